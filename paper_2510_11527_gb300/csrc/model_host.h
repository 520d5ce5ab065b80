// Host-side completion of a DevModel: the interior extrema of f_l' for the
// Buckley-Leverett flux (needed by the interval wave speed of the LLF flux, Section
// 5.2 of arXiv 2510.11527), |f_l'| there, and the float copies of all parameters.
#pragma once
#include <algorithm>
#include <cmath>

#include "af_model.cuh"

namespace af {

// SSP-RK(5,4) of Spiteri & Ruuth (2002) in Shu-Osher form: alpha[k][l], beta[k][l],
// row k producing stage value k+1 from u^(l) (Section 3.2 gives its stability
// polynomial, z^5 coefficient 0.004477718303076).
inline const double kA54[5][5] = {
    {1.0, 0, 0, 0, 0},
    {0.444370493651235, 0.555629506348765, 0, 0, 0},
    {0.620101851488403, 0, 0.379898148511597, 0, 0},
    {0.178079954393132, 0, 0, 0.821920045606868, 0},
    {0, 0, 0.517231671970585, 0.096059710526147, 0.386708617503269}};
inline const double kB54[5][5] = {
    {0.391752226571890, 0, 0, 0, 0},
    {0, 0.368410593050371, 0, 0, 0},
    {0, 0, 0.251891774271694, 0, 0},
    {0, 0, 0, 0.544974750228521, 0},
    {0, 0, 0, 0.063692468666290, 0.226007483236906}};

// Buckley-Leverett f_l'' (analytic) for locating the interior extrema of f_l'.
inline double bl_d2(int dir, double g, double u) {
  const double v = 1.0 - u, D = u * u + v * v, Dp = 2.0 * u - 2.0 * v;
  const double f1 = u * u / D;
  const double d1 = 2.0 * u * v / (D * D);
  const double dd1 = (2.0 * (v - u) * D - 4.0 * u * v * Dp) / (D * D * D);
  if (dir == 0) return dd1;
  return dd1 * (1.0 - g * v * v) + 4.0 * g * v * d1 - 2.0 * g * f1;
}

// |f_l'(u)| of the Buckley-Leverett flux
inline double bl_dabs(int dir, double g, double u) {
  const double v = 1.0 - u, D = u * u + v * v;
  const double f1 = u * u / D, d1 = 2.0 * u * v / (D * D);
  return std::fabs(dir == 0 ? d1 : d1 * (1.0 - g * v * v) + 2.0 * g * v * f1);
}

// roots of f_l'' on [-1, 2]: sign changes on a uniform grid refined by bisection
inline void bl_critical_points(DevModel& m) {
  for (int d = 0; d < 2; ++d) {
    m.ncrit[d] = 0;
    const double g = m.fp[0];
    const int n = 60000;
    const double a = -1.0, b = 2.0;
    double xprev = a, yprev = bl_d2(d, g, a);
    for (int k = 1; k <= n && m.ncrit[d] < 8; ++k) {
      const double x = a + (b - a) * k / n, y = bl_d2(d, g, x);
      if ((yprev < 0.0 && y > 0.0) || (yprev > 0.0 && y < 0.0) || y == 0.0) {
        double lo = xprev, hi = x, flo = yprev;
        for (int it = 0; it < 200 && y != 0.0; ++it) {
          const double mid = 0.5 * (lo + hi), fm = bl_d2(d, g, mid);
          if ((fm < 0.0) == (flo < 0.0)) {
            lo = mid;
            flo = fm;
          } else {
            hi = mid;
          }
        }
        const double c = y == 0.0 ? x : 0.5 * (lo + hi);
        m.critv[d][m.ncrit[d]] = bl_dabs(d, g, c);
        m.crit[d][m.ncrit[d]++] = c;
      }
      xprev = x;
      yprev = y;
    }
  }
}

// after fp/dp/umin/umax are set: flux-specific tables and float copies. In 1D the
// Buckley-Leverett flux is the gravity form f1 (1 - g (1-u)^2), the form of direction 1:
// its extrema tables are also placed in slot 0, which the 1D wave-speed code reads.
// 1 when the diffusion potential a(u) is constant (no diffusion term: kind NONE, or a
// kind whose coefficients of u are all zero), else 3; see DevModel::lim_parts.
inline int limiter_parts(int diff_kind, const double* p) {
  bool diffuses = false;
  switch (diff_kind) {
    case AF_DIFF_CONST: diffuses = p[0] != 0.0; break;
    case AF_DIFF_PWL: diffuses = p[0] != 0.0 || p[2] != 0.0; break;
    case AF_DIFF_PME: diffuses = true; break;
    case AF_DIFF_CUBIC:
    case AF_DIFF_CUBIC01: diffuses = p[0] != 0.0 || p[1] != 0.0 || p[2] != 0.0; break;
    case AF_DIFF_RAMP: diffuses = p[0] != 0.0; break;
    default: diffuses = false;
  }
  return diffuses ? 3 : 1;
}

inline void finish_model(DevModel& m, int flux_kind, int dim) {
  m.lim_parts = limiter_parts(m.diff_kind, m.dp);
  for (int d = 0; d < 2; ++d) {
    m.ncrit[d] = 0;
    for (int k = 0; k < 8; ++k) m.crit[d][k] = m.critv[d][k] = 0.0;
  }
  if (flux_kind == AF_FLUX_BL) {
    bl_critical_points(m);
    if (dim == 1) {
      m.ncrit[0] = m.ncrit[1];
      for (int k = 0; k < 8; ++k) {
        m.crit[0][k] = m.crit[1][k];
        m.critv[0][k] = m.critv[1][k];
      }
    }
  }
  fill_float_params(m);
}

// kappa(u) = a'(u) of the diffusion kinds
inline double kappa_of(const af_diff& df, double u) {
  switch (df.kind) {
    case AF_DIFF_CONST: return df.p[0];
    case AF_DIFF_PWL: return (u < df.p[1] ? df.p[0] : 0.0) + (u > df.p[3] ? df.p[2] : 0.0);
    case AF_DIFF_PME: return df.p[0] * std::pow(u, df.p[0] - 1.0);
    case AF_DIFF_CUBIC: return df.p[0] + 2.0 * df.p[1] * u + 3.0 * df.p[2] * u * u;
    case AF_DIFF_RAMP: return u <= df.p[1] ? 0.0 : (u < df.p[1] + df.p[2] ? df.p[0] * (u - df.p[1]) / df.p[2] : df.p[0]);
    case AF_DIFF_CUBIC01:
      return (u > 0.0 && u < 1.0) ? df.p[0] + 2.0 * df.p[1] * u + 3.0 * df.p[2] * u * u : 0.0;
    default: return 0.0;
  }
}

// kappa_max over [umin, umax] in closed form (Section 5.1.1)
inline double kappa_max_of(const af_diff& df, double lo, double hi) {
  double k = std::max(0.0, std::max(kappa_of(df, lo), kappa_of(df, hi)));
  if (df.kind == AF_DIFF_PWL) {
    if (lo < df.p[1]) k = std::max(k, df.p[0]);
    if (hi > df.p[3]) k = std::max(k, df.p[2]);
  }
  if ((df.kind == AF_DIFF_CUBIC || df.kind == AF_DIFF_CUBIC01) && df.p[2] != 0.0) {
    const double uv = -df.p[1] / (3.0 * df.p[2]);
    if (uv > lo && uv < hi) k = std::max(k, kappa_of(df, uv));
  }
  if (df.kind == AF_DIFF_CUBIC01) {
    // one-sided limits at the ends of [0, 1] inside the interval
    auto k4 = [&](double u) { return df.p[0] + 2.0 * df.p[1] * u + 3.0 * df.p[2] * u * u; };
    if (lo < 0.0 && hi > 0.0) k = std::max(k, k4(0.0));
    if (lo < 1.0 && hi > 1.0) k = std::max(k, k4(1.0));
  }
  return k;
}

}  // namespace af
