// Plain, slow FP64 CPU oracle for the compact fourth-order doubly conservative
// active flux (AF) method with monolithic convex MPP limiting (arXiv 2510.11527).
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may load, link or call this
// code: only the test suite, the package smoke check and the benchmark's CPU-baseline
// leg use it. It shares no code with the CUDA library.
//
// Everything is written in the paper's order and notation with plain loops over
// periodic index maps; each quantity is evaluated once per location and kept in its own
// array so that every step can be checked against the paper by eye. All functions are
// templated on the scalar type R so that the same source can be instantiated with a
// counting type (flop counts for the roofline); the exported entry points use double.
//
// Build: g++ -O2 -ffp-contract=off -std=c++17 -fPIC -shared (see oracle/build.py).
//
// DoF layout (2D, periodic, row-major [ny][nx], i fastest) -- Section 4, Fig. 2:
//   ub[j][i] cell average of cell (i,j)
//   V [j][i] point value at (x_{i+1/2}, y_{j+1/2})   (cell corner)
//   X [j][i] point value at (x_{i+1/2}, y_j)         (midpoint of the vertical edge)
//   Y [j][i] point value at (x_i, y_{j+1/2})         (midpoint of the horizontal edge)
// 1D (Section 2): ub[i] and P[i] = u_{i+1/2}; periodic, so u_{1/2} = u_{N+1/2}.
// 1D with a Dirichlet or outflow boundary: P[j+1] = u_{j+1/2}, j = -1..N-1 (N+1 values
// from the left to the right end of the interval).
// 3D (periodic, [nz][ny][nx], i fastest): 8 arrays ordered by kind s = sx + 2 sy + 4 sz
// of the location (i + sx/2, j + sy/2, k + sz/2): ub, then the x-face, y-face, xy-edge,
// z-face, xz-edge, yz-edge and corner values.
// 2D rectangle with outflow ends: ub [ny][nx]; V [ny+1][nx+1] (corners, from the
// bottom-left corner); X [ny][nx+1] (vertical edges, from the left side); Y [ny+1][nx]
// (horizontal edges, from the bottom side).
//
// Readings where the paper is silent (also listed in the design notes):
//   * 2D factors: directional split 1/(2d)=1/4, limiter factor 3*2d = 12, MPP CFL 1/4
//     (derived from the 1D factors 2,6 and the 3D factors 6,18 of Section 5).
//   * Without a diffusion term (a constant) each limited directional state has only
//     its face correction, so the face limiter factor is 2d instead of 3*2d (Example
//     6.2's limited results in Table 3 and its fourth-order rate need this factor).
//   * 2D cell potential A^H_l: tensor Simpson average of the 1D potential a-hat of
//     Proposition 2.1 along the transverse direction (Section 4, face averages).
//   * Low-order point residual used by the smoothness blend (Section 5.1.3 defers it):
//     first-order LLF + central second difference on the +-h/2 neighbours of the
//     5-point line, with a recovered centre replaced by that cell's average.
//   * Point blend weight in 2D: min of theta^{c,s} over the l-faces the point lies on,
//     else min of theta^{d,s}_l over the two cells sharing the point.
//   * Theta(zL,zH) is clipped to [0,1]; a limiter parameter equal to 1 returns the
//     (blended) high-order flux/potential itself (Remark after Proposition 5.2).
//   * After every RK stage, values outside [umin,umax] by at most clamp_tol are clamped
//     and counted; larger excesses are reported as an error.
//   * Boundaries of a 1D interval (Section 6 names Dirichlet and outflow conditions but
//     not their discrete form): ghost cells and ghost points beyond each end. Dirichlet:
//     every ghost DoF holds the boundary value and the boundary point value is held
//     at it. Outflow: even reflection of the DoFs about the boundary point (a
//     zero-gradient extension); the boundary point values evolve like interior ones.
//     The CFL maximum also runs over the two boundary faces. A 2D rectangle takes
//     outflow ends only (the paper's 2D examples with ends use outflow): the periodic
//     step on the rectangle padded with reflected ghost layers, restricted to it.
//   * AF method without double conservation (Appendix A, 1D): the cell average
//     receives the face flux f(u_{i+1/2}) - kappa(u_{i+1/2}) D_c(u)_{i+1/2}; the point
//     value the compact operator 4/h^2 sum b_mn kappa(z_m) z_n on its 5-point line.
//     Its limiter blends the total face flux with the low-order total face flux
//     F^L - (a(ub_{i+1}) - a(ub_i))/h, with Theta on u^{L,+-} and factor 2 (the
//     update is a mean of two states, each receiving one face correction).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------
// Counting scalar used only by ao_flop_count: every +,-,*,/ and exp is one flop.
struct FlopCounter {
  long long add = 0, mul = 0, div = 0, exp = 0, cmp = 0;
};
FlopCounter g_flops;

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { g_flops.add++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_flops.add++; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_flops.mul++; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_flops.div++; return Cnt(a.v / b.v); }
inline bool operator<(Cnt a, Cnt b) { g_flops.cmp++; return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { g_flops.cmp++; return a.v > b.v; }
inline bool operator<=(Cnt a, Cnt b) { g_flops.cmp++; return a.v <= b.v; }
inline bool operator>=(Cnt a, Cnt b) { g_flops.cmp++; return a.v >= b.v; }
inline bool operator==(Cnt a, Cnt b) { g_flops.cmp++; return a.v == b.v; }
inline bool operator!=(Cnt a, Cnt b) { g_flops.cmp++; return a.v != b.v; }
inline Cnt fabs_(Cnt a) { return Cnt(std::fabs(a.v)); }
inline Cnt exp_(Cnt a) { g_flops.exp++; return Cnt(std::exp(a.v)); }
inline double val(Cnt a) { return a.v; }

inline double fabs_(double a) { return std::fabs(a); }
inline double exp_(double a) { return std::exp(a); }
inline double val(double a) { return a; }

template <class R> inline R maxr(R a, R b) { return (a < b) ? b : a; }
template <class R> inline R minr(R a, R b) { return (b < a) ? b : a; }

inline int wrap(int i, int n) { return ((i % n) + n) % n; }

}  // namespace

extern "C" {

// Problem description shared with the Python side through ctypes.
// flux_kind: 0 zero, 1 linear f1=p0*u f2=p1*u (f3=p2*u), 2 Burgers f_l=p0*u^2,
//            3 Buckley-Leverett f1=u^2/(u^2+(1-u)^2), f2=f1*(1-p0*(1-u)^2); in 1D the
//              flux is the gravity form f1*(1-p0*(1-u)^2).
// diff_kind: 0 none, 1 constant a=p0*u, 2 piecewise linear
//            a = p0*min(u-p1,0) + p2*max(u-p3,0), 3 porous medium a=u^p0 (integer p0>=1),
//            4 cubic a = p0*u + p1*u^2 + p2*u^3,
//            6 the cubic of kind 4 at min(max(u, 0), 1) (constant outside [0, 1]),
//            5 ramp a = 0 (u <= p1), p0 (u-p1)^2 / (2 p2) (p1 < u < p1+p2),
//              p0 (u - p1 - p2/2) (u >= p1+p2)  (kappa rises linearly from 0 to p0).
// bc: 0 periodic, 1 Dirichlet (bc_left, bc_right; 1D only), 2 outflow (1D or 2D).
// nodc: 1 selects the AF method without double conservation of Appendix A (1D only,
//       blend off).
typedef struct {
  int dim;
  int nx, ny;
  double dx, dy;
  int flux_kind;
  double flux_p[4];
  int diff_kind;
  double diff_p[4];
  double umin, umax;
  int limiter;          // 1: monolithic convex limiter for averages + point projection
  int blend;            // 0 off, 1 smoothness indicator, 2 external per-cell indicator
  double gamma;         // blend strength (gamma = 1 in the paper's examples)
  double clamp_tol;     // absolute tolerance of the post-stage safeguard clamp
  int bc;               // 0 periodic, 1 Dirichlet, 2 outflow (1D)
  double bc_left, bc_right;
  int nodc;             // 1: Appendix A discretization of the diffusion term
  int nz;               // 3D: cells along z (periodic)
  double dz;
} ao_problem;

typedef struct {
  long long clamps;     // values clamped by the post-stage safeguard
  double max_excess;    // largest excess beyond [umin,umax] that was clamped
  int error;            // 1 if an excess above clamp_tol was met
} ao_stats;

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------------
// Problem functions: f_l, f_l', a, and the interval maximum of |f_l'| (Section 1 and
// eq. for the local wave speed in Section 5.1.1 / 5.2).

struct Model {
  ao_problem p;
  // interior local extrema of f_l' (Buckley-Leverett only), found once at set-up
  std::vector<double> crit[3];
};

template <class R> R flux(const Model& m, int dir, R u) {
  const ao_problem& p = m.p;
  switch (p.flux_kind) {
    case 1: return R(dir == 0 ? p.flux_p[0] : (dir == 1 ? p.flux_p[1] : p.flux_p[2])) * u;
    case 2: return R(p.flux_p[0]) * u * u;
    case 3: {
      R v = R(1.0) - u;
      R f1 = u * u / (u * u + v * v);
      // the gravity factor acts along y in 2D and 3D, and along the only axis in 1D
      // (Example 6.6: f = f1 (1 - 5 (1-u)^2) with gravity, p0 = 0 without)
      if (dir == 0 && p.dim != 1) return f1;
      return f1 * (R(1.0) - R(p.flux_p[0]) * v * v);
    }
    default: return R(0.0);
  }
}

template <class R> R dflux(const Model& m, int dir, R u) {
  const ao_problem& p = m.p;
  switch (p.flux_kind) {
    case 1: return R(dir == 0 ? p.flux_p[0] : (dir == 1 ? p.flux_p[1] : p.flux_p[2]));
    case 2: return R(2.0 * p.flux_p[0]) * u;
    case 3: {
      // f1 = u^2/D, D = u^2 + (1-u)^2, f1' = 2u(1-u)/D^2
      R v = R(1.0) - u;
      R D = u * u + v * v;
      R f1 = u * u / D;
      R d1 = R(2.0) * u * v / (D * D);
      if (dir == 0 && p.dim != 1) return d1;
      R g = R(p.flux_p[0]);
      // f2 = f1 (1 - g v^2), f2' = f1' (1 - g v^2) + f1 * 2 g v
      return d1 * (R(1.0) - g * v * v) + f1 * R(2.0) * g * v;
    }
    default: return R(0.0);
  }
}

template <class R> R apot(const Model& m, R u) {
  const ao_problem& p = m.p;
  switch (p.diff_kind) {
    case 1: return R(p.diff_p[0]) * u;
    case 2: return R(p.diff_p[0]) * minr(u - R(p.diff_p[1]), R(0.0)) +
                   R(p.diff_p[2]) * maxr(u - R(p.diff_p[3]), R(0.0));
    case 3: {
      int e = (int)p.diff_p[0];
      R r = u;
      for (int k = 1; k < e; ++k) r = r * u;
      return r;
    }
    case 4: return R(p.diff_p[0]) * u + R(p.diff_p[1]) * u * u + R(p.diff_p[2]) * u * u * u;
    case 6: {
      // the cubic of kind 4 on [0, 1], constant outside (Example 6.6)
      R v = minr(maxr(u, R(0.0)), R(1.0));
      return R(p.diff_p[0]) * v + R(p.diff_p[1]) * v * v + R(p.diff_p[2]) * v * v * v;
    }
    case 5: {
      R lo = R(p.diff_p[1]), w = R(p.diff_p[2]);
      if (u <= lo) return R(0.0);
      if (u < lo + w) return R(p.diff_p[0]) * (u - lo) * (u - lo) / (R(2.0) * w);
      return R(p.diff_p[0]) * (u - lo - R(0.5) * w);
    }
    default: return R(0.0);
  }
}

// kappa(u) = a'(u); at a kink of the piecewise forms the one-sided value nearer the
// degenerate side is taken (kappa is 0 exactly at u = p1 and u = p3 of kind 2).
template <class R> R kappa(const Model& m, R u) {
  const ao_problem& p = m.p;
  switch (p.diff_kind) {
    case 1: return R(p.diff_p[0]);
    case 2: return (u < R(p.diff_p[1]) ? R(p.diff_p[0]) : R(0.0)) + (u > R(p.diff_p[3]) ? R(p.diff_p[2]) : R(0.0));
    case 3: {
      int e = (int)p.diff_p[0];
      R r = R(double(e));
      for (int k = 1; k < e; ++k) r = r * u;
      return r;
    }
    case 4: return R(p.diff_p[0]) + R(2.0 * p.diff_p[1]) * u + R(3.0 * p.diff_p[2]) * u * u;
    case 6:
      if (!(u > R(0.0) && u < R(1.0))) return R(0.0);
      return R(p.diff_p[0]) + R(2.0 * p.diff_p[1]) * u + R(3.0 * p.diff_p[2]) * u * u;
    case 5: {
      R lo = R(p.diff_p[1]), w = R(p.diff_p[2]);
      if (u <= lo) return R(0.0);
      if (u < lo + w) return R(p.diff_p[0]) * (u - lo) / w;
      return R(p.diff_p[0]);
    }
    default: return R(0.0);
  }
}

// Whether the equation has a diffusion term at all: a(u) is constant for kind 0 and
// for every kind whose coefficients of u are all zero (the porous medium always
// diffuses).
bool has_diffusion(const ao_problem& p) {
  switch (p.diff_kind) {
    case 1: return p.diff_p[0] != 0.0;
    case 2: return p.diff_p[0] != 0.0 || p.diff_p[2] != 0.0;
    case 3: return true;
    case 4:
    case 6: return p.diff_p[0] != 0.0 || p.diff_p[1] != 0.0 || p.diff_p[2] != 0.0;
    case 5: return p.diff_p[0] != 0.0;
    default: return false;
  }
}

// Number of parts in the convex decomposition of each limited directional state
// u^{Lim,+-} (Section 5.1.1; Section 5.2 per direction). With diffusion each state is
// the mean of three parts -- the face correction and the two potential corrections --
// so a face correction enters its part with factor 3 * 2d (6 in 1D, 12 in 2D, 18 in
// 3D). Without a diffusion term the potential corrections vanish identically and the
// state consists of the face correction alone, factor 2d (reading of Example 6.2: the
// pure-convection limiter reproduces Table 3's limited columns and keeps the
// fourth-order rate only with this factor).
int lim_parts(const ao_problem& p) { return has_diffusion(p) ? 3 : 1; }

// Planted-mistake hook for the pins' sensitivity tests only (a separate build with
// -DAO_PLANT_FACE_SCALE=...; the oracle itself is built without it): scales the face
// limiter factor.
#ifndef AO_PLANT_FACE_SCALE
#define AO_PLANT_FACE_SCALE 1.0
#endif
double face_factor(const ao_problem& p, int d) { return 2.0 * d * lim_parts(p) * AO_PLANT_FACE_SCALE; }

// kappa_max = max over [umin, umax] of kappa (Section 5.1.1). Plain dense sampling
// plus the interval end points and the kinks of the piecewise form.
double kappa_max(const Model& m) {
  const ao_problem& p = m.p;
  double lo = p.umin, hi = p.umax, best = 0.0;
  const int n = 200000;
  for (int k = 0; k <= n; ++k) best = std::max(best, kappa<double>(m, lo + (hi - lo) * k / n));
  best = std::max(best, kappa<double>(m, lo));
  best = std::max(best, kappa<double>(m, hi));
  if (p.diff_kind == 2) {
    // one-sided limits at the kinks inside the interval
    if (p.diff_p[1] > lo) best = std::max(best, p.diff_p[0]);
    if (p.diff_p[3] < hi) best = std::max(best, p.diff_p[2]);
  }
  if ((p.diff_kind == 4 || p.diff_kind == 6) && p.diff_p[2] != 0.0) {
    double uv = -p.diff_p[1] / (3 * p.diff_p[2]);
    if (uv > lo && uv < hi) best = std::max(best, kappa<double>(m, uv));
  }
  if (p.diff_kind == 6) {
    // one-sided limits of kappa at the ends of [0, 1] inside the interval
    auto k4 = [&](double u) { return p.diff_p[0] + 2.0 * p.diff_p[1] * u + 3.0 * p.diff_p[2] * u * u; };
    if (lo < 0.0 && hi > 0.0) best = std::max(best, k4(0.0));
    if (lo < 1.0 && hi > 1.0) best = std::max(best, k4(1.0));
  }
  return best;
}

// Interior local extrema of f_l' on [-1, 2] by sampling and golden-section refinement
// (the value of f' at an extremum is insensitive to the location error).
void find_crit(Model& m) {
  for (int d = 0; d < 3; ++d) m.crit[d].clear();
  if (m.p.flux_kind != 3) return;
  for (int d = 0; d < 2; ++d) {
    const double a = -1.0, b = 2.0;
    const int n = 30000;
    auto fp = [&](double u) { return dflux<double>(m, d, u); };
    for (int k = 1; k < n; ++k) {
      double u0 = a + (b - a) * (k - 1) / n, u1 = a + (b - a) * k / n, u2 = a + (b - a) * (k + 1) / n;
      double g0 = fp(u0), g1 = fp(u1), g2 = fp(u2);
      int sgn = 0;
      if (g1 >= g0 && g1 > g2) sgn = 1;        // local max of f'
      else if (g1 <= g0 && g1 < g2) sgn = -1;  // local min of f'
      if (!sgn) continue;
      double lo = u0, hi = u2;
      const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
      for (int it = 0; it < 200; ++it) {
        double c = hi - gr * (hi - lo), e = lo + gr * (hi - lo);
        if (sgn * fp(c) > sgn * fp(e)) hi = e; else lo = c;
      }
      m.crit[d].push_back(0.5 * (lo + hi));
    }
  }
}

// alpha = max over u in [min(ua,ub), max(ua,ub)] of |f_l'(u)| (eq. of the local wave
// speed, Section 5.1.1; multi-D form in Section 5.2).
template <class R> R alpha_interval(const Model& m, int dir, R ua, R ub) {
  R lo = minr(ua, ub), hi = maxr(ua, ub);
  R best = maxr(fabs_(dflux<R>(m, dir, lo)), fabs_(dflux<R>(m, dir, hi)));
  for (double c : m.crit[dir]) {
    if (R(c) > lo && R(c) < hi) best = maxr(best, fabs_(dflux<R>(m, dir, R(c))));
  }
  return best;
}

// Theta(zL, zH): largest blend factor keeping (1-t) zL + t zH in [umin, umax]
// (definition in Section 5.1.1), clipped to [0,1].
template <class R> R Theta(const Model& m, R zL, R zH) {
  R umin = R(m.p.umin), umax = R(m.p.umax);
  R t;
  if (zH < umin) {
    if (zL == zH) return R(1.0);
    t = (zL - umin) / (zL - zH);
  } else if (zH > umax) {
    if (zL == zH) return R(1.0);
    t = (zL - umax) / (zL - zH);
  } else {
    return R(1.0);
  }
  if (t < R(0.0)) t = R(0.0);
  if (t > R(1.0)) t = R(1.0);
  return t;
}

// One 5-point line residual (spacing h/2, points z[0..4] at offsets -h..+h, the point
// being updated is z[2]). Convection: FVS-LLF split with biased D+ / D- (eqs.
// 1d_upwind_ops_4p / 4m) and alpha = max |f'| over the five points; diffusion: the
// compact fourth-order second derivative of a (eq. 1d_diff_compact_a).
template <class R>
R line_residual(const R z[5], const R f[5], const R df[5], const R a[5], R h) {
  R alpha = fabs_(df[0]);
  for (int k = 1; k < 5; ++k) alpha = maxr(alpha, fabs_(df[k]));
  R gp[5], gm[5];
  for (int k = 0; k < 5; ++k) {
    gp[k] = R(0.5) * (f[k] + alpha * z[k]);
    gm[k] = R(0.5) * (f[k] - alpha * z[k]);
  }
  R Dp = (gp[0] - R(6.0) * gp[1] + R(3.0) * gp[2] + R(2.0) * gp[3]) / (R(3.0) * h);
  R Dm = (R(-2.0) * gm[1] - R(3.0) * gm[2] + R(6.0) * gm[3] - gm[4]) / (R(3.0) * h);
  R D2 = (R(-1.0 / 3.0) * a[0] + R(16.0 / 3.0) * a[1] - R(10.0) * a[2] + R(16.0 / 3.0) * a[3] -
          R(1.0 / 3.0) * a[4]) / (h * h);
  return -(Dp + Dm) + D2;
}

// The diffusion part of line_residual alone (f = 0): the compact fourth-order second
// derivative of a, the same expression and order of operations.
template <class R>
R line_diffusion(const R a[5], R h) {
  return (R(-1.0 / 3.0) * a[0] + R(16.0 / 3.0) * a[1] - R(10.0) * a[2] + R(16.0 / 3.0) * a[3] -
          R(1.0 / 3.0) * a[4]) / (h * h);
}

// First-order point residual on the +-h/2 neighbours (reading for the blend's
// low-order point scheme): -(2/h)[F(z0,z+) - F(z-,z0)] + (4/h^2)(a+ - 2 a0 + a-).
template <class R>
R low_point_residual(const Model& m, int dir, R zm, R z0, R zp, R h) {
  auto llf = [&](R ul, R ur) {
    R al = alpha_interval<R>(m, dir, ul, ur);
    return R(0.5) * (flux<R>(m, dir, ul) + flux<R>(m, dir, ur)) - R(0.5) * al * (ur - ul);
  };
  R conv = (llf(z0, zp) - llf(zm, z0)) * (R(2.0) / h);
  R diff = (apot<R>(m, zp) - R(2.0) * apot<R>(m, z0) + apot<R>(m, zm)) * (R(4.0) / (h * h));
  return -conv + diff;
}

// Smoothness indicator along one line of cell averages (Section 5.1.3):
// s~_i = |u_{i-1} - 2u_i + u_{i+1}| / (|u_{i-1}| + 2|u_i| + |u_{i+1}| + 1e-13).
template <class R> R s_tilde(R um, R u0, R up) {
  return fabs_(um - R(2.0) * u0 + up) / (fabs_(um) + R(2.0) * fabs_(u0) + fabs_(up) + R(1e-13));
}

// Values on the index range [lo, hi), addressed by the mesh index itself: indices below
// 0 or at/above n are ghost entries beyond the two ends (or periodic images).
template <class R> struct Span {
  int lo;
  std::vector<R> v;
  Span(int lo_, int hi_) : lo(lo_), v((size_t)(hi_ - lo_), R(0.0)) {}
  R& operator[](int i) { return v.at((size_t)(i - lo)); }
  const R& operator[](int i) const { return v.at((size_t)(i - lo)); }
};

// Cell average ub_i and point value u_{j+1/2} at any index of a 1D mesh: stored values
// inside, the boundary rule outside (periodic image, Dirichlet value, or even
// reflection about the boundary point for outflow).
template <class R> R cell_at(const ao_problem& p, const R* ub, int i) {
  const int n = p.nx;
  if (p.bc == 0) return ub[wrap(i, n)];
  if (i >= 0 && i < n) return ub[i];
  if (p.bc == 1) return R(i < 0 ? p.bc_left : p.bc_right);
  return ub[i < 0 ? -1 - i : 2 * n - 1 - i];
}
template <class R> R point_at(const ao_problem& p, const R* P, int j) {
  const int n = p.nx;
  if (p.bc == 0) return P[wrap(j, n)];
  if (j >= -1 && j <= n - 1) return P[j + 1];
  if (p.bc == 1) return R(j < -1 ? p.bc_left : p.bc_right);
  return P[(j < -1 ? -2 - j : 2 * (n - 1) - j) + 1];
}

// Appendix A: B = [0 0; 0 M] - [M 0; 0 0] (5x5), b_mn for m, n = -2..2 at B[m+2][n+2].
inline double nodc_b(int r, int s) {
  static const double M[4][4] = {{1.0 / 8, -1.0 / 6, 1.0 / 24, 0.0},
                                 {-1.0 / 6, -3.0 / 8, 2.0 / 3, -1.0 / 8},
                                 {1.0 / 8, -2.0 / 3, 3.0 / 8, 1.0 / 6},
                                 {0.0, -1.0 / 24, 1.0 / 6, -1.0 / 8}};
  double v = 0.0;
  if (r >= 1 && s >= 1) v += M[r - 1][s - 1];
  if (r <= 3 && s <= 3) v -= M[r][s];
  return v;
}

// ---------------------------------------------------------------------------------
// 1D forward-Euler evaluation (Sections 2 and 5.1; Appendix A when p.nodc).
// Cells i = 0..n-1; point j is u_{j+1/2}, the right end of cell i = j. Updated points:
// j = 0..n-1 (periodic) or j = -1..n-1 (bounded). Everything is first gathered on the
// index range it is needed on, ghost entries included, then computed with plain loops.
template <class R>
void fe1d(const Model& m, const R* ub, const R* P, R tau, const R* s_ext, R* ub_o, R* P_o) {
  const ao_problem& p = m.p;
  const int n = p.nx, G = 3;
  const bool bounded = p.bc != 0;
  const int jlo = bounded ? -1 : 0;
  const R h = R(p.dx);
  Span<R> U(-G, n + G), Pt(-G - 1, n + G), c(-G, n + G);
  for (int i = -G; i < n + G; ++i) U[i] = cell_at<R>(p, ub, i);
  for (int j = -G - 1; j < n + G; ++j) Pt[j] = point_at<R>(p, P, j);
  // centre value by Simpson's rule: u_i = (6 ub_i - u_{i-1/2} - u_{i+1/2}) / 4
  for (int i = -G; i < n + G; ++i) c[i] = (R(6.0) * U[i] - Pt[i - 1] - Pt[i]) / R(4.0);
  Span<R> fP(-G - 1, n + G), dP(-G - 1, n + G), aP(-G - 1, n + G), kP(-G - 1, n + G);
  Span<R> fC(-G, n + G), dC(-G, n + G), aC(-G, n + G), kC(-G, n + G), fU(-G, n + G), aU(-G, n + G);
  for (int j = -G - 1; j < n + G; ++j) {
    fP[j] = flux<R>(m, 0, Pt[j]); dP[j] = dflux<R>(m, 0, Pt[j]); aP[j] = apot<R>(m, Pt[j]);
    if (p.nodc) kP[j] = kappa<R>(m, Pt[j]);
  }
  for (int i = -G; i < n + G; ++i) {
    fC[i] = flux<R>(m, 0, c[i]); dC[i] = dflux<R>(m, 0, c[i]); aC[i] = apot<R>(m, c[i]);
    if (p.nodc) kC[i] = kappa<R>(m, c[i]);
    fU[i] = flux<R>(m, 0, U[i]); aU[i] = apot<R>(m, U[i]);
  }
  // high-order flux f(u_{i+1/2}) on faces -1..n-1 and DC potential
  // a^_i = (-a_{i-1/2} + 8 a_i - a_{i+1/2})/6 on cells -1..n
  Span<R> FH(-1, n), AH(-1, n + 1), RH(jlo, n);
  for (int f = -1; f < n; ++f) FH[f] = fP[f];
  for (int i = -1; i <= n; ++i) AH[i] = (-aP[i - 1] + R(8.0) * aC[i] - aP[i]) / R(6.0);
  // point residual at x_{j+1/2}: line [u_{j-1/2}, u_j, u_{j+1/2}, u_{j+1}, u_{j+3/2}]
  for (int j = jlo; j < n; ++j) {
    R z[5] = {Pt[j - 1], c[j], Pt[j], c[j + 1], Pt[j + 1]};
    R f[5] = {fP[j - 1], fC[j], fP[j], fC[j + 1], fP[j + 1]};
    R d[5] = {dP[j - 1], dC[j], dP[j], dC[j + 1], dP[j + 1]};
    if (!p.nodc) {
      R a[5] = {aP[j - 1], aC[j], aP[j], aC[j + 1], aP[j + 1]};
      RH[j] = line_residual<R>(z, f, d, a, h);
    } else {
      // convection part of the same line (a = 0) plus the compact operator of
      // Appendix A: 4/h^2 sum_{m,n} b_mn kappa(z_m) z_n
      R a0[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
      R k[5] = {kP[j - 1], kC[j], kP[j], kC[j + 1], kP[j + 1]};
      R D2 = R(0.0);
      for (int r = 0; r < 5; ++r)
        for (int s = 0; s < 5; ++s) D2 = D2 + R(nodc_b(r, s)) * k[r] * z[s];
      RH[j] = line_residual<R>(z, f, d, a0, h) + R(4.0) * D2 / (h * h);
    }
  }
  const R mu = tau / h, nu = tau / (h * h);
  // low-order LLF scheme on faces -2..n and its directional states u^{L,+-} (Lemma 5.1)
  Span<R> FL(-2, n + 1), ULp(-2, n + 1), ULm(-1, n + 2);
  for (int f = -2; f <= n; ++f) {
    R al = alpha_interval<R>(m, 0, U[f], U[f + 1]);
    FL[f] = R(0.5) * (fU[f] + fU[f + 1]) - R(0.5) * al * (U[f + 1] - U[f]);
  }
  for (int i = -2; i <= n; ++i) ULp[i] = U[i] - R(2.0) * mu * (FL[i] - fU[i]) + R(2.0) * nu * (aU[i + 1] - aU[i]);
  for (int i = -1; i <= n + 1; ++i) ULm[i] = U[i] - R(2.0) * mu * (fU[i] - FL[i - 1]) - R(2.0) * nu * (aU[i] - aU[i - 1]);
  // optional smoothness blend (Section 5.1.3), applied before the limiter
  Span<R> Fh(-1, n), Ah(-1, n + 1), R_(jlo, n), thcs(-1, n);
  for (int f = -1; f < n; ++f) { Fh[f] = FH[f]; thcs[f] = R(1.0); }
  for (int i = -1; i <= n; ++i) Ah[i] = AH[i];
  for (int j = jlo; j < n; ++j) R_[j] = RH[j];
  if (p.blend) {
    Span<R> st(-2, n + 2), s(-1, n + 1), thds(-1, n + 1);
    if (p.blend == 1) {
      for (int i = -2; i < n + 2; ++i) st[i] = s_tilde<R>(U[i - 1], U[i], U[i + 1]);
      for (int i = -1; i <= n; ++i) s[i] = (st[i - 1] + R(4.0) * st[i] + st[i + 1]) / R(6.0);
    } else {
      for (int i = -1; i <= n; ++i) s[i] = s_ext[wrap(i, n)];
    }
    for (int f = -1; f < n; ++f) thcs[f] = exp_(-R(p.gamma) * (R(0.5) * (s[f] + s[f + 1])));
    for (int i = -1; i <= n; ++i) thds[i] = exp_(-R(p.gamma) * s[i]);
    for (int f = -1; f < n; ++f) Fh[f] = thcs[f] * FH[f] + (R(1.0) - thcs[f]) * FL[f];
    for (int i = -1; i <= n; ++i) Ah[i] = thds[i] * AH[i] + (R(1.0) - thds[i]) * aU[i];
    for (int j = jlo; j < n; ++j) {
      R RL = low_point_residual<R>(m, 0, U[j], Pt[j], U[j + 1], h);
      R_[j] = thcs[j] * RH[j] + (R(1.0) - thcs[j]) * RL;
    }
  }
  if (!p.nodc) {
    // monolithic convex limiter (eqs. 1d_convection_limiting_parameter and
    // 1d_diffusion_limiting_parameter), limited average (eq. 1d_limited_average)
    Span<R> Flim(-1, n), Alim(-1, n + 1);
    for (int f = -1; f < n; ++f) Flim[f] = Fh[f];
    for (int i = -1; i <= n; ++i) Alim[i] = Ah[i];
    if (p.limiter) {
      // face correction factor 2 * parts (6 with diffusion, 2 without)
      const R kc = R(face_factor(p, 1));
      for (int f = -1; f < n; ++f) {
        R dF = Fh[f] - FL[f];
        R t = minr(Theta<R>(m, ULp[f], ULp[f] - kc * mu * dF),
                   Theta<R>(m, ULm[f + 1], ULm[f + 1] + kc * mu * dF));
        Flim[f] = (t == R(1.0)) ? Fh[f] : FL[f] + t * dF;
      }
      for (int i = -1; i <= n; ++i) {
        R dA = Ah[i] - aU[i];
        R t = minr(minr(Theta<R>(m, ULp[i - 1], ULp[i - 1] + R(6.0) * nu * dA),
                        Theta<R>(m, ULp[i], ULp[i] - R(6.0) * nu * dA)),
                   minr(Theta<R>(m, ULm[i], ULm[i] - R(6.0) * nu * dA),
                        Theta<R>(m, ULm[i + 1], ULm[i + 1] + R(6.0) * nu * dA)));
        Alim[i] = (t == R(1.0)) ? Ah[i] : aU[i] + t * dA;
      }
    }
    for (int i = 0; i < n; ++i)
      ub_o[i] = ub[i] - mu * (Flim[i] - Flim[i - 1]) + nu * (Alim[i + 1] - R(2.0) * Alim[i] + Alim[i - 1]);
  } else {
    // Appendix A: total face flux G = f(u_{i+1/2}) - kappa(u_{i+1/2}) D_c(u)_{i+1/2},
    // D_c(u)_{i+1/2} = (u_{i-1/2} - 8 u_i + 8 u_{i+1} - u_{i+3/2}) / (6h); low-order
    // counterpart G^L = F^L - (a(ub_{i+1}) - a(ub_i)) / h
    Span<R> GH(-1, n), GL(-1, n), Glim(-1, n);
    for (int f = -1; f < n; ++f) {
      R Dc = (Pt[f - 1] - R(8.0) * c[f] + R(8.0) * c[f + 1] - Pt[f + 1]) / (R(6.0) * h);
      GH[f] = fP[f] - kP[f] * Dc;
      GL[f] = FL[f] - (aU[f + 1] - aU[f]) / h;
      Glim[f] = GH[f];
    }
    if (p.limiter) {
      for (int f = -1; f < n; ++f) {
        R dG = GH[f] - GL[f];
        R t = minr(Theta<R>(m, ULp[f], ULp[f] - R(2.0) * mu * dG),
                   Theta<R>(m, ULm[f + 1], ULm[f + 1] + R(2.0) * mu * dG));
        Glim[f] = (t == R(1.0)) ? GH[f] : GL[f] + t * dG;
      }
    }
    for (int i = 0; i < n; ++i) ub_o[i] = ub[i] - mu * (Glim[i] - Glim[i - 1]);
  }
  // point values: high-order update, then projection onto [umin, umax] (Section 5.1.2);
  // Dirichlet boundary points keep the boundary value
  for (int j = jlo; j < n; ++j) {
    R v = Pt[j] + tau * R_[j];
    if (p.limiter) v = minr(maxr(v, R(p.umin)), R(p.umax));
    if (p.bc == 1 && j == -1) v = R(p.bc_left);
    if (p.bc == 1 && j == n - 1) v = R(p.bc_right);
    P_o[bounded ? j + 1 : j] = v;
  }
}

// ---------------------------------------------------------------------------------
// Dimension-generic forward-Euler evaluation (Sections 4 and 5.2; d = 1, 2, 3) on the
// fine grid of half-cell spacing: the DoF at (i + s_0/2, j + s_1/2, k + s_2/2), s_l in
// {0, 1}, has fine index (2i + s_0, 2j + s_1, 2k + s_2). Its kind is s = s_0 + 2 s_1 +
// 4 s_2: kind 0 is the cell centre (recovered, not a DoF), kinds 1 .. 2^d - 1 are the
// point values (3D: 1 x-face, 2 y-face, 3 xy-edge, 4 z-face, 5 xz-edge, 6 yz-edge,
// 7 corner; 2D: 1 = X, 2 = Y, 3 = V). Every 5-point line of the paper is then the fine
// points p - 2e, p - e, p, p + e, p + 2e along one axis, and every Simpson average
// takes weights 1, 4, 1 (/6) per axis. Periodic in every direction.
template <class R>
void fend(const Model& m, int d, const int* n, const R* h, const R* ub, const R* const* P, R tau,
          const R* s_ext, R* ub_o, R* const* P_o) {
  const ao_problem& p = m.p;
  const int nk = 1 << d;
  // f = 0 (pure diffusion): the convection terms of the high-order face fluxes, the
  // point residuals and the low-order fluxes and states are identically zero and are
  // not formed (the values are the same: x - 0 and -(0 + 0) + y are exact); the flop
  // count then holds the pure-diffusion method's own operations
  const bool conv = p.flux_kind != 0;
  int nn[3] = {1, 1, 1};
  for (int l = 0; l < d; ++l) nn[l] = n[l];
  const size_t N = (size_t)nn[0] * nn[1] * nn[2];
  auto cell = [&](const int* c) {   // periodic cell index -> linear
    int w[3];
    for (int l = 0; l < 3; ++l) w[l] = wrap(c[l], nn[l]);
    return ((size_t)w[2] * nn[1] + w[1]) * nn[0] + w[0];
  };
  auto decode = [&](size_t q, int* c) {
    c[0] = (int)(q % nn[0]);
    c[1] = (int)((q / nn[0]) % nn[1]);
    c[2] = (int)(q / ((size_t)nn[0] * nn[1]));
  };
  // fine index f -> (kind, cell)
  auto split = [&](const int* f, int& kind, size_t& q) {
    int c[3] = {0, 0, 0};
    kind = 0;
    for (int l = 0; l < d; ++l) {
      const int w = wrap(f[l], 2 * nn[l]);
      c[l] = w >> 1;
      kind |= (w & 1) << l;
    }
    q = cell(c);
  };
  const R w1[3] = {R(1.0), R(4.0), R(1.0)};   // Simpson weights (/6) for offsets -1, 0, +1

  // (1) centre value from the tensor Simpson rule for the cell average:
  //     ub = sum_m (prod_l w1(m_l)/6) z(2i + m)  ->  solved for the centre m = 0
  std::vector<R> C(N);
  for (size_t q = 0; q < N; ++q) {
    int c[3];
    decode(q, c);
    R acc = R(0.0);
    for (int o = 0; o < 27; ++o) {
      int mm[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
      bool skip = false, centre = true;
      for (int l = 0; l < 3; ++l) {
        if (l >= d && mm[l] != 0) skip = true;
        if (mm[l] != 0) centre = false;
      }
      if (skip || centre) continue;
      R wgt = R(1.0);
      int f[3] = {0, 0, 0};
      for (int l = 0; l < d; ++l) { wgt = wgt * w1[mm[l] + 1]; f[l] = 2 * c[l] + mm[l]; }
      int kind;
      size_t qq;
      split(f, kind, qq);
      acc = acc + wgt * P[kind][qq];
    }
    R w0 = R(1.0), tot = R(1.0);
    for (int l = 0; l < d; ++l) { w0 = w0 * R(4.0); tot = tot * R(6.0); }
    C[q] = (tot * ub[q] - acc) / w0;
  }
  auto Z = [&](const int* f) {
    int kind;
    size_t qq;
    split(f, kind, qq);
    return kind == 0 ? C[qq] : P[kind][qq];
  };
  // pointwise nonlinearities at every fine location, evaluated once: f_l, f_l', a per
  // kind (kind 0: at the recovered centres)
  std::vector<R> Pf[8][3], Pd[8][3], Pa[8];
  for (int s = 0; s < nk; ++s) {
    const R* z = s == 0 ? C.data() : P[s];
    Pa[s].resize(N);
    for (int l = 0; l < d; ++l) { Pf[s][l].resize(N); Pd[s][l].resize(N); }
    for (size_t q = 0; q < N; ++q) {
      Pa[s][q] = apot<R>(m, z[q]);
      for (int l = 0; l < d; ++l) { Pf[s][l][q] = flux<R>(m, l, z[q]); Pd[s][l][q] = dflux<R>(m, l, z[q]); }
    }
  }
  auto at = [&](const int* f, int& kind) {
    size_t qq;
    split(f, kind, qq);
    return qq;
  };
  std::vector<R> fU[3], aU(N);
  for (int l = 0; l < d; ++l) fU[l].resize(N);
  for (size_t q = 0; q < N; ++q) {
    for (int l = 0; l < d; ++l) fU[l][q] = flux<R>(m, l, ub[q]);
    aU[q] = apot<R>(m, ub[q]);
  }
  // transverse Simpson offsets of a face / a cell: all m with m_l = 0 along the axis l
  auto transverse = [&](int l, auto&& fn) {
    for (int o = 0; o < 27; ++o) {
      int mm[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
      bool skip = mm[l] != 0;
      for (int t = d; t < 3; ++t) if (mm[t] != 0) skip = true;
      if (skip) continue;
      R wgt = R(1.0), tot = R(1.0);
      for (int t = 0; t < d; ++t)
        if (t != l) { wgt = wgt * w1[mm[t] + 1]; tot = tot * R(6.0); }
      fn(mm, wgt, tot);
    }
  };

  // (2) high-order face fluxes F^H_l (Simpson face average of f_l) and cell potentials
  //     A^H_l (transverse Simpson average of the 1D DC potential along l)
  std::vector<R> FH[3], AH[3];
  for (int l = 0; l < d; ++l) {
    FH[l].resize(N);
    AH[l].resize(N);
    for (size_t q = 0; q < N; ++q) {
      int c[3];
      decode(q, c);
      R fs = R(0.0), as = R(0.0), tot6 = R(1.0);
      transverse(l, [&](const int* mm, R wgt, R tot) {
        int f[3] = {0, 0, 0}, fm[3], fp[3];
        for (int t = 0; t < d; ++t) f[t] = 2 * c[t] + mm[t];
        for (int t = 0; t < 3; ++t) { fm[t] = f[t]; fp[t] = f[t]; }
        fm[l] -= 1;
        fp[l] += 1;
        int kp, km, k0;
        const size_t qp = at(fp, kp), qm = at(fm, km), q0 = at(f, k0);
        if (conv) fs = fs + wgt * Pf[kp][l][qp];   // face point at fine 2i + 1 along l
        R ahat = (-Pa[km][qm] + R(8.0) * Pa[k0][q0] - Pa[kp][qp]) / R(6.0);
        as = as + wgt * ahat;
        tot6 = tot;
      });
      FH[l][q] = fs / tot6;
      AH[l][q] = as / tot6;
    }
  }

  // (3) high-order point residuals, one 5-point line per axis
  std::vector<R> RH[8][3];
  for (int s = 1; s < nk; ++s)
    for (int l = 0; l < d; ++l) {
      RH[s][l].resize(N);
      for (size_t q = 0; q < N; ++q) {
        int c[3];
        decode(q, c);
        int f0[3] = {0, 0, 0};
        for (int t = 0; t < d; ++t) f0[t] = 2 * c[t] + ((s >> t) & 1);
        R z[5], fl[5], df[5], a[5];
        for (int t = 0; t < 5; ++t) {
          int f[3] = {f0[0], f0[1], f0[2]};
          f[l] += t - 2;
          int kt;
          const size_t qt = at(f, kt);
          z[t] = Z(f);
          fl[t] = Pf[kt][l][qt];
          df[t] = Pd[kt][l][qt];
          a[t] = Pa[kt][qt];
        }
        RH[s][l][q] = conv ? line_residual<R>(z, fl, df, a, h[l]) : line_diffusion<R>(a, h[l]);
      }
    }

  // (4) low-order LLF fluxes and directional states u^{L,+-}_l with factor 2d
  R mu[3], nu[3];
  std::vector<R> FL[3], ULp[3], ULm[3];
  const R twod = R(2.0 * d);
  auto nb = [&](size_t q, int l, int step) {
    int c[3];
    decode(q, c);
    c[l] += step;
    return cell(c);
  };
  for (int l = 0; l < d; ++l) {
    mu[l] = tau / h[l];
    nu[l] = tau / (h[l] * h[l]);
    FL[l].resize(N);
    ULp[l].resize(N);
    ULm[l].resize(N);
    for (size_t q = 0; q < N; ++q) {
      if (!conv) {
        FL[l][q] = R(0.0);
        continue;
      }
      size_t qp = nb(q, l, 1);
      R al = alpha_interval<R>(m, l, ub[q], ub[qp]);
      FL[l][q] = R(0.5) * (fU[l][q] + fU[l][qp]) - R(0.5) * al * (ub[qp] - ub[q]);
    }
    for (size_t q = 0; q < N; ++q) {
      size_t qp = nb(q, l, 1), qm = nb(q, l, -1);
      if (!conv) {
        ULp[l][q] = ub[q] + twod * nu[l] * (aU[qp] - aU[q]);
        ULm[l][q] = ub[q] - twod * nu[l] * (aU[q] - aU[qm]);
        continue;
      }
      ULp[l][q] = ub[q] - twod * mu[l] * (FL[l][q] - fU[l][q]) + twod * nu[l] * (aU[qp] - aU[q]);
      ULm[l][q] = ub[q] - twod * mu[l] * (fU[l][q] - FL[l][qm]) - twod * nu[l] * (aU[q] - aU[qm]);
    }
  }

  // (5) optional smoothness blend, axis by axis (Section 5.2.3)
  std::vector<R> Fh[3], Ah[3], RP[8];
  for (int l = 0; l < d; ++l) { Fh[l] = FH[l]; Ah[l] = AH[l]; }
  for (int s = 1; s < nk; ++s) {
    RP[s].assign(N, R(0.0));
    for (size_t q = 0; q < N; ++q) {
      R acc = RH[s][0][q];
      for (int l = 1; l < d; ++l) acc = acc + RH[s][l][q];
      RP[s][q] = acc;
    }
  }
  if (p.blend) {
    std::vector<R> sl[3], tc[3], td[3];
    const R g = R(p.gamma);
    for (int l = 0; l < d; ++l) {
      sl[l].resize(N);
      tc[l].resize(N);
      td[l].resize(N);
      if (p.blend == 1) {
        std::vector<R> st(N);
        for (size_t q = 0; q < N; ++q) st[q] = s_tilde<R>(ub[nb(q, l, -1)], ub[q], ub[nb(q, l, 1)]);
        for (size_t q = 0; q < N; ++q) sl[l][q] = (st[nb(q, l, -1)] + R(4.0) * st[q] + st[nb(q, l, 1)]) / R(6.0);
      } else {
        for (size_t q = 0; q < N; ++q) sl[l][q] = s_ext[q];
      }
      for (size_t q = 0; q < N; ++q) {
        tc[l][q] = exp_(-g * (R(0.5) * (sl[l][q] + sl[l][nb(q, l, 1)])));
        td[l][q] = exp_(-g * sl[l][q]);
      }
      for (size_t q = 0; q < N; ++q) {
        Fh[l][q] = tc[l][q] * FH[l][q] + (R(1.0) - tc[l][q]) * FL[l][q];
        Ah[l][q] = td[l][q] * AH[l][q] + (R(1.0) - td[l][q]) * aU[q];
      }
    }
    // point weight along l: on an l-face (s_l = 1), the min of theta^{c,s}_l over the
    // l-faces holding the point; otherwise the min of theta^{d,s}_l over the cells
    // holding it. Low-order residual on the +-h/2 neighbours, a centre replaced by its
    // cell average.
    for (int s = 1; s < nk; ++s)
      for (size_t q = 0; q < N; ++q) {
        int c[3];
        decode(q, c);
        int f0[3] = {0, 0, 0};
        for (int t = 0; t < d; ++t) f0[t] = 2 * c[t] + ((s >> t) & 1);
        R acc = R(0.0);
        for (int l = 0; l < d; ++l) {
          R w = R(2.0);
          const bool onface = (s >> l) & 1;
          // cells holding the point: along l its own cell c_l; across t, c_t and, on an
          // odd coordinate, c_t + 1
          for (int o = 0; o < 8; ++o) {
            int cc[3] = {c[0], c[1], c[2]};
            bool ok = true;
            for (int t = 0; t < 3; ++t) {
              const int bit = (o >> t) & 1;
              if (!bit) continue;
              if (t == l || t >= d || !((s >> t) & 1)) { ok = false; break; }
              cc[t] += 1;
            }
            if (!ok) continue;
            const size_t qq = cell(cc);
            const R v = onface ? tc[l][qq] : td[l][qq];
            w = (w == R(2.0)) ? v : minr(w, v);
          }
          R zz[3];
          for (int t = 0; t < 3; ++t) {
            int f[3] = {f0[0], f0[1], f0[2]};
            f[l] += t - 1;
            int kind;
            size_t qq;
            split(f, kind, qq);
            zz[t] = kind == 0 ? ub[qq] : P[kind][qq];
          }
          R RL = low_point_residual<R>(m, l, zz[0], zz[1], zz[2], h[l]);
          acc = (l == 0) ? (w * RH[s][l][q] + (R(1.0) - w) * RL) : acc + (w * RH[s][l][q] + (R(1.0) - w) * RL);
        }
        RP[s][q] = acc;
      }
  }

  // (6) monolithic convex limiter: potential corrections with factor 3 * 2d, face
  //     corrections with 2d times the number of parts (3 * 2d with diffusion, 2d without)
  std::vector<R> Fl[3], Al[3];
  for (int l = 0; l < d; ++l) { Fl[l] = Fh[l]; Al[l] = Ah[l]; }
  if (p.limiter) {
    const R kf = R(6.0 * d), kc = R(face_factor(p, d));
    for (int l = 0; l < d; ++l) {
      for (size_t q = 0; q < N; ++q) {
        size_t qp = nb(q, l, 1);
        R dF = Fh[l][q] - FL[l][q];
        R t = minr(Theta<R>(m, ULp[l][q], ULp[l][q] - kc * mu[l] * dF),
                   Theta<R>(m, ULm[l][qp], ULm[l][qp] + kc * mu[l] * dF));
        Fl[l][q] = (t == R(1.0)) ? Fh[l][q] : FL[l][q] + t * dF;
      }
      for (size_t q = 0; q < N; ++q) {
        size_t qm = nb(q, l, -1), qp = nb(q, l, 1);
        R dA = Ah[l][q] - aU[q];
        R t = minr(minr(Theta<R>(m, ULp[l][qm], ULp[l][qm] + kf * nu[l] * dA),
                        Theta<R>(m, ULp[l][q], ULp[l][q] - kf * nu[l] * dA)),
                   minr(Theta<R>(m, ULm[l][q], ULm[l][q] - kf * nu[l] * dA),
                        Theta<R>(m, ULm[l][qp], ULm[l][qp] + kf * nu[l] * dA)));
        Al[l][q] = (t == R(1.0)) ? Ah[l][q] : aU[q] + t * dA;
      }
    }
  }

  // (7) limited cell-average update and point values with projection
  for (size_t q = 0; q < N; ++q) {
    R v = ub[q];
    for (int l = 0; l < d; ++l) {
      size_t qm = nb(q, l, -1), qp = nb(q, l, 1);
      v = v - mu[l] * (Fl[l][q] - Fl[l][qm]) + nu[l] * (Al[l][qp] - R(2.0) * Al[l][q] + Al[l][qm]);
    }
    ub_o[q] = v;
  }
  const R umin = R(p.umin), umax = R(p.umax);
  for (int s = 1; s < nk; ++s)
    for (size_t q = 0; q < N; ++q) {
      R v = P[s][q] + tau * RP[s][q];
      if (p.limiter) v = minr(maxr(v, umin), umax);
      P_o[s][q] = v;
    }
}

// ---------------------------------------------------------------------------------
// 2D forward-Euler evaluation (Sections 4 and 5.2 with d = 2).
template <class R>
void fe2d(const Model& m, const R* ub, const R* V, const R* X, const R* Y, R tau, const R* s_ext,
          R* ub_o, R* V_o, R* X_o, R* Y_o) {
  const ao_problem& p = m.p;
  const int nx = p.nx, ny = p.ny;
  const R h1 = R(p.dx), h2 = R(p.dy);
  const size_t N = (size_t)nx * ny;
  auto at = [&](int i, int j) { return (size_t)wrap(j, ny) * nx + wrap(i, nx); };

  // (1) centre value z_{i,j} = [36 zbar - 4(X_{i-1,j}+X_{ij}+Y_{i,j-1}+Y_{ij})
  //                              - (V_{i-1,j-1}+V_{i,j-1}+V_{i-1,j}+V_{ij})] / 16  (Section 4)
  std::vector<R> C(N);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      C[at(i, j)] = (R(36.0) * ub[at(i, j)] -
                     R(4.0) * (X[at(i - 1, j)] + X[at(i, j)] + Y[at(i, j - 1)] + Y[at(i, j)]) -
                     (V[at(i - 1, j - 1)] + V[at(i, j - 1)] + V[at(i - 1, j)] + V[at(i, j)])) / R(16.0);

  // (2) pointwise nonlinearities at every point type and at the cell averages
  struct PF { std::vector<R> f1, f2, d1, d2, a; };
  auto eval = [&](const R* z) {
    PF q;
    q.f1.resize(N); q.f2.resize(N); q.d1.resize(N); q.d2.resize(N); q.a.resize(N);
    for (size_t k = 0; k < N; ++k) {
      q.f1[k] = flux<R>(m, 0, z[k]); q.f2[k] = flux<R>(m, 1, z[k]);
      q.d1[k] = dflux<R>(m, 0, z[k]); q.d2[k] = dflux<R>(m, 1, z[k]);
      q.a[k] = apot<R>(m, z[k]);
    }
    return q;
  };
  PF pV = eval(V), pX = eval(X), pY = eval(Y), pC = eval(C.data());
  std::vector<R> f1U(N), f2U(N), aU(N);
  for (size_t k = 0; k < N; ++k) {
    f1U[k] = flux<R>(m, 0, ub[k]); f2U[k] = flux<R>(m, 1, ub[k]); aU[k] = apot<R>(m, ub[k]);
  }

  // (3) high-order fluxes (Simpson face average of f_l at the face's three points) and
  //     cell potentials A^H_l (transverse Simpson average of the 1D DC potential).
  std::vector<R> FH1(N), FH2(N), AH1(N), AH2(N);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      // x-face (i+1/2, j): V_{i,j-1}, X_{ij}, V_{ij}
      FH1[at(i, j)] = (pV.f1[at(i, j - 1)] + R(4.0) * pX.f1[at(i, j)] + pV.f1[at(i, j)]) / R(6.0);
      // y-face (i, j+1/2): V_{i-1,j}, Y_{ij}, V_{ij}
      FH2[at(i, j)] = (pV.f2[at(i - 1, j)] + R(4.0) * pY.f2[at(i, j)] + pV.f2[at(i, j)]) / R(6.0);
      // a^ along x-lines at y_{j-1/2}, y_j, y_{j+1/2}, combined with Simpson weights 1,4,1
      R lo = (-pV.a[at(i - 1, j - 1)] + R(8.0) * pY.a[at(i, j - 1)] - pV.a[at(i, j - 1)]) / R(6.0);
      R mid = (-pX.a[at(i - 1, j)] + R(8.0) * pC.a[at(i, j)] - pX.a[at(i, j)]) / R(6.0);
      R hi = (-pV.a[at(i - 1, j)] + R(8.0) * pY.a[at(i, j)] - pV.a[at(i, j)]) / R(6.0);
      AH1[at(i, j)] = (lo + R(4.0) * mid + hi) / R(6.0);
      // a^ along y-lines at x_{i-1/2}, x_i, x_{i+1/2}
      R le = (-pV.a[at(i - 1, j - 1)] + R(8.0) * pX.a[at(i - 1, j)] - pV.a[at(i - 1, j)]) / R(6.0);
      R ce = (-pY.a[at(i, j - 1)] + R(8.0) * pC.a[at(i, j)] - pY.a[at(i, j)]) / R(6.0);
      R ri = (-pV.a[at(i, j - 1)] + R(8.0) * pX.a[at(i, j)] - pV.a[at(i, j)]) / R(6.0);
      AH2[at(i, j)] = (le + R(4.0) * ce + ri) / R(6.0);
    }

  // (4) high-order point residuals per direction on the 5-point lines (eq. 2d_af_dc;
  //     the operators are the 1D ones with half-index shifts)
  auto line = [&](const PF& q0, size_t k0, const PF& q1, size_t k1, const PF& q2, size_t k2,
                  const PF& q3, size_t k3, const PF& q4, size_t k4, const R* z0, const R* z1,
                  const R* z2, const R* z3, const R* z4, int dir, R h) {
    R z[5] = {z0[k0], z1[k1], z2[k2], z3[k3], z4[k4]};
    const PF* q[5] = {&q0, &q1, &q2, &q3, &q4};
    size_t kk[5] = {k0, k1, k2, k3, k4};
    R f[5], d[5], a[5];
    for (int t = 0; t < 5; ++t) {
      f[t] = dir == 0 ? q[t]->f1[kk[t]] : q[t]->f2[kk[t]];
      d[t] = dir == 0 ? q[t]->d1[kk[t]] : q[t]->d2[kk[t]];
      a[t] = q[t]->a[kk[t]];
    }
    return line_residual<R>(z, f, d, a, h);
  };
  const R* Cp = C.data();
  std::vector<R> RV1(N), RV2(N), RX1(N), RX2(N), RY1(N), RY2(N);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = at(i, j);
      RV1[k] = line(pV, at(i - 1, j), pY, at(i, j), pV, k, pY, at(i + 1, j), pV, at(i + 1, j),
                    V, Y, V, Y, V, 0, h1);
      RV2[k] = line(pV, at(i, j - 1), pX, at(i, j), pV, k, pX, at(i, j + 1), pV, at(i, j + 1),
                    V, X, V, X, V, 1, h2);
      RX1[k] = line(pX, at(i - 1, j), pC, at(i, j), pX, k, pC, at(i + 1, j), pX, at(i + 1, j),
                    X, Cp, X, Cp, X, 0, h1);
      RX2[k] = line(pX, at(i, j - 1), pV, at(i, j - 1), pX, k, pV, at(i, j), pX, at(i, j + 1),
                    X, V, X, V, X, 1, h2);
      RY1[k] = line(pY, at(i - 1, j), pV, at(i - 1, j), pY, k, pV, at(i, j), pY, at(i + 1, j),
                    Y, V, Y, V, Y, 0, h1);
      RY2[k] = line(pY, at(i, j - 1), pC, at(i, j), pY, k, pC, at(i, j + 1), pY, at(i, j + 1),
                    Y, Cp, Y, Cp, Y, 1, h2);
    }

  // (5) low-order LLF fluxes and the directional states u^{L,+-}_l with factor 2d = 4
  const R mu1 = tau / h1, mu2 = tau / h2, nu1 = tau / (h1 * h1), nu2 = tau / (h2 * h2);
  std::vector<R> FL1(N), FL2(N), ULp1(N), ULm1(N), ULp2(N), ULm2(N);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = at(i, j), kx = at(i + 1, j), ky = at(i, j + 1);
      R a1 = alpha_interval<R>(m, 0, ub[k], ub[kx]);
      FL1[k] = R(0.5) * (f1U[k] + f1U[kx]) - R(0.5) * a1 * (ub[kx] - ub[k]);
      R a2 = alpha_interval<R>(m, 1, ub[k], ub[ky]);
      FL2[k] = R(0.5) * (f2U[k] + f2U[ky]) - R(0.5) * a2 * (ub[ky] - ub[k]);
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = at(i, j);
      ULp1[k] = ub[k] - R(4.0) * mu1 * (FL1[k] - f1U[k]) + R(4.0) * nu1 * (aU[at(i + 1, j)] - aU[k]);
      ULm1[k] = ub[k] - R(4.0) * mu1 * (f1U[k] - FL1[at(i - 1, j)]) - R(4.0) * nu1 * (aU[k] - aU[at(i - 1, j)]);
      ULp2[k] = ub[k] - R(4.0) * mu2 * (FL2[k] - f2U[k]) + R(4.0) * nu2 * (aU[at(i, j + 1)] - aU[k]);
      ULm2[k] = ub[k] - R(4.0) * mu2 * (f2U[k] - FL2[at(i, j - 1)]) - R(4.0) * nu2 * (aU[k] - aU[at(i, j - 1)]);
    }

  // (6) optional smoothness blend, direction by direction (Section 5.2.3 / 5.1.3)
  std::vector<R> Fh1(FH1), Fh2(FH2), Ah1(AH1), Ah2(AH2);
  std::vector<R> RV(N), RX(N), RY(N);
  for (size_t k = 0; k < N; ++k) {
    RV[k] = RV1[k] + RV2[k]; RX[k] = RX1[k] + RX2[k]; RY[k] = RY1[k] + RY2[k];
  }
  if (p.blend) {
    std::vector<R> s1(N), s2(N);
    if (p.blend == 1) {
      std::vector<R> st1(N), st2(N);
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          st1[at(i, j)] = s_tilde<R>(ub[at(i - 1, j)], ub[at(i, j)], ub[at(i + 1, j)]);
          st2[at(i, j)] = s_tilde<R>(ub[at(i, j - 1)], ub[at(i, j)], ub[at(i, j + 1)]);
        }
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          s1[at(i, j)] = (st1[at(i - 1, j)] + R(4.0) * st1[at(i, j)] + st1[at(i + 1, j)]) / R(6.0);
          s2[at(i, j)] = (st2[at(i, j - 1)] + R(4.0) * st2[at(i, j)] + st2[at(i, j + 1)]) / R(6.0);
        }
    } else {
      for (size_t k = 0; k < N; ++k) { s1[k] = s_ext[k]; s2[k] = s_ext[k]; }
    }
    const R g = R(p.gamma);
    std::vector<R> tc1(N), tc2(N), td1(N), td2(N);
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t k = at(i, j);
        tc1[k] = exp_(-g * (R(0.5) * (s1[k] + s1[at(i + 1, j)])));
        tc2[k] = exp_(-g * (R(0.5) * (s2[k] + s2[at(i, j + 1)])));
        td1[k] = exp_(-g * s1[k]);
        td2[k] = exp_(-g * s2[k]);
      }
    for (size_t k = 0; k < N; ++k) {
      Fh1[k] = tc1[k] * FH1[k] + (R(1.0) - tc1[k]) * FL1[k];
      Fh2[k] = tc2[k] * FH2[k] + (R(1.0) - tc2[k]) * FL2[k];
      Ah1[k] = td1[k] * AH1[k] + (R(1.0) - td1[k]) * aU[k];
      Ah2[k] = td2[k] * AH2[k] + (R(1.0) - td2[k]) * aU[k];
    }
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t k = at(i, j);
        // low-order point residuals on the +-h/2 neighbours
        R LV1 = low_point_residual<R>(m, 0, Y[k], V[k], Y[at(i + 1, j)], h1);
        R LV2 = low_point_residual<R>(m, 1, X[k], V[k], X[at(i, j + 1)], h2);
        R LX1 = low_point_residual<R>(m, 0, ub[k], X[k], ub[at(i + 1, j)], h1);
        R LX2 = low_point_residual<R>(m, 1, V[at(i, j - 1)], X[k], V[k], h2);
        R LY1 = low_point_residual<R>(m, 0, V[at(i - 1, j)], Y[k], V[k], h1);
        R LY2 = low_point_residual<R>(m, 1, ub[k], Y[k], ub[at(i, j + 1)], h2);
        // direction weights at each point type
        R wV1 = minr(tc1[k], tc1[at(i, j + 1)]);
        R wV2 = minr(tc2[k], tc2[at(i + 1, j)]);
        R wX1 = tc1[k];
        R wX2 = minr(td2[k], td2[at(i + 1, j)]);
        R wY1 = minr(td1[k], td1[at(i, j + 1)]);
        R wY2 = tc2[k];
        RV[k] = (wV1 * RV1[k] + (R(1.0) - wV1) * LV1) + (wV2 * RV2[k] + (R(1.0) - wV2) * LV2);
        RX[k] = (wX1 * RX1[k] + (R(1.0) - wX1) * LX1) + (wX2 * RX2[k] + (R(1.0) - wX2) * LX2);
        RY[k] = (wY1 * RY1[k] + (R(1.0) - wY1) * LY1) + (wY2 * RY2[k] + (R(1.0) - wY2) * LY2);
      }
  }

  // (7) monolithic convex limiter (eqs. multid_convection_limiting_parameter,
  //     multid_diffusion_limiting_parameter): potential corrections with factor
  //     3*2d = 12, face corrections with 2d times the number of parts (12 with
  //     diffusion, 4 without)
  std::vector<R> Fl1(Fh1), Fl2(Fh2), Al1(Ah1), Al2(Ah2);
  if (p.limiter) {
    const R k12 = R(12.0), kc = R(face_factor(p, 2));
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t k = at(i, j), kx = at(i + 1, j), ky = at(i, j + 1);
        R dF1 = Fh1[k] - FL1[k];
        R t1 = minr(Theta<R>(m, ULp1[k], ULp1[k] - kc * mu1 * dF1),
                    Theta<R>(m, ULm1[kx], ULm1[kx] + kc * mu1 * dF1));
        Fl1[k] = (t1 == R(1.0)) ? Fh1[k] : FL1[k] + t1 * dF1;
        R dF2 = Fh2[k] - FL2[k];
        R t2 = minr(Theta<R>(m, ULp2[k], ULp2[k] - kc * mu2 * dF2),
                    Theta<R>(m, ULm2[ky], ULm2[ky] + kc * mu2 * dF2));
        Fl2[k] = (t2 == R(1.0)) ? Fh2[k] : FL2[k] + t2 * dF2;
      }
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t k = at(i, j);
        size_t xm = at(i - 1, j), xp = at(i + 1, j), ym = at(i, j - 1), yp = at(i, j + 1);
        R dA1 = Ah1[k] - aU[k];
        R t1 = minr(minr(Theta<R>(m, ULp1[xm], ULp1[xm] + k12 * nu1 * dA1),
                         Theta<R>(m, ULp1[k], ULp1[k] - k12 * nu1 * dA1)),
                    minr(Theta<R>(m, ULm1[k], ULm1[k] - k12 * nu1 * dA1),
                         Theta<R>(m, ULm1[xp], ULm1[xp] + k12 * nu1 * dA1)));
        Al1[k] = (t1 == R(1.0)) ? Ah1[k] : aU[k] + t1 * dA1;
        R dA2 = Ah2[k] - aU[k];
        R t2 = minr(minr(Theta<R>(m, ULp2[ym], ULp2[ym] + k12 * nu2 * dA2),
                         Theta<R>(m, ULp2[k], ULp2[k] - k12 * nu2 * dA2)),
                    minr(Theta<R>(m, ULm2[k], ULm2[k] - k12 * nu2 * dA2),
                         Theta<R>(m, ULm2[yp], ULm2[yp] + k12 * nu2 * dA2)));
        Al2[k] = (t2 == R(1.0)) ? Ah2[k] : aU[k] + t2 * dA2;
      }
  }

  // (8) limited cell-average update (eq. multid_limited_average)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = at(i, j);
      ub_o[k] = ub[k] - mu1 * (Fl1[k] - Fl1[at(i - 1, j)]) - mu2 * (Fl2[k] - Fl2[at(i, j - 1)]) +
                nu1 * (Al1[at(i + 1, j)] - R(2.0) * Al1[k] + Al1[at(i - 1, j)]) +
                nu2 * (Al2[at(i, j + 1)] - R(2.0) * Al2[k] + Al2[at(i, j - 1)]);
    }
  // (9) point values: high-order update and projection (Section 5.2.2)
  const R umin = R(p.umin), umax = R(p.umax);
  for (size_t k = 0; k < N; ++k) {
    R v = V[k] + tau * RV[k], x = X[k] + tau * RX[k], y = Y[k] + tau * RY[k];
    if (p.limiter) {
      v = minr(maxr(v, umin), umax); x = minr(maxr(x, umin), umax); y = minr(maxr(y, umin), umax);
    }
    V_o[k] = v; X_o[k] = x; Y_o[k] = y;
  }
}

// ---------------------------------------------------------------------------------
// Time integration (Section 3.2; SSP-RK3 of Gottlieb-Shu-Tadmor and SSP-RK(5,4) of
// Spiteri-Ruuth written as convex combinations of forward-Euler steps, Section 5).

// SSP-RK(5,4) Shu-Osher coefficients alpha[k][l], beta[k][l] (row k = stage output k+1,
// column l = input u^(l)); values from Spiteri & Ruuth (2002), pinned in the tests by
// the order-4 conditions and by the z^5 coefficient eta = 0.004477718303076 (Section 3.2).
const double RK54_A[5][5] = {
    {1.0, 0, 0, 0, 0},
    {0.444370493651235, 0.555629506348765, 0, 0, 0},
    {0.620101851488403, 0, 0.379898148511597, 0, 0},
    {0.178079954393132, 0, 0, 0.821920045606868, 0},
    {0, 0, 0.517231671970585, 0.096059710526147, 0.386708617503269}};
const double RK54_B[5][5] = {
    {0.391752226571890, 0, 0, 0, 0},
    {0, 0.368410593050371, 0, 0, 0},
    {0, 0, 0.251891774271694, 0, 0},
    {0, 0, 0, 0.544974750228521, 0},
    {0, 0, 0, 0.063692468666290, 0.226007483236906}};

struct State {
  std::vector<double> a[8];
};

int ncomp(const ao_problem& p) { return 1 << p.dim; }
size_t ncell(const ao_problem& p) {
  return (size_t)p.nx * (p.dim >= 2 ? p.ny : 1) * (p.dim == 3 ? p.nz : 1);
}
// values in component c: a bounded 1D mesh has n+1 point values
size_t comp_size(const ao_problem& p, int c) {
  if (p.bc == 0 || c == 0) return ncell(p);
  if (p.dim == 1) return ncell(p) + 1;
  const size_t nx = p.nx, ny = p.ny;
  return c == 1 ? (nx + 1) * (ny + 1) : (c == 2 ? (nx + 1) * ny : nx * (ny + 1));
}

// combinations the oracle implements: boundaries and Appendix A in 1D only, an
// external indicator only on a periodic mesh, Appendix A without the blend
bool supported(const ao_problem& p) {
  if (p.dim < 1 || p.dim > 3) return false;
  if (p.dim == 3 && (p.bc != 0 || p.flux_kind == 3)) return false;   // 3D: periodic, no Buckley-Leverett
  if ((p.bc == 1 || p.nodc) && p.dim != 1) return false;
  if (p.bc < 0 || p.bc > 2) return false;
  if (p.bc != 0 && (p.nx < 4 || (p.dim == 2 && p.ny < 4) || p.blend == 2)) return false;
  if (p.nodc && p.blend) return false;
  return true;
}

// Even extension of a bounded direction with n cells, periodic with period 2n: the cell
// index i (cell i spans [x_{i-1/2}, x_{i+1/2}]) and the face index k = j + 1 of the point
// u_{j+1/2} (k = 0 .. n from end to end) mapped into the stored range.
inline int reflect_cell(int i, int n) {
  int r = ((i % (2 * n)) + 2 * n) % (2 * n);
  return r < n ? r : 2 * n - 1 - r;
}
inline int reflect_face(int k, int n) {
  int r = ((k % (2 * n)) + 2 * n) % (2 * n);
  return r <= n ? r : 2 * n - r;
}

// Dirichlet boundary point values stay at the boundary data through every combination
void hold_dirichlet(const ao_problem& p, std::vector<double>* a) {
  if (p.dim != 1 || p.bc != 1) return;
  a[1][0] = p.bc_left;
  a[1][p.nx] = p.bc_right;
}

// Forward-Euler step on a 2D rectangle with outflow ends: the periodic step on the
// rectangle padded with G ghost layers on every side (every DoF kind evenly reflected
// about the boundary lines), restricted to the rectangle's DoFs. Each output reads
// inputs at most 3 cells away, so the wrap of the padded periodic mesh never reaches
// the rectangle's DoFs.
void fe2d_outflow(const Model& m, const State& in, double tau, State& out) {
  const ao_problem& p = m.p;
  const int nx = p.nx, ny = p.ny, G = 5, NX = nx + 2 * G, NY = ny + 2 * G;
  Model mp = m;
  mp.p.nx = NX;
  mp.p.ny = NY;
  mp.p.bc = 0;
  const size_t N = (size_t)NX * NY;
  std::vector<double> ub(N), V(N), X(N), Y(N), ubo(N), Vo(N), Xo(N), Yo(N);
  for (int J = 0; J < NY; ++J)
    for (int I = 0; I < NX; ++I) {
      const int i = I - G, j = J - G;   // cell (i, j); its corner V_{ij}, edges X_{ij}, Y_{ij}
      const int ci = reflect_cell(i, nx), cj = reflect_cell(j, ny);
      const int fi = reflect_face(i + 1, nx), fj = reflect_face(j + 1, ny);
      const size_t g = (size_t)J * NX + I;
      ub[g] = in.a[0][(size_t)cj * nx + ci];
      V[g] = in.a[1][(size_t)fj * (nx + 1) + fi];
      X[g] = in.a[2][(size_t)cj * (nx + 1) + fi];
      Y[g] = in.a[3][(size_t)fj * nx + ci];
    }
  fe2d<double>(mp, ub.data(), V.data(), X.data(), Y.data(), tau, nullptr, ubo.data(), Vo.data(), Xo.data(),
               Yo.data());
  auto P = [&](int i, int j) { return (size_t)(j + G) * NX + (i + G); };
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) out.a[0][(size_t)j * nx + i] = ubo[P(i, j)];
  for (int j = -1; j < ny; ++j)
    for (int i = -1; i < nx; ++i) out.a[1][(size_t)(j + 1) * (nx + 1) + (i + 1)] = Vo[P(i, j)];
  for (int j = 0; j < ny; ++j)
    for (int i = -1; i < nx; ++i) out.a[2][(size_t)j * (nx + 1) + (i + 1)] = Xo[P(i, j)];
  for (int j = -1; j < ny; ++j)
    for (int i = 0; i < nx; ++i) out.a[3][(size_t)(j + 1) * nx + i] = Yo[P(i, j)];
}

void fe(const Model& m, const State& in, double tau, const double* s_ext, State& out) {
  const ao_problem& p = m.p;
  for (int c = 0; c < ncomp(p); ++c) out.a[c].assign(comp_size(p, c), 0.0);
  if (p.dim == 3) {
    const int n[3] = {p.nx, p.ny, p.nz};
    const double h[3] = {p.dx, p.dy, p.dz};
    const double* P[8];
    double* Po[8];
    for (int c = 1; c < 8; ++c) { P[c] = in.a[c].data(); Po[c] = out.a[c].data(); }
    fend<double>(m, 3, n, h, in.a[0].data(), P, tau, s_ext, out.a[0].data(), Po);
  } else if (p.dim == 2 && p.bc != 0)
    fe2d_outflow(m, in, tau, out);
  else if (p.dim == 1)
    fe1d<double>(m, in.a[0].data(), in.a[1].data(), tau, s_ext, out.a[0].data(), out.a[1].data());
  else
    fe2d<double>(m, in.a[0].data(), in.a[1].data(), in.a[2].data(), in.a[3].data(), tau, s_ext,
                 out.a[0].data(), out.a[1].data(), out.a[2].data(), out.a[3].data());
}

// Post-stage safeguard: exact comparisons against [umin, umax]; excesses up to clamp_tol
// are clamped and counted, larger ones flag an error.
void safeguard(const ao_problem& p, State& s, ao_stats* st) {
  if (!p.limiter) return;
  for (int c = 0; c < ncomp(p); ++c)
    for (double& v : s.a[c]) {
      double e = 0.0;
      if (v < p.umin) e = p.umin - v;
      else if (v > p.umax) e = v - p.umax;
      if (e == 0.0) continue;
      if (e > p.clamp_tol) { if (st) st->error = 1; continue; }
      v = v < p.umin ? p.umin : p.umax;
      if (st) { st->clamps++; st->max_excess = std::max(st->max_excess, e); }
    }
}

State combine(const ao_problem& p, double a, const State& x, double b, const State& y) {
  State r;
  for (int c = 0; c < ncomp(p); ++c) {
    r.a[c].resize(x.a[c].size());
    for (size_t k = 0; k < x.a[c].size(); ++k) r.a[c][k] = a * x.a[c][k] + b * y.a[c][k];
  }
  hold_dirichlet(p, r.a);
  return r;
}

Model make_model(const ao_problem* p) {
  Model m;
  m.p = *p;
  find_crit(m);
  return m;
}

State load(const ao_problem& p, double* const* arr) {
  State s;
  for (int c = 0; c < ncomp(p); ++c) s.a[c].assign(arr[c], arr[c] + comp_size(p, c));
  return s;
}
void store(const ao_problem& p, const State& s, double* const* arr) {
  for (int c = 0; c < ncomp(p); ++c) std::memcpy(arr[c], s.a[c].data(), s.a[c].size() * sizeof(double));
}

}  // namespace

extern "C" {

// One forward-Euler evaluation out = FE(in, tau) with limiter/projection/blend as set
// in *p. Arrays: dim 1 -> {ub, P}; dim 2 -> {ub, V, X, Y}. s_ext: per-cell indicator
// (blend == 2) or NULL.
int ao_fe(const ao_problem* p, double* const* in, double tau, const double* s_ext, double* const* out) {
  if (!supported(*p)) return -2;
  Model m = make_model(p);
  State a = load(*p, in), b;
  fe(m, a, tau, s_ext, b);
  store(*p, b, out);
  return 0;
}

}  // extern "C"

namespace {

// One full time step with rk = 3 (SSP-RK3) or 54 (SSP-RK(5,4)); state updated in place.
int step_model(const Model& m, int rk, double* const* state, double dt, const double* s_ext, ao_stats* st) {
  const ao_problem* p = &m.p;
  State u0 = load(*p, state), t;
  if (rk == 3) {
    fe(m, u0, dt, s_ext, t);
    State u1 = t;
    safeguard(*p, u1, st);
    fe(m, u1, dt, s_ext, t);
    State u2 = combine(*p, 0.75, u0, 0.25, t);
    safeguard(*p, u2, st);
    fe(m, u2, dt, s_ext, t);
    State u3 = combine(*p, 1.0 / 3.0, u0, 2.0 / 3.0, t);
    safeguard(*p, u3, st);
    store(*p, u3, state);
    return st && st->error ? -4 : 0;
  }
  if (rk == 54) {
    const double(*A)[5] = RK54_A;
    const double(*B)[5] = RK54_B;
    State u[5];
    u[0] = u0;
    fe(m, u[0], B[0][0] / A[0][0] * dt, s_ext, t);
    u[1] = combine(*p, 0.0, u0, A[0][0], t);
    safeguard(*p, u[1], st);
    fe(m, u[1], B[1][1] / A[1][1] * dt, s_ext, t);
    u[2] = combine(*p, A[1][0], u[0], A[1][1], t);
    safeguard(*p, u[2], st);
    fe(m, u[2], B[2][2] / A[2][2] * dt, s_ext, t);
    u[3] = combine(*p, A[2][0], u[0], A[2][2], t);
    safeguard(*p, u[3], st);
    fe(m, u[3], B[3][3] / A[3][3] * dt, s_ext, t);
    u[4] = combine(*p, A[3][0], u[0], A[3][3], t);
    safeguard(*p, u[4], st);
    // last row: the same u^(3) enters with its own step ratio, so its limited FE step is
    // evaluated again at that ratio (the limiter is nonlinear in tau).
    fe(m, u[3], B[4][3] / A[4][3] * dt, s_ext, t);
    State part = combine(*p, A[4][2], u[2], A[4][3], t);
    fe(m, u[4], B[4][4] / A[4][4] * dt, s_ext, t);
    State u5 = combine(*p, 1.0, part, A[4][4], t);
    safeguard(*p, u5, st);
    store(*p, u5, state);
    return st && st->error ? -4 : 0;
  }
  return -1;
}

}  // namespace

extern "C" {

int ao_step(const ao_problem* p, int rk, double* const* state, double dt, const double* s_ext, ao_stats* st) {
  if (!supported(*p)) return -2;
  return step_model(make_model(p), rk, state, dt, s_ext, st);
}

}  // extern "C"

namespace {

// CFL time step dt = C / max_{faces,l} (alpha_face / h_l + kappa_max / h_l^2)
// (eq. multid_av_pp_dt; 1D eq. 1d_av_pp_dt), additionally capped by the linear
// stability of the unlimited high-order scheme for diffusion, dt <= Cd h_l^2 / kappa_max
// (cfl_diff <= 0 disables the cap). A bounded 1D mesh has faces -1..n-1, the two end
// faces between a boundary cell and its ghost cell included. km = kappa_max(m).
double dt_model(const Model& m, const double* ub, double cfl, double cfl_diff, double km) {
  const ao_problem* p = &m.p;
  double worst = 0.0;
  if (p->dim == 3) {
    const int n[3] = {p->nx, p->ny, p->nz};
    const double h[3] = {p->dx, p->dy, p->dz};
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          const double u = ub[((size_t)k * n[1] + j) * n[0] + i];
          const double un[3] = {ub[((size_t)k * n[1] + j) * n[0] + wrap(i + 1, n[0])],
                                ub[((size_t)k * n[1] + wrap(j + 1, n[1])) * n[0] + i],
                                ub[((size_t)wrap(k + 1, n[2]) * n[1] + j) * n[0] + i]};
          for (int l = 0; l < 3; ++l)
            worst = std::max(worst, alpha_interval<double>(m, l, u, un[l]) / h[l] + km / (h[l] * h[l]));
        }
  } else if (p->dim == 1) {
    for (int f = p->bc != 0 ? -1 : 0; f < p->nx; ++f) {
      double a = alpha_interval<double>(m, 0, cell_at<double>(*p, ub, f), cell_at<double>(*p, ub, f + 1));
      worst = std::max(worst, a / p->dx + km / (p->dx * p->dx));
    }
  } else {
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        double u = ub[(size_t)j * p->nx + i];
        // the neighbour across the right / top face (an outflow ghost repeats the cell)
        double ur = ub[(size_t)j * p->nx + wrap(i + 1, p->nx)], ut = ub[(size_t)wrap(j + 1, p->ny) * p->nx + i];
        if (p->bc != 0 && i + 1 == p->nx) ur = u;
        if (p->bc != 0 && j + 1 == p->ny) ut = u;
        double a1 = alpha_interval<double>(m, 0, u, ur);
        double a2 = alpha_interval<double>(m, 1, u, ut);
        worst = std::max(worst, a1 / p->dx + km / (p->dx * p->dx));
        worst = std::max(worst, a2 / p->dy + km / (p->dy * p->dy));
      }
  }
  double rate = worst / cfl;
  if (cfl_diff > 0.0 && km > 0.0) {
    double hmin = p->dim == 1 ? p->dx : std::min(p->dx, p->dy);
    if (p->dim == 3) hmin = std::min(hmin, p->dz);
    rate = std::max(rate, km / (hmin * hmin) / cfl_diff);
  }
  return rate > 0.0 ? 1.0 / rate : INFINITY;
}

}  // namespace

extern "C" {

double ao_dt(const ao_problem* p, const double* ub, double cfl, double cfl_diff) {
  Model m = make_model(p);
  return dt_model(m, ub, cfl, cfl_diff, kappa_max(m));
}

// Steps with the CFL time step until time T: each step is clipped to the time left,
// and stepping ends once less than T * 1e-14 is left. *nsteps = steps taken.
int ao_run(const ao_problem* p, int rk, double* const* state, double T, double cfl, double cfl_diff,
           long long* nsteps, ao_stats* st) {
  if (!supported(*p)) return -2;
  Model m = make_model(p);
  const double km = kappa_max(m);
  double t = 0.0;
  long long k = 0;
  while (T - t > T * 1e-14) {
    double dt = std::min(dt_model(m, state[0], cfl, cfl_diff, km), T - t);
    int rc = step_model(m, rk, state, dt, nullptr, st);
    if (rc) return rc;
    t += dt;
    ++k;
  }
  if (nsteps) *nsteps = k;
  return 0;
}

// First-order reference scheme for the cell averages alone (the kind of scheme the
// paper's reference solutions of Section 6 come from): forward Euler with the LLF
// flux (interval wave speed) and the central second difference of a,
//   ub_i <- ub_i - mu (F_{i+1/2} - F_{i-1/2}) + nu (a(ub_{i+1}) - 2 a(ub_i) + a(ub_{i-1})),
// ghost cells by the boundary rule, dt = cfl / max_faces(alpha/h + 2 kappa_max/h^2)
// (monotone for cfl <= 1), the last step clipped to T. 1D only.
int ao_first_order_run(const ao_problem* p, double* ub, double T, double cfl, long long* nsteps) {
  if (p->dim != 1 || !supported(*p)) return -2;
  Model m = make_model(p);
  const int n = p->nx;
  const double h = p->dx, km = kappa_max(m);
  std::vector<double> F(n + 1), un(n);
  double t = 0.0;
  long long k = 0;
  while (T - t > T * 1e-14) {
    double worst = 0.0;
    for (int f = -1; f < n; ++f) {
      double a = alpha_interval<double>(m, 0, cell_at<double>(*p, ub, f), cell_at<double>(*p, ub, f + 1));
      worst = std::max(worst, a / h + 2.0 * km / (h * h));
    }
    double dt = std::min(cfl / worst, T - t);
    const double mu = dt / h, nu = dt / (h * h);
    for (int f = -1; f < n; ++f) {
      double ul = cell_at<double>(*p, ub, f), ur = cell_at<double>(*p, ub, f + 1);
      double a = alpha_interval<double>(m, 0, ul, ur);
      F[f + 1] = 0.5 * (flux<double>(m, 0, ul) + flux<double>(m, 0, ur)) - 0.5 * a * (ur - ul);
    }
    for (int i = 0; i < n; ++i) {
      double am = apot<double>(m, cell_at<double>(*p, ub, i - 1)), a0 = apot<double>(m, ub[i]),
             ap = apot<double>(m, cell_at<double>(*p, ub, i + 1));
      un[i] = ub[i] - mu * (F[i + 1] - F[i]) + nu * (ap - 2.0 * a0 + am);
    }
    std::copy(un.begin(), un.end(), ub);
    t += dt;
    ++k;
  }
  if (nsteps) *nsteps = k;
  return 0;
}

double ao_kappa_max(const ao_problem* p) { return kappa_max(make_model(p)); }

// The dimension-generic fine-grid evaluation applied to a periodic 1D, 2D or 3D state in
// the library's array order (1D: ub, P; 2D: ub, V, X, Y; 3D: by kind). For 1D and 2D it
// restates the dedicated evaluations in another form; the two must agree.
int ao_fe_generic(const ao_problem* p, double* const* in, double tau, const double* s_ext, double* const* out) {
  if (!supported(*p) || p->bc != 0 || p->nodc) return -2;
  Model m = make_model(p);
  const int d = p->dim;
  const int n[3] = {p->nx, p->ny, p->nz};
  const double h[3] = {p->dx, p->dy, p->dz};
  const double* P[8] = {nullptr};
  double* Po[8] = {nullptr};
  // kind of each array after ub: 1D P -> 1; 2D V, X, Y -> 3, 1, 2; 3D by kind
  const int kind2[4] = {0, 3, 1, 2};
  for (int c = 1; c < (1 << d); ++c) {
    const int k = d == 2 ? kind2[c] : c;
    P[k] = in[c];
    Po[k] = out[c];
  }
  fend<double>(m, d, n, h, in[0], P, tau, s_ext, out[0], Po);
  return 0;
}

double ao_alpha_interval(const ao_problem* p, int dir, double a, double b) {
  return alpha_interval<double>(make_model(p), dir, a, b);
}

void ao_point_funcs(const ao_problem* p, int dir, double u, double* f, double* df, double* a) {
  Model m = make_model(p);
  *f = flux<double>(m, dir, u);
  *df = dflux<double>(m, dir, u);
  *a = apot<double>(m, u);
}

double ao_theta(const ao_problem* p, double zL, double zH) { return Theta<double>(make_model(p), zL, zH); }

void ao_rk54_coefs(double* alpha, double* beta) {
  for (int k = 0; k < 5; ++k)
    for (int l = 0; l < 5; ++l) { alpha[k * 5 + l] = RK54_A[k][l]; beta[k * 5 + l] = RK54_B[k][l]; }
}

// Flop count of one FE evaluation on the given state (counting scalar; every
// +,-,*,/ and exp counts one). out[0..4] = add, mul, div, exp, cmp.
void ao_flop_count(const ao_problem* p, double* const* in, double tau, const double* s_ext, long long* out) {
  for (int k = 0; k < 5; ++k) out[k] = 0;
  if (!supported(*p) || (p->dim == 2 && p->bc != 0)) return;   // periodic 2D / 3D and all 1D forms
  Model m = make_model(p);
  g_flops = FlopCounter();
  size_t n = ncell(*p);
  std::vector<Cnt> a[8], b[8], se;
  for (int c = 0; c < ncomp(*p); ++c) {
    a[c].resize(comp_size(*p, c)); b[c].resize(comp_size(*p, c));
    for (size_t k = 0; k < a[c].size(); ++k) a[c][k] = Cnt(in[c][k]);
  }
  if (s_ext) { se.resize(n); for (size_t k = 0; k < n; ++k) se[k] = Cnt(s_ext[k]); }
  if (p->dim == 3) {
    const int n[3] = {p->nx, p->ny, p->nz};
    const Cnt h[3] = {Cnt(p->dx), Cnt(p->dy), Cnt(p->dz)};
    const Cnt* P[8];
    Cnt* Po[8];
    for (int c = 1; c < 8; ++c) { P[c] = a[c].data(); Po[c] = b[c].data(); }
    fend<Cnt>(m, 3, n, h, a[0].data(), P, Cnt(tau), s_ext ? se.data() : nullptr, b[0].data(), Po);
  } else if (p->dim == 1)
    fe1d<Cnt>(m, a[0].data(), a[1].data(), Cnt(tau), s_ext ? se.data() : nullptr, b[0].data(), b[1].data());
  else
    fe2d<Cnt>(m, a[0].data(), a[1].data(), a[2].data(), a[3].data(), Cnt(tau), s_ext ? se.data() : nullptr,
              b[0].data(), b[1].data(), b[2].data(), b[3].data());
  out[0] = g_flops.add; out[1] = g_flops.mul; out[2] = g_flops.div; out[3] = g_flops.exp; out[4] = g_flops.cmp;
}

}  // extern "C"
