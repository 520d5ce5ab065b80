// Device-side problem functions for the active flux stage kernels: convection flux
// f_l, its derivative, the diffusion potential a(u) = int kappa, the interval maximum
// of |f_l'| used by the LLF low-order flux (Section 5.1.1 / 5.2 of arXiv 2510.11527),
// and the limiter function Theta (Section 5.1.1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "af.h"

namespace af {

// Flux kinds are template parameters of the kernels (compile-time dispatch).
enum : int { FLUX_ZERO = AF_FLUX_ZERO, FLUX_LINEAR = AF_FLUX_LINEAR, FLUX_BURGERS = AF_FLUX_BURGERS,
             FLUX_BL = AF_FLUX_BL };

// Problem parameters passed by value to every kernel.
struct DevModel {
  int flux_kind;
  int diff_kind;
  double fp[4];          // flux parameters
  double dp[4];          // diffusion parameters
  int ncrit[2];          // interior extrema of f_l' (Buckley-Leverett)
  double crit[2][8];
  double critv[2][8];    // |f_l'| at those extrema
  double umin, umax;
  double umid;           // (umin + umax) / 2: direction of the averages' FP32 conversion
  // the same parameters rounded to float, read by the FP32 stencils (GB300's FP64
  // unit also performs the double->float conversions, so none happen per use)
  float fpf[4], dpf[4], critf[2][8], critvf[2][8];
  int pme_e;             // AF_DIFF_PME: the integer exponent p0 (no conversion per use)
  // parts of the convex decomposition of each limited directional state u^{Lim,+-}
  // (Section 5.1.1, per direction in Section 5.2): 3 -- the face correction and the two
  // potential corrections -- when the equation diffuses, 1 when a(u) is constant and
  // only the face correction is present. The face limiter factor is 2d times this.
  int lim_parts;
};

// parameter k of a double/float pair in the stencil precision T
template <class T> __device__ __forceinline__ T par(const double* d, const float* f, int k);
template <> __device__ __forceinline__ double par<double>(const double* d, const float*, int k) { return d[k]; }
template <> __device__ __forceinline__ float par<float>(const double*, const float* f, int k) { return f[k]; }

inline void fill_float_params(DevModel& m) {
  m.umid = 0.5 * (m.umin + m.umax);
  for (int k = 0; k < 4; ++k) {
    m.fpf[k] = (float)m.fp[k];
    m.dpf[k] = (float)m.dp[k];
  }
  m.pme_e = m.diff_kind == AF_DIFF_PME ? (int)m.dp[0] : 0;
  for (int d = 0; d < 2; ++d)
    for (int k = 0; k < 8; ++k) {
      m.critf[d][k] = (float)m.crit[d][k];
      m.critvf[d][k] = (float)m.critv[d][k];
    }
}

// Comparisons, min and max of doubles run on the integer units through an
// order-preserving 64-bit key (key(a) < key(b) <=> a < b for non-NaN values; -0 orders
// just below +0): GB300's FP64 unit, which would otherwise execute DSETP/DMNMX, is the
// bottleneck of the FP64 stage.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ bool tlt(double a, double b) { return dkey(a) < dkey(b); }
__device__ __forceinline__ bool tlt(float a, float b) { return a < b; }
__device__ __forceinline__ bool is_one(double t) { return __double_as_longlong(t) == 0x3FF0000000000000LL; }
__device__ __forceinline__ bool is_one(float t) { return t == 1.0f; }

template <class T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <class T> __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <> __device__ __forceinline__ double tmax<double>(double a, double b) { return dkey(a) < dkey(b) ? b : a; }
template <> __device__ __forceinline__ double tmin<double>(double a, double b) { return dkey(b) < dkey(a) ? b : a; }
__device__ __forceinline__ double tabs(double a) {
  return __longlong_as_double(__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ float tabs(float a) { return fabsf(a); }

// exact float -> double with integer operations only (finite inputs). A subnormal
// float m * 2^-149 with leading bit p of m becomes the normal double
// 1.f * 2^(p - 149); the FP64 unit is never used.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned int u = (unsigned int)__float_as_int(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned int mant = u & 0x7FFFFFu;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0u) {
    if (mant == 0u) return __longlong_as_double((long long)s);
    const int p = 31 - __clz((int)mant);
    const unsigned long long fr = ((unsigned long long)mant << (52 - p)) & 0xFFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(s | ((unsigned long long)(p + 874) << 52) | fr));
  }
  const unsigned long long d = s | ((unsigned long long)(e - 127u + 1023u) << 52) | ((unsigned long long)mant << 29);
  return __longlong_as_double((long long)d);
}

// x == 0.0 (either sign) tested on the integer units
__device__ __forceinline__ bool is_zero_bits(double x) { return (__double_as_longlong(x) << 1) == 0; }

// Buckley-Leverett with gravity: f_1 = u^2 / (u^2 + (1-u)^2), f_2 = f_1 (1 - g (1-u)^2)
// and |f_1'|, |f_2'|, from one reciprocal of the denominator.
template <class T>
struct BLVals {
  T f[2], d[2];
};
// f_2 from u and f_1(u)
template <class T>
__device__ __forceinline__ T bl_f2(const DevModel& m, T u, T f1) {
  const T v = T(1) - u;
  return f1 * (T(1) - par<T>(m.fp, m.fpf, 0) * v * v);
}
template <class T>
__device__ __forceinline__ BLVals<T> bl_eval(const DevModel& m, T u) {
  const T v = T(1) - u, u2 = u * u;
  const T rD = T(1) / (u2 + v * v);
  const T g = par<T>(m.fp, m.fpf, 0);
  const T w = T(1) - g * v * v;
  const T f1 = u2 * rD;
  const T d1 = T(2) * u * v * rD * rD;   // f_1'
  BLVals<T> r;
  r.f[0] = f1;
  r.f[1] = bl_f2<T>(m, u, f1);
  r.d[0] = tabs(d1);
  r.d[1] = tabs(d1 * w + T(2) * g * v * f1);
  return r;
}

// f_l(u)
template <int FLUX, class T>
__device__ __forceinline__ T flux(const DevModel& m, int dir, T u) {
  if constexpr (FLUX == FLUX_LINEAR) {
    return par<T>(m.fp, m.fpf, dir) * u;
  } else if constexpr (FLUX == FLUX_BURGERS) {
    return par<T>(m.fp, m.fpf, 0) * u * u;
  } else if constexpr (FLUX == FLUX_BL) {
    return bl_eval<T>(m, u).f[dir];
  } else {
    return T(0);
  }
}

// |f_l'(u)|
template <int FLUX, class T>
__device__ __forceinline__ T dflux_abs(const DevModel& m, int dir, T u) {
  if constexpr (FLUX == FLUX_LINEAR) {
    return tabs(par<T>(m.fp, m.fpf, dir));
  } else if constexpr (FLUX == FLUX_BURGERS) {
    return tabs(T(2) * par<T>(m.fp, m.fpf, 0) * u);
  } else if constexpr (FLUX == FLUX_BL) {
    return bl_eval<T>(m, u).d[dir];
  } else {
    return T(0);
  }
}

// a(u)
template <class T>
__device__ __forceinline__ T apot(const DevModel& m, T u) {
  const double* d = m.dp;
  const float* f = m.dpf;
  switch (m.diff_kind) {
    case AF_DIFF_CONST:
      return par<T>(d, f, 0) * u;
    case AF_DIFF_PWL:
      // an exactly zero coefficient drops its branch (uniform integer test)
      if ((__double_as_longlong(d[0]) << 1) == 0) return par<T>(d, f, 2) * tmax(u - par<T>(d, f, 3), T(0));
      if ((__double_as_longlong(d[2]) << 1) == 0) return par<T>(d, f, 0) * tmin(u - par<T>(d, f, 1), T(0));
      return par<T>(d, f, 0) * tmin(u - par<T>(d, f, 1), T(0)) + par<T>(d, f, 2) * tmax(u - par<T>(d, f, 3), T(0));
    case AF_DIFF_PME: {
      const int e = m.pme_e;
      T r = u;
      for (int k = 1; k < e; ++k) r *= u;
      return r;
    }
    case AF_DIFF_CUBIC:
      return ((par<T>(d, f, 2) * u + par<T>(d, f, 1)) * u + par<T>(d, f, 0)) * u;
    case AF_DIFF_CUBIC01: {
      // the cubic at min(max(u, 0), 1): constant outside [0, 1]
      const T v = tmin(tmax(u, T(0)), T(1));
      return ((par<T>(d, f, 2) * v + par<T>(d, f, 1)) * v + par<T>(d, f, 0)) * v;
    }
    case AF_DIFF_RAMP: {
      // 0 below p1, p0 (u-p1)^2 / (2 p2) on the ramp, p0 (u - p1 - p2/2) above it
      const T k = par<T>(d, f, 0), lo = par<T>(d, f, 1), w = par<T>(d, f, 2), r = u - lo;
      if (!tlt(lo, u)) return T(0);
      if (tlt(u, lo + w)) return k * r * r / (T(2) * w);
      return k * (r - T(0.5) * w);
    }
    default:
      return T(0);
  }
}

// kappa(u) = a'(u), read by the diffusion form without double conservation; at a kink
// the one-sided value on the degenerate side (0 at u = p1, p3 of AF_DIFF_PWL)
template <class T>
__device__ __forceinline__ T kappa_fn(const DevModel& m, T u) {
  const double* d = m.dp;
  const float* f = m.dpf;
  switch (m.diff_kind) {
    case AF_DIFF_CONST:
      return par<T>(d, f, 0);
    case AF_DIFF_PWL:
      return (tlt(u, par<T>(d, f, 1)) ? par<T>(d, f, 0) : T(0)) + (tlt(par<T>(d, f, 3), u) ? par<T>(d, f, 2) : T(0));
    case AF_DIFF_PME: {
      const int e = m.pme_e;
      T r = T(e);
      for (int k = 1; k < e; ++k) r *= u;
      return r;
    }
    case AF_DIFF_CUBIC:
      return par<T>(d, f, 0) + (T(2) * par<T>(d, f, 1) + T(3) * par<T>(d, f, 2) * u) * u;
    case AF_DIFF_CUBIC01:
      if (!(tlt(T(0), u) && tlt(u, T(1)))) return T(0);
      return par<T>(d, f, 0) + (T(2) * par<T>(d, f, 1) + T(3) * par<T>(d, f, 2) * u) * u;
    case AF_DIFF_RAMP: {
      const T k = par<T>(d, f, 0), lo = par<T>(d, f, 1), w = par<T>(d, f, 2);
      if (!tlt(lo, u)) return T(0);
      if (tlt(u, lo + w)) return k * (u - lo) / w;
      return k;
    }
    default:
      return T(0);
  }
}

// max |f_l'| over [min(a,b), max(a,b)] given the end-point values da = |f_l'(a)| and
// db = |f_l'(b)|: the end points plus the interior extrema of f_l' that lie strictly
// inside (their |f_l'| is tabulated in the model).
template <int FLUX, class T>
__device__ __forceinline__ T alpha_interval_pre(const DevModel& m, int dir, T a, T b, T da, T db) {
  if constexpr (FLUX == FLUX_LINEAR) {
    return tabs(par<T>(m.fp, m.fpf, dir));
  } else if constexpr (FLUX == FLUX_BURGERS) {
    return tabs(T(2) * par<T>(m.fp, m.fpf, 0)) * tmax(tabs(a), tabs(b));
  } else if constexpr (FLUX == FLUX_BL) {
    const T lo = tmin(a, b), hi = tmax(a, b);
    T best = tmax(da, db);
    for (int k = 0; k < m.ncrit[dir]; ++k) {
      const T c = par<T>(m.crit[dir], m.critf[dir], k);
      if (tlt(lo, c) && tlt(c, hi)) best = tmax(best, par<T>(m.critv[dir], m.critvf[dir], k));
    }
    return best;
  } else {
    return T(0);
  }
}

// max |f_l'| over [min(a,b), max(a,b)]
template <int FLUX, class T>
__device__ __forceinline__ T alpha_interval(const DevModel& m, int dir, T a, T b) {
  if constexpr (FLUX == FLUX_BL) {
    return alpha_interval_pre<FLUX, T>(m, dir, a, b, dflux_abs<FLUX, T>(m, dir, a), dflux_abs<FLUX, T>(m, dir, b));
  } else {
    return alpha_interval_pre<FLUX, T>(m, dir, a, b, T(0), T(0));
  }
}

// Shu-Osher combination a*x + b*y with a pinned rounding sequence (b*y rounded, then
// one fused multiply-add), so every kernel that inlines it rounds identically whatever
// the compiler's contraction choices.
__device__ __forceinline__ double rk_comb(double a, double x, double b, double y) {
  return __fma_rn(a, x, __dmul_rn(b, y));
}
__device__ __forceinline__ float rk_comb(float a, float x, float b, float y) {
  return __fmaf_rn(a, x, __fmul_rn(b, y));
}
// a*x + y with one rounding (the point update z + tau R)
__device__ __forceinline__ double rk_fma(double a, double x, double y) { return __fma_rn(a, x, y); }
__device__ __forceinline__ float rk_fma(float a, float x, float y) { return __fmaf_rn(a, x, y); }
__device__ __forceinline__ double rk_scale(double b, double y) { return __dmul_rn(b, y); }
__device__ __forceinline__ float rk_scale(float b, float y) { return __fmul_rn(b, y); }

// double -> stencil precision. For float, the conversion is done with integer
// operations (truncation toward zero; underflow to signed zero): on GB300 the FP64 unit
// also executes F2F conversions, at 1/64 of the FP32 rate.
template <class T> __device__ __forceinline__ T to_stencil(double d);
template <> __device__ __forceinline__ double to_stencil<double>(double d) { return d; }
template <> __device__ __forceinline__ float to_stencil<float>(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned int hi = (unsigned int)(b >> 32);
  const unsigned int sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (e <= 0) return __int_as_float((int)sign);
  if (e >= 255) return __int_as_float((int)(sign | 0x7F800000u));
  return __int_as_float((int)(sign | ((unsigned int)e << 23) | (unsigned int)((b >> 29) & 0x7FFFFFull)));
}

// double -> stencil precision, rounded toward the nearer bound of [umin, umax]: upward
// above the midpoint mid of the bounds, downward below it (integer operations only).
// The stencils then see an average that lies between the FP64 average and the nearer
// bound, so the FP64 update built from their low-order fluxes is not shifted past that
// bound by the conversion (truncation toward zero would shift it by up to one FP32 ulp).
template <class T> __device__ __forceinline__ T to_stencil_nb(double d, double mid);
template <> __device__ __forceinline__ double to_stencil_nb<double>(double d, double) { return d; }
template <> __device__ __forceinline__ float to_stencil_nb<float>(double d, double mid) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned int hi = (unsigned int)(b >> 32);
  const unsigned int sign = hi & 0x80000000u;
  const bool up = dkey(mid) < dkey(d);
  const bool away = up != (sign != 0u);   // the magnitude grows
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (e <= 0) {   // below the normal FP32 range: 0, or the smallest normal away from zero
    if (!away || (b << 1) == 0) return __int_as_float((int)sign);
    return __int_as_float((int)(sign | 0x00800000u));
  }
  if (e >= 255) return __int_as_float((int)(sign | 0x7F800000u));
  unsigned int r = sign | ((unsigned int)e << 23) | (unsigned int)((b >> 29) & 0x7FFFFFull);
  if (away && (b & 0x1FFFFFFFull) != 0) r += 1u;   // next float away from zero
  return __int_as_float((int)r);
}

// error-free sum: s + err = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Theta(zL, zH): largest t in [0,1] with (1-t) zL + t zH inside [umin, umax].
template <class T>
__device__ __forceinline__ T theta_fn(T zL, T zH, T umin, T umax) {
  T bound;
  if (tlt(zH, umin)) bound = umin;
  else if (tlt(umax, zH)) bound = umax;
  else return T(1);
  T den = zL - zH;
  if (den == T(0)) return T(1);
  T t = (zL - bound) / den;
  return tmin(tmax(t, T(0)), T(1));
}

template <class T>
__device__ __forceinline__ bool inb(T z, T umin, T umax) {
  return !tlt(z, umin) & !tlt(umax, z);
}
// min of Theta over two / four (zL, zH) pairs. In FP64 the common case (every zH inside
// the bounds, so the minimum is 1) is tested first with integer compares; in FP32 the
// plain evaluation measured as fast.
template <class T>
__device__ __forceinline__ T theta_pair(T a0, T a1, T b0, T b1, T umin, T umax) {
  if constexpr (sizeof(T) == 8)
    if (inb(a1, umin, umax) & inb(b1, umin, umax)) return T(1);
  return tmin(theta_fn<T>(a0, a1, umin, umax), theta_fn<T>(b0, b1, umin, umax));
}
template <class T>
__device__ __forceinline__ T theta_quad(T a0, T a1, T b0, T b1, T c0, T c1, T d0, T d1, T umin, T umax) {
  if constexpr (sizeof(T) == 8)
    if (inb(a1, umin, umax) & inb(b1, umin, umax) & inb(c1, umin, umax) & inb(d1, umin, umax)) return T(1);
  return tmin(tmin(theta_fn<T>(a0, a1, umin, umax), theta_fn<T>(b0, b1, umin, umax)),
              tmin(theta_fn<T>(c0, c1, umin, umax), theta_fn<T>(d0, d1, umin, umax)));
}

// Stage statistics accumulated on the device (safeguard clamp of Section 5's
// "up to roundoff" MPP statement).
struct DevStats {
  unsigned long long clamps;
  unsigned long long errors;
  unsigned long long max_excess_bits;   // bit pattern of a non-negative double
  double ub_adjust;                     // sum of |clamped - raw| over cell averages
  unsigned long long avg_clamps;        // cell averages among the clamps
};

__device__ __forceinline__ void record_excess(DevStats* st, double e, double tol, bool* clamp_ok) {
  if (e <= tol) {
    *clamp_ok = true;
    atomicAdd(&st->clamps, 1ull);
    atomicMax(&st->max_excess_bits, (unsigned long long)__double_as_longlong(e));
  } else {
    *clamp_ok = false;
    atomicAdd(&st->errors, 1ull);
  }
}

// The rare path of the safeguard, kept out of line so that the excess (FP64 arithmetic
// and conversions) is never evaluated speculatively on the common path.
template <class S>
__device__ __noinline__ S safeguard_violation(S v, S umin, S umax, double tol, DevStats* st, bool is_avg) {
  const bool below = tlt(v, umin);
  const double e = below ? (double)umin - (double)v : (double)v - (double)umax;
  bool ok;
  record_excess(st, e, tol, &ok);
  if (ok && is_avg) {
    atomicAdd(&st->ub_adjust, e);
    atomicAdd(&st->avg_clamps, 1ull);
  }
  return ok ? (below ? umin : umax) : v;
}

// Safeguard on a stored value: exact comparison against the bounds, clamp if within
// tol. For cell averages (is_avg) the size of the change is accumulated: times dx dy it
// bounds the mass the clamps moved (later RK stages weight a stage output by <= 1).
template <class S>
__device__ __forceinline__ S safeguard(S v, S umin, S umax, double tol, DevStats* st, bool is_avg = false) {
  if (tlt(v, umin) | tlt(umax, v)) return safeguard_violation<S>(v, umin, umax, tol, st, is_avg);
  return v;
}

}  // namespace af
