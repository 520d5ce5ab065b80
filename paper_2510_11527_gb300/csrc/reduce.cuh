// Global reductions of the active flux driver: the CFL time step (eq.
// multid_av_pp_dt of arXiv 2510.11527 with the interval wave speed of Section 5.2),
// the total mass and the min/max over all DoFs. Every reduction is deterministic:
// max/min are order independent, and sums are formed per block in a fixed tree order
// and then summed by one block in block order.
#pragma once
#include "af_model.cuh"

namespace af {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;   // partial-result slots per reduction

// The CFL rate max over faces of alpha_face / h + kappa_max / h^2, with alpha_face =
// max |f_l'| over the interval spanned by the two cell averages. Its maximum over all
// faces equals the maximum over cells of |f_l'(u)| / h + kappa_max / h^2 (every cell
// average is an end point of faces in both directions, and rounding is monotone),
// together with |f_l'(c)| / h + kappa_max / h^2 for each interior extremum c of f_l'
// that lies strictly inside some face interval. The kernel reduces the first term into
// rate_bits[0] (non-negative doubles order like their bit patterns) and flags the
// extrema met (bit 8 l + k) in rate_bits[1]; dt_finalize_kernel adds their terms.
// A bounded 1D interval (bc != AF_BC_PERIODIC) has no wrap-around face; its two end
// faces join the end cells to their ghosts: the Dirichlet values gl / gr are then face
// end points too, while an outflow ghost repeats the end cell (nothing new). A 2D
// rectangle with outflow ends arrives in its padded layout (nx, ny = padded sizes): row
// and column 0 are skipped, and its last column / row has no face beyond.
template <int FLUX>
__device__ __forceinline__ unsigned crit_flags(const DevModel& m, int dir, double a, double b) {
  unsigned f = 0u;
  if constexpr (FLUX == FLUX_BL) {
    const double lo = tmin(a, b), hi = tmax(a, b);
    for (int k = 0; k < m.ncrit[dir]; ++k)
      if (tlt(lo, m.crit[dir][k]) && tlt(m.crit[dir][k], hi)) f |= 1u << k;
  }
  return f;
}

// The same rate for a flux whose |f_l'| is a nondecreasing function of |u| (Burgers) or a
// constant (linear, zero): rounding is monotone, so the largest rate is the rate at the
// largest |u|. A maximum of the magnitude bits (integer units only) per block, the rate
// formed once per block.
template <int FLUX>
__global__ void __launch_bounds__(RED_THREADS) dt_rate_maxu_kernel(const DevModel m, int dim, int nx, int ny,
                                                                    double inv_h1, double inv_h2, double kmax,
                                                                    const double* __restrict__ ub,
                                                                    unsigned long long* rate_bits, int bc, double gl,
                                                                    double gr) {
  const size_t n = (size_t)nx * ny;
  const double kd1 = kmax * inv_h1 * inv_h1, kd2 = kmax * inv_h2 * inv_h2;
  const bool rect = dim == 2 && bc != AF_BC_PERIODIC;
  unsigned long long mb = 0ull;
  if constexpr (FLUX == FLUX_BURGERS) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
      if (rect) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        if (i == 0 || j == 0) continue;
      }
      const unsigned long long b = (unsigned long long)__double_as_longlong(ub[k]) & 0x7FFFFFFFFFFFFFFFull;
      mb = b > mb ? b : mb;
    }
    if (dim == 1 && bc == AF_BC_DIRICHLET && blockIdx.x == 0 && threadIdx.x == 0) {
      const unsigned long long bl = (unsigned long long)__double_as_longlong(gl) & 0x7FFFFFFFFFFFFFFFull;
      const unsigned long long br = (unsigned long long)__double_as_longlong(gr) & 0x7FFFFFFFFFFFFFFFull;
      mb = bl > mb ? bl : mb;
      mb = br > mb ? br : mb;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = v > mb ? v : mb;
  }
  __shared__ unsigned long long smb[RED_THREADS / 32];
  if ((threadIdx.x & 31) == 0) smb[threadIdx.x >> 5] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < RED_THREADS / 32; ++w) mb = smb[w] > mb ? smb[w] : mb;
    const double u = __longlong_as_double((long long)mb);
    const double a1 = alpha_interval<FLUX, double>(m, 0, u, u), a2 = alpha_interval<FLUX, double>(m, 1, u, u);
    double b = a1 * inv_h1 + kd1;
    if (dim == 2) b = tmax(b, a2 * inv_h2 + kd2);
    atomicMax(rate_bits, (unsigned long long)__double_as_longlong(b));
  }
}

template <int FLUX>
__global__ void __launch_bounds__(RED_THREADS) dt_rate_kernel(const DevModel m, int dim, int nx, int ny,
                                                               double inv_h1, double inv_h2, double kmax,
                                                               const double* __restrict__ ub,
                                                               unsigned long long* rate_bits, int bc, double gl,
                                                               double gr) {
  const size_t n = (size_t)nx * ny;
  double best = 0.0;
  unsigned flags = 0u;
  const double kd1 = kmax * inv_h1 * inv_h1, kd2 = kmax * inv_h2 * inv_h2;
  const bool rect = dim == 2 && bc != AF_BC_PERIODIC;
  // The cell's rate max_l |f_l'(u)| / h_l + kappa_max / h_l^2 (1D: the gravity form,
  // whose extrema tables sit in slot 0), in FP64 and as an FP32 estimate (within a few
  // ulps). The FP64 one costs a division on GB300's slow FP64 unit, so it is formed only
  // for the cells whose estimate is within 2^-12 of the block's largest estimate: the
  // cell with the largest FP64 rate is always among them, so the maximum is the same.
  auto rate64 = [&](double u) {
    const BLVals<double> r = bl_eval<double>(m, u);
    double b = r.d[dim == 1 ? 1 : 0] * inv_h1 + kd1;
    if (dim == 2) b = tmax(b, r.d[1] * inv_h2 + kd2);
    return b;
  };
  const float ih1f = (float)inv_h1, ih2f = (float)inv_h2, kd1f = (float)kd1, kd2f = (float)kd2;
  auto rate32 = [&](double u) {
    const BLVals<float> r = bl_eval<float>(m, to_stencil<float>(u));
    float b = r.d[dim == 1 ? 1 : 0] * ih1f + kd1f;
    if (dim == 2) b = fmaxf(b, r.d[1] * ih2f + kd2f);
    return b;
  };
  float m32 = 0.0f;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(k % nx), j = (int)(k / nx);
    if (rect && (i == 0 || j == 0)) continue;
    const double u = ub[k];
    if constexpr (FLUX == FLUX_BL) {
      m32 = fmaxf(m32, rate32(u));
      double un = ub[(size_t)j * nx + (i + 1 == nx ? 0 : i + 1)];
      if (dim == 1 && bc != AF_BC_PERIODIC && i + 1 == nx) un = bc == AF_BC_DIRICHLET ? gr : u;
      if (rect && i + 1 == nx) un = u;
      flags |= crit_flags<FLUX>(m, 0, u, un);
      if (dim == 1 && bc == AF_BC_DIRICHLET && k == 0) flags |= crit_flags<FLUX>(m, 0, gl, u);
      if (dim == 2) {
        const double ut = (rect && j + 1 == ny) ? u : ub[(size_t)(j + 1 == ny ? 0 : j + 1) * nx + i];
        flags |= crit_flags<FLUX>(m, 1, u, ut) << 8;
      }
    } else {
      best = tmax(best, alpha_interval<FLUX, double>(m, 0, u, u) * inv_h1 + kd1);
      if (dim == 2) best = tmax(best, alpha_interval<FLUX, double>(m, 1, u, u) * inv_h2 + kd2);
    }
  }
  if constexpr (FLUX == FLUX_BL) {
    __shared__ float s32[RED_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) m32 = fmaxf(m32, __shfl_xor_sync(0xffffffffu, m32, o));
    if ((threadIdx.x & 31) == 0) s32[threadIdx.x >> 5] = m32;
    __syncthreads();
    for (int w = 0; w < RED_THREADS / 32; ++w) m32 = fmaxf(m32, s32[w]);
    const float thr = m32 - m32 * (1.0f / 4096.0f);
    unsigned long long last = ~0ull;   // bits of the last u evaluated in FP64 (NaN: none)
    double lastr = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
      if (rect) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        if (i == 0 || j == 0) continue;
      }
      const double u = ub[k];
      if (rate32(u) < thr) continue;
      const unsigned long long bits = (unsigned long long)__double_as_longlong(u);
      if (bits != last) {
        lastr = rate64(u);
        last = bits;
      }
      best = tmax(best, lastr);
    }
  }
  if (dim == 1 && bc == AF_BC_DIRICHLET && blockIdx.x == 0 && threadIdx.x == 0) {
    const double gv[2] = {gl, gr};
    for (int s = 0; s < 2; ++s) {
      double d;
      if constexpr (FLUX == FLUX_BL) d = bl_eval<double>(m, gv[s]).d[1];
      else d = alpha_interval<FLUX, double>(m, 0, gv[s], gv[s]);
      best = tmax(best, d * inv_h1 + kd1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) best = tmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  flags = __reduce_or_sync(0xffffffffu, flags);
  __shared__ double sm[RED_THREADS / 32];
  __shared__ unsigned sf[RED_THREADS / 32];
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5] = best;
    sf[threadIdx.x >> 5] = flags;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = sm[0];
    unsigned f = sf[0];
    for (int w = 1; w < RED_THREADS / 32; ++w) {
      b = tmax(b, sm[w]);
      f |= sf[w];
    }
    atomicMax(rate_bits, (unsigned long long)__double_as_longlong(b));
    if (f) atomicOr(rate_bits + 1, (unsigned long long)f);
  }
}

// rate over the flagged extrema (see dt_rate_kernel)
__device__ __forceinline__ double crit_rate(const DevModel& m, int dim, double inv_h1, double inv_h2, double kmax,
                                            unsigned long long flags, double rate) {
  const double kd1 = kmax * inv_h1 * inv_h1, kd2 = kmax * inv_h2 * inv_h2;
  for (int d = 0; d < dim; ++d)
    for (int k = 0; k < m.ncrit[d]; ++k)
      if ((flags >> (8 * d + k)) & 1ull)
        rate = tmax(rate, d == 0 ? m.critv[0][k] * inv_h1 + kd1 : m.critv[1][k] * inv_h2 + kd2);
  return rate;
}

// dt = 1 / max(rate / C, kappa_max / (h_min^2 Cd)). Resets the accumulators for the
// next step. When t_acc is given the step is also added to the simulated time; with
// t_end > 0 the step is first clipped to the time left before t_end (0 once less than
// t_end * 1e-14 is left) and each positive step is counted in *count.
static __global__ void dt_finalize_kernel(unsigned long long* rate_bits, const DevModel m, int dim, double inv_h1,
                                          double inv_h2, double cfl, double cfl_diff, double kmax, double inv_hmin2,
                                          double* dt_out, double* t_acc, double t_end, double* count) {
  const double rate =
      crit_rate(m, dim, inv_h1, inv_h2, kmax, rate_bits[1], __longlong_as_double((long long)rate_bits[0]));
  double r = rate / cfl;
  if (cfl_diff > 0.0 && kmax > 0.0) r = fmax(r, kmax * inv_hmin2 / cfl_diff);
  double dt = r > 0.0 ? 1.0 / r : 0.0;
  if (t_acc && t_end > 0.0) {
    const double left = t_end - *t_acc;
    dt = left > t_end * 1e-14 ? fmin(dt, left) : 0.0;
    if (dt > 0.0) *count += 1.0;
  }
  *dt_out = dt;
  if (t_acc) *t_acc += dt;
  rate_bits[0] = 0ull;
  rate_bits[1] = 0ull;
}

// *dt = v and, when t_acc is given, *t_acc += v
static __global__ void set_dt_kernel(double* dt, double* t_acc, double v) {
  *dt = v;
  if (t_acc) *t_acc += v;
}

// ---- deterministic sum / min / max ------------------------------------------------------
// op 0: sum of x; op 1: min; op 2: max. Each block reduces a contiguous chunk.
__device__ __forceinline__ double red_op(int op, double a, double b) {
  return op == 0 ? a + b : (op == 1 ? fmin(a, b) : fmax(a, b));
}

template <class S>
__global__ void __launch_bounds__(RED_THREADS) partial_kernel(const S* __restrict__ x, size_t n, int op,
                                                              double init, double* partial) {
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t beg = blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
  double acc = init;
  for (size_t k = beg + threadIdx.x; k < end; k += RED_THREADS) acc = red_op(op, acc, (double)x[k]);
  __shared__ double sm[RED_THREADS];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = red_op(op, sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

// the same over the entries of a row-major array with rows of width w whose column is
// >= ilo and row >= jlo (the DoFs of a padded 2D rectangle)
template <class S>
__global__ void __launch_bounds__(RED_THREADS) partial_masked_kernel(const S* __restrict__ x, size_t n, int w,
                                                                     int ilo, int jlo, int op, double init,
                                                                     double* partial) {
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t beg = blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
  double acc = init;
  for (size_t k = beg + threadIdx.x; k < end; k += RED_THREADS)
    if ((int)(k % w) >= ilo && (int)(k / w) >= jlo) acc = red_op(op, acc, (double)x[k]);
  __shared__ double sm[RED_THREADS];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = red_op(op, sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

// combine nparts partials into *out (op as above; combined with the existing *out when
// accumulate != 0). One block of RED_THREADS: thread t folds partials t, t + RED_THREADS,
// ... in order, then a fixed tree; the result depends only on nparts and the partials.
static __global__ void __launch_bounds__(RED_THREADS) finalize_kernel(const double* partial, int nparts, int op,
                                                                      double* out, int accumulate) {
  __shared__ double sm[RED_THREADS];
  const int t = threadIdx.x;
  // partial[0] is neutral for min/max over a set that contains it
  double acc = op == 0 ? 0.0 : partial[0];
  for (int k = t; k < nparts; k += RED_THREADS) acc = red_op(op, acc, partial[k]);
  sm[t] = acc;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (t < s) sm[t] = red_op(op, sm[t], sm[t + s]);
    __syncthreads();
  }
  if (t == 0) *out = accumulate ? red_op(op, *out, sm[0]) : sm[0];
}

}  // namespace af
