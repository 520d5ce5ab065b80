// 3D stage of the compact fourth-order doubly conservative active flux method with the
// monolithic convex limiter (arXiv 2510.11527, Section 4's 3D DoFs; Section 5.2 with
// d = 3: directional split 1/6, limiter factor 18, face factor 6 without a diffusion
// term). Four kernels per stage, one thread per cell, FP64:
//   K1 centre values from the tensor Simpson rule of the cell average;
//   K2 per direction: high-order face flux (Simpson face average of f_l), DC cell
//      potential (transverse Simpson average of the 1D potential along l), LLF face
//      flux with the interval wave speed, smoothness value s_l;
//   K3 per output: blend, low-order states u^{L,+-}_l, limiting parameters
//      theta^c (faces) and theta^d (cells), limited face fluxes and cell potentials;
//   K4 per output: limited cell-average update and the 7 point values of the cell
//      (5-point lines along each axis, blend with the low-order point residual,
//      projection), RK combination and post-stage safeguard.
// T is the stencil precision: FP64, or FP32 in the FP32-mixed form, whose point values
// and stencils are FP32 while the cell averages, their update and their RK combination
// stay FP64 (conversions run on the integer pipe).
// All locations are addressed on the fine grid of half-cell spacing: the DoF at
// (i + sx/2, j + sy/2, k + sz/2) has fine index (2i + sx, 2j + sy, 2k + sz), so a
// 5-point line is the fine points p - 2e .. p + 2e and a Simpson average weighs 1, 4, 1
// per axis. Inputs are read from global memory (reuse through L1 / L2).
#include "launch.h"
#include "stage3d.cuh"

namespace af {
namespace {

constexpr int T3 = 256;

template <class T>
__device__ __forceinline__ size_t cells3(const StageArgs3D<T>& A) { return (size_t)A.n[0] * A.n[1] * A.n[2]; }

// cell coordinates of a linear index (32-bit: meshes hold < 2^31 cells)
template <class T>
__device__ __forceinline__ void decode3(const StageArgs3D<T>& A, size_t q, int* c) {
  const unsigned qq = (unsigned)q, n0 = (unsigned)A.n[0], n1 = (unsigned)A.n[1];
  const unsigned r = qq / n0;
  c[0] = (int)(qq - r * n0);
  c[1] = (int)(r % n1);
  c[2] = (int)(r / n1);
}

// periodic cell index
template <class T>
__device__ __forceinline__ size_t cell3(const StageArgs3D<T>& A, const int* c) {
  return ((size_t)wrapi(c[2], A.n[2]) * A.n[1] + wrapi(c[1], A.n[1])) * A.n[0] + wrapi(c[0], A.n[0]);
}

// neighbour step cells along l of the cell at coordinates c (|step| <= 2, no division)
template <class T>
__device__ __forceinline__ size_t nbr3(const StageArgs3D<T>& A, const int* c, int l, int step) {
  int d[3] = {c[0], c[1], c[2]};
  d[l] += step;
  if (d[l] < 0) d[l] += A.n[l];
  if (d[l] >= A.n[l]) d[l] -= A.n[l];
  if (d[l] < 0 || d[l] >= A.n[l]) d[l] = wrapi(d[l], A.n[l]);   // meshes thinner than the step
  return ((size_t)d[2] * A.n[1] + d[1]) * A.n[0] + d[0];
}

// Simpson weights 1, 4, 1 per axis as exact tables (no FP64 multiplies per term): the
// full 3D weight of offset o = mx + 1 + 3 (my + 1) + 9 (mz + 1), and the transverse 2D
// weight for each axis l (the factor along l is 1)
__constant__ double kW27[27] = {1, 4, 1, 4, 16, 4, 1, 4, 1, 4, 16, 4, 16, 64, 16, 4, 16, 4, 1, 4, 1, 4, 16, 4, 1, 4, 1};
__constant__ float kW27f[27] = {1, 4, 1, 4, 16, 4, 1, 4, 1, 4, 16, 4, 16, 64, 16, 4, 16, 4, 1, 4, 1, 4, 16, 4, 1, 4, 1};
template <class T> __device__ __forceinline__ T w27(int o);
template <> __device__ __forceinline__ double w27<double>(int o) { return kW27[o]; }
template <> __device__ __forceinline__ float w27<float>(int o) { return kW27f[o]; }
template <class T>
__device__ __forceinline__ T wtrans(int o, int l) {
  // drop the factor of axis l from the 3D weight: divide by its 1D weight (4 or 1)
  const int ml = l == 0 ? o % 3 : (l == 1 ? (o / 3) % 3 : o / 9);
  return ml == 1 ? w27<T>(o) * T(0.25) : w27<T>(o);
}

// The wrapped fine coordinates of offsets -2 .. +3 from the cell's fine origin 2c along
// each axis, formed once per cell: a fine access is then two shifts and a lookup.
// exact widening of a stencil value to FP64 (FP32 on the integer pipe)
__device__ __forceinline__ double wide(double v) { return v; }
__device__ __forceinline__ double wide(float v) { return f2d_exact(v); }

struct FineAxes {
  int f[3][6];
};
template <class T>
__device__ __forceinline__ FineAxes fine_axes(const StageArgs3D<T>& A, const int* c) {
  FineAxes fa;
  for (int l = 0; l < 3; ++l)
    for (int o = 0; o < 6; ++o) fa.f[l][o] = wrapi(2 * c[l] + o - 2, 2 * A.n[l]);
  return fa;
}
// fine value at offsets (ox, oy, oz) in [-2, 3] from 2c: kind 0 is the recovered centre,
// or the cell average when avg is set (the low-order neighbours of the blend)
template <class T>
__device__ __forceinline__ T zoff(const StageArgs3D<T>& A, const FineAxes& fa, int ox, int oy, int oz, bool avg = false) {
  const int fx = fa.f[0][ox + 2], fy = fa.f[1][oy + 2], fz = fa.f[2][oz + 2];
  const int kind = (fx & 1) | ((fy & 1) << 1) | ((fz & 1) << 2);
  const size_t q = ((size_t)(fz >> 1) * A.n[1] + (fy >> 1)) * A.n[0] + (fx >> 1);
  if (kind == 0) return avg ? to_stencil<T>(A.ub[q]) : A.C[q];
  return A.pt[kind][q];
}

template <class T>
__global__ void __launch_bounds__(T3) centre3d_kernel(const StageArgs3D<T> A) {
  if (*A.dt == 0.0) return;
  const size_t N = cells3(A);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    int c[3];
    decode3(A, q, c);
    // the fine point at offset m in {-1, 0, 1}^3 from the centre is of kind
    // s = [m_x != 0] + 2 [m_y != 0] + 4 [m_z != 0], stored with the cell c - [m = -1]:
    // the 8 cells of the block c - {0, 1}^3 hold all 26 (same order and weights as
    // the fine-grid walk)
    size_t cq[8];
    {
      int lo[3];
      for (int l = 0; l < 3; ++l) lo[l] = c[l] == 0 ? A.n[l] - 1 : c[l] - 1;
      for (int a = 0; a < 8; ++a) {
        const int x = (a & 1) ? lo[0] : c[0], y = (a & 2) ? lo[1] : c[1], z = (a & 4) ? lo[2] : c[2];
        cq[a] = ((size_t)z * A.n[1] + y) * A.n[0] + x;
      }
    }
    T acc = T(0);
#pragma unroll
    for (int o = 0; o < 27; ++o) {
      const int mx = o % 3 - 1, my = (o / 3) % 3 - 1, mz = o / 9 - 1;
      if (mx == 0 && my == 0 && mz == 0) continue;
      const int kind = (mx != 0) | ((my != 0) << 1) | ((mz != 0) << 2);
      const int a = (mx < 0) | ((my < 0) << 1) | ((mz < 0) << 2);
      acc = acc + w27<T>(o) * A.pt[kind][cq[a]];
    }
    A.C[q] = (T(216) * to_stencil<T>(A.ub[q]) - acc) * T(1.0 / 64.0);
  }
}

// low-order directional states of a cell along l (Lemma 5.1 with factor 2d = 6), from
// its average u, f_l(u), a(u), the LLF flux of its face after (FLp) or before (FLm) and
// a at its neighbour after (an) or before (am): each f and a is formed once per cell
template <class T>
__device__ __forceinline__ T ulp3(T u, T fu, T au, T FLp, T an, T mu6, T nu6) {
  return u - mu6 * (FLp - fu) + nu6 * (an - au);
}
template <class T>
__device__ __forceinline__ T ulm3(T u, T fu, T au, T FLm, T am, T mu6, T nu6) {
  return u - mu6 * (fu - FLm) - nu6 * (au - am);
}

template <int FLUX, class T>
__global__ void __launch_bounds__(T3) limit3d_kernel(const DevModel m, const StageArgs3D<T> A, int o) {
  const double dtv = *A.dt;
  if (dtv == 0.0) return;   // uniform over the grid
  // per-direction factors of this launch, formed once per block in FP64 and rounded to
  // the stencil type (a double -> float rounding is an FP64-unit instruction on GB300)
  __shared__ T sK[3][4];   // 6 mu, 6 nu, face factor (18 or 6) mu, 18 nu
  if (threadIdx.x < 3) {
    const int l = threadIdx.x;
    const double mu = A.tcoef[o] * dtv * A.inv_h[l], nu = mu * A.inv_h[l];
    sK[l][0] = T(6.0 * mu);
    sK[l][1] = T(6.0 * nu);
    sK[l][2] = T(double(6 * m.lim_parts) * mu);   // 18 mu, or 6 mu without diffusion
    sK[l][3] = T(18.0 * nu);
  }
  __syncthreads();
  const size_t N = cells3(A);
  const T g = T(A.gamma), umin = T(m.umin), umax = T(m.umax);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    int c[3];
    decode3(A, q, c);
    const T u = to_stencil<T>(A.ub[q]), au = apot<T>(m, u);
    for (int l = 0; l < 3; ++l) {
      const size_t qp = nbr3(A, c, l, 1), qm = nbr3(A, c, l, -1);
      T fh = A.FH[l][q], ah = A.AH[l][q];
      const T fl = A.FL[l][q];
      if (A.blend) {
        const T tc = exp(-g * (T(0.5) * (A.S[l][q] + A.S[l][qp])));
        const T td = exp(-g * A.S[l][q]);
        fh = tc * fh + (T(1) - tc) * fl;
        ah = td * ah + (T(1) - td) * au;
      }
      T flim = fh, alim = ah;
      if (A.limiter) {
        const T mu6 = sK[l][0], nu6 = sK[l][1];
        const T k = sK[l][2], kd = sK[l][3];
        const T dF = fh - fl;
        // the cell (u), its neighbours after (up) and before (um) along l
        const T up = to_stencil<T>(A.ub[qp]), um = to_stencil<T>(A.ub[qm]);
        const T fu = flux<FLUX, T>(m, l, u), fup = flux<FLUX, T>(m, l, up), fum = flux<FLUX, T>(m, l, um);
        const T aup = apot<T>(m, up), aum = apot<T>(m, um);
        const T flm = A.FL[l][qm];
        const T zp = ulp3<T>(u, fu, au, fl, aup, mu6, nu6), zm = ulm3<T>(up, fup, aup, fl, au, mu6, nu6);
        const T tcl = tmin(theta_fn<T>(zp, zp - k * dF, umin, umax), theta_fn<T>(zm, zm + k * dF, umin, umax));
        flim = is_one(tcl) ? fh : fl + tcl * dF;
        const T dA = ah - au;
        const T p0 = ulp3<T>(um, fum, aum, flm, au, mu6, nu6), q0 = ulm3<T>(u, fu, au, flm, aum, mu6, nu6);
        const T td = tmin(tmin(theta_fn<T>(p0, p0 + kd * dA, umin, umax), theta_fn<T>(zp, zp - kd * dA, umin, umax)),
                          tmin(theta_fn<T>(q0, q0 - kd * dA, umin, umax), theta_fn<T>(zm, zm + kd * dA, umin, umax)));
        alim = is_one(td) ? ah : au + td * dA;
      }
      A.Flim[l][q] = flim;
      A.Alim[l][q] = alim;
    }
  }
}

template <int FLUX, class T>
__global__ void __launch_bounds__(T3) update3d_kernel(const DevModel m, const StageArgs3D<T> A, int o) {
  const double dtv = *A.dt;
  if (dtv == 0.0) return;   // uniform over the grid
  const double tau = A.tcoef[o] * dtv;
  const double cA = A.cA[o], cF = A.cF[o];
  // mu_l = tau / h_l and nu_l = tau / h_l^2 of this launch, once per block
  __shared__ double sMu[3], sNu[3];
  if (threadIdx.x < 3) {
    const int l = threadIdx.x;
    sMu[l] = tau * A.inv_h[l];
    sNu[l] = sMu[l] * A.inv_h[l];
  }
  __syncthreads();
  const size_t N = cells3(A);
  const T taut = T(tau), cAt = T(cA), cFt = T(cF), umin = T(m.umin), umax = T(m.umax), g = T(A.gamma);
  // an integer test: GB300 runs FP64 compares on its slow FP64 unit
  const bool comb = !is_zero_bits(cA);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    int c[3];
    decode3(A, q, c);
    const FineAxes fa = fine_axes(A, c);
    // limited cell-average update (eq. multid_limited_average), in FP64
    double v = A.ub[q];
    for (int l = 0; l < 3; ++l) {
      const double mu = sMu[l], nu = sNu[l];
      const size_t qm = nbr3(A, c, l, -1), qp = nbr3(A, c, l, 1);
      const double f0 = wide(A.Flim[l][q]), fm = wide(A.Flim[l][qm]);
      const double a0 = wide(A.Alim[l][q]), am = wide(A.Alim[l][qm]), ap = wide(A.Alim[l][qp]);
      v = v - mu * (f0 - fm) + nu * (ap - 2.0 * a0 + am);
    }
    double ubo = comb ? rk_comb(cA, A.Aub[o][q], cF, v) : rk_scale(cF, v);
    if (A.limiter && A.sg[o]) ubo = safeguard<double>(ubo, m.umin, m.umax, A.tol, A.stats, true);
    A.Oub[o][q] = ubo;
    // point values owned by the cell: kinds 1..7 at fine 2c + s
    for (int s = 1; s < 8; ++s) {
      const int p[3] = {s & 1, (s >> 1) & 1, (s >> 2) & 1};   // offsets from 2c
      T acc = T(0);
      for (int l = 0; l < 3; ++l) {
        const T ih = A.inv_hT[l];
        T z[5], fz[5], dz[5], az[5];
        for (int t = 0; t < 5; ++t) {
          int f[3] = {p[0], p[1], p[2]};
          f[l] += t - 2;
          z[t] = zoff(A, fa, f[0], f[1], f[2]);
          fz[t] = flux<FLUX, T>(m, l, z[t]);
          dz[t] = dflux_abs<FLUX, T>(m, l, z[t]);
          az[t] = apot<T>(m, z[t]);
        }
        T rh;
        if constexpr (FLUX == FLUX_ZERO) {
          // the diffusion part of line_res alone (its convection part is an exact zero)
          rh = (T(16) * (az[1] + az[3]) - (az[0] + az[4]) - T(30) * az[2]) * A.i3h2T[l];
        } else {
          const T alpha = tmax(tmax(tmax(dz[0], dz[1]), tmax(dz[3], dz[4])), dz[2]);
          rh = line_res<T>(z[0], z[1], z[2], z[3], z[4], fz[0], fz[1], fz[3], fz[4], alpha, az[0], az[1], az[2], az[3],
                           az[4], A.i6hT[l], A.i3h2T[l]);
        }
        T r = rh;
        if (A.blend) {
          // weight: min of theta^{c,s}_l over the l-faces holding the point (s_l = 1),
          // else of theta^{d,s}_l over the cells holding it
          const bool onface = (s >> l) & 1;
          T w = T(2);
          for (int bits = 0; bits < 8; ++bits) {
            int cc[3] = {c[0], c[1], c[2]};
            bool ok = true;
            for (int t = 0; t < 3; ++t) {
              if (!((bits >> t) & 1)) continue;
              if (t == l || !((s >> t) & 1)) { ok = false; break; }
              cc[t] = cc[t] + 1 == A.n[t] ? 0 : cc[t] + 1;   // periodic, so nbr3 below sees wrapped coordinates
            }
            if (!ok) continue;
            const size_t qq = cell3(A, cc);
            const T sv = A.S[l][qq];
            const T wv = onface ? exp(-g * (T(0.5) * (sv + A.S[l][nbr3(A, cc, l, 1)]))) : exp(-g * sv);
            w = (w == T(2)) ? wv : tmin(w, wv);
          }
          // low-order residual on the +-h/2 neighbours (a centre replaced by its average)
          int fm[3] = {p[0], p[1], p[2]}, fp[3] = {p[0], p[1], p[2]};
          fm[l] -= 1;
          fp[l] += 1;
          const T zm = zoff(A, fa, fm[0], fm[1], fm[2], true), z0 = z[2],
                  zp = zoff(A, fa, fp[0], fp[1], fp[2], true);
          const T Fr = T(0.5) * (flux<FLUX, T>(m, l, z0) + flux<FLUX, T>(m, l, zp)) -
                       T(0.5) * alpha_interval<FLUX, T>(m, l, z0, zp) * (zp - z0);
          const T Fl = T(0.5) * (flux<FLUX, T>(m, l, zm) + flux<FLUX, T>(m, l, z0)) -
                       T(0.5) * alpha_interval<FLUX, T>(m, l, zm, z0) * (z0 - zm);
          const T RL = (apot<T>(m, zp) - T(2) * apot<T>(m, z0) + apot<T>(m, zm)) * (T(4) * ih * ih) - (Fr - Fl) * (T(2) * ih);
          r = w * rh + (T(1) - w) * RL;
        }
        acc = (l == 0) ? r : acc + r;
      }
      T pv = A.pt[s][q] + taut * acc;
      if (A.limiter) pv = tmin(tmax(pv, umin), umax);
      T po = comb ? rk_comb(cAt, A.Apt[o][s][q], cFt, pv) : rk_scale(cFt, pv);
      if (A.limiter && A.sg[o]) po = safeguard<T>(po, umin, umax, A.tol, A.stats);
      A.Opt[o][s][q] = po;
    }
  }
}

// K4 with the point values staged: one CTA per tile of U3X x U3Y x U3Z cells loads the
// centres and the 7 point kinds of the tile and a one-cell halo into shared memory
// once, with a(z) evaluated once per location; every 5-point line of the tile's points
// then reads there (a line of a point owned by cell c spans the cells c - 1 .. c + 1
// along its axis). Values, order of operations and results are those of the gathered
// form; the blend's extra neighbours (averages, smoothness values) are still read
// from global memory.
constexpr int U3X = 8, U3Y = 4, U3Z = 4, U3T = U3X * U3Y * U3Z;
constexpr int B3X = U3X + 2, B3Y = U3Y + 2, B3Z = U3Z + 2, B3N = B3X * B3Y * B3Z;

// the launch's scalars of K4, formed once per CTA by the lanes of warp 0 at once (GB300's
// FP64 unit spends as long on a warp instruction with one active lane as with 32)
template <class T>
struct K4Scal {
  double mu[3], nu[3];                 // tau / h_l, tau / h_l^2
  T taut, cAt, cFt, umin, umax, g;
};

// warp 0 only: lane l < 3 forms mu_l = fl(tau / h_l), nu_l = fl(mu_l / h_l) (tau =
// fl(tcoef dt)); lanes 3 .. 8 round tau, cA, cF, u_min, u_max, gamma to T
template <class T>
__device__ __forceinline__ void k4_scalars(const DevModel& m, const StageArgs3D<T>& A, int o, double dtv,
                                           K4Scal<T>& sc) {
  const int l = threadIdx.x & 31;
  const double tau = A.tcoef[o] * dtv;
  const double ih = A.inv_h[l < 3 ? l : 0];
  const double x = l == 4 ? A.cA[o] : (l == 5 ? A.cF[o] : (l == 6 ? m.umin : (l == 7 ? m.umax : (l == 8 ? A.gamma : tau))));
  const double mu = x * (l < 3 ? ih : 1.0);
  const double nu = mu * ih;
  const T v = T(mu);
  switch (l) {
    case 0: case 1: case 2: sc.mu[l] = mu; sc.nu[l] = nu; break;
    case 3: sc.taut = v; break;
    case 4: sc.cAt = v; break;
    case 5: sc.cFt = v; break;
    case 6: sc.umin = v; break;
    case 7: sc.umax = v; break;
    case 8: sc.g = v; break;
    default: break;
  }
}

// centres (kind 0) and point kinds 1 .. 7 of the tile at c0 and its one-cell halo, with
// a(z), by `nthreads` threads
template <class T>
__device__ __forceinline__ void k4_load(const DevModel& m, const StageArgs3D<T>& A, int c0x, int c0y, int c0z,
                                        int nthreads, T (*sZ)[B3N], T (*sAz)[B3N]) {
  const int n0 = A.n[0], n1 = A.n[1], n2 = A.n[2];
  for (int k = threadIdx.x; k < 8 * B3N; k += nthreads) {
    const int sk = k / B3N, b = k - sk * B3N;
    const int bx = b % B3X, by = (b / B3X) % B3Y, bz = b / (B3X * B3Y);
    const size_t q = ((size_t)wrapi(c0z - 1 + bz, n2) * n1 + wrapi(c0y - 1 + by, n1)) * n0 + wrapi(c0x - 1 + bx, n0);
    const T z = sk == 0 ? A.C[q] : A.pt[sk][q];
    sZ[sk][b] = z;
    sAz[sk][b] = apot<T>(m, z);
  }
}

// limited cell-average update (eq. multid_limited_average) of cell c, in FP64, with the
// RK combination and the post-stage safeguard
template <class T>
__device__ __forceinline__ void k4_average(const DevModel& m, const StageArgs3D<T>& A, int o, const int* c, size_t q,
                                           const K4Scal<T>& sc, bool comb) {
  double v = A.ub[q];
  for (int l = 0; l < 3; ++l) {
    const double mu = sc.mu[l], nu = sc.nu[l];
    const size_t qm = nbr3(A, c, l, -1), qp = nbr3(A, c, l, 1);
    const double f0 = wide(A.Flim[l][q]), fm = wide(A.Flim[l][qm]);
    const double a0 = wide(A.Alim[l][q]), am = wide(A.Alim[l][qm]), ap = wide(A.Alim[l][qp]);
    v = v - mu * (f0 - fm) + nu * (ap - 2.0 * a0 + am);
  }
  double ubo = comb ? rk_comb(A.cA[o], A.Aub[o][q], A.cF[o], v) : rk_scale(A.cF[o], v);
  if (A.limiter && A.sg[o]) ubo = safeguard<double>(ubo, m.umin, m.umax, A.tol, A.stats, true);
  A.Oub[o][q] = ubo;
}

// the point value of kind s owned by cell c (tile-local lx, ly, lz), from the staged
// lines; RK combination and safeguard (indices are scalars, so that nothing indexed by
// the loop variables lands in local memory)
template <int FLUX, class T>
__device__ __forceinline__ void k4_point(const DevModel& m, const StageArgs3D<T>& A, int o, const int* c, size_t q,
                                         int lx, int ly, int lz, int s, const T (*sZ)[B3N], const T (*sAz)[B3N],
                                         const K4Scal<T>& sc, bool comb) {
  const int px = s & 1, py = (s >> 1) & 1, pz = (s >> 2) & 1;   // offsets from 2c
  T acc = T(0);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const T ih = A.inv_hT[l];
    const int pl = l == 0 ? px : (l == 1 ? py : pz);
    T z[5], fz[5], dz[5], az[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      // fine offset F = p_l + t - 2 along l: cell offset floor(F / 2), kind bit F & 1
      const int F = pl + t - 2, dc = F >> 1, kbit = F & 1;
      const int b = (lx + 1 + (l == 0 ? dc : 0)) + B3X * ((ly + 1 + (l == 1 ? dc : 0)) + B3Y * (lz + 1 + (l == 2 ? dc : 0)));
      const int kind = (l == 0 ? kbit : px) | ((l == 1 ? kbit : py) << 1) | ((l == 2 ? kbit : pz) << 2);
      z[t] = sZ[kind][b];
      fz[t] = flux<FLUX, T>(m, l, z[t]);
      dz[t] = dflux_abs<FLUX, T>(m, l, z[t]);
      az[t] = sAz[kind][b];
    }
    T rh;
    if constexpr (FLUX == FLUX_ZERO) {
      // the diffusion part of line_res alone (its convection part is an exact zero)
      rh = (T(16) * (az[1] + az[3]) - (az[0] + az[4]) - T(30) * az[2]) * A.i3h2T[l];
    } else {
      const T alpha = tmax(tmax(tmax(dz[0], dz[1]), tmax(dz[3], dz[4])), dz[2]);
      rh = line_res<T>(z[0], z[1], z[2], z[3], z[4], fz[0], fz[1], fz[3], fz[4], alpha, az[0], az[1], az[2], az[3],
                       az[4], A.i6hT[l], A.i3h2T[l]);
    }
    T r = rh;
    if (A.blend) {
      const FineAxes fa = fine_axes(A, c);
      // weight: min of theta^{c,s}_l over the l-faces holding the point (s_l = 1),
      // else of theta^{d,s}_l over the cells holding it
      const bool onface = (s >> l) & 1;
      T w = T(2);
      for (int bits = 0; bits < 8; ++bits) {
        int cc[3] = {c[0], c[1], c[2]};
        bool ok = true;
        for (int t = 0; t < 3; ++t) {
          if (!((bits >> t) & 1)) continue;
          if (t == l || !((s >> t) & 1)) { ok = false; break; }
          cc[t] = cc[t] + 1 == A.n[t] ? 0 : cc[t] + 1;   // periodic, so nbr3 below sees wrapped coordinates
        }
        if (!ok) continue;
        const size_t qq = cell3(A, cc);
        const T sv = A.S[l][qq];
        const T wv = onface ? exp(-sc.g * (T(0.5) * (sv + A.S[l][nbr3(A, cc, l, 1)]))) : exp(-sc.g * sv);
        w = (w == T(2)) ? wv : tmin(w, wv);
      }
      // low-order residual on the +-h/2 neighbours (a centre replaced by its average)
      int fm[3] = {px, py, pz}, fp[3] = {px, py, pz};
      fm[l] -= 1;
      fp[l] += 1;
      const T zm = zoff(A, fa, fm[0], fm[1], fm[2], true), z0 = z[2], zp = zoff(A, fa, fp[0], fp[1], fp[2], true);
      const T Fr = T(0.5) * (flux<FLUX, T>(m, l, z0) + flux<FLUX, T>(m, l, zp)) -
                   T(0.5) * alpha_interval<FLUX, T>(m, l, z0, zp) * (zp - z0);
      const T Fl = T(0.5) * (flux<FLUX, T>(m, l, zm) + flux<FLUX, T>(m, l, z0)) -
                   T(0.5) * alpha_interval<FLUX, T>(m, l, zm, z0) * (z0 - zm);
      const T RL = (apot<T>(m, zp) - T(2) * apot<T>(m, z0) + apot<T>(m, zm)) * (T(4) * ih * ih) - (Fr - Fl) * (T(2) * ih);
      r = w * rh + (T(1) - w) * RL;
    }
    acc = (l == 0) ? r : acc + r;
  }
  T pv = A.pt[s][q] + sc.taut * acc;
  if (A.limiter) pv = tmin(tmax(pv, sc.umin), sc.umax);
  T po = comb ? rk_comb(sc.cAt, A.Apt[o][s][q], sc.cFt, pv) : rk_scale(sc.cFt, pv);
  if (A.limiter && A.sg[o]) po = safeguard<T>(po, sc.umin, sc.umax, A.tol, A.stats);
  A.Opt[o][s][q] = po;
}

// One thread per cell: the average, then the 7 point kinds. MINB resident CTAs per SM:
// FP64 4 (the most its 46 KB of shared memory allow; 90-99 registers, none spilled;
// porous medium 128^3 stage 2.59 ms at the compiler's 149 registers and 3 CTAs, 2.39 ms
// at 4); FP32-mixed 8 at <= 64 registers (stage 1.24 ms with the compiler's 127
// registers and 4 CTAs per SM; 0.92 / 0.90 / 0.90 ms at 6 / 8 / 10 CTAs per SM;
// splitting a cell's 8 values over 2, 4 or 8 threads measured 0.97, 1.09, 1.35 ms)
template <int FLUX, class T, int MINB>
__global__ void __launch_bounds__(U3T, MINB) update3d_tile_kernel(const DevModel m, const StageArgs3D<T> A, int o) {
  const double dtv = *A.dt;
  if (is_zero_bits(dtv)) return;   // uniform over the grid
  __shared__ K4Scal<T> sc;
  __shared__ T sZ[8][B3N], sAz[8][B3N];
  if (threadIdx.x < 32) k4_scalars<T>(m, A, o, dtv, sc);
  const int n0 = A.n[0], n1 = A.n[1], n2 = A.n[2];
  const int tiles_x = (n0 + U3X - 1) / U3X, tiles_y = (n1 + U3Y - 1) / U3Y;
  const int tb = blockIdx.x;
  const int c0x = (tb % tiles_x) * U3X, c0y = ((tb / tiles_x) % tiles_y) * U3Y, c0z = (tb / (tiles_x * tiles_y)) * U3Z;
  k4_load<T>(m, A, c0x, c0y, c0z, U3T, sZ, sAz);
  __syncthreads();
  const int lx = threadIdx.x % U3X, ly = (threadIdx.x / U3X) % U3Y, lz = threadIdx.x / (U3X * U3Y);
  const int c[3] = {c0x + lx, c0y + ly, c0z + lz};
  if (c[0] >= n0 || c[1] >= n1 || c[2] >= n2) return;   // after the only barrier
  const size_t q = ((size_t)c[2] * n1 + c[1]) * n0 + c[0];
  // an integer test: GB300 runs FP64 compares on its slow FP64 unit
  const bool comb = !is_zero_bits(A.cA[o]);
  k4_average<T>(m, A, o, c, q, sc, comb);
  for (int s = 1; s < 8; ++s) k4_point<FLUX, T>(m, A, o, c, q, lx, ly, lz, s, sZ, sAz, sc, comb);
}

// K2 over the same tiles: the cell's Simpson block (fine offsets {-1, 0, 1}^3 around 2c,
// index o = mx + 1 + 3 (my + 1) + 9 (mz + 1)) lies in the cells c - 1 .. c along each
// axis, so each CTA stages the 8 kinds of its cells and of the cells one step lower
// (a (U3X + 1) x (U3Y + 1) x (U3Z + 1) box) with a(z) once per location, instead of 27
// gathers and a(z) evaluations per cell. Sums run in the gathered form's order.
constexpr int C3X = U3X + 1, C3Y = U3Y + 1, C3Z = U3Z + 1, C3N = C3X * C3Y * C3Z;

template <int FLUX, class T>
__global__ void __launch_bounds__(U3T) cellq3d_kernel(const DevModel m, const StageArgs3D<T> A) {
  if (is_zero_bits(*A.dt)) return;   // uniform over the grid
  __shared__ T sZ[8][C3N], sAz[8][C3N];
  const int n0 = A.n[0], n1 = A.n[1], n2 = A.n[2];
  const int tiles_x = (n0 + U3X - 1) / U3X, tiles_y = (n1 + U3Y - 1) / U3Y;
  const int tb = blockIdx.x;
  const int c0x = (tb % tiles_x) * U3X, c0y = ((tb / tiles_x) % tiles_y) * U3Y, c0z = (tb / (tiles_x * tiles_y)) * U3Z;
  for (int k = threadIdx.x; k < 8 * C3N; k += U3T) {
    const int sk = k / C3N, b = k - sk * C3N;
    const int bx = b % C3X, by = (b / C3X) % C3Y, bz = b / (C3X * C3Y);
    const size_t q = ((size_t)wrapi(c0z - 1 + bz, n2) * n1 + wrapi(c0y - 1 + by, n1)) * n0 + wrapi(c0x - 1 + bx, n0);
    const T z = sk == 0 ? A.C[q] : A.pt[sk][q];
    sZ[sk][b] = z;
    sAz[sk][b] = apot<T>(m, z);
  }
  __syncthreads();
  const int lx = threadIdx.x % U3X, ly = (threadIdx.x / U3X) % U3Y, lz = threadIdx.x / (U3X * U3Y);
  const int c[3] = {c0x + lx, c0y + ly, c0z + lz};
  if (c[0] >= n0 || c[1] >= n1 || c[2] >= n2) return;   // after the only barrier
  const size_t q = ((size_t)c[2] * n1 + c[1]) * n0 + c[0];
  // fine offset m in {-1, 0, 1} along an axis: box cell (local + 1) + (m >> 1), kind bit
  // m & 1. In FP32 the loops are unrolled (every offset below a constant: the index
  // arithmetic would otherwise outweigh the stencil's); in FP64, bound by the FP64 unit,
  // they are not (the unrolled form doubles the registers)
  constexpr int UNR_L = sizeof(T) == 4 ? 3 : 1, UNR_O = sizeof(T) == 4 ? 27 : 1;
  const int base = (lx + 1) + C3X * ((ly + 1) + C3Y * (lz + 1));
  auto at = [&](int o, int& kind) {
    const int mx = o % 3 - 1, my = (o / 3) % 3 - 1, mz = o / 9 - 1;
    kind = (mx & 1) | ((my & 1) << 1) | ((mz & 1) << 2);
    return base + (mx >> 1) + C3X * ((my >> 1) + C3Y * (mz >> 1));
  };
  const T u = to_stencil<T>(A.ub[q]);
#pragma unroll UNR_L
  for (int l = 0; l < 3; ++l) {
    const int st = l == 0 ? 1 : (l == 1 ? 3 : 9);
    T fs = T(0), as = T(0);
#pragma unroll UNR_O
    for (int o = 0; o < 27; ++o) {
      const int mm[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
      if (mm[l] != 0) continue;
      const T w = wtrans<T>(o, l);
      int km, k0, kp;
      const int bm = at(o - st, km), b0 = at(o, k0), bp = at(o + st, kp);
      // without a flux (pure diffusion) its terms are exact zeros: not formed
      if constexpr (FLUX != FLUX_ZERO) fs = fs + w * flux<FLUX, T>(m, l, sZ[kp][bp]);
      const T ahat = (-sAz[km][bm] + T(8) * sAz[k0][b0] - sAz[kp][bp]) * T(1.0 / 6.0);
      as = as + w * ahat;
    }
    A.FH[l][q] = fs * T(1.0 / 36.0);
    A.AH[l][q] = as * T(1.0 / 36.0);
    if constexpr (FLUX == FLUX_ZERO) {
      A.FL[l][q] = T(0);
    } else {
      const T un = to_stencil<T>(A.ub[nbr3(A, c, l, 1)]);
      const T al = alpha_interval<FLUX, T>(m, l, u, un);
      A.FL[l][q] = T(0.5) * (flux<FLUX, T>(m, l, u) + flux<FLUX, T>(m, l, un)) - T(0.5) * al * (un - u);
    }
    if (A.blend) {
      T v[5];
      for (int t = 0; t < 5; ++t) v[t] = to_stencil<T>(A.ub[nbr3(A, c, l, t - 2)]);
      auto stv = [](T a, T b, T cc) {
        return tabs(a - T(2) * b + cc) / (tabs(a) + T(2) * tabs(b) + tabs(cc) + T(1e-13));
      };
      A.S[l][q] = (stv(v[0], v[1], v[2]) + T(4) * stv(v[1], v[2], v[3]) + stv(v[2], v[3], v[4])) * T(1.0 / 6.0);
    }
  }
}

template <int FLUX, class T>
cudaError_t run3d(const DevModel& m, const StageArgs3D<T>& a, cudaStream_t s) {
  const size_t N = (size_t)a.n[0] * a.n[1] * a.n[2];
  const int grid = (int)std::min<size_t>((N + T3 - 1) / T3, 152 * 16);
  const long long tiles = (long long)((a.n[0] + U3X - 1) / U3X) * ((a.n[1] + U3Y - 1) / U3Y) * ((a.n[2] + U3Z - 1) / U3Z);
  if (tiles > 0x7FFFFFFFLL) return cudaErrorInvalidConfiguration;
  centre3d_kernel<T><<<grid, T3, 0, s>>>(a);
  cellq3d_kernel<FLUX, T><<<(unsigned)tiles, U3T, 0, s>>>(m, a);
  for (int o = 0; o < a.nout; ++o) {
    limit3d_kernel<FLUX, T><<<grid, T3, 0, s>>>(m, a, o);
    update3d_tile_kernel<FLUX, T, sizeof(T) == 4 ? 8 : 4><<<(unsigned)tiles, U3T, 0, s>>>(m, a, o);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t dispatch3d(int flux, const DevModel& m, const StageArgs3D<T>& a, cudaStream_t s) {
  switch (flux) {
    case FLUX_ZERO: return run3d<FLUX_ZERO, T>(m, a, s);
    case FLUX_LINEAR: return run3d<FLUX_LINEAR, T>(m, a, s);
    case FLUX_BURGERS: return run3d<FLUX_BURGERS, T>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_stage3d_f64(int flux, const DevModel& m, const StageArgs3D<double>& a, cudaStream_t s) {
  return dispatch3d<double>(flux, m, a, s);
}
cudaError_t launch_stage3d_f32(int flux, const DevModel& m, const StageArgs3D<float>& a, cudaStream_t s) {
  return dispatch3d<float>(flux, m, a, s);
}

// CFL rate of a 3D mesh: max over cells and directions of |f_l'(ub)| / h_l +
// kappa_max / h_l^2 (the fluxes of 3D meshes have no interior extrema of f_l', so the
// interval maximum over a face is taken at its end points, both cell averages)
template <int FLUX>
__global__ void __launch_bounds__(RED_THREADS) rate3d_kernel(const DevModel m, size_t N, const double* __restrict__ ub,
                                                              double ih0, double ih1, double ih2, double kmax,
                                                              unsigned long long* rate_bits) {
  const double inv_h[3] = {ih0, ih1, ih2};
  double best = 0.0;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    const double u = ub[q];
    for (int l = 0; l < 3; ++l) best = tmax(best, dflux_abs<FLUX, double>(m, l, u) * inv_h[l] + kmax * inv_h[l] * inv_h[l]);
  }
  for (int off = 16; off > 0; off >>= 1) best = tmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomicMax(rate_bits, (unsigned long long)__double_as_longlong(best));
}

cudaError_t launch_rate3d(int flux, const DevModel& m, const int* n, const double* ub, const double* inv_h, double kmax,
                          unsigned long long* rate_bits, cudaStream_t s) {
  const int blocks = 152 * 4;
  const size_t N = (size_t)n[0] * n[1] * n[2];
  switch (flux) {
    case FLUX_ZERO:
      rate3d_kernel<FLUX_ZERO><<<blocks, RED_THREADS, 0, s>>>(m, N, ub, inv_h[0], inv_h[1], inv_h[2], kmax, rate_bits);
      break;
    case FLUX_LINEAR:
      rate3d_kernel<FLUX_LINEAR><<<blocks, RED_THREADS, 0, s>>>(m, N, ub, inv_h[0], inv_h[1], inv_h[2], kmax, rate_bits);
      break;
    case FLUX_BURGERS:
      rate3d_kernel<FLUX_BURGERS><<<blocks, RED_THREADS, 0, s>>>(m, N, ub, inv_h[0], inv_h[1], inv_h[2], kmax, rate_bits);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace af
