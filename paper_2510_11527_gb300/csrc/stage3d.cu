// 3D stage of the compact fourth-order doubly conservative active flux method with the
// monolithic convex limiter (arXiv 2510.11527, Section 4's 3D DoFs; Section 5.2 with
// d = 3: directional split 1/6, limiter factor 18). Four kernels per stage, one thread
// per cell, FP64:
//   K1 centre values from the tensor Simpson rule of the cell average;
//   K2 per direction: high-order face flux (Simpson face average of f_l), DC cell
//      potential (transverse Simpson average of the 1D potential along l), LLF face
//      flux with the interval wave speed, smoothness value s_l;
//   K3 per output: blend, low-order states u^{L,+-}_l, limiting parameters
//      theta^c (faces) and theta^d (cells), limited face fluxes and cell potentials;
//   K4 per output: limited cell-average update and the 7 point values of the cell
//      (5-point lines along each axis, blend with the low-order point residual,
//      projection), RK combination and post-stage safeguard.
// All locations are addressed on the fine grid of half-cell spacing: the DoF at
// (i + sx/2, j + sy/2, k + sz/2) has fine index (2i + sx, 2j + sy, 2k + sz), so a
// 5-point line is the fine points p - 2e .. p + 2e and a Simpson average weighs 1, 4, 1
// per axis. Inputs are read from global memory (reuse through L1 / L2).
#include "launch.h"
#include "stage3d.cuh"

namespace af {
namespace {

constexpr int T3 = 256;

__device__ __forceinline__ size_t cells3(const StageArgs3D& A) { return (size_t)A.n[0] * A.n[1] * A.n[2]; }

// cell coordinates of a linear index (32-bit: meshes hold < 2^31 cells)
__device__ __forceinline__ void decode3(const StageArgs3D& A, size_t q, int* c) {
  const unsigned qq = (unsigned)q, n0 = (unsigned)A.n[0], n1 = (unsigned)A.n[1];
  const unsigned r = qq / n0;
  c[0] = (int)(qq - r * n0);
  c[1] = (int)(r % n1);
  c[2] = (int)(r / n1);
}

// periodic cell index
__device__ __forceinline__ size_t cell3(const StageArgs3D& A, const int* c) {
  return ((size_t)wrapi(c[2], A.n[2]) * A.n[1] + wrapi(c[1], A.n[1])) * A.n[0] + wrapi(c[0], A.n[0]);
}

// neighbour step cells along l of the cell at coordinates c (|step| <= 2, no division)
__device__ __forceinline__ size_t nbr3(const StageArgs3D& A, const int* c, int l, int step) {
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
__device__ __forceinline__ double wtrans(int o, int l) {
  // drop the factor of axis l from the 3D weight: divide by its 1D weight (4 or 1)
  const int ml = l == 0 ? o % 3 : (l == 1 ? (o / 3) % 3 : o / 9);
  return ml == 1 ? kW27[o] * 0.25 : kW27[o];
}

// The wrapped fine coordinates of offsets -2 .. +3 from the cell's fine origin 2c along
// each axis, formed once per cell: a fine access is then two shifts and a lookup.
struct FineAxes {
  int f[3][6];
};
__device__ __forceinline__ FineAxes fine_axes(const StageArgs3D& A, const int* c) {
  FineAxes fa;
  for (int l = 0; l < 3; ++l)
    for (int o = 0; o < 6; ++o) fa.f[l][o] = wrapi(2 * c[l] + o - 2, 2 * A.n[l]);
  return fa;
}
// fine value at offsets (ox, oy, oz) in [-2, 3] from 2c: kind 0 is the recovered centre,
// or the cell average when avg is set (the low-order neighbours of the blend)
__device__ __forceinline__ double zoff(const StageArgs3D& A, const FineAxes& fa, int ox, int oy, int oz, bool avg = false) {
  const int fx = fa.f[0][ox + 2], fy = fa.f[1][oy + 2], fz = fa.f[2][oz + 2];
  const int kind = (fx & 1) | ((fy & 1) << 1) | ((fz & 1) << 2);
  const size_t q = ((size_t)(fz >> 1) * A.n[1] + (fy >> 1)) * A.n[0] + (fx >> 1);
  return (kind == 0 && !avg) ? A.C[q] : A.in[kind][q];
}

__global__ void __launch_bounds__(T3) centre3d_kernel(const StageArgs3D A) {
  if (*A.dt == 0.0) return;
  const size_t N = cells3(A);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    int c[3];
    decode3(A, q, c);
    const FineAxes fa = fine_axes(A, c);
    double acc = 0.0;
    for (int o = 0; o < 27; ++o) {
      const int mm[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
      if (mm[0] == 0 && mm[1] == 0 && mm[2] == 0) continue;
      acc = acc + kW27[o] * zoff(A, fa, mm[0], mm[1], mm[2]);
    }
    A.C[q] = (216.0 * A.in[0][q] - acc) / 64.0;
  }
}

template <int FLUX>
__global__ void __launch_bounds__(T3) cellq3d_kernel(const DevModel m, const StageArgs3D A) {
  if (*A.dt == 0.0) return;
  const size_t N = cells3(A);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    int c[3];
    decode3(A, q, c);
    const double u = A.in[0][q];
    // the cell's Simpson block: fine offsets {-1, 0, 1}^3 around 2c (index o = mx + 1 +
    // 3 (my + 1) + 9 (mz + 1)), with a(z) evaluated once per location
    const FineAxes fa = fine_axes(A, c);
    double zb[27], ab[27];
    for (int o = 0; o < 27; ++o) {
      zb[o] = zoff(A, fa, o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1);
      ab[o] = apot<double>(m, zb[o]);
    }
    for (int l = 0; l < 3; ++l) {
      const int st = l == 0 ? 1 : (l == 1 ? 3 : 9);
      double fs = 0.0, as = 0.0;
      for (int o = 0; o < 27; ++o) {
        const int mm[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
        if (mm[l] != 0) continue;
        const double w = wtrans(o, l);
        fs = fs + w * flux<FLUX, double>(m, l, zb[o + st]);
        const double ahat = (-ab[o - st] + 8.0 * ab[o] - ab[o + st]) * (1.0 / 6.0);
        as = as + w * ahat;
      }
      A.FH[l][q] = fs * (1.0 / 36.0);
      A.AH[l][q] = as * (1.0 / 36.0);
      const double un = A.in[0][nbr3(A, c, l, 1)];
      const double al = alpha_interval<FLUX, double>(m, l, u, un);
      A.FL[l][q] = 0.5 * (flux<FLUX, double>(m, l, u) + flux<FLUX, double>(m, l, un)) - 0.5 * al * (un - u);
      if (A.blend) {
        double v[5];
        for (int t = 0; t < 5; ++t) v[t] = A.in[0][nbr3(A, c, l, t - 2)];
        auto st = [](double a, double b, double cc) {
          return tabs(a - 2.0 * b + cc) / (tabs(a) + 2.0 * tabs(b) + tabs(cc) + 1e-13);
        };
        A.S[l][q] = (st(v[0], v[1], v[2]) + 4.0 * st(v[1], v[2], v[3]) + st(v[2], v[3], v[4])) * (1.0 / 6.0);
      }
    }
  }
}

// low-order directional states of cell q along l (Lemma 5.1 with factor 2d = 6)
// (q: the cell, qp / qm: its neighbour after / before it along l)
template <int FLUX>
__device__ __forceinline__ double ulp3(const DevModel& m, const StageArgs3D& A, size_t q, size_t qp, int l, double mu,
                                       double nu) {
  const double u = A.in[0][q], un = A.in[0][qp];
  return u - 6.0 * mu * (A.FL[l][q] - flux<FLUX, double>(m, l, u)) + 6.0 * nu * (apot<double>(m, un) - apot<double>(m, u));
}
template <int FLUX>
__device__ __forceinline__ double ulm3(const DevModel& m, const StageArgs3D& A, size_t q, size_t qm, int l, double mu,
                                       double nu) {
  const double u = A.in[0][q], um = A.in[0][qm];
  return u - 6.0 * mu * (flux<FLUX, double>(m, l, u) - A.FL[l][qm]) - 6.0 * nu * (apot<double>(m, u) - apot<double>(m, um));
}

template <int FLUX>
__global__ void __launch_bounds__(T3) limit3d_kernel(const DevModel m, const StageArgs3D A, int o) {
  const double dtv = *A.dt;
  if (dtv == 0.0) return;
  const double tau = A.tcoef[o] * dtv;
  const size_t N = cells3(A);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    int c[3];
    decode3(A, q, c);
    const double u = A.in[0][q], au = apot<double>(m, u);
    for (int l = 0; l < 3; ++l) {
      const double mu = tau * A.inv_h[l], nu = mu * A.inv_h[l];
      const size_t qp = nbr3(A, c, l, 1), qm = nbr3(A, c, l, -1);
      double fh = A.FH[l][q], ah = A.AH[l][q];
      const double fl = A.FL[l][q];
      if (A.blend) {
        const double tc = exp(-A.gamma * (0.5 * (A.S[l][q] + A.S[l][qp])));
        const double td = exp(-A.gamma * A.S[l][q]);
        fh = tc * fh + (1.0 - tc) * fl;
        ah = td * ah + (1.0 - td) * au;
      }
      double flim = fh, alim = ah;
      if (A.limiter) {
        const double umin = m.umin, umax = m.umax;
        const double k = 18.0 * mu, kd = 18.0 * nu;
        const double dF = fh - fl;
        const double zp = ulp3<FLUX>(m, A, q, qp, l, mu, nu), zm = ulm3<FLUX>(m, A, qp, q, l, mu, nu);
        const double tcl = tmin(theta_fn<double>(zp, zp - k * dF, umin, umax), theta_fn<double>(zm, zm + k * dF, umin, umax));
        flim = is_one(tcl) ? fh : fl + tcl * dF;
        const double dA = ah - au;
        const double p0 = ulp3<FLUX>(m, A, qm, q, l, mu, nu), q0 = ulm3<FLUX>(m, A, q, qm, l, mu, nu);
        const double td = tmin(tmin(theta_fn<double>(p0, p0 + kd * dA, umin, umax), theta_fn<double>(zp, zp - kd * dA, umin, umax)),
                               tmin(theta_fn<double>(q0, q0 - kd * dA, umin, umax), theta_fn<double>(zm, zm + kd * dA, umin, umax)));
        alim = is_one(td) ? ah : au + td * dA;
      }
      A.Flim[l][q] = flim;
      A.Alim[l][q] = alim;
    }
  }
}

template <int FLUX>
__global__ void __launch_bounds__(T3) update3d_kernel(const DevModel m, const StageArgs3D A, int o) {
  const double dtv = *A.dt;
  if (dtv == 0.0) return;
  const double tau = A.tcoef[o] * dtv;
  const double cA = A.cA[o], cF = A.cF[o];
  const size_t N = cells3(A);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    int c[3];
    decode3(A, q, c);
    const FineAxes fa = fine_axes(A, c);
    // limited cell-average update (eq. multid_limited_average)
    double v = A.in[0][q];
    for (int l = 0; l < 3; ++l) {
      const double mu = tau * A.inv_h[l], nu = mu * A.inv_h[l];
      const size_t qm = nbr3(A, c, l, -1), qp = nbr3(A, c, l, 1);
      v = v - mu * (A.Flim[l][q] - A.Flim[l][qm]) + nu * (A.Alim[l][qp] - 2.0 * A.Alim[l][q] + A.Alim[l][qm]);
    }
    double ubo = cA != 0.0 ? rk_comb(cA, A.A[o][0][q], cF, v) : rk_scale(cF, v);
    if (A.limiter && A.sg[o]) ubo = safeguard<double>(ubo, m.umin, m.umax, A.tol, A.stats, true);
    A.O[o][0][q] = ubo;
    // point values owned by the cell: kinds 1..7 at fine 2c + s
    for (int s = 1; s < 8; ++s) {
      const int p[3] = {s & 1, (s >> 1) & 1, (s >> 2) & 1};   // offsets from 2c
      double acc = 0.0;
      for (int l = 0; l < 3; ++l) {
        const double ih = A.inv_h[l];
        double z[5], fz[5], dz[5], az[5];
        for (int t = 0; t < 5; ++t) {
          int f[3] = {p[0], p[1], p[2]};
          f[l] += t - 2;
          z[t] = zoff(A, fa, f[0], f[1], f[2]);
          fz[t] = flux<FLUX, double>(m, l, z[t]);
          dz[t] = dflux_abs<FLUX, double>(m, l, z[t]);
          az[t] = apot<double>(m, z[t]);
        }
        const double alpha = tmax(tmax(tmax(dz[0], dz[1]), tmax(dz[3], dz[4])), dz[2]);
        const double rh = line_res<double>(z[0], z[1], z[2], z[3], z[4], fz[0], fz[1], fz[3], fz[4], alpha, az[0], az[1],
                                           az[2], az[3], az[4], A.i6h[l], A.i3h2[l]);
        double r = rh;
        if (A.blend) {
          // weight: min of theta^{c,s}_l over the l-faces holding the point (s_l = 1),
          // else of theta^{d,s}_l over the cells holding it
          const bool onface = (s >> l) & 1;
          double w = 2.0;
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
            const double sv = A.S[l][qq];
            const double wv = onface ? exp(-A.gamma * (0.5 * (sv + A.S[l][nbr3(A, cc, l, 1)]))) : exp(-A.gamma * sv);
            w = (w == 2.0) ? wv : tmin(w, wv);
          }
          // low-order residual on the +-h/2 neighbours (a centre replaced by its average)
          int fm[3] = {p[0], p[1], p[2]}, fp[3] = {p[0], p[1], p[2]};
          fm[l] -= 1;
          fp[l] += 1;
          const double zm = zoff(A, fa, fm[0], fm[1], fm[2], true), z0 = z[2],
                       zp = zoff(A, fa, fp[0], fp[1], fp[2], true);
          const double Fr = 0.5 * (flux<FLUX, double>(m, l, z0) + flux<FLUX, double>(m, l, zp)) -
                            0.5 * alpha_interval<FLUX, double>(m, l, z0, zp) * (zp - z0);
          const double Fl = 0.5 * (flux<FLUX, double>(m, l, zm) + flux<FLUX, double>(m, l, z0)) -
                            0.5 * alpha_interval<FLUX, double>(m, l, zm, z0) * (z0 - zm);
          const double RL = (apot<double>(m, zp) - 2.0 * apot<double>(m, z0) + apot<double>(m, zm)) * (4.0 * ih * ih) -
                            (Fr - Fl) * (2.0 * ih);
          r = w * rh + (1.0 - w) * RL;
        }
        acc = (l == 0) ? r : acc + r;
      }
      double pv = A.in[s][q] + tau * acc;
      if (A.limiter) pv = tmin(tmax(pv, m.umin), m.umax);
      double po = cA != 0.0 ? rk_comb(cA, A.A[o][s][q], cF, pv) : rk_scale(cF, pv);
      if (A.limiter && A.sg[o]) po = safeguard<double>(po, m.umin, m.umax, A.tol, A.stats);
      A.O[o][s][q] = po;
    }
  }
}

template <int FLUX>
cudaError_t run3d(const DevModel& m, const StageArgs3D& a, cudaStream_t s) {
  const size_t N = (size_t)a.n[0] * a.n[1] * a.n[2];
  const int grid = (int)std::min<size_t>((N + T3 - 1) / T3, 152 * 16);
  centre3d_kernel<<<grid, T3, 0, s>>>(a);
  cellq3d_kernel<FLUX><<<grid, T3, 0, s>>>(m, a);
  for (int o = 0; o < a.nout; ++o) {
    limit3d_kernel<FLUX><<<grid, T3, 0, s>>>(m, a, o);
    update3d_kernel<FLUX><<<grid, T3, 0, s>>>(m, a, o);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stage3d_f64(int flux, const DevModel& m, const StageArgs3D& a, cudaStream_t s) {
  switch (flux) {
    case FLUX_ZERO: return run3d<FLUX_ZERO>(m, a, s);
    case FLUX_LINEAR: return run3d<FLUX_LINEAR>(m, a, s);
    case FLUX_BURGERS: return run3d<FLUX_BURGERS>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

// CFL rate of a 3D mesh: max over cells and directions of |f_l'(ub)| / h_l +
// kappa_max / h_l^2 (the fluxes of 3D meshes have no interior extrema of f_l', so the
// interval maximum over a face is taken at its end points, both cell averages)
template <int FLUX>
__global__ void __launch_bounds__(RED_THREADS) rate3d_kernel(const DevModel m, const StageArgs3D A, double kmax,
                                                              unsigned long long* rate_bits) {
  const size_t N = cells3(A);
  double best = 0.0;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    const double u = A.in[0][q];
    for (int l = 0; l < 3; ++l)
      best = tmax(best, dflux_abs<FLUX, double>(m, l, u) * A.inv_h[l] + kmax * A.inv_h[l] * A.inv_h[l]);
  }
  for (int off = 16; off > 0; off >>= 1) best = tmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomicMax(rate_bits, (unsigned long long)__double_as_longlong(best));
}

cudaError_t launch_rate3d(int flux, const DevModel& m, const StageArgs3D& a, double kmax, unsigned long long* rate_bits,
                          cudaStream_t s) {
  const int blocks = 152 * 4;
  switch (flux) {
    case FLUX_ZERO: rate3d_kernel<FLUX_ZERO><<<blocks, RED_THREADS, 0, s>>>(m, a, kmax, rate_bits); break;
    case FLUX_LINEAR: rate3d_kernel<FLUX_LINEAR><<<blocks, RED_THREADS, 0, s>>>(m, a, kmax, rate_bits); break;
    case FLUX_BURGERS: rate3d_kernel<FLUX_BURGERS><<<blocks, RED_THREADS, 0, s>>>(m, a, kmax, rate_bits); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace af
