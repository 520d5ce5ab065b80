// Fused 1D stage kernel of the compact fourth-order doubly conservative active flux
// method (arXiv 2510.11527, Sections 2 and 5.1). Same structure as the 2D kernel:
// each CTA owns TX cells (cell average ub_i and the point value P_i = u_{i+1/2}) and
// stages a +-3 cell halo in shared memory.
//   centre          u_i = (6 ub_i - u_{i-1/2} - u_{i+1/2}) / 4
//   point residual  5-point line [P_{i-1}, c_i, P_i, c_{i+1}, P_{i+1}]
//   DC potential    a^_i = (-a(P_{i-1}) + 8 a(c_i) - a(P_i)) / 6   (Proposition 2.1)
//   low order       LLF with interval wave speed, states u^{L,+-} with factor 2
//   limiter         theta^c (2 states) and theta^d (4 states) with factor 6
#pragma once
#include "stage2d.cuh"

namespace af {

template <int FLUX, class T>
struct Tile1D {
  static constexpr int TX = 256, NT = TX, H = 3, BX = TX + 2 * H;
};

template <int FLUX, class T, class PT>
__global__ void __launch_bounds__(256) stage1d_kernel(const DevModel m, const StageArgs2D<PT> A) {
  using L = Tile1D<FLUX, T>;
  constexpr int TX = L::TX, NT = L::NT, H = L::H, BX = L::BX;
  __shared__ T sU[BX], sP[BX], sC[BX];
  __shared__ T fP[BX], aP[BX], fC[BX], aC[BX], dP[BX], dC[BX], fU[BX], aU[BX];
  __shared__ T sFH[BX], sAH[BX], sFL[BX], sULp[BX], sULm[BX], sFlim[BX], sAlim[BX];
  __shared__ T sS[BX], sTC[BX], sTD[BX];

  const double dtv = *A.dt;
  if (dtv == 0.0) return;
  const int nx = A.nx;
  const int i0 = blockIdx.x * TX;
  const int tid = threadIdx.x;
  const T umin = T(m.umin), umax = T(m.umax);
  const bool blend = A.blend != 0;
  const bool ext = A.blend == 2;

  for (int k = tid; k < BX; k += NT) {
    const size_t g = (size_t)wrapi(i0 - H + k, nx);
    sU[k] = T(A.ub[g]);
    sP[k] = T(A.V[g]);
  }
  __syncthreads();
  for (int b = tid; b < BX; b += NT) {
    const T u = sU[b];
    fU[b] = flux<FLUX, T>(m, 0, u);
    aU[b] = apot<T>(m, u);
    const T p = sP[b];
    fP[b] = flux<FLUX, T>(m, 0, p);
    dP[b] = dflux_abs<FLUX, T>(m, 0, p);
    aP[b] = apot<T>(m, p);
    if (b >= 1) {
      const T c = (T(6) * u - sP[b - 1] - p) * T(0.25);
      sC[b] = c;
      fC[b] = flux<FLUX, T>(m, 0, c);
      dC[b] = dflux_abs<FLUX, T>(m, 0, c);
      aC[b] = apot<T>(m, c);
    }
    if (blend && !ext && b >= 1 && b < BX - 1) {
      const T um = sU[b - 1], up = sU[b + 1];
      sTC[b] = tabs(um - T(2) * u + up) / (tabs(um) + T(2) * tabs(u) + tabs(up) + T(1e-13));
    }
  }
  __syncthreads();
  const T ih = T(A.inv_h1);
  const T i6h = T(A.inv_h1 / 6.0), i3h2 = T(A.inv_h1 * A.inv_h1 / 3.0);
  const int bo = H + tid;
  // high-order point residual of the owned point
  T rH;
  {
    const int b = bo;
    const T alpha = tmax(tmax(tmax(dP[b - 1], dC[b]), tmax(dC[b + 1], dP[b + 1])), dP[b]);
    rH = line_res<T>(sP[b - 1], sC[b], sP[b], sC[b + 1], sP[b + 1], fP[b - 1], fC[b], fC[b + 1], fP[b + 1], alpha,
                     aP[b - 1], aC[b], aP[b], aC[b + 1], aP[b + 1], i6h, i3h2);
  }
  for (int b = H - 2 + tid; b <= H + TX; b += NT) {
    if (b >= H - 1 && b < H + TX) sFH[b] = fP[b];
    if (b >= H - 1) sAH[b] = (T(8) * aC[b] - aP[b - 1] - aP[b]) * T(1.0 / 6.0);
    const T ul = sU[b], ur = sU[b + 1];
    sFL[b] = T(0.5) * (fU[b] + fU[b + 1]) - T(0.5) * alpha_interval<FLUX, T>(m, 0, ul, ur) * (ur - ul);
  }
  if (blend) {
    for (int b = H - 1 + tid; b <= H + TX; b += NT) {
      sS[b] = ext ? T(A.s_ext[wrapi(i0 - H + b, nx)]) : (sTC[b - 1] + T(4) * sTC[b] + sTC[b + 1]) * T(1.0 / 6.0);
    }
  }
  __syncthreads();
  T rP = rH;
  if (blend) {
    const T g = T(A.gamma);
    for (int b = H - 1 + tid; b <= H + TX; b += NT) {
      sTD[b] = exp(-g * sS[b]);
      if (b < H + TX) sTC[b] = exp(-g * (T(0.5) * (sS[b] + sS[b + 1])));
    }
    __syncthreads();
    for (int b = H - 1 + tid; b <= H + TX; b += NT) {
      if (b < H + TX) sFH[b] = sTC[b] * sFH[b] + (T(1) - sTC[b]) * sFL[b];
      sAH[b] = sTD[b] * sAH[b] + (T(1) - sTD[b]) * aU[b];
    }
    {
      const int b = bo;
      const T zm = sU[b], z0 = sP[b], zp = sU[b + 1];
      const T Fr = T(0.5) * (fP[b] + fU[b + 1]) - T(0.5) * alpha_interval<FLUX, T>(m, 0, z0, zp) * (zp - z0);
      const T Fl = T(0.5) * (fU[b] + fP[b]) - T(0.5) * alpha_interval<FLUX, T>(m, 0, zm, z0) * (z0 - zm);
      const T RL = (aU[b + 1] - T(2) * aP[b] + aU[b]) * (T(4) * ih * ih) - (Fr - Fl) * (T(2) * ih);
      rP = sTC[b] * rH + (T(1) - sTC[b]) * RL;
    }
    __syncthreads();
  }
  const int gi = i0 + tid;
  const bool own = gi < nx;
  T* Flim = A.limiter ? sFlim : sFH;
  T* Alim = A.limiter ? sAlim : sAH;
  for (int o = 0; o < A.nout; ++o) {
    const double tau = A.tcoef[o] * dtv;
    const double mu = tau * A.inv_h1, nu = mu * A.inv_h1;
    if (A.limiter) {
      const T m2 = T(2.0 * mu), n2 = T(2.0 * nu);
      for (int b = H - 2 + tid; b <= H + TX + 1; b += NT) {
        const T u = sU[b], f = fU[b], a = aU[b];
        if (b <= H + TX) sULp[b] = u - m2 * (sFL[b] - f) + n2 * (aU[b + 1] - a);
        if (b >= H - 1) sULm[b] = u - m2 * (f - sFL[b - 1]) - n2 * (a - aU[b - 1]);
      }
      __syncthreads();
      const T k6 = T(6.0 * mu), q6 = T(6.0 * nu);
      for (int b = H - 1 + tid; b <= H + TX; b += NT) {
        if (b < H + TX) {
          const T fh = sFH[b], fl = sFL[b], dF = fh - fl;
          const T zp = sULp[b], zm = sULm[b + 1];
          const T t = tmin(theta_fn<T>(zp, zp - k6 * dF, umin, umax), theta_fn<T>(zm, zm + k6 * dF, umin, umax));
          sFlim[b] = is_one(t) ? fh : fl + t * dF;
        }
        const T ah = sAH[b], al = aU[b], d = q6 * (ah - al);
        const T t = tmin(tmin(theta_fn<T>(sULp[b - 1], sULp[b - 1] + d, umin, umax),
                              theta_fn<T>(sULp[b], sULp[b] - d, umin, umax)),
                         tmin(theta_fn<T>(sULm[b], sULm[b] - d, umin, umax),
                              theta_fn<T>(sULm[b + 1], sULm[b + 1] + d, umin, umax)));
        sAlim[b] = is_one(t) ? ah : al + t * (ah - al);
      }
      __syncthreads();
    }
    if (own) {
      const int b = bo;
      const size_t g = (size_t)gi;
      const double ubfe = A.ub[g] - mu * ((double)Flim[b] - (double)Flim[b - 1]) +
                          nu * (((double)Alim[b + 1] - 2.0 * (double)Alim[b]) + (double)Alim[b - 1]);
      T p = sP[b] + T(tau) * rP;
      if (A.limiter) p = tmin(tmax(p, umin), umax);
      const double cA = A.cA[o], cF = A.cF[o];
      double ubo;
      PT po;
      if (cA != 0.0) {
        ubo = rk_comb(cA, A.Aub[o][g], cF, ubfe);
        po = PT(rk_comb(T(cA), T(A.AV[o][g]), T(cF), p));
      } else {
        ubo = rk_scale(cF, ubfe);
        po = PT(rk_scale(T(cF), p));
      }
      if (A.limiter && A.sg[o]) {
        ubo = safeguard<double>(ubo, m.umin, m.umax, A.tol, A.stats, true);
        po = safeguard<PT>(po, PT(m.umin), PT(m.umax), A.tol, A.stats);
      }
      A.Oub[o][g] = ubo;
      A.OV[o][g] = po;
    }
    if (o + 1 < A.nout) __syncthreads();
  }
}

}  // namespace af
