// Fused 1D stage kernel of the compact fourth-order doubly conservative active flux
// method (arXiv 2510.11527, Sections 2 and 5.1; Appendix A for the diffusion form
// without double conservation). Same structure as the 2D kernel: each CTA owns TX cells
// (cell average ub_i and the point value P_i = u_{i+1/2}) and stages a +-3 cell halo
// in shared memory.
//   centre          u_i = (6 ub_i - u_{i-1/2} - u_{i+1/2}) / 4
//   point residual  5-point line [P_{i-1}, c_i, P_i, c_{i+1}, P_{i+1}]
//   DC potential    a^_i = (-a(P_{i-1}) + 8 a(c_i) - a(P_i)) / 6   (Proposition 2.1)
//   low order       LLF with interval wave speed, states u^{L,+-} with factor 2
//   limiter         theta^c (2 states; factor 6, or 2 without a diffusion term) and
//                   theta^d (4 states; factor 6)
// Without double conservation (Appendix A) the face flux is f(P_i) - kappa(P_i) D_c(u),
// D_c(u) = (P_{i-1} - 8 c_i + 8 c_{i+1} - P_{i+1}) / (6 dx), the point value takes
// 4/dx^2 sum_{m,n} b_mn kappa(z_m) z_n on its line, and the limiter blends the total
// face flux with F^L - (a(ub_{i+1}) - a(ub_i))/dx by Theta with factor 2.
// A bounded interval (Dirichlet / outflow ends) reads ghost cells and points from the
// boundary rule, updates the extra left end point u_{-1/2} in CTA 0, and holds
// Dirichlet end points at the boundary values.
#pragma once
#include "stage2d.cuh"

namespace af {

template <int FLUX, class T>
struct Tile1D {
  static constexpr int TX = 256, NT = TX, H = 3, BX = TX + 2 * H;
};

// Cell average ub_i and point value u_{j+1/2} at any index: stored values inside, the
// boundary rule outside (periodic image; Dirichlet value; even reflection about the
// end point for outflow). Indices far beyond an end (never read by an owned output)
// are clamped to the first H ghosts so that every load stays inside the arrays.
template <class PT>
__device__ __forceinline__ double cell1d(const StageArgs2D<PT>& A, int i, int H) {
  const int n = A.nx;
  if (A.bc == AF_BC_PERIODIC) return A.ub[wrapi(i, n)];
  if (i >= 0 && i < n) return A.ub[i];
  if (A.bc == AF_BC_DIRICHLET) return i < 0 ? A.bc_left : A.bc_right;
  i = i < -H ? -H : (i >= n + H ? n + H - 1 : i);
  return A.ub[i < 0 ? -1 - i : 2 * n - 1 - i];
}
template <class PT>
__device__ __forceinline__ PT point1d(const StageArgs2D<PT>& A, int j, int H) {
  const int n = A.nx;
  if (A.bc == AF_BC_PERIODIC) return A.V[wrapi(j, n)];
  if (j >= -1 && j <= n - 1) return A.V[j + 1];
  if (A.bc == AF_BC_DIRICHLET) return PT(j < -1 ? A.bc_left : A.bc_right);
  j = j < -H - 1 ? -H - 1 : (j >= n + H ? n + H - 1 : j);
  return A.V[(j < -1 ? -2 - j : 2 * (n - 1) - j) + 1];
}

// 4 sum_{m,n} b_mn k_m z_n of Appendix A, B = [0 0; 0 M] - [M 0; 0 0] written out row
// by row (each row sums to zero)
template <class T>
__device__ __forceinline__ T nodc_d2(const T z[5], const T k[5]) {
  const T r0 = T(-1.0 / 8) * z[0] + T(1.0 / 6) * z[1] - T(1.0 / 24) * z[2];
  const T r1 = T(1.0 / 6) * z[0] + T(0.5) * z[1] - T(5.0 / 6) * z[2] + T(1.0 / 6) * z[3];
  const T r2 = T(-1.0 / 8) * (z[0] + z[4]) + T(0.5) * (z[1] + z[3]) - T(0.75) * z[2];
  const T r3 = T(1.0 / 6) * z[1] - T(5.0 / 6) * z[2] + T(0.5) * z[3] + T(1.0 / 6) * z[4];
  const T r4 = T(-1.0 / 24) * z[2] + T(1.0 / 6) * z[3] - T(1.0 / 8) * z[4];
  return T(4) * ((k[0] * r0 + k[1] * r1) + (k[2] * r2 + (k[3] * r3 + k[4] * r4)));
}

// double -> exact widening of a stencil value (FP32 on the integer pipe)
__device__ __forceinline__ double d_of(double v) { return v; }
__device__ __forceinline__ double d_of(float v) { return f2d_exact(v); }

// The launch's scalars, formed once per CTA by one thread: GB300 runs FP64 arithmetic,
// FP64 compares and double <-> float conversions on its FP64 unit at 1/64 of the FP32
// rate, so per-thread copies would cost each cell as much as its own FP64 work.
template <class T>
struct Scal1D {
  T umin, umax, ih, i6h, i3h2, g, i4hh, i2h;
  T taut[2], m2[2], n2[2], k6[2], q6[2], cAt[2], cFt[2];
  double mu[2], nu[2];
  int comb[2];
};

template <int FLUX, class T, class PT>
__global__ void __launch_bounds__(256, 4) stage1d_kernel(const DevModel m, const StageArgs2D<PT> A) {
  using L = Tile1D<FLUX, T>;
  constexpr int TX = L::TX, NT = L::NT, H = L::H, BX = L::BX;
  // flux direction of the model functions: the 1D Buckley-Leverett flux is the gravity
  // form f1 (1 - g (1-u)^2), which the model keeps as direction 1 (Example 6.6)
  constexpr int XD = FLUX == FLUX_BL ? 1 : 0;
  __shared__ T sU[BX], sP[BX], sC[BX];
  // aP / aC hold kappa instead of a without double conservation (no DC potential)
  __shared__ T fP[BX], aP[BX], fC[BX], aC[BX], dP[BX], dC[BX], fU[BX], aU[BX];
  __shared__ T sFH[BX], sAH[BX], sFL[BX], sULp[BX], sULm[BX], sFlim[BX], sAlim[BX];
  __shared__ T sS[BX], sTC[BX], sTD[BX];

  const double dtv = *A.dt;
  if (is_zero_bits(dtv)) return;   // uniform over the grid
  const int nx = A.nx;
  const int i0 = blockIdx.x * TX;
  const int tid = threadIdx.x;
  __shared__ Scal1D<T> sc;
  // formed at once by the lanes of warp o (output o) and the upper lanes of warp 0 (the
  // mesh's values): GB300's FP64 unit takes as long for a warp instruction with one
  // active lane as with 32. Lane l evaluates fl(fl(fl(x y1) y2) y3) with the factors of
  // its value's formula (a factor 1 is exact, so each value is rounded as its formula
  // is; the divided line scales come from the host); only the stores differ between
  // lanes.
  if ((tid >> 5) < A.nout) {
    const int o = tid >> 5, l = tid & 31;
    const double ih = A.inv_h1, tau = A.tcoef[o] * dtv;
    double x = tau, y1 = 1.0, y2 = 1.0, y3 = 1.0;
    if (l < 16) {
      // 0: tau; 1: mu; 2: nu; 3: 2 mu; 4: 2 nu; 5: (2 or 2 P) mu; 6: 6 nu; 7, 8: cA, cF
      if (l >= 1 && l <= 6) y1 = ih;
      if (l == 2 || l == 4 || l == 6) y2 = ih;
      if (l == 3) y2 = 2.0;
      if (l == 5) y2 = A.nodc ? 2.0 : double(2 * m.lim_parts);
      if (l == 4) y3 = 2.0;
      if (l == 6) y3 = 6.0;
      if (l == 7) x = A.cA[o];
      if (l == 8) x = A.cF[o];
    } else {
      // 16, 17: u_min, u_max; 18: 1/h; 19: 1/(6h); 20: (1/h/h)/3; 21: gamma; 22: (4/h)/h;
      // 23: 2/h
      x = l == 16   ? m.umin
          : l == 17 ? m.umax
          : l == 21 ? A.gamma
          : l == 22 ? 4.0
          : l == 23 ? 2.0
          : l == 19 ? A.i6h[0]
          : l == 20 ? A.i3h2[0]
                    : ih;
      y1 = (l == 22 || l == 23) ? ih : 1.0;
      y2 = l == 22 ? ih : 1.0;
    }
    const double d = ((x * y1) * y2) * y3;
    const T dt = T(d);
    switch (o == 0 || l < 16 ? l : 31) {
      case 0: sc.taut[o] = dt; sc.comb[o] = !is_zero_bits(A.cA[o]); break;
      case 1: sc.mu[o] = d; break;
      case 2: sc.nu[o] = d; break;
      case 3: sc.m2[o] = dt; break;
      case 4: sc.n2[o] = dt; break;
      case 5: sc.k6[o] = dt; break;
      case 6: sc.q6[o] = dt; break;
      case 7: sc.cAt[o] = dt; break;
      case 8: sc.cFt[o] = dt; break;
      case 16: sc.umin = dt; break;
      case 17: sc.umax = dt; break;
      case 18: sc.ih = dt; break;
      case 19: sc.i6h = dt; break;
      case 20: sc.i3h2 = dt; break;
      case 21: sc.g = dt; break;
      case 22: sc.i4hh = dt; break;
      case 23: sc.i2h = dt; break;
      default: break;
    }
  }
  __syncthreads();
  const T umin = sc.umin, umax = sc.umax;
  const bool blend = A.blend != 0;
  const bool ext = A.blend == 2;
  const bool nodc = A.nodc != 0;
  const bool bounded = A.bc != AF_BC_PERIODIC;
  const int poff = bounded ? 1 : 0;   // point u_{j+1/2} is stored at index j + poff

  for (int k = tid; k < BX; k += NT) {
    // rounded toward the nearer bound, as the 2D stages round the averages (integer ops)
    sU[k] = to_stencil_nb<T>(cell1d(A, i0 - H + k, H), m.umid);
    sP[k] = T(point1d(A, i0 - H + k, H));
  }
  __syncthreads();
  for (int b = tid; b < BX; b += NT) {
    const T u = sU[b];
    fU[b] = flux<FLUX, T>(m, XD, u);
    aU[b] = apot<T>(m, u);
    const T p = sP[b];
    fP[b] = flux<FLUX, T>(m, XD, p);
    if constexpr (FLUX != FLUX_BURGERS) dP[b] = dflux_abs<FLUX, T>(m, XD, p);
    aP[b] = nodc ? kappa_fn<T>(m, p) : apot<T>(m, p);
    if (b >= 1) {
      const T c = (T(6) * u - sP[b - 1] - p) * T(0.25);
      sC[b] = c;
      fC[b] = flux<FLUX, T>(m, XD, c);
      if constexpr (FLUX != FLUX_BURGERS) dC[b] = dflux_abs<FLUX, T>(m, XD, c);
      aC[b] = nodc ? kappa_fn<T>(m, c) : apot<T>(m, c);
    }
    if (blend && !ext && b >= 1 && b < BX - 1) {
      const T um = sU[b - 1], up = sU[b + 1];
      sTC[b] = tabs(um - T(2) * u + up) / (tabs(um) + T(2) * tabs(u) + tabs(up) + T(1e-13));
    }
  }
  __syncthreads();
  const T ih = sc.ih, i6h = sc.i6h, i3h2 = sc.i3h2;
  // points updated by this thread: its own u_{i+1/2} and, in CTA 0 of a bounded
  // interval, thread 0 also the left end point u_{-1/2} (held at the boundary value
  // when the end is Dirichlet)
  const bool extra = bounded && blockIdx.x == 0 && tid == 0;
  const int nq = extra ? 2 : 1;
  const int bq[2] = {H + tid, H - 1};
  // high-order point residual
  T rH[2] = {T(0), T(0)};
  for (int q = 0; q < nq; ++q) {
    const int b = bq[q];
    // max |f'| over the line; for Burgers |2p| max |z| (the same value: rounding is
    // monotone), which spares two FP64 multiplies per cell
    T alpha;
    if constexpr (FLUX == FLUX_BURGERS)
      alpha = tabs(T(2) * par<T>(m.fp, m.fpf, 0)) *
              tmax(tmax(tmax(tabs(sP[b - 1]), tabs(sC[b])), tmax(tabs(sC[b + 1]), tabs(sP[b + 1]))), tabs(sP[b]));
    else
      alpha = tmax(tmax(tmax(dP[b - 1], dC[b]), tmax(dC[b + 1], dP[b + 1])), dP[b]);
    if (!nodc) {
      rH[q] = line_res<T>(sP[b - 1], sC[b], sP[b], sC[b + 1], sP[b + 1], fP[b - 1], fC[b], fC[b + 1], fP[b + 1],
                          alpha, aP[b - 1], aC[b], aP[b], aC[b + 1], aP[b + 1], i6h, i3h2);
    } else {
      const T z[5] = {sP[b - 1], sC[b], sP[b], sC[b + 1], sP[b + 1]};
      const T k[5] = {aP[b - 1], aC[b], aP[b], aC[b + 1], aP[b + 1]};
      rH[q] = line_res<T>(z[0], z[1], z[2], z[3], z[4], fP[b - 1], fC[b], fC[b + 1], fP[b + 1], alpha, T(0), T(0),
                          T(0), T(0), T(0), i6h, i3h2) +
              nodc_d2<T>(z, k) * (T(3) * i3h2);
    }
  }
  for (int b = H - 2 + tid; b <= H + TX; b += NT) {
    const T ul = sU[b], ur = sU[b + 1];
    // LLF flux (f_l + f_r - alpha (u_r - u_l)) / 2: one multiply-add and one multiply
    const T fl = T(0.5) * ((fU[b] + fU[b + 1]) - alpha_interval<FLUX, T>(m, XD, ul, ur) * (ur - ul));
    if (!nodc) {
      if (b >= H - 1 && b < H + TX) sFH[b] = fP[b];
      if (b >= H - 1) sAH[b] = (T(8) * aC[b] - aP[b - 1] - aP[b]) * T(1.0 / 6.0);
      sFL[b] = fl;
    } else {
      // total face fluxes: f(P) - kappa(P) D_c(u) and F^L - (a(ub_{i+1}) - a(ub_i)) / dx
      if (b >= H - 1 && b < H + TX)
        sFH[b] = fP[b] - aP[b] * (((sP[b - 1] - sP[b + 1]) + T(8) * (sC[b + 1] - sC[b])) * i6h);
      sFL[b] = fl - (aU[b + 1] - aU[b]) * ih;
    }
  }
  if (blend) {
    for (int b = H - 1 + tid; b <= H + TX; b += NT) {
      sS[b] = ext ? T(A.s_ext[wrapi(i0 - H + b, nx)]) : (sTC[b - 1] + T(4) * sTC[b] + sTC[b + 1]) * T(1.0 / 6.0);
    }
  }
  __syncthreads();
  T rP[2] = {rH[0], rH[1]};
  if (blend) {
    const T g = sc.g;
    for (int b = H - 1 + tid; b <= H + TX; b += NT) {
      sTD[b] = exp(-g * sS[b]);
      if (b < H + TX) sTC[b] = exp(-g * (T(0.5) * (sS[b] + sS[b + 1])));
    }
    __syncthreads();
    for (int b = H - 1 + tid; b <= H + TX; b += NT) {
      if (b < H + TX) sFH[b] = sTC[b] * sFH[b] + (T(1) - sTC[b]) * sFL[b];
      sAH[b] = sTD[b] * sAH[b] + (T(1) - sTD[b]) * aU[b];
    }
    for (int q = 0; q < nq; ++q) {
      const int b = bq[q];
      const T zm = sU[b], z0 = sP[b], zp = sU[b + 1];
      const T Fr = T(0.5) * (fP[b] + fU[b + 1]) - T(0.5) * alpha_interval<FLUX, T>(m, XD, z0, zp) * (zp - z0);
      const T Fl = T(0.5) * (fU[b] + fP[b]) - T(0.5) * alpha_interval<FLUX, T>(m, XD, zm, z0) * (z0 - zm);
      const T RL = (aU[b + 1] - T(2) * aP[b] + aU[b]) * sc.i4hh - (Fr - Fl) * sc.i2h;
      rP[q] = sTC[b] * rH[q] + (T(1) - sTC[b]) * RL;
    }
    __syncthreads();
  }
  const int gi = i0 + tid;
  const bool own = gi < nx;
  T* Flim = A.limiter ? sFlim : sFH;
  T* Alim = A.limiter ? sAlim : sAH;
  for (int o = 0; o < A.nout; ++o) {
    const double mu = sc.mu[o], nu = sc.nu[o];
    if (A.limiter) {
      const T m2 = sc.m2[o], n2 = sc.n2[o];
      for (int b = H - 2 + tid; b <= H + TX + 1; b += NT) {
        const T u = sU[b], f = fU[b], a = aU[b];
        if (!nodc) {
          if (b <= H + TX) sULp[b] = u - m2 * (sFL[b] - f) + n2 * (aU[b + 1] - a);
          if (b >= H - 1) sULm[b] = u - m2 * (f - sFL[b - 1]) - n2 * (a - aU[b - 1]);
        } else {
          // sFL already holds the total low-order face flux (diffusion included)
          if (b <= H + TX) sULp[b] = u - m2 * (sFL[b] - f);
          if (b >= H - 1) sULm[b] = u - m2 * (f - sFL[b - 1]);
        }
      }
      __syncthreads();
      // face factor 2 * parts (6 with diffusion, 2 without); the total face flux of the
      // form without double conservation takes factor 2 (the average is the mean of
      // u^{L,+} and u^{L,-}, one face correction each)
      const T k6 = sc.k6[o], q6 = sc.q6[o];
      for (int b = H - 1 + tid; b <= H + TX; b += NT) {
        if (b < H + TX) {
          const T fh = sFH[b], fl = sFL[b], dF = fh - fl;
          const T zp = sULp[b], zm = sULm[b + 1];
          const T t = tmin(theta_fn<T>(zp, zp - k6 * dF, umin, umax), theta_fn<T>(zm, zm + k6 * dF, umin, umax));
          sFlim[b] = is_one(t) ? fh : fl + t * dF;
        }
        if (!nodc) {
          const T ah = sAH[b], al = aU[b], d = q6 * (ah - al);
          const T t = tmin(tmin(theta_fn<T>(sULp[b - 1], sULp[b - 1] + d, umin, umax),
                                theta_fn<T>(sULp[b], sULp[b] - d, umin, umax)),
                           tmin(theta_fn<T>(sULm[b], sULm[b] - d, umin, umax),
                                theta_fn<T>(sULm[b + 1], sULm[b + 1] + d, umin, umax)));
          sAlim[b] = is_one(t) ? ah : al + t * (ah - al);
        }
      }
      __syncthreads();
    }
    if (own) {
      const int b = H + tid;
      const size_t g = (size_t)gi;
      double ubfe = A.ub[g] - mu * (d_of(Flim[b]) - d_of(Flim[b - 1]));
      if (!nodc) ubfe += nu * ((d_of(Alim[b + 1]) - 2.0 * d_of(Alim[b])) + d_of(Alim[b - 1]));
      double ubo = sc.comb[o] ? rk_comb(A.cA[o], A.Aub[o][g], A.cF[o], ubfe) : rk_scale(A.cF[o], ubfe);
      if (A.limiter && A.sg[o]) ubo = safeguard<double>(ubo, m.umin, m.umax, A.tol, A.stats, true);
      A.Oub[o][g] = ubo;
    }
    for (int q = 0; q < nq; ++q) {
      const int gj = q == 0 ? gi : -1;   // point index j of u_{j+1/2}
      if (gj >= nx) continue;
      const size_t g = (size_t)(gj + poff);
      PT po;
      if (A.bc == AF_BC_DIRICHLET && (gj == -1 || gj == nx - 1)) {
        po = PT(gj == -1 ? A.bc_left : A.bc_right);
      } else {
        T p = sP[bq[q]] + sc.taut[o] * rP[q];
        if (A.limiter) p = tmin(tmax(p, umin), umax);
        po = sc.comb[o] ? PT(rk_comb(sc.cAt[o], T(A.AV[o][g]), sc.cFt[o], p)) : PT(rk_scale(sc.cFt[o], p));
        if (A.limiter && A.sg[o]) po = safeguard<PT>(po, PT(umin), PT(umax), A.tol, A.stats);
      }
      A.OV[o][g] = po;
    }
    if (o + 1 < A.nout) __syncthreads();
  }
}

}  // namespace af
