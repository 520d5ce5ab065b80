// Fused 2D stage kernel of the compact fourth-order doubly conservative active flux
// method with monolithic convex MPP limiting (arXiv 2510.11527, Sections 4 and 5.2,
// d = 2).
//
// One launch performs, for every cell of a periodic nx x ny mesh, one or two limited
// forward-Euler evaluations FE(u, tau_k) of the same input state followed by the
// Shu-Osher combination out_k = cA_k * A_k + cF_k * FE(u, tau_k), the point-value
// projection and the post-stage safeguard. Each CTA owns a TX x TY tile and stages a
// halo box of +-H cells (H = 2; 3 with the smoothness blend) of all four DoF arrays in
// shared memory; every derived quantity is evaluated once per box location, kept in
// shared memory, and consumed by the neighbouring threads:
//
//   P0  load ub, V, X, Y (periodic wrap)
//   P1  centre values c (Simpson recovery, Section 4) and pointwise f_l, |f_l'|, a
//   P2  high-order point residuals (registers), Simpson face fluxes F^H_l, cell
//       potentials A^H_l, LLF fluxes F^L_l
//   P2b/P2c (blend) smoothness s_l, weights theta^{c,s}, theta^{d,s}; blended F, A, R
//   P3  directional low-order states u^{L,+-}_l (factor 2d = 4)
//   P4  limiter parameters theta^c (faces; factor 3*2d = 12, or 2d = 4 without a
//       diffusion term), theta^d (cells; factor 12)
//   P5  limited cell-average update (eq. multid_limited_average), point update and
//       projection, RK combination, safeguard, store.
//
// Face arrays are indexed by the box position of the face's left (x) / lower (y) cell:
// F_1(b) lives on the x-face between b and b+1, F_2(b) on the y-face between b and
// b+BX. Both tiles adjacent to a face compute it with the same instructions from the
// same values, so conservation and double conservation hold bit for bit.
#pragma once
#include <type_traits>

#include "af_model.cuh"

namespace af {

template <class PT>
struct StageArgs2D {
  int nx, ny;
  double inv_h1, inv_h2;             // 1/dx, 1/dy
  double i6h[2], i3h2[2];            // 1/(6 h_l), (1/h_l^2)/3: line scales, formed on the host
  float i6hf[2], i3h2f[2];           // the same rounded to FP32
  const double* ub;                  // FE input (read with halo)
  const PT* V;
  const PT* X;
  const PT* Y;
  int nout;                          // 1 or 2 limited FE evaluations of the same input
  double tcoef[2];                   // tau_k = tcoef_k * (*dt)
  double cA[2], cF[2];               // out_k = cA_k * A_k + cF_k * FE(u, tau_k)
  const double* Aub[2];
  const PT* AV[2];
  const PT* AX[2];
  const PT* AY[2];
  double* Oub[2];
  PT* OV[2];
  PT* OX[2];
  PT* OY[2];
  const double* dt;                  // device scalar
  const double* s_ext;               // external per-cell indicator (blend external)
  const float* sb[2];                // s_1, s_2 per cell (column-marching FP32 blend)
  int limiter;
  int blend;                         // 0 off, 1 smoothness indicator, 2 external indicator
  int blend_external;
  int sg[2];                         // per output: apply the post-stage safeguard
  double gamma;
  double tol;                        // safeguard tolerance (absolute)
  DevStats* stats;
  // 1D only: ends of the interval (AF_BC_*) and the diffusion form (AF_FORM_*). On a
  // bounded interval the point arrays hold nx+1 values, index k <-> u(x0 + k dx).
  int bc;
  double bc_left, bc_right;
  int nodc;
};

// Per flux kind: which pointwise quantities are stored per point and per cell average
// (a is always last). Buckley-Leverett stores f1, f2, |f1'|, |f2'|, a in FP64; in FP32
// f2 = f1 (1 - g (1-u)^2) is formed at each use instead (3 FP32 operations), which keeps
// the blended FP32 tile at 3 CTAs per SM.
template <int FLUX, class T> struct PointStore {
  static constexpr bool F2 = false;
  static constexpr int NQ = FLUX == FLUX_BURGERS ? 2 : 1, NQU = NQ, DOFF = 1;
};
template <class T> struct PointStore<FLUX_BL, T> {
  static constexpr bool F2 = sizeof(T) == 8;   // f2 stored
  static constexpr int DOFF = F2 ? 2 : 1;      // index of |f1'| (|f2'| follows)
  static constexpr int NQ = DOFF + 3, NQU = NQ;
};

template <int FLUX, class T, bool BLEND, int TX_ = 32, int TY_ = 8>
struct Tile2D {
  static constexpr int TX = TX_, TY = TY_, NT = TX * TY;
  static_assert(NT == 256, "stage tiles use 256 threads");
  static constexpr int H = BLEND ? 3 : 2;
  static constexpr int BX = TX + 2 * H, BY = TY + 2 * H, BN = BX * BY;
  static constexpr int NQ = PointStore<FLUX, T>::NQ, NQU = PointStore<FLUX, T>::NQU;
  // shared arrays (all of length BN, element type T)
  static constexpr int A_U = 0, A_V = 1, A_X = 2, A_Y = 3, A_C = 4;
  static constexpr int A_QU = 5;                       // NQU arrays: funcs at ub
  static constexpr int A_FH1 = A_QU + NQU, A_FH2 = A_FH1 + 1, A_AH1 = A_FH1 + 2, A_AH2 = A_FH1 + 3;
  static constexpr int A_FL1 = A_FH1 + 4, A_FL2 = A_FH1 + 5;
  static constexpr int A_BL0 = A_FH1 + 6;              // blend: s1 (then td1), s2 (then td2), tc1, tc2
  static constexpr int NBL = BLEND ? 4 : 0;
  static constexpr int A_Q = A_BL0 + NBL;              // 4 point types x NQ, aliased later
  static constexpr int NQREG = (4 * NQ > 8 ? 4 * NQ : 8);
  static constexpr int NARR = A_Q + NQREG;
  static constexpr size_t SMEM = (size_t)NARR * BN * sizeof(T);
  // aliases inside the Q region (valid after P2)
  static constexpr int A_ULP1 = A_Q, A_ULM1 = A_Q + 1, A_ULP2 = A_Q + 2, A_ULM2 = A_Q + 3;
  static constexpr int A_FLIM1 = A_Q + 4, A_FLIM2 = A_Q + 5, A_ALIM1 = A_Q + 6, A_ALIM2 = A_Q + 7;
};

// Scalars uniform over a tile (grid spacings, dt-dependent limiter factors, RK weights)
template <class T>
struct TileScal {
  double tau[2], mu1[2], mu2[2], nu1[2], nu2[2];
  float mu1f[2], mu2f[2], nu1f[2], nu2f[2];
  T taut[2], m4_1[2], n4_1[2], m4_2[2], n4_2[2], k1[2], k2[2], q1[2], q2[2], cAt[2], cFt[2];
  T umin, umax, i6h1, i6h2, i3h21, i3h22, i2h1, i2h2, i4h21, i4h22, g;
};

template <int NT, class F>
__device__ __forceinline__ void for_rect(int x0, int x1, int y0, int y1, F&& f) {
  const int w = x1 - x0, n = w * (y1 - y0);
  for (int k = threadIdx.x; k < n; k += NT) f(x0 + k % w, y0 + k / w);
}

// A rectangle [X0, X1) x [Y0, Y1) of box positions with the body applied to each.
template <int X0_, int X1_, int Y0_, int Y1_, class F>
struct Seg {
  static constexpr int X0 = X0_, Y0 = Y0_, W = X1_ - X0_, N = (X1_ - X0_) * (Y1_ - Y0_);
  F f;
};
template <int X0, int X1, int Y0, int Y1, class F>
__device__ __forceinline__ Seg<X0, X1, Y0, Y1, F> seg(F f) {
  return Seg<X0, X1, Y0, Y1, F>{f};
}
template <int NT, class S>
__device__ __forceinline__ void for_seg(const S& s) {
  for (int k = threadIdx.x; k < S::N; k += NT) s.f(S::X0 + k % S::W, S::Y0 + k / S::W);
}
// The independent loops of one phase, one after the other. (Merging them into one
// balanced iteration space was measured slower on GB300: the per-item dispatch costs
// more branches than the shorter barrier waits save.)
template <int NT, class... Ss>
__device__ __forceinline__ void for_segs(const Ss&... ss) {
  (for_seg<NT>(ss), ...);
}

// periodic index; the halo never reaches further than one period except on meshes
// smaller than the halo, which take the modulo path
__device__ __forceinline__ int wrapi(int i, int n) {
  if (i < 0) {
    i += n;
    if (i < 0) {
      i %= n;
      if (i < 0) i += n;
    }
  } else if (i >= n) {
    i -= n;
    if (i >= n) i %= n;
  }
  return i;
}

// Residual of one 5-point line (spacing h/2; points 0..4 at offsets -h..+h, point 2
// is updated), algebraically identical to the FVS-LLF split with the biased D+/D-
// operators and the compact second derivative of a:
//   R = -[(f0 - f4) + 8 (f3 - f1) + alpha ((z0 + z4) - 4 (z1 + z3) + 6 z2)] / (6h)
//       + [16 (a1 + a3) - (a0 + a4) - 30 a2] / (3h^2)
template <class T>
__device__ __forceinline__ T line_res(T z0, T z1, T z2, T z3, T z4, T f0, T f1, T f3, T f4, T alpha, T a0,
                                      T a1, T a2, T a3, T a4, T i6h, T i3h2) {
  T cf = (f0 - f4) + T(8) * (f3 - f1);
  T dz = (z0 + z4) - T(4) * (z1 + z3) + T(6) * z2;
  T da = T(16) * (a1 + a3) - (a0 + a4) - T(30) * a2;
  return da * i3h2 - (cf + alpha * dz) * i6h;
}

// Padded index of a 2D rectangle with outflow ends (n cells in this direction, padded
// index I = cell index + 1): the evenly reflected source of a cell-type entry (ub; X in
// y; Y in x) and of a face-type entry (V; X in x; Y in y). Indices further out than any
// owned output reads are clamped first, so every load stays inside the arrays (n >= 4).
__device__ __forceinline__ int rect_cell(int I, int n) {
  I = I < -3 ? -3 : (I > n + 4 ? n + 4 : I);
  return I < 1 ? 1 - I : (I > n ? 2 * n + 1 - I : I);
}
__device__ __forceinline__ int rect_face(int I, int n) {
  I = I < -3 ? -3 : (I > n + 4 ? n + 4 : I);
  return I < 0 ? -I : (I > n ? 2 * n - I : I);
}

// One TX x TY tile with origin (i0, j0) of one mesh: all phases P0-P5. Every thread of
// the CTA must call it (it contains __syncthreads); smem_raw holds Tile2D::SMEM bytes.
// PAIRED enables the paired vector loads of interior halo boxes (P0). RECT selects a 2D
// rectangle with outflow ends in its padded layout (reflected ghost loads, masked stores);
// periodic meshes compile without any of it.
template <int FLUX, class T, class PT, bool BLEND, int TX_ = 32, int TY_ = 8, bool PAIRED = true, bool RECT = false>
__device__ __forceinline__ void stage_tile(const DevModel& m, const StageArgs2D<PT>& A, const int i0, const int j0,
                                           unsigned char* smem_raw) {
  using L = Tile2D<FLUX, T, BLEND, TX_, TY_>;
  using PS = PointStore<FLUX, T>;
  constexpr int TX = L::TX, TY = L::TY, NT = L::NT, H = L::H, BX = L::BX, BY = L::BY, BN = L::BN;
  constexpr int NQ = L::NQ;
  T* S = reinterpret_cast<T*>(smem_raw);
  auto arr = [&](int a) -> T* { return S + (size_t)a * BN; };
  T* sU = arr(L::A_U);
  T* sZ[4] = {arr(L::A_V), arr(L::A_X), arr(L::A_Y), arr(L::A_C)};   // V, X, Y, centre
  T* sQU = arr(L::A_QU);
  T* sQ = arr(L::A_Q);
  auto Q = [&](int type, int k) -> T* { return sQ + (size_t)(type * NQ + k) * BN; };

  const double dtv = *A.dt;
  if (is_zero_bits(dtv)) return;
  const int nx = A.nx, ny = A.ny;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;

  // tile-uniform scalars, formed once in FP64 and rounded. GB300's FP64 unit takes as
  // long for a warp instruction with one active lane as with 32, so the lanes of warp o
  // form output o's values at once and the upper lanes of warp 0 the mesh's: lane l
  // evaluates fl(fl(fl(x y1) y2) y3) with the factors of its value's formula (a factor 1
  // is exact, so each value is rounded as its formula is; the divided line scales come
  // from the host), then only the stores differ between lanes.
  __shared__ TileScal<T> sc;
  if ((tid >> 5) < A.nout) {
    const int o = tid >> 5, l = tid & 31;
    const double tau = A.tcoef[o] * dtv;
    // direction: the second of each pair of lanes 1 .. 14 (odd, even), 18 .. 25 (even, odd)
    const bool second = l < 16 ? !(l & 1) : (l & 1);
    const double ih = second ? A.inv_h2 : A.inv_h1;
    double x = tau, y1 = 1.0, y2 = 1.0, y3 = 1.0;
    if (l >= 1 && l < 15) {
      // 1, 2: mu_l; 3, 4: nu_l; 5, 6: 4 mu_l; 7, 8: 4 nu_l; 9, 10: 4 P mu_l; 11, 12: 12 nu_l
      const int kind = (l - 1) >> 1;
      y1 = ih;
      y2 = (kind & 1) ? ih : (kind == 2 ? 4.0 : (kind == 4 ? double(4 * m.lim_parts) : 1.0));
      y3 = kind == 3 ? 4.0 : (kind == 5 ? 12.0 : 1.0);
      if (kind == 6) {   // lanes 13, 14: cA, cF of the output
        x = l == 13 ? A.cA[o] : A.cF[o];
        y1 = y2 = 1.0;
      }
    } else if (l >= 16) {
      // 16, 17: u_min, u_max; 18, 19: 2 / h_l; 20, 21: (4 / h_l) / h_l; 22, 23: 1 / (6 h_l);
      // 24, 25: (1 / h_l / h_l) / 3; 26: gamma
      x = l == 16 ? m.umin : (l == 17 ? m.umax : (l == 26 ? A.gamma : 1.0));
      if (l >= 18 && l < 26) {
        const int kind = (l - 18) >> 1;
        x = kind == 0 ? 2.0 : (kind == 1 ? 4.0 : (kind == 2 ? (second ? A.i6h[1] : A.i6h[0])
                                                                : (second ? A.i3h2[1] : A.i3h2[0])));
        y1 = kind < 2 ? ih : 1.0;
        y2 = kind == 1 ? ih : 1.0;
      }
    }
    const double d = ((x * y1) * y2) * y3;
    const T dt = T(d);
    const float df = (float)d;
    switch (o == 0 || l < 16 ? l : 31) {
      case 0: sc.tau[o] = d; sc.taut[o] = dt; break;
      case 1: sc.mu1[o] = d; sc.mu1f[o] = df; break;
      case 2: sc.mu2[o] = d; sc.mu2f[o] = df; break;
      case 3: sc.nu1[o] = d; sc.nu1f[o] = df; break;
      case 4: sc.nu2[o] = d; sc.nu2f[o] = df; break;
      case 5: sc.m4_1[o] = dt; break;
      case 6: sc.m4_2[o] = dt; break;
      case 7: sc.n4_1[o] = dt; break;
      case 8: sc.n4_2[o] = dt; break;
      case 9: sc.k1[o] = dt; break;
      case 10: sc.k2[o] = dt; break;
      case 11: sc.q1[o] = dt; break;
      case 12: sc.q2[o] = dt; break;
      case 13: sc.cAt[o] = dt; break;
      case 14: sc.cFt[o] = dt; break;
      case 16: sc.umin = dt; break;
      case 17: sc.umax = dt; break;
      case 18: sc.i2h1 = dt; break;
      case 19: sc.i2h2 = dt; break;
      case 20: sc.i4h21 = dt; break;
      case 21: sc.i4h22 = dt; break;
      case 22: sc.i6h1 = dt; break;
      case 23: sc.i6h2 = dt; break;
      case 24: sc.i3h21 = dt; break;
      case 25: sc.i3h22 = dt; break;
      case 26: sc.g = dt; break;
      default: break;
    }
  }

  // ---- P0: load the halo box --------------------------------------------------------
  // Tiles whose halo box lies inside an even-width mesh load the box as aligned pairs
  // (8- or 16-byte vector loads; rows start at the even column i0 - 2); other tiles
  // (periodic wrap, odd widths, the +-3 blend halo, the sides of a rectangle with
  // outflow ends) load element by element. In both, all loads of a thread are issued
  // before its first store, so their latencies overlap. A rectangle (A.bc) is tiled in
  // its padded layout: a paired box never reaches row or column 0 or beyond the last.
  bool paired = false;
  if constexpr (H == 2 && PAIRED) {
    paired = (nx % 2 == 0) && i0 - H >= 0 && i0 + TX + H <= nx && j0 - H >= 0 && j0 + TY + H <= ny;
  }
  if (paired) {
    using P2 = std::conditional_t<sizeof(PT) == 4, float2, double2>;
    constexpr int PW = BX / 2, NV = PW * BY, NPV = (NV + NT - 1) / NT;
    double2 ldU[NPV];
    P2 ldV[NPV], ldX[NPV], ldY[NPV];
#pragma unroll
    for (int it = 0; it < NPV; ++it) {
      const int k = tid + it * NT;
      if (k < NV) {
        const size_t g = (size_t)(j0 - H + k / PW) * nx + (i0 - H + 2 * (k % PW));
        ldU[it] = *reinterpret_cast<const double2*>(A.ub + g);
        ldV[it] = *reinterpret_cast<const P2*>(A.V + g);
        ldX[it] = *reinterpret_cast<const P2*>(A.X + g);
        ldY[it] = *reinterpret_cast<const P2*>(A.Y + g);
      }
    }
#pragma unroll
    for (int it = 0; it < NPV; ++it) {
      const int k = tid + it * NT;
      if (k < NV) {
        const int b = (k / PW) * BX + 2 * (k % PW);
        sU[b] = to_stencil_nb<T>(ldU[it].x, m.umid);
        sU[b + 1] = to_stencil_nb<T>(ldU[it].y, m.umid);
        sZ[0][b] = T(ldV[it].x);
        sZ[0][b + 1] = T(ldV[it].y);
        sZ[1][b] = T(ldX[it].x);
        sZ[1][b + 1] = T(ldX[it].y);
        sZ[2][b] = T(ldY[it].x);
        sZ[2][b + 1] = T(ldY[it].y);
      }
    }
  } else {
    constexpr int NP0 = (BN + NT - 1) / NT;
    double ldU[NP0];
    PT ldV[NP0], ldX[NP0], ldY[NP0];
#pragma unroll
    for (int it = 0; it < NP0; ++it) {
      const int k = tid + it * NT;
      if (k < BN) {
        const int bx = k % BX, by = k / BX;
        if constexpr (RECT) {
          // cell-type and face-type source indices in the padded layout
          const int ci = rect_cell(i0 - H + bx, nx - 1), fi = rect_face(i0 - H + bx, nx - 1);
          const int cj = rect_cell(j0 - H + by, ny - 1), fj = rect_face(j0 - H + by, ny - 1);
          ldU[it] = A.ub[(size_t)cj * nx + ci];
          ldV[it] = A.V[(size_t)fj * nx + fi];
          ldX[it] = A.X[(size_t)cj * nx + fi];
          ldY[it] = A.Y[(size_t)fj * nx + ci];
        } else {
          const int gi = wrapi(i0 - H + bx, nx), gj = wrapi(j0 - H + by, ny);
          const size_t g = (size_t)gj * nx + gi;
          ldU[it] = A.ub[g];
          ldV[it] = A.V[g];
          ldX[it] = A.X[g];
          ldY[it] = A.Y[g];
        }
      }
    }
#pragma unroll
    for (int it = 0; it < NP0; ++it) {
      const int k = tid + it * NT;
      if (k < BN) {
        sU[k] = to_stencil_nb<T>(ldU[it], m.umid);
        sZ[0][k] = T(ldV[it]);
        sZ[1][k] = T(ldX[it]);
        sZ[2][k] = T(ldY[it]);
      }
    }
  }
  __syncthreads();
  const T umin = sc.umin, umax = sc.umax;

  // ---- P1: centres and pointwise nonlinearities ----------------------------------------
  auto eval_point = [&](int type, int b) {
    const T z = sZ[type][b];
    if constexpr (FLUX == FLUX_BURGERS) {
      Q(type, 0)[b] = flux<FLUX, T>(m, 0, z);
    } else if constexpr (FLUX == FLUX_BL) {
      const BLVals<T> r = bl_eval<T>(m, z);
      Q(type, 0)[b] = r.f[0];
      if constexpr (PS::F2) Q(type, 1)[b] = r.f[1];
      Q(type, PS::DOFF)[b] = r.d[0];
      Q(type, PS::DOFF + 1)[b] = r.d[1];
    }
    Q(type, NQ - 1)[b] = apot<T>(m, z);
  };
  T* sS1 = nullptr;
  T* sS2 = nullptr;
  T* sTC1 = nullptr;
  T* sTC2 = nullptr;
  T* sTD1 = nullptr;
  T* sTD2 = nullptr;
  if constexpr (BLEND) {
    sS1 = arr(L::A_BL0);
    sS2 = arr(L::A_BL0 + 1);
    sTC1 = arr(L::A_BL0 + 2);
    sTC2 = arr(L::A_BL0 + 3);
    sTD1 = sS1;   // theta^{d,s} replaces s in place once theta^{c,s} is formed
    sTD2 = sS2;
  }
  const auto p1_qu = seg<0, BX, 0, BY>([&](int bx, int by) {
    const int k = by * BX + bx;
    const T u = sU[k];
    if constexpr (FLUX == FLUX_BURGERS) {
      sQU[k] = flux<FLUX, T>(m, 0, u);
    } else if constexpr (FLUX == FLUX_BL) {
      const BLVals<T> r = bl_eval<T>(m, u);
      sQU[k] = r.f[0];
      if constexpr (PS::F2) sQU[BN + k] = r.f[1];
      sQU[PS::DOFF * BN + k] = r.d[0];
      sQU[(PS::DOFF + 1) * BN + k] = r.d[1];
    }
    sQU[(L::NQU - 1) * BN + k] = apot<T>(m, u);
  });
  const auto p1_pts = seg<H - 2, H + TX + 1, H - 2, H + TY + 1>([&](int bx, int by) {
    const int b = by * BX + bx;
    eval_point(0, b);
    eval_point(1, b);
    eval_point(2, b);
  });
  const auto p1_ctr = seg<H - 1, H + TX + 1, H - 1, H + TY + 1>([&](int bx, int by) {
    const int b = by * BX + bx;
    const T* V = sZ[0];
    const T* X = sZ[1];
    const T* Y = sZ[2];
    // z_ij = [36 zbar - 4 (X_{i-1,j} + X_ij + Y_{i,j-1} + Y_ij) - (four corners)] / 16
    const T c = (T(36) * sU[b] - T(4) * ((X[b - 1] + X[b]) + (Y[b - BX] + Y[b])) -
                 ((V[b - BX - 1] + V[b - BX]) + (V[b - 1] + V[b]))) * T(0.0625);
    sZ[3][b] = c;
    eval_point(3, b);
  });
  if constexpr (BLEND) {
    if (!A.blend_external) {
      // s~_l = |u_- - 2u + u_+| / (|u_-| + 2|u| + |u_+| + 1e-13) (Section 5.1.3); kept
      // temporarily in the TC arrays
      for_segs<NT>(p1_qu, p1_pts, p1_ctr, seg<1, BX - 1, 1, BY - 1>([&](int bx, int by) {
                     const int b = by * BX + bx;
                     const T u = sU[b];
                     const T au2 = T(2) * tabs(u);
                     sTC1[b] = tabs(sU[b - 1] - T(2) * u + sU[b + 1]) /
                               (tabs(sU[b - 1]) + au2 + tabs(sU[b + 1]) + T(1e-13));
                     sTC2[b] = tabs(sU[b - BX] - T(2) * u + sU[b + BX]) /
                               (tabs(sU[b - BX]) + au2 + tabs(sU[b + BX]) + T(1e-13));
                   }));
    } else {
      for_segs<NT>(p1_qu, p1_pts, p1_ctr);
    }
  } else {
    for_segs<NT>(p1_qu, p1_pts, p1_ctr);
  }
  __syncthreads();

  // ---- P2: high-order residuals, Simpson fluxes, DC potentials, LLF fluxes -------------
  const T i6h1 = sc.i6h1, i6h2 = sc.i6h2;
  const T i3h21 = sc.i3h21, i3h22 = sc.i3h22;
  // value / flux / |f'| / a of a stored point of the given type, direction dir
  auto Fz = [&](int type, int b, int dir) -> T {
    if constexpr (FLUX == FLUX_BURGERS) return Q(type, 0)[b];
    else if constexpr (FLUX == FLUX_BL) {
      if constexpr (PS::F2) return Q(type, dir)[b];
      else return dir == 0 ? Q(type, 0)[b] : bl_f2<T>(m, sZ[type][b], Q(type, 0)[b]);
    }
    else return flux<FLUX, T>(m, dir, sZ[type][b]);
  };
  auto Az = [&](int type, int b) -> T { return Q(type, NQ - 1)[b]; };
  // one 5-point line given (type, box index) of its points
  auto line = [&](int dir, int t0, int b0, int t1, int b1, int t2, int b2, int t3, int b3, int t4, int b4) -> T {
    const T z0 = sZ[t0][b0], z1 = sZ[t1][b1], z2 = sZ[t2][b2], z3 = sZ[t3][b3], z4 = sZ[t4][b4];
    T alpha;
    if constexpr (FLUX == FLUX_BURGERS) {
      // |2 p0| rounded to T equals |2 T(p0)| (scaling by 2 is exact)
      alpha = tabs(T(2) * par<T>(m.fp, m.fpf, 0)) *
              tmax(tmax(tmax(tabs(z0), tabs(z1)), tmax(tabs(z3), tabs(z4))), tabs(z2));
    } else if constexpr (FLUX == FLUX_BL) {
      const int k = PS::DOFF + dir;
      alpha = tmax(tmax(tmax(Q(t0, k)[b0], Q(t1, k)[b1]), tmax(Q(t3, k)[b3], Q(t4, k)[b4])), Q(t2, k)[b2]);
    } else if constexpr (FLUX == FLUX_LINEAR) {
      alpha = tabs(T(dir == 0 ? m.fp[0] : m.fp[1]));
    } else {
      alpha = T(0);
    }
    const T i6h = dir == 0 ? i6h1 : i6h2, i3h2 = dir == 0 ? i3h21 : i3h22;
    return line_res<T>(z0, z1, z2, z3, z4, Fz(t0, b0, dir), Fz(t1, b1, dir), Fz(t3, b3, dir), Fz(t4, b4, dir), alpha,
                       Az(t0, b0), Az(t1, b1), Az(t2, b2), Az(t3, b3), Az(t4, b4), i6h, i3h2);
  };
  constexpr int tV = 0, tX = 1, tY = 2, tC = 3;
  const int bo = (ty + H) * BX + (tx + H);   // own box index
  T rV1, rV2, rX1, rX2, rY1, rY2;
  rV1 = line(0, tV, bo - 1, tY, bo, tV, bo, tY, bo + 1, tV, bo + 1);
  rV2 = line(1, tV, bo - BX, tX, bo, tV, bo, tX, bo + BX, tV, bo + BX);
  rX1 = line(0, tX, bo - 1, tC, bo, tX, bo, tC, bo + 1, tX, bo + 1);
  rX2 = line(1, tX, bo - BX, tV, bo - BX, tX, bo, tV, bo, tX, bo + BX);
  rY1 = line(0, tY, bo - 1, tV, bo - 1, tY, bo, tV, bo, tY, bo + 1);
  rY2 = line(1, tY, bo - BX, tC, bo, tY, bo, tC, bo + BX, tY, bo + BX);

  T* sFH1 = arr(L::A_FH1);
  T* sFH2 = arr(L::A_FH2);
  T* sAH1 = arr(L::A_AH1);
  T* sAH2 = arr(L::A_AH2);
  T* sFL1 = arr(L::A_FL1);
  T* sFL2 = arr(L::A_FL2);
  auto fU = [&](int b, int dir) -> T {
    if constexpr (FLUX == FLUX_BURGERS) return sQU[b];
    else if constexpr (FLUX == FLUX_BL) {
      if constexpr (PS::F2) return sQU[dir * BN + b];
      else return dir == 0 ? sQU[b] : bl_f2<T>(m, sU[b], sQU[b]);
    }
    else return flux<FLUX, T>(m, dir, sU[b]);
  };
  auto aU = [&](int b) -> T { return sQU[(L::NQU - 1) * BN + b]; };
  // |f_dir'| at a cell average (stored for the Buckley-Leverett flux only)
  auto dU = [&](int b, int dir) -> T {
    if constexpr (FLUX == FLUX_BL) return sQU[(PS::DOFF + dir) * BN + b];
    else return T(0);
  };
  // |f_dir'| at a stored point
  auto Dz = [&](int type, int b, int dir) -> T {
    if constexpr (FLUX == FLUX_BL) return Q(type, PS::DOFF + dir)[b];
    else return T(0);
  };
  const T sixth = T(1.0 / 6.0), r36 = T(1.0 / 36.0);
  // x-faces (Simpson over the face: V below, X middle, V above)
  const auto p2_fh1 = seg<H - 1, H + TX, H, H + TY>([&](int bx, int by) {
    const int b = by * BX + bx;
    sFH1[b] = (Fz(tV, b - BX, 0) + T(4) * Fz(tX, b, 0) + Fz(tV, b, 0)) * sixth;
  });
  const auto p2_fh2 = seg<H, H + TX, H - 1, H + TY>([&](int bx, int by) {
    const int b = by * BX + bx;
    sFH2[b] = (Fz(tV, b - 1, 1) + T(4) * Fz(tY, b, 1) + Fz(tV, b, 1)) * sixth;
  });
  // cell potentials: tensor Simpson average of the DC potential a^ along each direction
  auto pot = [&](int b, int dir) -> T {
    const T sv = (Az(tV, b - BX - 1) + Az(tV, b - BX)) + (Az(tV, b - 1) + Az(tV, b));
    const T sx = Az(tX, b - 1) + Az(tX, b);
    const T sy = Az(tY, b - BX) + Az(tY, b);
    const T ac = Az(tC, b);
    return dir == 0 ? (T(8) * sy - T(4) * sx + T(32) * ac - sv) * r36
                    : (T(8) * sx - T(4) * sy + T(32) * ac - sv) * r36;
  };
  const auto p2_ah1 = seg<H - 1, H + TX + 1, H, H + TY>([&](int bx, int by) { sAH1[by * BX + bx] = pot(by * BX + bx, 0); });
  const auto p2_ah2 = seg<H, H + TX, H - 1, H + TY + 1>([&](int bx, int by) { sAH2[by * BX + bx] = pot(by * BX + bx, 1); });
  // LLF fluxes with the interval wave speed
  const auto p2_fl1 = seg<H - 2, H + TX + 1, H, H + TY>([&](int bx, int by) {
    const int b = by * BX + bx;
    const T ul = sU[b], ur = sU[b + 1];
    const T al = alpha_interval_pre<FLUX, T>(m, 0, ul, ur, dU(b, 0), dU(b + 1, 0));
    sFL1[b] = T(0.5) * (fU(b, 0) + fU(b + 1, 0)) - T(0.5) * al * (ur - ul);
  });
  const auto p2_fl2 = seg<H, H + TX, H - 2, H + TY + 1>([&](int bx, int by) {
    const int b = by * BX + bx;
    const T ul = sU[b], ur = sU[b + BX];
    const T al = alpha_interval_pre<FLUX, T>(m, 1, ul, ur, dU(b, 1), dU(b + BX, 1));
    sFL2[b] = T(0.5) * (fU(b, 1) + fU(b + BX, 1)) - T(0.5) * al * (ur - ul);
  });
  if constexpr (BLEND) {
    if (A.blend_external) {
      for_segs<NT>(p2_fh1, p2_fh2, p2_ah1, p2_ah2, p2_fl1, p2_fl2,
                   seg<H - 1, H + TX + 1, H - 1, H + TY + 1>([&](int bx, int by) {
                     const int gi = wrapi(i0 - H + bx, nx), gj = wrapi(j0 - H + by, ny);
                     const T s = T(A.s_ext[(size_t)gj * nx + gi]);
                     sS1[by * BX + bx] = s;
                     sS2[by * BX + bx] = s;
                   }));
    } else {
      // s_l = (s~_{-1} + 4 s~ + s~_{+1}) / 6 along direction l
      for_segs<NT>(p2_fh1, p2_fh2, p2_ah1, p2_ah2, p2_fl1, p2_fl2,
                   seg<H - 1, H + TX + 1, H - 1, H + TY + 1>([&](int bx, int by) {
                     const int b = by * BX + bx;
                     sS1[b] = (sTC1[b - 1] + T(4) * sTC1[b] + sTC1[b + 1]) * sixth;
                     sS2[b] = (sTC2[b - BX] + T(4) * sTC2[b] + sTC2[b + BX]) * sixth;
                   }));
    }
  } else {
    for_segs<NT>(p2_fh1, p2_fh2, p2_ah1, p2_ah2, p2_fl1, p2_fl2);
  }
  __syncthreads();

  T rV, rX, rY;
  if constexpr (BLEND) {
    // ---- P2b: blend weights theta^{c,s} = exp(-gamma (s_i + s_{i+1})/2), theta^{d,s} = exp(-gamma s_i)
    const T g = sc.g;
    for_rect<NT>(H - 1, H + TX + 1, H - 1, H + TY + 1, [&](int bx, int by) {
      const int b = by * BX + bx;
      const T s1 = sS1[b], s2 = sS2[b];
      if (bx < H + TX) sTC1[b] = exp(-g * (T(0.5) * (s1 + sS1[b + 1])));
      if (by < H + TY) sTC2[b] = exp(-g * (T(0.5) * (s2 + sS2[b + BX])));
    });
    __syncthreads();
    for_rect<NT>(H - 1, H + TX + 1, H - 1, H + TY + 1, [&](int bx, int by) {
      const int b = by * BX + bx;
      sTD1[b] = exp(-g * sS1[b]);
      sTD2[b] = exp(-g * sS2[b]);
    });
    __syncthreads();
    // ---- P2c: blended fluxes/potentials (in place) and blended point residuals
    for_segs<NT>(seg<H - 1, H + TX, H, H + TY>([&](int bx, int by) {
                   const int b = by * BX + bx;
                   const T t = sTC1[b];
                   sFH1[b] = t * sFH1[b] + (T(1) - t) * sFL1[b];
                 }),
                 seg<H, H + TX, H - 1, H + TY>([&](int bx, int by) {
                   const int b = by * BX + bx;
                   const T t = sTC2[b];
                   sFH2[b] = t * sFH2[b] + (T(1) - t) * sFL2[b];
                 }),
                 seg<H - 1, H + TX + 1, H, H + TY>([&](int bx, int by) {
                   const int b = by * BX + bx;
                   const T t = sTD1[b];
                   sAH1[b] = t * sAH1[b] + (T(1) - t) * aU(b);
                 }),
                 seg<H, H + TX, H - 1, H + TY + 1>([&](int bx, int by) {
                   const int b = by * BX + bx;
                   const T t = sTD2[b];
                   sAH2[b] = t * sAH2[b] + (T(1) - t) * aU(b);
                 }));
    // first-order point residual on the +-h/2 neighbours (centre -> cell average):
    //   -(2/h)[F(z0,z+) - F(z-,z0)] + (4/h^2)(a+ - 2 a0 + a-)
    const T i2h1 = sc.i2h1, i2h2 = sc.i2h2;
    const T i4h21 = sc.i4h21, i4h22 = sc.i4h22;
    // value, flux, potential and |f'| (direction dir) at a stored point / a cell average
    struct PV {
      T z, f, a, d;
    };
    auto pt = [&](int type, int bb, int dir) -> PV {
      return PV{sZ[type][bb], Fz(type, bb, dir), Az(type, bb), Dz(type, bb, dir)};
    };
    auto cu = [&](int bb, int dir) -> PV { return PV{sU[bb], fU(bb, dir), aU(bb), dU(bb, dir)}; };
    auto lowres = [&](int dir, const PV& pm, const PV& p0, const PV& pp) -> T {
      const T Fr = T(0.5) * (p0.f + pp.f) -
                   T(0.5) * alpha_interval_pre<FLUX, T>(m, dir, p0.z, pp.z, p0.d, pp.d) * (pp.z - p0.z);
      const T Fl = T(0.5) * (pm.f + p0.f) -
                   T(0.5) * alpha_interval_pre<FLUX, T>(m, dir, pm.z, p0.z, pm.d, p0.d) * (p0.z - pm.z);
      return (pp.a - T(2) * p0.a + pm.a) * (dir == 0 ? i4h21 : i4h22) - (Fr - Fl) * (dir == 0 ? i2h1 : i2h2);
    };
    const int b = bo;
    const T LV1 = lowres(0, pt(tY, b, 0), pt(tV, b, 0), pt(tY, b + 1, 0));
    const T LV2 = lowres(1, pt(tX, b, 1), pt(tV, b, 1), pt(tX, b + BX, 1));
    const T LX1 = lowres(0, cu(b, 0), pt(tX, b, 0), cu(b + 1, 0));
    const T LX2 = lowres(1, pt(tV, b - BX, 1), pt(tX, b, 1), pt(tV, b, 1));
    const T LY1 = lowres(0, pt(tV, b - 1, 0), pt(tY, b, 0), pt(tV, b, 0));
    const T LY2 = lowres(1, cu(b, 1), pt(tY, b, 1), cu(b + BX, 1));
    const T wV1 = tmin(sTC1[b], sTC1[b + BX]), wV2 = tmin(sTC2[b], sTC2[b + 1]);
    const T wX1 = sTC1[b], wX2 = tmin(sTD2[b], sTD2[b + 1]);
    const T wY1 = tmin(sTD1[b], sTD1[b + BX]), wY2 = sTC2[b];
    rV = (wV1 * rV1 + (T(1) - wV1) * LV1) + (wV2 * rV2 + (T(1) - wV2) * LV2);
    rX = (wX1 * rX1 + (T(1) - wX1) * LX1) + (wX2 * rX2 + (T(1) - wX2) * LX2);
    rY = (wY1 * rY1 + (T(1) - wY1) * LY1) + (wY2 * rY2 + (T(1) - wY2) * LY2);
    __syncthreads();
  } else {
    rV = rV1 + rV2;
    rX = rX1 + rX2;
    rY = rY1 + rY2;
  }

  // ---- per output: low-order states, limiter, update ------------------------------------
  const int gi = i0 + tx, gj = j0 + ty;
  const bool own = gi < nx && gj < ny;
  const size_t g = (size_t)gj * nx + gi;
  T* sULp1 = arr(L::A_ULP1);
  T* sULm1 = arr(L::A_ULM1);
  T* sULp2 = arr(L::A_ULP2);
  T* sULm2 = arr(L::A_ULM2);
  T* sFlim1 = A.limiter ? arr(L::A_FLIM1) : sFH1;
  T* sFlim2 = A.limiter ? arr(L::A_FLIM2) : sFH2;
  T* sAlim1 = A.limiter ? arr(L::A_ALIM1) : sAH1;
  T* sAlim2 = A.limiter ? arr(L::A_ALIM2) : sAH2;
  // kept rolled: one copy of the per-output body, compiled identically in every kernel
  // that inlines this tile
#pragma unroll 1
  for (int o = 0; o < A.nout; ++o) {
    const double mu1 = sc.mu1[o], mu2 = sc.mu2[o];
    const double nu1 = sc.nu1[o], nu2 = sc.nu2[o];
    if (A.limiter) {
      // ---- P3: directional low-order states u^{L,+-}_l = ub -+ 4 mu (...) +- 4 nu (...)
      const T m4_1 = sc.m4_1[o], n4_1 = sc.n4_1[o], m4_2 = sc.m4_2[o], n4_2 = sc.n4_2[o];
      for_segs<NT>(seg<H - 2, H + TX + 2, H, H + TY>([&](int bx, int by) {
                     const int b = by * BX + bx;
                     const T u = sU[b], f = fU(b, 0), a = aU(b);
                     if (bx < H + TX + 1) sULp1[b] = u - m4_1 * (sFL1[b] - f) + n4_1 * (aU(b + 1) - a);
                     if (bx > H - 2) sULm1[b] = u - m4_1 * (f - sFL1[b - 1]) - n4_1 * (a - aU(b - 1));
                   }),
                   seg<H, H + TX, H - 2, H + TY + 2>([&](int bx, int by) {
                     const int b = by * BX + bx;
                     const T u = sU[b], f = fU(b, 1), a = aU(b);
                     if (by < H + TY + 1) sULp2[b] = u - m4_2 * (sFL2[b] - f) + n4_2 * (aU(b + BX) - a);
                     if (by > H - 2) sULm2[b] = u - m4_2 * (f - sFL2[b - BX]) - n4_2 * (a - aU(b - BX));
                   }));
      __syncthreads();
      // ---- P4: theta^c per face (2 states), theta^d per cell (4 states), factor 12
      const T k1 = sc.k1[o], k2 = sc.k2[o], q1 = sc.q1[o], q2 = sc.q2[o];
      for_segs<NT>(seg<H - 1, H + TX, H, H + TY>([&](int bx, int by) {
                     const int b = by * BX + bx;
                     const T fh = sFH1[b], fl = sFL1[b], dF = fh - fl;
                     const T zp = sULp1[b], zm = sULm1[b + 1];
                     const T t = theta_pair<T>(zp, zp - k1 * dF, zm, zm + k1 * dF, umin, umax);
                     sFlim1[b] = is_one(t) ? fh : fl + t * dF;
                   }),
                   seg<H, H + TX, H - 1, H + TY>([&](int bx, int by) {
                     const int b = by * BX + bx;
                     const T fh = sFH2[b], fl = sFL2[b], dF = fh - fl;
                     const T zp = sULp2[b], zm = sULm2[b + BX];
                     const T t = theta_pair<T>(zp, zp - k2 * dF, zm, zm + k2 * dF, umin, umax);
                     sFlim2[b] = is_one(t) ? fh : fl + t * dF;
                   }),
                   seg<H - 1, H + TX + 1, H, H + TY>([&](int bx, int by) {
                     const int b = by * BX + bx;
                     const T ah = sAH1[b], al = aU(b), d = q1 * (ah - al);
                     const T p0 = sULp1[b - 1], p1 = sULp1[b], q0 = sULm1[b], q1 = sULm1[b + 1];
                     const T t = theta_quad<T>(p0, p0 + d, p1, p1 - d, q0, q0 - d, q1, q1 + d, umin, umax);
                     sAlim1[b] = is_one(t) ? ah : al + t * (ah - al);
                   }),
                   seg<H, H + TX, H - 1, H + TY + 1>([&](int bx, int by) {
                     const int b = by * BX + bx;
                     const T ah = sAH2[b], al = aU(b), d = q2 * (ah - al);
                     const T p0 = sULp2[b - BX], p1 = sULp2[b], q0 = sULm2[b], q1 = sULm2[b + BX];
                     const T t = theta_quad<T>(p0, p0 + d, p1, p1 - d, q0, q0 - d, q1, q1 + d, umin, umax);
                     sAlim2[b] = is_one(t) ? ah : al + t * (ah - al);
                   }));
      __syncthreads();
    }
    // ---- P5: limited average update, point update + projection, RK combination ----
    if (own) {
      const int b = bo;
      const double ubin = A.ub[g];
      // explicit roundings: every kernel inlining this tile (single mesh or batch)
      // produces bit-identical results
      double ubfe;
      if constexpr (sizeof(T) == 8) {
        const double dflux = rk_comb(mu1, (double)sFlim1[b] - (double)sFlim1[b - 1], mu2,
                                     (double)sFlim2[b] - (double)sFlim2[b - BX]);
        const double dpot = rk_comb(nu1, ((double)sAlim1[b + 1] - 2.0 * (double)sAlim1[b]) + (double)sAlim1[b - 1],
                                    nu2, ((double)sAlim2[b + BX] - 2.0 * (double)sAlim2[b]) + (double)sAlim2[b - BX]);
        ubfe = (ubin - dflux) + dpot;
      } else {
        // FP32 stencils: each face contributes mu F (convection) and nu (A_+ - A)
        // (diffusion), formed in FP32 by both adjacent cells from the same operands, so
        // the contributions cancel exactly across faces; the eight terms of a cell are
        // summed without rounding error (TwoSum) and added once to the FP64 average.
        const float m1 = sc.mu1f[o], m2 = sc.mu2f[o], n1 = sc.nu1f[o], n2 = sc.nu2f[o];
        const float t[8] = {__fmul_rn(m1, sFlim1[b - 1]), -__fmul_rn(m1, sFlim1[b]),
                            __fmul_rn(m2, sFlim2[b - BX]), -__fmul_rn(m2, sFlim2[b]),
                            __fmul_rn(n1, __fsub_rn(sAlim1[b + 1], sAlim1[b])),
                            -__fmul_rn(n1, __fsub_rn(sAlim1[b], sAlim1[b - 1])),
                            __fmul_rn(n2, __fsub_rn(sAlim2[b + BX], sAlim2[b])),
                            -__fmul_rn(n2, __fsub_rn(sAlim2[b], sAlim2[b - BX]))};
        float hi = t[0], lo = 0.0f;
#pragma unroll
        for (int q = 1; q < 8; ++q) {
          float e;
          two_sum(hi, t[q], hi, e);
          lo = __fadd_rn(lo, e);
        }
        ubfe = ubin + (f2d_exact(hi) + f2d_exact(lo));
      }
      const T taut = sc.taut[o];
      T v = rk_fma(taut, rV, sZ[tV][b]), x = rk_fma(taut, rX, sZ[tX][b]), y = rk_fma(taut, rY, sZ[tY][b]);
      if (A.limiter) {
        v = tmin(tmax(v, umin), umax);
        x = tmin(tmax(x, umin), umax);
        y = tmin(tmax(y, umin), umax);
      }
      const double cA = A.cA[o], cF = A.cF[o];
      const T cAt = sc.cAt[o], cFt = sc.cFt[o];
      double ubo;
      PT vo, xo, yo;
      if (!is_zero_bits(cA)) {
        ubo = rk_comb(cA, A.Aub[o][g], cF, ubfe);
        vo = PT(rk_comb(cAt, T(A.AV[o][g]), cFt, v));
        xo = PT(rk_comb(cAt, T(A.AX[o][g]), cFt, x));
        yo = PT(rk_comb(cAt, T(A.AY[o][g]), cFt, y));
      } else {
        ubo = rk_scale(cF, ubfe);
        vo = PT(rk_scale(cFt, v));
        xo = PT(rk_scale(cFt, x));
        yo = PT(rk_scale(cFt, y));
      }
      if constexpr (RECT) {
        // the padded rectangle stores the average from (1, 1), X from row 1, Y from column 1
        const bool wU = gi > 0 && gj > 0, wX = gj > 0, wY = gi > 0;
        if (A.limiter && A.sg[o]) {
          if (wU) ubo = safeguard<double>(ubo, m.umin, m.umax, A.tol, A.stats, true);
          vo = safeguard<PT>(vo, PT(umin), PT(umax), A.tol, A.stats);
          if (wX) xo = safeguard<PT>(xo, PT(umin), PT(umax), A.tol, A.stats);
          if (wY) yo = safeguard<PT>(yo, PT(umin), PT(umax), A.tol, A.stats);
        }
        if (wU) A.Oub[o][g] = ubo;
        A.OV[o][g] = vo;
        if (wX) A.OX[o][g] = xo;
        if (wY) A.OY[o][g] = yo;
      } else {
        if (A.limiter && A.sg[o]) {
          ubo = safeguard<double>(ubo, m.umin, m.umax, A.tol, A.stats, true);
          vo = safeguard<PT>(vo, PT(umin), PT(umax), A.tol, A.stats);
          xo = safeguard<PT>(xo, PT(umin), PT(umax), A.tol, A.stats);
          yo = safeguard<PT>(yo, PT(umin), PT(umax), A.tol, A.stats);
        }
        A.Oub[o][g] = ubo;
        A.OV[o][g] = vo;
        A.OX[o][g] = xo;
        A.OY[o][g] = yo;
      }
    }
    if (o + 1 < A.nout) __syncthreads();
  }
}

// One CTA per 32 x 8 tile of a single mesh (row-major tile index in blockIdx.x).
template <int FLUX, class T, class PT, bool BLEND, bool RECT = false>
__global__ void __launch_bounds__(256) stage2d_kernel(const DevModel m, const StageArgs2D<PT> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tiles_x = (A.nx + 31) / 32, t = blockIdx.x;   // 1D grid: no 65535 limit on rows
  stage_tile<FLUX, T, PT, BLEND, 32, 8, true, RECT>(m, A, (t % tiles_x) * 32, (t / tiles_x) * 8, smem_raw);
}

// The same for the FP32 stencils without the blend, compiled for 6 resident CTAs per SM
// (<= 40 registers; its 36 KB of shared memory allow 6): measured 8% faster than the
// compiler's own 48-register choice at 5 CTAs per SM.
template <int FLUX, bool RECT = false>
__global__ void __launch_bounds__(256, 6) stage2d_kernel_f32occ6(const DevModel m, const StageArgs2D<float> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tiles_x = (A.nx + 31) / 32, t = blockIdx.x;
  stage_tile<FLUX, float, float, false, 32, 8, true, RECT>(m, A, (t % tiles_x) * 32, (t / tiles_x) * 8, smem_raw);
}

}  // namespace af
