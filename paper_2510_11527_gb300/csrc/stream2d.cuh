// Column-marching 2D stage kernel (periodic meshes, with or without the smoothness
// blend): the same limited forward-Euler evaluation and Shu-Osher combination as
// stage_tile (Sections 4 and 5.2 of arXiv 2510.11527, d = 2), organised so that every
// derived quantity is formed once per location and kept in registers.
//
// Each warp owns a band of 28 output columns and a strip of S output rows. Lane L holds
// column 28 * band - 2 + L (periodic image): lanes 2..29 produce outputs, lanes 0, 1,
// 30, 31 only supply the +-2 halo of the x-stencils, which reach neighbouring columns
// through warp shuffles. The warp marches up its strip one input row per step, so the
// y-stencils read the rows before it from registers: at step r it loads row r, forms
// the row's centres, pointwise f, a, its x-face and cell quantities, the y-face between
// rows r-1 and r, the point residuals of row r-1, the x-limiter of row r and the
// y-limiter of row r-1, and finalises the cells of row r-2. Three row slots hold what
// later steps read (the loop is unrolled by three so the slots rotate without copies).
//
// Conservation: every face term of the FP32 update (mu F and nu (A_+ - A)) reaches both
// adjacent cells unchanged (a shuffle or a register); a face on a band or strip edge is
// formed by both warps that meet there, from the same values with the same rounding
// (the kernel's translation unit is compiled without contraction), so the terms cancel
// exactly across faces. Each cell sums its eight terms without rounding error (TwoSum)
// and adds them once to the FP64 average, as stage_tile does.
#pragma once
#include "stage2d.cuh"

namespace af {

constexpr int STREAM_BAND = 28;   // output columns per warp
constexpr int STREAM_WPB = 4;     // warps per block
// Resident blocks per SM the kernel is compiled for: 4 (128 registers per thread, 16
// warps per SM) measured fastest; Buckley-Leverett's and the blend's longer live
// ranges spill there and take 3.
template <int FLUX, int BK = 0>
constexpr int stream_min_blocks() { return FLUX == FLUX_BL || BK != 0 ? 3 : 4; }

// per-lane constants of one launch
template <class T>
struct StreamScal {
  T umin, umax, i6h1, i6h2, i3h21, i3h22, m4_1, n4_1, m4_2, n4_2, k1, k2, q1, q2, taut, cAt, cFt, half, sixth, r36;
  float m1f, m2f, n1f, n2f;
  double cA, cF, umid;
};

// per-warp constants of the smoothness blend (kept apart from StreamScal: a larger
// StreamScal cost the kernels without the blend registers); static shared memory of
// the kernel's translation unit, one slot per warp of a block
struct BlendScal {
  float g, i2h1, i2h2, i4h21, i4h22;   // gamma; 2/h and 4/h^2 of the low-order residual
};
static __shared__ BlendScal stream_kb[STREAM_WPB];

// values of one input row that later steps read (a row slot)
template <class T>
struct RowSlot {
  T V, X, Y, C, U;                 // points, recovered centre, cell average (stencil type)
  T fV, fX, fY, fC, fU;            // f_2 at V, X, Y, centre, average (y-direction flux)
  T fV1;                           // f_1 at V (x-face Simpson flux of the next row)
  T dV, dX, dY, dC, dU;            // |f_2'| (Buckley-Leverett)
  T aV, aX, aY, aC, aU;            // a
  T Vm, aVm;                       // V and a(V) of the left neighbour column
  T FH2, AH2;                      // high-order flux of the y-face above, cell potential (y)
  T rV, rX, rY;                    // point residuals (x-lines, then x + y)
  T ULp2, ULm2, Alim2;             // y low-order states, limited potential (y)
  T tF2lo, tD2lo;                  // update terms of the y-face below the row's cell
  T tF1, tD1;                      // update terms of the x-face right of the cell
  // smoothness blend: s_2 of the cell, theta^{c,s} of the x-face right of the cell,
  // theta^{d,s}_1 of the cell, low-order residuals of the row's x-lines (V, X, Y)
  T s2, tc1, td1, LV1, LX1, LY1;
  T FVX;   // LLF flux (y) between V of the row below and X of this row
};

// max / min for values that are never NaN in a valid state: one FMNMX in FP32 (tmax /
// tmin keep the select semantics of the tile kernel); FP64 keeps the integer compare
__device__ __forceinline__ float fmx(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float fmn(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double fmx(double a, double b) { return tmax(a, b); }
__device__ __forceinline__ double fmn(double a, double b) { return tmin(a, b); }

// Diffusion kinds compiled into the column-marching kernel (DK_GENERIC takes the
// model's runtime kind).
enum : int { DK_GENERIC = -1, DK_NONE = 0, DK_CONST = 1, DK_PWL = 2, DK_PME2 = 3, DK_CUBIC = 4 };

template <int DIFF, class T>
__device__ __forceinline__ T apot_k(const DevModel& m, T u) {
  if constexpr (DIFF == DK_NONE) {
    return T(0);
  } else if constexpr (DIFF == DK_CONST) {
    return par<T>(m.dp, m.dpf, 0) * u;
  } else if constexpr (DIFF == DK_PWL) {
    // both branches always: a zero coefficient contributes a signed zero, which does not
    // change the sum
    return par<T>(m.dp, m.dpf, 0) * fmn(u - par<T>(m.dp, m.dpf, 1), T(0)) +
           par<T>(m.dp, m.dpf, 2) * fmx(u - par<T>(m.dp, m.dpf, 3), T(0));
  } else if constexpr (DIFF == DK_PME2) {
    return u * u;
  } else if constexpr (DIFF == DK_CUBIC) {
    return ((par<T>(m.dp, m.dpf, 2) * u + par<T>(m.dp, m.dpf, 1)) * u + par<T>(m.dp, m.dpf, 0)) * u;
  } else {
    return apot<T>(m, u);
  }
}

// a * b + c with one rounding, written out (the translation unit of this kernel is
// compiled without contraction)
__device__ __forceinline__ float sfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double sfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// line residual of stage_tile's line_res with its multiply-adds fused explicitly
template <class T>
__device__ __forceinline__ T line_res_s(T z0, T z1, T z2, T z3, T z4, T f0, T f1, T f3, T f4, T alpha, T a0, T a1,
                                        T a2, T a3, T a4, T i6h, T i3h2) {
  const T cf = sfma(T(8), f3 - f1, f0 - f4);
  const T dz = sfma(T(6), z2, sfma(T(-4), z1 + z3, z0 + z4));
  const T da = sfma(T(-30), a2, sfma(T(16), a1 + a3, -(a0 + a4)));
  return sfma(da, i3h2, -(sfma(alpha, dz, cf) * i6h));
}

template <class T>
__device__ __forceinline__ T shup(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <class T>
__device__ __forceinline__ T shdn(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// f_l, |f_l'| and a at one value: returns f_1 in f1, f_2 in f2, |f_1'| in d1, |f_2'| in d2
template <int FLUX, int DIFF, class T>
__device__ __forceinline__ void point_eval(const DevModel& m, T z, T& f1, T& f2, T& d1, T& d2, T& a) {
  if constexpr (FLUX == FLUX_BURGERS) {
    f1 = flux<FLUX, T>(m, 0, z);
    f2 = f1;
    d1 = d2 = T(0);
  } else if constexpr (FLUX == FLUX_BL) {
    const BLVals<T> r = bl_eval<T>(m, z);
    f1 = r.f[0];
    f2 = r.f[1];
    d1 = r.d[0];
    d2 = r.d[1];
  } else {
    f1 = flux<FLUX, T>(m, 0, z);
    f2 = flux<FLUX, T>(m, 1, z);
    d1 = d2 = T(0);
  }
  a = apot_k<DIFF, T>(m, z);
}

// alpha of a 5-point line along dir from the values (Burgers: |z|) or |f'| (Buckley-Leverett)
template <int FLUX, class T>
__device__ __forceinline__ T line_alpha(const DevModel& m, int dir, T z0, T z1, T z2, T z3, T z4, T d0, T d1, T d2,
                                        T d3, T d4) {
  if constexpr (FLUX == FLUX_BURGERS) {
    return tabs(T(2) * par<T>(m.fp, m.fpf, 0)) * fmx(fmx(fmx(tabs(z0), tabs(z1)), fmx(tabs(z3), tabs(z4))), tabs(z2));
  } else if constexpr (FLUX == FLUX_BL) {
    return fmx(fmx(fmx(d0, d1), fmx(d3, d4)), d2);
  } else if constexpr (FLUX == FLUX_LINEAR) {
    return tabs(T(dir == 0 ? m.fp[0] : m.fp[1]));
  } else {
    return T(0);
  }
}

template <int FLUX, class T>
__device__ __forceinline__ T llf(const DevModel& m, int dir, T ul, T ur, T fl, T fr, T dl, T dr, T half) {
  const T al = alpha_interval_pre<FLUX, T>(m, dir, ul, ur, dl, dr);
  return sfma(-(half * al), ur - ul, half * (fl + fr));
}

// first-order point residual of the smoothness blend on the +-h/2 neighbours (m, 0, p)
// of a point along dir: -(2/h) [F(z0, zp) - F(zm, z0)] + (4/h^2) (a_p - 2 a_0 + a_m),
// F the LLF flux (a recovered centre enters as its cell's average)
// from the two LLF fluxes (left Fl = F(zm, z0), right Fr = F(z0, zp)), which the
// neighbouring points' residuals share
template <class T>
__device__ __forceinline__ T lowres_s(T Fl, T Fr, T am, T a0, T ap, T i2h, T i4h2) {
  return sfma(sfma(T(-2), a0, ap + am), i4h2, -((Fr - Fl) * i2h));
}

// w h + (1 - w) l: a blend weight applied to a high-order and a low-order value
template <class T>
__device__ __forceinline__ T blendw(T w, T h, T l) { return sfma(w, h - l, l); }

// cell potential (tensor Simpson average of the DC potential along dir): for x,
// (8 sy - 4 sx + 32 ac - sv) / 36
template <class T>
__device__ __forceinline__ T cell_pot(T sv, T sx, T sy, T ac, bool ydir, T r36) {
  const T a = ydir ? sx : sy, b = ydir ? sy : sx;
  return sfma(T(32), ac, sfma(T(8), a, sfma(T(-4), b, -sv))) * r36;
}

template <int FLUX, int DIFF, class T>
struct StreamCtx {
  const DevModel& m;
  const StageArgs2D<T>& A;
  const StreamScal<T>& k;
  int nx, ny, gi, lane, rs, re;
  bool col_out;          // this lane's column produces outputs
  bool comb;             // the output combines an earlier state (cA != 0)
};

// per-row input registers (the next row is prefetched one step ahead)
template <class T>
struct RowIn {
  double ub;
  T V, X, Y;
  T s1, s2;   // smoothness indicators (blend)
};
template <class T>
struct OutIn {
  double ub, Aub;   // FE input and RK combination input of the output cell
  T V, X, Y;        // RK combination inputs of the point values
};

// BK: the smoothness blend's indicator. 0: no blend; 1: s_1 and s_2 per cell (FP32
// arrays A.sb[0], A.sb[1]); 2: one external indicator per cell for both directions
// (FP64 array A.s_ext).
template <class T, int BK = 0>
__device__ __forceinline__ RowIn<T> load_row(const StageArgs2D<T>& A, size_t g) {
  RowIn<T> in;
  in.ub = __ldg(A.ub + g);
  in.V = __ldg(A.V + g);
  in.X = __ldg(A.X + g);
  in.Y = __ldg(A.Y + g);
  if constexpr (BK == 1) {
    in.s1 = __ldg(A.sb[0] + g);
    in.s2 = __ldg(A.sb[1] + g);
  } else if constexpr (BK == 2) {
    // integer conversion (toward zero): GB300 runs double -> float on its FP64 unit
    in.s1 = in.s2 = to_stencil<T>(__ldg(A.s_ext + g));
  } else {
    in.s1 = in.s2 = T(0);
  }
  return in;
}

// One step: input row r arrives (in), slots p2 (row r-2), p1 (row r-1), cur (row r;
// held row r-3 before). Finalises the cells of row r-2 if they belong to the strip.
template <int FLUX, int DIFF, class T, int BK>
__device__ __forceinline__ void stream_step(const StreamCtx<FLUX, DIFF, T>& c, int r, const RowIn<T>& in,
                                            const OutIn<T>& oin, RowSlot<T>& p2, RowSlot<T>& p1, RowSlot<T>& cur) {
  const DevModel& m = c.m;
  const StageArgs2D<T>& A = c.A;
  const StreamScal<T>& k = c.k;
  const T half = k.half, sixth = k.sixth;
  const bool lim = A.limiter != 0;
  constexpr bool BL = FLUX == FLUX_BL;

  // ---- row r: points, centre, pointwise functions
  cur.U = to_stencil_nb<T>(in.ub, k.umid);
  cur.V = in.V;
  cur.X = in.X;
  cur.Y = in.Y;
  const T Xm = shup(cur.X);
  cur.Vm = shup(cur.V);
  // z_ij = [36 zbar - 4 (X_{i-1,j} + X_ij + Y_{i,j-1} + Y_ij) - (four corners)] / 16
  cur.C = sfma(T(36), cur.U, sfma(T(-4), (Xm + cur.X) + (p1.Y + cur.Y), -((p1.Vm + p1.V) + (cur.Vm + cur.V)))) *
          T(0.0625);
  T f1V, f1X, f1Y, f1C, f1U, d1V, d1X, d1Y, d1C, d1U;
  point_eval<FLUX, DIFF, T>(m, cur.V, f1V, cur.fV, d1V, cur.dV, cur.aV);
  point_eval<FLUX, DIFF, T>(m, cur.X, f1X, cur.fX, d1X, cur.dX, cur.aX);
  point_eval<FLUX, DIFF, T>(m, cur.Y, f1Y, cur.fY, d1Y, cur.dY, cur.aY);
  point_eval<FLUX, DIFF, T>(m, cur.C, f1C, cur.fC, d1C, cur.dC, cur.aC);
  point_eval<FLUX, DIFF, T>(m, cur.U, f1U, cur.fU, d1U, cur.dU, cur.aU);
  cur.fV1 = f1V;
  // smoothness blend (Section 5.1.3, direction by direction as in Section 5.2):
  // theta^{d,s}_1 of cell (i, r) and theta^{c,s}_1 of the x-face right of it
  T td1 = T(1), tc1 = T(1);
  const BlendScal& kb = stream_kb[threadIdx.x >> 5];
  if constexpr (BK != 0) {
    cur.s2 = in.s2;
    td1 = expf(-kb.g * in.s1);
    tc1 = expf(-kb.g * (half * (in.s1 + shdn(in.s1))));
    cur.td1 = td1;
    cur.tc1 = tc1;
  }

  // ---- neighbour values (|f'| only where the flux needs it)
  auto dup = [](T v) { if constexpr (BL) return shup(v); else return T(0); };
  auto ddn = [](T v) { if constexpr (BL) return shdn(v); else return T(0); };
  cur.aVm = shup(cur.aV);
  const T aXm = shup(cur.aX);
  const T f1Vm = shup(f1V), d1Vm = dup(d1V);
  T fVm2;   // f_2(V_{i-1,r})
  if constexpr (FLUX == FLUX_BURGERS) fVm2 = f1Vm; else fVm2 = shup(cur.fV);
  const T f1Xm = shup(f1X), d1Xm = dup(d1X);
  const T Ym = shup(cur.Y), f1Ym = shup(f1Y), aYm = shup(cur.aY), d1Ym = dup(d1Y);
  const T Up = shdn(cur.U), f1Up = shdn(f1U), aUp = shdn(cur.aU), d1Up = ddn(d1U);
  const T Um = shup(cur.U), f1Um = shup(f1U), aUm = shup(cur.aU), d1Um = dup(d1U);
  const T Vp = shdn(cur.V), f1Vp = shdn(f1V), aVp = shdn(cur.aV), d1Vp = ddn(d1V);
  const T Yp = shdn(cur.Y), f1Yp = shdn(f1Y), aYp = shdn(cur.aY), d1Yp = ddn(d1Y);
  const T Xp = shdn(cur.X), f1Xp = shdn(f1X), aXp = shdn(cur.aX), d1Xp = ddn(d1X);
  const T Cp = shdn(cur.C), f1Cp = shdn(f1C), aCp = shdn(cur.aC), d1Cp = ddn(d1C);

  // ---- faces and cell potentials of row r
  // x-face right of cell (i, r): Simpson over V_{i,r-1}, X_{i,r}, V_{i,r}
  T FH1 = sfma(T(4), f1X, p1.fV1 + f1V) * sixth;
  // y-face above cell (i, r): Simpson over V_{i-1,r}, Y_{i,r}, V_{i,r}
  cur.FH2 = sfma(T(4), cur.fY, fVm2 + cur.fV) * sixth;
  T AH1;   // lives only in this step (x-limiter of row r)
  {
    const T sv = (p1.aVm + p1.aV) + (cur.aVm + cur.aV);
    const T sx = aXm + cur.aX;
    const T sy = p1.aY + cur.aY;
    cur.AH2 = cell_pot<T>(sv, sx, sy, cur.aC, true, k.r36);
    AH1 = cell_pot<T>(sv, sx, sy, cur.aC, false, k.r36);
    if constexpr (BK != 0) AH1 = blendw(td1, AH1, cur.aU);
  }
  const T FL1 = llf<FLUX, T>(m, 0, cur.U, Up, f1U, f1Up, d1U, d1Up, half);
  // the face on the left, formed here as its owner forms it (same inputs, same code)
  const T FL1m = llf<FLUX, T>(m, 0, Um, cur.U, f1Um, f1U, d1Um, d1U, half);
  // y-face between rows r-1 and r
  const T FL2 = llf<FLUX, T>(m, 1, p1.U, cur.U, p1.fU, cur.fU, p1.dU, cur.dU, half);
  // blend: the x-face of row r; theta^{c,s}_2 of the y-face between rows r-1 and r and
  // theta^{d,s}_2 of cell (i, r-1), with the y-face flux and the y cell potential of
  // row r-1 (both first used by this step's y-limiter); the low-order residuals of the
  // x-lines of row r
  T tc2 = T(1), td2 = T(1);
  if constexpr (BK != 0) {
    FH1 = blendw(tc1, FH1, FL1);
    tc2 = expf(-kb.g * (half * (p1.s2 + cur.s2)));
    td2 = expf(-kb.g * p1.s2);
    p1.FH2 = blendw(tc2, p1.FH2, FL2);
    p1.AH2 = blendw(td2, p1.AH2, p1.aU);
    // x-lines: V between Y_i and Y_{i+1}, X between the averages of cells i and i+1,
    // Y between V_{i-1} and V_i; F(V_{i-1}, Y_i) is the left lane's F(V, Y_{+1})
    const T FYV = llf<FLUX, T>(m, 0, cur.Y, cur.V, f1Y, f1V, d1Y, d1V, half);
    const T FVY = llf<FLUX, T>(m, 0, cur.V, Yp, f1V, f1Yp, d1V, d1Yp, half);
    const T FUX = llf<FLUX, T>(m, 0, cur.U, cur.X, f1U, f1X, d1U, d1X, half);
    const T FXU = llf<FLUX, T>(m, 0, cur.X, Up, f1X, f1Up, d1X, d1Up, half);
    cur.LV1 = lowres_s<T>(FYV, FVY, cur.aY, cur.aV, aYp, kb.i2h1, kb.i4h21);
    cur.LX1 = lowres_s<T>(FUX, FXU, cur.aU, cur.aX, aUp, kb.i2h1, kb.i4h21);
    cur.LY1 = lowres_s<T>(shup(FVY), FYV, cur.aVm, cur.aY, cur.aV, kb.i2h1, kb.i4h21);
    // y-direction flux between V of row r-1 and X of row r (the next step's X-line)
    cur.FVX = llf<FLUX, T>(m, 1, p1.V, cur.X, p1.fV, cur.fX, p1.dV, cur.dX, half);
  }

  // ---- point residuals: x-lines of row r
  cur.rV = line_res_s<T>(cur.Vm, cur.Y, cur.V, Yp, Vp, f1Vm, f1Y, f1Yp, f1Vp,
                       line_alpha<FLUX, T>(m, 0, cur.Vm, cur.Y, cur.V, Yp, Vp, d1Vm, d1Y, d1V, d1Yp, d1Vp), cur.aVm,
                       cur.aY, cur.aV, aYp, aVp, k.i6h1, k.i3h21);
  cur.rX = line_res_s<T>(Xm, cur.C, cur.X, Cp, Xp, f1Xm, f1C, f1Cp, f1Xp,
                       line_alpha<FLUX, T>(m, 0, Xm, cur.C, cur.X, Cp, Xp, d1Xm, d1C, d1X, d1Cp, d1Xp), aXm, cur.aC,
                       cur.aX, aCp, aXp, k.i6h1, k.i3h21);
  cur.rY = line_res_s<T>(Ym, cur.Vm, cur.Y, cur.V, Yp, f1Ym, f1Vm, f1V, f1Yp,
                       line_alpha<FLUX, T>(m, 0, Ym, cur.Vm, cur.Y, cur.V, Yp, d1Ym, d1Vm, d1Y, d1V, d1Yp), aYm,
                       cur.aVm, cur.aY, cur.aV, aYp, k.i6h1, k.i3h21);
  // y-lines of row r-1, added to its x-lines (same order as stage_tile: x + y)
  {
    const T rV2 = line_res_s<T>(p2.V, p1.X, p1.V, cur.X, cur.V, p2.fV, p1.fX, cur.fX, cur.fV,
                              line_alpha<FLUX, T>(m, 1, p2.V, p1.X, p1.V, cur.X, cur.V, p2.dV, p1.dX, p1.dV, cur.dX, cur.dV),
                              p2.aV, p1.aX, p1.aV, cur.aX, cur.aV, k.i6h2, k.i3h22);
    const T rX2 = line_res_s<T>(p2.X, p2.V, p1.X, p1.V, cur.X, p2.fX, p2.fV, p1.fV, cur.fX,
                              line_alpha<FLUX, T>(m, 1, p2.X, p2.V, p1.X, p1.V, cur.X, p2.dX, p2.dV, p1.dX, p1.dV, cur.dX),
                              p2.aX, p2.aV, p1.aX, p1.aV, cur.aX, k.i6h2, k.i3h22);
    const T rY2 = line_res_s<T>(p2.Y, p1.C, p1.Y, cur.C, cur.Y, p2.fY, p1.fC, cur.fC, cur.fY,
                              line_alpha<FLUX, T>(m, 1, p2.Y, p1.C, p1.Y, cur.C, cur.Y, p2.dY, p1.dC, p1.dY, cur.dC, cur.dY),
                              p2.aY, p1.aC, p1.aY, cur.aC, cur.aY, k.i6h2, k.i3h22);
    if constexpr (BK != 0) {
      // blended residuals: each direction's high-order residual against its low-order one
      // with the weight of the faces / cells the point lies on
      const T tc2p = shdn(tc2), td2p = shdn(td2);
      // y-lines of row r-1: V between X_{r-1} and X_r, X between V_{r-2} and V_{r-1}
      // (F(V_{r-2}, X_{r-1}) formed one step earlier), Y between the averages of rows
      // r-1 and r
      const T FXV = llf<FLUX, T>(m, 1, p1.X, p1.V, p1.fX, p1.fV, p1.dX, p1.dV, half);
      const T FUY = llf<FLUX, T>(m, 1, p1.U, p1.Y, p1.fU, p1.fY, p1.dU, p1.dY, half);
      const T FYU = llf<FLUX, T>(m, 1, p1.Y, cur.U, p1.fY, cur.fU, p1.dY, cur.dU, half);
      const T LV2 = lowres_s<T>(FXV, cur.FVX, p1.aX, p1.aV, cur.aX, kb.i2h2, kb.i4h22);
      const T LX2 = lowres_s<T>(p1.FVX, FXV, p2.aV, p1.aX, p1.aV, kb.i2h2, kb.i4h22);
      const T LY2 = lowres_s<T>(FUY, FYU, p1.aU, p1.aY, cur.aU, kb.i2h2, kb.i4h22);
      p1.rV = blendw(tmin(p1.tc1, tc1), p1.rV, p1.LV1) + blendw(tmin(tc2, tc2p), rV2, LV2);
      p1.rX = blendw(p1.tc1, p1.rX, p1.LX1) + blendw(tmin(td2, td2p), rX2, LX2);
      p1.rY = blendw(tmin(p1.td1, td1), p1.rY, p1.LY1) + blendw(tc2, rY2, LY2);
    } else {
      p1.rV = p1.rV + rV2;
      p1.rX = p1.rX + rX2;
      p1.rY = p1.rY + rY2;
    }
  }

  // ---- limiter: x-direction of row r, y-direction of row r-1
  T Flim1 = FH1, Alim1 = AH1, Flim2 = p1.FH2;
  p1.Alim2 = p1.AH2;
  if (lim) {
    // x low-order states of this cell and of both neighbours (the neighbours' formed
    // here from the shuffled values, no further shuffle round)
    auto ulp = [&](T u, T f, T a, T FLr, T ar) { return sfma(k.n4_1, ar - a, sfma(-k.m4_1, FLr - f, u)); };
    auto ulm = [&](T u, T f, T a, T FLl, T al) { return sfma(-k.n4_1, a - al, sfma(-k.m4_1, f - FLl, u)); };
    const T ULp1 = ulp(cur.U, f1U, cur.aU, FL1, aUp);
    const T ULm1 = ulm(cur.U, f1U, cur.aU, FL1m, aUm);
    const T ULm1p = ulm(Up, f1Up, aUp, FL1, cur.aU);
    const T ULp1m = ulp(Um, f1Um, aUm, FL1m, cur.aU);
    // y: low-order states u^{L,+}_{r-1} and u^{L,-}_r around the face between them
    p1.ULp2 = sfma(k.n4_2, cur.aU - p1.aU, sfma(-k.m4_2, FL2 - p1.fU, p1.U));
    cur.ULm2 = sfma(-k.n4_2, cur.aU - p1.aU, sfma(-k.m4_2, cur.fU - FL2, cur.U));
    // the twelve (low, high) pairs of the two face limiters and the two potential
    // limiters; Theta = 1 for all of them unless a high-order part leaves the bounds
    const T dF1 = FH1 - FL1, dA1 = AH1 - cur.aU, e1 = k.q1 * dA1;
    const T dF2 = p1.FH2 - FL2, dA2 = p1.AH2 - p1.aU, e2 = k.q2 * dA2;
    T zl[12] = {ULp1, ULm1p, ULp1m, ULp1, ULm1, ULm1p, p1.ULp2, cur.ULm2, p2.ULp2, p1.ULp2, p1.ULm2, cur.ULm2};
    T zh[12] = {sfma(-k.k1, dF1, ULp1), sfma(k.k1, dF1, ULm1p), ULp1m + e1, ULp1 - e1, ULm1 - e1, ULm1p + e1,
                sfma(-k.k2, dF2, p1.ULp2), sfma(k.k2, dF2, cur.ULm2), p2.ULp2 + e2, p1.ULp2 - e2, p1.ULm2 - e2,
                cur.ULm2 + e2};
    T lo = zh[0], hi = zh[0];
#pragma unroll
    for (int q = 1; q < 12; ++q) {
      lo = fmn(lo, zh[q]);
      hi = fmx(hi, zh[q]);
    }
    if (tlt(lo, k.umin) | tlt(k.umax, hi)) {
      T t[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) t[q] = theta_fn<T>(zl[q], zh[q], k.umin, k.umax);
      const T tc1 = tmin(t[0], t[1]), td1 = tmin(tmin(t[2], t[3]), tmin(t[4], t[5]));
      const T tc2 = tmin(t[6], t[7]), td2 = tmin(tmin(t[8], t[9]), tmin(t[10], t[11]));
      Flim1 = is_one(tc1) ? FH1 : sfma(tc1, dF1, FL1);
      Alim1 = is_one(td1) ? AH1 : sfma(td1, dA1, cur.aU);
      Flim2 = is_one(tc2) ? p1.FH2 : sfma(tc2, dF2, FL2);
      p1.Alim2 = is_one(td2) ? p1.AH2 : sfma(td2, dA2, p1.aU);
    }
  }
  // update terms: x-face right of (i, r); y-face between rows r-1 and r (stored with
  // the upper row); the diffusion term of that face needs A_{r}, so it is formed one
  // step later: here the y-face between rows r-2 and r-1
  const T Alim1p = shdn(Alim1);
  cur.tF1 = __fmul_rn(k.m1f, Flim1);
  cur.tD1 = __fmul_rn(k.n1f, __fsub_rn(Alim1p, Alim1));
  cur.tF2lo = __fmul_rn(k.m2f, Flim2);
  p1.tD2lo = __fmul_rn(k.n2f, __fsub_rn(p1.Alim2, p2.Alim2));

  // ---- finalise the cells of row j = r - 2
  const int j = r - 2;
  const T tF1m = shup(p2.tF1), tD1m = shup(p2.tD1);
  if (j >= c.rs && j < c.re && c.col_out) {
    const size_t g = (size_t)j * c.nx + c.gi;
    // eight face terms in stage_tile's order, summed without rounding error
    const float t[8] = {tF1m, -p2.tF1, p2.tF2lo, -p1.tF2lo, p2.tD1, -tD1m, p1.tD2lo, -p2.tD2lo};
    float hs = t[0], ls = 0.0f;
#pragma unroll
    for (int q = 1; q < 8; ++q) {
      float e;
      two_sum(hs, t[q], hs, e);
      ls = __fadd_rn(ls, e);
    }
    const double ubfe = oin.ub + (f2d_exact(hs) + f2d_exact(ls));
    T v = rk_fma(k.taut, p2.rV, p2.V), x = rk_fma(k.taut, p2.rX, p2.X), y = rk_fma(k.taut, p2.rY, p2.Y);
    if (lim) {
      v = fmn(fmx(v, k.umin), k.umax);
      x = fmn(fmx(x, k.umin), k.umax);
      y = fmn(fmx(y, k.umin), k.umax);
    }
    double ubo;
    T vo, xo, yo;
    if (c.comb) {
      ubo = rk_comb(k.cA, oin.Aub, k.cF, ubfe);
      vo = rk_comb(k.cAt, oin.V, k.cFt, v);
      xo = rk_comb(k.cAt, oin.X, k.cFt, x);
      yo = rk_comb(k.cAt, oin.Y, k.cFt, y);
    } else {
      ubo = rk_scale(k.cF, ubfe);
      vo = rk_scale(k.cFt, v);
      xo = rk_scale(k.cFt, x);
      yo = rk_scale(k.cFt, y);
    }
    // post-stage safeguard: one test for the four values, the clamp path only if needed
    if (lim && A.sg[0] &&
        (tlt(ubo, m.umin) | tlt(m.umax, ubo) | (fmn(fmn(vo, xo), yo) < k.umin) | (fmx(fmx(vo, xo), yo) > k.umax))) {
      ubo = safeguard<double>(ubo, m.umin, m.umax, A.tol, A.stats, true);
      vo = safeguard<T>(vo, k.umin, k.umax, A.tol, A.stats);
      xo = safeguard<T>(xo, k.umin, k.umax, A.tol, A.stats);
      yo = safeguard<T>(yo, k.umin, k.umax, A.tol, A.stats);
    }
    A.Oub[0][g] = ubo;
    A.OV[0][g] = vo;
    A.OX[0][g] = xo;
    A.OY[0][g] = yo;
  }
}

// One warp's march over its band and strip of rows (all 32 lanes; the single-mesh
// kernel and the batch kernel call it).
template <int FLUX, int DIFF, int BK>
__device__ __forceinline__ void stream_run(const DevModel& m, const StageArgs2D<float>& A, int S, int band,
                                           int strip) {
  using T = float;
  const double dtv = *A.dt;
  if (is_zero_bits(dtv)) return;   // uniform over the mesh
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nx = A.nx, ny = A.ny;
  const int rs = strip * S;
  if (rs >= ny) return;   // whole warp
  const int re = min(rs + S, ny);
  const int giu = band * STREAM_BAND - 2 + lane;
  // the launch's scalars, kept in shared memory (one slot per warp, so that no warp
  // waits for another): a value the compiler does not keep in a register is reloaded
  // rather than formed again on GB300's slow FP64 unit. The FP64 unit takes as long
  // for a warp instruction with one active lane as with 32, so the lanes form one
  // scalar each at once: lane l rounds fl(fl(fl(x y1) y2) y3) to FP32, the products in
  // the order of tau = tcoef dt, mu_l = tau / h_l, nu_l = mu_l / h_l and their scaled
  // copies (a factor 1 is exact, so every value is rounded as its own formula is).
  // The divided line scales come from the host (StageArgs2D::i6hf, i3h2f).
  __shared__ StreamScal<T> skw[STREAM_WPB];
  {
    const double tau = A.tcoef[0] * dtv;
    const int q = lane & 1;   // direction of lanes 0 .. 11 and 18 .. 21
    const double ih = q ? A.inv_h2 : A.inv_h1;
    double x = tau, y1 = ih, y2 = 1.0, y3 = 1.0;
    if (lane < 12) {
      const int kind = lane >> 1;   // 4 mu, 4 nu, 4 P mu, 12 nu, mu, nu
      y2 = (kind == 1 || kind == 3 || kind == 5) ? ih : (kind == 2 ? double(4 * m.lim_parts) : (kind == 0 ? 4.0 : 1.0));
      y3 = kind == 1 ? 4.0 : (kind == 3 ? 12.0 : 1.0);
    } else if (lane < 18) {
      // tau, u_min, u_max, cA, cF, gamma
      x = lane == 12 ? tau
                     : (lane == 13 ? m.umin : (lane == 14 ? m.umax : (lane == 15 ? A.cA[0] : (lane == 16 ? A.cF[0] : A.gamma))));
      y1 = 1.0;
    } else {
      // 2 / h_l and (4 / h_l) / h_l of the blend's low-order residual
      x = lane < 20 ? 2.0 : 4.0;
      y2 = lane < 20 ? 1.0 : ih;
    }
    const float v = (float)(((x * y1) * y2) * y3);
    auto at = [&](int l) { return __shfl_sync(0xffffffffu, v, l); };
    StreamScal<T> k;
    k.m4_1 = at(0);
    k.m4_2 = at(1);
    k.n4_1 = at(2);
    k.n4_2 = at(3);
    k.k1 = at(4);
    k.k2 = at(5);
    k.q1 = at(6);
    k.q2 = at(7);
    k.m1f = at(8);
    k.m2f = at(9);
    k.n1f = at(10);
    k.n2f = at(11);
    k.taut = at(12);
    k.umin = at(13);
    k.umax = at(14);
    k.cAt = at(15);
    k.cFt = at(16);
    k.i6h1 = A.i6hf[0];
    k.i6h2 = A.i6hf[1];
    k.i3h21 = A.i3h2f[0];
    k.i3h22 = A.i3h2f[1];
    k.cA = A.cA[0];
    k.cF = A.cF[0];
    k.half = T(0.5);
    k.sixth = T(1.0 / 6.0);
    k.r36 = T(1.0 / 36.0);
    k.umid = m.umid;
    if constexpr (BK != 0) {
      BlendScal b;
      b.g = at(17);
      b.i2h1 = at(18);
      b.i2h2 = at(19);
      b.i4h21 = at(20);
      b.i4h22 = at(21);
      if (lane == 0) stream_kb[wib] = b;
    }
    if (lane == 0) skw[wib] = k;
  }
  __syncwarp();
  const StreamScal<T>& k = skw[wib];
  const bool comb = !is_zero_bits(A.cA[0]);
  StreamCtx<FLUX, DIFF, T> c{m, A, k, nx, ny, wrapi(giu, nx), lane, rs, re,
                             lane >= 2 && lane < 2 + STREAM_BAND && giu < nx, comb};

  RowSlot<T> s0, s1, s2;
  // rows rs-3 .. rs-1 feed the first steps; their slots start as the wrapped row rs-3
  // so that the warm-up steps read finite values (their results are never stored)
  int gj = wrapi(rs - 3, ny);
  {
    const RowIn<T> a = load_row<T, BK>(A, (size_t)gj * nx + c.gi);
    s0 = RowSlot<T>{};
    s1 = RowSlot<T>{};
    s2 = RowSlot<T>{};
    s0.U = s1.U = s2.U = to_stencil_nb<T>(a.ub, k.umid);
    s0.V = s1.V = s2.V = a.V;
    s0.X = s1.X = s2.X = a.X;
    s0.Y = s1.Y = s2.Y = a.Y;
  }
  const int r0 = rs - 2, r1 = re + 1;   // steps r0 .. r1
  gj = gj + 1 == ny ? 0 : gj + 1;       // row r0
  RowIn<T> in = load_row<T, BK>(A, (size_t)gj * nx + c.gi);
  auto next_row = [&]() {
    gj = gj + 1 == ny ? 0 : gj + 1;
    return load_row<T, BK>(A, (size_t)gj * nx + c.gi);
  };
  // RK combination inputs of the cells finalised at step r (row r - 2)
  auto out_in = [&](int r) {
    OutIn<T> o{0.0, 0.0, T(0), T(0), T(0)};
    const int j = r - 2;
    if (j >= rs && j < re) {
      const size_t g = (size_t)j * nx + c.gi;
      o.ub = __ldg(A.ub + g);
      if (comb) {
        o.Aub = A.Aub[0][g];
        o.V = __ldg(A.AV[0] + g);
        o.X = __ldg(A.AX[0] + g);
        o.Y = __ldg(A.AY[0] + g);
      }
    }
    return o;
  };
  OutIn<T> oin = out_in(r0);
  if constexpr (BK != 0) {
    // the blended step is too large to unroll three times (the unrolled loop misses the
    // instruction cache): one step per iteration, the slots rotated by copies
#pragma unroll 1
    for (int r = r0; r <= r1; ++r) {
      const RowIn<T> nin = next_row();
      const OutIn<T> noin = out_in(r + 1);
      stream_step<FLUX, DIFF, T, BK>(c, r, in, oin, s1, s2, s0);
      const RowSlot<T> t = s1;
      s1 = s2;
      s2 = s0;
      s0 = t;
      in = nin;
      oin = noin;
    }
  } else {
    for (int r = r0; r <= r1; r += 3) {
      {
        const RowIn<T> nin = next_row();
        const OutIn<T> noin = out_in(r + 1);
        stream_step<FLUX, DIFF, T, BK>(c, r, in, oin, s1, s2, s0);
        in = nin;
        oin = noin;
      }
      if (r + 1 > r1) break;
      {
        const RowIn<T> nin = next_row();
        const OutIn<T> noin = out_in(r + 2);
        stream_step<FLUX, DIFF, T, BK>(c, r + 1, in, oin, s2, s0, s1);
        in = nin;
        oin = noin;
      }
      if (r + 2 > r1) break;
      {
        const RowIn<T> nin = next_row();
        const OutIn<T> noin = out_in(r + 3);
        stream_step<FLUX, DIFF, T, BK>(c, r + 2, in, oin, s0, s1, s2);
        in = nin;
        oin = noin;
      }
    }
  }
}

// One launch: one output of the stage (the launcher calls it once per output); warp w
// takes band w % bands and strip w / bands.
template <int FLUX, int DIFF, int BK = 0>
__global__ void __launch_bounds__(32 * STREAM_WPB, stream_min_blocks<FLUX, BK>())
    stream2d_kernel(const DevModel m, const StageArgs2D<float> A, int S, int bands) {
  const int w = blockIdx.x * STREAM_WPB + (threadIdx.x >> 5);
  stream_run<FLUX, DIFF, BK>(m, A, S, w % bands, w / bands);
}

// Plain smoothness indicator of Section 5.1.3 per cell, direction by direction
// (Section 5.2): s~_l = |u_- - 2u + u_+| / (|u_-| + 2|u| + |u_+| + 1e-13) along l, then
// s_l = (s~_{l,-1} + 4 s~_l + s~_{l,+1}) / 6, from the cell averages of the stage input
// in the stencil precision (rounded as the stage kernel rounds them), for the 32 x 8
// tile at (i0, j0) of a periodic mesh: the averages of the tile and a +-2 halo are
// converted once in shared memory. Called by all 256 threads of a CTA; compiled without
// multiply-add contraction (the column-marching translation units), so every caller
// forms the same values.
constexpr int BS_TX = 32, BS_TY = 8, BS_H = 2, BS_BX = BS_TX + 2 * BS_H, BS_BY = BS_TY + 2 * BS_H;

__device__ __forceinline__ void blend_s_tile(const double* __restrict__ ub, int nx, int ny, double umid, int i0,
                                             int j0, float* __restrict__ s1, float* __restrict__ s2) {
  __shared__ float su[BS_BY][BS_BX];
  __shared__ float st1[BS_TY][BS_TX + 2];   // s~_1 on columns -1 .. TX
  __shared__ float st2[BS_TY + 2][BS_TX];   // s~_2 on rows -1 .. TY
  for (int q = threadIdx.x; q < BS_BX * BS_BY; q += blockDim.x) {
    const int bx = q % BS_BX, by = q / BS_BX;
    const int gi = wrapi(i0 - BS_H + bx, nx), gj = wrapi(j0 - BS_H + by, ny);
    su[by][bx] = to_stencil_nb<float>(ub[(size_t)gj * nx + gi], umid);
  }
  __syncthreads();
  // the quotient with the fast approximate division (2 ulp): the indicator only sets
  // the blend weights, and the IEEE division cost this pass most of its time
  auto stl = [](float a, float b, float c) {
    return __fdividef(fabsf(a - 2.0f * b + c), fabsf(a) + 2.0f * fabsf(b) + fabsf(c) + 1e-13f);
  };
  for (int q = threadIdx.x; q < BS_TY * (BS_TX + 2); q += blockDim.x) {
    const int x = q % (BS_TX + 2), y = q / (BS_TX + 2);
    const int bx = x + BS_H - 1, by = y + BS_H;
    st1[y][x] = stl(su[by][bx - 1], su[by][bx], su[by][bx + 1]);
  }
  for (int q = threadIdx.x; q < (BS_TY + 2) * BS_TX; q += blockDim.x) {
    const int x = q % BS_TX, y = q / BS_TX;
    const int bx = x + BS_H, by = y + BS_H - 1;
    st2[y][x] = stl(su[by - 1][bx], su[by][bx], su[by + 1][bx]);
  }
  __syncthreads();
  const int x = threadIdx.x % BS_TX, y = threadIdx.x / BS_TX;
  const int gi = i0 + x, gj = j0 + y;
  if (gi < nx && gj < ny) {
    const float sixth = 1.0f / 6.0f;
    const size_t g = (size_t)gj * nx + gi;
    s1[g] = (st1[y][x] + 4.0f * st1[y][x + 1] + st1[y][x + 2]) * sixth;
    s2[g] = (st2[y][x] + 4.0f * st2[y + 1][x] + st2[y + 2][x]) * sixth;
  }
}


// ---- launch (host)

// Strip height of the column-marching kernel, at least 16 rows (the warm-up of a strip
// is 4 rows). At 16 resident warps per SM (4 CTAs): about two and a half waves, at most
// 128 rows (measured stage times, degenerate Burgers: 1024^2 S = 8/12/16:
// 0.0549/0.0544/0.0543 ms; 2048^2 S = 16/24/32/48: 0.1487/0.1451/0.1468/0.1494 ms;
// 4096^2 S = 62/96/128: 0.477/0.471/0.508 ms). The heavier kernels at 12 warps per SM
// (Buckley-Leverett, the blend) keep about four waves of 16 warps and at most 64 rows:
// the blended Buckley-Leverett stage at 4096^2 lost 4 % at S = 100 (3.3 waves, the last
// one partly filled) against S = 62.
static int stream_strip(int nx, int ny, bool heavy) {
  const long long bands = (nx + STREAM_BAND - 1) / STREAM_BAND;
  const long long target = heavy ? 152LL * 16 * 4 : 152LL * 16 * 5 / 2;
  long long S = (bands * ny + target - 1) / target;
  if (S < 16) S = 16;
  if (S > (heavy ? 64 : 128)) S = heavy ? 64 : 128;
  return (int)S;
}

// one launch per output of the stage
template <int FLUX, int DIFF, int BK = 0>
static cudaError_t stream2d_go(const DevModel& m, const StageArgs2D<float>& a, cudaStream_t s) {
  const int S = stream_strip(a.nx, a.ny, stream_min_blocks<FLUX, BK>() < 4);
  const int bands = (a.nx + STREAM_BAND - 1) / STREAM_BAND;
  const long long warps = (long long)bands * ((a.ny + S - 1) / S);
  const long long blocks = (warps + STREAM_WPB - 1) / STREAM_WPB;
  if (blocks > 0x7FFFFFFFLL) return cudaErrorInvalidConfiguration;
  for (int o = 0; o < a.nout; ++o) {
    StageArgs2D<float> b = a;
    b.nout = 1;
    b.tcoef[0] = a.tcoef[o];
    b.cA[0] = a.cA[o];
    b.cF[0] = a.cF[o];
    b.Aub[0] = a.Aub[o];
    b.AV[0] = a.AV[o];
    b.AX[0] = a.AX[o];
    b.AY[0] = a.AY[o];
    b.Oub[0] = a.Oub[o];
    b.OV[0] = a.OV[o];
    b.OX[0] = a.OX[o];
    b.OY[0] = a.OY[o];
    b.sg[0] = a.sg[o];
    stream2d_kernel<FLUX, DIFF, BK><<<(unsigned)blocks, 32 * STREAM_WPB, 0, s>>>(m, b, S, bands);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace af
