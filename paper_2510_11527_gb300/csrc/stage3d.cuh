// Stage arguments of the 3D active flux evaluation (arXiv 2510.11527, Section 4's 3D
// DoFs, Section 5.2 with d = 3). A 3D state is the FP64 cell averages plus 7 point arrays
// [nz][ny][nx] (i fastest) ordered by the kind s = sx + 2 sy + 4 sz of the location
// (i + sx/2, j + sy/2, k + sz/2): the x-face, y-face, xy-edge, z-face, xz-edge, yz-edge
// and corner values, stored as PT (FP64, or FP32 in the FP32-mixed form). Periodic in
// every direction. T is the stencil precision (T = PT).
#pragma once
#include <cuda_runtime.h>

#include "af_model.cuh"

namespace af {

template <class T>
struct StageArgs3D {
  int n[3];                          // cells per direction
  double inv_h[3];                   // 1/dx, 1/dy, 1/dz
  double i6h[3], i3h2[3];            // 1/(6 h_l), 1/(3 h_l^2)
  T inv_hT[3], i6hT[3], i3h2T[3];    // the same three, rounded to the stencil type
  const double* ub;                  // FE input: cell averages
  const T* pt[8];                    // FE input: point values by kind (pt[0] unused)
  int nout;                          // 1 or 2 limited FE evaluations of the same input
  double tcoef[2];                   // tau_k = tcoef_k * (*dt)
  double cA[2], cF[2];               // out_k = cA_k * A_k + cF_k * FE(u, tau_k)
  const double* Aub[2];
  const T* Apt[2][8];
  double* Oub[2];
  T* Opt[2][8];
  const double* dt;                  // device scalar
  int limiter;
  int blend;                         // 0 off, 1 smoothness indicator
  int sg[2];                         // per output: apply the post-stage safeguard
  double gamma;
  double tol;
  DevStats* stats;
  // scratch, n cells each: centres; per direction l the high-order face flux (upper
  // face), the DC cell potential, the low-order face flux (upper face), the smoothness
  // value s_l, and the limited face flux and cell potential
  T* C;
  T* FH[3];
  T* AH[3];
  T* FL[3];
  T* S[3];
  T* Flim[3];
  T* Alim[3];
};

}  // namespace af
