// Internal definition of af_ctx (single-mesh solver context), shared by the
// translation units of libaf. Not installed.
#pragma once
#include <cuda_runtime.h>

#include "af.h"
#include "af_model.cuh"

struct af_ctx {
  af_grid grid;
  af_flux flux;
  af_diff diff;
  af_bounds_t bnd;
  af_opts opts;
  af::DevModel m;
  int dim = 2, nx = 1, ny = 1, prec = AF_PREC_FP64, nbuf = 3;
  size_t n = 0;
  size_t np = 0;                      // point values per point array (n, or n + 1 on a bounded 1D interval)
  // device layout: a 2D rectangle with outflow ends is stored padded, (nx + 1) x (ny + 1)
  // entries per array, padded cell (I, J) holding the average of cell (I - 1, J - 1) and
  // the corner V, vertical-edge X and horizontal-edge Y values at its top-right; row 0
  // and column 0 hold the bottom / left side points (the averages there, X in row 0
  // and Y in column 0 are not DoFs). Otherwise pnx = nx, pny = ny.
  int pnx = 1, pny = 1;
  // 3D: cells along z, the 8 arrays of each buffer by kind (k3[b][0] == ub[b]; points
  // in the context's precision) and the stage scratch (centres; per direction FH, AH,
  // FL, s, limited F and A)
  int nz = 1;
  double dz = 1, inv_h3 = 0;
  void* k3[4][8] = {};                // [b][0]: FP64 averages; [b][1..7]: points (FP64 or FP32)
  void* scr3[19] = {};                // stencil precision
  size_t pn = 0;                      // pnx * pny entries per device array (1D: max(n, np))
  double dx = 1, dy = 1, inv_h1 = 1, inv_h2 = 1, kmax = 0, cfl = 0.165, cfl_diff = 0, tol = 0;
  bool bounds_pending = false;
  unsigned char* block = nullptr;     // one allocation for every device buffer
  double* ub[4] = {nullptr, nullptr, nullptr, nullptr};
  void* pv[4] = {nullptr, nullptr, nullptr, nullptr};
  void* px[4] = {nullptr, nullptr, nullptr, nullptr};
  void* py[4] = {nullptr, nullptr, nullptr, nullptr};
  double* dt_dev = nullptr;
  double* t_dev = nullptr;
  double* red = nullptr;              // 8 reduction result slots
  double* partial = nullptr;          // RED_MAX_BLOCKS partials
  unsigned long long* rate_bits = nullptr;
  af::DevStats* stats = nullptr;
  double* s_ext = nullptr;            // n doubles
  const double* s_ext_user = nullptr; // caller-provided device indicator
  double* host_pinned = nullptr;      // 8 doubles for small read-backs
  const struct af_mlp* mlp = nullptr; // learned indicator run before every stage
  cudaStream_t stream = nullptr;
  char err[512] = {0};
};

namespace af {
// Fused learned-indicator inference on state buffer `buf` of the context into out
// (n doubles); defined with the network kernels.
cudaError_t mlp_indicator_launch(const af_ctx* c, const struct af_mlp* net, int buf, double* out);
}  // namespace af
