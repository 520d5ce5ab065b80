// Batched FP32-mixed stage with the smoothness blend on the column-marching kernel (see
// batch2d_stream.cuh): bk 1, the plain indicator of Section 5.1.3, formed per stage for
// every instance by blend_s_batch_kernel into its two FP32 arrays; bk 2, the learned
// indicator (BatchInst::s, formed by the batched inference). Compiled with -fmad=false,
// like stream2d_blend_f32.cu, so the indicator and the stage are the single mesh's.
#include "batch2d_stream.cuh"
#include "launch.h"

namespace af {

// The plain indicator of state buffer `in` of every instance into its arrays sb[0],
// sb[1]: the 32 x 8 tiles of instance k are numbered from inst[k].ind_begin on (the
// numbering of the learned inference), so a tile's instance is found by bisection.
__global__ void __launch_bounds__(256) blend_s_batch_kernel(const BatchInst* __restrict__ inst, int n, int total,
                                                            int in) {
  static_assert(BS_TX == 32 && BS_TY == 8, "tiles of the batch's indicator numbering");
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    int lo = 0, hi = n - 1;   // the last instance whose first tile is <= w
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (inst[mid].ind_begin <= w) lo = mid;
      else hi = mid - 1;
    }
    const BatchInst& I = inst[lo];
    const int t = w - I.ind_begin, tiles_x = (I.nx + BS_TX - 1) / BS_TX;
    blend_s_tile(I.ub[in], I.nx, I.ny, I.m.umid, (t % tiles_x) * BS_TX, (t / tiles_x) * BS_TY, I.sb[0], I.sb[1]);
  }
}

cudaError_t batch_launch_blend_s(const BatchInst* inst, int n, int total, int in, cudaStream_t s) {
  if (n < 1 || total < 1) return cudaErrorInvalidValue;
  const int grid = std::min(total, 152 * 8);
  blend_s_batch_kernel<<<grid, 256, 0, s>>>(inst, n, total, in);
  return cudaGetLastError();
}

// the diffusion kind: compiled in for the cubic potential shared by every instance
// (Buckley-Leverett), else each instance's runtime kind (as on a single mesh)
template <int FLUX, int BK>
static cudaError_t batch_stream_blend_diff(int diff, const BatchInst* inst, const int* items, int total,
                                           const BatchStage& St, DevStats* stats, int S, cudaStream_t s) {
  if (diff == AF_DIFF_CUBIC) return batch_stream_go<FLUX, DK_CUBIC, BK>(inst, items, total, St, stats, S, s);
  return batch_stream_go<FLUX, DK_GENERIC, BK>(inst, items, total, St, stats, S, s);
}

template <int BK>
static cudaError_t batch_stream_blend_flux(int flux, int diff, const BatchInst* inst, const int* items, int total,
                                           const BatchStage& St, DevStats* stats, int S, cudaStream_t s) {
  switch (flux) {
    case FLUX_ZERO: return batch_stream_blend_diff<FLUX_ZERO, BK>(diff, inst, items, total, St, stats, S, s);
    case FLUX_LINEAR: return batch_stream_blend_diff<FLUX_LINEAR, BK>(diff, inst, items, total, St, stats, S, s);
    case FLUX_BURGERS: return batch_stream_blend_diff<FLUX_BURGERS, BK>(diff, inst, items, total, St, stats, S, s);
    case FLUX_BL: return batch_stream_blend_diff<FLUX_BL, BK>(diff, inst, items, total, St, stats, S, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_launch_stream_blend(int flux, int bk, int diff, const BatchInst* inst, const int* items, int total,
                                      const BatchStage& St, DevStats* stats, int S, cudaStream_t s) {
  if (bk == 1) return batch_stream_blend_flux<1>(flux, diff, inst, items, total, St, stats, S, s);
  if (bk == 2) return batch_stream_blend_flux<2>(flux, diff, inst, items, total, St, stats, S, s);
  return cudaErrorInvalidValue;
}

}  // namespace af
