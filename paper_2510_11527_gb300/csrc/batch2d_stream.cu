// Batched FP32-mixed stage without the blend on the column-marching kernel (see
// batch2d_stream.cuh). Compiled with -fmad=false, like stream2d_f32.cu.
#include "batch2d_stream.cuh"
#include "launch.h"

namespace af {

// diff: the diffusion kind shared by every instance (AF_DIFF_*; pme_e its PME exponent),
// or -1 when they differ (the model's runtime kind is then read per instance)
template <int FLUX>
static cudaError_t batch_stream_diff(int diff, int pme_e, const BatchInst* inst, const int* items, int total,
                                     const BatchStage& St, DevStats* stats, int S, cudaStream_t s) {
  switch (diff) {
    case AF_DIFF_NONE: return batch_stream_go<FLUX, DK_NONE, 0>(inst, items, total, St, stats, S, s);
    case AF_DIFF_CONST: return batch_stream_go<FLUX, DK_CONST, 0>(inst, items, total, St, stats, S, s);
    case AF_DIFF_PWL: return batch_stream_go<FLUX, DK_PWL, 0>(inst, items, total, St, stats, S, s);
    case AF_DIFF_PME:
      return pme_e == 2 ? batch_stream_go<FLUX, DK_PME2, 0>(inst, items, total, St, stats, S, s)
                        : batch_stream_go<FLUX, DK_GENERIC, 0>(inst, items, total, St, stats, S, s);
    case AF_DIFF_CUBIC: return batch_stream_go<FLUX, DK_CUBIC, 0>(inst, items, total, St, stats, S, s);
    default: return batch_stream_go<FLUX, DK_GENERIC, 0>(inst, items, total, St, stats, S, s);
  }
}

cudaError_t batch_launch_stream(int flux, int diff, int pme_e, const BatchInst* inst, const int* items, int total,
                                const BatchStage& St, DevStats* stats, int S, cudaStream_t s) {
  switch (flux) {
    case FLUX_ZERO: return batch_stream_diff<FLUX_ZERO>(diff, pme_e, inst, items, total, St, stats, S, s);
    case FLUX_LINEAR: return batch_stream_diff<FLUX_LINEAR>(diff, pme_e, inst, items, total, St, stats, S, s);
    case FLUX_BURGERS: return batch_stream_diff<FLUX_BURGERS>(diff, pme_e, inst, items, total, St, stats, S, s);
    case FLUX_BL: return batch_stream_diff<FLUX_BL>(diff, pme_e, inst, items, total, St, stats, S, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace af
