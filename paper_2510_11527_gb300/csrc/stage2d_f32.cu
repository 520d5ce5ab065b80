// Instantiations of the fused 2D stage kernel on periodic meshes, FP32-mixed form (FP32
// point values and stencil arithmetic, FP64 cell averages and update).
#include "stage2d_launch.cuh"

namespace af {

cudaError_t launch_stage2d_f32(int flux, bool blend, const DevModel& m, const StageArgs2D<float>& a,
                               cudaStream_t s) {
  return stage2d_dispatch<float, false>(flux, blend, m, a, s);
}

}  // namespace af
