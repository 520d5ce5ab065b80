// Instantiations of the fused 2D stage kernel on periodic meshes, FP64 form (all DoFs and
// stencils FP64).
#include "stage2d_launch.cuh"

namespace af {

cudaError_t launch_stage2d_f64(int flux, bool blend, const DevModel& m, const StageArgs2D<double>& a,
                               cudaStream_t s) {
  return stage2d_dispatch<double, false>(flux, blend, m, a, s);
}

}  // namespace af
