// Instantiations of the fused 2D stage kernel on rectangles with outflow ends (padded
// layout, reflected ghost loads, masked stores), FP64 and FP32-mixed forms.
#include "stage2d_launch.cuh"

namespace af {

cudaError_t launch_stage2d_rect_f64(int flux, bool blend, const DevModel& m, const StageArgs2D<double>& a,
                                    cudaStream_t s) {
  return stage2d_dispatch<double, true>(flux, blend, m, a, s);
}
cudaError_t launch_stage2d_rect_f32(int flux, bool blend, const DevModel& m, const StageArgs2D<float>& a,
                                    cudaStream_t s) {
  return stage2d_dispatch<float, true>(flux, blend, m, a, s);
}

}  // namespace af
