// Instantiations of the fused 1D stage kernel (FP64 and FP32-mixed forms).
#include "launch.h"
#include "stage1d.cuh"

namespace af {

template <int FLUX, class T, class PT>
static cudaError_t go1(const DevModel& m, const StageArgs2D<PT>& a, cudaStream_t s) {
  using L = Tile1D<FLUX, T>;
  dim3 grid((a.nx + L::TX - 1) / L::TX);
  stage1d_kernel<FLUX, T, PT><<<grid, L::NT, 0, s>>>(m, a);
  return cudaGetLastError();
}

template <class T, class PT>
static cudaError_t disp(int flux, const DevModel& m, const StageArgs2D<PT>& a, cudaStream_t s) {
  switch (flux) {
    case FLUX_ZERO: return go1<FLUX_ZERO, T, PT>(m, a, s);
    case FLUX_LINEAR: return go1<FLUX_LINEAR, T, PT>(m, a, s);
    case FLUX_BURGERS: return go1<FLUX_BURGERS, T, PT>(m, a, s);
    case FLUX_BL: return go1<FLUX_BL, T, PT>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stage1d_f64(int flux, const DevModel& m, const StageArgs2D<double>& a, cudaStream_t s) {
  return disp<double, double>(flux, m, a, s);
}
cudaError_t launch_stage1d_f32(int flux, const DevModel& m, const StageArgs2D<float>& a, cudaStream_t s) {
  return disp<float, float>(flux, m, a, s);
}

}  // namespace af
