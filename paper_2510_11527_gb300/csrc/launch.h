// Internal launch helpers shared by the translation units of libaf (not installed).
#pragma once
#include <cuda_runtime.h>

#include "reduce.cuh"
#include "stage2d.cuh"
#include "stage3d.cuh"

namespace af {

cudaError_t launch_stage2d_f64(int flux, bool blend, const DevModel& m, const StageArgs2D<double>& a,
                               cudaStream_t s);
cudaError_t launch_stage2d_f32(int flux, bool blend, const DevModel& m, const StageArgs2D<float>& a,
                               cudaStream_t s);
// bk: 0 no blend, 1 smoothness blend with the plain indicator, 2 with the external one
cudaError_t launch_stream2d_f32(int flux, int bk, const DevModel& m, const StageArgs2D<float>& a, cudaStream_t s);
cudaError_t launch_stream2d_blend_f32(int flux, int bk, const DevModel& m, const StageArgs2D<float>& a,
                                      cudaStream_t s);
cudaError_t launch_stage2d_rect_f64(int flux, bool blend, const DevModel& m, const StageArgs2D<double>& a,
                                    cudaStream_t s);
cudaError_t launch_stage2d_rect_f32(int flux, bool blend, const DevModel& m, const StageArgs2D<float>& a,
                                    cudaStream_t s);
cudaError_t launch_stage3d_f64(int flux, const DevModel& m, const StageArgs3D<double>& a, cudaStream_t s);
cudaError_t launch_stage3d_f32(int flux, const DevModel& m, const StageArgs3D<float>& a, cudaStream_t s);
cudaError_t launch_rate3d(int flux, const DevModel& m, const int* n, const double* ub, const double* inv_h, double kmax,
                          unsigned long long* rate_bits, cudaStream_t s);
cudaError_t launch_stage1d_f64(int flux, const DevModel& m, const StageArgs2D<double>& a, cudaStream_t s);
cudaError_t launch_stage1d_f32(int flux, const DevModel& m, const StageArgs2D<float>& a, cudaStream_t s);

}  // namespace af
