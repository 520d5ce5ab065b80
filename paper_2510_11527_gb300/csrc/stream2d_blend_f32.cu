// The column-marching 2D stage kernel with the smoothness blend (FP32-mixed form,
// periodic meshes; compiled with -fmad=false like stream2d_f32.cu, for the same
// reason), and the pass that forms the plain indicator for it.
#include "launch.h"
#include "stream2d.cuh"

namespace af {

__global__ void __launch_bounds__(256) blend_s_kernel(const double* __restrict__ ub, int nx, int ny, double umid,
                                                      float* __restrict__ s1, float* __restrict__ s2) {
  const int tiles_x = (nx + BS_TX - 1) / BS_TX;
  blend_s_tile(ub, nx, ny, umid, (blockIdx.x % tiles_x) * BS_TX, (blockIdx.x / tiles_x) * BS_TY, s1, s2);
}

// the diffusion kind: compiled in for the cubic potential (Buckley-Leverett), else the
// model's runtime kind
template <int FLUX, int BK>
static cudaError_t stream2d_blend_dispatch(const DevModel& m, const StageArgs2D<float>& a, cudaStream_t s) {
  if (m.diff_kind == AF_DIFF_CUBIC) return stream2d_go<FLUX, DK_CUBIC, BK>(m, a, s);
  return stream2d_go<FLUX, DK_GENERIC, BK>(m, a, s);
}

template <int BK>
static cudaError_t stream2d_blend_flux(int flux, const DevModel& m, const StageArgs2D<float>& a, cudaStream_t s) {
  switch (flux) {
    case FLUX_ZERO: return stream2d_blend_dispatch<FLUX_ZERO, BK>(m, a, s);
    case FLUX_LINEAR: return stream2d_blend_dispatch<FLUX_LINEAR, BK>(m, a, s);
    case FLUX_BURGERS: return stream2d_blend_dispatch<FLUX_BURGERS, BK>(m, a, s);
    case FLUX_BL: return stream2d_blend_dispatch<FLUX_BL, BK>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

// bk 1: the plain indicator, formed first into a.sb[0], a.sb[1] (two FP32 arrays of
// nx * ny); bk 2: the external indicator a.s_ext (one FP64 value per cell)
cudaError_t launch_stream2d_blend_f32(int flux, int bk, const DevModel& m, const StageArgs2D<float>& a,
                                      cudaStream_t s) {
  if (bk == 1) {
    if (!a.sb[0] || !a.sb[1]) return cudaErrorInvalidValue;
    const long long tiles = (long long)((a.nx + BS_TX - 1) / BS_TX) * ((a.ny + BS_TY - 1) / BS_TY);
    if (tiles > 0x7FFFFFFFLL) return cudaErrorInvalidConfiguration;
    blend_s_kernel<<<(unsigned)tiles, 256, 0, s>>>(a.ub, a.nx, a.ny, m.umid,
                                                   const_cast<float*>(a.sb[0]), const_cast<float*>(a.sb[1]));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return stream2d_blend_flux<1>(flux, m, a, s);
  }
  if (bk == 2) {
    if (!a.s_ext) return cudaErrorInvalidValue;
    return stream2d_blend_flux<2>(flux, m, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace af
