// Launchers of the fused 2D stage kernels (internal). The FP32-mixed form of a periodic
// mesh runs the column-marching kernel (stream2d.cuh), with or without the blend. The
// others run one CTA per 32 x 8 tile of the mesh, or of the padded layout of a
// rectangle with ends (RECT): the FP64 form and the blended FP32 rectangle
// stage2d_kernel, the FP32 rectangle without the blend the 6-CTAs-per-SM compilation. The translation units instantiate
// the periodic (RECT = false) and the rectangle (RECT = true) launchers separately, so
// they compile in parallel and the periodic kernels are unaffected by the rectangle's
// code.
#pragma once
#include <type_traits>

#include "launch.h"

namespace af {

template <int FLUX, class T, bool BLEND, bool RECT>
static auto stage2d_kernel_for() {
  if constexpr (std::is_same_v<T, float> && !BLEND) return stage2d_kernel_f32occ6<FLUX, RECT>;
  else return stage2d_kernel<FLUX, T, T, BLEND, RECT>;
}

template <int FLUX, class T, bool BLEND, bool RECT>
static cudaError_t stage2d_go(const DevModel& m, const StageArgs2D<T>& a, cudaStream_t s) {
  if constexpr (std::is_same_v<T, float> && !RECT)
    return launch_stream2d_f32(FLUX, BLEND ? (a.blend_external ? 2 : 1) : 0, m, a, s);
  using L = Tile2D<FLUX, T, BLEND>;
  static bool attr = false;
  auto k = stage2d_kernel_for<FLUX, T, BLEND, RECT>();
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long tiles = (long long)((a.nx + L::TX - 1) / L::TX) * ((a.ny + L::TY - 1) / L::TY);
  if (tiles > 0x7FFFFFFFLL) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)tiles);
  k<<<grid, L::NT, L::SMEM, s>>>(m, a);
  return cudaGetLastError();
}

template <class T, bool RECT>
static cudaError_t stage2d_dispatch(int flux, bool blend, const DevModel& m, const StageArgs2D<T>& a,
                                    cudaStream_t s) {
  switch (flux) {
    case FLUX_ZERO: return blend ? stage2d_go<FLUX_ZERO, T, true, RECT>(m, a, s) : stage2d_go<FLUX_ZERO, T, false, RECT>(m, a, s);
    case FLUX_LINEAR:
      return blend ? stage2d_go<FLUX_LINEAR, T, true, RECT>(m, a, s) : stage2d_go<FLUX_LINEAR, T, false, RECT>(m, a, s);
    case FLUX_BURGERS:
      return blend ? stage2d_go<FLUX_BURGERS, T, true, RECT>(m, a, s) : stage2d_go<FLUX_BURGERS, T, false, RECT>(m, a, s);
    case FLUX_BL: return blend ? stage2d_go<FLUX_BL, T, true, RECT>(m, a, s) : stage2d_go<FLUX_BL, T, false, RECT>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace af
