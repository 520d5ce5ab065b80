// Instantiations of the fused 2D stage kernel, FP64 form (all DoFs and stencils FP64).
#include "launch.h"

namespace af {

template <int FLUX, bool BLEND>
static cudaError_t go(const DevModel& m, const StageArgs2D<double>& a, cudaStream_t s) {
  using L = Tile2D<FLUX, double, BLEND>;
  static bool attr = false;
  auto k = stage2d_kernel<FLUX, double, double, BLEND>;
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

cudaError_t launch_stage2d_f64(int flux, bool blend, const DevModel& m, const StageArgs2D<double>& a,
                               cudaStream_t s) {
  switch (flux) {
    case FLUX_ZERO: return blend ? go<FLUX_ZERO, true>(m, a, s) : go<FLUX_ZERO, false>(m, a, s);
    case FLUX_LINEAR: return blend ? go<FLUX_LINEAR, true>(m, a, s) : go<FLUX_LINEAR, false>(m, a, s);
    case FLUX_BURGERS: return blend ? go<FLUX_BURGERS, true>(m, a, s) : go<FLUX_BURGERS, false>(m, a, s);
    case FLUX_BL: return blend ? go<FLUX_BL, true>(m, a, s) : go<FLUX_BL, false>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace af
