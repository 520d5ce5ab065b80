// Instantiations of the column-marching 2D stage kernel (FP32-mixed form, periodic
// meshes) without the blend; the blended ones are in stream2d_blend_f32.cu. Both
// translation units are compiled with -fmad=false: a face term is formed by two warps
// whenever the face lies on a band or strip edge (and in different copies of the
// unrolled step body), and only an arithmetic without compiler contraction makes both
// copies round alike, which conservation needs. Fused multiply-adds appear only where
// written explicitly.
#include "launch.h"
#include "stream2d.cuh"

namespace af {

// the diffusion kind is compiled in for the common kinds
template <int FLUX>
static cudaError_t stream2d_dispatch(const DevModel& m, const StageArgs2D<float>& a, cudaStream_t s) {
  switch (m.diff_kind) {
    case AF_DIFF_NONE: return stream2d_go<FLUX, DK_NONE>(m, a, s);
    case AF_DIFF_CONST: return stream2d_go<FLUX, DK_CONST>(m, a, s);
    case AF_DIFF_PWL: return stream2d_go<FLUX, DK_PWL>(m, a, s);
    case AF_DIFF_PME: return m.pme_e == 2 ? stream2d_go<FLUX, DK_PME2>(m, a, s) : stream2d_go<FLUX, DK_GENERIC>(m, a, s);
    case AF_DIFF_CUBIC: return stream2d_go<FLUX, DK_CUBIC>(m, a, s);
    default: return stream2d_go<FLUX, DK_GENERIC>(m, a, s);
  }
}

cudaError_t launch_stream2d_f32(int flux, int bk, const DevModel& m, const StageArgs2D<float>& a, cudaStream_t s) {
  if (bk != 0) return launch_stream2d_blend_f32(flux, bk, m, a, s);
  switch (flux) {
    case FLUX_ZERO: return stream2d_dispatch<FLUX_ZERO>(m, a, s);
    case FLUX_LINEAR: return stream2d_dispatch<FLUX_LINEAR>(m, a, s);
    case FLUX_BURGERS: return stream2d_dispatch<FLUX_BURGERS>(m, a, s);
    case FLUX_BL: return stream2d_dispatch<FLUX_BL>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace af
