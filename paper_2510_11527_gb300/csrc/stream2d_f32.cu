// Instantiations of the column-marching 2D stage kernel (FP32-mixed form, periodic
// meshes without the blend). This translation unit is compiled with -fmad=false: a face
// term is formed by two warps whenever the face lies on a band or strip edge (and in
// different copies of the unrolled step body), and only an arithmetic without compiler
// contraction makes both copies round alike, which conservation needs. Fused
// multiply-adds appear only where written explicitly, in values formed once per
// output (the point residuals and the point update).
#include "launch.h"
#include "stream2d.cuh"

namespace af {

// Strip height of the column-marching kernel: about four waves of 16 resident warps
// per SM, at least 16 rows (the warm-up of a strip is 4 rows) and at most 64 (measured
// on 1024^2 to 4096^2 meshes).
static int stream_strip(int nx, int ny) {
  const long long bands = (nx + STREAM_BAND - 1) / STREAM_BAND;
  const long long target = 152LL * 16 * 4;
  long long S = (bands * ny + target - 1) / target;
  if (S < 16) S = 16;
  if (S > 64) S = 64;
  return (int)S;
}

// one launch per output of the stage
template <int FLUX, int DIFF>
static cudaError_t stream2d_go(const DevModel& m, const StageArgs2D<float>& a, cudaStream_t s) {
  const int S = stream_strip(a.nx, a.ny);
  const int bands = (a.nx + STREAM_BAND - 1) / STREAM_BAND;
  const long long warps = (long long)bands * ((a.ny + S - 1) / S);
  const long long blocks = (warps + STREAM_WPB - 1) / STREAM_WPB;
  if (blocks > 0x7FFFFFFFLL) return cudaErrorInvalidConfiguration;
  for (int o = 0; o < a.nout; ++o) {
    StageArgs2D<float> b = a;
    b.nout = 1;
    b.tcoef[0] = a.tcoef[o];
    b.cA[0] = a.cA[o];
    b.cF[0] = a.cF[o];
    b.Aub[0] = a.Aub[o];
    b.AV[0] = a.AV[o];
    b.AX[0] = a.AX[o];
    b.AY[0] = a.AY[o];
    b.Oub[0] = a.Oub[o];
    b.OV[0] = a.OV[o];
    b.OX[0] = a.OX[o];
    b.OY[0] = a.OY[o];
    b.sg[0] = a.sg[o];
    stream2d_kernel<FLUX, DIFF><<<(unsigned)blocks, 32 * STREAM_WPB, 0, s>>>(m, b, S, bands);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

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

cudaError_t launch_stream2d_f32(int flux, const DevModel& m, const StageArgs2D<float>& a, cudaStream_t s) {
  switch (flux) {
    case FLUX_ZERO: return stream2d_dispatch<FLUX_ZERO>(m, a, s);
    case FLUX_LINEAR: return stream2d_dispatch<FLUX_LINEAR>(m, a, s);
    case FLUX_BURGERS: return stream2d_dispatch<FLUX_BURGERS>(m, a, s);
    case FLUX_BL: return stream2d_dispatch<FLUX_BL>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace af
