// The column-marching 2D stage kernel with the smoothness blend (FP32-mixed form,
// periodic meshes; compiled with -fmad=false like stream2d_f32.cu, for the same
// reason), and the pass that forms the plain indicator for it.
#include "launch.h"
#include "stream2d.cuh"

namespace af {

// Plain smoothness indicator of Section 5.1.3 per cell, direction by direction
// (Section 5.2): s~_l = |u_- - 2u + u_+| / (|u_-| + 2|u| + |u_+| + 1e-13) along l, then
// s_l = (s~_{l,-1} + 4 s~_l + s~_{l,+1}) / 6, from the cell averages of the stage input
// in the stencil precision (rounded as the stage kernel rounds them). One CTA per 32 x 8
// tile: the averages of the tile and a +-2 halo are converted once in shared memory.
constexpr int BS_TX = 32, BS_TY = 8, BS_H = 2, BS_BX = BS_TX + 2 * BS_H, BS_BY = BS_TY + 2 * BS_H;

__global__ void __launch_bounds__(256) blend_s_kernel(const double* __restrict__ ub, int nx, int ny, double umid,
                                                      float* __restrict__ s1, float* __restrict__ s2) {
  __shared__ float su[BS_BY][BS_BX];
  __shared__ float st1[BS_TY][BS_TX + 2];   // s~_1 on columns -1 .. TX
  __shared__ float st2[BS_TY + 2][BS_TX];   // s~_2 on rows -1 .. TY
  const int tiles_x = (nx + BS_TX - 1) / BS_TX;
  const int i0 = (blockIdx.x % tiles_x) * BS_TX, j0 = (blockIdx.x / tiles_x) * BS_TY;
  for (int q = threadIdx.x; q < BS_BX * BS_BY; q += blockDim.x) {
    const int bx = q % BS_BX, by = q / BS_BX;
    const int gi = wrapi(i0 - BS_H + bx, nx), gj = wrapi(j0 - BS_H + by, ny);
    su[by][bx] = to_stencil_nb<float>(ub[(size_t)gj * nx + gi], umid);
  }
  __syncthreads();
  // the quotient with the fast approximate division (2 ulp): the indicator only sets
  // the blend weights, and the IEEE division cost this pass most of its time
  auto stl = [](float a, float b, float c) {
    return __fdividef(fabsf(a - 2.0f * b + c), fabsf(a) + 2.0f * fabsf(b) + fabsf(c) + 1e-13f);
  };
  for (int q = threadIdx.x; q < BS_TY * (BS_TX + 2); q += blockDim.x) {
    const int x = q % (BS_TX + 2), y = q / (BS_TX + 2);
    const int bx = x + BS_H - 1, by = y + BS_H;
    st1[y][x] = stl(su[by][bx - 1], su[by][bx], su[by][bx + 1]);
  }
  for (int q = threadIdx.x; q < (BS_TY + 2) * BS_TX; q += blockDim.x) {
    const int x = q % BS_TX, y = q / BS_TX;
    const int bx = x + BS_H, by = y + BS_H - 1;
    st2[y][x] = stl(su[by - 1][bx], su[by][bx], su[by + 1][bx]);
  }
  __syncthreads();
  const int x = threadIdx.x % BS_TX, y = threadIdx.x / BS_TX;
  const int gi = i0 + x, gj = j0 + y;
  if (gi < nx && gj < ny) {
    const float sixth = 1.0f / 6.0f;
    const size_t g = (size_t)gj * nx + gi;
    s1[g] = (st1[y][x] + 4.0f * st1[y][x + 1] + st1[y][x + 2]) * sixth;
    s2[g] = (st2[y][x] + 4.0f * st2[y + 1][x] + st2[y + 2][x]) * sixth;
  }
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
