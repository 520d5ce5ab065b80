// Learned smoothness indicator for the blend of Section 5.1.3 / 5.2 of arXiv
// 2510.11527: a 21 -> 32 -> 32 -> 1 network maps a normalised patch of cell averages and
// point values around a cell to s >= 0, which replaces the smoothness indicator s in
// theta^{c,s} = exp(-gamma s_face), theta^{d,s} = exp(-gamma s). The MPP limiter and the
// projection still run after it, so bounds and conservation do not depend on it.
//
// Kernels:
//   indicator (fused inference): gather + normalise the patch, two bf16 tensor-core
//     layers (mma.sync m16n8k16, FP32 accumulate, layer-1 accumulators reused as layer-2
//     A fragments), FP32 output layer, softplus; one warp per 16 cells.
//   features: training data (the same patch in FP32) and the plain indicator's label.
//   train: per-sample FP32 forward (same bf16 rounding points as the tensor-core path)
//     and backward, gradients accumulated per CTA in shared memory.
//   adam: Adam update of the FP32 master weights and refresh of their bf16 copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "af.h"
#include "batch2d.cuh"
#include "ctx.h"

namespace {

constexpr int NIN = 21, NH = 32;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH, NPARAM = OFF_B3 + 1;   // 1793
static_assert(NPARAM == AF_MLP_NPARAM, "parameter count");

// periodic index for offsets of a few cells (one compare each way; the modulo only on
// meshes smaller than the offset)
__device__ __forceinline__ int wrapm(int i, int n) {
  if (i < 0) {
    i += n;
    if (i < 0) {
      i %= n;
      if (i < 0) i += n;
    }
  } else if (i >= n) {
    i -= n;
    if (i >= n) i %= n;
  }
  return i;
}

// FP32 copies of state values without the FP64 unit (truncating, as the stage kernels)
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(double x) { return af::to_stencil<float>(x); }

// normalised patch from values in FP32: (v_k - v_4) / (max_k |v_k| + 1e-13), v_4 being
// the cell's own average
__device__ __forceinline__ void normalise(const float v[NIN], float f[NIN]) {
  float sc = 0.0f;
#pragma unroll
  for (int k = 0; k < NIN; ++k) sc = fmaxf(sc, fabsf(v[k]));
  const float r = 1.0f / (sc + 1e-13f), m = v[4];
#pragma unroll
  for (int k = 0; k < NIN; ++k) f[k] = (v[k] - m) * r;
}

// normalised patch of cell (i, j) in FP32: (v_k - ub_ij) / (max_k |v_k| + 1e-13)
template <class PT>
__device__ __forceinline__ void gather(const double* __restrict__ ub, const PT* __restrict__ V,
                                       const PT* __restrict__ X, const PT* __restrict__ Y, int nx, int ny, int i,
                                       int j, float f[NIN]) {
  // patch offsets of the 13 cell averages (a along x, b along y)
  constexpr int kPatchA[13] = {-1, 0, 1, -1, 0, 1, -1, 0, 1, -2, 2, 0, 0};
  constexpr int kPatchB[13] = {-1, -1, -1, 0, 0, 0, 1, 1, 1, 0, 0, -2, 2};
  float v[NIN];
  // wrapped columns i-2..i+2 and row offsets j-2..j+2, formed once
  int ci[5];
  size_t rj[5];
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    ci[d] = wrapm(i + d - 2, nx);
    rj[d] = (size_t)wrapm(j + d - 2, ny) * nx;
  }
#pragma unroll
  for (int k = 0; k < 13; ++k) v[k] = af::to_stencil<float>(ub[rj[kPatchB[k] + 2] + ci[kPatchA[k] + 2]]);
  const int im = ci[1], jm = wrapm(j - 1, ny);
  const size_t c = (size_t)j * nx + i;
  v[13] = to_f32(V[(size_t)jm * nx + im]);
  v[14] = to_f32(V[(size_t)jm * nx + i]);
  v[15] = to_f32(V[(size_t)j * nx + im]);
  v[16] = to_f32(V[c]);
  v[17] = to_f32(X[(size_t)j * nx + im]);
  v[18] = to_f32(X[c]);
  v[19] = to_f32(Y[(size_t)jm * nx + i]);
  v[20] = to_f32(Y[c]);
  normalise(v, f);
}

__device__ __forceinline__ float softplusf(float z) { return z > 20.0f ? z : log1pf(expf(z)); }

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&p);
}

// Tensor-core network on 16 rows held (bf16, [16][40]) in shared memory; returns the
// output pre-activation z (s = softplus(z)) of rows g and g + 8 in all four lanes of
// quad g.
struct NetFrags {
  uint32_t b1[2][4][2], b2[2][4][2];
  float bias1[4][2], bias2[4][2], w3[4][2], b3;
};

__device__ __forceinline__ void load_frags(NetFrags& F, const __nv_bfloat16* w1q, const __nv_bfloat16* w2q,
                                           const float* params, int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int kb = 0; kb < 2; ++kb)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int n = 8 * nt + g, k0 = 16 * kb + 2 * t;
      F.b1[kb][nt][0] = *reinterpret_cast<const uint32_t*>(w1q + n * 32 + k0);
      F.b1[kb][nt][1] = *reinterpret_cast<const uint32_t*>(w1q + n * 32 + k0 + 8);
      F.b2[kb][nt][0] = *reinterpret_cast<const uint32_t*>(w2q + n * 32 + k0);
      F.b2[kb][nt][1] = *reinterpret_cast<const uint32_t*>(w2q + n * 32 + k0 + 8);
    }
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int col = 8 * nt + 2 * t + e;
      F.bias1[nt][e] = params[OFF_B1 + col];
      F.bias2[nt][e] = params[OFF_B2 + col];
      F.w3[nt][e] = params[OFF_W3 + col];
    }
  F.b3 = params[OFF_B3];
}

__device__ __forceinline__ void net_rows(const NetFrags& F, const __nv_bfloat16 (*sx)[40], int lane, float* s0,
                                         float* s8) {
  const int g = lane >> 2, t = lane & 3;
  float c1[4][4];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) c1[nt][0] = c1[nt][1] = c1[nt][2] = c1[nt][3] = 0.0f;
#pragma unroll
  for (int kb = 0; kb < 2; ++kb) {
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t*>(&sx[g][16 * kb + 2 * t]);
    a[1] = *reinterpret_cast<const uint32_t*>(&sx[g + 8][16 * kb + 2 * t]);
    a[2] = *reinterpret_cast<const uint32_t*>(&sx[g][16 * kb + 2 * t + 8]);
    a[3] = *reinterpret_cast<const uint32_t*>(&sx[g + 8][16 * kb + 2 * t + 8]);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) mma16816(c1[nt], a, F.b1[kb][nt]);
  }
  // bias + ReLU, rounded to bf16: the layer-1 accumulator tiles 2kb, 2kb+1 are exactly
  // the A fragment of layer-2 k-block kb
  uint32_t a2[2][4];
#pragma unroll
  for (int kb = 0; kb < 2; ++kb) {
    const int n0 = 2 * kb, n1 = 2 * kb + 1;
    a2[kb][0] = pack_bf16(fmaxf(c1[n0][0] + F.bias1[n0][0], 0.f), fmaxf(c1[n0][1] + F.bias1[n0][1], 0.f));
    a2[kb][1] = pack_bf16(fmaxf(c1[n0][2] + F.bias1[n0][0], 0.f), fmaxf(c1[n0][3] + F.bias1[n0][1], 0.f));
    a2[kb][2] = pack_bf16(fmaxf(c1[n1][0] + F.bias1[n1][0], 0.f), fmaxf(c1[n1][1] + F.bias1[n1][1], 0.f));
    a2[kb][3] = pack_bf16(fmaxf(c1[n1][2] + F.bias1[n1][0], 0.f), fmaxf(c1[n1][3] + F.bias1[n1][1], 0.f));
  }
  float c2[4][4];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) c2[nt][0] = c2[nt][1] = c2[nt][2] = c2[nt][3] = 0.0f;
#pragma unroll
  for (int kb = 0; kb < 2; ++kb)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) mma16816(c2[nt], a2[kb], F.b2[kb][nt]);
  float r0 = 0.f, r8 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      r0 += F.w3[nt][e] * fmaxf(c2[nt][e] + F.bias2[nt][e], 0.f);
      r8 += F.w3[nt][e] * fmaxf(c2[nt][2 + e] + F.bias2[nt][e], 0.f);
    }
  r0 += __shfl_xor_sync(0xffffffffu, r0, 1);
  r0 += __shfl_xor_sync(0xffffffffu, r0, 2);
  r8 += __shfl_xor_sync(0xffffffffu, r8, 1);
  r8 += __shfl_xor_sync(0xffffffffu, r8, 2);
  (void)t;
  *s0 = r0 + F.b3;
  *s8 = r8 + F.b3;
}

// Fused inference on a state, s (double) per cell. Each CTA takes 32 x 8 tiles of
// cells: the tile's cell averages with a +-2 halo and its point values with a -1 halo
// are staged in shared memory (coalesced row loads, converted to FP32 once), every lane
// builds the patch of one cell from there, and each warp runs the network on its 32
// patches as two 16-row blocks.
// Resident CTAs per SM the indicator kernel is compiled for (3: 85 registers, the
// weight fragments partly spilled; 2: 122 registers, no spill).
#ifndef AF_INDICATOR_MIN_CTAS
#define AF_INDICATOR_MIN_CTAS 3
#endif

// One 32 x 8 tile (cells i0 .. i0 + 31, j0 .. j0 + 7) of a periodic mesh: the patches
// are gathered into shared memory, each warp runs the network on its row of 32 cells
// and writes s. Called by all 256 threads of the CTA, which it leaves synchronised.
template <class PT>
__device__ __forceinline__ void indicator_tile(const NetFrags& F, const double* __restrict__ ub,
                                               const PT* __restrict__ V, const PT* __restrict__ X,
                                               const PT* __restrict__ Y, int nx, int ny, int i0, int j0,
                                               double* __restrict__ out) {
  constexpr int UX = 36, UY = 12, PX = 33, PY = 9;
  constexpr int kPatchA[13] = {-1, 0, 1, -1, 0, 1, -1, 0, 1, -2, 2, 0, 0};
  constexpr int kPatchB[13] = {-1, -1, -1, 0, 0, 0, 1, 1, 1, 0, 0, -2, 2};
  __shared__ float sU[UY][UX];
  __shared__ float sV[PY][PX], sX[PY][PX], sY[PY][PX];
  __shared__ __align__(16) __nv_bfloat16 sx[8][32][40];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {
    for (int k = tid; k < UX * UY; k += 256) {
      const int bx = k % UX, by = k / UX;
      sU[by][bx] = af::to_stencil<float>(ub[(size_t)wrapm(j0 - 2 + by, ny) * nx + wrapm(i0 - 2 + bx, nx)]);
    }
    for (int k = tid; k < PX * PY; k += 256) {
      const int bx = k % PX, by = k / PX;
      const size_t g = (size_t)wrapm(j0 - 1 + by, ny) * nx + wrapm(i0 - 1 + bx, nx);
      sV[by][bx] = to_f32(V[g]);
      sX[by][bx] = to_f32(X[g]);
      sY[by][bx] = to_f32(Y[g]);
    }
    __syncthreads();
    {
      // cell (i0 + lane, j0 + warp)
      const int tx = lane, ty = warp;
      float v[NIN], f[NIN];
#pragma unroll
      for (int k = 0; k < 13; ++k) v[k] = sU[ty + 2 + kPatchB[k]][tx + 2 + kPatchA[k]];
      v[13] = sV[ty][tx];
      v[14] = sV[ty][tx + 1];
      v[15] = sV[ty + 1][tx];
      v[16] = sV[ty + 1][tx + 1];
      v[17] = sX[ty + 1][tx];
      v[18] = sX[ty + 1][tx + 1];
      v[19] = sY[ty][tx + 1];
      v[20] = sY[ty + 1][tx + 1];
      normalise(v, f);
#pragma unroll
      for (int k = 0; k < 32; k += 2)
        *reinterpret_cast<uint32_t*>(&sx[warp][lane][k]) =
            pack_bf16(k < NIN ? f[k] : 0.f, k + 1 < NIN ? f[k + 1] : 0.f);
    }
    __syncwarp();
    const int j = j0 + warp;
    float z[2][2];
#pragma unroll
    for (int h = 0; h < 2; ++h) net_rows(F, sx[warp] + 16 * h, lane, &z[h][0], &z[h][1]);
    {
      // the four lanes of a quad share the four pre-activations (rows g, g + 8 of both
      // 16-row blocks): each applies the output activation to one of them
      const int t = lane & 3, h = t >> 1, w = t & 1;
      const float s = softplusf(z[h][w]);
      const int i = i0 + 16 * h + (lane >> 2) + 8 * w;
      if (j < ny && i < nx) out[(size_t)j * nx + i] = af::f2d_exact(s);
    }
    __syncthreads();
  }
}

template <class PT>
__global__ void __launch_bounds__(256, AF_INDICATOR_MIN_CTAS) indicator_kernel(const double* __restrict__ ub, const PT* __restrict__ V,
                                                           const PT* __restrict__ X, const PT* __restrict__ Y, int nx,
                                                           int ny, const __nv_bfloat16* __restrict__ w1q,
                                                           const __nv_bfloat16* __restrict__ w2q,
                                                           const float* __restrict__ params, double* __restrict__ out) {
  NetFrags F;
  load_frags(F, w1q, w2q, params, threadIdx.x & 31);
  const int tiles_x = (nx + 31) / 32, tiles = tiles_x * ((ny + 7) / 8);
  for (int t = blockIdx.x; t < tiles; t += gridDim.x)
    indicator_tile<PT>(F, ub, V, X, Y, nx, ny, (t % tiles_x) * 32, (t / tiles_x) * 8, out);
}

// The same over every instance of a batch (state buffer `in` of each, s into its
// indicator array): the 32 x 8 tiles of instance k are numbered from inst[k].ind_begin
// on, so a tile's instance is found by bisection.
template <class PT>
__global__ void __launch_bounds__(256, AF_INDICATOR_MIN_CTAS)
    indicator_batch_kernel(const af::BatchInst* __restrict__ inst, int n, int total, int in,
                           const __nv_bfloat16* __restrict__ w1q, const __nv_bfloat16* __restrict__ w2q,
                           const float* __restrict__ params) {
  NetFrags F;
  load_frags(F, w1q, w2q, params, threadIdx.x & 31);
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    int lo = 0, hi = n - 1;   // the last instance whose first tile is <= w
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (inst[mid].ind_begin <= w) lo = mid;
      else hi = mid - 1;
    }
    const af::BatchInst& I = inst[lo];
    const int t = w - I.ind_begin, tiles_x = (I.nx + 31) / 32;
    indicator_tile<PT>(F, I.ub[in], (const PT*)I.pv[in], (const PT*)I.px[in], (const PT*)I.py[in], I.nx, I.ny,
                       (t % tiles_x) * 32, (t / tiles_x) * 8, I.s);
  }
}

// network on given FP32 feature rows (n x 21) -> out (n)
__global__ void __launch_bounds__(256) infer_rows_kernel(const float* __restrict__ feat, long long n,
                                                         const __nv_bfloat16* __restrict__ w1q,
                                                         const __nv_bfloat16* __restrict__ w2q,
                                                         const float* __restrict__ params, float* __restrict__ out) {
  __shared__ __align__(16) __nv_bfloat16 sx[8][16][40];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  NetFrags F;
  load_frags(F, w1q, w2q, params, lane);
  for (long long base = ((long long)blockIdx.x * 8 + warp) * 16; base < n; base += (long long)gridDim.x * 128) {
    if (lane < 16) {
      const long long row = base + lane;
#pragma unroll
      for (int k = 0; k < 32; k += 2) {
        const float lo = (row < n && k < NIN) ? feat[row * NIN + k] : 0.f;
        const float hi = (row < n && k + 1 < NIN) ? feat[row * NIN + k + 1] : 0.f;
        *reinterpret_cast<uint32_t*>(&sx[warp][lane][k]) = pack_bf16(lo, hi);
      }
    }
    __syncwarp();
    float z0, z8;
    net_rows(F, sx[warp], lane, &z0, &z8);
    // lanes t = 0, 1 of each quad apply the output activation to rows g, g + 8
    const int t = lane & 3;
    if (t < 2) {
      const long long row = base + (lane >> 2) + 8 * t;
      const float s = softplusf(t ? z8 : z0);
      if (row < n) out[row] = s;
    }
    __syncwarp();
  }
}

// training data: FP32 patch and the plain indicator max(s_1, s_2) (FP64) per cell
template <class PT>
__global__ void features_kernel(const double* __restrict__ ub, const PT* __restrict__ V, const PT* __restrict__ X,
                                const PT* __restrict__ Y, int nx, int ny, float* __restrict__ feat,
                                float* __restrict__ label) {
  const long long n = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)(c / nx);
    float f[NIN];
    gather<PT>(ub, V, X, Y, nx, ny, i, j, f);
#pragma unroll
    for (int k = 0; k < NIN; ++k) feat[c * NIN + k] = f[k];
    if (label) {
      auto U = [&](int a, int b) { return ub[(size_t)wrapm(j + b, ny) * nx + wrapm(i + a, nx)]; };
      auto st = [](double um, double uc, double up) {
        return fabs(um - 2.0 * uc + up) / (fabs(um) + 2.0 * fabs(uc) + fabs(up) + 1e-13);
      };
      const double s1 = (st(U(-2, 0), U(-1, 0), U(0, 0)) + 4.0 * st(U(-1, 0), U(0, 0), U(1, 0)) +
                         st(U(0, 0), U(1, 0), U(2, 0))) / 6.0;
      const double s2 = (st(U(0, -2), U(0, -1), U(0, 0)) + 4.0 * st(U(0, -1), U(0, 0), U(0, 1)) +
                         st(U(0, 0), U(0, 1), U(0, 2))) / 6.0;
      label[c] = (float)fmax(s1, s2);
    }
  }
}

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// per-sample forward + backward in FP32 with the tensor-core path's rounding points
// (bf16 inputs and weights of the two hidden layers); gradient of the batch-mean loss
// accumulated into grad, loss into loss_acc. sample k of the batch is k itself when
// seed == 0, else a splitmix64 draw over [0, nsamples).
__global__ void __launch_bounds__(256) train_kernel(const float* __restrict__ feat, const float* __restrict__ label,
                                                    long long nsamples, int batch, unsigned long long seed, int step,
                                                    const float* __restrict__ params, float* __restrict__ grad,
                                                    float* __restrict__ loss_acc) {
  __shared__ float W1[NH * NIN], W2[NH * NH], b1[NH], b2[NH], w3[NH];
  __shared__ float G[NPARAM];
  __shared__ float b3s;
  for (int k = threadIdx.x; k < NH * NIN; k += blockDim.x) W1[k] = bfr(params[OFF_W1 + k]);
  for (int k = threadIdx.x; k < NH * NH; k += blockDim.x) W2[k] = bfr(params[OFF_W2 + k]);
  for (int k = threadIdx.x; k < NH; k += blockDim.x) {
    b1[k] = params[OFF_B1 + k];
    b2[k] = params[OFF_B2 + k];
    w3[k] = params[OFF_W3 + k];
  }
  if (threadIdx.x == 0) b3s = params[OFF_B3];
  for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) G[k] = 0.f;
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  float lossv = 0.f;
  if (k < batch) {
    long long idx = seed == 0 ? k
                              : (long long)(splitmix64(seed ^ ((unsigned long long)step << 32) ^ (unsigned long long)k) %
                                            (unsigned long long)nsamples);
    float x[NIN], z1[NH], h1[NH], z2[NH];
    for (int q = 0; q < NIN; ++q) x[q] = bfr(feat[idx * NIN + q]);
    for (int o = 0; o < NH; ++o) {
      float a = 0.f;
      for (int q = 0; q < NIN; ++q) a = fmaf(W1[o * NIN + q], x[q], a);
      z1[o] = a + b1[o];
      h1[o] = bfr(fmaxf(z1[o], 0.f));
    }
    float z3 = 0.f;
    for (int o = 0; o < NH; ++o) {
      float a = 0.f;
      for (int q = 0; q < NH; ++q) a = fmaf(W2[o * NH + q], h1[q], a);
      z2[o] = a + b2[o];
      z3 = fmaf(w3[o], fmaxf(z2[o], 0.f), z3);
    }
    z3 += b3s;
    const float out = softplusf(z3), r = out - label[idx];
    lossv = r * r / (float)batch;
    const float dz3 = 2.f / (float)batch * r / (1.f + expf(-z3));
    atomicAdd(&G[OFF_B3], dz3);
    float dh1[NH];
    for (int q = 0; q < NH; ++q) dh1[q] = 0.f;
    for (int o = 0; o < NH; ++o) {
      atomicAdd(&G[OFF_W3 + o], dz3 * fmaxf(z2[o], 0.f));
      if (z2[o] > 0.f) {
        const float dz2 = dz3 * w3[o];
        atomicAdd(&G[OFF_B2 + o], dz2);
        for (int q = 0; q < NH; ++q) {
          atomicAdd(&G[OFF_W2 + o * NH + q], dz2 * h1[q]);
          dh1[q] = fmaf(dz2, W2[o * NH + q], dh1[q]);
        }
      }
    }
    for (int q = 0; q < NH; ++q) {
      if (z1[q] > 0.f) {
        const float dz1 = dh1[q];
        atomicAdd(&G[OFF_B1 + q], dz1);
        for (int p = 0; p < NIN; ++p) atomicAdd(&G[OFF_W1 + q * NIN + p], dz1 * x[p]);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) lossv += __shfl_xor_sync(0xffffffffu, lossv, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, lossv);
  __syncthreads();
  for (int q = threadIdx.x; q < NPARAM; q += blockDim.x) atomicAdd(&grad[q], G[q]);
}

// Adam on the FP32 master weights; refreshes the bf16 copies and clears the gradient
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            float* __restrict__ grad, float lr, float c1, float c2, __nv_bfloat16* w1q,
                            __nv_bfloat16* w2q) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NPARAM) return;
  const float g = grad[q];
  const float mq = 0.9f * m[q] + 0.1f * g, vq = 0.999f * v[q] + 0.001f * g * g;
  m[q] = mq;
  v[q] = vq;
  const float w = p[q] - lr * (mq / c1) / (sqrtf(vq / c2) + 1e-8f);
  p[q] = w;
  grad[q] = 0.f;
  if (q < OFF_B1) w1q[(q / NIN) * 32 + q % NIN] = __float2bfloat16_rn(w);
  else if (q >= OFF_W2 && q < OFF_B2) w2q[q - OFF_W2] = __float2bfloat16_rn(w);
}

__global__ void quantize_kernel(const float* __restrict__ p, __nv_bfloat16* w1q, __nv_bfloat16* w2q) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 32 * 32) {
    const int n = q / 32, k = q % 32;
    w1q[q] = __float2bfloat16_rn(k < NIN ? p[OFF_W1 + n * NIN + k] : 0.f);
    w2q[q] = __float2bfloat16_rn(p[OFF_W2 + q]);
  }
}

}  // namespace

struct af_mlp {
  unsigned char* block = nullptr;
  float* params = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  float* loss = nullptr;
  __nv_bfloat16* w1q = nullptr;
  __nv_bfloat16* w2q = nullptr;
  int t = 0;
  cudaStream_t stream = nullptr;
};

namespace af {
cudaError_t mlp_indicator_launch(const af_ctx* c, const af_mlp* net, int buf, double* out) {
  if (c->dim != 2) return cudaErrorInvalidValue;
  const long long tiles = (long long)((c->nx + 31) / 32) * ((c->ny + 7) / 8);
  const int grid = (int)std::min<long long>(tiles, 152LL * AF_INDICATOR_MIN_CTAS);
  if (c->prec == AF_PREC_FP64)
    indicator_kernel<double><<<grid, 256, 0, c->stream>>>(c->ub[buf], (const double*)c->pv[buf],
                                                          (const double*)c->px[buf], (const double*)c->py[buf],
                                                          c->nx, c->ny, net->w1q, net->w2q, net->params, out);
  else
    indicator_kernel<float><<<grid, 256, 0, c->stream>>>(c->ub[buf], (const float*)c->pv[buf],
                                                         (const float*)c->px[buf], (const float*)c->py[buf], c->nx,
                                                         c->ny, net->w1q, net->w2q, net->params, out);
  return cudaGetLastError();
}

cudaError_t mlp_indicator_batch_launch(const af_mlp* net, const BatchInst* inst, int n, int total, int in, int prec,
                                       cudaStream_t s) {
  if (total < 1 || n < 1) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(total, 152LL * AF_INDICATOR_MIN_CTAS);
  if (prec == AF_PREC_FP64)
    indicator_batch_kernel<double><<<grid, 256, 0, s>>>(inst, n, total, in, net->w1q, net->w2q, net->params);
  else
    indicator_batch_kernel<float><<<grid, 256, 0, s>>>(inst, n, total, in, net->w1q, net->w2q, net->params);
  return cudaGetLastError();
}
}  // namespace af

extern "C" {

af_status af_mlp_create(af_mlp** out) {
  if (!out) return AF_E_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return AF_E_UNSUPPORTED;
  af_mlp* net = new (std::nothrow) af_mlp;
  if (!net) return AF_E_OOM;
  const size_t bytes = 4 * 1024 * 5 * sizeof(float) + 2 * 32 * 32 * sizeof(__nv_bfloat16) + 256;
  if (cudaMalloc(&net->block, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete net;
    return AF_E_OOM;
  }
  cudaMemset(net->block, 0, bytes);
  float* f = (float*)net->block;
  net->params = f;
  net->m = f + 2048;
  net->v = f + 4096;
  net->grad = f + 6144;
  net->loss = f + 8192;
  net->w1q = (__nv_bfloat16*)(f + 10240);
  net->w2q = net->w1q + 32 * 32;
  *out = net;
  return AF_OK;
}

af_status af_mlp_destroy(af_mlp* net) {
  if (!net) return AF_E_ARG;
  cudaDeviceSynchronize();
  cudaFree(net->block);
  delete net;
  return AF_OK;
}

af_status af_mlp_set_params(af_mlp* net, const float* host, int n) {
  if (!net || !host || n != NPARAM) return AF_E_ARG;
  if (cudaMemcpy(net->params, host, NPARAM * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return AF_E_CUDA;
  cudaMemset(net->m, 0, NPARAM * sizeof(float));
  cudaMemset(net->v, 0, NPARAM * sizeof(float));
  cudaMemset(net->grad, 0, NPARAM * sizeof(float));
  net->t = 0;
  quantize_kernel<<<4, 256>>>(net->params, net->w1q, net->w2q);
  return cudaDeviceSynchronize() == cudaSuccess ? AF_OK : AF_E_CUDA;
}

af_status af_mlp_get_params(const af_mlp* net, float* host) {
  if (!net || !host) return AF_E_ARG;
  return cudaMemcpy(host, net->params, NPARAM * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? AF_OK
                                                                                                      : AF_E_CUDA;
}

af_status af_mlp_features(af_ctx* c, float* feat_dev, float* label_dev) {
  if (!c || !feat_dev || c->dim != 2 || c->bounds_pending) return AF_E_ARG;
  const int grid = (int)std::min<size_t>((c->n + 255) / 256, 152 * 32);
  if (c->prec == AF_PREC_FP64)
    features_kernel<double><<<grid, 256, 0, c->stream>>>(c->ub[0], (const double*)c->pv[0], (const double*)c->px[0],
                                                         (const double*)c->py[0], c->nx, c->ny, feat_dev, label_dev);
  else
    features_kernel<float><<<grid, 256, 0, c->stream>>>(c->ub[0], (const float*)c->pv[0], (const float*)c->px[0],
                                                        (const float*)c->py[0], c->nx, c->ny, feat_dev, label_dev);
  if (cudaGetLastError() != cudaSuccess) return AF_E_CUDA;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? AF_OK : AF_E_CUDA;
}

af_status af_mlp_infer(const af_mlp* net, const float* feat_dev, long long n, float* out_dev) {
  if (!net || !feat_dev || !out_dev || n < 1) return AF_E_ARG;
  const int grid = (int)std::min<long long>((n + 127) / 128, 152 * 16);
  infer_rows_kernel<<<grid, 256>>>(feat_dev, n, net->w1q, net->w2q, net->params, out_dev);
  if (cudaGetLastError() != cudaSuccess) return AF_E_CUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? AF_OK : AF_E_CUDA;
}

af_status af_mlp_indicator(const af_mlp* net, af_ctx* c, double* s_dev) {
  if (!net || !c || !s_dev || c->dim != 2 || c->bounds_pending) return AF_E_ARG;
  if (af::mlp_indicator_launch(c, net, 0, s_dev) != cudaSuccess) return AF_E_CUDA;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? AF_OK : AF_E_CUDA;
}

af_status af_mlp_grad(af_mlp* net, const float* feat_dev, const float* label_dev, int nsamples, float* grad_host,
                      float* loss_host) {
  if (!net || !feat_dev || !label_dev || nsamples < 1) return AF_E_ARG;
  cudaMemset(net->grad, 0, NPARAM * sizeof(float));
  cudaMemset(net->loss, 0, sizeof(float));
  train_kernel<<<(nsamples + 255) / 256, 256>>>(feat_dev, label_dev, nsamples, nsamples, 0ull, 0, net->params,
                                               net->grad, net->loss);
  if (cudaGetLastError() != cudaSuccess) return AF_E_CUDA;
  if (grad_host && cudaMemcpy(grad_host, net->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return AF_E_CUDA;
  if (loss_host && cudaMemcpy(loss_host, net->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return AF_E_CUDA;
  cudaMemset(net->grad, 0, NPARAM * sizeof(float));
  return AF_OK;
}

af_status af_mlp_train(af_mlp* net, const float* feat_dev, const float* label_dev, long long nsamples, int batch,
                       int steps, float lr, unsigned long long seed, float* loss_host) {
  if (!net || !feat_dev || !label_dev || nsamples < 1 || batch < 1 || steps < 0 || !(lr > 0.f)) return AF_E_ARG;
  if (seed == 0 && batch > nsamples) return AF_E_ARG;   // seed 0: rows 0..batch-1 in order
  float last = 0.f;
  for (int s = 0; s < steps; ++s) {
    cudaMemset(net->loss, 0, sizeof(float));
    train_kernel<<<(batch + 255) / 256, 256>>>(feat_dev, label_dev, nsamples, batch, seed, s,
                                               net->params, net->grad, net->loss);
    net->t += 1;
    const float c1 = 1.f - powf(0.9f, (float)net->t), c2 = 1.f - powf(0.999f, (float)net->t);
    adam_kernel<<<(NPARAM + 255) / 256, 256>>>(net->params, net->m, net->v, net->grad, lr, c1, c2, net->w1q,
                                                net->w2q);
    if (cudaGetLastError() != cudaSuccess) return AF_E_CUDA;
    if (s == steps - 1 && loss_host) {
      if (cudaMemcpy(&last, net->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return AF_E_CUDA;
      *loss_host = last;
    }
  }
  return cudaDeviceSynchronize() == cudaSuccess ? AF_OK : AF_E_CUDA;
}

af_status af_set_mlp(af_ctx* c, const af_mlp* net) {
  if (!c) return AF_E_ARG;
  if (net && (c->dim != 2 || c->opts.blend != AF_BLEND_EXTERNAL)) return AF_E_ARG;
  c->mlp = net;
  return AF_OK;
}

}  // extern "C"
