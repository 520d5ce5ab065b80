// Device part of the batched stage (internal): instance and stage descriptors and the
// persistent tile-walking stage kernels, shared by the translation units that
// instantiate them (batch2d.cu without the blend, batch2d_blend.cu with it).
#pragma once
#include <cuda_runtime.h>

#include "af.h"
#include "stage2d.cuh"

namespace af {

constexpr int BATCH_STREAM_BAND = 28;   // output columns per warp of the column-marching kernel

struct BatchInst {
  DevModel m;
  int nx, ny;
  double inv_h1, inv_h2, inv_hmin2, kmax, tol;
  double i6h[2], i3h2[2];        // 1/(6 h_l), (1/h_l^2)/3 (line scales)
  float i6hf[2], i3h2f[2];       // the same in FP32
  int tile_begin, tiles_x;       // first work item of this instance, tiles along x
  int item_begin, bands;         // column-marching items: first item, bands of 28 columns
  int ind_begin;                 // first 32 x 8 tile of the indicators' launches
  double* s;                     // learned indicator per cell (blend with the network)
  float* sb[2];                  // plain indicator s_1, s_2 per cell (FP32-mixed blend)
  double* ub[4];
  void* pv[4];
  void* px[4];
  void* py[4];
  double* dt;                    // this instance's step
  double* t;                     // this instance's time
};

struct BatchStage {              // uniform over the batch for one launch
  int in, nout;
  int out[2], aidx[2], sg[2];
  double cA[2], cF[2], tcoef[2];
  int limiter;
  int blend;                     // smoothness-indicator blend (Section 5.1.3): 0 off, 1 plain,
                                 // 2 the learned indicator (BatchInst::s)
  double gamma;
};

template <int FLUX, class T, class PT, int TX, int TY, bool BLEND>
__device__ __forceinline__ void batch_stage_body(const BatchInst* __restrict__ inst,
                                                 const int* __restrict__ work_inst, int total, const BatchStage& S,
                                                 DevStats* stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the tile's arguments live in shared memory, written by one thread: a per-thread
  // copy would sit in local memory (its arrays are indexed at run time)
  __shared__ StageArgs2D<PT> A;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const BatchInst& I = inst[work_inst[w]];
    const int t = w - I.tile_begin;
    const int i0 = (t % I.tiles_x) * TX, j0 = (t / I.tiles_x) * TY;
    if (threadIdx.x == 0) {
    A.nx = I.nx;
    A.ny = I.ny;
    A.inv_h1 = I.inv_h1;
    A.inv_h2 = I.inv_h2;
    for (int l = 0; l < 2; ++l) {
      A.i6h[l] = I.i6h[l];
      A.i3h2[l] = I.i3h2[l];
      A.i6hf[l] = I.i6hf[l];
      A.i3h2f[l] = I.i3h2f[l];
    }
    A.ub = I.ub[S.in];
    A.V = (const PT*)I.pv[S.in];
    A.X = (const PT*)I.px[S.in];
    A.Y = (const PT*)I.py[S.in];
    A.nout = S.nout;
    for (int o = 0; o < 2; ++o) {
      const int a = S.aidx[o], d = S.out[o];
      A.tcoef[o] = S.tcoef[o];
      A.cA[o] = S.cA[o];
      A.cF[o] = S.cF[o];
      A.Aub[o] = a >= 0 ? I.ub[a] : nullptr;
      A.AV[o] = a >= 0 ? (const PT*)I.pv[a] : nullptr;
      A.AX[o] = a >= 0 ? (const PT*)I.px[a] : nullptr;
      A.AY[o] = a >= 0 ? (const PT*)I.py[a] : nullptr;
      A.Oub[o] = d >= 0 ? I.ub[d] : nullptr;
      A.OV[o] = d >= 0 ? (PT*)I.pv[d] : nullptr;
      A.OX[o] = d >= 0 ? (PT*)I.px[d] : nullptr;
      A.OY[o] = d >= 0 ? (PT*)I.py[d] : nullptr;
      A.sg[o] = S.sg[o];
    }
    A.dt = I.dt;
    A.s_ext = I.s;
    A.limiter = S.limiter;
    A.blend = S.blend;
    A.blend_external = S.blend == 2;
    A.gamma = S.gamma;
    A.tol = I.tol;
    A.stats = stats;
    A.bc = AF_BC_PERIODIC;
    A.nodc = 0;
    }
    __syncthreads();
    // element-wise halo loads: the paired path's extra registers spill in this kernel
    stage_tile<FLUX, T, PT, BLEND, TX, TY, false>(I.m, A, i0, j0, smem_raw);
    __syncthreads();
  }
}

// FP64 stencils (and the blended FP32 ones): 72.6 KB of shared memory per CTA leave
// room for 3 CTAs per SM, which the registers must not undercut (<= 80 per thread)
template <int FLUX, class T, class PT, int TX, int TY, bool BLEND>
__global__ void __launch_bounds__(256, 3) batch_stage_kernel(const BatchInst* __restrict__ inst,
                                                          const int* __restrict__ work_inst, int total,
                                                          const BatchStage S, DevStats* stats) {
  batch_stage_body<FLUX, T, PT, TX, TY, BLEND>(inst, work_inst, total, S, stats);
}

// FP32 stencils: compiled for 6 resident CTAs per SM (measured 8% faster than the
// compiler's 64-register choice at 4 CTAs per SM, despite a few spilled words)
template <int FLUX, int TX, int TY>
__global__ void __launch_bounds__(256, 6) batch_stage_kernel_f32occ6(const BatchInst* __restrict__ inst,
                                                                     const int* __restrict__ work_inst, int total,
                                                                     const BatchStage S, DevStats* stats) {
  batch_stage_body<FLUX, float, float, TX, TY, false>(inst, work_inst, total, S, stats);
}

// The blended FP64 stage kernels (instantiated in batch2d_blend.cu): one persistent
// launch (the occupancy limit times the SM count) for tile shape tx x ty; prec must be
// AF_PREC_FP64 (the FP32-mixed batch blends on the column-marching items).
cudaError_t batch_launch_blend(int prec, int flux, int tx, int ty, const BatchInst* inst, const int* work, int total,
                               const BatchStage& S, DevStats* stats, cudaStream_t stream);

// The FP32-mixed stage without the blend on the column-marching kernel
// (batch2d_stream.cu): `total` (instance, band, strip) items of strips of S rows; diff
// the diffusion kind all instances share (pme_e its PME exponent), -1 if they differ.
cudaError_t batch_launch_stream(int flux, int diff, int pme_e, const BatchInst* inst, const int* items, int total,
                                const BatchStage& St, DevStats* stats, int S, cudaStream_t s);

// The FP32-mixed stage with the blend on the column-marching kernel
// (batch2d_stream_blend.cu): bk 1 the plain indicator (BatchInst::sb, formed first by
// batch_launch_blend_s from the same input), bk 2 the learned one (BatchInst::s); diff
// as for batch_launch_stream (AF_DIFF_CUBIC compiled in, any other kind read per
// instance).
cudaError_t batch_launch_stream_blend(int flux, int bk, int diff, const BatchInst* inst, const int* items, int total,
                                      const BatchStage& St, DevStats* stats, int S, cudaStream_t s);
// The plain indicator of every instance's state buffer `in` into its arrays sb: `total`
// 32 x 8 tiles, instance k's from inst[k].ind_begin on.
cudaError_t batch_launch_blend_s(const BatchInst* inst, int n, int total, int in, cudaStream_t s);

// The learned indicator (mlp.cu) of every instance's state buffer `in` into its array
// s: `total` 32 x 8 tiles, instance k's from inst[k].ind_begin on; prec AF_PREC_*.
cudaError_t mlp_indicator_batch_launch(const af_mlp* net, const BatchInst* inst, int n, int total, int in, int prec,
                                       cudaStream_t s);

}  // namespace af
