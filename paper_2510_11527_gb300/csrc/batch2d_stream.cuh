// The batched FP32-mixed stage on the column-marching kernel (stream2d.cuh), shared by
// batch2d_stream.cu (without the blend) and batch2d_stream_blend.cu (plain or learned
// indicator): one persistent launch per stage; each warp walks a list of (instance,
// band, strip) items and marches each as the single-mesh kernel does, for every output
// of the stage. The instance's model and stage arguments are copied into the warp's
// shared slot first. The translation units are compiled with -fmad=false, like the
// single-mesh kernels, so a batched instance evolves bit for bit as the single mesh
// does.
#pragma once
#include <algorithm>

#include "batch2d.cuh"
#include "stream2d.cuh"

namespace af {

static_assert(BATCH_STREAM_BAND == STREAM_BAND, "band width of the batch items");

template <int FLUX, int DIFF, int BK>
__global__ void __launch_bounds__(32 * STREAM_WPB, stream_min_blocks<FLUX, BK>())
    batch_stream_kernel(const BatchInst* __restrict__ inst, const int* __restrict__ item_inst, int total,
                        const BatchStage St, DevStats* stats, int S) {
  __shared__ DevModel sm_m[STREAM_WPB];
  __shared__ StageArgs2D<float> sm_a[STREAM_WPB];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nw = gridDim.x * STREAM_WPB;
  for (int w = blockIdx.x * STREAM_WPB + wib; w < total; w += nw) {
    const int k = item_inst[w];
    const BatchInst& I = inst[k];
    const int local = w - I.item_begin;
    const int band = local % I.bands, strip = local / I.bands;
    for (int o = 0; o < St.nout; ++o) {
      __syncwarp();   // every lane is done with the slot's previous contents
      {
        const unsigned* src = reinterpret_cast<const unsigned*>(&I.m);
        unsigned* dst = reinterpret_cast<unsigned*>(&sm_m[wib]);
        for (int q = lane; q < (int)(sizeof(DevModel) / 4); q += 32) dst[q] = src[q];
      }
      if (lane == 0) {
        StageArgs2D<float>& A = sm_a[wib];
        const int a = St.aidx[o], d = St.out[o];
        A.nx = I.nx;
        A.ny = I.ny;
        A.inv_h1 = I.inv_h1;
        A.inv_h2 = I.inv_h2;
        A.i6hf[0] = I.i6hf[0];
        A.i6hf[1] = I.i6hf[1];
        A.i3h2f[0] = I.i3h2f[0];
        A.i3h2f[1] = I.i3h2f[1];
        A.ub = I.ub[St.in];
        A.V = (const float*)I.pv[St.in];
        A.X = (const float*)I.px[St.in];
        A.Y = (const float*)I.py[St.in];
        A.nout = 1;
        A.tcoef[0] = St.tcoef[o];
        A.cA[0] = St.cA[o];
        A.cF[0] = St.cF[o];
        A.Aub[0] = a >= 0 ? I.ub[a] : nullptr;
        A.AV[0] = a >= 0 ? (const float*)I.pv[a] : nullptr;
        A.AX[0] = a >= 0 ? (const float*)I.px[a] : nullptr;
        A.AY[0] = a >= 0 ? (const float*)I.py[a] : nullptr;
        A.Oub[0] = I.ub[d];
        A.OV[0] = (float*)I.pv[d];
        A.OX[0] = (float*)I.px[d];
        A.OY[0] = (float*)I.py[d];
        A.sg[0] = St.sg[o];
        A.dt = I.dt;
        A.s_ext = I.s;
        A.sb[0] = I.sb[0];
        A.sb[1] = I.sb[1];
        A.limiter = St.limiter;
        A.blend = St.blend;
        A.blend_external = St.blend == 2;
        A.gamma = St.gamma;
        A.tol = I.tol;
        A.stats = stats;
        A.bc = AF_BC_PERIODIC;
        A.nodc = 0;
      }
      __syncwarp();
      stream_run<FLUX, DIFF, BK>(sm_m[wib], sm_a[wib], S, band, strip);
    }
  }
}

template <int FLUX, int DIFF, int BK>
static cudaError_t batch_stream_go(const BatchInst* inst, const int* items, int total, const BatchStage& St,
                                   DevStats* stats, int S, cudaStream_t stream) {
  static int blocks = 0;
  if (!blocks) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_stream_kernel<FLUX, DIFF, BK>,
                                                                  32 * STREAM_WPB, 0);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    blocks = (per_sm > 0 ? per_sm : 1) * sms;
  }
  const int grid = std::min(blocks, (total + STREAM_WPB - 1) / STREAM_WPB);
  batch_stream_kernel<FLUX, DIFF, BK><<<grid, 32 * STREAM_WPB, 0, stream>>>(inst, items, total, St, stats, S);
  return cudaGetLastError();
}

}  // namespace af
