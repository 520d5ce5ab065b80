// Instantiations of the batched FP64 stage with the smoothness-indicator blend (Section
// 5.1.3) on the tile kernel, kept in their own translation unit so that they compile in
// parallel with the rest of the batch code. (The FP32-mixed batch runs the blend on the
// column-marching items, batch2d_stream_blend.cu.)
#include <algorithm>

#include "batch2d.cuh"

namespace af {
namespace {

template <int FLUX, class T, int TX, int TY>
cudaError_t go(const BatchInst* inst, const int* work, int total, const BatchStage& S, DevStats* stats,
               cudaStream_t stream) {
  using L = Tile2D<FLUX, T, true, TX, TY>;
  auto k = batch_stage_kernel<FLUX, T, T, TX, TY, true>;
  static int blocks = 0;
  if (!blocks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, L::SMEM);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    blocks = std::max(1, per_sm) * sms;
  }
  const int grid = std::min(blocks, total);
  k<<<grid, 256, L::SMEM, stream>>>(inst, work, total, S, stats);
  return cudaGetLastError();
}

template <int FLUX, class T>
cudaError_t shape(int tx, int ty, const BatchInst* inst, const int* work, int total, const BatchStage& S,
                  DevStats* stats, cudaStream_t stream) {
  if (tx == 32 && ty == 8) return go<FLUX, T, 32, 8>(inst, work, total, S, stats, stream);
  if (tx == 64 && ty == 4) return go<FLUX, T, 64, 4>(inst, work, total, S, stats, stream);
  if (tx == 16 && ty == 16) return go<FLUX, T, 16, 16>(inst, work, total, S, stats, stream);
  return cudaErrorInvalidValue;
}

template <class T>
cudaError_t flux(int fk, int tx, int ty, const BatchInst* inst, const int* work, int total, const BatchStage& S,
                 DevStats* stats, cudaStream_t stream) {
  switch (fk) {
    case AF_FLUX_ZERO: return shape<FLUX_ZERO, T>(tx, ty, inst, work, total, S, stats, stream);
    case AF_FLUX_LINEAR: return shape<FLUX_LINEAR, T>(tx, ty, inst, work, total, S, stats, stream);
    case AF_FLUX_BURGERS: return shape<FLUX_BURGERS, T>(tx, ty, inst, work, total, S, stats, stream);
    default: return shape<FLUX_BL, T>(tx, ty, inst, work, total, S, stats, stream);
  }
}

}  // namespace

cudaError_t batch_launch_blend(int prec, int fk, int tx, int ty, const BatchInst* inst, const int* work, int total,
                               const BatchStage& S, DevStats* stats, cudaStream_t stream) {
  if (prec != AF_PREC_FP64) return cudaErrorInvalidValue;
  return flux<double>(fk, tx, ty, inst, work, total, S, stats, stream);
}

}  // namespace af
