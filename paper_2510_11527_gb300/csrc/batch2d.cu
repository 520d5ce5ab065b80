// Batched execution of many independent periodic 2D meshes (uneven sizes and
// coefficients) of the active flux method (arXiv 2510.11527): one persistent launch per
// SSP-RK stage walks a list of (instance, tile) work items with the same tile body as
// the single-mesh kernel; per-instance CFL steps stay on the device; a whole time step
// (CFL reduction + stages) is captured once as a CUDA graph and replayed. The tile
// shape is a template parameter chosen by an autotuner that times the candidates on
// the batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "af.h"
#include "model_host.h"
#include "reduce.cuh"
#include "batch2d.cuh"

namespace af {

// per-tile part of the CFL rate for the Buckley-Leverett flux (see dt_rate_kernel) into
// rate_bits[2 instance] and the interior-extremum flags of f_l' into
// rate_bits[2 instance + 1]; the other fluxes take batch_rate_maxu_kernel
template <int FLUX, int TX, int TY>
__global__ void __launch_bounds__(256) batch_rate_kernel(const BatchInst* __restrict__ inst,
                                                         const int* __restrict__ work_inst, int total, int in,
                                                         unsigned long long* rate_bits) {
  __shared__ double sm[8];
  __shared__ unsigned sf[8];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int k = work_inst[w];
    const BatchInst& I = inst[k];
    const int t = w - I.tile_begin;
    const int i = (t % I.tiles_x) * TX + (int)threadIdx.x % TX, j = (t / I.tiles_x) * TY + (int)threadIdx.x / TX;
    double best = 0.0;
    unsigned flags = 0u;
    if (i < I.nx && j < I.ny) {
      const double* ub = I.ub[in];
      const double u = ub[(size_t)j * I.nx + i];
      const double kd1 = I.kmax * I.inv_h1 * I.inv_h1, kd2 = I.kmax * I.inv_h2 * I.inv_h2;
      const BLVals<double> r = bl_eval<double>(I.m, u);
      flags = crit_flags<FLUX>(I.m, 0, u, ub[(size_t)j * I.nx + (i + 1 == I.nx ? 0 : i + 1)]) |
              (crit_flags<FLUX>(I.m, 1, u, ub[(size_t)(j + 1 == I.ny ? 0 : j + 1) * I.nx + i]) << 8);
      best = tmax(r.d[0] * I.inv_h1 + kd1, r.d[1] * I.inv_h2 + kd2);
    }
    for (int o = 16; o > 0; o >>= 1) best = tmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    flags = __reduce_or_sync(0xffffffffu, flags);
    if ((threadIdx.x & 31) == 0) {
      sm[threadIdx.x >> 5] = best;
      sf[threadIdx.x >> 5] = flags;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = sm[0];
      unsigned f = sf[0];
      for (int q = 1; q < 8; ++q) {
        b = tmax(b, sm[q]);
        f |= sf[q];
      }
      atomicMax(rate_bits + 2 * k, (unsigned long long)__double_as_longlong(b));
      if (f) atomicOr(rate_bits + 2 * k + 1, (unsigned long long)f);
    }
    __syncthreads();
  }
}

// The same for a flux whose |f_l'| is nondecreasing in |u| (Burgers) or constant: the
// tile's rate is the rate at its largest |u|, a maximum of magnitude bits (integer
// units; per cell the rate would cost GB300's slow FP64 unit several operations). One
// warp per tile, no block-wide synchronisation.
template <int FLUX, int TX, int TY>
__global__ void __launch_bounds__(256) batch_rate_maxu_kernel(const BatchInst* __restrict__ inst,
                                                              const int* __restrict__ work_inst, int total, int in,
                                                              unsigned long long* rate_bits) {
  const int lane = threadIdx.x & 31;
  for (int w = blockIdx.x * 8 + (threadIdx.x >> 5); w < total; w += gridDim.x * 8) {
    const int k = work_inst[w];
    const BatchInst& I = inst[k];
    const int t = w - I.tile_begin;
    const int i0 = (t % I.tiles_x) * TX, j0 = (t / I.tiles_x) * TY;
    const double* ub = I.ub[in];
    unsigned long long mb = 0ull;
    for (int c = lane; c < TX * TY; c += 32) {
      const int i = i0 + c % TX, j = j0 + c / TX;
      if (i < I.nx && j < I.ny) {
        const unsigned long long v =
            (unsigned long long)__double_as_longlong(ub[(size_t)j * I.nx + i]) & 0x7FFFFFFFFFFFFFFFull;
        mb = v > mb ? v : mb;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, mb, o);
      mb = v > mb ? v : mb;
    }
    if (lane == 0) {
      const double u = __longlong_as_double((long long)mb);
      const double kd1 = I.kmax * I.inv_h1 * I.inv_h1, kd2 = I.kmax * I.inv_h2 * I.inv_h2;
      const double b = tmax(alpha_interval<FLUX, double>(I.m, 0, u, u) * I.inv_h1 + kd1,
                            alpha_interval<FLUX, double>(I.m, 1, u, u) * I.inv_h2 + kd2);
      atomicMax(rate_bits + 2 * k, (unsigned long long)__double_as_longlong(b));
    }
  }
}

__global__ void batch_dt_kernel(const BatchInst* __restrict__ inst, int n, double cfl, double cfl_diff,
                                unsigned long long* rate_bits) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const BatchInst& I = inst[k];
  const double rate = crit_rate(I.m, 2, I.inv_h1, I.inv_h2, I.kmax, rate_bits[2 * k + 1],
                                __longlong_as_double((long long)rate_bits[2 * k]));
  double r = rate / cfl;
  if (cfl_diff > 0.0 && I.kmax > 0.0) r = fmax(r, I.kmax * I.inv_hmin2 / cfl_diff);
  const double dt = r > 0.0 ? 1.0 / r : 0.0;
  *I.dt = dt;
  *I.t += dt;
  rate_bits[2 * k] = 0ull;
  rate_bits[2 * k + 1] = 0ull;
}

}  // namespace af

using af::BatchInst;
using af::BatchStage;
using af::DevModel;
using af::DevStats;

namespace {


struct Shape {
  int tx, ty;
};
const Shape kShapes[] = {{32, 8}, {64, 4}, {16, 16}};

}  // namespace

struct af_batch {
  int n = 0, flux = 0, prec = AF_PREC_FP64, rk = AF_RK_SSP3, nbuf = 3, limiter = 1, blend = 0;
  double cfl = 0.165, cfl_diff = 0.0, gamma = 1.0;
  int tx = 32, ty = 8, total_tiles = 0;
  // FP32-mixed without the blend: column-marching items (strips of stream_S rows,
  // chosen in build_work)
  int stream_S = 32, total_items = 0, diff_uniform = -1, pme_e = 0;
  int* d_items = nullptr;
  // the learned indicator (blend 2): the attached network, its 32 x 8 tiles over every
  // instance and the per-cell indicator arrays of all instances
  const af_mlp* mlp = nullptr;
  int ind_total = 0;
  double* d_s = nullptr;
  long long cells = 0;
  std::vector<BatchInst> h_inst;
  std::vector<af_grid> grids;
  unsigned char* block = nullptr;
  BatchInst* d_inst = nullptr;
  int* d_work = nullptr;
  unsigned long long* d_rate = nullptr;
  double* d_dt = nullptr;
  double* d_t = nullptr;
  DevStats* d_stats = nullptr;
  double* d_partial = nullptr;
  double* d_red = nullptr;
  double* h_pinned = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraphExec_t graph = nullptr;
  int persistent_blocks = 0;
  char err[512] = {0};
};

#define BFAIL(b, code, ...)                                        \
  do {                                                             \
    if (b) snprintf((b)->err, sizeof((b)->err), __VA_ARGS__);      \
    return code;                                                   \
  } while (0)
#define BCK(b, call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) BFAIL(b, AF_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

namespace {

template <int FLUX, class T, class PT, int TX, int TY, bool BLEND>
cudaError_t launch_stage_t(af_batch* b, const BatchStage& S) {
  using L = af::Tile2D<FLUX, T, BLEND, TX, TY>;
  auto k = [] {
    if constexpr (sizeof(T) == 4 && !BLEND) return af::batch_stage_kernel_f32occ6<FLUX, TX, TY>;
    else return af::batch_stage_kernel<FLUX, T, PT, TX, TY, BLEND>;
  }();
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
  const int grid = std::min(blocks, b->total_tiles);
  k<<<grid, 256, L::SMEM, b->stream>>>(b->d_inst, b->d_work, b->total_tiles, S, b->d_stats);
  return cudaGetLastError();
}

template <int FLUX, class T, class PT, bool BLEND>
cudaError_t launch_stage_bshape(af_batch* b, const BatchStage& S) {
  if (b->tx == 32 && b->ty == 8) return launch_stage_t<FLUX, T, PT, 32, 8, BLEND>(b, S);
  if (b->tx == 64 && b->ty == 4) return launch_stage_t<FLUX, T, PT, 64, 4, BLEND>(b, S);
  if (b->tx == 16 && b->ty == 16) return launch_stage_t<FLUX, T, PT, 16, 16, BLEND>(b, S);
  return cudaErrorInvalidValue;
}
template <int FLUX, class T, class PT>
cudaError_t launch_stage_shape(af_batch* b, const BatchStage& S) {
  if (sizeof(T) == 4 && !b->blend)
    return af::batch_launch_stream(b->flux, b->diff_uniform, b->pme_e, b->d_inst, b->d_items, b->total_items, S,
                                   b->d_stats, b->stream_S, b->stream);
  if (sizeof(T) == 4)
    return af::batch_launch_stream_blend(b->flux, b->blend, b->diff_uniform, b->d_inst, b->d_items, b->total_items,
                                         S, b->d_stats, b->stream_S, b->stream);
  if (b->blend)
    return af::batch_launch_blend(b->prec, b->flux, b->tx, b->ty, b->d_inst, b->d_work, b->total_tiles, S,
                                  b->d_stats, b->stream);
  return launch_stage_bshape<FLUX, T, PT, false>(b, S);
}

template <class T, class PT>
cudaError_t launch_stage_flux(af_batch* b, const BatchStage& S) {
  switch (b->flux) {
    case AF_FLUX_ZERO: return launch_stage_shape<af::FLUX_ZERO, T, PT>(b, S);
    case AF_FLUX_LINEAR: return launch_stage_shape<af::FLUX_LINEAR, T, PT>(b, S);
    case AF_FLUX_BURGERS: return launch_stage_shape<af::FLUX_BURGERS, T, PT>(b, S);
    default: return launch_stage_shape<af::FLUX_BL, T, PT>(b, S);
  }
}

cudaError_t launch_stage(af_batch* b, const BatchStage& S) {
  return b->prec == AF_PREC_FP64 ? launch_stage_flux<double, double>(b, S) : launch_stage_flux<float, float>(b, S);
}

template <int FLUX, int TX, int TY>
cudaError_t launch_rate_t(af_batch* b) {
  if constexpr (FLUX == af::FLUX_BL) {
    const int grid = std::min(b->total_tiles, 152 * 8);
    af::batch_rate_kernel<FLUX, TX, TY><<<grid, 256, 0, b->stream>>>(b->d_inst, b->d_work, b->total_tiles, 0,
                                                                     b->d_rate);
  } else {
    const int grid = std::min((b->total_tiles + 7) / 8, 152 * 8);
    af::batch_rate_maxu_kernel<FLUX, TX, TY><<<grid, 256, 0, b->stream>>>(b->d_inst, b->d_work, b->total_tiles, 0,
                                                                          b->d_rate);
  }
  return cudaGetLastError();
}

template <int FLUX>
cudaError_t launch_rate_shape(af_batch* b) {
  if (b->tx == 32) return launch_rate_t<FLUX, 32, 8>(b);
  if (b->tx == 64) return launch_rate_t<FLUX, 64, 4>(b);
  return launch_rate_t<FLUX, 16, 16>(b);
}

cudaError_t launch_dt(af_batch* b) {
  cudaError_t e;
  switch (b->flux) {
    case AF_FLUX_ZERO: e = launch_rate_shape<af::FLUX_ZERO>(b); break;
    case AF_FLUX_LINEAR: e = launch_rate_shape<af::FLUX_LINEAR>(b); break;
    case AF_FLUX_BURGERS: e = launch_rate_shape<af::FLUX_BURGERS>(b); break;
    default: e = launch_rate_shape<af::FLUX_BL>(b); break;
  }
  if (e != cudaSuccess) return e;
  af::batch_dt_kernel<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->d_inst, b->n, b->cfl, b->cfl_diff, b->d_rate);
  return cudaGetLastError();
}

BatchStage make_stage(int in, int nout) {
  BatchStage S;
  std::memset(&S, 0, sizeof(S));
  S.in = in;
  S.nout = nout;
  S.out[0] = S.out[1] = -1;
  S.aidx[0] = S.aidx[1] = -1;
  return S;
}
void set_o(BatchStage& S, int o, int out, double cA, int aidx, double cF, double tcoef, int sg) {
  S.out[o] = out;
  S.cA[o] = cA;
  S.aidx[o] = aidx;
  S.cF[o] = cF;
  S.tcoef[o] = tcoef;
  S.sg[o] = sg;
}

// the stages of one step, same buffer roles as the single-mesh driver
std::vector<BatchStage> stages_of(const af_batch* b) {
  std::vector<BatchStage> v;
  if (b->rk == AF_RK_SSP3) {
    BatchStage s0 = make_stage(0, 1); set_o(s0, 0, 1, 0.0, -1, 1.0, 1.0, 1); v.push_back(s0);
    BatchStage s1 = make_stage(1, 1); set_o(s1, 0, 2, 0.75, 0, 0.25, 1.0, 1); v.push_back(s1);
    BatchStage s2 = make_stage(2, 1); set_o(s2, 0, 0, 1.0 / 3.0, 0, 2.0 / 3.0, 1.0, 1); v.push_back(s2);
  } else {
    const double(*A)[5] = af::kA54;
    const double(*B)[5] = af::kB54;
    BatchStage s0 = make_stage(0, 1); set_o(s0, 0, 1, 0.0, -1, A[0][0], B[0][0] / A[0][0], 1); v.push_back(s0);
    BatchStage s1 = make_stage(1, 1); set_o(s1, 0, 2, A[1][0], 0, A[1][1], B[1][1] / A[1][1], 1); v.push_back(s1);
    BatchStage s2 = make_stage(2, 1); set_o(s2, 0, 3, A[2][0], 0, A[2][2], B[2][2] / A[2][2], 1); v.push_back(s2);
    BatchStage s3 = make_stage(3, 2);
    set_o(s3, 0, 1, A[3][0], 0, A[3][3], B[3][3] / A[3][3], 1);
    set_o(s3, 1, 2, A[4][2], 2, A[4][3], B[4][3] / A[4][3], 0);
    v.push_back(s3);
    BatchStage s4 = make_stage(1, 1); set_o(s4, 0, 0, 1.0, 2, A[4][4], B[4][4] / A[4][4], 1); v.push_back(s4);
  }
  for (auto& s : v) {
    s.limiter = b->limiter;
    s.blend = b->blend;
    s.gamma = b->gamma;
  }
  return v;
}

// work list for the current tile shape
af_status build_work(af_batch* b) {
  std::vector<int> work;
  for (int k = 0; k < b->n; ++k) {
    BatchInst& I = b->h_inst[k];
    I.tiles_x = (I.nx + b->tx - 1) / b->tx;
    const int tiles_y = (I.ny + b->ty - 1) / b->ty;
    I.tile_begin = (int)work.size();
    for (int t = 0; t < I.tiles_x * tiles_y; ++t) work.push_back(k);
  }
  b->total_tiles = (int)work.size();
  // column-marching items of every instance (FP32-mixed without the blend). Strip
  // height: the tallest of 128, 64, 32 rows that still gives every resident warp slot
  // (SMs x resident warps) at least 8 items -- each strip repeats a 4-row warm-up and its
  // setup, so taller strips cost less per row (256 instances of 64^2..1024^2: S = 32
  // 1.57e10, 64 1.77e10, 128 1.86e10 cell-stage/s)
  {
    long long rows = 0;
    for (int k = 0; k < b->n; ++k)
      rows += (long long)((b->h_inst[k].nx + af::BATCH_STREAM_BAND - 1) / af::BATCH_STREAM_BAND) * b->h_inst[k].ny;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    // resident warps per SM of the column-marching kernel: 12 for Buckley-Leverett and
    // the blend (3 CTAs of 4 warps), else 16
    const long long want = 8LL * ((b->blend || b->flux == AF_FLUX_BL) ? 12 : 16) * sms;
    b->stream_S = rows / 128 >= want ? 128 : (rows / 64 >= want ? 64 : 32);
  }
  std::vector<int> items;
  for (int k = 0; k < b->n; ++k) {
    BatchInst& I = b->h_inst[k];
    I.bands = (I.nx + af::BATCH_STREAM_BAND - 1) / af::BATCH_STREAM_BAND;
    const int strips = (I.ny + b->stream_S - 1) / b->stream_S;
    I.item_begin = (int)items.size();
    for (int t = 0; t < I.bands * strips; ++t) items.push_back(k);
  }
  b->total_items = (int)items.size();
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  BCK(b, cudaMalloc(&b->d_items, items.size() * sizeof(int)));
  BCK(b, cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (b->d_work) cudaFree(b->d_work);
  b->d_work = nullptr;
  BCK(b, cudaMalloc(&b->d_work, work.size() * sizeof(int)));
  BCK(b, cudaMemcpy(b->d_work, work.data(), work.size() * sizeof(int), cudaMemcpyHostToDevice));
  BCK(b, cudaMemcpy(b->d_inst, b->h_inst.data(), b->n * sizeof(BatchInst), cudaMemcpyHostToDevice));
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return AF_OK;
}

af_status enqueue_step(af_batch* b) {
  BCK(b, launch_dt(b));
  for (const auto& s : stages_of(b)) {
    // the indicator of every instance from this stage's input first: learned, or the
    // plain one for the FP32-mixed column-marching stage (the tile kernels form it)
    if (b->blend == 2)
      BCK(b, af::mlp_indicator_batch_launch(b->mlp, b->d_inst, b->n, b->ind_total, s.in, b->prec, b->stream));
    else if (b->blend == 1 && b->prec == AF_PREC_FP32_MIXED)
      BCK(b, af::batch_launch_blend_s(b->d_inst, b->n, b->ind_total, s.in, b->stream));
    BCK(b, launch_stage(b, s));
  }
  return AF_OK;
}

af_status read_dev(af_batch* b, const double* dev, double* out) {
  BCK(b, cudaMemcpyAsync(b->h_pinned, dev, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  *out = b->h_pinned[0];
  return AF_OK;
}

template <class S>
af_status reduce_inst(af_batch* b, const S* x, size_t n, int op, double init, double* out_dev, int acc) {
  const int blocks = (int)std::min<size_t>(af::RED_MAX_BLOCKS, (n + af::RED_THREADS - 1) / af::RED_THREADS);
  af::partial_kernel<S><<<blocks, af::RED_THREADS, 0, b->stream>>>(x, n, op, init, b->d_partial);
  BCK(b, cudaGetLastError());
  af::finalize_kernel<<<1, af::RED_THREADS, 0, b->stream>>>(b->d_partial, blocks, op, out_dev, acc);
  BCK(b, cudaGetLastError());
  return AF_OK;
}

}  // namespace

extern "C" {

af_status af_batch_create(int n, const af_grid* grids, const af_flux* fluxes, const af_diff* diffs,
                          const af_bounds_t* bounds, const af_opts* opts, af_batch** out) {
  if (n < 1 || !grids || !fluxes || !diffs || !bounds || !opts || !out) return AF_E_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return AF_E_UNSUPPORTED;
  if (opts->precision != AF_PREC_FP64 && opts->precision != AF_PREC_FP32_MIXED) return AF_E_ARG;
  if (opts->rk != AF_RK_SSP3 && opts->rk != AF_RK_SSP54) return AF_E_ARG;
  // the plain blend, or the external indicator computed by a network attached with
  // af_batch_set_mlp (a batch has no per-cell indicator input of its own)
  if (opts->diffusion_form != AF_FORM_DC) return AF_E_UNSUPPORTED;
  if (opts->blend != AF_BLEND_OFF && opts->blend != AF_BLEND_PLAIN && opts->blend != AF_BLEND_EXTERNAL) return AF_E_ARG;
  for (int k = 0; k < n; ++k) {
    if (grids[k].dim != 2 || grids[k].nx < 1 || grids[k].ny < 1) return AF_E_ARG;
    if (grids[k].bc != AF_BC_PERIODIC) return AF_E_UNSUPPORTED;
    if (!(grids[k].x1 > grids[k].x0) || !(grids[k].y1 > grids[k].y0)) return AF_E_ARG;
    if (fluxes[k].kind != fluxes[0].kind || fluxes[k].kind < 0 || fluxes[k].kind > AF_FLUX_BL) return AF_E_ARG;
    if (diffs[k].kind < AF_DIFF_NONE || diffs[k].kind > AF_DIFF_CUBIC01) return AF_E_ARG;
    if (diffs[k].kind == AF_DIFF_RAMP && !(diffs[k].p[2] > 0.0)) return AF_E_ARG;
    if (bounds[k].from_initial_data || !(bounds[k].umax > bounds[k].umin)) return AF_E_ARG;
  }
  af_batch* b = new (std::nothrow) af_batch;
  if (!b) return AF_E_OOM;
  b->n = n;
  b->flux = fluxes[0].kind;
  b->prec = opts->precision;
  b->rk = opts->rk;
  b->nbuf = opts->rk == AF_RK_SSP54 ? 4 : 3;
  b->limiter = opts->limiter;
  b->blend = opts->blend == AF_BLEND_PLAIN ? 1 : (opts->blend == AF_BLEND_EXTERNAL ? 2 : 0);
  b->gamma = opts->gamma;
  b->cfl = opts->cfl > 0.0 ? opts->cfl : 0.33 / 2;
  b->cfl_diff = opts->cfl_diff > 0.0 ? opts->cfl_diff
                                     : (opts->cfl_diff < 0.0 ? 0.0 : 0.9 * (opts->rk == AF_RK_SSP54 ? 0.1307 : 0.0616));
  b->grids.assign(grids, grids + n);
  const size_t ps = b->prec == AF_PREC_FP64 ? 8 : 4;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t total = 0;
  for (int k = 0; k < n; ++k) {
    const size_t c = (size_t)grids[k].nx * grids[k].ny;
    b->cells += (long long)c;
    total += b->nbuf * (al(c * 8) + 3 * al(c * ps));
  }
  if (cudaMalloc(&b->block, total) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return AF_E_OOM;
  }
  cudaMemset(b->block, 0, total);
  b->h_inst.resize(n);
  unsigned char* p = b->block;
  for (int k = 0; k < n; ++k) {
    BatchInst& I = b->h_inst[k];
    std::memset(&I, 0, sizeof(I));
    const af_grid& g = grids[k];
    const size_t c = (size_t)g.nx * g.ny;
    I.nx = g.nx;
    I.ny = g.ny;
    const double dx = (g.x1 - g.x0) / g.nx, dy = (g.y1 - g.y0) / g.ny;
    I.inv_h1 = 1.0 / dx;
    I.inv_h2 = 1.0 / dy;
    I.inv_hmin2 = 1.0 / (std::min(dx, dy) * std::min(dx, dy));
    I.i6h[0] = I.inv_h1 / 6.0;
    I.i6h[1] = I.inv_h2 / 6.0;
    I.i3h2[0] = I.inv_h1 * I.inv_h1 / 3.0;
    I.i3h2[1] = I.inv_h2 * I.inv_h2 / 3.0;
    for (int l = 0; l < 2; ++l) {
      I.i6hf[l] = (float)I.i6h[l];
      I.i3h2f[l] = (float)I.i3h2[l];
    }
    I.m.flux_kind = fluxes[k].kind;
    I.m.diff_kind = diffs[k].kind;
    for (int q = 0; q < 4; ++q) { I.m.fp[q] = fluxes[k].p[q]; I.m.dp[q] = diffs[k].p[q]; }
    I.m.umin = bounds[k].umin;
    I.m.umax = bounds[k].umax;
    af::finish_model(I.m, fluxes[k].kind, 2);
    I.kmax = af::kappa_max_of(diffs[k], bounds[k].umin, bounds[k].umax);
    const double scale = std::max(std::fabs(bounds[k].umin), std::fabs(bounds[k].umax));
    I.tol = (b->prec == AF_PREC_FP64 ? 8.0 * 2.220446049250313e-16 : 64.0 * 1.1920929e-07) * scale;
    for (int s = 0; s < b->nbuf; ++s) {
      I.ub[s] = (double*)p; p += al(c * 8);
      I.pv[s] = p; p += al(c * ps);
      I.px[s] = p; p += al(c * ps);
      I.py[s] = p; p += al(c * ps);
    }
    I.ind_begin = b->ind_total;
    b->ind_total += ((g.nx + 31) / 32) * ((g.ny + 7) / 8);
  }
  // indicator arrays: the learned one (one double per cell), or the plain one of the
  // FP32-mixed column-marching stage (s_1, s_2 as FP32)
  const bool plain32 = b->blend == 1 && b->prec == AF_PREC_FP32_MIXED;
  if (b->blend == 2 || plain32) {
    size_t stotal = 0;
    for (int k = 0; k < n; ++k) stotal += al((size_t)grids[k].nx * grids[k].ny * 8);
    if (cudaMalloc(&b->d_s, stotal) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(b->block);
      delete b;
      return AF_E_OOM;
    }
    unsigned char* q = (unsigned char*)b->d_s;
    for (int k = 0; k < n; ++k) {
      const size_t c = (size_t)grids[k].nx * grids[k].ny;
      if (plain32) {
        b->h_inst[k].sb[0] = (float*)q;
        b->h_inst[k].sb[1] = (float*)q + c;
      } else {
        b->h_inst[k].s = (double*)q;
      }
      q += al(c * 8);
    }
  }
  // the diffusion kind every instance shares (compiled into the column-marching stage)
  b->diff_uniform = b->h_inst[0].m.diff_kind;
  b->pme_e = b->h_inst[0].m.pme_e;
  for (int k = 1; k < n; ++k)
    if (b->h_inst[k].m.diff_kind != b->diff_uniform || b->h_inst[k].m.pme_e != b->pme_e) b->diff_uniform = -1;
  bool ok = cudaMalloc(&b->d_inst, n * sizeof(BatchInst)) == cudaSuccess &&
            cudaMalloc(&b->d_rate, 2 * n * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&b->d_dt, n * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&b->d_t, n * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&b->d_stats, sizeof(DevStats)) == cudaSuccess &&
            cudaMalloc(&b->d_partial, af::RED_MAX_BLOCKS * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&b->d_red, 8 * sizeof(double)) == cudaSuccess &&
            cudaMallocHost(&b->h_pinned, 8 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    af_batch_destroy(b);
    return AF_E_OOM;
  }
  cudaMemset(b->d_rate, 0, 2 * n * sizeof(unsigned long long));
  cudaMemset(b->d_dt, 0, n * sizeof(double));
  cudaMemset(b->d_t, 0, n * sizeof(double));
  cudaMemset(b->d_stats, 0, sizeof(DevStats));
  for (int k = 0; k < n; ++k) {
    b->h_inst[k].dt = b->d_dt + k;
    b->h_inst[k].t = b->d_t + k;
  }
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    af_batch_destroy(b);
    return AF_E_CUDA;
  }
  b->own_stream = true;
  if (build_work(b) != AF_OK) {
    af_batch_destroy(b);
    return AF_E_OOM;
  }
  *out = b;
  return AF_OK;
}

af_status af_batch_destroy(af_batch* b) {
  if (!b) return AF_E_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->block);
  cudaFree(b->d_s);
  cudaFree(b->d_inst);
  cudaFree(b->d_work);
  cudaFree(b->d_items);
  cudaFree(b->d_rate);
  cudaFree(b->d_dt);
  cudaFree(b->d_t);
  cudaFree(b->d_stats);
  cudaFree(b->d_partial);
  cudaFree(b->d_red);
  if (b->h_pinned) cudaFreeHost(b->h_pinned);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return AF_OK;
}

const char* af_batch_last_error(const af_batch* b) { return b ? b->err : "null batch"; }

af_status af_batch_set_stream(af_batch* b, void* stream) {
  if (!b || !stream) return AF_E_ARG;
  cudaStreamSynchronize(b->stream);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->own_stream = false;
  b->stream = (cudaStream_t)stream;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return AF_OK;
}

af_status af_batch_info(const af_batch* b, long long* cells, int* tiles, int* tx, int* ty) {
  if (!b) return AF_E_ARG;
  if (cells) *cells = b->cells;
  if (tiles) *tiles = b->total_tiles;
  if (tx) *tx = b->tx;
  if (ty) *ty = b->ty;
  return AF_OK;
}

af_status af_batch_set_mlp(af_batch* b, const af_mlp* net) {
  if (!b) return AF_E_ARG;
  if (b->blend != 2) BFAIL(b, AF_E_STATE, "af_batch_set_mlp needs a batch created with blend = AF_BLEND_EXTERNAL");
  cudaStreamSynchronize(b->stream);   // no step in flight uses the previous network
  b->mlp = net;
  if (b->graph) {   // the captured step holds the previous network's buffers
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return AF_OK;
}

af_status af_batch_set_tile(af_batch* b, int tx, int ty) {
  if (!b) return AF_E_ARG;
  bool known = false;
  for (const Shape& s : kShapes) known |= (s.tx == tx && s.ty == ty);
  if (!known) BFAIL(b, AF_E_ARG, "tile %dx%d not built (32x8, 64x4, 16x16)", tx, ty);
  BCK(b, cudaStreamSynchronize(b->stream));
  b->tx = tx;
  b->ty = ty;
  return build_work(b);
}

af_status af_batch_set_state(af_batch* b, int i, const double* ub, const double* V, const double* X, const double* Y) {
  if (!b || i < 0 || i >= b->n || !ub || !V || !X || !Y) return AF_E_ARG;
  BatchInst& I = b->h_inst[i];
  const size_t c = (size_t)I.nx * I.ny;
  const double* src[4] = {ub, V, X, Y};
  for (int a = 0; a < 4; ++a)
    for (size_t k = 0; k < c; ++k) {
      const double v = src[a][k];
      if (!(v == v)) BFAIL(b, AF_E_STATE, "NaN in instance %d", i);
      if (b->limiter && (v < I.m.umin || v > I.m.umax)) BFAIL(b, AF_E_STATE, "instance %d outside its bounds", i);
    }
  BCK(b, cudaMemcpyAsync(I.ub[0], ub, c * 8, cudaMemcpyHostToDevice, b->stream));
  void* dst[3] = {I.pv[0], I.px[0], I.py[0]};
  if (b->prec == AF_PREC_FP64) {
    for (int a = 1; a < 4; ++a) BCK(b, cudaMemcpyAsync(dst[a - 1], src[a], c * 8, cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
  } else {
    std::vector<float> tmp(c);
    for (int a = 1; a < 4; ++a) {
      for (size_t k = 0; k < c; ++k) tmp[k] = (float)src[a][k];
      BCK(b, cudaMemcpyAsync(dst[a - 1], tmp.data(), c * 4, cudaMemcpyHostToDevice, b->stream));
      BCK(b, cudaStreamSynchronize(b->stream));
    }
  }
  return AF_OK;
}

af_status af_batch_get_state(af_batch* b, int i, double* ub, double* V, double* X, double* Y) {
  if (!b || i < 0 || i >= b->n || !ub || !V || !X || !Y) return AF_E_ARG;
  BatchInst& I = b->h_inst[i];
  const size_t c = (size_t)I.nx * I.ny;
  double* dst[4] = {ub, V, X, Y};
  void* src[3] = {I.pv[0], I.px[0], I.py[0]};
  BCK(b, cudaMemcpyAsync(ub, I.ub[0], c * 8, cudaMemcpyDeviceToHost, b->stream));
  if (b->prec == AF_PREC_FP64) {
    for (int a = 1; a < 4; ++a) BCK(b, cudaMemcpyAsync(dst[a], src[a - 1], c * 8, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
  } else {
    std::vector<float> tmp(c);
    for (int a = 1; a < 4; ++a) {
      BCK(b, cudaMemcpyAsync(tmp.data(), src[a - 1], c * 4, cudaMemcpyDeviceToHost, b->stream));
      BCK(b, cudaStreamSynchronize(b->stream));
      for (size_t k = 0; k < c; ++k) dst[a][k] = (double)tmp[k];
    }
  }
  BCK(b, cudaStreamSynchronize(b->stream));
  return AF_OK;
}

af_status af_batch_device_ptrs(af_batch* b, int i, void* ptrs[4], int dtype[2]) {
  if (!b || i < 0 || i >= b->n || !ptrs) return AF_E_ARG;
  const BatchInst& I = b->h_inst[i];
  ptrs[0] = I.ub[0];
  ptrs[1] = I.pv[0];
  ptrs[2] = I.px[0];
  ptrs[3] = I.py[0];
  if (dtype) { dtype[0] = 8; dtype[1] = b->prec == AF_PREC_FP64 ? 8 : 4; }
  return AF_OK;
}

af_status af_batch_step(af_batch* b, int nsteps) {
  if (!b || nsteps < 0) return AF_E_ARG;
  if (b->blend == 2 && !b->mlp) BFAIL(b, AF_E_STATE, "blend with the external indicator needs af_batch_set_mlp");
  if (!b->graph) {
    cudaGraph_t g = nullptr;
    BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    af_status s = enqueue_step(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (s != AF_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) BFAIL(b, AF_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) BFAIL(b, AF_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  for (int s = 0; s < nsteps; ++s) BCK(b, cudaGraphLaunch(b->graph, b->stream));
  return AF_OK;
}

af_status af_batch_sync(af_batch* b) {
  if (!b) return AF_E_ARG;
  BCK(b, cudaStreamSynchronize(b->stream));
  return AF_OK;
}

af_status af_batch_time(af_batch* b, int i, double* t) {
  if (!b || i < 0 || i >= b->n || !t) return AF_E_ARG;
  return read_dev(b, b->d_t + i, t);
}

af_status af_batch_mass(af_batch* b, int i, double* mass) {
  if (!b || i < 0 || i >= b->n || !mass) return AF_E_ARG;
  const BatchInst& I = b->h_inst[i];
  af_status s = reduce_inst<double>(b, I.ub[0], (size_t)I.nx * I.ny, 0, 0.0, b->d_red, 0);
  if (s != AF_OK) return s;
  double v;
  s = read_dev(b, b->d_red, &v);
  if (s != AF_OK) return s;
  *mass = v / (I.inv_h1 * I.inv_h2);
  return AF_OK;
}

af_status af_batch_bounds(af_batch* b, int i, double* umin, double* umax) {
  if (!b || i < 0 || i >= b->n || !umin || !umax) return AF_E_ARG;
  const BatchInst& I = b->h_inst[i];
  const size_t c = (size_t)I.nx * I.ny;
  void* arrs[4] = {I.ub[0], I.pv[0], I.px[0], I.py[0]};
  for (int op = 1; op <= 2; ++op)
    for (int a = 0; a < 4; ++a) {
      af_status s;
      const double init = op == 1 ? INFINITY : -INFINITY;
      if (a == 0 || b->prec == AF_PREC_FP64)
        s = reduce_inst<double>(b, (const double*)arrs[a], c, op, init, b->d_red + op, a > 0);
      else
        s = reduce_inst<float>(b, (const float*)arrs[a], c, op, init, b->d_red + op, a > 0);
      if (s != AF_OK) return s;
    }
  af_status s = read_dev(b, b->d_red + 1, umin);
  if (s != AF_OK) return s;
  return read_dev(b, b->d_red + 2, umax);
}

af_status af_batch_stats(af_batch* b, long long* clamps, long long* errors, double* max_excess) {
  if (!b) return AF_E_ARG;
  DevStats st;
  BCK(b, cudaMemcpyAsync(&st, b->d_stats, sizeof(st), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  if (clamps) *clamps = (long long)st.clamps;
  if (errors) *errors = (long long)st.errors;
  if (max_excess) std::memcpy(max_excess, &st.max_excess_bits, sizeof(double));
  return AF_OK;
}

// Time one step of every candidate tile shape on this batch (median of 3 after a warm-up)
// and keep the fastest. The state is saved and restored around the trials.
af_status af_batch_autotune(af_batch* b, int* tx, int* ty) {
  if (!b) return AF_E_ARG;
  if (b->blend == 2 && !b->mlp) BFAIL(b, AF_E_STATE, "blend with the external indicator needs af_batch_set_mlp");
  BCK(b, cudaStreamSynchronize(b->stream));
  // snapshot U0 and the clocks so the trials leave no trace
  size_t bytes0 = 0;
  for (const auto& I : b->h_inst) bytes0 += (size_t)I.nx * I.ny * (8 + 3 * (b->prec == AF_PREC_FP64 ? 8 : 4));
  unsigned char* save = nullptr;
  BCK(b, cudaMalloc(&save, bytes0 + 2 * b->n * sizeof(double) + sizeof(DevStats)));
  auto copy_state = [&](bool to_save) -> af_status {
    size_t off = 0;
    const size_t ps = b->prec == AF_PREC_FP64 ? 8 : 4;
    for (const auto& I : b->h_inst) {
      const size_t c = (size_t)I.nx * I.ny;
      void* arrs[4] = {I.ub[0], I.pv[0], I.px[0], I.py[0]};
      for (int a = 0; a < 4; ++a) {
        const size_t n = c * (a == 0 ? 8 : ps);
        if (to_save) BCK(b, cudaMemcpyAsync(save + off, arrs[a], n, cudaMemcpyDeviceToDevice, b->stream));
        else BCK(b, cudaMemcpyAsync(arrs[a], save + off, n, cudaMemcpyDeviceToDevice, b->stream));
        off += n;
      }
    }
    if (to_save) {
      BCK(b, cudaMemcpyAsync(save + off, b->d_t, b->n * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
      BCK(b, cudaMemcpyAsync(save + off + b->n * 8, b->d_dt, b->n * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
      BCK(b, cudaMemcpyAsync(save + off + 2 * b->n * 8, b->d_stats, sizeof(DevStats), cudaMemcpyDeviceToDevice, b->stream));
    } else {
      BCK(b, cudaMemcpyAsync(b->d_t, save + off, b->n * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
      BCK(b, cudaMemcpyAsync(b->d_dt, save + off + b->n * 8, b->n * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
      BCK(b, cudaMemcpyAsync(b->d_stats, save + off + 2 * b->n * 8, sizeof(DevStats), cudaMemcpyDeviceToDevice, b->stream));
    }
    return AF_OK;
  };
  af_status s = copy_state(true);
  if (s != AF_OK) { cudaFree(save); return s; }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  Shape pick = kShapes[0];
  for (const Shape& sh : kShapes) {
    if ((s = af_batch_set_tile(b, sh.tx, sh.ty)) != AF_OK) break;
    std::vector<float> t;
    for (int rep = 0; rep < 4 && s == AF_OK; ++rep) {
      cudaEventRecord(e0, b->stream);
      s = enqueue_step(b);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep) t.push_back(ms);
      if (s == AF_OK) s = copy_state(false);
    }
    if (s != AF_OK) break;
    std::sort(t.begin(), t.end());
    if (t[t.size() / 2] < best) { best = t[t.size() / 2]; pick = sh; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == AF_OK) s = copy_state(false);
  cudaStreamSynchronize(b->stream);
  cudaFree(save);
  if (s != AF_OK) return s;
  s = af_batch_set_tile(b, pick.tx, pick.ty);
  if (tx) *tx = pick.tx;
  if (ty) *ty = pick.ty;
  return s;
}

}  // extern "C"
