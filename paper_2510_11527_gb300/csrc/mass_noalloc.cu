// Allocation-free total-mass reduction: a variant of the deterministic mass reduction
// behind af_mass whose scratch lives in a file-scope device array instead of memory
// the library or the caller allocates. The paper has no counterpart; this exists for
// callers that cannot allocate device memory (see include/af.h).
#include <cuda_runtime.h>

#include "af.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr long long kPerBlock = (long long)kThreads * kPerThread;         // 2048 cells per block
constexpr int kMaxParts = (int)(AF_MASS_NOALLOC_MAX_CELLS / kPerBlock);   // 65536 partial sums
static_assert((long long)kMaxParts * kPerBlock == AF_MASS_NOALLOC_MAX_CELLS, "size mismatch");

// Scratch shared by every call on a device: kMaxParts block partials followed by the
// final sum (512 KiB + 8 B per device that loads the library, held until exit).
static __device__ __align__(256) double g_mass_scratch[kMaxParts + 1];

// Block b sums cells [b * 2048, (b + 1) * 2048) in a fixed order: each thread adds its
// 8 strided cells, then a shared-memory tree of halving strides.
__global__ void __launch_bounds__(kThreads) mass_partial_static(const double* __restrict__ x, long long n,
                                                                double* parts) {
  const long long base = (long long)blockIdx.x * kPerBlock + threadIdx.x;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const long long i = base + (long long)k * kThreads;
    if (i < n) acc += x[i];
  }
  __shared__ double sm[kThreads];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) parts[blockIdx.x] = sm[0];
}

// One block combines the partials in a fixed order; the result goes to parts[kMaxParts].
__global__ void __launch_bounds__(1024) mass_final_static(double* parts, int nparts) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < nparts; k += 1024) acc += parts[k];
  __shared__ double sm[1024];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) parts[kMaxParts] = sm[0];
}

// Device address of the current device's scratch array, resolved on every call (the
// host-side name of the array is only a stand-in and must never be passed to a kernel;
// resolving per call also stays right after the caller resets the device, which
// reloads the module at a new address). With CUDA's lazy module loading the first
// resolution on a device loads this module and allocates the array there.
cudaError_t scratch_for_current_device(double** out) {
  return cudaGetSymbolAddress((void**)out, g_mass_scratch);
}

// ub_dev must be device (or managed) memory of the current device: a pointer into
// another device's memory would run the reduction on the wrong GPU.
bool on_current_device(const void* p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
    (void)cudaGetLastError();   // the failed query's own error: the call reports AF_E_ARG
    return false;
  }
  return (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) && pa.device == dev;
}

}  // namespace

extern "C" af_status af_mass_noalloc(const double* ub_dev, long long ncells, double cell_area, double* mass,
                                     void* stream) {
  if (!ub_dev || !mass) return AF_E_ARG;
  if (ncells <= 0 || ncells > AF_MASS_NOALLOC_MAX_CELLS) return AF_E_ARG;
  if (!on_current_device(ub_dev)) return AF_E_ARG;
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return AF_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int nparts = (int)((ncells + kPerBlock - 1) / kPerBlock);
  // launch errors are taken from the launch calls themselves, so an unrelated error
  // left pending by an earlier call is neither reported here nor cleared
  void* a1[] = {(void*)&ub_dev, (void*)&ncells, (void*)&scratch};
  if (cudaLaunchKernel((const void*)mass_partial_static, dim3(nparts), dim3(kThreads), a1, 0, s) != cudaSuccess)
    return AF_E_CUDA;
  void* a2[] = {(void*)&scratch, (void*)&nparts};
  if (cudaLaunchKernel((const void*)mass_final_static, dim3(1), dim3(1024), a2, 0, s) != cudaSuccess)
    return AF_E_CUDA;
  double sum = 0.0;
  if (cudaMemcpyAsync(&sum, scratch + kMaxParts, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return AF_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return AF_E_CUDA;
  *mass = sum * cell_area;
  return AF_OK;
}
