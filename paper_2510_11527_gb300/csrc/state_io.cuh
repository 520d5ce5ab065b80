// Device side of af_set_state / af_get_state: host arrays are copied as doubles into a
// staging area (the RK temporaries, free between steps), checked there (NaN count, min,
// max over all values) and only then converted into the state buffers, so a rejected
// input leaves the state untouched and the host never scans the arrays.
#pragma once
#include <climits>

#include "reduce.cuh"

namespace af {

constexpr int STATE_IO_BLOCKS = RED_MAX_BLOCKS / 3;   // three partial slots per block

__device__ __forceinline__ double undkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL));
}

// (NaN count, min key, max key) over the block; the result is valid in thread 0
__device__ __forceinline__ void block_nan_min_max(unsigned long long& nan, long long& lo, long long& hi) {
  for (int o = 16; o > 0; o >>= 1) {
    nan += __shfl_xor_sync(0xffffffffu, nan, o);
    const long long l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  __shared__ unsigned long long sn[RED_THREADS / 32];
  __shared__ long long sl[RED_THREADS / 32], sh[RED_THREADS / 32];
  if ((threadIdx.x & 31) == 0) {
    sn[threadIdx.x >> 5] = nan;
    sl[threadIdx.x >> 5] = lo;
    sh[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < RED_THREADS / 32; ++w) {
      nan += sn[w];
      lo = sl[w] < lo ? sl[w] : lo;
      hi = sh[w] > hi ? sh[w] : hi;
    }
  }
}

// per block: number of NaNs, min and max (as order-preserving keys) of x[0, n)
__global__ void __launch_bounds__(RED_THREADS) validate_partial_kernel(const double* __restrict__ x, size_t n,
                                                                       unsigned long long* partial) {
  unsigned long long nan = 0;
  long long lo = LLONG_MAX, hi = LLONG_MIN;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const long long b = __double_as_longlong(x[k]);
    if ((b & 0x7FFFFFFFFFFFFFFFLL) > 0x7FF0000000000000LL) {
      ++nan;
    } else {
      const long long key = b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
      lo = key < lo ? key : lo;
      hi = key > hi ? key : hi;
    }
  }
  block_nan_min_max(nan, lo, hi);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = nan;
    partial[gridDim.x + blockIdx.x] = (unsigned long long)lo;
    partial[2 * gridDim.x + blockIdx.x] = (unsigned long long)hi;
  }
}

// out[0] = NaN count, out[1] = min, out[2] = max over the nb block partials (one block
// of RED_THREADS)
static __global__ void __launch_bounds__(RED_THREADS) validate_final_kernel(const unsigned long long* partial,
                                                                            int nb, double* out) {
  unsigned long long nan = 0;
  long long lo = LLONG_MAX, hi = LLONG_MIN;
  for (int b = threadIdx.x; b < nb; b += RED_THREADS) {
    nan += partial[b];
    const long long l = (long long)partial[nb + b], h = (long long)partial[2 * nb + b];
    lo = l < lo ? l : lo;
    hi = h > hi ? h : hi;
  }
  block_nan_min_max(nan, lo, hi);
  if (threadIdx.x == 0) {
    out[0] = (double)nan;
    out[1] = undkey(lo);
    out[2] = undkey(hi);
  }
}

// staged doubles (ub: n values, then na - 1 point arrays of np >= n values, back to
// back) -> state buffers (points rounded to nearest when stored in FP32)
template <class PT>
__global__ void __launch_bounds__(RED_THREADS) scatter_state_kernel(const double* __restrict__ stg, size_t n,
                                                                    size_t np, int na, double* ub, PT* V, PT* X,
                                                                    PT* Y) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < np; k += (size_t)gridDim.x * blockDim.x) {
    if (k < n) ub[k] = stg[k];
    V[k] = (PT)stg[n + k];
    if (na == 4) {
      X[k] = (PT)stg[n + np + k];
      Y[k] = (PT)stg[n + 2 * np + k];
    }
  }
}

// FP32 point arrays (np values each) -> staged doubles (exact widening) for the copy to
// the host
__global__ void __launch_bounds__(RED_THREADS) gather_points_kernel(const float* __restrict__ V,
                                                                    const float* __restrict__ X,
                                                                    const float* __restrict__ Y, size_t n, int na,
                                                                    double* stg) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    stg[k] = f2d_exact(V[k]);
    if (na == 4) {
      stg[n + k] = f2d_exact(X[k]);
      stg[2 * n + k] = f2d_exact(Y[k]);
    }
  }
}

}  // namespace af
