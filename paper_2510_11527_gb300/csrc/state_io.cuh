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

// exact widening of a stored point value
__device__ __forceinline__ double wide(double v) { return v; }
__device__ __forceinline__ double wide(float v) { return f2d_exact(v); }

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

// dst[k] = src[k] rounded to nearest float / widened exactly (3D FP32-mixed point arrays)
__global__ void __launch_bounds__(RED_THREADS) narrow_kernel(const double* __restrict__ src, float* dst, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    dst[k] = (float)src[k];
}
__global__ void __launch_bounds__(RED_THREADS) widen_kernel(const float* __restrict__ src, double* dst, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    dst[k] = f2d_exact(src[k]);
}

// 2D rectangle with ends: the caller's layout (ub [ny][nx], V [ny+1][nx+1],
// X [ny][nx+1], Y [ny+1][nx], staged back to back as doubles) <-> the padded device
// layout ((nx+1) x (ny+1) per array; entry (I, J) holds ub(I-1, J-1), V(I-1, J-1),
// X(I-1, J-1), Y(I-1, J-1) in cell / point indices, i.e. corner and edges of padded cell
// (I, J)). Padded entries that are not DoFs (ub in row / column 0, X in row 0, Y in
// column 0) are written as 0 and never read as data.
template <class PT>
__global__ void __launch_bounds__(RED_THREADS) scatter_rect_kernel(const double* __restrict__ stg, int nx, int ny,
                                                                   double* ub, PT* V, PT* X, PT* Y) {
  const int NX = nx + 1, NY = ny + 1;
  const size_t pn = (size_t)NX * NY, oV = (size_t)nx * ny, oX = oV + pn, oY = oX + (size_t)NX * ny;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < pn; k += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(k % NX), J = (int)(k / NX);
    ub[k] = (I > 0 && J > 0) ? stg[(size_t)(J - 1) * nx + (I - 1)] : 0.0;
    V[k] = (PT)stg[oV + k];
    X[k] = J > 0 ? (PT)stg[oX + (size_t)(J - 1) * NX + I] : PT(0);
    Y[k] = I > 0 ? (PT)stg[oY + (size_t)J * nx + (I - 1)] : PT(0);
  }
}

template <class PT>
__global__ void __launch_bounds__(RED_THREADS) gather_rect_kernel(const double* __restrict__ ub,
                                                                  const PT* __restrict__ V, const PT* __restrict__ X,
                                                                  const PT* __restrict__ Y, int nx, int ny,
                                                                  double* stg) {
  const int NX = nx + 1, NY = ny + 1;
  const size_t pn = (size_t)NX * NY, oV = (size_t)nx * ny, oX = oV + pn, oY = oX + (size_t)NX * ny;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < pn; k += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(k % NX), J = (int)(k / NX);
    if (I > 0 && J > 0) stg[(size_t)(J - 1) * nx + (I - 1)] = ub[k];
    stg[oV + k] = wide(V[k]);
    if (J > 0) stg[oX + (size_t)(J - 1) * NX + I] = wide(X[k]);
    if (I > 0) stg[oY + (size_t)J * nx + (I - 1)] = wide(Y[k]);
  }
}

}  // namespace af
