// One signal cut into contiguous slices (one per GPU): the fold of Eq. (2)
// is a sum over the signal's entries, so the extended folds of the slices
// add up to the signal's folds. Each slice's fold restricted to its entries
// comes from the fold kernel (rows counted from the slice's first element,
// FoldQ::e0) plus this completion: per column k < M the slots' counts or
// sums, the slice's last entries past the fold kernel's 16-byte multiple,
// and the wrap-around entry x_{k-Rw} of the short last row (Rw = N - (L-1)M)
// when it lies in the slice; the extension k = M+i (i < K-1) follows
// y[M+i] = y[i] - x_i + x_{(i+LM) mod N}, each term kept only when its index
// lies in the slice (the index sets of the two sides differ by exactly those
// two entries). Also the partial exact scores of step 9 over a slice.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "tm_internal.h"

namespace ftm {
namespace {

// Entry n of the full signal (n in the slice) from the slice's storage.
__device__ __forceinline__ double slice_val(const void* x, int32_t dtype, int64_t n0, int64_t n) {
  const int64_t u = n - n0;
  switch (dtype) {
    case TM_I8_PM1: return (static_cast<const uint8_t*>(x)[u] & 2u) ? -1.0 : 1.0;
    case TM_BITS_PM1: return ((static_cast<const uint8_t*>(x)[u >> 3] >> (u & 7)) & 1u) ? 1.0 : -1.0;
    case TM_F16: return double(__half2float(static_cast<const __half*>(x)[u]));
    default: return double(static_cast<const float*>(x)[u]);
  }
}

// Number of n in [0, b) with n = k (mod M), b >= 0.
__device__ __forceinline__ int64_t count_below(int64_t b, int64_t k, int64_t M) {
  return b > k ? (b - k - 1) / M + 1 : 0;
}

__global__ void fold_slice_complete_kernel(const SliceFoldArgs a) {
  const int j = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.P) return;
  const int64_t M = a.M[j], L = a.L[j];
  const bool ints = a.xdtype == TM_I8_PM1 || a.xdtype == TM_BITS_PM1;
  const int64_t s0 = a.n0, s1 = a.n0 + a.len;   // the slice
  auto in_slice = [&](int64_t n) { return n >= s0 && n < s1; };
  const int64_t Rw = a.N - (L - 1) * M;
  // column c < M of the slice's M-fold, the value kept as double (exact for
  // integers; reals are summed in fp32 in a fixed order first)
  auto column = [&](int64_t c) -> double {
    double v;
    if (ints) {
      long long cnt = 0;
      for (int s = 0; s < a.nslots; ++s)
        for (int r = 0; r < a.R[j]; ++r) cnt += a.partial[int64_t(s) * a.stride + a.moff[j] + c + r * M];
      // entries of the folded range [n0, n0 + nfold) in this column
      const int64_t nk = count_below(s0 + a.nfold, c, M) - count_below(s0, c, M);
      v = double(a.xdtype == TM_BITS_PM1 ? 2 * cnt - nk : nk - 2 * cnt);
    } else {
      const float* pf = reinterpret_cast<const float*>(a.partial);
      float f = 0.f;
      for (int s = 0; s < a.nslots; ++s)
        for (int r = 0; r < a.R[j]; ++r) f += pf[int64_t(s) * a.stride + a.moff[j] + c + r * M];
      v = double(f);
    }
    for (int64_t n = s0 + a.nfold; n < s1; ++n)
      if (n % M == c) v += slice_val(a.x, a.xdtype, s0, n);
    if (c >= Rw && in_slice(c - Rw)) v += slice_val(a.x, a.xdtype, s0, c - Rw);
    return v;
  };
  double y = 0.0;
  if (k < M) {
    y = column(k);
  } else if (k < M + a.K - 1) {
    const int64_t i = k - M;
    int64_t w = i + L * M - a.N;
    if (w >= a.N) w %= a.N;
    y = column(i);
    if (in_slice(i)) y -= slice_val(a.x, a.xdtype, s0, i);
    if (in_slice(w)) y += slice_val(a.x, a.xdtype, s0, w);
  }
  if (ints) static_cast<int32_t*>(a.y)[int64_t(j) * a.P + k] = int32_t(y);
  else static_cast<float*>(a.y)[int64_t(j) * a.P + k] = float(y);
}

constexpr int kScoreThreads = 256;

__global__ void score_slice_kernel(const SliceScoreArgs a) {
  __shared__ double red[kScoreThreads / 32];
  const int64_t m = a.m[blockIdx.x];
  double acc = 0.0;
  for (int i = threadIdx.x; i < a.K; i += kScoreThreads) {
    int64_t n = m + i;
    if (n >= a.N) n -= a.N;
    if (n >= a.n0 && n < a.n0 + a.len) acc = fma(double(a.t[i]), slice_val(a.x, a.xdtype, a.n0, n), acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kScoreThreads / 32; ++w) s += red[w];
    a.out[blockIdx.x] = s;
  }
}

}  // namespace

cudaError_t launch_fold_slice_complete(const SliceFoldArgs& a, cudaStream_t s) {
  const dim3 grid(unsigned((a.P + 255) / 256), 2);
  fold_slice_complete_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_score_slice(const SliceScoreArgs& a, cudaStream_t s) {
  if (a.nm <= 0) return cudaSuccess;
  score_slice_kernel<<<a.nm, kScoreThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ftm
