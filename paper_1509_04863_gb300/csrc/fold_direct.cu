// Step 3 of Algorithm 1 (Eq. (2)) for moduli too wide for the streaming
// fold kernel's register-resident columns (M above about 2^14 entries): one
// thread per fold entry k < M+K-1, summing the L terms x_{(k+lM) mod N}
// directly. A warp's consecutive k read consecutive entries of x, so every
// row is read with coalesced loads; x is read about (M+K-1)/M times per
// modulus. The entries are written complete (wrap-around terms and the
// extension included, zeros from M+K-1 up to P), so the correlation kernels
// take them as given folds. With the Thm. 2 sampling, terms past N are the
// zero padding and the extension repeats the first entries.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "tm_internal.h"

namespace ftm {
namespace {

template <int DT>
__device__ __forceinline__ float entry(const void* x, int64_t n) {
  if constexpr (DT == TM_I8_PM1) return (__ldg(static_cast<const uint8_t*>(x) + n) & 2u) ? -1.0f : 1.0f;
  else if constexpr (DT == TM_BITS_PM1)
    return ((__ldg(static_cast<const uint8_t*>(x) + (n >> 3)) >> (n & 7)) & 1u) ? 1.0f : -1.0f;
  else if constexpr (DT == TM_F16) return __half2float(static_cast<const __half*>(x)[n]);
  else return __ldg(static_cast<const float*>(x) + n);
}

template <int DT>
__device__ __forceinline__ void fold_entry(const CorrQ& Q, int j, int64_t k, void* y) {
  const int64_t N = Q.N, M = Q.M[j], L = Q.L[j];
  const int64_t P = Q.P;
  constexpr bool kInt = DT == TM_I8_PM1 || DT == TM_BITS_PM1;
  int64_t si = 0;     // +-1 signals: exact integer sum
  float sf = 0.f;     // real signals: fp32, terms in the order l = 0, 1, ...
  if (k < M + Q.K - 1) {
    const int64_t c = Q.thm2 && k >= M ? k - M : k;   // Thm. 2: periodic extension
    for (int64_t l = 0; l < L; ++l) {
      int64_t n = c + l * M;
      if (n >= N) {
        if (Q.thm2) break;                             // zero padding
        n -= N;
        if (n >= N) n %= N;
      }
      const float v = entry<DT>(Q.x, n);
      if constexpr (kInt) si += v > 0.f ? 1 : -1;
      else sf += v;
    }
  }
  if constexpr (kInt) static_cast<int32_t*>(y)[int64_t(j) * P + k] = int32_t(si);
  else static_cast<float*>(y)[int64_t(j) * P + k] = sf;
}

__global__ void fold_direct_kernel(const CorrQ* q, const int32_t* idx, void* y_base) {
  const CorrQ Q = q[idx[blockIdx.z]];
  const int j = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= Q.nmod || k >= Q.P) return;
  void* y = static_cast<char*>(y_base) + Q.y_off * 4;
  switch (Q.xdtype) {
    case TM_I8_PM1: fold_entry<TM_I8_PM1>(Q, j, k, y); break;
    case TM_BITS_PM1: fold_entry<TM_BITS_PM1>(Q, j, k, y); break;
    case TM_F16: fold_entry<TM_F16>(Q, j, k, y); break;
    default: fold_entry<TM_F32>(Q, j, k, y); break;
  }
}

}  // namespace

cudaError_t launch_fold_direct(const CorrQ* q, const int32_t* idx, int32_t n, int32_t maxP, int32_t maxmod, void* y,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid(unsigned((maxP + 255) / 256), unsigned(maxmod), unsigned(n));
  fold_direct_kernel<<<grid, 256, 0, s>>>(q, idx, y);
  return cudaGetLastError();
}

}  // namespace ftm
