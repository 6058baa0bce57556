// Step 3 of Algorithm 1 (Eq. (2)) for moduli too wide for the streaming
// fold kernel's register-resident columns (M above about 2^14 entries), in
// two launches.
//
//  1. Partial sums: the L rows x_{k + l M} (l < L, k < M) are cut into dh
//     groups of about 16 consecutive rows; one thread per (four columns,
//     group) sums its rows' natural entries (k + l M < N) with the loads of
//     eight rows in flight at once. A warp's consecutive threads read
//     consecutive entries of x, so every row is read with coalesced loads.
//  2. Completion, one thread per fold entry k < M+K-1: the group sums in
//     group order, the wrap-around entry x_{k + (L-1) M - N} when the last
//     row runs past N, and for k >= M the extension
//     y[M+i] = y[i] - x_i + x_{(i + L M) mod N}; zeros from M+K-1 up to P.
//     With the Thm. 2 sampling, terms past N are the zero padding and the
//     extension repeats the first entries (y[M+i] = y[i]).
// +-1 signals are summed exactly in int32; real signals in fp32 in a fixed
// order (rows within a group, then the groups), so the folds do not depend
// on the launch.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "tm_internal.h"

namespace ftm {
namespace {

constexpr int kDirThreads = 256;

template <int DT>
__device__ __forceinline__ float entry(const void* x, int64_t n) {
  if constexpr (DT == TM_I8_PM1) return (__ldg(static_cast<const uint8_t*>(x) + n) & 2u) ? -1.0f : 1.0f;
  else if constexpr (DT == TM_BITS_PM1)
    return ((__ldg(static_cast<const uint8_t*>(x) + (n >> 3)) >> (n & 7)) & 1u) ? 1.0f : -1.0f;
  else if constexpr (DT == TM_F16) return __half2float(static_cast<const __half*>(x)[n]);
  else return __ldg(static_cast<const float*>(x) + n);
}

// Sums of the group's natural entries for columns k0 .. k0+3 (those < M).
// Rows l < L-1 are natural for every column; the last row only where
// k + (L-1) M < N. int8 rows are read as aligned 32-bit words (a funnel
// shift picks the four bytes of the row) and summed bytewise (__vadd4: each
// byte lane keeps its column's sum modulo 256, unpacked every 64 rows, so
// the +-1 sums stay within a signed byte) while the words lie within the
// signal's 16-byte-aligned prefix; other rows and storage types entry by
// entry.
template <int DT>
__device__ __forceinline__ void part_cols(const CorrQ& Q, int j, int h, int64_t k0, int32_t* partial) {
  constexpr bool kInt = DT == TM_I8_PM1 || DT == TM_BITS_PM1;
  const int64_t N = Q.N, M = Q.M[j], L = Q.L[j];
  const int64_t l0 = int64_t(h) * Q.drows;
  const int64_t lend = min(L, l0 + Q.drows);
  const int64_t lfull = min(lend, L - 1);
  int si[kDirCols] = {0, 0, 0, 0};
  float sf[kDirCols] = {0.f, 0.f, 0.f, 0.f};
  int64_t l = l0;
  if constexpr (DT == TM_I8_PM1) {
    const int64_t n16 = Q.N & ~int64_t(15);   // bytes readable as whole words
    // rows whose two words end inside the aligned prefix: k0 + l M + 8 <= n16
    const int64_t lw = n16 >= k0 + 8 ? min(lfull, (n16 - 8 - k0) / M + 1) : l0;
    const uint32_t* X = static_cast<const uint32_t*>(Q.x);
    while (l < lw) {
      const int64_t lb = min(lw, l + 64);
      uint32_t acc = 0;
      for (; l + 8 <= lb; l += 8) {
        uint32_t w[8][2];
        int sh[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int64_t a = k0 + (l + u) * M;
          w[u][0] = __ldg(&X[a >> 2]);
          w[u][1] = __ldg(&X[(a >> 2) + 1]);
          sh[u] = int(a & 3) * 8;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = __vadd4(acc, __funnelshift_r(w[u][0], w[u][1], sh[u]));
      }
      for (; l < lb; ++l) {
        const int64_t a = k0 + l * M;
        acc = __vadd4(acc, __funnelshift_r(__ldg(&X[a >> 2]), __ldg(&X[(a >> 2) + 1]), int(a & 3) * 8));
      }
#pragma unroll
      for (int u = 0; u < kDirCols; ++u) si[u] += int(int8_t(uint8_t(acc >> (8 * u))));
    }
  }
  for (; l < lfull; ++l) {
#pragma unroll
    for (int u = 0; u < kDirCols; ++u) {
      if (k0 + u >= M) break;
      const float v = entry<DT>(Q.x, k0 + u + l * M);
      if constexpr (kInt) si[u] += v > 0.f ? 1 : -1;
      else sf[u] += v;
    }
  }
  if (lend == L && L - 1 >= l0) {   // the group holds the last row
#pragma unroll
    for (int u = 0; u < kDirCols; ++u) {
      const int64_t n = k0 + u + (L - 1) * M;
      if (k0 + u >= M || n >= N) continue;
      const float v = entry<DT>(Q.x, n);
      if constexpr (kInt) si[u] += v > 0.f ? 1 : -1;
      else sf[u] += v;
    }
  }
  int32_t* dst = partial + Q.dpart + (int64_t(j) * Q.dh + h) * M + k0;
#pragma unroll
  for (int u = 0; u < kDirCols; ++u) {
    if (k0 + u >= M) break;
    if constexpr (kInt) dst[u] = si[u];
    else reinterpret_cast<float*>(dst)[u] = sf[u];
  }
}

__global__ void __launch_bounds__(kDirThreads) fold_direct_part_kernel(const CorrQ* q, const int32_t* idx,
                                                                       int32_t* partial) {
  const CorrQ& Q = q[idx[blockIdx.z]];   // read in place: no per-thread copy
  const int j = blockIdx.y % Q.nmod, h = blockIdx.y / Q.nmod;
  const int64_t k0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * kDirCols;
  if (h >= Q.dh || k0 >= Q.M[j]) return;
  switch (Q.xdtype) {
    case TM_I8_PM1: part_cols<TM_I8_PM1>(Q, j, h, k0, partial); break;
    case TM_BITS_PM1: part_cols<TM_BITS_PM1>(Q, j, h, k0, partial); break;
    case TM_F16: part_cols<TM_F16>(Q, j, h, k0, partial); break;
    default: part_cols<TM_F32>(Q, j, h, k0, partial); break;
  }
}

// The fields of one query's modulus j that the completion needs, in
// registers (stores through y could alias the descriptor otherwise).
struct DirQ {
  const void* x;
  int64_t N, M, L, P, dpart;
  int32_t K, dh, thm2;
};

// Value of fold entry k (int32 bits for +-1 signals, else fp32 bits).
template <int DT>
__device__ __forceinline__ uint32_t complete_entry(const DirQ& Q, int j, int64_t k, const int32_t* partial) {
  constexpr bool kInt = DT == TM_I8_PM1 || DT == TM_BITS_PM1;
  const int64_t N = Q.N, M = Q.M, L = Q.L;
  float vf = 0.f;
  int vi = 0;
  if (k < M + Q.K - 1) {
    const int64_t c = k < M ? k : k - M;
    const int32_t* ps = partial + Q.dpart + int64_t(j) * Q.dh * M + c;
    // group sums in group order, eight loads in flight
    for (int h0 = 0; h0 < Q.dh; h0 += 8) {
      uint32_t w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) w[u] = h0 + u < Q.dh ? __ldg(reinterpret_cast<const uint32_t*>(ps) + int64_t(h0 + u) * M) : 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if constexpr (kInt) vi += int(w[u]);
        else vf += __uint_as_float(w[u]);
      }
    }
    auto add = [&](int64_t n, int sign) {
      const float v = entry<DT>(Q.x, n);
      if constexpr (kInt) vi += sign * (v > 0.f ? 1 : -1);
      else vf = sign > 0 ? vf + v : vf - v;
    };
    if (!Q.thm2) {
      const int64_t w = c + (L - 1) * M - N;   // the last row's entry past N wraps around
      if (w >= 0) add(w, 1);
      if (k >= M) {   // extension: y[M+c] = y[c] - x_c + x_{(c + L M) mod N}
        add(c, -1);
        int64_t e = c + L * M - N;
        if (e >= N) e %= N;
        add(e, 1);
      }
    }
  }
  if constexpr (kInt) return uint32_t(vi);
  else return __float_as_uint(vf);
}

// kDirCols entries per thread (a block's threads on consecutive k): all
// loads first, then the stores.
template <int DT>
__device__ __forceinline__ void complete_cols(const DirQ& D, int j, const int32_t* partial, void* y) {
  uint32_t v[kDirCols];
#pragma unroll
  for (int u = 0; u < kDirCols; ++u) {
    const int64_t k = (int64_t(blockIdx.x) * kDirCols + u) * blockDim.x + threadIdx.x;
    v[u] = k < D.P ? complete_entry<DT>(D, j, k, partial) : 0u;
  }
  uint32_t* yo = static_cast<uint32_t*>(y) + int64_t(j) * D.P;
#pragma unroll
  for (int u = 0; u < kDirCols; ++u) {
    const int64_t k = (int64_t(blockIdx.x) * kDirCols + u) * blockDim.x + threadIdx.x;
    if (k < D.P) yo[k] = v[u];
  }
}

__global__ void __launch_bounds__(kDirThreads) fold_direct_complete_kernel(const CorrQ* q, const int32_t* idx,
                                                                           const int32_t* partial, void* y_base) {
  const CorrQ& Q = q[idx[blockIdx.z]];
  const int j = blockIdx.y;
  if (j >= Q.nmod) return;
  DirQ D;
  D.x = Q.x; D.N = Q.N; D.M = Q.M[j]; D.L = Q.L[j]; D.P = Q.P; D.dpart = Q.dpart;
  D.K = Q.K; D.dh = Q.dh; D.thm2 = Q.thm2;
  const int dt = Q.xdtype;
  void* y = static_cast<char*>(y_base) + Q.y_off * 4;
  // kDirCols entries per thread, a block's threads on consecutive k
  switch (dt) {
    case TM_I8_PM1: complete_cols<TM_I8_PM1>(D, j, partial, y); break;
    case TM_BITS_PM1: complete_cols<TM_BITS_PM1>(D, j, partial, y); break;
    case TM_F16: complete_cols<TM_F16>(D, j, partial, y); break;
    default: complete_cols<TM_F32>(D, j, partial, y); break;
  }
}

}  // namespace

cudaError_t launch_fold_direct(const CorrQ* q, const int32_t* idx, int32_t n, int32_t maxP, int32_t maxmod,
                               int32_t maxM, int32_t maxHM, int32_t* partial, void* y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t per = int64_t(kDirThreads) * kDirCols;
  const dim3 g1(unsigned((maxM + per - 1) / per), unsigned(maxHM), unsigned(n));
  fold_direct_part_kernel<<<g1, kDirThreads, 0, s>>>(q, idx, partial);
  const dim3 g2(unsigned((maxP + per - 1) / per), unsigned(maxmod), unsigned(n));
  fold_direct_complete_kernel<<<g2, kDirThreads, 0, s>>>(q, idx, partial, y);
  return cudaGetLastError();
}

}  // namespace ftm
