// Step 3 of Algorithm 1 (Eq. (2)) for moduli too wide for the streaming
// fold kernel's register-resident columns (M above about 2^14 entries), in
// two launches.
//
//  1. Partial sums: the L rows x_{k + l M} (l < L, k < M) are cut into dh
//     groups of about 16 consecutive rows; one thread per (four columns,
//     group) sums its rows' natural entries (k + l M < N) with the loads of
//     eight rows in flight at once. A warp's consecutive threads read
//     consecutive entries of x, so every row is read with coalesced loads.
//     int8 signals with at most 16 rows skip this stage (dh = 0).
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
  // the row pitch is a multiple of four columns: one 16-byte store (columns
  // past M land in the row's padding)
  int4* dst = reinterpret_cast<int4*>(partial + Q.dpart + (int64_t(j) * Q.dh + h) * Q.dpitch + k0);
  if constexpr (kInt) *dst = make_int4(si[0], si[1], si[2], si[3]);
  else *dst = make_int4(__float_as_int(sf[0]), __float_as_int(sf[1]), __float_as_int(sf[2]), __float_as_int(sf[3]));
}

__device__ __forceinline__ int i8b(const uint8_t* x, int64_t n) { return (__ldg(x + n) & 2u) ? -1 : 1; }

// int8 signals: the first stage for every modulus at once. A thread folds
// columns k0 .. k0+3 of each modulus over the group's rows; row l of
// modulus j starts at k0 + l M_j, so the rows of the moduli (M, M+1, ...)
// lie a few bytes apart and the second and third reads mostly hit L1.
// Eight rows of every modulus are in flight at a time; the byte lanes are
// unpacked every 64 rows.
template <int NM>
__device__ __forceinline__ void part_i8_all(const CorrQ& Q, int h, int64_t k0, int32_t* partial) {
  const int64_t N = Q.N, n16 = Q.N & ~int64_t(15);
  const uint32_t* X = static_cast<const uint32_t*>(Q.x);
  const uint8_t* x8 = static_cast<const uint8_t*>(Q.x);
  const int64_t l0 = int64_t(h) * Q.drows;
  int64_t lend[NM];
  uint32_t M[NM];
  int64_t lmain = INT64_MAX, Mmax = 0;
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    M[j] = uint32_t(Q.M[j]);
    const int64_t L = Q.L[j];
    lend[j] = min(L, l0 + Q.drows);
    lmain = min(lmain, min(lend[j], L - 1));   // rows natural for every column
    Mmax = max(Mmax, int64_t(M[j]));
  }
  // rows whose words stay inside the aligned prefix for every modulus:
  // k0 + l M + 8 <= n16 (int8 signals are below 2^31 bytes: 32-bit offsets)
  const int64_t lsafe = n16 >= k0 + 8 ? (n16 - 8 - k0) / Mmax + 1 : 0;
  const int64_t lfast = max(l0, min(lmain, lsafe));
  int s[NM][4];
  uint32_t acc[NM], a[NM];
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    acc[j] = 0u;
    a[j] = uint32_t(k0 + l0 * int64_t(M[j]));
#pragma unroll
    for (int c = 0; c < 4; ++c) s[j][c] = 0;
  }
  int64_t l = l0;
  int rows = 0;
  for (; l + 8 <= lfast; l += 8) {
    uint32_t w0[NM][8], w1[NM][8];
#pragma unroll
    for (int j = 0; j < NM; ++j) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint32_t au = a[j] + uint32_t(u) * M[j];
        w0[j][u] = __ldg(&X[au >> 2]);
        w1[j][u] = __ldg(&X[(au >> 2) + 1]);
      }
    }
#pragma unroll
    for (int j = 0; j < NM; ++j) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint32_t au = a[j] + uint32_t(u) * M[j];
        acc[j] = __vadd4(acc[j], __funnelshift_r(w0[j][u], w1[j][u], (au & 3u) << 3));
      }
      a[j] += 8u * M[j];
    }
    rows += 8;
    if (rows >= 56) {   // at most 64 rows per byte lane
#pragma unroll
      for (int j = 0; j < NM; ++j) {
#pragma unroll
        for (int c = 0; c < 4; ++c) s[j][c] += int(int8_t(uint8_t(acc[j] >> (8 * c))));
        acc[j] = 0u;
      }
      rows = 0;
    }
  }
#pragma unroll
  for (int j = 0; j < NM; ++j) {
#pragma unroll
    for (int c = 0; c < 4; ++c) s[j][c] += int(int8_t(uint8_t(acc[j] >> (8 * c))));
  }
  // the other rows of each modulus byte by byte (a short remainder, rows near
  // the end of the signal and the last row: natural entries only)
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    for (int64_t r = l; r < lend[j]; ++r) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t n = k0 + c + r * int64_t(M[j]);
        if (k0 + c < M[j] && n < N) s[j][c] += i8b(x8, n);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    if (k0 >= M[j]) continue;
    int4* dst = reinterpret_cast<int4*>(partial + Q.dpart + (int64_t(j) * Q.dh + h) * Q.dpitch + k0);
    *dst = make_int4(s[j][0], s[j][1], s[j][2], s[j][3]);
  }
}

__global__ void __launch_bounds__(kDirThreads) fold_direct_part_kernel(const CorrQ* q, const int32_t* idx,
                                                                       int32_t* partial) {
  const CorrQ& Q = q[idx[blockIdx.z]];   // read in place: no per-thread copy
  if (Q.xdtype == TM_I8_PM1) {          // every modulus in one thread: blockIdx.y is the group
    const int h = blockIdx.y;
    const int64_t k0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * kDirCols;
    int mmax = Q.M[0];
    for (int j = 1; j < Q.nmod; ++j) mmax = max(mmax, Q.M[j]);
    if (h >= Q.dh || k0 >= mmax) return;
    if (Q.nmod == 3) part_i8_all<3>(Q, h, k0, partial);
    else part_i8_all<2>(Q, h, k0, partial);
    return;
  }
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
  int32_t K, dh, thm2, pitch;
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
    const int32_t* ps = partial + Q.dpart + int64_t(j) * Q.dh * Q.pitch + c;
    // group sums in group order, eight loads in flight
    for (int h0 = 0; h0 < Q.dh; h0 += 8) {
      uint32_t w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        w[u] = h0 + u < Q.dh ? __ldg(reinterpret_cast<const uint32_t*>(ps) + int64_t(h0 + u) * Q.pitch) : 0u;
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
// int8 signals: four consecutive entries k0 .. k0+3 per thread, 32-bit
// index arithmetic where it fits, the group loads of the four entries in
// flight together.
__device__ __forceinline__ int i8v(const uint8_t* x, int64_t n) { return (__ldg(x + n) & 2u) ? -1 : 1; }

__device__ __forceinline__ void complete4_i8(const DirQ& D, int j, const int32_t* partial, int32_t* yj) {
  const int M = int(D.M), P = int(D.P), kend = int(D.M) + D.K - 1, dh = D.dh, pitch = D.pitch;
  const int k0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (k0 >= P) return;
  int c[4], s[4];
  bool live[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int k = k0 + u;
    live[u] = k < kend;
    c[u] = k < M ? k : k - M;
    s[u] = 0;
  }
  const int32_t* base = partial + D.dpart + int64_t(j) * dh * pitch;
#pragma unroll 4
  for (int h = 0; h < dh; ++h) {
    const int32_t* ph = base + int64_t(h) * pitch;
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] += live[u] ? __ldg(ph + c[u]) : 0;
  }
  if (!D.thm2) {
    const uint8_t* x = static_cast<const uint8_t*>(D.x);
    const int64_t wr = (D.L - 1) * D.M - D.N, ex = D.L * D.M - D.N;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!live[u]) continue;
      const int64_t w = c[u] + wr;   // the last row's entry past N wraps around
      if (w >= 0) s[u] += i8v(x, w);
      if (k0 + u >= M) {              // extension: y[M+c] = y[c] - x_c + x_{(c + L M) mod N}
        int64_t e = c[u] + ex;
        if (e >= D.N) e %= D.N;
        s[u] += i8v(x, e) - i8v(x, c[u]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) if (!live[u]) s[u] = 0;
  int32_t* o = yj + k0;
  if ((reinterpret_cast<uintptr_t>(o) & 15) == 0) {
    *reinterpret_cast<int4*>(o) = make_int4(s[0], s[1], s[2], s[3]);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) o[u] = s[u];   // P is a multiple of 4: k0 + 3 < P
  }
}

// int8 signals with at most 16 rows (no first stage, dh = 0): sixteen
// consecutive entries per thread summed from the definition,
// y[k] = sum_{l<L} x_{(k + l M) mod N} (Thm. 2: terms below N of entry
// k mod M). Each row's sixteen bytes come from five aligned words and four
// funnel shifts and are added bytewise (at most 16 terms per byte lane), so
// the index arithmetic of a row is shared by sixteen entries; rows whose
// words would leave the signal's 16-byte-aligned prefix, or that wrap within
// the sixteen bytes, go byte by byte.
constexpr int kDirRun = 16;   // consecutive entries per thread of the direct int8 path

__device__ __forceinline__ void direct16_i8(const DirQ& D, int32_t* yj) {
  const int M = int(D.M), P = int(D.P), kend = int(D.M) + D.K - 1, L = int(D.L);
  const int64_t N = D.N, n16 = D.N & ~int64_t(15);
  const int k0 = (blockIdx.x * blockDim.x + threadIdx.x) * kDirRun;
  if (k0 >= P) return;
  int s[kDirRun];
#pragma unroll
  for (int u = 0; u < kDirRun; ++u) s[u] = 0;
  if (k0 < kend) {
    const uint8_t* x = static_cast<const uint8_t*>(D.x);
    const uint32_t* X = static_cast<const uint32_t*>(D.x);
    if (D.thm2 && k0 < M && k0 + kDirRun > M) {
      // Thm. 2 with the sixteen entries on both sides of M: entry by entry
      for (int u = 0; u < kDirRun; ++u) {
        const int k = k0 + u;
        const int64_t c = k >= M ? k - M : k;
        for (int l = 0; l < L; ++l) {
          const int64_t n = c + int64_t(l) * M;
          if (n >= N) break;
          s[u] += i8v(x, n);
        }
      }
    } else {
      const int64_t cb = D.thm2 && k0 >= M ? k0 - M : k0;   // consecutive columns cb .. cb+15
      uint32_t acc[kDirRun / 4] = {0u, 0u, 0u, 0u};
#pragma unroll 2
      for (int l = 0; l < L; ++l) {
        int64_t n = cb + int64_t(l) * M;
        if (n >= N && !D.thm2) {
          n -= N;
          if (n >= N) n %= N;
        }
        if (n + kDirRun + 4 <= n16) {
          const uint32_t* w = X + (n >> 2);
          uint32_t v[kDirRun / 4 + 1];
#pragma unroll
          for (int b = 0; b <= kDirRun / 4; ++b) v[b] = __ldg(w + b);
          const int sh = int(n & 3) * 8;
#pragma unroll
          for (int b = 0; b < kDirRun / 4; ++b) acc[b] = __vadd4(acc[b], __funnelshift_r(v[b], v[b + 1], sh));
        } else {
          // near the end of the signal: byte by byte
#pragma unroll
          for (int u = 0; u < kDirRun; ++u) {
            int64_t nn = n + u;
            if (nn >= N) {
              if (D.thm2) continue;   // zero padding
              nn -= N;
            }
            s[u] += i8v(x, nn);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kDirRun; ++u) s[u] += int(int8_t(uint8_t(acc[u >> 2] >> (8 * (u & 3)))));
    }
#pragma unroll
    for (int u = 0; u < kDirRun; ++u)
      if (k0 + u >= kend) s[u] = 0;
  }
  // The warp's 512 entries are contiguous (P is a multiple of 512, so whole
  // warps return above): they go out through shared memory as 16-byte
  // stores of consecutive lanes. Slot s of the staging area sits at
  // s ^ ((s >> 3) & 7), so both the writes (lane stride four slots) and the
  // reads (consecutive slots) hit eight distinct 16-byte bank groups per
  // quarter warp.
  __shared__ int4 stage[kDirThreads / 32][32 * kDirRun / 4];
  int4* st = stage[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  int32_t* o = yj + (k0 - lane * kDirRun);   // the warp's first entry
  if ((reinterpret_cast<uintptr_t>(o) & 15) == 0) {
#pragma unroll
    for (int b = 0; b < kDirRun / 4; ++b) {
      const int sl = lane * (kDirRun / 4) + b;
      st[sl ^ ((sl >> 3) & 7)] = make_int4(s[4 * b], s[4 * b + 1], s[4 * b + 2], s[4 * b + 3]);
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < kDirRun / 4; ++b) {
      const int sl = b * 32 + lane;
      reinterpret_cast<int4*>(o)[sl] = st[sl ^ ((sl >> 3) & 7)];
    }
  } else {
    int32_t* ot = yj + k0;
#pragma unroll
    for (int u = 0; u < kDirRun; ++u) ot[u] = s[u];   // P is a multiple of 16: k0 + 15 < P
  }
}

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

__global__ void __launch_bounds__(kDirThreads, 4) fold_direct_complete_kernel(const CorrQ* q, const int32_t* idx,
                                                                           const int32_t* partial, void* y_base) {
  const CorrQ& Q = q[idx[blockIdx.z]];
  const int j = blockIdx.y;
  if (j >= Q.nmod) return;
  DirQ D;
  D.x = Q.x; D.N = Q.N; D.M = Q.M[j]; D.L = Q.L[j]; D.P = Q.P; D.dpart = Q.dpart;
  D.K = Q.K; D.dh = Q.dh; D.thm2 = Q.thm2; D.pitch = Q.dpitch;
  const int dt = Q.xdtype;
  void* y = static_cast<char*>(y_base) + Q.y_off * 4;
  // kDirCols entries per thread, a block's threads on consecutive k
  switch (dt) {
    case TM_I8_PM1:
      if (D.dh == 0) direct16_i8(D, static_cast<int32_t*>(y) + int64_t(j) * D.P);
      else complete4_i8(D, j, partial, static_cast<int32_t*>(y) + int64_t(j) * D.P);
      break;
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
  if (maxHM > 0) {   // some query has row groups (dh > 0)
    const dim3 g1(unsigned((maxM + per - 1) / per), unsigned(maxHM), unsigned(n));
    fold_direct_part_kernel<<<g1, kDirThreads, 0, s>>>(q, idx, partial);
  }
  // every query int8 with at most 16 rows: sixteen entries per thread
  const int64_t per2 = maxHM > 0 ? per : int64_t(kDirThreads) * kDirRun;
  const dim3 g2(unsigned((maxP + per2 - 1) / per2), unsigned(maxmod), unsigned(n));
  fold_direct_complete_kernel<<<g2, kDirThreads, 0, s>>>(q, idx, partial, y);
  return cudaGetLastError();
}

}  // namespace ftm
