// Step 3 of Algorithm 1 (Eq. (2)) for +-1 signals stored as int8:
// column sums of x viewed as rows of length M, for both moduli, from a
// single read of x.
//
// Design: the signals of a batch are concatenated (16-byte-aligned prefixes)
// into one byte space that is split into equal contiguous shares, one per
// CTA. A producer warp streams a CTA's share through a ring of shared-memory
// stages with bulk asynchronous copies (TMA, cp.async.bulk). Consumer lanes
// own fixed 16-column units of one modulus, dealt out in chunks of 32
// consecutive units per warp (8 warps for M1, 9 for M2, so that K and K+1
// columns both come to one chunk per warp when K = 4096). For a stage holding
// bytes [s, e) of a signal every lane of a warp walks the same rows l of its
// modulus: rows strictly inside the stage take the fast path (one or two
// aligned 16-byte shared-memory reads, re-aligned by funnel shifts by the
// warp-uniform offset (l*Mp - s) mod 16), the first and last row the same
// read followed by a byte mask for the part inside the stage. Stages carry
// 16 bytes of slack on both sides so every read stays in bounds.
//
// A byte holding -1 (0xFF) has bit 1 set and +1 (0x01) has not, so
// w & 0x02020202 adds 2 per -1 entry into four packed byte-lane counters.
// A unit narrower than 16 columns (the last one of a row) still counts all
// 16 bytes; the lanes past its width see bytes of the next row and are never
// written out. Byte lanes are widened into 16-bit lanes every few stages and
// written as int32 counts of -1 entries per (share, column) at the end of a
// share. The correlation kernel turns the counts into y (Eq. (2)) and adds
// the wrap-around term and the extension k >= M.
//
// To keep every lane busy the fold runs with an effective modulus
// Mp = R*M >= 4096 (R = ceil(4096/M)); the correlation kernel sums the R
// columns k + rM of the Mp-fold into column k of the M-fold.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "tm_internal.h"

namespace ftm {
namespace {

constexpr int kStageBytes = kFoldTile + 32;   // 16 bytes of slack before and after the data
constexpr uint32_t kNegBit = 0x02020202u;

__device__ __forceinline__ uint32_t fsr(uint32_t lo, uint32_t hi, uint32_t sh) {
  return __funnelshift_r(lo, hi, sh);
}

// Bytes [o, o+16) of a stage as 4 words, -16 < o < valid + 16 (the slack
// keeps both aligned reads inside the stage); r = o & 15 must be the same
// in every lane of the warp.
__device__ __forceinline__ void load16(const uint8_t* buf, int o, uint32_t (&w)[4]) {
  const uint4* p = reinterpret_cast<const uint4*>(buf + (o & ~15));
  const uint4 a = p[0];
  const int r = o & 15;
  if (r == 0) {
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    return;
  }
  const uint4 b = p[1];
  const uint32_t sh = uint32_t(r & 3) * 8u;
  switch (r >> 2) {
    case 0: w[0] = fsr(a.x, a.y, sh); w[1] = fsr(a.y, a.z, sh); w[2] = fsr(a.z, a.w, sh); w[3] = fsr(a.w, b.x, sh); break;
    case 1: w[0] = fsr(a.y, a.z, sh); w[1] = fsr(a.z, a.w, sh); w[2] = fsr(a.w, b.x, sh); w[3] = fsr(b.x, b.y, sh); break;
    case 2: w[0] = fsr(a.z, a.w, sh); w[1] = fsr(a.w, b.x, sh); w[2] = fsr(b.x, b.y, sh); w[3] = fsr(b.y, b.z, sh); break;
    default: w[0] = fsr(a.w, b.x, sh); w[1] = fsr(b.x, b.y, sh); w[2] = fsr(b.y, b.z, sh); w[3] = fsr(b.z, b.w, sh); break;
  }
}

// Low n bytes of a word set (n clamped to [0, 4]).
__device__ __forceinline__ uint32_t low_bytes(int n) {
  return n <= 0 ? 0u : n >= 4 ? 0xFFFFFFFFu : (1u << (8 * n)) - 1u;
}

// Counts the bytes of [o, o+16) that lie inside the stage [0, len).
__device__ __forceinline__ void count_masked(const uint8_t* buf, int o, int len, uint32_t (&c8)[4]) {
  uint32_t w[4];
  load16(buf, o, w);
  const int lo = -o, hi = len - o;   // valid byte positions lo <= i < hi
#pragma unroll
  for (int k = 0; k < 4; ++k) c8[k] += w[k] & (kNegBit & low_bytes(hi - 4 * k) & ~low_bytes(lo - 4 * k));
}

__device__ __forceinline__ void count(uint32_t (&c8)[4], const uint32_t (&w)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) c8[i] += w[i] & kNegBit;
}

__device__ __forceinline__ void count2(uint32_t (&c8)[4], const uint32_t (&w)[4], const uint32_t (&v)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) c8[i] += (w[i] & kNegBit) + (v[i] & kNegBit);
}

// First query whose byte range ends after `pos`.
__device__ __forceinline__ int first_query(const FoldQ* q, int nq, int64_t pos) {
  int lo = 0, hi = nq;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (q[mid].goff + q[mid].nbytes > pos) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// One consumer lane's work on one share [lo, hi) (signal-local bytes) for
// the effective modulus Mp: units lane + 32 (wig + W j), j < J, where wig is
// the warp's index among the W warps of its modulus. Returns false when a
// bounded wait ran out.
template <int J>
__device__ __forceinline__ bool consume_share(const uint8_t* smem, uint64_t* full, uint64_t* empty, int lo, int hi,
                                              int Mp, int W, int wig, int32_t* dst, uint32_t& it) {
  const int lane = threadIdx.x & 31;
  const int G = (Mp + 15) >> 4;
  // Stages between widenings: a unit meets at most kFoldTile/Mp + 2 rows
  // per stage and a byte lane holds up to 127 of them (2 per -1 entry).
  const int F = max(1, 127 / (kFoldTile / Mp + 2));

  int col[J];
  bool live[J];
  uint32_t c8[J][4], c16[J][8];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int g = lane + 32 * (wig + W * j);
    col[j] = 16 * g;
    live[j] = g < G;
#pragma unroll
    for (int i = 0; i < 4; ++i) c8[j][i] = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) c16[j][i] = 0u;
  }

  int since = 0;
  for (int s = lo; s < hi; s += kFoldTile) {
    const uint32_t st = it % kFoldStages;
    // every lane waits; the warp gives up together so no lane is left
    // behind at the __syncwarp below
    if (!__all_sync(0xffffffffu, mbar_wait(&full[st], (it / kFoldStages) & 1u))) return false;
    const uint8_t* buf = smem + st * kStageBytes + 16;
    const int len = min(kFoldTile, hi - s);
    const int l0 = s / Mp;               // rows meeting [s, s+len)
    const int l1 = (s + len - 1) / Mp;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (!live[j]) continue;
      // first row: the unit may start before the stage (or end after it)
      {
        const int o = l0 * Mp + col[j] - s;
        if (o > -16 && o < len) count_masked(buf, o, len, c8[j]);
      }
      if (l1 > l0) {
        // rows strictly inside the stage: all 16 bytes are present (a narrow
        // last unit reads at most 15 bytes of slack, counted in lanes that
        // are never written)
        int l = l0 + 1;
        for (; l + 1 < l1; l += 2) {
          uint32_t w[4], v[4];
          const int o = l * Mp + col[j] - s;
          load16(buf, o, w);
          load16(buf, o + Mp, v);
          count2(c8[j], w, v);
        }
        if (l < l1) {
          uint32_t w[4];
          load16(buf, l * Mp + col[j] - s, w);
          count(c8[j], w);
        }
        // last row: the unit may run past the stage
        const int o = l1 * Mp + col[j] - s;
        if (o < len) count_masked(buf, o, len, c8[j]);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    ++it;
    if (++since == F) {
      since = 0;
#pragma unroll
      for (int j = 0; j < J; ++j) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          c16[j][2 * i] += c8[j][i] & 0x00FF00FFu;
          c16[j][2 * i + 1] += (c8[j][i] >> 8) & 0x00FF00FFu;
          c8[j][i] = 0u;
        }
      }
    }
  }

  // Widen the remainder and write this share's counts of -1 entries.
#pragma unroll
  for (int j = 0; j < J; ++j) {
    if (!live[j]) continue;
    int32_t cnt[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t e0 = c16[j][2 * i] + (c8[j][i] & 0x00FF00FFu);
      const uint32_t e1 = c16[j][2 * i + 1] + ((c8[j][i] >> 8) & 0x00FF00FFu);
      cnt[4 * i + 0] = int32_t((e0 & 0xFFFFu) >> 1);
      cnt[4 * i + 2] = int32_t(e0 >> 17);
      cnt[4 * i + 1] = int32_t((e1 & 0xFFFFu) >> 1);
      cnt[4 * i + 3] = int32_t(e1 >> 17);
    }
    const int width = min(16, Mp - col[j]);
    if (width == 16) {
      int4* d4 = reinterpret_cast<int4*>(dst + col[j]);
      d4[0] = make_int4(cnt[0], cnt[1], cnt[2], cnt[3]);
      d4[1] = make_int4(cnt[4], cnt[5], cnt[6], cnt[7]);
      d4[2] = make_int4(cnt[8], cnt[9], cnt[10], cnt[11]);
      d4[3] = make_int4(cnt[12], cnt[13], cnt[14], cnt[15]);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (i < width) dst[col[j] + i] = cnt[i];
    }
  }
  return true;
}

// JMAX: the most units any lane of the launch needs (3 covers moduli up to
// 12288; larger moduli use the 5-unit instantiation).
template <int JMAX>
__global__ void __launch_bounds__(kFoldThreads, 1) fold_i8_kernel(const FoldArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kFoldStages * kStageBytes);
  uint64_t* empty = full + kFoldStages;

  const int tid = threadIdx.x;
  const int64_t cb = fold_cta_begin(a.W, a.nctas, blockIdx.x);
  const int64_t ce = fold_cta_begin(a.W, a.nctas, blockIdx.x + 1);

  if (tid == 0) {
    for (int s = 0; s < kFoldStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kFoldConsumers / 32);
    }
    mbar_init_fence();
  }
  __syncthreads();
  if (cb >= ce) return;
  const int q0 = first_query(a.q, a.nq, cb);

  // ---------------------------------------------------------------- producer
  if (tid >= kFoldConsumers) {
    if (tid == kFoldConsumers) {
      const uint64_t pol = l2_policy_evict_first();
      uint32_t it = 0;
      bool ok = true;
      for (int qi = q0; qi < a.nq && ok; ++qi) {
        const int64_t goff = a.q[qi].goff;
        const int32_t nbytes = a.q[qi].nbytes;
        const uint8_t* x = a.q[qi].x;
        if (goff >= ce) break;
        if (nbytes == 0) continue;
        const int64_t lo = max(cb, goff) - goff;
        const int64_t hi = min(ce, goff + nbytes) - goff;
        for (int64_t s = lo; s < hi; s += kFoldTile) {
          const uint32_t st = it % kFoldStages;
          if (it >= kFoldStages && !mbar_wait(&empty[st], ((it / kFoldStages) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          const uint32_t len = uint32_t(hi - s < kFoldTile ? hi - s : int64_t(kFoldTile));
          mbar_arrive_expect_tx(&full[st], len);
          bulk_load(smem + st * kStageBytes + 16, x + s, len, &full[st], pol);
          ++it;
        }
      }
      if (!ok) atomicOr(a.err, 1);
      // Let every copy this thread issued land before the CTA may exit.
      for (uint32_t k = it > kFoldStages ? it - kFoldStages : 0; k < it; ++k)
        (void)mbar_wait(&full[k % kFoldStages], (k / kFoldStages) & 1u);
    }
    return;
  }

  // ---------------------------------------------------------------- consumers
  const int warp = tid >> 5;
  const int m = warp < kFoldWarps0 ? 0 : 1;         // modulus handled by this warp
  const int W = m == 0 ? kFoldWarps0 : kFoldWarps1;
  const int wig = m == 0 ? warp : warp - kFoldWarps0;
  uint32_t it = 0;
  bool ok = true;
  for (int qi = q0; qi < a.nq && ok; ++qi) {
    const int64_t goff = a.q[qi].goff;
    const int32_t nbytes = a.q[qi].nbytes;
    if (goff >= ce) break;
    if (nbytes == 0) continue;
    const int lo = int(max(cb, goff) - goff);
    const int hi = int(min(ce, goff + nbytes) - goff);
    const int Mp = a.q[qi].Mp[m];
    int32_t* dst = a.partial + a.q[qi].part + int64_t(blockIdx.x - a.q[qi].first_cta) * a.q[qi].stride +
                   a.q[qi].moff[m];
    const int J = fold_units_per_lane(Mp, W);
    if (J <= 1) ok = consume_share<1>(smem, full, empty, lo, hi, Mp, W, wig, dst, it);
    else if (J == 2) ok = consume_share<2>(smem, full, empty, lo, hi, Mp, W, wig, dst, it);
    else if (J == 3 || JMAX == 3) ok = consume_share<3>(smem, full, empty, lo, hi, Mp, W, wig, dst, it);
    else ok = consume_share<(JMAX > 3 ? JMAX : 3)>(smem, full, empty, lo, hi, Mp, W, wig, dst, it);
  }
  if (!ok) atomicOr(a.err, 1);
}

}  // namespace

cudaError_t fold_configure() {
  const int smem = kFoldStages * kStageBytes + 2 * kFoldStages * 8;
  cudaError_t e = cudaFuncSetAttribute(fold_i8_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fold_i8_kernel<kFoldJMax>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_fold_i8(const FoldArgs& a, int jmax, cudaStream_t s) {
  const int smem = kFoldStages * kStageBytes + 2 * kFoldStages * 8;
  if (jmax <= 3) fold_i8_kernel<3><<<a.nctas, kFoldThreads, smem, s>>>(a);
  else fold_i8_kernel<kFoldJMax><<<a.nctas, kFoldThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ftm
