// Step 3 of Algorithm 1 (Eq. (2)) for +-1 signals stored as int8:
// column sums of x viewed as rows of length M, for both moduli, from a
// single read of x.
//
// Design: the signals of a batch are concatenated (16-byte-aligned prefixes)
// into one byte space that is split into equal contiguous shares, one per
// CTA. A producer warp streams a CTA's share through a ring of shared-memory
// stages with bulk asynchronous copies (TMA, cp.async.bulk). Each consumer
// thread owns fixed 16-column units of one modulus and, for every row of
// that modulus crossing the stage, adds the unit's 16 bytes into packed
// byte-lane counters (a byte holding -1 = 0xFF has bit 1 set, +1 = 0x01 has
// not). Rows of the odd modulus start at every byte offset, so the unit is
// re-aligned from two aligned 16-byte shared-memory reads with funnel
// shifts. Byte lanes are widened into 16-bit lanes every few stages and
// written out as int32 counts of -1 entries per (share, column) at the end
// of a share. The correlation kernel turns counts into y (Eq. (2)) and adds
// the wrap-around term and the extension k >= M.
//
// To keep every consumer busy the fold runs with an effective modulus
// Mp = R*M >= 4096 (R = ceil(4096/M)); the correlation kernel sums the R
// columns k + rM of the Mp-fold into column k of the M-fold.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "tm_internal.h"

namespace ftm {
namespace {

constexpr int kStageBytes = kFoldTile + 16;   // slack: the re-aligning read may run 15 bytes past

__device__ __forceinline__ uint32_t fsr(uint32_t lo, uint32_t hi, uint32_t sh) {
  return __funnelshift_r(lo, hi, sh);
}

// Bytes [o, o+16) of a stage, o >= 0 and o + 16 <= valid bytes.
__device__ __forceinline__ void load16(const uint8_t* buf, int o, uint32_t& w0, uint32_t& w1, uint32_t& w2,
                                       uint32_t& w3) {
  const uint4* p = reinterpret_cast<const uint4*>(buf + (o & ~15));
  const uint4 a = p[0];
  const int r = o & 15;
  if (r == 0) {
    w0 = a.x; w1 = a.y; w2 = a.z; w3 = a.w;
    return;
  }
  const uint4 b = p[1];
  const uint32_t sh = uint32_t(r & 3) * 8u;
  switch (r >> 2) {
    case 0: w0 = fsr(a.x, a.y, sh); w1 = fsr(a.y, a.z, sh); w2 = fsr(a.z, a.w, sh); w3 = fsr(a.w, b.x, sh); break;
    case 1: w0 = fsr(a.y, a.z, sh); w1 = fsr(a.z, a.w, sh); w2 = fsr(a.w, b.x, sh); w3 = fsr(b.x, b.y, sh); break;
    case 2: w0 = fsr(a.z, a.w, sh); w1 = fsr(a.w, b.x, sh); w2 = fsr(b.x, b.y, sh); w3 = fsr(b.y, b.z, sh); break;
    default: w0 = fsr(a.w, b.x, sh); w1 = fsr(b.x, b.y, sh); w2 = fsr(b.y, b.z, sh); w3 = fsr(b.z, b.w, sh); break;
  }
}

// Bytes i < width of the unit at stage offset o that lie inside [0, len);
// everything else reads as 0 (counts nothing).
__device__ __forceinline__ void load_masked(const uint8_t* buf, int o, int len, int width, uint32_t& w0,
                                            uint32_t& w1, uint32_t& w2, uint32_t& w3) {
  w0 = w1 = w2 = w3 = 0u;
  const int i0 = o < 0 ? -o : 0;
  const int i1 = min(width, len - o);
  for (int i = i0; i < i1; ++i) {
    const uint32_t v = uint32_t(buf[o + i]) << (8 * (i & 3));
    const int k = i >> 2;
    w0 |= (k == 0) ? v : 0u;
    w1 |= (k == 1) ? v : 0u;
    w2 |= (k == 2) ? v : 0u;
    w3 |= (k == 3) ? v : 0u;
  }
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

// One consumer thread's work on one share [lo, hi) (query-local bytes) of a
// signal, for J units of the effective modulus Mp: units t + 256 j, j < J.
// Returns false when a bounded wait ran out.
template <int J>
__device__ __forceinline__ bool consume_share(const uint8_t* smem, uint64_t* full, uint64_t* empty, int lo, int hi,
                                              int Mp, int tm, int32_t* dst, uint32_t& it) {
  const int lane = threadIdx.x & 31;
  const int G = (Mp + 15) >> 4;
  // Stages between widenings: a unit meets at most kFoldTile/Mp + 2 rows
  // per stage and a byte lane holds up to 127 of them (2 per -1 entry).
  const int F = max(1, 127 / (kFoldTile / Mp + 2));

  int pos[J], wid[J];
  uint32_t c8[J][4], c16[J][8];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int g = tm + j * kFoldModThreads;
    const int col = 16 * g;
    wid[j] = g < G ? min(16, Mp - col) : 0;
    // first row whose unit reaches past byte `lo`
    const int need = lo - col - wid[j] + 1;
    const int l = need > 0 ? (need + Mp - 1) / Mp : 0;
    pos[j] = l * Mp + col;
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
    const uint8_t* buf = smem + st * kStageBytes;
    const int len = min(kFoldTile, hi - s);
    const int e = s + len;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (wid[j] == 0) continue;
      int p = pos[j];
      while (p < e) {
        const int o = p - s;
        uint32_t w0, w1, w2, w3;
        if (o >= 0 && o + 16 <= len && wid[j] == 16) load16(buf, o, w0, w1, w2, w3);
        else load_masked(buf, o, len, wid[j], w0, w1, w2, w3);
        c8[j][0] += w0 & 0x02020202u;
        c8[j][1] += w1 & 0x02020202u;
        c8[j][2] += w2 & 0x02020202u;
        c8[j][3] += w3 & 0x02020202u;
        if (p + wid[j] > e) break;   // unit continues in the next stage
        p += Mp;
      }
      pos[j] = p;
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
    if (wid[j] == 0) continue;
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
    const int col = 16 * (tm + j * kFoldModThreads);
    if (wid[j] == 16) {
      int4* d4 = reinterpret_cast<int4*>(dst + col);
      d4[0] = make_int4(cnt[0], cnt[1], cnt[2], cnt[3]);
      d4[1] = make_int4(cnt[4], cnt[5], cnt[6], cnt[7]);
      d4[2] = make_int4(cnt[8], cnt[9], cnt[10], cnt[11]);
      d4[3] = make_int4(cnt[12], cnt[13], cnt[14], cnt[15]);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (i < wid[j]) dst[col + i] = cnt[i];
    }
  }
  return true;
}

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
        const FoldQ Q = a.q[qi];
        if (Q.goff >= ce) break;
        if (Q.nbytes == 0) continue;
        const int64_t lo = max(cb, Q.goff) - Q.goff;
        const int64_t hi = min(ce, Q.goff + Q.nbytes) - Q.goff;
        for (int64_t s = lo; s < hi; s += kFoldTile) {
          const uint32_t st = it % kFoldStages;
          if (it >= kFoldStages && !mbar_wait(&empty[st], ((it / kFoldStages) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          const uint32_t len = uint32_t(hi - s < kFoldTile ? hi - s : int64_t(kFoldTile));
          mbar_arrive_expect_tx(&full[st], len);
          bulk_load(smem + st * kStageBytes, Q.x + s, len, &full[st], pol);
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
  const int m = tid >> 8;           // modulus handled by this thread
  const int tm = tid & (kFoldModThreads - 1);
  uint32_t it = 0;
  bool ok = true;
  for (int qi = q0; qi < a.nq && ok; ++qi) {
    const FoldQ& Q = a.q[qi];
    if (Q.goff >= ce) break;
    if (Q.nbytes == 0) continue;
    const int lo = int(max(cb, Q.goff) - Q.goff);
    const int hi = int(min(ce, Q.goff + Q.nbytes) - Q.goff);
    const int G = (Q.Mp[m] + 15) >> 4;
    int32_t* dst = a.partial + Q.part + int64_t(blockIdx.x - Q.first_cta) * Q.stride + Q.moff[m];
    switch ((G + kFoldModThreads - 1) / kFoldModThreads) {
      case 1: ok = consume_share<1>(smem, full, empty, lo, hi, Q.Mp[m], tm, dst, it); break;
      case 2: ok = consume_share<2>(smem, full, empty, lo, hi, Q.Mp[m], tm, dst, it); break;
      case 3: ok = consume_share<3>(smem, full, empty, lo, hi, Q.Mp[m], tm, dst, it); break;
      case 4: ok = consume_share<4>(smem, full, empty, lo, hi, Q.Mp[m], tm, dst, it); break;
      default: ok = consume_share<kFoldJMax>(smem, full, empty, lo, hi, Q.Mp[m], tm, dst, it); break;
    }
  }
  if (!ok) atomicOr(a.err, 1);
}

}  // namespace

cudaError_t fold_configure() {
  const int smem = kFoldStages * kStageBytes + 2 * kFoldStages * 8;
  return cudaFuncSetAttribute(fold_i8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_fold_i8(const FoldArgs& a, cudaStream_t s) {
  const int smem = kFoldStages * kStageBytes + 2 * kFoldStages * 8;
  fold_i8_kernel<<<a.nctas, kFoldThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ftm
