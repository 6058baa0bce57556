// Step 3 of Algorithm 1 (Eq. (2)): column sums of x viewed as rows of
// length M, for both moduli, from a single read of x.
//
// Design: the signals of one storage type in a batch are concatenated
// (16-byte-aligned prefixes) into one byte space that is split into equal
// contiguous shares, one per CTA. A producer warp streams a CTA's share
// through a ring of shared-memory stages with bulk asynchronous copies (TMA,
// cp.async.bulk, L2 evict-first). Consumer lanes own fixed units of E
// consecutive columns of one modulus, dealt out in chunks of 32 consecutive
// units per warp (8 warps for M1, 9 for M2, so that K and K+1 columns both
// come to one chunk per warp for the paper's moduli). For a stage holding
// elements [s, e) of a signal every lane of a warp walks the same rows l of
// its modulus. Int8, fp16 and fp32 units read whole rows through row walkers
// that keep each unit's next row offset from stage to stage; a row cut by a
// stage edge is read in two parts, the bytes past either edge being slack
// that holds a neutral value (+1 for int8, which adds to no count; +0.0 for
// reals). Bit-packed units take a fast path for rows strictly inside the
// stage and a masked path for the first and last row. Stages carry 16
// bytes of slack on both sides so every read stays in bounds. A unit
// narrower than E (the last one of a row) still reads E columns; the
// columns past its width see the next row and are never written out. Each
// CTA writes one slot of per-column results per signal share; the
// correlation kernel adds the slots, the wrap-around term and the
// extension k >= M.
//
// Units (one per storage type):
//  int8 +-1 : 16 bytes; whole words added (raw sums, carries included)
//             and decoded into per-column counts every few stages (see
//             UnitI8), widened into 16-bit lanes; output: count of -1
//             entries.
//  bits     : 32 columns in one word (LSB first, 1 = +1); bit-sliced
//             vertical counters (5 planes, up to 31 rows) flushed into byte
//             then 16-bit lanes; output: count of +1 entries.
//  fp16/fp32: 8 / 4 columns, fp32 accumulators added row by row in a fixed
//             order (the result does not depend on timing); output: sums.
//
// To keep every lane busy the fold runs with an effective modulus
// Mp = R*M >= fold_geom(dtype).min_mp; the correlation kernel sums the R
// columns k + rM of the Mp-fold into column k of the M-fold.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "tm_internal.h"

namespace ftm {
namespace {

constexpr int kSlack = 32;   // 16 bytes of slack before and after each stage's data

// Position in the ring of stages: stage index and the parity of its
// current phase, advanced without divisions.
struct RingPos {
  uint32_t st = 0, ph = 0, used = 0;   // used: stages filled so far (saturates at the ring size)
  __device__ __forceinline__ void advance(int stages) {
    if (++st == uint32_t(stages)) {
      st = 0;
      ph ^= 1u;
    }
    if (used < uint32_t(stages)) ++used;
  }
};

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

// Bytes [o, o+16) of a stage whose phase o & 15 == P is known at compile
// time (o - P is 16-byte aligned).
template <int P>
__device__ __forceinline__ void load16p(const uint8_t* buf, int o, uint32_t (&w)[4]) {
  const uint4* p = reinterpret_cast<const uint4*>(buf + (o - P));
  const uint4 a = p[0];
  if constexpr (P == 0) {
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  } else {
    const uint4 b = p[1];
    const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    constexpr int q = P >> 2;
    constexpr uint32_t sh = uint32_t(P & 3) * 8u;
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = sh == 0 ? v[q + k] : fsr(v[q + k], v[q + k + 1], sh);
  }
}

// The two aligned 16-byte words around byte o of a stage (-16 < o < valid
// + 16), and the 16 bytes [o, o+16) extracted from them (r = o & 15 warp-
// uniform). Split so that a batch of rows issues all its loads first.
__device__ __forceinline__ void load32raw(const uint8_t* buf, int o, uint4& a, uint4& b) {
  const uint4* p = reinterpret_cast<const uint4*>(buf + (o & ~15));
  a = p[0];
  b = p[1];
}
__device__ __forceinline__ void extract16(const uint4& a, const uint4& b, int o, uint32_t (&w)[4]) {
  const int r = o & 15;
  const uint32_t sh = uint32_t(r & 3) * 8u;
  switch (r >> 2) {
    case 0: w[0] = fsr(a.x, a.y, sh); w[1] = fsr(a.y, a.z, sh); w[2] = fsr(a.z, a.w, sh); w[3] = fsr(a.w, b.x, sh); break;
    case 1: w[0] = fsr(a.y, a.z, sh); w[1] = fsr(a.z, a.w, sh); w[2] = fsr(a.w, b.x, sh); w[3] = fsr(b.x, b.y, sh); break;
    case 2: w[0] = fsr(a.z, a.w, sh); w[1] = fsr(a.w, b.x, sh); w[2] = fsr(b.x, b.y, sh); w[3] = fsr(b.y, b.z, sh); break;
    default: w[0] = fsr(a.w, b.x, sh); w[1] = fsr(b.x, b.y, sh); w[2] = fsr(b.y, b.z, sh); w[3] = fsr(b.z, b.w, sh); break;
  }
}

// ---------------------------------------------------------------- int8 +-1
// An entry is 0x01 (+1) or 0xFF (-1), i.e. 1 + 254 [entry = -1]. Whole
// 32-bit words are added, carries between byte lanes included, so after R
// row reads a lane word holds
//   S = R * 0x01010101 + 254 * C  (mod 2^32),   C = sum_b n_b 256^b,
// n_b the number of -1 entries in byte lane b. While R <= 127 each n_b
// fits 7 bits, C < 2^31, and C = ((S - R * 0x01010101) >> 1) * 127^-1
// (mod 2^31) gives the four counts back exactly. Bytes just outside a
// stage read as 0x01 (the stage slack holds that value), which adds to R
// but not to the counts: a row cut by a stage boundary is read in two
// parts, one per stage, with no mask.
struct UnitI8 {
  static constexpr int kE = 16, kBits = 8;
  static constexpr bool kWalk = true;
  static constexpr uint32_t kInv127 = 0x6FDFBF7Fu;   // 127 * kInv127 = 1 (mod 2^31)
  uint32_t s[4];      // raw word sums since the last widening
  uint32_t c16[8];    // counts in 16-bit lanes: word 2i columns 4i, 4i+2; word 2i+1 columns 4i+1, 4i+3
  uint32_t rows;      // row reads since the last widening
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < 4; ++i) s[i] = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) c16[i] = 0u;
    rows = 0u;
  }
  // stages between widenings: a unit reads at most tile/Mp + 2 rows per stage
  static __device__ __forceinline__ int widen_every(int Mp, int tile) { return max(1, 127 / (tile / Mp + 2)); }
  template <int P>
  __device__ __forceinline__ void addp(const uint8_t* buf, int o) {
    uint32_t w[4];
    load16p<P>(buf, o, w);
#pragma unroll
    for (int i = 0; i < 4; ++i) s[i] += w[i];
    ++rows;
  }
  __device__ __forceinline__ void add(const uint8_t* buf, int o) {
    uint32_t w[4];
    load16(buf, o, w);
#pragma unroll
    for (int i = 0; i < 4; ++i) s[i] += w[i];
    ++rows;
  }
  // two rows at 16-byte aligned offsets
  __device__ __forceinline__ void add2_aligned(const uint8_t* buf, int o, int o2) {
    const uint4 a = *reinterpret_cast<const uint4*>(buf + o);
    const uint4 b = *reinterpret_cast<const uint4*>(buf + o2);
    s[0] += a.x + b.x;
    s[1] += a.y + b.y;
    s[2] += a.z + b.z;
    s[3] += a.w + b.w;
    rows += 2u;
  }
  __device__ __forceinline__ void add_words(const uint32_t (&w)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) s[i] += w[i];
    ++rows;
  }
  __device__ __forceinline__ void widen() {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t c = (((s[i] - rows * 0x01010101u) >> 1) * kInv127) & 0x7FFFFFFFu;
      c16[2 * i] += c & 0x00FF00FFu;
      c16[2 * i + 1] += (c >> 8) & 0x00FF00FFu;
      s[i] = 0u;
    }
    rows = 0u;
  }
  __device__ __forceinline__ void write(int32_t* dst, int col, int width) {
    widen();
    int32_t cnt[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      cnt[4 * i + 0] = int32_t(c16[2 * i] & 0xFFFFu);
      cnt[4 * i + 2] = int32_t(c16[2 * i] >> 16);
      cnt[4 * i + 1] = int32_t(c16[2 * i + 1] & 0xFFFFu);
      cnt[4 * i + 3] = int32_t(c16[2 * i + 1] >> 16);
    }
    if (width == 16) {
      int4* d4 = reinterpret_cast<int4*>(dst + col);
      d4[0] = make_int4(cnt[0], cnt[1], cnt[2], cnt[3]);
      d4[1] = make_int4(cnt[4], cnt[5], cnt[6], cnt[7]);
      d4[2] = make_int4(cnt[8], cnt[9], cnt[10], cnt[11]);
      d4[3] = make_int4(cnt[12], cnt[13], cnt[14], cnt[15]);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (i < width) dst[col + i] = cnt[i];
    }
  }
};

// Row walkers for units that read past stage edges without masks: read
// the rows o, o + Mp, ... with o < el and return the first offset >= el.
// Offsets and Mp multiples of 16: aligned loads, two rows per step.
template <class U, int G>
__device__ __forceinline__ int walk_aligned(U& u, const uint8_t* buf, int o, int el, int Mp) {
  if constexpr (G == 4) {
    for (; o + 3 * Mp < el; o += 4 * Mp) {
      u.add2_aligned(buf, o, o + Mp);
      u.add2_aligned(buf, o + 2 * Mp, o + 3 * Mp);
    }
  }
  for (; o + Mp < el; o += 2 * Mp) u.add2_aligned(buf, o, o + Mp);
  if (o < el) {
    u.template addp<0>(buf, o);
    o += Mp;
  }
  return o;
}

// Four rows o + k Mp (k < 4) with Mp = 1 (mod 16), the first at phase P:
// all eight loads are issued before any sum, so the rows' shared-memory
// round trips overlap.
template <int P, class U>
__device__ __forceinline__ void add4_step1(U& u, const uint8_t* buf, int o, int Mp) {
  uint32_t w0[4], w1[4], w2[4], w3[4];
  load16p<P>(buf, o, w0);
  load16p<(P + 1) & 15>(buf, o + Mp, w1);
  load16p<(P + 2) & 15>(buf, o + 2 * Mp, w2);
  load16p<(P + 3) & 15>(buf, o + 3 * Mp, w3);
  u.add_words(w0);
  u.add_words(w1);
  u.add_words(w2);
  u.add_words(w3);
}

// Mp = 1 (mod 16), as for the modulus K+1 with K a multiple of 16: the
// phase o & 15 advances by one per row. Rows go four at a time (the phase
// of the group's first row taken at run time, the others following at
// compile time), the last ones through a cycle of 16 compile-time phases
// entered at the first remaining row's phase.
template <class U, int G>
__device__ __forceinline__ int walk_step1(U& u, const uint8_t* buf, int o, int el, int Mp) {
#define FTM_GROUP(P)                       \
  case P:                                  \
    add4_step1<P>(u, buf, o, Mp);          \
    break;
  if constexpr (G == 4) {
    for (; o + 3 * Mp < el; o += 4 * Mp) {
      switch (o & 15) {
        FTM_GROUP(0) FTM_GROUP(1) FTM_GROUP(2) FTM_GROUP(3) FTM_GROUP(4) FTM_GROUP(5) FTM_GROUP(6) FTM_GROUP(7)
        FTM_GROUP(8) FTM_GROUP(9) FTM_GROUP(10) FTM_GROUP(11) FTM_GROUP(12) FTM_GROUP(13) FTM_GROUP(14) FTM_GROUP(15)
      }
    }
  }
#undef FTM_GROUP
#define FTM_ROW(P)            \
  case P:                     \
    if (o >= el) return o;    \
    u.template addp<P>(buf, o); \
    o += Mp;
  switch (o & 15) {
    for (;;) {
      FTM_ROW(0) FTM_ROW(1) FTM_ROW(2) FTM_ROW(3) FTM_ROW(4) FTM_ROW(5) FTM_ROW(6) FTM_ROW(7)
      FTM_ROW(8) FTM_ROW(9) FTM_ROW(10) FTM_ROW(11) FTM_ROW(12) FTM_ROW(13) FTM_ROW(14) FTM_ROW(15)
    }
  }
#undef FTM_ROW
  return o;
}

// Any other Mp: the phase is taken at run time. Int8 rows go G at a time,
// their loads first; real units keep one row per step (batching them was
// measured slower: the fp32 fold of the uneven mix 3.98 -> 4.27 ms).
template <class U, int G>
__device__ __forceinline__ int walk_any(U& u, const uint8_t* buf, int o, int el, int Mp) {
  if constexpr (U::kBits > 8) {
    for (; o < el; o += Mp) u.add(buf, o);
    return o;
  }
  for (; o + (G - 1) * Mp < el; o += G * Mp) {
    uint4 a[G], b[G];
#pragma unroll
    for (int k = 0; k < G; ++k) load32raw(buf, o + k * Mp, a[k], b[k]);
#pragma unroll
    for (int k = 0; k < G; ++k) {
      uint32_t w[4];
      extract16(a[k], b[k], o + k * Mp, w);
      u.add_words(w);
    }
  }
  for (; o < el; o += Mp) u.add(buf, o);
  return o;
}

// ---------------------------------------------------------------- bit-packed +-1
// A unit is one 32-bit word of a row: 32 columns, bit i = column i, 1 = +1.
// Rows are added bit-sliced. A carry-save state (planes of weight 1, 2, 4)
// takes eight rows at a time through a tree of seven 3-input full adders
// (each a bitwise sum and majority); the tree's weight-8 output feeds a
// vertical counter (planes of weight 8 .. 256). Single rows (the masked
// first and last rows of a stage, leftovers) ripple through the same
// planes. Before the vertical counter can overflow (63 weight-8 steps) all
// planes are flushed into 16-bit lane counts. Output: count of +1 entries
// per column.
struct UnitBits {
  static constexpr int kE = 32, kBits = 1;
  static constexpr bool kWalk = false;
  static constexpr int kV = 6;            // vertical counter planes, weights 8 .. 256
  uint32_t ones, twos, fours;
  uint32_t v[kV];
  uint32_t c16[16];                       // 16-bit lanes: word k holds columns k (low) and k+16 (high)
  int steps;                              // weight-8 steps into v since the last flush
  __device__ __forceinline__ void clear() {
    ones = twos = fours = 0u;
#pragma unroll
    for (int i = 0; i < kV; ++i) v[i] = 0u;
#pragma unroll
    for (int i = 0; i < 16; ++i) c16[i] = 0u;
    steps = 0;
  }
  static __device__ __forceinline__ int widen_every(int, int) { return 1 << 30; }   // planes flush themselves
  // 32 bits starting at bit o of the stage (o > -32; the word before the
  // stage lies in the 16-byte slack); o & 31 is warp-uniform
  static __device__ __forceinline__ uint32_t load32(const uint8_t* buf, int o) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(buf);
    const int q = o >> 5;
    return fsr(w[q], w[q + 1], uint32_t(o & 31));
  }
  // full adder on bit planes: a + b + c = l + 2 h
  static __device__ __forceinline__ void csa(uint32_t& h, uint32_t& l, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
  }
  // all planes into the 16-bit lanes, weight by weight
  __device__ __forceinline__ void flush() {
    const uint32_t pl[3 + kV] = {ones, twos, fours, v[0], v[1], v[2], v[3], v[4], v[5]};
#pragma unroll
    for (int b = 0; b < 3 + kV; ++b) {
#pragma unroll
      for (int k = 0; k < 16; ++k) c16[k] += ((pl[b] >> k) & 0x00010001u) << b;
    }
    ones = twos = fours = 0u;
#pragma unroll
    for (int i = 0; i < kV; ++i) v[i] = 0u;
    steps = 0;
  }
  // one weight-8 step: e (0/1 per column) into the vertical counter
  __device__ __forceinline__ void step8(uint32_t e) {
#pragma unroll
    for (int b = 0; b < kV; ++b) {
      const uint32_t c = v[b] & e;
      v[b] ^= e;
      e = c;
    }
    if (++steps == 63) flush();
  }
  // one row (0/1 per column, weight 1)
  __device__ __forceinline__ void add1(uint32_t w) {
    const uint32_t c1 = ones & w;
    ones ^= w;
    const uint32_t c2 = twos & c1;
    twos ^= c1;
    const uint32_t c4 = fours & c2;
    fours ^= c2;
    step8(c4);
  }
  __device__ __forceinline__ void add(const uint8_t* buf, int o) { add1(load32(buf, o)); }
  __device__ __forceinline__ void add2(const uint8_t* buf, int o, int o2) {
    const uint32_t a = load32(buf, o), b = load32(buf, o2);
    add1(a);
    add1(b);
  }
  // eight rows o + i Mp, i < 8, all inside the stage: loads first, then the
  // adder tree
  __device__ __forceinline__ void add8(const uint8_t* buf, int o, int Mp) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = load32(buf, o + i * Mp);
    uint32_t twosA, twosB, foursA, foursB, e;
    csa(twosA, ones, ones, w[0], w[1]);
    csa(twosB, ones, ones, w[2], w[3]);
    csa(foursA, twos, twos, twosA, twosB);
    csa(twosA, ones, ones, w[4], w[5]);
    csa(twosB, ones, ones, w[6], w[7]);
    csa(foursB, twos, twos, twosA, twosB);
    csa(e, fours, fours, foursA, foursB);
    step8(e);
  }
  __device__ __forceinline__ void add_masked(const uint8_t* buf, int o, int len) {
    uint32_t w = load32(buf, o);
    // keep bits i with 0 <= o + i < len
    if (o < 0) w &= 0xFFFFFFFFu << (-o);
    if (len - o < 32) w &= (len - o) <= 0 ? 0u : (0xFFFFFFFFu >> (32 - (len - o)));
    add1(w);
  }
  __device__ __forceinline__ void widen() {}
  __device__ __forceinline__ void write(int32_t* dst, int col, int width) {
    flush();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k < width) dst[col + k] = int32_t(c16[k] & 0xFFFFu);
      if (k + 16 < width) dst[col + k + 16] = int32_t(c16[k] >> 16);
    }
  }
};

// ---------------------------------------------------------------- fp32
struct UnitF32 {
  static constexpr int kE = 4, kBits = 32;
  static constexpr bool kWalk = true;   // stage slack reads as +0.0f
  float acc[4];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = 0.f;
  }
  static __device__ __forceinline__ int widen_every(int, int) { return 1 << 30; }
  // 16 bytes at byte offset ob (a multiple of 4): whole words, no shifts
  __device__ __forceinline__ void add(const uint8_t* buf, int ob) {
    const uint4* p = reinterpret_cast<const uint4*>(buf + (ob & ~15));
    const uint4 a = p[0];
    uint32_t w[4];
    switch ((ob >> 2) & 3) {
      case 0: w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; break;
      case 1: { const uint4 b = p[1]; w[0] = a.y; w[1] = a.z; w[2] = a.w; w[3] = b.x; break; }
      case 2: { const uint4 b = p[1]; w[0] = a.z; w[1] = a.w; w[2] = b.x; w[3] = b.y; break; }
      default: { const uint4 b = p[1]; w[0] = a.w; w[1] = b.x; w[2] = b.y; w[3] = b.z; break; }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] += __uint_as_float(w[i]);
  }
  template <int P>
  __device__ __forceinline__ void addp(const uint8_t* buf, int ob) { add(buf, ob); }
  __device__ __forceinline__ void add_words(const uint32_t (&w)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] += __uint_as_float(w[i]);
  }
  __device__ __forceinline__ void add2_aligned(const uint8_t* buf, int o, int o2) {
    const float4 a = *reinterpret_cast<const float4*>(buf + o);
    const float4 b = *reinterpret_cast<const float4*>(buf + o2);
    acc[0] += a.x; acc[1] += a.y; acc[2] += a.z; acc[3] += a.w;
    acc[0] += b.x; acc[1] += b.y; acc[2] += b.z; acc[3] += b.w;
  }
  __device__ __forceinline__ void widen() {}
  __device__ __forceinline__ void write(int32_t* dst, int col, int width) {
    float* d = reinterpret_cast<float*>(dst) + col;
    if (width == 4) *reinterpret_cast<float4*>(d) = make_float4(acc[0], acc[1], acc[2], acc[3]);
    else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i < width) d[i] = acc[i];
    }
  }
};

// ---------------------------------------------------------------- fp16
struct UnitF16 {
  static constexpr int kE = 8, kBits = 16;
  static constexpr bool kWalk = true;   // stage slack reads as +0.0
  float acc[8];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.f;
  }
  static __device__ __forceinline__ int widen_every(int, int) { return 1 << 30; }
  __device__ __forceinline__ void add_words(const uint32_t (&w)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
      acc[2 * i] += f.x;
      acc[2 * i + 1] += f.y;
    }
  }
  // 16 bytes at byte offset ob (a multiple of 2)
  __device__ __forceinline__ void add(const uint8_t* buf, int ob) {
    uint32_t w[4];
    load16(buf, ob, w);
    add_words(w);
  }
  template <int P>
  __device__ __forceinline__ void addp(const uint8_t* buf, int ob) { add(buf, ob); }
  __device__ __forceinline__ void add2_aligned(const uint8_t* buf, int o, int o2) {
    const uint4 a = *reinterpret_cast<const uint4*>(buf + o);
    const uint4 b = *reinterpret_cast<const uint4*>(buf + o2);
    const uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wb[4] = {b.x, b.y, b.z, b.w};
    add_words(wa);
    add_words(wb);
  }
  __device__ __forceinline__ void widen() {}
  __device__ __forceinline__ void write(int32_t* dst, int col, int width) {
    float* d = reinterpret_cast<float*>(dst) + col;
    if (width == 8) {
      reinterpret_cast<float4*>(d)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      reinterpret_cast<float4*>(d)[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < width) d[i] = acc[i];
    }
  }
};

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
// the effective modulus Mp (in elements): units lane + 32 (wig + W j), j < J,
// where wig is the warp's index among the W warps of its modulus. Returns
// false when a bounded wait ran out.
template <class U, int J>
__device__ __forceinline__ bool consume_share(const uint8_t* smem, uint64_t* full, uint64_t* empty, int tile,
                                              int stages, int lo, int hi, int Mp, int ph, int W, int wig,
                                              int32_t* dst, RingPos& rp) {
  const int lane = threadIdx.x & 31;
  const int F = U::widen_every(Mp, tile);
  // unit j of this lane starts at column col(j); it exists when col(j) < Mp
  auto col = [&](int j) { return U::kE * (lane + 32 * (wig + W * j)); };
  U u[J];
#pragma unroll
  for (int j = 0; j < J; ++j) u[j].clear();

  int since = 0;
  for (int s = lo; s < hi; s += tile) {
    const uint32_t st = rp.st;
    // every lane waits; the warp gives up together so no lane is left
    // behind at the __syncwarp below
    if (!__all_sync(0xffffffffu, mbar_wait(&full[st], rp.ph))) return false;
    const uint8_t* buf = smem + st * (tile + kSlack) + 16;
    const int len = min(tile, hi - s);
    // the stage in elements: [es, es + el)
    const int es = int((int64_t(s) * 8) / U::kBits) + ph;   // the stage's first element, row phase included
    const int el = int((int64_t(len) * 8) / U::kBits);
    const int l0 = es / Mp;               // rows meeting the stage
    const int l1 = (es + el - 1) / Mp;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int cj = col(j);
      if (cj >= Mp) continue;
      // first row: the unit may start before the stage (or end after it)
      {
        const int o = l0 * Mp + cj - es;
        if (o > -U::kE && o < el) u[j].add_masked(buf, o, el);
      }
      if (l1 > l0) {
        // rows strictly inside the stage: all E columns are present (a
        // narrow last unit reads past its width into the next row or the
        // slack, in columns that are never written)
        int l = l0 + 1;
        if constexpr (U::kBits == 1) {
          for (; l + 7 < l1; l += 8) u[j].add8(buf, l * Mp + cj - es, Mp);
        }
        for (; l + 1 < l1; l += 2) {
          const int o = l * Mp + cj - es;
          u[j].add2(buf, o, o + Mp);
        }
        if (l < l1) u[j].add(buf, l * Mp + cj - es);
        // last row: the unit may run past the stage
        const int o = l1 * Mp + cj - es;
        if (o < el) u[j].add_masked(buf, o, el);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    rp.advance(stages);
    if (++since == F) {
      since = 0;
#pragma unroll
      for (int j = 0; j < J; ++j) u[j].widen();
    }
  }
#pragma unroll
  for (int j = 0; j < J; ++j)
    if (col(j) < Mp) u[j].write(dst, col(j), min(U::kE, Mp - col(j)));
  return true;
}

// The same for units read through the row walkers (kWalk): each unit keeps
// the offset of its next row relative to the next stage, so no row index
// is recomputed per stage and no read is masked.
// The same for units read through the row walkers (kWalk): each unit keeps
// the byte offset of its next row relative to the next stage, so no row
// index is recomputed per stage and no read is masked. Rows are Mb = Mp *
// bytes-per-element bytes long; a unit covers 16 bytes of a row.
template <class U, int J>
__device__ __forceinline__ bool consume_share_walk(const uint8_t* smem, uint64_t* full, uint64_t* empty, int tile,
                                                   int stages, int lo, int hi, int Mp, int ph, int W, int wig,
                                                   int32_t* dst, RingPos& rp) {
  constexpr int kEB = U::kBits / 8;   // bytes per element
  const int lane = threadIdx.x & 31;
  const int F = U::widen_every(Mp, tile);
  const int Mb = Mp * kEB;
  auto colb = [&](int j) { return 16 * (lane + 32 * (wig + W * j)); };   // unit j's first byte in a row
  U u[J];
  int o[J];   // next row of unit j, relative to the current stage (bytes)
  const int g = lo + ph * kEB;        // the share's first byte, counted from the row phase
  const int l = g / Mb;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    u[j].clear();
    o[j] = l * Mb + colb(j) - g;
    if (o[j] <= -16) o[j] += Mb;
  }
  const int step = Mb & 15;
  int since = 0;
  for (int s = lo; s < hi; s += tile) {
    const uint32_t st = rp.st;
    if (!__all_sync(0xffffffffu, mbar_wait(&full[st], rp.ph))) return false;
    const uint8_t* buf = smem + st * (tile + kSlack) + 16;
    const int el = min(tile, hi - s);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (colb(j) >= Mb) continue;
      int e;
      // rows in groups of G (loads first): four for one unit per lane, two
      // for more (register pressure)
      constexpr int G = J == 1 ? 4 : 2;
      if (step == 0) e = walk_aligned<U, G>(u[j], buf, o[j], el, Mb);
      else if constexpr (kEB == 1) e = step == 1 ? walk_step1<U, G>(u[j], buf, o[j], el, Mb) : walk_any<U, G>(u[j], buf, o[j], el, Mb);
      else e = walk_any<U, G>(u[j], buf, o[j], el, Mb);
      // a last row that started within 16 bytes of the end continues in
      // the next stage (its first bytes there fall at negative offsets)
      o[j] = e - Mb > el - 16 ? e - Mb - el : e - el;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    rp.advance(stages);
    if (++since == F) {
      since = 0;
#pragma unroll
      for (int j = 0; j < J; ++j) u[j].widen();
    }
  }
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int col = colb(j) / kEB;
    if (col < Mp) u[j].write(dst, col, min(U::kE, Mp - col));
  }
  return true;
}

template <class U, int JMAX>
__global__ void __launch_bounds__(kFoldThreads, 1) fold_kernel(const FoldArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int tile = a.tile, stages = kFoldRingBytes / a.tile;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kFoldRingBytes + kFoldMaxStages * kSlack);
  uint64_t* empty = full + kFoldMaxStages;

  const int tid = threadIdx.x;
  const int64_t cb = fold_share_begin(a, blockIdx.x);
  const int64_t ce = fold_share_begin(a, blockIdx.x + 1);
  // a correlation launched as a dependent may start its template work now
  // (it waits for this grid before reading the partial sums)
  pdl_release();

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kFoldConsumers / 32);
    }
    mbar_init_fence();
  }
  // The 16 bytes before and after each stage's data hold a neutral value
  // (walker units read across stage edges): +1 entries of an int8 signal,
  // which add to no count; zero bytes, +0.0 for real signals. Bulk copies
  // never write there.
  const uint32_t neutral = a.dtype == TM_I8_PM1 ? 0x01010101u : 0u;   // +1 entries / +0.0 / no bits set
  if (tid < 8 * stages) {
    const int st = tid >> 3, k = tid & 7;
    uint32_t* w = reinterpret_cast<uint32_t*>(smem + st * (tile + kSlack) + (k < 4 ? 0 : 16 + tile));
    w[k & 3] = neutral;
  }
  __syncthreads();
  if (cb >= ce) return;
  const int q0 = a.has_q0 ? a.q0[blockIdx.x] : first_query(a.q, a.nq, cb);

  // ---------------------------------------------------------------- producer
  if (tid >= kFoldConsumers) {
    if (tid == kFoldConsumers) {
      const uint64_t pol = l2_policy_evict_first();
      RingPos rp;
      uint32_t fills = 0;
      bool ok = true;
      for (int qi = q0; qi < a.nq && ok; ++qi) {
        const int64_t goff = a.q[qi].goff;
        const int32_t nbytes = a.q[qi].nbytes;
        const uint8_t* x = a.q[qi].x;
        if (goff >= ce) break;
        if (nbytes == 0) continue;
        const int64_t lo = max(cb, goff) - goff;
        const int64_t hi = min(ce, goff + nbytes) - goff;
        for (int64_t s = lo; s < hi; s += tile) {
          const uint32_t st = rp.st;
          // a stage filled before is free again once its consumers arrived
          if (rp.used == uint32_t(stages) && !mbar_wait(&empty[st], rp.ph ^ 1u)) {
            ok = false;
            break;
          }
          const uint32_t len = uint32_t(hi - s < tile ? hi - s : int64_t(tile));
          if (len < uint32_t(tile)) {
            // a short stage: the 16 bytes after its data read as +1 too; a
            // later bulk copy into this stage overwrites them, so order the
            // store before the async proxy's writes
            *reinterpret_cast<uint4*>(smem + st * (tile + kSlack) + 16 + len) =
                make_uint4(neutral, neutral, neutral, neutral);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          }
          mbar_arrive_expect_tx(&full[st], len);
          bulk_load(smem + st * (tile + kSlack) + 16, x + s, len, &full[st], pol);
          rp.advance(stages);
          ++fills;
        }
      }
      if (!ok) atomicOr(a.err, 1);
      // Let every copy this thread issued land before the CTA may exit.
      for (uint32_t k = fills > uint32_t(stages) ? fills - stages : 0; k < fills; ++k)
        (void)mbar_wait(&full[k % stages], (k / stages) & 1u);
    }
    return;
  }

  // ---------------------------------------------------------------- consumers
  const int warp = tid >> 5;
  RingPos rp;
  bool ok = true;
  for (int qi = q0; qi < a.nq && ok; ++qi) {
    const int64_t goff = a.q[qi].goff;
    const int32_t nbytes = a.q[qi].nbytes;
    if (goff >= ce) break;
    if (nbytes == 0) continue;
    // the modulus this warp folds for this signal (warps split 8/9 between
    // two moduli, 6/6/5 between three)
    const int nm = a.q[qi].nmod;
    const int m = nm == 3 ? (warp < 6 ? 0 : warp < 12 ? 1 : 2) : (warp < kFoldWarps0 ? 0 : 1);
    const int W = fold_warp_count(nm, m);
    const int wig = warp - fold_warp_first(nm, m);
    const int lo = int(max(cb, goff) - goff);
    const int hi = int(min(ce, goff + nbytes) - goff);
    const int Mp = a.q[qi].Mp[m];
    // rows are counted from element e0 of the signal (0 unless x is a slice)
    const int ph = int(a.q[qi].e0 % Mp);
    const int J = fold_units_per_lane(Mp, W, U::kE);
    if constexpr (U::kWalk) {
      // one slot per CTA share, or (piece > 0) one per fixed piece of the
      // signal, the share then holding whole pieces
      const int64_t piece = a.q[qi].piece;
      const int64_t step = piece > 0 ? piece : int64_t(hi - lo);
      for (int64_t plo = lo; plo < hi && ok; plo += step) {
        const int phi = int(min(int64_t(hi), plo + step));
        const int64_t slot = piece > 0 ? plo / piece : int64_t(blockIdx.x - a.q[qi].first_cta);
        int32_t* dst = a.partial + a.q[qi].part + slot * a.q[qi].stride + a.q[qi].moff[m];
        const int pl = int(plo);
        if (J <= 1) ok = consume_share_walk<U, 1>(smem, full, empty, tile, stages, pl, phi, Mp, ph, W, wig, dst, rp);
        else if (J == 2 || JMAX == 2) ok = consume_share_walk<U, 2>(smem, full, empty, tile, stages, pl, phi, Mp, ph, W, wig, dst, rp);
        else if (J <= 3 || JMAX <= 3) ok = consume_share_walk<U, (JMAX < 3 ? JMAX : 3)>(smem, full, empty, tile, stages, pl, phi, Mp, ph, W, wig, dst, rp);
        else ok = consume_share_walk<U, JMAX>(smem, full, empty, tile, stages, pl, phi, Mp, ph, W, wig, dst, rp);
      }
    } else {
      int32_t* dst = a.partial + a.q[qi].part + int64_t(blockIdx.x - a.q[qi].first_cta) * a.q[qi].stride +
                     a.q[qi].moff[m];
      if (J <= 1) ok = consume_share<U, 1>(smem, full, empty, tile, stages, lo, hi, Mp, ph, W, wig, dst, rp);
      else if (J == 2 || JMAX == 2) ok = consume_share<U, 2>(smem, full, empty, tile, stages, lo, hi, Mp, ph, W, wig, dst, rp);
      else if (J <= 4 || JMAX <= 4) ok = consume_share<U, (JMAX < 4 ? JMAX : 4)>(smem, full, empty, tile, stages, lo, hi, Mp, ph, W, wig, dst, rp);
      else ok = consume_share<U, JMAX>(smem, full, empty, tile, stages, lo, hi, Mp, ph, W, wig, dst, rp);
    }
  }
  if (!ok) atomicOr(a.err, 1);
}

constexpr int kFoldSmem = kFoldRingBytes + kFoldMaxStages * kSlack + 2 * kFoldMaxStages * 8;

template <class K>
cudaError_t set_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFoldSmem);
}

}  // namespace

cudaError_t fold_configure() {
  cudaError_t e;
  if ((e = set_smem(fold_kernel<UnitI8, 3>)) != cudaSuccess) return e;
  if ((e = set_smem(fold_kernel<UnitI8, 5>)) != cudaSuccess) return e;
  if ((e = set_smem(fold_kernel<UnitBits, 2>)) != cudaSuccess) return e;
  if ((e = set_smem(fold_kernel<UnitF16, 4>)) != cudaSuccess) return e;
  if ((e = set_smem(fold_kernel<UnitF16, 8>)) != cudaSuccess) return e;
  if ((e = set_smem(fold_kernel<UnitF32, 8>)) != cudaSuccess) return e;
  return set_smem(fold_kernel<UnitF32, 16>);
}

// Each storage type has a register-lean instantiation for the common moduli
// and a wider one (moduli up to fold_geom().jmax units per lane).
cudaError_t launch_fold(const FoldArgs& a, int jmax, cudaStream_t s) {
  if (a.tile != 16384 && a.tile != 32768 && a.tile != 65536) return cudaErrorInvalidValue;
  switch (a.dtype) {
    case TM_I8_PM1:
      if (jmax <= 3) fold_kernel<UnitI8, 3><<<a.nctas, kFoldThreads, kFoldSmem, s>>>(a);
      else fold_kernel<UnitI8, 5><<<a.nctas, kFoldThreads, kFoldSmem, s>>>(a);
      break;
    case TM_BITS_PM1: fold_kernel<UnitBits, 2><<<a.nctas, kFoldThreads, kFoldSmem, s>>>(a); break;
    case TM_F16:
      if (jmax <= 4) fold_kernel<UnitF16, 4><<<a.nctas, kFoldThreads, kFoldSmem, s>>>(a);
      else fold_kernel<UnitF16, 8><<<a.nctas, kFoldThreads, kFoldSmem, s>>>(a);
      break;
    default:
      if (jmax <= 8) fold_kernel<UnitF32, 8><<<a.nctas, kFoldThreads, kFoldSmem, s>>>(a);
      else fold_kernel<UnitF32, 16><<<a.nctas, kFoldThreads, kFoldSmem, s>>>(a);
      break;
  }
  return cudaGetLastError();
}

}  // namespace ftm
