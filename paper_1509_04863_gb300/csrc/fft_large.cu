// Steps 4-9 of Algorithm 1 for one query with a long FFT (P = 2^14 .. 2^26
// points), spread over all SMs as a sequence of launches.
//
// Transform. P is viewed as dims L_1 x .. x L_D x 8192 (outermost first,
// D = 1 or 2 strided dims of at most 512 points, the 8192-point rows
// contiguous). A decimation-in-frequency pass over dim d takes, for every
// inner index n' < S_d (the product of the inner dims) of every block of
// P_d = L_d S_d points, the L_d-point DFT along d and multiplies output k_d
// by W_{P_d}^{n' k_d}; the rows are 512 x 16 blocks done the same way inside
// one CTA. The spectrum ends in digit-reversed mixed-radix order, the same
// for the signal and the template, so the product conj(T) Z needs no
// reordering; the inverse runs the passes backwards in conjugated form
// (conj(IDFT(v)) L = DFT(conj(v)), the twiddle applied before each DFT).
//
// Both folds ride one complex signal z = y_1 + i y_2 (the inverse of
// conj(T) Z is r_1 + i r_2). Step 7 keeps every index whose FFT value is
// within 2 delta of the maximum (delta: the normwise rounding bound of the
// correlation) and rescores them exactly from the folds in fixed-size
// chunks; when more than kLargeCap indices qualify, every index is rescored
// if M K <= 2^36, else the FFT maximum is reported with
// TM_RF_UNCERTIFIED. Steps 8-9 use the closed-form intersection (crt.h) and
// the exact (Tx)_m of the members, again in chunks.
//
// Inside a CTA: 8192 points in shared memory (one entry of padding per 16),
// 512 threads, 16 points per thread, Stockham passes of radix 16 (one
// radix-2/4/8 pass first) with the butterfly's column index fastest across
// lanes, so that the strided layouts are conflict-free and a warp reads at
// most two distinct twiddles of the 8192-entry table per load. Twiddles
// between dims come from sincospif of exactly representable arguments
// (two factors above 2^24).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "crt.h"
#include "device_util.cuh"
#include "tm_internal.h"

namespace ftm {
namespace {

constexpr int kLT = 512;              // threads per transform CTA
constexpr int kLPts = 8192;           // points per transform CTA
constexpr int kLPPT = kLPts / kLT;    // points per thread
constexpr int kLW = kLT / 32;
constexpr int kLRowLog = 13;
constexpr int kSmemPts = kLPts + kLPts / 16;

__device__ float2 g_tw13[8192];       // W_8192^m = e^{-2 pi i m / 8192}

struct LHdr {
  unsigned long long z2i;   // sum of y^2 over both folds (integer folds)
  double z2f;               // the same for real folds
  double t1, t2sq;          // ||t||_1, ||t||_2^2
  unsigned long long rkey[2];   // max of r_j: order key of the value << 32 | (2^32-1 - index)
  int maxy, tbad;           // max |y| (integer folds); t not integral (or too large)
  unsigned int tc2, zc2;    // bits of max |T~_k|^2, max |Z~_k|^2
  int ncand[2];
  int mode[2];              // 0: list, 1: every index rescored, 2: uncertified
  int m[2];
  double rv[2];
  int flags;
  int nch;                  // chunks per listed candidate (set by the rescoring)
  int nchm;                 // chunks per listed member (set by the scoring)
  int nbest;                // CTAs per query of the rescoring and scoring launches
  CrtSet crt;
  long long ncs;
};

// Workspace layout (bytes from ws).
constexpr size_t kOffHdr = 0;
constexpr size_t kOffCand = 512;
constexpr size_t kOffPart = kOffCand + 2 * kLargeCap * sizeof(int);
constexpr size_t kOffBest = kOffPart + size_t(kLargePart) * 8;
constexpr size_t kOffMPart = kOffBest + size_t(2) * kLargeCtas * 16;
constexpr size_t kOffMBest = kOffMPart + size_t(kLargeMPart) * 8;
constexpr size_t kWsBytes = kOffMBest + size_t(kLargeCtas) * 16;
static_assert(sizeof(LHdr) <= kOffCand, "header");

struct Ws {
  LHdr* h;
  int* cand;          // [2][kLargeCap]
  long long* part;    // [listed candidate][nch] int64 or double bits (modulus 0's first)
  long long* best;    // [2][kLargeCtas] x (value bits, index)
  long long* mpart;   // [listed member][nchm]
  long long* mbest;   // [kLargeCtas] x (value bits, member)
};
__device__ __forceinline__ Ws ws_of(void* p) {
  char* b = static_cast<char*>(p);
  return Ws{reinterpret_cast<LHdr*>(b + kOffHdr), reinterpret_cast<int*>(b + kOffCand),
            reinterpret_cast<long long*>(b + kOffPart), reinterpret_cast<long long*>(b + kOffBest),
            reinterpret_cast<long long*>(b + kOffMPart), reinterpret_cast<long long*>(b + kOffMBest)};
}

// ---------------------------------------------------------------- complex helpers
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// cos and sin of 2 pi m / 16, m < 8.
__device__ __forceinline__ float cs16(int m) {
  constexpr float C[8] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                          0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f};
  return C[m];
}
__device__ __forceinline__ float sn16(int m) {
  constexpr float S[8] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                          1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f};
  return S[m];
}

template <int R>
__host__ __device__ constexpr int brev(int r) {
  int o = 0;
  for (int b = 1; b < R; b <<= 1) {
    o = (o << 1) | (r & 1);
    r >>= 1;
  }
  return o;
}
template <int R>
__host__ __device__ constexpr int lg(void) {
  return R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
}

// In-register forward DFT of size R by radix-2 decimation in frequency;
// output r lands at position brev(r).
template <int R>
__device__ __forceinline__ void dftr(float2 (&v)[R]) {
#pragma unroll
  for (int len = R; len >= 2; len >>= 1) {
    const int half = len >> 1;
#pragma unroll
    for (int s = 0; s < R; s += len) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const float2 a = v[s + k], b = v[s + k + half];
        v[s + k] = cadd(a, b);
        const float2 d = csub(a, b);
        const int m = k * (16 / len);
        if (m == 0) {
          v[s + k + half] = d;
        } else if (m == 4) {
          v[s + k + half] = make_float2(d.y, -d.x);
        } else {
          const float c = cs16(m), sn = sn16(m);
          v[s + k + half] = make_float2(d.x * c + d.y * sn, d.y * c - d.x * sn);
        }
      }
    }
  }
}

// W_{2^a}^e for 0 <= e < 2^a, a <= 26, from sincospif of exact arguments.
__device__ __forceinline__ float2 wsc(int a, int e) {
  float s, c;
  if (e < (1 << 24)) {
    sincospif(__int_as_float((128 - a) << 23) * float(e), &s, &c);   // 2 e / 2^a
    return make_float2(c, -s);
  }
  float s2, c2;
  sincospif(__int_as_float((140 - a) << 23) * float(e >> 12), &s, &c);      // 2 (e - e mod 4096) / 2^a
  sincospif(__int_as_float((128 - a) << 23) * float(e & 4095), &s2, &c2);
  return cmul(make_float2(c, -s), make_float2(c2, -s2));
}

// Twiddles along a thread's elements. A thread's elements of a tile share
// the column c and step down the rows by s = kLT / C, so their twiddles
// W^{(n0+c) i} form a geometric sequence in the element number u. TwSeq
// gives them in order: exact values (sincospif) at u = 0, 4, 8, 12 and up
// to three multiplications by the exact step W^{(n0+c) s} in between
// (about 10 ulp at most, inside the rounding bound's margin).
struct TwSeq {
  int a;
  uint32_t e0, d;
  float2 step, w;
  __device__ __forceinline__ TwSeq(int a_, uint32_t e0_, uint32_t d_) : a(a_), e0(e0_), d(d_) {
    step = wsc(a, d & ((1u << a) - 1));
  }
  __device__ __forceinline__ float2 at(int u) {   // called for u = 0, 1, 2, ... in order
    if ((u & 3) == 0) w = wsc(a, (e0 + uint32_t(u) * d) & ((1u << a) - 1));
    else w = cmul(w, step);
    return w;
  }
};

// One Stockham pass of radix R over NC = 2^logNC independent DFTs of
// length L = 2^logL (NC L = 8192) held in buf at pad(i NC + col): butterfly
// j of a column takes i = j + r L/R, twiddles by W_{Ns R}^{r (j mod Ns)} and
// writes to (j - j mod Ns) R + j mod Ns + r Ns. With NC L = 8192 the read
// index of leg r is bi + r 8192/R (bi = j NC + col, the butterfly number)
// and the write index W0 + r Ns NC, both multiples of 16 apart, so the
// padded addresses step by constants.
template <int R>
__device__ __forceinline__ void bpass(float2* buf, int logL, int logNs, int logNC) {
  constexpr int NB = kLPPT / R;
  constexpr int LR = lg<R>();
  constexpr int kRead = (kLPts / R) / 16 * 17;   // padded step between legs
  const int Ns = 1 << logNs;
  const int twsh = kLRowLog - logNs - LR;
  const int cmask = (1 << logNC) - 1;
  const int wstep = ((Ns << logNC) >> 4) * 17;    // padded step between outputs
  float2 v[NB][R];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int bi = threadIdx.x + b * kLT;
    const int k = (bi >> logNC) & (Ns - 1);
    const int a0 = pad(bi);
#pragma unroll
    for (int r = 0; r < R; ++r) v[b][r] = buf[a0 + r * kRead];
    if (Ns > 1) {
      const int tk = k << twsh;
#pragma unroll
      for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], __ldg(&g_tw13[r * tk]));
    }
    dftr<R>(v[b]);
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int bi = threadIdx.x + b * kLT;
    const int col = bi & cmask, jp = bi >> logNC;
    const int k = jp & (Ns - 1);
    const int w0 = pad((((jp - k) * R + k) << logNC) + col);
#pragma unroll
    for (int r = 0; r < R; ++r) buf[w0 + r * wstep] = v[b][brev<R>(r)];
  }
  __syncthreads();
}

// Forward DFTs of length 2^logL (natural order in and out) of 8192 >> logL
// columns at pad(i 2^logNC + col); caller synchronised before.
__device__ void bfft(float2* buf, int logL, int logNC) {
  const int first = logL & 3;
  if (first == 1) bpass<2>(buf, logL, 0, logNC);
  else if (first == 2) bpass<4>(buf, logL, 0, logNC);
  else if (first == 3) bpass<8>(buf, logL, 0, logNC);
  for (int logNs = first; logNs < logL; logNs += 4) bpass<16>(buf, logL, logNs, logNC);
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ unsigned fkey(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

template <class T, class Op>
__device__ __forceinline__ T warp_red(T v, Op op) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// Block reduction to thread 0 (valid there); red holds kLW entries.
template <class T, class Op>
__device__ __forceinline__ T block_red(T v, T* red, Op op) {
  v = warp_red(v, op);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < int(blockDim.x >> 5); ++w) v = op(v, red[w]);
  return v;
}
// Two block reductions with one pair of barriers (valid in thread 0).
template <class T1, class Op1, class T2, class Op2>
__device__ __forceinline__ void block_red2(T1& a, T1* ra, Op1 op1, T2& b, T2* rb, Op2 op2) {
  a = warp_red(a, op1);
  b = warp_red(b, op2);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { ra[threadIdx.x >> 5] = a; rb[threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < int(blockDim.x >> 5); ++w) { a = op1(a, ra[w]); b = op2(b, rb[w]); }
}
struct OpAdd {
  template <class T>
  __device__ T operator()(T a, T b) const { return a + b; }
};
struct OpMax {
  template <class T>
  __device__ T operator()(T a, T b) const { return a > b ? a : b; }
};

// (value, index) with the larger value, then the smaller index.
__device__ __forceinline__ void better(double& bv, long long& bi, double v, long long i) {
  if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}
__device__ __forceinline__ void block_best(double& bv, long long& bi, double* rv, long long* ri) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
    better(bv, bi, ov, oi);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = bv; ri[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < int(blockDim.x >> 5); ++w) better(bv, bi, rv[w], ri[w]);
}

__device__ __forceinline__ bool int_dtype(int dt) { return dt == TM_I8_PM1 || dt == TM_BITS_PM1; }

template <int DT>
__device__ __forceinline__ float sval(const void* x, int64_t n) {
  if constexpr (DT == TM_I8_PM1) return (__ldg(static_cast<const uint8_t*>(x) + n) & 2u) ? -1.0f : 1.0f;
  else if constexpr (DT == TM_BITS_PM1)
    return ((__ldg(static_cast<const uint8_t*>(x) + (n >> 3)) >> (n & 7)) & 1u) ? 1.0f : -1.0f;
  else if constexpr (DT == TM_F16) return __half2float(static_cast<const __half*>(x)[n]);
  else return __ldg(static_cast<const float*>(x) + n);
}

// The query of this block: a single query's descriptor is a kernel
// parameter (q1); in a batch (B) the descriptor of query blockIdx.z is
// copied to shared memory and every thread reads its fields there.
#define TM_LQ(q)                       \
  __shared__ LQ sq_;                   \
  if constexpr (B) load_lq(lqs, sq_);  \
  const LQ& q = B ? sq_ : q1;

__device__ __forceinline__ void load_lq(const LQ* __restrict__ lqs, LQ& sq) {
  static_assert(sizeof(LQ) % 4 == 0, "LQ words");
  const int* src = reinterpret_cast<const int*>(lqs + blockIdx.z);
  for (int i = threadIdx.x; i < int(sizeof(LQ) / 4); i += blockDim.x) reinterpret_cast<int*>(&sq)[i] = src[i];
  __syncthreads();
}

// ---------------------------------------------------------------- strided passes
// Tile of pass d: C = 8192 >> logL columns (inner indices n0 .. n0+C-1) of
// one block, all L rows; element e = i C + c at global block + i S + n0 + c.
struct Tile {
  int logL, logC, logS, logPd;
  int64_t base;   // global index of (i = 0, c = 0)
  int n0;
  int cmask;
};
__device__ __forceinline__ Tile tile_of(const LQ& q, int d) {
  Tile t;
  t.logL = d == 0 ? q.logL[0] : q.logL[1];
  t.logC = kLRowLog - t.logL;
  t.logS = kLRowLog + (d == 0 && q.nsd == 2 ? q.logL[1] : 0);
  t.logPd = t.logL + t.logS;
  const int tiles = 1 << (t.logS - t.logC);
  const int64_t blk = blockIdx.x >> (t.logS - t.logC);
  t.n0 = (blockIdx.x & (tiles - 1)) << t.logC;
  t.base = (blk << t.logPd) + t.n0;
  t.cmask = (1 << t.logC) - 1;
  return t;
}
// Offset of tile element e from t.base (below P_d <= 2^26: 32-bit).
__device__ __forceinline__ int tile_off(const Tile& t, int e) {
  return ((e >> t.logC) << t.logS) + (e & t.cmask);
}
__device__ __forceinline__ int64_t tile_gidx(const Tile& t, int e) { return t.base + tile_off(t, e); }

enum { kSrcBuf = 0, kSrcY = 1, kSrcT = 2 };

// Forward pass over strided dim d: source buffer, the folds (first pass of
// z) or the template (first pass of t); result to dst.
// src_b / dst_b: 0 for the signal buffer A, 1 for the template buffer B.
template <int SRC, bool B>
__global__ void __launch_bounds__(kLT, 2) lfwd_kernel(const LQ q1, const LQ* __restrict__ lqs, int d, int src_b,
                                                      int dst_b) {
  extern __shared__ __align__(16) float2 sm[];
  TM_LQ(q)
  if (blockIdx.x >= unsigned(q.P >> kLRowLog) || d >= q.nsd) return;
  const float2* src = src_b ? q.B : q.A;
  float2* dst = dst_b ? q.B : q.A;
  __shared__ float redf[kLW], redf2[kLW];
  __shared__ unsigned long long redu[kLW];
  __shared__ int redi[kLW];
  const Tile tl = tile_of(q, d);
  const Ws w = ws_of(q.ws);
  // loads of eight elements in flight before their first use
  if constexpr (SRC == kSrcY) {
    const bool ints = int_dtype(q.xdtype);
    const int32_t* yi = static_cast<const int32_t*>(q.y);
    const float* yf = static_cast<const float*>(q.y);
    unsigned long long s2 = 0;
    float f2 = 0.f;   // fp32 sums within the CTA (see below), then fp64
    int my = 0;
#pragma unroll
    for (int u0 = 0; u0 < kLPPT; u0 += 8) {
      float2 v[8];
      if (ints) {
        int a[8], b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int64_t n = tile_gidx(tl, threadIdx.x + (u0 + u) * kLT);
          a[u] = yi[n];
          b[u] = yi[int64_t(q.P) + n];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          s2 += (unsigned long long)((long long)a[u] * a[u] + (long long)b[u] * b[u]);
          my = max(my, max(abs(a[u]), abs(b[u])));
          v[u] = make_float2(float(a[u]), float(b[u]));
        }
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int64_t n = tile_gidx(tl, threadIdx.x + (u0 + u) * kLT);
          v[u] = make_float2(yf[n], yf[int64_t(q.P) + n]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) f2 = fmaf(v[u].x, v[u].x, fmaf(v[u].y, v[u].y, f2));
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) sm[pad(threadIdx.x + (u0 + u) * kLT)] = v[u];
    }
    if (ints) {
      block_red2(s2, redu, OpAdd(), my, redi, OpMax());
      if (threadIdx.x == 0) { atomicAdd(&w.h->z2i, s2); atomicMax(&w.h->maxy, my); }
    } else {
      // nonnegative terms, each through at most 32 + 5 + 15 fp32 additions
      // (thread, warp tree, warps in turn): relative error < 52 u < 4e-6,
      // so the scaled sum bounds the exact one from above; FP64 only in
      // thread 0 (this part has few FP64 units)
      f2 = block_red(f2, redf, OpAdd());
      if (threadIdx.x == 0) atomicAdd(&w.h->z2f, double(f2) * (1.0 + 4e-6));
    }
  } else if constexpr (SRC == kSrcT) {
    float a1 = 0.f, a2 = 0.f;   // fp32 within the CTA, fp64 across CTAs
    int bad = 0;
#pragma unroll
    for (int u0 = 0; u0 < kLPPT; u0 += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t n = tile_gidx(tl, threadIdx.x + (u0 + u) * kLT);
        v[u] = n < q.K ? __ldg(&q.t[n]) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        a1 += fabsf(v[u]);
        a2 = fmaf(v[u], v[u], a2);
        bad |= (v[u] == rintf(v[u]) && fabsf(v[u]) <= 1048576.f) ? 0 : 1;
        sm[pad(threadIdx.x + (u0 + u) * kLT)] = make_float2(v[u], 0.f);
      }
    }
    // nonnegative terms, each through at most 16 + 5 + 15 fp32 additions:
    // relative error < 36 u < 4e-6 (the scaled sums are upper bounds)
    bad = __syncthreads_or(bad);
    block_red2(a1, redf, OpAdd(), a2, redf2, OpAdd());
    if (threadIdx.x == 0) {
      atomicAdd(&w.h->t1, double(a1) * (1.0 + 4e-6));
      atomicAdd(&w.h->t2sq, double(a2) * (1.0 + 4e-6));
      if (bad) atomicOr(&w.h->tbad, 1);
    }
  } else {
    const float2* s0 = src + tl.base;
#pragma unroll 8
    for (int u = 0; u < kLPPT; ++u) {
      const int e = threadIdx.x + u * kLT;
      sm[pad(e)] = s0[tile_off(tl, e)];
    }
  }
  __syncthreads();
  bfft(sm, tl.logL, tl.logC);
  float2* d0 = dst + tl.base;
  if (tl.logC <= 9) {   // C <= kLT: the thread's elements share their column
    const int c = threadIdx.x & tl.cmask;
    const uint32_t nc = uint32_t(tl.n0 + c);
    TwSeq tw(tl.logPd, nc * uint32_t(threadIdx.x >> tl.logC), nc * uint32_t(kLT >> tl.logC));
#pragma unroll
    for (int u = 0; u < kLPPT; ++u) {
      const int e = threadIdx.x + u * kLT;
      d0[tile_off(tl, e)] = cmul(sm[pad(e)], tw.at(u));
    }
  } else {
    for (int u = 0; u < kLPPT; ++u) {
      const int e = threadIdx.x + u * kLT;
      const int i = e >> tl.logC, c = e & tl.cmask;
      d0[tile_off(tl, e)] = cmul(sm[pad(e)], wsc(tl.logPd, (tl.n0 + c) * i));
    }
  }
}

// Inverse pass over strided dim d in conjugated form (twiddle, then DFT).
// OUT: the outermost dim, results r_1 = Re/P (n < M1), r_2 = -Im/P (n < M2)
// and their maxima.
template <bool OUT, bool B>
__global__ void __launch_bounds__(kLT, 2) linv_kernel(const LQ q1, const LQ* __restrict__ lqs, int d) {
  extern __shared__ __align__(16) float2 sm[];
  TM_LQ(q)
  if (blockIdx.x >= unsigned(q.P >> kLRowLog) || d >= q.nsd) return;
  __shared__ unsigned long long redu[kLW], redu2[kLW];
  const Tile tl = tile_of(q, d);
  float2* a0 = q.A + tl.base;
  // loads of eight elements in flight before their twiddles
  static_assert(kLPPT % 8 == 0, "load batches");
  if (tl.logC <= 9) {   // C <= kLT: the thread's elements share their column
    const int c = threadIdx.x & tl.cmask;
    const uint32_t nc = uint32_t(tl.n0 + c);
    TwSeq tw(tl.logPd, nc * uint32_t(threadIdx.x >> tl.logC), nc * uint32_t(kLT >> tl.logC));
#pragma unroll
    for (int u0 = 0; u0 < kLPPT; u0 += 8) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = a0[tile_off(tl, threadIdx.x + (u0 + u) * kLT)];
#pragma unroll
      for (int u = 0; u < 8; ++u) sm[pad(threadIdx.x + (u0 + u) * kLT)] = cmul(v[u], tw.at(u0 + u));
    }
  } else {
    for (int u0 = 0; u0 < kLPPT; u0 += 8) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = a0[tile_off(tl, threadIdx.x + (u0 + u) * kLT)];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = threadIdx.x + (u0 + u) * kLT;
        const int i = e >> tl.logC, c = e & tl.cmask;
        sm[pad(e)] = cmul(v[u], wsc(tl.logPd, (tl.n0 + c) * i));
      }
    }
  }
  __syncthreads();
  bfft(sm, tl.logL, tl.logC);
  if constexpr (!OUT) {
    for (int u = 0; u < kLPPT; ++u) {
      const int e = threadIdx.x + u * kLT;
      a0[tile_off(tl, e)] = sm[pad(e)];
    }
  } else {
    const float invP = 1.0f / float(q.P);   // exact: P is a power of two
    unsigned long long k1 = 0, k2 = 0;
    for (int u = 0; u < kLPPT; ++u) {
      const int e = threadIdx.x + u * kLT;
      const int64_t n = tile_gidx(tl, e);
      const float2 g = sm[pad(e)];
      if (n < q.M[0]) {
        const float v = g.x * invP;
        q.r[n] = v;
        k1 = max(k1, (static_cast<unsigned long long>(fkey(v)) << 32) | (0xffffffffull - n));
      }
      if (n < q.M[1]) {
        const float v = -g.y * invP;
        q.r[int64_t(q.P) + n] = v;
        k2 = max(k2, (static_cast<unsigned long long>(fkey(v)) << 32) | (0xffffffffull - n));
      }
    }
    const Ws w = ws_of(q.ws);
    block_red2(k1, redu, OpMax(), k2, redu2, OpMax());
    if (threadIdx.x == 0 && k1) atomicMax(&w.h->rkey[0], k1);
    if (threadIdx.x == 0 && k2) atomicMax(&w.h->rkey[1], k2);
  }
}

// ---------------------------------------------------------------- row blocks
// 8192 contiguous points as 512 x 16 (n = i 16 + c): DFT over i (stride 16),
// twiddle W_8192^{c k_i}, DFT over c; output (k_i, k_c) at k_i 16 + k_c.
// TEMPLATE: forward only (spectrum of t, its maximum). Otherwise the signal
// block: forward, maximum of |Z~|, product with the template spectrum in
// conjugated form g = T~ conj(Z~), then the inverse of the row (DFT over c,
// twiddle, DFT over i).
template <bool TEMPLATE, bool B>
__global__ void __launch_bounds__(kLT, 2) lrow_kernel(const LQ q1, const LQ* __restrict__ lqs) {
  extern __shared__ __align__(16) float2 sm[];
  TM_LQ(q)
  if (blockIdx.x >= unsigned(q.P >> kLRowLog)) return;
  __shared__ float redf[kLW];
  const int64_t base = int64_t(blockIdx.x) << kLRowLog;
  float2* buf = TEMPLATE ? q.B : q.A;
  for (int u = 0; u < kLPPT; ++u) {
    const int e = threadIdx.x + u * kLT;
    sm[pad(e)] = buf[base + e];
  }
  __syncthreads();
  bfft(sm, 9, 4);
  float mx = 0.f;
  // each thread: rows k_i = tid + h kLT
#pragma unroll
  for (int h = 0; h < 512 / kLT; ++h) {
    const int ki = threadIdx.x + h * kLT;
    // W_8192^{c k_i}: the table's exact values at c = 4, 8, 12, steps by W^{k_i} between
    const float2 wst = __ldg(&g_tw13[ki]);
    float2 rw[16];
    rw[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int c = 1; c < 16; ++c) rw[c] = (c & 3) == 0 ? __ldg(&g_tw13[(c * ki) & 8191]) : cmul(rw[c - 1], wst);
    float2 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float2 x = sm[pad(ki * 16 + c)];
      v[c] = c == 0 ? x : cmul(x, rw[c]);
    }
    dftr<16>(v);   // v[brev(k_c)] = spectrum at (k_i, k_c)
    if constexpr (TEMPLATE) {
#pragma unroll
      for (int kc = 0; kc < 16; ++kc) {
        const float2 s = v[brev<16>(kc)];
        mx = fmaxf(mx, fmaf(s.x, s.x, s.y * s.y));
        sm[pad(ki * 16 + kc)] = s;
      }
    } else {
      const float4* T4 = reinterpret_cast<const float4*>(q.B + base + ki * 16);
      float2 g[16];
#pragma unroll
      for (int h2 = 0; h2 < 8; ++h2) {
        const float4 tt = __ldg(&T4[h2]);
        const float2 T0 = make_float2(tt.x, tt.y), T1 = make_float2(tt.z, tt.w);
        const float2 Z0 = v[brev<16>(2 * h2)], Z1 = v[brev<16>(2 * h2 + 1)];
        mx = fmaxf(mx, fmaf(Z0.x, Z0.x, Z0.y * Z0.y));
        mx = fmaxf(mx, fmaf(Z1.x, Z1.x, Z1.y * Z1.y));
        g[2 * h2] = cmul(T0, cconj(Z0));
        g[2 * h2 + 1] = cmul(T1, cconj(Z1));
      }
      dftr<16>(g);   // inverse of the inner dim (conjugated form): g[brev(c)]
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const float2 x = g[brev<16>(c)];
        sm[pad(ki * 16 + c)] = c == 0 ? x : cmul(x, rw[c]);
      }
    }
  }
  __syncthreads();
  if constexpr (!TEMPLATE) bfft(sm, 9, 4);
  for (int u = 0; u < kLPPT; ++u) {
    const int e = threadIdx.x + u * kLT;
    buf[base + e] = sm[pad(e)];
  }
  mx = block_red(mx, redf, OpMax());
  if (threadIdx.x == 0) {
    const Ws w = ws_of(q.ws);
    atomicMax(TEMPLATE ? &w.h->tc2 : &w.h->zc2, __float_as_uint(mx));
  }
}

// ---------------------------------------------------------------- step 7
// delta of the correlation through length-P FFTs (u = 2^-24): one FFT has
// relative 2-norm error <= epsF = 14 u log2 P; with Tp >= max |T_k| (exact
// spectrum), Zc = max |Z~_k| and the 2-norms t2, z2 the inverse of the
// product is off by at most epsF (t2 Zc + 2 Tp z2) + 4 u Tp z2 in every
// entry (the normwise bound of the shared-memory path with one term).
__device__ __forceinline__ float large_delta(const LHdr& h, int logP, bool ints) {
  const float u = 5.9604644775390625e-08f;
  const float epsF = 14.0f * u * float(logP);
  const float t2 = sqrtf(float(h.t2sq)) * 1.0001f;
  const float z2 = (ints ? sqrtf(float(h.z2i)) : sqrtf(float(h.z2f))) * 1.0001f;
  const float Tp = 1.0001f * sqrtf(__uint_as_float(h.tc2)) + epsF * sqrtf(float(1 << logP)) * t2;
  const float Zc = 1.0001f * sqrtf(__uint_as_float(h.zc2));
  return 1.02f * (epsF * (t2 * Zc + 2.0f * Tp * z2) + 4.0f * u * Tp * z2) + 1e-30f;
}

// Every index with r~_j >= max_j - 2 delta joins the candidate list of j
// (grid: kCandPer entries per CTA, modulus j = blockIdx.y).
constexpr int kCandPer = 8 * kLT;
template <bool B>
__global__ void __launch_bounds__(kLT) lcand_kernel(const LQ q1, const LQ* __restrict__ lqs) {
  TM_LQ(q)
  const Ws w = ws_of(q.ws);
  const LHdr& h = *w.h;
  const int j = blockIdx.y;
  const int Mj = j == 0 ? q.M[0] : q.M[1];
  const int64_t base = int64_t(blockIdx.x) * kCandPer + threadIdx.x;
  if (base >= Mj) return;
  const float delta = large_delta(h, q.logP, int_dtype(q.xdtype));
  const float thr = fkey_inv(unsigned(h.rkey[j] >> 32)) - 2.0f * delta;
  const float* r = q.r + int64_t(j) * q.P;
  float v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int64_t n = base + u * kLT;
    v[u] = n < Mj ? r[n] : -INFINITY;
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (v[u] >= thr) {
      const int c = atomicAdd(&w.h->ncand[j], 1);
      if (c < kLargeCap) w.cand[j * kLargeCap + c] = int(base + u * kLT);
    }
  }
}

// Chunk h of nch over K: [h ceil(K/nch), ...).
__device__ __forceinline__ void chunk_range(int K, int nch, int h, int& i0, int& i1) {
  const int len = (K + nch - 1) / nch;
  i0 = min(K, h * len);
  i1 = min(K, i0 + len);
}

// Exact partial dot sum_{i0<=i<i1} t_i v(i) over the block: int64 for
// integer data (t integral), else double-float pairs (DF) in a fixed order,
// added across the block as pairs (warps in index order) and converted to
// fp64 once. Thread 0 gets it.
// The loads of eight terms per thread are in flight before any is used.
template <class F>
__device__ __forceinline__ long long block_dot(const float* t, int i0, int i1, bool exact, F v, double* rd,
                                               long long* rl) {
  constexpr int U = 8;
  long long ai = 0;
  DF ad;
  for (int i = i0 + threadIdx.x; i < i1; i += U * kLT) {
    float tv[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int ii = i + u * kLT;
      tv[u] = ii < i1 ? __ldg(&t[ii]) : 0.f;
      xv[u] = ii < i1 ? v(ii) : 0.f;
    }
    if (exact) {
#pragma unroll
      for (int u = 0; u < U; ++u) ai += (long long)__float2int_rn(tv[u]) * (long long)__float2int_rn(xv[u]);
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) ad.add_prod(tv[u], xv[u]);
    }
  }
  if (exact) return block_red(ai, rl, OpAdd());
  DF s[1] = {ad};
  block_sum_df<kLW>(s, reinterpret_cast<float2*>(rd));   // a double per warp holds a float2
  return __double_as_longlong(s[0].value());
}

// Chunks per listed item: enough items for two waves of the launch's CTAs
// of this query, chunks of at least 2048 terms, at most cap partial sums.
__device__ __forceinline__ int chunks_for(int items, int K, int cap) {
  if (items <= 0) return 1;
  int n = (2 * int(gridDim.x) + items - 1) / items;
  n = min(n, (K + 2047) / 2048);
  n = min(n, cap / items);
  return max(n, 1);
}
template <class F>
__device__ __forceinline__ double warp_dot(const float* t, int K, bool exact, F v) {
  const int lane = threadIdx.x & 31;
  if (exact) {
    long long a = 0;
    for (int i = lane; i < K; i += 32) a += (long long)__float2int_rn(__ldg(&t[i])) * (long long)v(i);
    return double(warp_red(a, OpAdd()));
  }
  DF a;
  for (int i = lane; i < K; i += 32) a.add_prod(__ldg(&t[i]), float(v(i)));
  return warp_sum_df(a).value();
}

__device__ __forceinline__ float yval(const LQ& q, int j, int64_t k) {
  return int_dtype(q.xdtype) ? float(static_cast<const int32_t*>(q.y)[int64_t(j) * q.P + k])
                             : static_cast<const float*>(q.y)[int64_t(j) * q.P + k];
}

constexpr int64_t kFullRescoreWork = int64_t(1) << 36;

// Exact rescoring: the candidates of each modulus in chunks (partial sums),
// or, above kLargeCap candidates, every index (a warp per index, the best
// per CTA) when M K <= 2^36.
template <bool B>
__global__ void __launch_bounds__(kLT) lrescore_kernel(const LQ q1, const LQ* __restrict__ lqs) {
  TM_LQ(q)
  __shared__ double rd[kLW];
  __shared__ long long rl[kLW];
  __shared__ double bv_s[kLW];
  __shared__ long long bi_s[kLW];
  const Ws w = ws_of(q.ws);
  const bool ints = int_dtype(q.xdtype);
  const bool exact = ints && w.h->tbad == 0;
  const int nc0 = w.h->ncand[0], nc1 = w.h->ncand[1];
  const int n0 = nc0 <= kLargeCap ? nc0 : 0, n1 = nc1 <= kLargeCap ? nc1 : 0;   // listed
  const int nch = chunks_for(n0 + n1, q.K, kLargePart);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    w.h->nch = nch;
    w.h->nbest = int(gridDim.x);
  }
  for (int it = blockIdx.x; it < (n0 + n1) * nch; it += gridDim.x) {
    const int cg = it / nch, hh = it - cg * nch;
    const int j = cg < n0 ? 0 : 1;
    const int64_t m = w.cand[j * kLargeCap + (j == 0 ? cg : cg - n0)];
    int i0, i1;
    chunk_range(q.K, nch, hh, i0, i1);
    const long long s = block_dot(q.t, i0, i1, exact, [&](int i) { return yval(q, j, m + i); }, rd, rl);
    if (threadIdx.x == 0) w.part[int64_t(it)] = s;
  }
  for (int j = 0; j < 2; ++j) {
    const int nc = j == 0 ? nc0 : nc1;
    const int Mj = j == 0 ? q.M[0] : q.M[1];
    if (nc <= kLargeCap) {
      continue;
    } else if (int64_t(Mj) * q.K <= kFullRescoreWork) {
      double bv = -INFINITY;
      long long bi = 0x7fffffffffffffffll;
      const int warp = threadIdx.x >> 5;
      for (int64_t m = int64_t(blockIdx.x) * kLW + warp; m < Mj; m += int64_t(gridDim.x) * kLW) {
        const double v = warp_dot(q.t, q.K, exact, [&](int i) { return yval(q, j, m + i); });
        better(bv, bi, v, m);
      }
      block_best(bv, bi, bv_s, bi_s);
      if (threadIdx.x == 0) {
        w.best[(int64_t(j) * kLargeCtas + blockIdx.x) * 2] = __double_as_longlong(bv);
        w.best[(int64_t(j) * kLargeCtas + blockIdx.x) * 2 + 1] = bi;
      }
    }
  }
}

// Sum of n partial dot products (int64, or fp64 bits) over one warp:
// lane-strided, then a fixed shuffle tree; the value is in every lane.
__device__ __forceinline__ double sum_chunks(const long long* p, int n, bool exact) {
  const int lane = threadIdx.x & 31;
  if (exact) {
    long long s = 0;
    for (int i = lane; i < n; i += 32) s += p[i];
    return double(warp_red(s, OpAdd()));
  }
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += __longlong_as_double(p[i]);
  return warp_red(s, OpAdd());
}

// Step 7 decisions and steps 8 (one CTA).
template <bool B>
__global__ void __launch_bounds__(kLT) lselect_kernel(const LQ q1, const LQ* __restrict__ lqs) {
  TM_LQ(q)
  __shared__ double bv_s[kLW];
  __shared__ long long bi_s[kLW];
  const Ws w = ws_of(q.ws);
  LHdr& h = *w.h;
  const bool exact = int_dtype(q.xdtype) && h.tbad == 0;
  const int nch = h.nch;
  const int n0 = h.ncand[0] <= kLargeCap ? h.ncand[0] : 0;
  for (int j = 0; j < 2; ++j) {
    const int nc = h.ncand[j];
    const int Mj = j == 0 ? q.M[0] : q.M[1];
    double bv = -INFINITY;
    long long bi = 0x7fffffffffffffffll;
    int mode;
    if (nc <= kLargeCap) {
      mode = 0;
      const int warp = threadIdx.x >> 5;
      for (int c = warp; c < nc; c += kLW) {   // a warp per candidate, its chunks in a fixed order
        const double v = sum_chunks(w.part + int64_t(j == 0 ? c : n0 + c) * nch, nch, exact);
        if ((threadIdx.x & 31) == 0) better(bv, bi, v, w.cand[j * kLargeCap + c]);
      }
    } else if (int64_t(Mj) * q.K <= kFullRescoreWork) {
      mode = 1;
      for (int b = threadIdx.x; b < h.nbest; b += blockDim.x)
        better(bv, bi, __longlong_as_double(w.best[(int64_t(j) * kLargeCtas + b) * 2]),
               w.best[(int64_t(j) * kLargeCtas + b) * 2 + 1]);
    } else {
      mode = 2;
      if (threadIdx.x == 0) {
        bv = double(fkey_inv(unsigned(h.rkey[j] >> 32)));
        bi = (long long)(0xffffffffull - (h.rkey[j] & 0xffffffffull));
      }
    }
    block_best(bv, bi, bv_s, bi_s);
    if (threadIdx.x == 0) {
      h.mode[j] = mode;
      h.m[j] = int(bi);
      h.rv[j] = bv;
      if (mode == 1) h.flags |= TM_RF_FULL_RESCORE;
      if (mode == 2) h.flags |= TM_RF_UNCERTIFIED;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    CrtSet c = crt_intersect(q.N, q.M[0], q.M[1], q.inv, h.m[0], h.m[1]);
    if (q.thm2) c.nw = 0;   // wrapped members fall in the zero padding
    h.crt = c;
    h.ncs = c.nnat + c.nw;
  }
}

__device__ __forceinline__ int64_t member(const CrtSet& c, int64_t i) {
  return i < c.nnat ? c.m0 + i * c.step : c.w[i - c.nnat];
}

// Step 9 scores (Tx)_m of the members: chunked partial sums for up to
// kLargeMembers members, else a warp per member and the best per CTA.
template <int DT>
__device__ void lscore_impl(const LQ& q) {
  __shared__ double rd[kLW];
  __shared__ long long rl[kLW];
  __shared__ double bv_s[kLW];
  __shared__ long long bi_s[kLW];
  const Ws w = ws_of(q.ws);
  const CrtSet c = w.h->crt;
  const int64_t ncs = w.h->ncs;
  const bool exact = int_dtype(q.xdtype) && w.h->tbad == 0;
  const int nch = ncs <= kLargeMembers ? chunks_for(int(ncs), q.K, kLargeMPart) : 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) w.h->nchm = nch;
  const int64_t N = q.N;
  auto xv = [&](int64_t m, int i) {
    int64_t n = m + i;
    if (n >= N) n -= N;
    return sval<DT>(q.x, n);
  };
  if (ncs <= kLargeMembers) {
    const int items = int(ncs) * nch;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
      const int mi = it / nch, hh = it - mi * nch;
      const int64_t m = member(c, mi);
      int i0, i1;
      chunk_range(q.K, nch, hh, i0, i1);
      const long long s = block_dot(q.t, i0, i1, exact, [&](int i) { return xv(m, i); }, rd, rl);
      if (threadIdx.x == 0) w.mpart[int64_t(it)] = s;
    }
  } else {
    double bv = -INFINITY;
    long long bi = 0x7fffffffffffffffll;
    const int warp = threadIdx.x >> 5;
    for (int64_t mi = int64_t(blockIdx.x) * kLW + warp; mi < ncs; mi += int64_t(gridDim.x) * kLW) {
      const int64_t m = member(c, mi);
      better(bv, bi, warp_dot(q.t, q.K, exact, [&](int i) { return xv(m, i); }), m);
    }
    block_best(bv, bi, bv_s, bi_s);
    if (threadIdx.x == 0) {
      w.mbest[int64_t(blockIdx.x) * 2] = __double_as_longlong(bv);
      w.mbest[int64_t(blockIdx.x) * 2 + 1] = bi;
    }
  }
}
template <bool B>
__global__ void __launch_bounds__(kLT) lscore_kernel(const LQ q1, const LQ* __restrict__ lqs) {
  TM_LQ(q)
  switch (q.xdtype) {
    case TM_I8_PM1: lscore_impl<TM_I8_PM1>(q); break;
    case TM_BITS_PM1: lscore_impl<TM_BITS_PM1>(q); break;
    case TM_F16: lscore_impl<TM_F16>(q); break;
    default: lscore_impl<TM_F32>(q); break;
  }
}

// The result record (one CTA).
template <bool B>
__global__ void __launch_bounds__(kLT) lfinish_kernel(const LQ q1, const LQ* __restrict__ lqs, tm_result* out) {
  TM_LQ(q)
  __shared__ double bv_s[kLW];
  __shared__ long long bi_s[kLW];
  const Ws w = ws_of(q.ws);
  const LHdr& h = *w.h;
  const int64_t ncs = h.ncs;
  const bool exact = int_dtype(q.xdtype) && h.tbad == 0;
  const int nch = h.nchm;
  double bv = -INFINITY;
  long long bi = 0x7fffffffffffffffll;
  if (ncs <= kLargeMembers) {
    const int warp = threadIdx.x >> 5;
    for (int mi = warp; mi < ncs; mi += kLW) {
      const double v = sum_chunks(w.mpart + int64_t(mi) * nch, nch, exact);
      if ((threadIdx.x & 31) == 0) better(bv, bi, v, member(h.crt, mi));
    }
  } else {
    for (int b = threadIdx.x; b < h.nbest; b += blockDim.x)
      better(bv, bi, __longlong_as_double(w.mbest[2 * b]), w.mbest[2 * b + 1]);
  }
  block_best(bv, bi, bv_s, bi_s);
  if (threadIdx.x == 0) {
    tm_result res;
    res.n_cand = int32_t(ncs > 0x7fffffff ? 0x7fffffff : ncs);
    if (ncs == 0) { res.shift = -1; res.status = TM_EMPTY; res.score = 0.0; }
    else { res.shift = bi; res.status = ncs == 1 ? TM_FOUND : TM_RESOLVED; res.score = bv; }
    res.status |= h.flags;
    if (*q.err) res.status |= TM_RF_DEVICE_ERROR;
    res.m1 = h.m[0];
    res.m2 = h.m[1];
    res.r1 = h.rv[0];
    res.r2 = h.rv[1];
    res.m3 = 0;
    res.reserved = 0;
    res.r3 = 0.0;
    out[q.qi] = res;
  }
}

__global__ void linit_kernel(const LQ* __restrict__ lqs, void* ws1) {
  void* ws = lqs != nullptr ? lqs[blockIdx.z].ws : ws1;
  LHdr* h = ws_of(ws).h;
  unsigned* p = reinterpret_cast<unsigned*>(h);
  for (int i = threadIdx.x; i < int(sizeof(LHdr) / 4); i += blockDim.x) p[i] = 0u;
}

constexpr int kSmemBytes = kSmemPts * int(sizeof(float2));

// The template spectra (the workspace headers first): they read only t and
// may run beside the fold.
template <bool B>
cudaError_t launch_large_tpl(const LQ& q1, const LQ* d_lq, int n, int maxP, bool two_dims, cudaStream_t s) {
  const dim3 g(unsigned(maxP / kLPts), 1, unsigned(n));
  const LQ* lq = B ? d_lq : nullptr;
  linit_kernel<<<dim3(1, 1, unsigned(n)), 128, 0, s>>>(lq, q1.ws);
  lfwd_kernel<kSrcT, B><<<g, kLT, kSmemBytes, s>>>(q1, lq, 0, 1, 1);
  if (two_dims) lfwd_kernel<kSrcBuf, B><<<g, kLT, kSmemBytes, s>>>(q1, lq, 1, 1, 1);
  lrow_kernel<true, B><<<g, kLT, kSmemBytes, s>>>(q1, lq);
  return cudaGetLastError();
}

// The signal spectra, product and inverse, then steps 7-9 (after the folds
// and the template spectra).
template <bool B>
cudaError_t launch_large_sig(const LQ& q1, const LQ* d_lq, int n, int maxP, bool two_dims, int maxM, tm_result* out,
                             cudaStream_t s) {
  const dim3 g(unsigned(maxP / kLPts), 1, unsigned(n));
  // rescoring and scoring: about kLargeCtas CTAs in all, at least 64 per query
  const unsigned per = unsigned(std::max(64, kLargeCtas / n));
  const LQ* lq = B ? d_lq : nullptr;
  // signal spectrum, product and the row inverse
  lfwd_kernel<kSrcY, B><<<g, kLT, kSmemBytes, s>>>(q1, lq, 0, 0, 0);
  if (two_dims) lfwd_kernel<kSrcBuf, B><<<g, kLT, kSmemBytes, s>>>(q1, lq, 1, 0, 0);
  lrow_kernel<false, B><<<g, kLT, kSmemBytes, s>>>(q1, lq);
  // the rest of the inverse, outermost dim last
  if (two_dims) linv_kernel<false, B><<<g, kLT, kSmemBytes, s>>>(q1, lq, 1);
  linv_kernel<true, B><<<g, kLT, kSmemBytes, s>>>(q1, lq, 0);
  // steps 7-9
  lcand_kernel<B><<<dim3(unsigned((maxM + kCandPer - 1) / kCandPer), 2, unsigned(n)), kLT, 0, s>>>(q1, lq);
  lrescore_kernel<B><<<dim3(per, 1, unsigned(n)), kLT, 0, s>>>(q1, lq);
  lselect_kernel<B><<<dim3(1, 1, unsigned(n)), kLT, 0, s>>>(q1, lq);
  lscore_kernel<B><<<dim3(per, 1, unsigned(n)), kLT, 0, s>>>(q1, lq);
  lfinish_kernel<B><<<dim3(1, 1, unsigned(n)), kLT, 0, s>>>(q1, lq, out);
  return cudaGetLastError();
}

}  // namespace

size_t large_ws_bytes() { return kWsBytes; }

int large_launches(int nsd) { return 1 + 2 * (nsd + 1) + nsd + 5; }   // per batch (nsd: most strided dims)

cudaError_t large_configure() {
  cudaError_t e;
#define TM_SMEM(k)                                                                          \
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);    \
  if (e != cudaSuccess) return e;
  TM_SMEM((lfwd_kernel<kSrcBuf, false>));
  TM_SMEM((lfwd_kernel<kSrcY, false>));
  TM_SMEM((lfwd_kernel<kSrcT, false>));
  TM_SMEM((linv_kernel<false, false>));
  TM_SMEM((linv_kernel<true, false>));
  TM_SMEM((lrow_kernel<false, false>));
  TM_SMEM((lrow_kernel<true, false>));
  TM_SMEM((lfwd_kernel<kSrcBuf, true>));
  TM_SMEM((lfwd_kernel<kSrcY, true>));
  TM_SMEM((lfwd_kernel<kSrcT, true>));
  TM_SMEM((linv_kernel<false, true>));
  TM_SMEM((linv_kernel<true, true>));
  TM_SMEM((lrow_kernel<false, true>));
  TM_SMEM((lrow_kernel<true, true>));
#undef TM_SMEM
  float2 h[8192];
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < 8192; ++m) {
    const double a = two_pi * double(m) / 8192.0;
    h[m] = make_float2(float(cos(a)), float(-sin(a)));
  }
  return cudaMemcpyToSymbol(g_tw13, h, sizeof(h));
}

cudaError_t launch_large_template(const LQ* d_lq, const LQ* h_lq, int n, int maxP, bool two_dims, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (maxP < (1 << kLogPMinLarge) || maxP > (1 << kLogPMaxLarge)) return cudaErrorInvalidValue;
  if (n == 1) return launch_large_tpl<false>(h_lq[0], d_lq, 1, maxP, two_dims, s);
  return launch_large_tpl<true>(h_lq[0], d_lq, n, maxP, two_dims, s);
}

cudaError_t launch_large_signal(const LQ* d_lq, const LQ* h_lq, int n, int maxP, bool two_dims, int maxM,
                                tm_result* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (maxP < (1 << kLogPMinLarge) || maxP > (1 << kLogPMaxLarge)) return cudaErrorInvalidValue;
  if (n == 1) return launch_large_sig<false>(h_lq[0], d_lq, 1, maxP, two_dims, maxM, out, s);
  return launch_large_sig<true>(h_lq[0], d_lq, n, maxP, two_dims, maxM, out, s);
}

cudaError_t launch_correlate_large(const LQ* d_lq, const LQ* h_lq, int n, int maxP, bool two_dims, int maxM,
                                   tm_result* out, cudaStream_t s) {
  const cudaError_t e = launch_large_template(d_lq, h_lq, n, maxP, two_dims, s);
  if (e != cudaSuccess) return e;
  return launch_large_signal(d_lq, h_lq, n, maxP, two_dims, maxM, out, s);
}

}  // namespace ftm
