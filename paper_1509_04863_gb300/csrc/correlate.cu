// Steps 3 (completion) and 4-9 of Algorithm 1, one CTA per query.
//
//  a. Template spectrum T = FFT_P([t 0]) (steps 4-5), kept in shared memory
//     when the launch left room for it (P <= 8192), else in global scratch.
//  b. Folds: y_j[k] (k < M_j) from the fold kernel's per-share counts, plus
//     the wrap-around entry x_{k-R} for k >= R = N-(L-1)M (indexing mod N)
//     and the (< 16) signal bytes the fold kernel did not cover; then the
//     extension y[M+i] = y[i] - x_i + x_{(i+LM) mod N}, i < K-1 (the fold
//     of Eq. (2) over k = 0..M+K-2). Written to global memory exactly.
//  c. Both folds ride one complex FFT, z = y_1 + i y_2 (step 5). Since
//     conj(T) Z = conj(T) Y_1 + i conj(T) Y_2 and both correlations are real,
//     one inverse transform of conj(T) Z (step 6, with the conjugate that
//     turns the product into a cross-correlation) gives r_1 in its real part
//     and r_2 in its imaginary part. The inverse is taken as
//     IFFT(W) = conj(FFT(conj(W)))/P, so conj(T) Z becomes T conj(Z).
//  d. Step 7: argmax of r_j over j < M_j. The FFT values carry rounding
//     error |dr| <= delta (a normwise bound, below); every j with
//     r_j >= max - 2 delta is rescored exactly from the folds (integers in
//     int32/int64, reals in double-float pairs on the FP32 pipes, reduced as
//     pairs), which makes the chosen index exact.
//  e. Steps 8-9: closed-form intersection (crt.h); several members are
//     resolved by their exact (Tx)_m.
//
// FFT: Stockham autosort, radix 16 (plus one radix 2/4/8 pass, computed
// from registers by the producing loop for P = 8192 and 16384), shared
// memory resident (P <= 16384 complex entries, padded one entry per 16 to
// avoid bank conflicts). Twiddles W_P^m, m < P/2, are copied once per CTA
// into shared memory from a table computed on the host in double precision
// (W_P^{m+P/2} = -W_P^m gives the other half).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "crt.h"
#include "device_util.cuh"
#include "tm_internal.h"

namespace ftm {
namespace {

constexpr int kWarps = kCorrThreads / 32;

__device__ __forceinline__ int pad_idx(int i) { return i + (i >> 4); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// cos(2 pi m / 16) and sin(2 pi m / 16), m < 8.
__device__ __forceinline__ float c16(int m) {
  constexpr float C[8] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                          0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f};
  return C[m];
}
__device__ __forceinline__ float s16(int m) {
  constexpr float S[8] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                          1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f};
  return S[m];
}

template <int R>
__host__ __device__ constexpr int bitrev(int r) {
  int o = 0;
  for (int b = 1; b < R; b <<= 1) {
    o = (o << 1) | (r & 1);
    r >>= 1;
  }
  return o;
}

// In-register DFT of size R (forward, e^{-2 pi i/R}) by radix-2 decimation in
// frequency; output index r is found at position bitrev(r).
template <int R>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
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
        const int m = k * (16 / len);   // W_len^k = W_16^m
        if (m == 0) {
          v[s + k + half] = d;
        } else if (m == 4) {            // -i
          v[s + k + half] = make_float2(d.y, -d.x);
        } else {
          const float c = c16(m), sn = s16(m);
          v[s + k + half] = make_float2(d.x * c + d.y * sn, d.y * c - d.x * sn);
        }
      }
    }
  }
}

// W_P^e for 0 <= e < P from the half table tw[m] = W_P^m, m < P/2.
__device__ __forceinline__ float2 twiddle(const float2* tw, int e, int halfP) {
  const float2 w = tw[e & (halfP - 1)];
  return (e & halfP) ? make_float2(-w.x, -w.y) : w;
}

// One Stockham pass of radix R over P points whose sub-transforms of length
// Ns are done: butterfly j takes x[j + r P/R], twiddles by W_{Ns R}^{r (j mod Ns)},
// and writes to (j - j mod Ns) R + j mod Ns + r Ns. The twiddles come from
// the pass table stab[(r-1) Ns + k] = W_{16 Ns}^{r k} when given (lanes with
// consecutive k read consecutive entries), else from the half table tw.
template <int R, int NBMAX>
__device__ __forceinline__ void fft_pass(float2* buf, int P, int Ns, int twshift, const float2* tw,
                                         const float2* stab) {
  // butterflies per thread: NBMAX radix-16 butterflies' worth of points
  constexpr int NB = (NBMAX * 16) / R;
  const int nbf = P / R;
  float2 v[NB][R];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = threadIdx.x + b * kCorrThreads;
    if (j < nbf) {
      const int k = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = buf[pad_idx(j + r * nbf)];
      if (Ns > 1) {
        if (stab != nullptr) {
#pragma unroll
          for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], stab[(r - 1) * Ns + k]);
        } else {
#pragma unroll
          for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], twiddle(tw, (r * k) << twshift, P >> 1));
        }
      }
      dft<R>(v[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = threadIdx.x + b * kCorrThreads;
    if (j < nbf) {
      const int k = j & (Ns - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[pad_idx(base + r * Ns)] = v[b][bitrev<R>(r)];
    }
  }
  __syncthreads();
}

// Pass tables for every radix-16 pass but the last (16 Ns < P), packed one
// after the other: 15 Ns entries W_{16 Ns}^{r k}, r = 1..15, k < Ns. At most
// 15 (4 + 64) = 1020 entries for P <= 16384.
constexpr int kPassTw = 1024;
__device__ __forceinline__ int pass_first(int logP) { return logP & 3; }

// Fills the pass tables from the global table gtw[m] = W_{kPMax}^m.
__device__ void build_pass_twiddles(float2* stw, int logP, const float2* __restrict__ gtw) {
  const int P = 1 << logP;
  int off = 0;
  for (int Ns = 1 << pass_first(logP); 16 * Ns < P; Ns <<= 4) {
    if (Ns > 1) {
      const int stride = kPMax / (16 * Ns);
      for (int i = threadIdx.x; i < 15 * Ns; i += kCorrThreads) {
        const int r = i / Ns + 1, k = i - (r - 1) * Ns;
        stw[off + i] = __ldg(&gtw[r * k * stride]);
      }
      off += 15 * Ns;
    }
  }
}

// Forward FFT of length 2^logP <= 8192 NBMAX in place (padded layout,
// natural order); tw holds W_P^m for m < P/2, stw the pass tables of
// build_pass_twiddles. Each thread holds NBMAX x 16 points per pass.
template <int NBMAX>
__device__ __forceinline__ void fft(float2* buf, int logP, const float2* tw, const float2* stw,
                                    bool skip_first = false) {
  const int P = 1 << logP;
  int logNs = 0;
  const int first = pass_first(logP);
  if (first && skip_first) {
    logNs = first;   // done by first_pass_regs
  } else if (first) {
    const int twshift = logP - first;
    if (first == 1) fft_pass<2, NBMAX>(buf, P, 1, twshift, tw, nullptr);
    else if (first == 2) fft_pass<4, NBMAX>(buf, P, 1, twshift, tw, nullptr);
    else fft_pass<8, NBMAX>(buf, P, 1, twshift, tw, nullptr);
    logNs = first;
  }
  int off = 0;
  while (logNs < logP) {
    const int Ns = 1 << logNs;
    const bool last = logNs + 4 == logP;
    fft_pass<16, NBMAX>(buf, P, Ns, logP - (logNs + 4), tw, (last || Ns == 1) ? nullptr : stw + off);
    if (!last && Ns > 1) off += 15 * Ns;
    logNs += 4;
  }
}

// The first pass of fft() for P = 8192 (radix 2) or 16384 (radix 4), whose
// sub-transforms have length 1 (no twiddles), from registers: the thread
// holds x[b] = the input at k = tid + 512 b, and since P / R0 = 8 x 512,
// butterfly j = tid + 512 b takes the inputs j + r P / R0 = x[b + 8 r] of
// the same thread. Writes buf (padded) exactly as fft_pass<R0> with Ns = 1;
// the caller orders the writes (barrier) before fft(..., skip_first).
__device__ __forceinline__ bool first_pass_in_regs(int logP) { return logP == 13 || logP == 14; }

template <int R0, int NV>
__device__ __forceinline__ void first_pass_regs_r(float2* buf, const float2 (&x)[NV]) {
  constexpr int per = 8;   // butterflies per thread: P / R0 / 512
  static_assert(R0 * per <= NV, "inputs of the thread's butterflies");
#pragma unroll
  for (int b = 0; b < per; ++b) {
    float2 v[R0];
#pragma unroll
    for (int r = 0; r < R0; ++r) v[r] = x[b + r * per];
    dft<R0>(v);
    const int j = threadIdx.x + b * kCorrThreads;
#pragma unroll
    for (int r = 0; r < R0; ++r) buf[pad_idx(j * R0 + r)] = v[bitrev<R0>(r)];
  }
}

template <int NV>
__device__ __forceinline__ void first_pass_regs(float2* buf, int logP, const float2 (&x)[NV]) {
  if (logP == 13) first_pass_regs_r<2>(buf, x);
  else if constexpr (NV >= 32) first_pass_regs_r<4>(buf, x);
}

// ---------------------------------------------------------------- block reductions
template <class T>
__device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s += red[w];
  return s;
}

// Two float sums and an AND over the block in one exchange (red: 2 kWarps floats).
__device__ __forceinline__ void block_sum2_and(float& a, float& b, int& c, float* red, int* redi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  c = __all_sync(0xffffffffu, c);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = a;
    red[kWarps + (threadIdx.x >> 5)] = b;
    redi[threadIdx.x >> 5] = c;
  }
  __syncthreads();
  a = 0.f;
  b = 0.f;
  c = 1;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    a += red[w];
    b += red[kWarps + w];
    c &= redi[w];
  }
}

// Four 64-bit sums over the block in one exchange (red: 4 kWarps entries);
// valid in thread 0.
template <class T>
__device__ __forceinline__ void block_sum4(T (&v)[4], T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < 4; ++i) red[4 * (threadIdx.x >> 5) + i] = v[i];
  __syncthreads();
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    T s = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += red[4 * w + i];
    v[i] = s;
  }
}

__device__ __forceinline__ int block_and(int v, int* redi) {
  v = __all_sync(0xffffffffu, v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) redi[threadIdx.x >> 5] = v;
  __syncthreads();
  int s = 1;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s &= redi[w];
  return s;
}

__device__ __forceinline__ int block_max(int v, int* redi) {
  v = __reduce_max_sync(0xffffffffu, v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) redi[threadIdx.x >> 5] = v;
  __syncthreads();
  int s = redi[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) s = max(s, redi[w]);
  return s;
}

// max value, smallest index on ties
__device__ __forceinline__ float block_maxf(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = red[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) m = fmaxf(m, red[w]);
  return m;
}

__device__ __forceinline__ void better(float& v, int& i, float v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}
__device__ __forceinline__ void betterd(double& v, int64_t& i, double v2, int64_t i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__device__ __forceinline__ void block_argmax(float& v, int& i, float* redv, int* redi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) better(v, i, __shfl_xor_sync(0xffffffffu, v, o), __shfl_xor_sync(0xffffffffu, i, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { redv[threadIdx.x >> 5] = v; redi[threadIdx.x >> 5] = i; }
  __syncthreads();
  v = redv[0]; i = redi[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) better(v, i, redv[w], redi[w]);
}

// ---------------------------------------------------------------- signal access
struct Sig {
  const void* x;
  int32_t dtype;
  __device__ __forceinline__ float val(int64_t n) const {
    switch (dtype) {
      case TM_I8_PM1: return (static_cast<const uint8_t*>(x)[n] & 2u) ? -1.0f : 1.0f;
      case TM_BITS_PM1: return ((static_cast<const uint8_t*>(x)[n >> 3] >> (n & 7)) & 1u) ? 1.0f : -1.0f;
      case TM_F16: return __half2float(static_cast<const __half*>(x)[n]);
      default: return static_cast<const float*>(x)[n];
    }
  }
  __device__ __forceinline__ int ival(int64_t n) const {
    if (dtype == TM_I8_PM1) return (static_cast<const uint8_t*>(x)[n] & 2u) ? -1 : 1;
    return ((static_cast<const uint8_t*>(x)[n >> 3] >> (n & 7)) & 1u) ? 1 : -1;
  }
};

__device__ __forceinline__ bool is_int_dtype(int d) { return d == TM_I8_PM1 || d == TM_BITS_PM1; }

// The same accessors with the storage type fixed at compile time, so that
// batches of loads carry no branches and can all be in flight at once.
template <int DT>
struct SigT {
  const void* x;
  __device__ __forceinline__ float val(int64_t n) const {
    if constexpr (DT == TM_I8_PM1) return (__ldg(static_cast<const uint8_t*>(x) + n) & 2u) ? -1.0f : 1.0f;
    else if constexpr (DT == TM_BITS_PM1)
      return ((__ldg(static_cast<const uint8_t*>(x) + (n >> 3)) >> (n & 7)) & 1u) ? 1.0f : -1.0f;
    else if constexpr (DT == TM_F16) return __half2float(static_cast<const __half*>(x)[n]);
    else return __ldg(static_cast<const float*>(x) + n);
  }
};

// Calls f(SigT<dtype>{x}).
template <class F>
__device__ __forceinline__ void with_sig(int dtype, const void* x, F&& f) {
  switch (dtype) {
    case TM_I8_PM1: f(SigT<TM_I8_PM1>{x}); break;
    case TM_BITS_PM1: f(SigT<TM_BITS_PM1>{x}); break;
    case TM_F16: f(SigT<TM_F16>{x}); break;
    default: f(SigT<TM_F32>{x}); break;
  }
}

// Asks L2 for the signal elements [e0, e1) (128-byte lines; no data comes
// back to the SM). Loads of them later in the kernel then wait for L2
// instead of HBM: the fold kernel streamed the signal with evict-first.
__device__ __forceinline__ void prefetch_elems(const void* x, int dtype, int64_t e0, int64_t e1) {
  if (e1 <= e0) return;
  const int sh = dtype == TM_F32 ? 2 : (dtype == TM_F16 ? 1 : 0);
  int64_t b0 = dtype == TM_BITS_PM1 ? e0 >> 3 : e0 << sh;
  const int64_t b1 = dtype == TM_BITS_PM1 ? (e1 + 7) >> 3 : e1 << sh;
  b0 &= ~int64_t(127);
  const char* c = static_cast<const char*>(x);
  for (int64_t o = b0 + int64_t(threadIdx.x) * 128; o < b1; o += int64_t(kCorrThreads) * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

// Exact sum_{i<K} t_i * v(i) over one warp: integer terms in int32 when
// `small` guarantees no partial sum reaches 2^31, else int64; reals in
// double-float pairs (DF), the lanes' pairs added in fp64.
template <class F>
__device__ __forceinline__ double warp_dot(const float* __restrict__ t, int K, bool integral, bool small, F v) {
  const int lane = threadIdx.x & 31;
  if (integral && small) {
    int acc = 0;
#pragma unroll 4
    for (int i = lane; i < K; i += 32) acc += __float2int_rn(t[i]) * int(v(i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return double(acc);
  }
  if (integral) {
    long long acc = 0;
#pragma unroll 4
    for (int i = lane; i < K; i += 32) acc += (long long)__float2int_rn(t[i]) * (long long)v(i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return double(acc);
  }
  DF df;
#pragma unroll 4
  for (int i = lane; i < K; i += 32) df.add_prod(t[i], float(v(i)));
  return warp_sum_df(df).value();
}

// Bound on max_j |r~_j - r_j| for a correlation computed through length-P
// FFTs as the inverse transform of a sum of `terms` spectrum products
// T_b conj(Z_s). Inputs: t2 >= ||t_b||_2 and z2 >= ||z_s||_2 (the blocks'
// 2-norms), Tp >= max_k |T_k| of the exact template spectra, Zc = max_k |Z~_k|
// of the computed signal spectra. Derivation (u = 2^-24; one length-P FFT
// has relative 2-norm error <= epsF = 14 u log2 P, the radix-2 bound
// log2(P) (mu + gamma_4 (sqrt 2 + mu)) with a safety factor of two; the
// unnormalised transform scales 2-norms by sqrt P):
//   T~ Z~* - T Z* = dT Z~* + T dZ*, so each product is off by at most
//   epsF sqrt(P) (t2 Zc + Tp z2) in 2-norm, plus its own rounding and that
//   of the sum, (3 + terms) u |T~ Z~*| <= (3 + terms) u Tp sqrt(P) z2;
//   the inverse transform adds epsF times the 2-norm of its input, at most
//   epsF terms Tp sqrt(P) z2, and divides every 2-norm by sqrt(P) on the
//   way back (the 1/P scaling is exact).
// Hence max_j |dr_j| <= ||dr||_2 <= terms (epsF (t2 Zc + 2 Tp z2) + (3 + terms) u Tp z2).
// The factor 1.02 covers the fp32 rounding of the norms and maxima.
__device__ __forceinline__ float fft_corr_error_bound(int logP, float t2, float Tp, float Zc, float z2, int terms) {
  const float u = 5.9604644775390625e-08f;
  const float epsF = 14.0f * u * float(logP > 0 ? logP : 1);
  return 1.02f * float(terms) *
             (epsF * (t2 * Zc + 2.0f * Tp * z2) + float(3 + terms) * u * Tp * z2) + 1e-30f;
}

// A rigorous bound on max_k |T_k| from the computed spectrum's maximum:
// |T_k - T~_k| <= ||dT||_2 <= epsF sqrt(P) ||t||_2.
__device__ __forceinline__ float spectrum_max_bound(float Tc, int logP, float t2) {
  const float u = 5.9604644775390625e-08f;
  const float epsF = 14.0f * u * float(logP > 0 ? logP : 1);
  return 1.0001f * Tc + epsF * sqrtf(float(1 << logP)) * t2;
}

// Step 7 candidates of each modulus of a query: the argmax of the FFT
// values and every index within 2 delta of it.
struct Cands {
  int cand[3][kCandCap];
  int ncand[3];
};

// Step 7 for modulus mj (rv(k) = r~_mj[k], k < M).
template <class RFn>
__device__ void collect_candidates(Cands& cs, int mj, int M, float delta, RFn rv) {
  __shared__ float redv[kWarps];
  __shared__ int redi[kWarps];
  const int tid = threadIdx.x;
  float bv = -INFINITY;
  int bi = 0x7fffffff;
  for (int k = tid; k < M; k += kCorrThreads) better(bv, bi, rv(k), k);
  block_argmax(bv, bi, redv, redi);
  if (tid == 0) cs.ncand[mj] = 0;
  __syncthreads();
  const float thr = bv - 2.0f * delta;
  for (int k = tid; k < M; k += kCorrThreads) {
    if (rv(k) >= thr) {
      const int c = atomicAdd(&cs.ncand[mj], 1);
      if (c < kCandCap) cs.cand[mj][c] = k;
    }
  }
  __syncthreads();
}

// Step 7 for moduli 0 and 1 together (rv0, rv1 as above): one pass over
// the columns for both maxima, one for both candidate lists, half the
// barriers of two collect_candidates calls. The same lists in the same
// order of discovery per modulus is not guaranteed (atomic slots), as
// with collect_candidates; the rescoring takes the exact maximum with the
// smallest index whatever the order.
template <class RFn0, class RFn1>
__device__ void collect_candidates2(Cands& cs, int M0, int M1, float delta, RFn0 rv0, RFn1 rv1) {
  __shared__ float redv[2 * kWarps];
  __shared__ int redi[2 * kWarps];
  const int tid = threadIdx.x;
  float bv0 = -INFINITY, bv1 = -INFINITY;
  int bi0 = 0x7fffffff, bi1 = 0x7fffffff;
  const int Mx = max(M0, M1);
  for (int k = tid; k < Mx; k += kCorrThreads) {
    if (k < M0) better(bv0, bi0, rv0(k), k);
    if (k < M1) better(bv1, bi1, rv1(k), k);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    better(bv0, bi0, __shfl_xor_sync(0xffffffffu, bv0, o), __shfl_xor_sync(0xffffffffu, bi0, o));
    better(bv1, bi1, __shfl_xor_sync(0xffffffffu, bv1, o), __shfl_xor_sync(0xffffffffu, bi1, o));
  }
  __syncthreads();
  if ((tid & 31) == 0) {
    redv[tid >> 5] = bv0; redi[tid >> 5] = bi0;
    redv[kWarps + (tid >> 5)] = bv1; redi[kWarps + (tid >> 5)] = bi1;
  }
  if (tid == 0) { cs.ncand[0] = 0; cs.ncand[1] = 0; }
  __syncthreads();
  bv0 = redv[0]; bi0 = redi[0];
  bv1 = redv[kWarps]; bi1 = redi[kWarps];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) {
    better(bv0, bi0, redv[w], redi[w]);
    better(bv1, bi1, redv[kWarps + w], redi[kWarps + w]);
  }
  const float thr0 = bv0 - 2.0f * delta, thr1 = bv1 - 2.0f * delta;
  for (int k = tid; k < Mx; k += kCorrThreads) {
    if (k < M0 && rv0(k) >= thr0) {
      const int c = atomicAdd(&cs.ncand[0], 1);
      if (c < kCandCap) cs.cand[0][c] = k;
    }
    if (k < M1 && rv1(k) >= thr1) {
      const int c = atomicAdd(&cs.ncand[1], 1);
      if (c < kCandCap) cs.cand[1][c] = k;
    }
  }
  __syncthreads();
}

// Steps 7-9 after the candidates of every modulus are collected: exact
// rescoring of each candidate from the exported folds (the chosen index is
// the exact argmax), the closed-form intersection of the candidate sets
// (crt.h), the exact (Tx)_m of its member(s) and the result record.
__device__ void resolve(const CorrArgs& a, const CorrQ& Q, int qi, bool t_integral, float t1, int maxy, Cands& cs) {
  __shared__ long long redl[kWarps];
  __shared__ float2 redf2[kWarps];
  __shared__ long long redl4[4 * kWarps];
  __shared__ float2 redf4[4 * kWarps];
  __shared__ double wbest_v[kWarps];
  __shared__ int64_t wbest_i[kWarps];
  __shared__ int s_m[3];
  __shared__ double s_r[3];
  __shared__ int s_flags;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = Q.P, K = Q.K;
  const int64_t N = Q.N;
  const Sig sig{Q.x, Q.xdtype};
  const bool ints = is_int_dtype(Q.xdtype);
  const float* __restrict__ t = Q.t;
  if (tid == 0) {
    s_flags = 0;
    s_m[2] = 0;
    s_r[2] = 0.0;
  }
  __syncthreads();
  const bool exact_int = ints && t_integral;
  // int32 rescoring is exact when every partial sum stays below 2^31:
  // |sum| <= ||t||_1 max|y|
  const bool small = exact_int && double(t1) * double(maxy) < 2.0e9;
  const void* yv = Q.y_in != nullptr ? Q.y_in : static_cast<const void*>(static_cast<const char*>(a.y) + Q.y_off * 4);

  // exact rescoring: the listed candidates of every modulus together, four
  // at a time, each summed by the whole block
  int nlist[3] = {0, 0, 0};
  for (int j = 0; j < Q.nmod; ++j) nlist[j] = cs.ncand[j] <= kCandCap ? cs.ncand[j] : 0;
  const int b1 = nlist[0], b2 = nlist[0] + nlist[1], total = b2 + nlist[2];
  double bvj[3] = {-INFINITY, -INFINITY, -INFINITY};
  int64_t bij[3] = {0x7fffffffffffffffll, 0x7fffffffffffffffll, 0x7fffffffffffffffll};
  for (int c0 = 0; c0 < total; c0 += 4) {
    const int nb = min(4, total - c0);
    int jj[4], mj[4];
    const int32_t* ypi[4];
    const float* ypf[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int v = c0 + (b < nb ? b : 0);
      mj[b] = v < b1 ? 0 : (v < b2 ? 1 : 2);
      jj[b] = cs.cand[mj[b]][v - (mj[b] == 0 ? 0 : (mj[b] == 1 ? b1 : b2))];
      ypi[b] = static_cast<const int32_t*>(yv) + int64_t(mj[b]) * P + jj[b];
      ypf[b] = static_cast<const float*>(yv) + int64_t(mj[b]) * P + jj[b];
    }
    double v[4] = {0.0, 0.0, 0.0, 0.0};   // thread 0's: the sums it compares
    // loads for four indices i per thread go out before any is used
    constexpr int kU = 4;
    if (exact_int) {
      long long acc[4] = {0, 0, 0, 0};
      for (int i0 = tid; i0 < K; i0 += kU * kCorrThreads) {
        float tv[kU];
        int yw[kU][4];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int i = i0 + u * kCorrThreads;
          tv[u] = i < K ? __ldg(&t[i]) : 0.f;
#pragma unroll
          for (int b = 0; b < 4; ++b) yw[u][b] = i < K ? ypi[b][i] : 0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const long long ti = __float2int_rn(tv[u]);
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[b] += ti * yw[u][b];
        }
      }
      block_sum4(acc, redl4);
      if (tid == 0)
#pragma unroll
        for (int b = 0; b < 4; ++b) v[b] = double(acc[b]);
    } else {
      DF df[4];
      for (int i0 = tid; i0 < K; i0 += kU * kCorrThreads) {
        float tv[kU], yw[kU][4];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int i = i0 + u * kCorrThreads;
          tv[u] = i < K ? __ldg(&t[i]) : 0.f;
#pragma unroll
          for (int b = 0; b < 4; ++b) yw[u][b] = i < K ? (ints ? float(ypi[b][i]) : ypf[b][i]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
#pragma unroll
          for (int b = 0; b < 4; ++b) df[b].add_prod(tv[u], yw[u][b]);
      }
      block_sum_df<kWarps>(df, redf4);
      if (tid == 0)
#pragma unroll
        for (int b = 0; b < 4; ++b) v[b] = df[b].value();
    }
    if (tid == 0) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (b >= nb) continue;
        if (mj[b] == 0) betterd(bvj[0], bij[0], v[b], jj[b]);
        else if (mj[b] == 1) betterd(bvj[1], bij[1], v[b], jj[b]);
        else betterd(bvj[2], bij[2], v[b], jj[b]);
      }
    }
  }
  if (tid == 0) {
    for (int j = 0; j < Q.nmod; ++j) {
      if (nlist[j] == 0) continue;
      s_m[j] = int(j == 0 ? bij[0] : (j == 1 ? bij[1] : bij[2]));
      s_r[j] = j == 0 ? bvj[0] : (j == 1 ? bvj[1] : bvj[2]);
    }
  }
  __syncthreads();
  for (int j = 0; j < Q.nmod; ++j) {
    if (cs.ncand[j] <= kCandCap) continue;
    // more candidates than the list holds: every index, one per warp
    const int32_t* yi = static_cast<const int32_t*>(yv) + int64_t(j) * P;
    const float* yf = static_cast<const float*>(yv) + int64_t(j) * P;
    const int M = Q.M[j];
    double wv = -INFINITY;
    int64_t wi = 0x7fffffffffffffffll;
    for (int c = warp; c < M; c += kWarps) {
      double v;
      if (ints) v = warp_dot(t, K, exact_int, small, [&](int i) { return yi[c + i]; });
      else v = warp_dot(t, K, false, false, [&](int i) { return yf[c + i]; });
      betterd(wv, wi, v, c);
    }
    if (lane == 0) { wbest_v[warp] = wv; wbest_i[warp] = wi; }
    __syncthreads();
    if (tid == 0) {
      double v = wbest_v[0];
      int64_t i = wbest_i[0];
      for (int w = 1; w < kWarps; ++w) betterd(v, i, wbest_v[w], wbest_i[w]);
      s_m[j] = int(i);
      s_r[j] = v;
      s_flags |= TM_RF_FULL_RESCORE;
    }
    __syncthreads();
  }

  // ------------------------------------------------ e. steps 8-9
  CrtSet crt;
  if (Q.nmod == 3) {
    const int64_t Ms[3] = {Q.M[0], Q.M[1], Q.M[2]}, ms[3] = {s_m[0], s_m[1], s_m[2]};
    crt = crt_intersect3(N, Ms, Q.inv, Q.inv3, ms);
  } else {
    crt = crt_intersect_L(N, Q.M[0], Q.M[1], Q.L[0], Q.L[1], Q.inv, s_m[0], s_m[1]);
  }
  if (Q.thm2) crt.nw = 0;   // wrapped members fall in the zero padding
  const int64_t ncs = crt.nnat + crt.nw;
  auto member = [&](int64_t c) -> int64_t { return c < crt.nnat ? crt.m0 + c * crt.step : crt.w[c - crt.nnat]; };
  double best_v = 0.0;
  int64_t best_m = -1;
  const bool have_x = Q.x != nullptr;
  if (!have_x) {
    // folds without the signal: the member(s) are reported unscored
    best_m = ncs > 0 ? member(0) : -1;
  } else if (ncs == 1) {
    // a single member: its exact (Tx)_m, spread over the whole block
    const int64_t mm = member(0);
    if (exact_int) {
      long long acc = 0;
      for (int i = tid; i < K; i += kCorrThreads) {
        int64_t n = mm + i;
        if (n >= N) n -= N;
        acc += (long long)__float2int_rn(t[i]) * sig.ival(n);
      }
      best_v = double(block_sum(acc, redl));
    } else {
      DF df;
      for (int i = tid; i < K; i += kCorrThreads) {
        int64_t n = mm + i;
        if (n >= N) n -= N;
        df.add_prod(t[i], sig.val(n));
      }
      DF s[1] = {df};
      block_sum_df<kWarps>(s, redf2);
      best_v = tid == 0 ? s[0].value() : 0.0;   // thread 0 writes the result
    }
    best_m = mm;
  } else if (ncs > 1) {
    double wv = -INFINITY;
    int64_t wi = 0x7fffffffffffffffll;
    for (int64_t c = warp; c < ncs; c += kWarps) {
      const int64_t mm = member(c);
      const double v = warp_dot(t, K, exact_int, false, [&](int i) {
        int64_t n = mm + i;
        if (n >= N) n -= N;
        return ints ? double(sig.ival(n)) : double(sig.val(n));
      });
      betterd(wv, wi, v, mm);
    }
    if (lane == 0) { wbest_v[warp] = wv; wbest_i[warp] = wi; }
    __syncthreads();
    best_v = wbest_v[0];
    best_m = wbest_i[0];
    for (int w = 1; w < kWarps; ++w) betterd(best_v, best_m, wbest_v[w], wbest_i[w]);
  }
  if (tid == 0) {
    tm_result res;
    res.n_cand = int32_t(ncs > 0x7fffffff ? 0x7fffffff : ncs);
    if (ncs == 0) { res.shift = -1; res.status = TM_EMPTY; res.score = 0.0; }
    else { res.shift = best_m; res.status = ncs == 1 ? TM_FOUND : TM_RESOLVED; res.score = best_v; }
    res.status |= s_flags;
    if (!have_x && ncs > 0) res.status |= TM_RF_SCORE_PENDING;
    if (*a.err) res.status |= TM_RF_DEVICE_ERROR;
    res.m1 = s_m[0];
    res.m2 = s_m[1];
    res.r1 = s_r[0];
    res.r2 = s_r[1];
    res.m3 = s_m[2];
    res.reserved = 0;
    res.r3 = s_r[2];
    a.out[qi] = res;
  }
}

// Steps 7-9 for two moduli whose FFT values are all available at once
// (rval(j, k) = r~_j[k]).
template <class RFn>
__device__ void select_and_resolve(const CorrArgs& a, const CorrQ& Q, int qi, float delta, bool t_integral, float t1,
                                   int maxy, RFn rval) {
  __shared__ Cands cs;
  collect_candidates(cs, 0, Q.M[0], delta, [&](int k) { return rval(0, k); });
  collect_candidates(cs, 1, Q.M[1], delta, [&](int k) { return rval(1, k); });
  resolve(a, Q, qi, t_integral, t1, maxy, cs);
}

// Steps 3 (completion) to 9 for query qi. The twiddle table and the pass
// tables are loaded only when logP differs from the previous query's
// (loaded_logP).
template <int NBMAX>
__device__ __forceinline__ void corr_query(const CorrArgs& a, int qi, float2* sbuf, int& loaded_logP) {
  __shared__ float redf[2 * kWarps];
  __shared__ long long redl[kWarps];
  __shared__ int redi[kWarps];

  const int tid = threadIdx.x;
  // the descriptor, once per CTA in shared memory (its moduli are indexed at
  // run time: a per-thread copy would sit in local memory)
  __shared__ CorrQ sQ;
  __syncthreads();   // the previous query's readers are done
  if (tid < int(sizeof(CorrQ) / 4))
    reinterpret_cast<int*>(&sQ)[tid] = a.lone >= 0 ? reinterpret_cast<const int*>(&a.q1)[tid]
                                                    : reinterpret_cast<const int*>(a.q + qi)[tid];
  __syncthreads();
  const CorrQ& Q = sQ;
  const int P = Q.P, logP = Q.logP, K = Q.K;
  const int64_t N = Q.N;
  const Sig sig{Q.x, Q.xdtype};
  if (Q.y_in == nullptr && Q.y_core == nullptr && !Q.thm2 && Q.x != nullptr) {
    // the signal entries of the wrap-around and extension terms (part b):
    // x_n for n < max(K-1, w_j) and n in [w_j, w_j + K - 1), w_j = L_j M_j - N
    int64_t lo = K - 1;
    for (int j = 0; j < Q.nmod; ++j) {
      const int64_t w = Q.L[j] * Q.M[j] - N;
      lo = max(lo, w);
      prefetch_elems(Q.x, Q.xdtype, w, min(N, w + K - 1));
    }
    prefetch_elems(Q.x, Q.xdtype, 0, min(N, lo));
  }
  const bool ints = is_int_dtype(Q.xdtype);
  const float* __restrict__ t = Q.t;
  const int npad = P + (P >> 4);
  const int halfP = P >> 1;
  float2* tw = sbuf + npad;   // W_P^m, m < P/2
  // pass tables at the end of the launch's shared memory
  float2* stw = reinterpret_cast<float2*>(reinterpret_cast<char*>(sbuf) + a.smem_bytes) - kPassTw;

  // ------------------------------------------------ twiddles, a. template spectrum
  // Twiddles, pass tables and the template are independent loads: the
  // template's (this thread's entries k = tid + b 512, kept in registers)
  // go out first, then the twiddles' in batches, before any is stored.
  constexpr int kTB = 8;
  constexpr int kTper = (NBMAX == 1 ? kPMax / 2 : kPMax) / kCorrThreads;   // P / 512 at most
  float tv[kTper];
#pragma unroll
  for (int b = 0; b < kTper; ++b) {
    const int k = tid + b * kCorrThreads;
    tv[b] = k < K ? __ldg(&t[k]) : 0.f;
  }
  if (logP != loaded_logP) {
    loaded_logP = logP;
    const int stride = kPMax >> logP;
    for (int m0 = tid; m0 < halfP; m0 += kTB * kCorrThreads) {
      float2 v[kTB];
#pragma unroll
      for (int b = 0; b < kTB; ++b) {
        const int m = m0 + b * kCorrThreads;
        v[b] = m < halfP ? __ldg(&a.tw[m * stride]) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int b = 0; b < kTB; ++b)
        if (m0 + b * kCorrThreads < halfP) tw[m0 + b * kCorrThreads] = v[b];
    }
    build_pass_twiddles(stw, logP, a.tw);
  }
  float t1 = 0.f, t2 = 0.f;
  int tint = 1;
  // the padded template (the padding slots of sbuf are never read), or for
  // P = 8192 and 16384 the FFT's first pass of it
#pragma unroll
  for (int b = 0; b < kTper; ++b) {
    t1 += fabsf(tv[b]);
    t2 = fmaf(tv[b], tv[b], t2);
    tint &= (tv[b] == rintf(tv[b]) && fabsf(tv[b]) <= 1048576.f) ? 1 : 0;
  }
  const bool fuse_t = first_pass_in_regs(logP);
  if (fuse_t) {
    float2 x[kTper];
#pragma unroll
    for (int b = 0; b < kTper; ++b) x[b] = make_float2(tv[b], 0.f);
    first_pass_regs(sbuf, logP, x);
  } else {
#pragma unroll
    for (int b = 0; b < kTper; ++b) {
      const int k = tid + b * kCorrThreads;
      if (k < P) sbuf[pad_idx(k)] = make_float2(tv[b], 0.f);
    }
  }
  block_sum2_and(t1, t2, tint, redf, redi);   // also orders the writes above
  t2 = sqrtf(t2);
  const bool t_integral = tint != 0;
  fft<NBMAX>(sbuf, logP, tw, stw, fuse_t);
  // the spectrum stays in shared memory when the launch left room for it
  float2* spec = (npad + halfP + P + kPassTw) * int(sizeof(float2)) <= a.smem_bytes ? tw + halfP
                                                                                   : a.spec + Q.spec_off;
  float tc2 = 0.f;
  for (int k = tid; k < P; k += kCorrThreads) {
    const float2 T = sbuf[pad_idx(k)];
    spec[k] = T;
    tc2 = fmaxf(tc2, fmaf(T.x, T.x, T.y * T.y));
  }
  const float Tp = spectrum_max_bound(sqrtf(block_maxf(tc2, redf)), logP, t2);
  // everything above reads only the template; the folds come from the
  // kernel before this one (a programmatic dependent launch starts early)
  pdl_acquire();

  // ------------------------------------------------ b-d, per pass: the first
  // pass carries M1 (real part) and M2 (imaginary part) through one complex
  // FFT pipeline, a second pass (three moduli) carries M3
  __shared__ Cands cands;
  int maxy_all = 0;
  auto run_pass = [&](const int pass) {
  // ------------------------------------------------ b. folds
  // Loads are issued in batches (kB per thread) before their results are
  // used, so each pass waits for about one memory round trip.
  constexpr int kB = 8;
  int* ib = reinterpret_cast<int*>(sbuf);     // int view: entry e -> ib[2e] (M1), ib[2e+1] (M2)
  float* fb = reinterpret_cast<float*>(sbuf);
  if (Q.y_in != nullptr) {
    // complete folds supplied by the caller (e.g. summed slice folds)
    const int32_t* yin = static_cast<const int32_t*>(Q.y_in);
    for (int k = tid; k < P; k += kCorrThreads) {
      ib[2 * pad_idx(k)] = yin[k];           // int32 or float bits alike
      ib[2 * pad_idx(k) + 1] = yin[P + k];
    }
  } else {
    // +-1 signals: the slots are summed and turned into fold values in one
    // pass over the columns, which writes every entry k < M_j (no zeroing
    // of them first)
    const int ma = pass == 0 ? 0 : 2, mb = pass == 0 ? 1 : -1;   // moduli in complex slots 0, 1
    const bool fused = ints && Q.y_core == nullptr;
    if (fused) {
      // zero what no fold value writes: k >= M_j (the extension then
      // overwrites [M_j, M_j + K - 1) after a barrier), all of a slot
      // without a modulus
      const int Ma = Q.M[ma], Mb = mb >= 0 ? Q.M[mb] : 0;
      for (int k = tid; k < P; k += kCorrThreads) {
        if (k >= Ma) ib[2 * pad_idx(k)] = 0;
        if (k >= Mb) ib[2 * pad_idx(k) + 1] = 0;
      }
    } else {
      for (int k = tid; k < npad; k += kCorrThreads) sbuf[k] = make_float2(0.f, 0.f);
      __syncthreads();
    }
    if (Q.y_core != nullptr) {
      // the folds over k < M_j from a cache of this signal's folds (int32 or
      // float bits alike)
      const int32_t* yc = static_cast<const int32_t*>(Q.y_core);
      for (int j = 0; j < 2; ++j) {
        const int mj = pass == 0 ? j : (j == 0 ? 2 : -1);
        if (mj < 0) continue;
        for (int k = tid; k < Q.M[mj]; k += kCorrThreads) ib[2 * pad_idx(k) + j] = yc[int64_t(mj) * Q.core_pitch + k];
      }
    } else if (fused) {
      // column k of the M-fold: its slot counts c (of -1 entries for int8,
      // +1 entries for bits) over the nk rows that reach it give the fold
      // value nk - 2c (int8) or 2c - nk (bits); k >= Rw (the last row is
      // short) also takes the wrap-around entry x_{k-Rw}. Slot rows are
      // padded to 16 columns, so a quad read at k < M stays inside the row.
      const bool ones = Q.xdtype == TM_BITS_PM1;
      for (int j = 0; j < 2; ++j) {
        const int mj = j == 0 ? ma : mb;
        if (mj < 0) continue;
        const int M = Q.M[mj], Rr = Q.R[mj];
        const int L = int(Q.L[mj]);
        const int Rw = int(N - int64_t(L - 1) * M);   // length of the last (partial) row, 1..M
        const int32_t* part = a.partial + Q.part + Q.moff[mj];
        const int nq4 = (M + 3) >> 2;
        if (Rr == 1) {
          with_sig(Q.xdtype, Q.x, [&](auto sx) {
            for (int q0 = tid; q0 < nq4; q0 += 4 * kCorrThreads) {
              float xw[4][4];
#pragma unroll
              for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  const int k = 4 * (q0 + b * kCorrThreads) + i;
                  xw[b][i] = (k < M && k >= Rw && !Q.thm2) ? sx.val(k - Rw) : 0.f;
                }
              int4 c[4];
#pragma unroll
              for (int b = 0; b < 4; ++b) c[b] = make_int4(0, 0, 0, 0);
#pragma unroll 2
              for (int sl = 0; sl < Q.nslots; ++sl) {
                const int32_t* ps = part + int64_t(sl) * Q.stride;
                int4 v[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                  const int q = q0 + b * kCorrThreads;
                  v[b] = q < nq4 ? __ldg(reinterpret_cast<const int4*>(ps) + q) : make_int4(0, 0, 0, 0);
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                  c[b].x += v[b].x; c[b].y += v[b].y; c[b].z += v[b].z; c[b].w += v[b].w;
                }
              }
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                const int cc[4] = {c[b].x, c[b].y, c[b].z, c[b].w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  const int k = 4 * (q0 + b * kCorrThreads) + i;
                  if (k < M) {
                    const int nk = L - 1 + (k < Rw ? 1 : 0);
                    ib[2 * pad_idx(k) + j] = (ones ? 2 * cc[i] - nk : nk - 2 * cc[i]) + int(xw[b][i]);
                  }
                }
              }
            }
          });
        } else {
          // column k gathers the counts at k + r M, r < R, of every slot:
          // kC columns per thread, their (slot, replica) terms eight at a
          // time, all loads of a batch issued before any is added (no
          // shared-memory atomics on the R replicas of a column)
          constexpr int kC = 4, kT = 8;
          const int nt = Q.nslots * Rr;
          with_sig(Q.xdtype, Q.x, [&](auto sx) {
            for (int k0 = tid; k0 < M; k0 += kC * kCorrThreads) {
              float xw[kC];
              int c[kC];
#pragma unroll
              for (int b = 0; b < kC; ++b) {
                const int k = k0 + b * kCorrThreads;
                xw[b] = (k < M && k >= Rw && !Q.thm2) ? sx.val(k - Rw) : 0.f;
                c[b] = 0;
              }
              int sl = 0, r = 0;
              for (int t0 = 0; t0 < nt; t0 += kT) {
                int v[kT][kC];
#pragma unroll
                for (int u = 0; u < kT; ++u) {
                  const int32_t* ps = part + int64_t(sl) * Q.stride + r * M;
#pragma unroll
                  for (int b = 0; b < kC; ++b) {
                    const int k = k0 + b * kCorrThreads;
                    v[u][b] = (t0 + u < nt && k < M) ? __ldg(&ps[k]) : 0;
                  }
                  if (++r == Rr) { r = 0; ++sl; }
                }
#pragma unroll
                for (int u = 0; u < kT; ++u)
#pragma unroll
                  for (int b = 0; b < kC; ++b) c[b] += v[u][b];
              }
#pragma unroll
              for (int b = 0; b < kC; ++b) {
                const int k = k0 + b * kCorrThreads;
                if (k < M) {
                  const int nk = L - 1 + (k < Rw ? 1 : 0);
                  ib[2 * pad_idx(k) + j] = (ones ? 2 * c[b] - nk : nk - 2 * c[b]) + int(xw[b]);
                }
              }
            }
          });
        }
      }
    } else {
      // partial slots hold fp32 column sums, added in a fixed order
      for (int j = 0; j < 2; ++j) {
      const int mj = pass == 0 ? j : (j == 0 ? 2 : -1);   // modulus in complex slot j
      if (mj < 0) continue;
        const int M = Q.M[mj], Rr = Q.R[mj];
        const int L = int(Q.L[mj]);
        const int Rw = int(N - int64_t(L - 1) * M);
        const float* pf = reinterpret_cast<const float*>(a.partial + Q.part + Q.moff[mj]);
        for (int k0 = tid; k0 < M; k0 += kB * kCorrThreads) {
          float acc[kB];
          with_sig(Q.xdtype, Q.x, [&](auto sx) {
#pragma unroll
            for (int b = 0; b < kB; ++b) {
              const int k = k0 + b * kCorrThreads;
              acc[b] = (k < M && k >= Rw && !Q.thm2) ? sx.val(k - Rw) : 0.f;
            }
          });
          float yk[kB];
#pragma unroll
          for (int b = 0; b < kB; ++b) yk[b] = 0.f;
          // the terms (slot sl, replica r) in the order t = sl Rr + r,
          // loaded four at a time before they are added in that order
          const int nsr = Q.nslots * Rr;
          int sl = 0, r = 0;
          for (int t0 = 0; t0 < nsr; t0 += 4) {
            float v[4][kB];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float* ps = pf + int64_t(sl) * Q.stride + r * M;
#pragma unroll
              for (int b = 0; b < kB; ++b) {
                const int k = k0 + b * kCorrThreads;
                v[u][b] = (t0 + u < nsr && k < M) ? __ldg(&ps[k]) : 0.f;
              }
              if (++r == Rr) { r = 0; ++sl; }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (t0 + u < nsr) {
#pragma unroll
                for (int b = 0; b < kB; ++b) yk[b] += v[u][b];
              }
            }
          }
#pragma unroll
          for (int b = 0; b < kB; ++b) {
            const int k = k0 + b * kCorrThreads;
            if (k < M) fb[2 * pad_idx(k) + j] = yk[b] + acc[b];
          }
        }
      }
    }
    __syncthreads();
    if (Q.y_core == nullptr) {
      // the entries after the fold kernel's 16-byte blocks (fewer than 16
      // bytes' worth); the count L or L-1 above includes each of them: as +1
      // for int8 (counted -1 entries), as -1 for bits (counted +1 entries).
      // Consecutive entries fall in distinct columns when there are no
      // more of them than columns: one thread each, else thread 0 in order.
      const int ntail = int(N - Q.nelem16);
      const bool spread = ntail <= Q.M[ma] && (mb < 0 || ntail <= Q.M[mb]);
      auto tail = [&](int64_t n) {
        for (int j = 0; j < 2; ++j) {
          const int mj = j == 0 ? ma : mb;   // modulus in complex slot j
          if (mj < 0) continue;
          const int e = 2 * pad_idx(int(n % Q.M[mj])) + j;
          if (Q.xdtype == TM_I8_PM1) ib[e] -= sig.ival(n) < 0 ? 2 : 0;
          else if (Q.xdtype == TM_BITS_PM1) ib[e] += sig.ival(n) > 0 ? 2 : 0;
          else fb[e] += sig.val(n);
        }
      };
      if (spread) {
        if (tid < ntail) tail(Q.nelem16 + tid);
      } else if (tid == 0) {
        for (int64_t n = Q.nelem16; n < N; ++n) tail(n);
      }
    }
    __syncthreads();
    // extension y[M+i] = y[i] - x_i + x_{(i+LM) mod N}, i < K-1, both
    // complex slots at once (x_i is shared)
    {
      const int m0 = pass == 0 ? 0 : 2, m1 = pass == 0 ? 1 : -1;   // moduli in complex slots 0, 1
      const int M0 = Q.M[m0], M1 = m1 >= 0 ? Q.M[m1] : 0;
      const int64_t LM0 = Q.L[m0] * M0, LM1 = m1 >= 0 ? Q.L[m1] * M1 : 0;
      for (int i0 = tid; i0 < K - 1; i0 += kB * kCorrThreads) {
        float xi[kB], xw0[kB], xw1[kB];
        with_sig(Q.xdtype, Q.x, [&](auto sx) {
#pragma unroll
          for (int b = 0; b < kB; ++b) {
            const int i = i0 + b * kCorrThreads;
            xi[b] = xw0[b] = xw1[b] = 0.f;
            if (i < K - 1 && !Q.thm2) {   // Thm. 2: periodic, y[M+i] = y[i]
              int64_t w0 = i + LM0 - N;   // LM >= N and i + LM - N < 2M, so one reduction is rare
              if (w0 >= N) w0 %= N;
              xi[b] = sx.val(i);
              xw0[b] = sx.val(w0);
              if (m1 >= 0) {
                int64_t w1 = i + LM1 - N;
                if (w1 >= N) w1 %= N;
                xw1[b] = sx.val(w1);
              }
            }
          }
        });
#pragma unroll
        for (int b = 0; b < kB; ++b) {
          const int i = i0 + b * kCorrThreads;
          if (i < K - 1) {
            const int e = 2 * pad_idx(M0 + i), ee = 2 * pad_idx(i);
            if (ints) ib[e] = ib[ee] - int(xi[b]) + int(xw0[b]);
            else fb[e] = fb[ee] - xi[b] + xw0[b];
            if (m1 >= 0) {
              const int e1 = 2 * pad_idx(M1 + i) + 1;
              if (ints) ib[e1] = ib[ee + 1] - int(xi[b]) + int(xw1[b]);
              else fb[e1] = fb[ee + 1] - xi[b] + xw1[b];
            }
          }
        }
      }
    }
  }
  __syncthreads();
  // export exact folds, convert to float, norms of z (exact integers for +-1
  // signals; fp32 sums for reals)
  float z2 = 0.f;
  int maxy = 0;
  // P = 8192 (one radix-16 butterfly per thread and pass): z and, below,
  // T conj(Z) are kept in registers and written as the FFT's first pass
  constexpr int kZper = kPMax / 2 / kCorrThreads;   // 16
  const bool fuse_z = NBMAX == 1 && logP == 13;
  float2 zr[kZper];
  if (ints) {
    long long s2 = 0;
    int32_t* yi = static_cast<int32_t*>(a.y) + Q.y_off;
    if (fuse_z) {
#pragma unroll
      for (int b = 0; b < kZper; ++b) {
        const int k = tid + b * kCorrThreads;
        const int e = 2 * pad_idx(k);
        const int v0 = ib[e], v1 = ib[e + 1];
        if (Q.y_in == nullptr) {
          yi[(pass == 0 ? 0 : 2) * P + k] = v0;
          if (pass == 0) yi[P + k] = v1;
        }
        zr[b] = make_float2(float(v0), float(v1));
        s2 += (long long)v0 * v0 + (long long)v1 * v1;
        maxy = max(maxy, max(abs(v0), abs(v1)));
      }
    } else {
      for (int k = tid; k < P; k += kCorrThreads) {
        const int e = 2 * pad_idx(k);
        const int v0 = ib[e], v1 = ib[e + 1];
        if (Q.y_in == nullptr) {
          yi[(pass == 0 ? 0 : 2) * P + k] = v0;
          if (pass == 0) yi[P + k] = v1;
        }
        sbuf[pad_idx(k)] = make_float2(float(v0), float(v1));
        s2 += (long long)v0 * v0 + (long long)v1 * v1;
        maxy = max(maxy, max(abs(v0), abs(v1)));
      }
    }
    s2 = block_sum(s2, redl);
    z2 = sqrtf(float(s2));
    maxy = block_max(maxy, redi);
  } else {
    float* yf = static_cast<float*>(a.y) + Q.y_off;
    if (fuse_z) {
#pragma unroll
      for (int b = 0; b < kZper; ++b) {
        const int k = tid + b * kCorrThreads;
        const float2 v = sbuf[pad_idx(k)];
        if (Q.y_in == nullptr) {
          yf[(pass == 0 ? 0 : 2) * P + k] = v.x;
          if (pass == 0) yf[P + k] = v.y;
        }
        z2 = fmaf(v.x, v.x, fmaf(v.y, v.y, z2));
        zr[b] = v;
      }
    } else {
      for (int k = tid; k < P; k += kCorrThreads) {
        const float2 v = sbuf[pad_idx(k)];
        if (Q.y_in == nullptr) {
          yf[(pass == 0 ? 0 : 2) * P + k] = v.x;
          if (pass == 0) yf[P + k] = v.y;
        }
        z2 = fmaf(v.x, v.x, fmaf(v.y, v.y, z2));
      }
    }
    z2 = sqrtf(block_sum(z2, redf));
  }

  // ------------------------------------------------ c. correlation by FFT
  if (fuse_z) {
    first_pass_regs(sbuf, logP, zr);   // every read of sbuf above precedes the block sums' barriers
    __syncthreads();
  }
  fft<NBMAX>(sbuf, logP, tw, stw, fuse_z);
  float zc2 = 0.f;
  if (fuse_z) {
#pragma unroll
    for (int b = 0; b < kZper; ++b) {
      const int k = tid + b * kCorrThreads;
      const float2 z = sbuf[pad_idx(k)], T = spec[k];
      zc2 = fmaxf(zc2, fmaf(z.x, z.x, z.y * z.y));
      zr[b] = make_float2(T.x * z.x + T.y * z.y, T.y * z.x - T.x * z.y);   // T conj(Z)
    }
  } else {
    for (int k = tid; k < P; k += kCorrThreads) {
      const float2 z = sbuf[pad_idx(k)], T = spec[k];
      zc2 = fmaxf(zc2, fmaf(z.x, z.x, z.y * z.y));
      sbuf[pad_idx(k)] = make_float2(T.x * z.x + T.y * z.y, T.y * z.x - T.x * z.y);   // T conj(Z)
    }
  }
  const float Zc = 1.0001f * sqrtf(block_maxf(zc2, redf));   // block_maxf also orders the writes above
  if (fuse_z) {
    first_pass_regs(sbuf, logP, zr);   // the reads of sbuf above precede block_maxf's barriers
    __syncthreads();
  }
  fft<NBMAX>(sbuf, logP, tw, stw, fuse_z);
  const float invP = 1.0f / float(P);   // exact: P is a power of two

  if (a.r != nullptr && Q.r_off >= 0) {
    float* r = a.r + Q.r_off;
    if (pass == 0) {
      for (int k = tid; k < Q.M[0]; k += kCorrThreads) r[k] = sbuf[pad_idx(k)].x * invP;
      for (int k = tid; k < Q.M[1]; k += kCorrThreads) r[P + k] = -sbuf[pad_idx(k)].y * invP;
    } else {
      for (int k = tid; k < Q.M[2]; k += kCorrThreads) r[2 * P + k] = sbuf[pad_idx(k)].x * invP;
    }
  }

  // ------------------------------------------------ d. step 7 candidates
  // Rounding bound on every r_j (fft_corr_error_bound, one product term).
  const float delta = fft_corr_error_bound(logP, t2, Tp, Zc, z2, 1);
  if (pass == 0) {
    collect_candidates2(cands, Q.M[0], Q.M[1], delta, [&](int k) { return sbuf[pad_idx(k)].x * invP; },
                        [&](int k) { return -sbuf[pad_idx(k)].y * invP; });
  } else {
    collect_candidates(cands, 2, Q.M[2], delta, [&](int k) { return sbuf[pad_idx(k)].x * invP; });
  }
  maxy_all = max(maxy_all, maxy);
  };
  run_pass(0);
  if (Q.nmod == 3) {
    __syncthreads();   // the first pass's values are no longer read
    run_pass(1);
  }
  // ------------------------------------------------ e. steps 7-9
  resolve(a, Q, qi, t_integral, t1, maxy_all, cands);
}

// One CTA per query, in a.order (largest FFT first) from a.first on; the
// hardware hands the next query to whichever SM frees up. (A loop over
// queries inside a CTA was tried: the state it carries across iterations
// pushes this kernel past its 128 registers and into local memory. A
// launch limited to fewer CTAs is therefore cut into waves of launches.)
template <int NBMAX>
__global__ void __launch_bounds__(kCorrThreads, 1) corr_kernel(const CorrArgs a) {
  extern __shared__ __align__(16) float2 sbuf[];
  int loaded_logP = -1;
  corr_query<NBMAX>(a, a.lone >= 0 ? a.lone : a.order[a.first + blockIdx.x], sbuf, loaded_logP);
}

// ---------------------------------------------------------------- blocked correlation
// For max(M)+K-1 > 16384 the correlation is cut into blocks of B = 8192
// (overlap-save): with t_b = t[bB, bB+B), the y-segments seg_s = y[sB, sB+2B)
// and output blocks j = aB + jj, jj < B,
//   r_j = sum_b sum_{ii<B} t_b[ii] seg_{a+b}[jj + ii],
// a linear correlation of length-2B arrays that a 2B-point FFT computes
// without wrap-around. All spectra go to global scratch: T_b (b < Bt), Z_s
// (s < A+Bt-1, z = y_1 + i y_2 as above); block a is the inverse transform
// of sum_b T_b conj(Z_{a+b}). The folds are built straight into global memory.
constexpr int kBlk = 8192;
constexpr int kBlkLog = 14;   // FFT length 2 kBlk

__global__ void __launch_bounds__(kCorrThreads, 1) corr_blocked_kernel(const CorrArgs a) {
  extern __shared__ __align__(16) float2 sbuf[];
  __shared__ float redf[kWarps];
  __shared__ long long redl[kWarps];
  __shared__ int redi[kWarps];

  const int tid = threadIdx.x;
  const int qi = a.order[blockIdx.x];
  __shared__ CorrQ sQ;   // the descriptor, once per CTA
  if (tid < int(sizeof(CorrQ) / 4)) reinterpret_cast<int*>(&sQ)[tid] = reinterpret_cast<const int*>(a.q + qi)[tid];
  __syncthreads();
  const CorrQ& Q = sQ;
  const int P = Q.P, K = Q.K;
  const int64_t N = Q.N;
  const Sig sig{Q.x, Q.xdtype};
  const bool ints = is_int_dtype(Q.xdtype);
  const float* __restrict__ t = Q.t;
  constexpr int PB = 2 * kBlk;
  constexpr int npad = PB + (PB >> 4);
  float2* tw = sbuf + npad;   // W_PB^m, m < PB/2
  const int Bt = (K + kBlk - 1) / kBlk;
  const int A = (max(Q.M[0], Q.M[1]) + kBlk - 1) / kBlk;
  const int S = A + Bt - 1;
  float2* spec = a.spec + Q.spec_off;   // [Bt + S][PB]
  float* rb = a.r + Q.r_off;            // [2][P]: r_1 then r_2
  float2* stw = reinterpret_cast<float2*>(reinterpret_cast<char*>(sbuf) + a.smem_bytes) - kPassTw;

  {
    const int stride = kPMax >> kBlkLog;
    for (int m = tid; m < PB / 2; m += kCorrThreads) tw[m] = __ldg(&a.tw[m * stride]);
    build_pass_twiddles(stw, kBlkLog, a.tw);
  }
  // template norms
  float t1 = 0.f, t2 = 0.f;
  int tint = 1;
  for (int k = tid; k < K; k += kCorrThreads) {
    const float v = t[k];
    t1 += fabsf(v);
    t2 = fmaf(v, v, t2);
    tint &= (v == rintf(v) && fabsf(v) <= 1048576.f) ? 1 : 0;
  }
  t1 = block_sum(t1, redf);
  t2 = sqrtf(block_sum(t2, redf));
  const bool t_integral = block_and(tint, redi) != 0;

  // ------------------------------------------------ folds, straight to global memory
  int32_t* yi = static_cast<int32_t*>(a.y) + Q.y_off;
  float* yf = static_cast<float*>(a.y) + Q.y_off;
  if (Q.y_in == nullptr) {   // else the folds are given, complete, at y_off
    for (int j = 0; j < 2; ++j) {
      const int M = Q.M[j], Rr = Q.R[j];
      const int L = int(Q.L[j]);
      const int Rw = int(N - int64_t(L - 1) * M);
      const int32_t* part = a.partial + Q.part + Q.moff[j];
      for (int k = tid; k < M; k += kCorrThreads) {
        if (ints) {
          int c = 0;
          for (int s = 0; s < Q.nslots; ++s) {
            const int32_t* ps = part + int64_t(s) * Q.stride;
            for (int r = 0; r < Rr; ++r) c += ps[k + r * M];
          }
          const int nk = L - 1 + (k < Rw ? 1 : 0);
          int yk = Q.xdtype == TM_BITS_PM1 ? 2 * c - nk : nk - 2 * c;
          if (k >= Rw && !Q.thm2) yk += sig.ival(k - Rw);
          yi[int64_t(j) * P + k] = yk;
        } else {
          const float* pf = reinterpret_cast<const float*>(part);
          float yk = 0.f;
          for (int s = 0; s < Q.nslots; ++s) {
            const float* ps = pf + int64_t(s) * Q.stride;
            for (int r = 0; r < Rr; ++r) yk += ps[k + r * M];
          }
          if (k >= Rw && !Q.thm2) yk += sig.val(k - Rw);
          yf[int64_t(j) * P + k] = yk;
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      for (int64_t n = Q.nelem16; n < N; ++n) {
        for (int j = 0; j < 2; ++j) {
          const int64_t e = int64_t(j) * P + n % Q.M[j];
          if (Q.xdtype == TM_I8_PM1) yi[e] -= sig.ival(n) < 0 ? 2 : 0;
          else if (Q.xdtype == TM_BITS_PM1) yi[e] += sig.ival(n) > 0 ? 2 : 0;
          else yf[e] += sig.val(n);
        }
      }
    }
    __syncthreads();
    for (int j = 0; j < 2; ++j) {
      const int M = Q.M[j];
      const int64_t LM = Q.L[j] * M;
      for (int i = tid; i < K - 1; i += kCorrThreads) {
        int64_t w = i + LM - N;
        if (w >= N) w %= N;
        const int64_t e = int64_t(j) * P + M + i, e0 = int64_t(j) * P + i;
        if (Q.thm2) {   // periodic extension
          if (ints) yi[e] = yi[e0];
          else yf[e] = yf[e0];
        } else if (ints) {
          yi[e] = yi[e0] - sig.ival(i) + sig.ival(w);
        } else {
          yf[e] = yf[e0] - sig.val(i) + sig.val(w);
        }
      }
    }
    __syncthreads();
  }
  // norms of z = y_1 + i y_2
  auto yval = [&](int j, int64_t k) -> float {
    if (k >= Q.M[j] + K - 1) return 0.f;
    return ints ? float(yi[int64_t(j) * P + k]) : yf[int64_t(j) * P + k];
  };
  float z2 = 0.f;
  int maxy = 0;
  {
    long long s2 = 0;
    float f2 = 0.f;
    for (int j = 0; j < 2; ++j) {
      for (int k = tid; k < Q.M[j] + K - 1; k += kCorrThreads) {
        if (ints) {
          const int v = yi[int64_t(j) * P + k];
          s2 += (long long)v * v;
          maxy = max(maxy, abs(v));
        } else {
          const float v = yf[int64_t(j) * P + k];
          f2 = fmaf(v, v, f2);
        }
      }
    }
    if (ints) {
      s2 = block_sum(s2, redl);
      z2 = sqrtf(float(s2));
      maxy = block_max(maxy, redi);
    } else {
      z2 = sqrtf(block_sum(f2, redf));
    }
  }

  // ------------------------------------------------ spectra of template blocks and signal segments
  float tc2 = 0.f, zc2 = 0.f;   // largest |T~_k|^2, |Z~_k|^2 over all blocks
  for (int b = 0; b < Bt; ++b) {
    for (int k = tid; k < npad; k += kCorrThreads) sbuf[k] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int i = tid; i < kBlk && b * kBlk + i < K; i += kCorrThreads) sbuf[pad_idx(i)].x = t[b * kBlk + i];
    __syncthreads();
    fft<2>(sbuf, kBlkLog, tw, stw);
    for (int k = tid; k < PB; k += kCorrThreads) {
      const float2 T = sbuf[pad_idx(k)];
      spec[int64_t(b) * PB + k] = T;
      tc2 = fmaxf(tc2, fmaf(T.x, T.x, T.y * T.y));
    }
    __syncthreads();
  }
  for (int s = 0; s < S; ++s) {
    for (int i = tid; i < PB; i += kCorrThreads) {
      const int64_t k = int64_t(s) * kBlk + i;
      sbuf[pad_idx(i)] = make_float2(yval(0, k), yval(1, k));
    }
    __syncthreads();
    fft<2>(sbuf, kBlkLog, tw, stw);
    for (int k = tid; k < PB; k += kCorrThreads) {
      const float2 Z = sbuf[pad_idx(k)];
      spec[int64_t(Bt + s) * PB + k] = Z;
      zc2 = fmaxf(zc2, fmaf(Z.x, Z.x, Z.y * Z.y));
    }
    __syncthreads();
  }
  const float Tp = spectrum_max_bound(sqrtf(block_maxf(tc2, redf)), kBlkLog, t2);
  const float Zc = 1.0001f * sqrtf(block_maxf(zc2, redf));
  // ------------------------------------------------ output blocks
  const float invPB = 1.0f / float(PB);
  for (int ab = 0; ab < A; ++ab) {
    for (int k = tid; k < PB; k += kCorrThreads) {
      float2 acc = make_float2(0.f, 0.f);
      for (int b = 0; b < Bt; ++b) {
        const float2 T = spec[int64_t(b) * PB + k], z = spec[int64_t(Bt + ab + b) * PB + k];
        acc.x += T.x * z.x + T.y * z.y;   // T conj(Z)
        acc.y += T.y * z.x - T.x * z.y;
      }
      sbuf[pad_idx(k)] = acc;
    }
    __syncthreads();
    fft<2>(sbuf, kBlkLog, tw, stw);
    for (int i = tid; i < kBlk; i += kCorrThreads) {
      const int jj = ab * kBlk + i;
      const float2 w = sbuf[pad_idx(i)];
      if (jj < Q.M[0]) rb[jj] = w.x * invPB;
      if (jj < Q.M[1]) rb[P + jj] = -w.y * invPB;
    }
    __syncthreads();
  }
  // ------------------------------------------------ steps 7-9
  const float delta = fft_corr_error_bound(kBlkLog, t2, Tp, Zc, z2, Bt);
  select_and_resolve(a, Q, qi, delta, t_integral, t1, maxy,
                     [&](int j, int k) { return rb[int64_t(j) * P + k]; });
}

int corr_blocked_smem_bytes() { return (2 * kBlk + 2 * kBlk / 16 + kBlk + kPassTw) * int(sizeof(float2)); }

// Shared memory of a launch whose largest FFT is P: the padded work buffer,
// the half twiddle table, for P <= 8192 the template spectrum, and the pass
// twiddle tables.
int corr_smem_bytes(int P) {
  return (P + P / 16 + P / 2 + (P <= 8192 ? P : 0) + kPassTw) * int(sizeof(float2));
}

}  // namespace

cudaError_t corr_configure() {
  cudaError_t e = cudaFuncSetAttribute(corr_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       corr_smem_bytes(kPMax / 2));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(corr_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, corr_smem_bytes(kPMax));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(corr_blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              corr_blocked_smem_bytes());
}

cudaError_t launch_correlate(const CorrArgs& a, int32_t maxP, cudaStream_t s) {
  CorrArgs b = a;
  b.smem_bytes = corr_smem_bytes(maxP);
  // at most a.ctas CTAs at a time (so that a concurrent fold keeps its
  // SMs): waves of launches over the order
  const int wave = (a.ctas > 0 && a.ctas < a.nq) ? a.ctas : a.nq;
  for (int f = 0; f < a.nq; f += wave) {
    b.first = a.first + f;
    const int grid = min(wave, a.nq - f);
    // one butterfly of radix 16 per thread and pass up to P = 8192, two above
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t c = launch_config(dim3(grid), dim3(kCorrThreads), size_t(b.smem_bytes), s,
                                               a.pdl != 0 && wave == a.nq, attr);
    const cudaError_t e = maxP <= kPMax / 2 ? cudaLaunchKernelEx(&c, corr_kernel<1>, b)
                                            : cudaLaunchKernelEx(&c, corr_kernel<2>, b);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_correlate_blocked(const CorrArgs& a, cudaStream_t s) {
  CorrArgs b = a;
  b.smem_bytes = corr_blocked_smem_bytes();
  corr_blocked_kernel<<<a.nq, kCorrThreads, b.smem_bytes, s>>>(b);
  return cudaGetLastError();
}

int blocked_spectra(int K, int maxM) {
  const int Bt = (K + kBlk - 1) / kBlk, A = (maxM + kBlk - 1) / kBlk;
  return Bt + A + Bt - 1;
}

}  // namespace ftm
