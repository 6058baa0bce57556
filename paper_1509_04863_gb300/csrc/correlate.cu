// Steps 3 (completion) and 4-9 of Algorithm 1, one CTA per query.
//
//  a. Template spectrum T = FFT_P([t 0]) (steps 4-5), kept in global scratch.
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
//     int64, reals in fp64), which makes the chosen index exact.
//  e. Steps 8-9: closed-form intersection (crt.h); several members are
//     resolved by their exact (Tx)_m.
//
// FFT: Stockham autosort, radix 16 (plus one radix 2/4/8 pass), shared
// memory resident (P <= 16384 complex entries, padded one entry per 16 to
// avoid bank conflicts), twiddles from a table W_{16384}^m computed on the
// host in double precision.
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

// One Stockham pass of radix R over P points whose sub-transforms of length
// Ns are done: butterfly j takes x[j + r P/R], twiddles by W_{Ns R}^{r (j mod Ns)},
// and writes to (j - j mod Ns) R + j mod Ns + r Ns.
template <int R>
__device__ __forceinline__ void fft_pass(float2* buf, int P, int Ns, int twshift, const float2* __restrict__ tw) {
  constexpr int NB = (kPMax / R + kCorrThreads - 1) / kCorrThreads;
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
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], __ldg(&tw[(r * k) << twshift]));
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

// Forward FFT of length 2^logP in place (padded layout, natural order).
__device__ void fft(float2* buf, int logP, const float2* __restrict__ tw) {
  const int P = 1 << logP;
  int logNs = 0;
  const int first = logP & 3;
  if (first) {
    const int twshift = kLogPMax - first;
    if (first == 1) fft_pass<2>(buf, P, 1, twshift, tw);
    else if (first == 2) fft_pass<4>(buf, P, 1, twshift, tw);
    else fft_pass<8>(buf, P, 1, twshift, tw);
    logNs = first;
  }
  while (logNs < logP) {
    fft_pass<16>(buf, P, 1 << logNs, kLogPMax - (logNs + 4), tw);
    logNs += 4;
  }
}

// ---------------------------------------------------------------- block reductions
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s += red[w];
  return s;
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

// max value, smallest index on ties
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

__device__ __forceinline__ void warp_argmaxd(double& v, int64_t& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int64_t i2 = __shfl_xor_sync(0xffffffffu, i, o);
    betterd(v, i, v2, i2);
  }
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
  __device__ __forceinline__ int ival(int64_t n) const { return int(val(n)); }
};

__device__ __forceinline__ bool is_int_dtype(int d) { return d == TM_I8_PM1 || d == TM_BITS_PM1; }

// Exact sum_{i<K} t_i * v(i) over one warp; v integer-valued when `integral`.
template <class F>
__device__ __forceinline__ double warp_dot(const float* __restrict__ t, int K, bool integral, F v) {
  const int lane = threadIdx.x & 31;
  if (integral) {
    long long acc = 0;
    for (int i = lane; i < K; i += 32) acc += (long long)__float2int_rn(t[i]) * (long long)v(i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return double(acc);
  }
  double acc = 0.0;
  for (int i = lane; i < K; i += 32) acc = fma(double(t[i]), double(v(i)), acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

__global__ void __launch_bounds__(kCorrThreads, 1) corr_kernel(const CorrArgs a) {
  extern __shared__ __align__(16) float2 sbuf[];
  __shared__ double red[kWarps];
  __shared__ float redv[kWarps];
  __shared__ int redi[kWarps];
  __shared__ int cand[2][kCandCap];
  __shared__ int ncand[2];
  __shared__ double wbest_v[kWarps];
  __shared__ int64_t wbest_i[kWarps];
  __shared__ int s_m[2];
  __shared__ double s_r[2];
  __shared__ int s_flags;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const CorrQ Q = a.q[a.order[blockIdx.x]];
  const int qi = a.order[blockIdx.x];
  const int P = Q.P, logP = Q.logP, K = Q.K;
  const int64_t N = Q.N;
  const Sig sig{Q.x, Q.xdtype};
  const bool ints = is_int_dtype(Q.xdtype);
  const float* __restrict__ t = Q.t;
  const int npad = P + (P >> 4);
  if (tid == 0) s_flags = 0;

  // ------------------------------------------------ a. template spectrum
  double t1 = 0.0, t2 = 0.0;
  int tint = 1;
  for (int k = tid; k < npad; k += kCorrThreads) sbuf[k] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int k = tid; k < K; k += kCorrThreads) {
    const float v = t[k];
    sbuf[pad_idx(k)] = make_float2(v, 0.f);
    t1 += fabs(double(v));
    t2 += double(v) * double(v);
    tint &= (v == rintf(v) && fabsf(v) <= 1048576.f) ? 1 : 0;
  }
  __syncthreads();
  t1 = block_sum(t1, red);
  t2 = sqrt(block_sum(t2, red));
  const bool t_integral = block_and(tint, redi) != 0;
  fft(sbuf, logP, a.tw);
  float2* spec = a.spec + Q.spec_off;
  for (int k = tid; k < P; k += kCorrThreads) spec[k] = sbuf[pad_idx(k)];
  __syncthreads();

  // ------------------------------------------------ b. folds
  int* ib = reinterpret_cast<int*>(sbuf);     // int view: entry e -> ib[2e] (M1), ib[2e+1] (M2)
  float* fb = reinterpret_cast<float*>(sbuf);
  for (int k = tid; k < 2 * npad; k += kCorrThreads) ib[k] = 0;
  __syncthreads();
  for (int j = 0; j < 2; ++j) {
    const int M = Q.M[j], Rr = Q.R[j];
    const int64_t L = Q.L[j];
    const int64_t Rw = N - (L - 1) * M;    // length of the last (partial) row
    const int32_t* part = a.partial + Q.part + Q.moff[j];
    for (int k = tid; k < M; k += kCorrThreads) {
      if (ints) {
        // partial slots hold counts of -1 entries per column of the Mp-fold
        int neg = 0;
        for (int s = 0; s < Q.nslots; ++s) {
          const int32_t* ps = part + int64_t(s) * Q.stride;
          for (int r = 0; r < Rr; ++r) neg += ps[k + r * M];
        }
        const int64_t nk = (k < N) ? (N - 1 - k) / M + 1 : 0;   // entries n < N, n = k mod M
        int yk = int(nk) - 2 * neg;
        if (k >= Rw) yk += sig.ival(k - Rw);
        ib[2 * pad_idx(k) + j] = yk;
      } else {
        // partial slots hold fp32 column sums, added in a fixed order
        const float* pf = reinterpret_cast<const float*>(part);
        float yk = 0.f;
        for (int s = 0; s < Q.nslots; ++s) {
          const float* ps = pf + int64_t(s) * Q.stride;
          for (int r = 0; r < Rr; ++r) yk += ps[k + r * M];
        }
        if (k >= Rw) yk += sig.val(k - Rw);
        fb[2 * pad_idx(k) + j] = yk;
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int64_t n = Q.nelem16; n < N; ++n) {
      for (int j = 0; j < 2; ++j) {
        const int e = 2 * pad_idx(int(n % Q.M[j])) + j;
        // the count n_k already includes this entry as +1
        if (ints) ib[e] -= sig.ival(n) < 0 ? 2 : 0;
        else fb[e] += sig.val(n);
      }
    }
  }
  __syncthreads();
  for (int j = 0; j < 2; ++j) {
    const int M = Q.M[j];
    const int64_t LM = Q.L[j] * M;
    for (int i = tid; i < K - 1; i += kCorrThreads) {
      const int e = 2 * pad_idx(M + i) + j, e0 = 2 * pad_idx(i) + j;
      if (ints) ib[e] = ib[e0] - sig.ival(i) + sig.ival((i + LM) % N);
      else fb[e] = fb[e0] - sig.val(i) + sig.val((i + LM) % N);
    }
  }
  __syncthreads();
  // export exact folds, convert to float, norms of z
  double z1 = 0.0, z2 = 0.0;
  {
    int32_t* yi = static_cast<int32_t*>(a.y) + Q.y_off;
    float* yf = static_cast<float*>(a.y) + Q.y_off;
    for (int k = tid; k < P; k += kCorrThreads) {
      const int e = 2 * pad_idx(k);
      float v0, v1;
      if (ints) {
        const int i0 = ib[e], i1 = ib[e + 1];
        yi[k] = i0; yi[P + k] = i1;
        v0 = float(i0); v1 = float(i1);
        sbuf[pad_idx(k)] = make_float2(v0, v1);
      } else {
        v0 = fb[e]; v1 = fb[e + 1];
        yf[k] = v0; yf[P + k] = v1;
      }
      z1 += fabs(double(v0)) + fabs(double(v1));
      z2 += double(v0) * v0 + double(v1) * v1;
    }
  }
  z1 = block_sum(z1, red);
  z2 = sqrt(block_sum(z2, red));

  // ------------------------------------------------ c. correlation by FFT
  fft(sbuf, logP, a.tw);
  for (int k = tid; k < P; k += kCorrThreads) {
    const float2 z = sbuf[pad_idx(k)], T = spec[k];
    sbuf[pad_idx(k)] = make_float2(T.x * z.x + T.y * z.y, T.y * z.x - T.x * z.y);   // T conj(Z)
  }
  __syncthreads();
  fft(sbuf, logP, a.tw);
  const float invP = 1.0f / float(P);   // exact: P is a power of two

  if (a.r != nullptr && Q.r_off >= 0) {
    float* r = a.r + Q.r_off;
    for (int k = tid; k < Q.M[0]; k += kCorrThreads) r[k] = sbuf[pad_idx(k)].x * invP;
    for (int k = tid; k < Q.M[1]; k += kCorrThreads) r[P + k] = -sbuf[pad_idx(k)].y * invP;
  }

  // ------------------------------------------------ d. step 7 with exact rescoring
  // Rounding bound (normwise, fp32 unit roundoff u): one length-P FFT has
  // relative 2-norm error <= epsF = 14 u log2 P (the radix-2 bound
  // log2(P) (mu + gamma_4 (sqrt 2 + mu)) with a safety factor of two); with
  // |T_k| <= ||t||_1, |Z_k| <= ||z||_1 and the 1/P scaling of the inverse,
  // max_j |dr_j| <= ||dw||_2 <= epsF (||t||_2 ||z||_1 + 2 ||t||_1 ||z||_2) + 3u ||t||_1 ||z||_2.
  const double u = 5.9604644775390625e-08;
  const double epsF = 14.0 * u * double(logP > 0 ? logP : 1);
  const double delta = epsF * (t2 * z1 + 2.0 * t1 * z2) + 3.0 * u * t1 * z2 + 1e-30;
  const bool exact_int = ints && t_integral;
  const void* yv = static_cast<const char*>(a.y) + Q.y_off * 4;

  for (int j = 0; j < 2; ++j) {
    const int M = Q.M[j];
    float bv = -INFINITY;
    int bi = 0x7fffffff;
    for (int k = tid; k < M; k += kCorrThreads) {
      const float2 w = sbuf[pad_idx(k)];
      better(bv, bi, j == 0 ? w.x * invP : -w.y * invP, k);
    }
    block_argmax(bv, bi, redv, redi);
    if (tid == 0) ncand[j] = 0;
    __syncthreads();
    const float thr = float(double(bv) - 2.0 * delta);
    for (int k = tid; k < M; k += kCorrThreads) {
      const float2 w = sbuf[pad_idx(k)];
      const float rv = j == 0 ? w.x * invP : -w.y * invP;
      if (rv >= thr) {
        const int c = atomicAdd(&ncand[j], 1);
        if (c < kCandCap) cand[j][c] = k;
      }
    }
    __syncthreads();
    const int nc = ncand[j];
    const bool all = nc > kCandCap;
    const int ncheck = all ? M : nc;
    double wv = -INFINITY;
    int64_t wi = 0x7fffffffffffffffll;
    for (int c = warp; c < ncheck; c += kWarps) {
      const int jj = all ? c : cand[j][c];
      double v;
      if (ints) {
        const int32_t* y = static_cast<const int32_t*>(yv) + int64_t(j) * P + jj;
        v = warp_dot(t, K, exact_int, [&](int i) { return y[i]; });
      } else {
        const float* y = static_cast<const float*>(yv) + int64_t(j) * P + jj;
        v = warp_dot(t, K, false, [&](int i) { return y[i]; });
      }
      betterd(wv, wi, v, jj);
    }
    if (lane == 0) { wbest_v[warp] = wv; wbest_i[warp] = wi; }
    __syncthreads();
    if (tid == 0) {
      double v = wbest_v[0];
      int64_t i = wbest_i[0];
      for (int w = 1; w < kWarps; ++w) betterd(v, i, wbest_v[w], wbest_i[w]);
      s_m[j] = int(i);
      s_r[j] = v;
      if (all) s_flags |= TM_RF_FULL_RESCORE;
    }
    __syncthreads();
  }

  // ------------------------------------------------ e. steps 8-9
  const CrtSet cs = crt_intersect(N, Q.M[0], Q.M[1], Q.inv, s_m[0], s_m[1]);
  const int64_t ncs = cs.nnat + cs.nw;
  auto member = [&](int64_t c) -> int64_t { return c < cs.nnat ? cs.m0 + c * cs.step : cs.w[c - cs.nnat]; };
  auto tx = [&](int64_t m) -> double {
    return warp_dot(t, K, exact_int, [&](int i) {
      int64_t n = m + i;
      if (n >= N) n -= N;
      return ints ? double(sig.ival(n)) : double(sig.val(n));
    });
  };
  double wv = -INFINITY;
  int64_t wi = 0x7fffffffffffffffll;
  for (int64_t c = warp; c < ncs; c += kWarps) {
    const int64_t mm = member(c);
    betterd(wv, wi, tx(mm), mm);
  }
  if (lane == 0) { wbest_v[warp] = wv; wbest_i[warp] = wi; }
  __syncthreads();
  if (tid == 0) {
    tm_result res;
    double v = wbest_v[0];
    int64_t i = wbest_i[0];
    for (int w = 1; w < kWarps; ++w) betterd(v, i, wbest_v[w], wbest_i[w]);
    res.n_cand = int32_t(ncs > 0x7fffffff ? 0x7fffffff : ncs);
    if (ncs == 0) { res.shift = -1; res.status = TM_EMPTY; res.score = 0.0; }
    else { res.shift = i; res.status = ncs == 1 ? TM_FOUND : TM_RESOLVED; res.score = v; }
    res.status |= s_flags;
    if (*a.err) res.status |= TM_RF_DEVICE_ERROR;
    res.m1 = s_m[0];
    res.m2 = s_m[1];
    res.r1 = s_r[0];
    res.r2 = s_r[1];
    a.out[qi] = res;
  }
}

}  // namespace

cudaError_t corr_configure() {
  const int smem = (kPMax + kPMax / 16) * int(sizeof(float2));
  return cudaFuncSetAttribute(corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_correlate(const CorrArgs& a, int32_t maxP, cudaStream_t s) {
  const int smem = (maxP + maxP / 16) * int(sizeof(float2));
  corr_kernel<<<a.nq, kCorrThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ftm
