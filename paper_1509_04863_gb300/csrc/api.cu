// Host runtime and C ABI: planning (Algorithm 1 step 2), batch workspaces,
// launches and error reporting. See include/tm.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "crt.h"
#include "device_util.cuh"
#include "runtime.h"

namespace ftm {

namespace {
thread_local std::string g_err;
}  // namespace

std::string& last_error() { return g_err; }

tm_status fail(tm_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

tm_status cuda_fail(cudaError_t e, const char* what) {
  return fail(TM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

int64_t gcd64(int64_t a, int64_t b) {
  while (b) { const int64_t t = a % b; a = b; b = t; }
  return a;
}

// Least s with s (s+1) > N.
int64_t least_s(int64_t N) {
  int64_t s = std::max<int64_t>(1, int64_t(std::sqrt(double(N))) - 2);
  while (s * (s + 1) <= N) ++s;
  while (s > 1 && (s - 1) * s > N) --s;
  return s;
}

}  // namespace

int64_t signal_bytes(int32_t dtype, int64_t N) {
  switch (dtype) {
    case TM_I8_PM1: return N;
    case TM_BITS_PM1: return ceil_div(N, 8);
    case TM_F16: return 2 * N;
    default: return 4 * N;
  }
}

// Algorithm 1 step 2 and the derived sizes.
// Least integer s with s (s+1) (s+2) > N.
int64_t least_s3(int64_t N) {
  int64_t s = std::max<int64_t>(1, int64_t(std::cbrt(double(N))) - 2);
  while (s * (s + 1) * (s + 2) <= N) ++s;
  while (s > 1 && (s - 1) * s * (s + 1) > N) --s;
  return s;
}

tm_status make_plan(int64_t N, int32_t K, int32_t xdtype, int32_t mode, int32_t M1, int32_t M2, uint32_t flags,
                    PlanCore& pc, int32_t M3) {
  if (N < 1 || K < 1 || K > N) return fail(TM_EINVAL, "need 1 <= K <= N");
  if (xdtype < TM_I8_PM1 || xdtype > TM_F32) return fail(TM_EINVAL, "unknown signal dtype");
  const bool three = (flags & TM_THREE_MODULI) != 0;
  if (three && (flags & TM_THM2_SAMPLING)) return fail(TM_EUNSUPPORTED, "three moduli with the Thm. 2 sampling");
  int64_t m[3] = {0, 0, 0};
  if (three) {
    if (mode == TM_MODE_PAPER || mode == TM_MODE_AUTO) {
      int64_t c = mode == TM_MODE_PAPER ? K : std::max<int64_t>(K, least_s3(N));
      c += 1 - (c & 1);   // odd: c, c+1, c+2 pairwise co-prime
      m[0] = c; m[1] = c + 1; m[2] = c + 2;
    } else if (mode == TM_MODE_EXPLICIT) {
      m[0] = M1; m[1] = M2; m[2] = M3;
    } else {
      return fail(TM_EINVAL, "unknown mode");
    }
  } else if (mode == TM_MODE_PAPER) { m[0] = K; m[1] = int64_t(K) + 1; }
  else if (mode == TM_MODE_AUTO) { m[0] = std::max<int64_t>(K, least_s(N)); m[1] = m[0] + 1; }
  else if (mode == TM_MODE_EXPLICIT) { m[0] = M1; m[1] = M2; }
  else return fail(TM_EINVAL, "unknown mode");
  const int nm = three ? 3 : 2;
  for (int j = 0; j < nm; ++j) {
    if (m[j] < K) return fail(TM_EINVAL, "step 2 needs every modulus >= K");
    if (m[j] > 2 * N) return fail(TM_EINVAL, "moduli above 2N are not meaningful");
  }
  for (int i = 0; i < nm; ++i)
    for (int j = i + 1; j < nm; ++j)
      if (gcd64(m[i], m[j]) != 1) return fail(TM_EINVAL, "step 2 needs pairwise co-prime moduli");
  // the product of the moduli must exceed N (checked without overflow)
  bool above = m[0] > N / m[1] || m[0] * m[1] > N;
  if (three && !above) above = m[0] * m[1] > N / m[2] || m[0] * m[1] * m[2] > N;
  if (!above && !(flags & TM_ALLOW_AMBIG))
    return fail(TM_EINVAL, "step 2 needs the moduli's product above N (set TM_ALLOW_AMBIG to accept several solutions)");
  int64_t mmax = 0;
  for (int j = 0; j < nm; ++j) mmax = std::max(mmax, m[j]);
  const int64_t need = mmax + K - 1;
  int32_t logP = 0;
  while ((int64_t(1) << logP) < need) ++logP;
  if (logP > kLogPMaxLarge) return fail(TM_EUNSUPPORTED, "FFT length above 2^26 (max(M)+K-1 > 67108864)");
  if (three && logP > kLogPMax) return fail(TM_EUNSUPPORTED, "three moduli: FFT lengths up to 16384");
  if (signal_bytes(xdtype, N) > kMaxQueryBytes) return fail(TM_EUNSUPPORTED, "signal larger than 2^31-2^16 bytes");
  pc.N = N; pc.K = K; pc.xdtype = xdtype; pc.nmod = nm;
  for (int j = 0; j < 3; ++j) {
    pc.M[j] = int32_t(m[j]);
    pc.L[j] = j < nm ? ceil_div(N, m[j]) : 0;
  }
  pc.logP = logP; pc.P = 1 << logP;
  pc.inv = int32_t(mod_inverse(m[0], m[1]));
  pc.inv3 = three ? int32_t(mod_inverse((m[0] % m[2]) * (m[1] % m[2]) % m[2], m[2])) : 0;
  if (xdtype == TM_BITS_PM1 && N > kMaxQueryBytes)
    return fail(TM_EUNSUPPORTED, "bit-packed signal longer than 2^31-2^16 elements");
  const FoldGeom g = fold_geom(xdtype);
  for (int j = 0; j < 3; ++j) {
    if (j >= nm) { pc.R[j] = 1; pc.Mp[j] = 0; continue; }
    pc.R[j] = int32_t(std::max<int64_t>(1, ceil_div(g.min_mp, pc.M[j])));
    pc.Mp[j] = pc.R[j] * pc.M[j];
    // wider moduli: folded entry by entry (fold_direct.cu)
    if (fold_units_per_lane(pc.Mp[j], fold_warp_count(nm, j), g.E) > g.jmax) pc.direct = 1;
  }
  const long double prod = (long double)m[0] * (long double)m[1] * (three ? (long double)m[2] : 1.0L);
  pc.max_cand = int64_t(std::ceil((long double)N / prod)) + 3;
  pc.flags = flags;
  // FFTs longer than the blocked correlation's: passes over all SMs, on
  // folds computed entry by entry
  if (logP > kLogPMaxBlocked) pc.large = pc.direct = 1;
  return TM_OK;
}

// Bytes of a signal the fold kernel streams: a multiple of 16 holding whole
// elements (the correlation kernel adds the few elements after it).
int64_t fold_bytes(int32_t dtype, int64_t N) {
  const int64_t b = dtype == TM_BITS_PM1 ? N / 8 : signal_bytes(dtype, N);
  return b & ~int64_t(15);
}

// Elements covered by fold_bytes.
int64_t fold_elems(int32_t dtype, int64_t N) {
  const int64_t b = fold_bytes(dtype, N);
  switch (dtype) {
    case TM_I8_PM1: return b;
    case TM_BITS_PM1: return 8 * b;
    case TM_F16: return b / 2;
    default: return b / 4;
  }
}

// ---------------------------------------------------------------- per-device state
namespace {
std::mutex g_mu;
std::vector<float2*> g_twiddles;   // per device
std::vector<int> g_configured;
}  // namespace

tm_status device_setup(int dev, float2** tw) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (int(g_twiddles.size()) <= dev) { g_twiddles.resize(dev + 1, nullptr); g_configured.resize(dev + 1, 0); }
  if (!g_configured[dev]) {
    TM_CUDA(fold_configure());
    TM_CUDA(corr_configure());
    TM_CUDA(large_configure());
    std::vector<float2> h(kPMax);
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < kPMax; ++m) {
      const double a = two_pi * double(m) / double(kPMax);
      h[m] = make_float2(float(std::cos(a)), float(-std::sin(a)));   // W^m = e^{-2 pi i m / PMax}
    }
    float2* d = nullptr;
    TM_CUDA(cudaMalloc(&d, kPMax * sizeof(float2)));
    TM_CUDA(cudaMemcpy(d, h.data(), kPMax * sizeof(float2), cudaMemcpyHostToDevice));
    g_twiddles[dev] = d;
    g_configured[dev] = 1;
  }
  *tw = g_twiddles[dev];
  return TM_OK;
}

}  // namespace ftm

// ---------------------------------------------------------------- objects
// Device scratch of the slice entry points (tm_fold_slice and friends),
// allocated on first use and grown when a larger slice arrives.
struct SliceWs {
  int device = -1;
  int64_t part_cap = 0;            // int32 entries of `partial`
  ftm::FoldQ* d_fq = nullptr;
  ftm::CorrQ* d_cq = nullptr;
  int32_t* d_order = nullptr;
  int32_t* d_partial = nullptr;
  int32_t* d_err = nullptr;
  float2* d_spec = nullptr;
  ~SliceWs() {
    cudaFree(d_fq); cudaFree(d_cq); cudaFree(d_order); cudaFree(d_partial); cudaFree(d_err); cudaFree(d_spec);
  }
};

struct tm_plan_s {
  tm_plan_desc d;
  ftm::PlanCore pc;
  tm_batch_t b = nullptr;
  SliceWs* sw = nullptr;
};

namespace ftm {

void batch_free(tm_batch_t b) {
  if (!b) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->ev_stage) { cudaEventSynchronize(b->ev_stage); cudaEventDestroy(b->ev_stage); }
  if (b->aux) cudaStreamDestroy(b->aux);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->cstream) { cudaStreamSynchronize(b->cstream); cudaStreamDestroy(b->cstream); }
  if (b->ev_pfork) cudaEventDestroy(b->ev_pfork);
  if (b->ev_pjoin) cudaEventDestroy(b->ev_pjoin);
  if (b->owns_memory) {
    cudaFree(b->d_partial2);
    cudaFree(b->d_fq); cudaFree(b->d_cq); cudaFree(b->d_lq); cudaFree(b->d_ssum); cudaFree(b->d_order); cudaFree(b->d_partial);
    cudaFree(b->d_y); cudaFree(b->d_spec); cudaFree(b->d_r); cudaFree(b->d_err); cudaFree(b->d_out);
    cudaFree(b->d_x); cudaFree(b->d_t);
    if (b->h_stage) cudaFreeHost(b->h_stage);
  }
  cudaSetDevice(cur);
  delete b;
}

// Fill x/t pointers of the descriptors from b->q (or the batch's own copies).
void bind_pointers(tm_batch_t b) {
  for (int i = 0; i < b->n; ++i) {
    const void* x = (b->flags & TM_BATCH_HOST_INPUTS) ? static_cast<const void*>(b->d_x + b->xoff[i]) : b->q[i].x;
    const float* t = (b->flags & TM_BATCH_HOST_INPUTS) ? b->d_t + b->toff[i] : b->q[i].t;
    b->fq[b->fold_of[i]].x = static_cast<const uint8_t*>(x);
    b->cq[i].x = x;
    b->cq[i].t = t;
    // entry-by-entry folds land in the batch's fold buffer and are given to
    // the correlation as complete folds
    b->cq[i].y_in = b->cq[i].direct ? static_cast<const void*>(static_cast<const char*>(b->d_y) + b->cq[i].y_off * 4)
                                    : nullptr;
    if (b->lq_of.size() == size_t(b->n) && b->lq_of[i] >= 0) {
      LQ& l = b->lq[b->lq_of[i]];
      const CorrQ& c = b->cq[i];
      l.x = x;
      l.t = t;
      l.y = c.y_in;
      l.r = b->d_r + c.r_off;
      l.A = b->d_spec + c.spec_off;
      l.B = l.A + c.P;
      l.ws = l.B + c.P;
      l.err = b->d_err;
    }
  }
}

// Upload descriptors on `s` through pinned staging (reuse waits for the
// previous upload to have been consumed by the copy engine).
tm_status upload_descriptors(tm_batch_t b, cudaStream_t s) {
  const size_t nf = b->fq.size() * sizeof(FoldQ), nc = b->cq.size() * sizeof(CorrQ);
  const size_t nl = b->lq.size() * sizeof(LQ);
  const size_t nj = b->ssum.size() * sizeof(SlotSumJob);
  TM_CUDA(cudaEventSynchronize(b->ev_stage));
  char* h = static_cast<char*>(b->h_stage);
  std::memcpy(h, b->fq.data(), nf);
  std::memcpy(h + nf, b->cq.data(), nc);
  if (nl > 0) std::memcpy(h + nf + nc, b->lq.data(), nl);
  if (nj > 0) std::memcpy(h + nf + nc + nl, b->ssum.data(), nj);
  TM_CUDA(cudaMemcpyAsync(b->d_fq, h, nf, cudaMemcpyHostToDevice, s));
  TM_CUDA(cudaMemcpyAsync(b->d_cq, h + nf, nc, cudaMemcpyHostToDevice, s));
  if (nl > 0) TM_CUDA(cudaMemcpyAsync(b->d_lq, h + nf + nc, nl, cudaMemcpyHostToDevice, s));
  if (nj > 0) TM_CUDA(cudaMemcpyAsync(b->d_ssum, h + nf + nc + nl, nj, cudaMemcpyHostToDevice, s));
  TM_CUDA(cudaEventRecord(b->ev_stage, s));
  return TM_OK;
}

tm_status batch_plan(tm_batch_s* b, const tm_query* q, int32_t n, uint32_t flags, const uint8_t* nofold) {
  if (n < 1 || !q) return fail(TM_EINVAL, "empty batch");
  b->flags = flags;
  b->n = n;
  b->groups.clear();   // planning again (tm_batch_set_grid) starts afresh
  b->W = 0;
  b->nctas = 0;
  b->maxP = 0;
  b->q.assign(q, q + n);
  b->pc.resize(n);
  for (int i = 0; i < n; ++i) {
    tm_status st = make_plan(q[i].N, q[i].K, q[i].xdtype, q[i].mode, q[i].M1, q[i].M2, q[i].flags, b->pc[i], q[i].M3);
    if (st != TM_OK) {
      g_err = "query " + std::to_string(i) + ": " + g_err;
      return st;
    }
    if (!(flags & TM_BATCH_HOST_INPUTS)) {
      if (!q[i].x || !q[i].t) return fail(TM_EINVAL, "null x or t pointer");
      if (reinterpret_cast<uintptr_t>(q[i].x) & 15) return fail(TM_EINVAL, "x must be 16-byte aligned");
      if (reinterpret_cast<uintptr_t>(q[i].t) & 3) return fail(TM_EINVAL, "t must be 4-byte aligned");
    }
  }
  // few queries with long FFTs: each on all SMs instead of one CTA
  int nbig = 0;
  for (int i = 0; i < n; ++i) nbig += b->pc[i].P > kPMax ? 1 : 0;
  b->is_large.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    PlanCore& p = b->pc[i];
    if (p.P > kPMax && (p.large || p.logP >= kLogPLargeAlways || nbig <= kLargeMaxQueries) && !(nofold && nofold[i])) {
      p.large = p.direct = 1;
      b->is_large[i] = 1;
    }
    if (p.large && !b->is_large[i]) return fail(TM_EUNSUPPORTED, "FFT length above 2^18 with cached folds");
  }
  TM_CUDA(cudaGetDevice(&b->device));
  int sms = 0;
  TM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  tm_status st = device_setup(b->device, &b->tw);
  if (st != TM_OK) return st;

  // ---- fold geometry: per storage type, a flattened byte space split into
  // equal shares, one per CTA
  b->fq.resize(n);
  b->cq.resize(n);
  b->fold_of.assign(n, 0);
  b->dh.assign(n, 0);
  b->drows.assign(n, 0);
  b->dpitch.assign(n, 0);
  b->dpart.assign(n, 0);
  b->ssum.clear();
  b->ssum_of.assign(n, -1);
  b->ssum_cols = 0;
  std::vector<uint8_t> fine_of(size_t(n), 0);   // fold descriptor -> TM_FINE_PIECES
  int64_t part = 0;
  for (int32_t dt = TM_I8_PM1; dt <= TM_F32; ++dt) {
    tm_batch_s::FoldGroup gr;
    gr.dtype = dt;
    gr.first = int32_t(b->groups.empty() ? 0 : b->groups.back().first + b->groups.back().count);
    gr.count = 0;
    gr.jmax = 1;
    const FoldGeom geo = fold_geom(dt);
    int64_t W = 0, max_share = INT64_MAX;
    for (int i = 0; i < n; ++i) {
      const PlanCore& p = b->pc[i];
      if (p.xdtype != dt) continue;
      const int32_t pos = gr.first + gr.count++;
      b->fold_of[i] = pos;
      fine_of[pos] = (p.flags & TM_FINE_PIECES) ? 1 : 0;
      const int64_t nb = ((nofold && nofold[i]) || p.direct) ? 0 : fold_bytes(p.xdtype, p.N);
      FoldQ& f = b->fq[pos];
      f = FoldQ{};
      f.goff = W;
      f.nbytes = int32_t(nb);
      f.nmod = p.nmod;
      int32_t off = 0;
      for (int j = 0; j < 3; ++j) {
        f.Mp[j] = j < p.nmod ? p.Mp[j] : 0;
        f.moff[j] = off;
        off += j < p.nmod ? int32_t(pad16(p.Mp[j])) : 0;
      }
      f.stride = off;
      W += nb;
      // rows of Mp elements per share stay below the lane counters' capacity
      max_share = std::min<int64_t>(max_share, int64_t(kFoldMaxRowsPerSlot - 2) *
                                                   std::min(p.Mp[0], p.nmod == 3 ? std::min(p.Mp[1], p.Mp[2]) : p.Mp[1]) *
                                                   geo.bits / 8);
      for (int j = 0; j < p.nmod; ++j)
        gr.jmax = std::max<int32_t>(gr.jmax, fold_units_per_lane(p.Mp[j], fold_warp_count(p.nmod, j), geo.E));
    }
    if (gr.count == 0) continue;
    gr.W = W;
    const int64_t cap = b->fold_cap > 0 ? std::min<int64_t>(sms, b->fold_cap) : sms;
    int64_t nctas = std::min<int64_t>(cap, std::max<int64_t>(1, ceil_div(W, 65536)));
    if (W > 0) nctas = std::max<int64_t>(nctas, ceil_div(W, max_share));
    gr.nctas = int32_t(nctas);
    auto cta_of = [&](int64_t pos) {   // CTA whose share holds byte pos
      int32_t lo = 0, hi = gr.nctas - 1;
      while (lo < hi) {
        const int32_t mid = (lo + hi + 1) / 2;
        if (fold_cta_begin(W, gr.nctas, mid) <= pos) lo = mid; else hi = mid - 1;
      }
      return lo;
    };
    const bool real = dt == TM_F16 || dt == TM_F32;
    gr.cb.clear();
    if (real && W > 0 && gr.nctas <= kFoldMaxCtas) {
      // real signals: fixed pieces per signal, one slot each, and shares
      // that start on piece boundaries (the nearest to the equal split), so
      // every fp32 column sum is the same whatever else the batch holds
      std::vector<int64_t> bounds;
      for (int32_t k = gr.first; k < gr.first + gr.count; ++k) {
        FoldQ& f = b->fq[k];
        if (f.nbytes == 0) continue;
        f.piece = fold_piece_bytes(f.nbytes, fine_of[k] != 0);
        for (int64_t o = 0; o < f.nbytes; o += f.piece) bounds.push_back(f.goff + o);
      }
      bounds.push_back(W);
      gr.cb.assign(size_t(gr.nctas) + 1, 0);
      gr.cb[gr.nctas] = W;
      for (int32_t c = 1; c < gr.nctas; ++c) {
        const int64_t want = fold_cta_begin(W, gr.nctas, c);
        auto it = std::lower_bound(bounds.begin(), bounds.end(), want);
        int64_t v = it == bounds.end() ? W : *it;
        if (it != bounds.begin() && want - *(it - 1) < v - want) v = *(it - 1);
        gr.cb[c] = std::max(gr.cb[c - 1], v);
      }
    }
    auto share_of = [&](int64_t pos) {   // CTA whose share holds byte pos
      if (gr.cb.empty()) return cta_of(pos);
      return int32_t(std::upper_bound(gr.cb.begin(), gr.cb.end() - 1, pos) - gr.cb.begin()) - 1;
    };
    for (int32_t k = gr.first; k < gr.first + gr.count; ++k) {
      FoldQ& f = b->fq[k];
      if (f.nbytes == 0) { f.first_cta = 0; f.nslots = 0; f.part = part; continue; }
      f.first_cta = share_of(f.goff);
      f.nslots = f.piece > 0 ? int32_t(ceil_div(f.nbytes, f.piece))
                             : share_of(f.goff + f.nbytes - 1) - f.first_cta + 1;
      f.part = part;
      part += int64_t(f.nslots) * f.stride;
      if (f.nslots >= kSlotSumMin) {
        // many rows: summed into a row of their own ahead of the correlation
        SlotSumJob j;
        j.src = f.part; j.dst = part; j.nslots = f.nslots; j.cols = f.stride; j.real = real ? 1 : 0;
        b->ssum_of[k] = int32_t(b->ssum.size());
        b->ssum.push_back(j);
        b->ssum_cols = std::max(b->ssum_cols, f.stride);
        part += f.stride;
      }
    }
    b->W += W;
    b->nctas = std::max(b->nctas, gr.nctas);
    b->groups.push_back(gr);
  }
  // partial sums of the entry-by-entry folds follow the streaming fold's slots
  b->maxM_direct = b->maxHM_direct = 0;
  for (int i = 0; i < n; ++i) {
    const PlanCore& p = b->pc[i];
    if (!p.direct) continue;
    // int8 with at most 16 rows: the completion sums the rows itself (dh = 0)
    const int32_t dh = (p.xdtype == TM_I8_PM1 && p.L[0] <= 16) ? 0 : direct_row_groups(p.L[0], p.xdtype);
    const int32_t mmax = *std::max_element(p.M, p.M + p.nmod);
    const int32_t pitch = (mmax + 3) & ~3;   // rows of 16-byte multiples: vector stores
    part = (part + 3) & ~int64_t(3);
    b->dh[i] = dh;
    b->drows[i] = dh > 0 ? int32_t(ceil_div(p.L[0], dh)) : 0;
    b->dpitch[i] = pitch;
    b->dpart[i] = part;
    part += int64_t(p.nmod) * dh * pitch;
    b->maxM_direct = std::max(b->maxM_direct, mmax);
    // first-stage grid rows: groups (int8: all moduli per thread) or groups x moduli
    b->maxHM_direct = std::max(b->maxHM_direct, p.xdtype == TM_I8_PM1 ? dh : dh * p.nmod);   // 0: no launch
  }
  b->part_elems = std::max<int64_t>(part, 16);

  // ---- correlation descriptors and output layout
  int64_t yo = 0, so = 0, ro = 0;
  for (int i = 0; i < n; ++i) {
    const PlanCore& p = b->pc[i];
    const FoldQ& f = b->fq[b->fold_of[i]];
    CorrQ& c = b->cq[i];
    c.N = p.N; c.K = p.K; c.xdtype = p.xdtype;
    c.nmod = p.nmod;
    for (int j = 0; j < 3; ++j) { c.M[j] = p.M[j]; c.R[j] = p.R[j]; c.L[j] = p.L[j]; c.moff[j] = f.moff[j]; }
    c.P = p.P; c.logP = p.logP; c.inv = p.inv; c.inv3 = p.inv3;
    c.direct = p.direct;
    c.dh = b->dh[i];
    c.drows = b->drows[i];
    c.dpitch = b->dpitch[i];
    c.dpart = b->dpart[i];
    c.thm2 = (p.flags & TM_THM2_SAMPLING) ? 1 : 0;
    c.nelem16 = int32_t(fold_elems(p.xdtype, p.N));
    c.nslots = f.nslots; c.stride = f.stride; c.part = f.part;
    if (b->ssum_of[b->fold_of[i]] >= 0) {   // the slot sums' row
      c.nslots = 1;
      c.part = b->ssum[b->ssum_of[b->fold_of[i]]].dst;
    }
    c.y_off = yo; yo += int64_t(p.nmod) * p.P;
    const bool large = b->is_large[i];
    const bool blocked = p.P > kPMax && !large;   // correlation in blocks (overlap-save), r kept in global memory
    if (large) so = (so + 31) & ~int64_t(31);   // 256-byte aligned spectra (vector loads)
    c.spec_off = so;
    if (large) so += (2 * int64_t(p.P) + int64_t(large_ws_bytes() / sizeof(float2)) + 31) & ~int64_t(31);
    else so += blocked ? int64_t(blocked_spectra(p.K, std::max(p.M[0], p.M[1]))) * kPMax : p.P;
    c.r_off = ((flags & TM_BATCH_KEEP_CORR) || blocked || large) ? ro : -1;
    if (c.r_off >= 0) ro += int64_t(p.nmod) * p.P;
    if (!blocked && !large) b->maxP = std::max(b->maxP, p.P);
  }
  b->y_elems = yo; b->spec_elems = so; b->r_elems = ro;
  b->direct.clear();
  b->maxP_direct = b->maxmod_direct = 0;
  for (int i = 0; i < n; ++i) {
    if (!b->pc[i].direct) continue;
    b->direct.push_back(i);
    b->maxP_direct = std::max(b->maxP_direct, b->pc[i].P);
    b->maxmod_direct = std::max(b->maxmod_direct, b->pc[i].nmod);
  }
  // processing order: shared-memory queries (largest P first), then blocked
  // ones, then those on the multi-CTA path
  auto cls = [&](int i) { return b->is_large[i] ? 2 : (b->pc[i].P > kPMax ? 1 : 0); };
  b->order.resize(n);
  for (int i = 0; i < n; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) {
    if (cls(a) != cls(c)) return cls(a) < cls(c);
    return b->pc[a].P > b->pc[c].P;
  });
  b->n_blocked = b->n_large = 0;
  for (int i = 0; i < n; ++i) {
    b->n_blocked += cls(i) == 1 ? 1 : 0;
    b->n_large += cls(i) == 2 ? 1 : 0;
  }
  b->lq.clear();
  b->lq_of.assign(n, -1);
  b->lq_maxP = b->lq_maxM = b->lq_two = 0;
  for (int k = 0; k < n; ++k) {
    const int i = b->order[k];   // the order puts these queries last, largest P first
    if (!b->is_large[i]) continue;
    const PlanCore& p = b->pc[i];
    b->lq_of[i] = int32_t(b->lq.size());
    b->lq.push_back(LQ{});
    LQ& l = b->lq.back();
    l.qi = i;
    l.N = p.N; l.K = p.K; l.xdtype = p.xdtype;
    l.M[0] = p.M[0]; l.M[1] = p.M[1];
    l.inv = p.inv; l.P = p.P; l.logP = p.logP;
    l.thm2 = (p.flags & TM_THM2_SAMPLING) ? 1 : 0;
    l.nsd = large_dims(p.logP, l.logL);
    b->lq_maxP = std::max(b->lq_maxP, p.P);
    b->lq_maxM = std::max(b->lq_maxM, std::max(p.M[0], p.M[1]));
    b->lq_two = b->lq_two || l.nsd == 2;
  }

  return TM_OK;
}

tm_status batch_alloc(tm_batch_s* b) {
  const int32_t n = b->n;
  const uint32_t flags = b->flags;
  auto alloc = [&](void** ptr, size_t bytes) -> cudaError_t {
    b->ws_bytes += int64_t(bytes);
    return cudaMalloc(ptr, std::max<size_t>(bytes, 16));
  };
  bool ok = alloc((void**)&b->d_fq, n * sizeof(FoldQ)) == cudaSuccess &&
            alloc((void**)&b->d_cq, n * sizeof(CorrQ)) == cudaSuccess &&
            alloc((void**)&b->d_lq, std::max<size_t>(b->lq.size(), 1) * sizeof(LQ)) == cudaSuccess &&
            alloc((void**)&b->d_ssum, n * sizeof(SlotSumJob)) == cudaSuccess &&
            alloc((void**)&b->d_order, 2 * n * sizeof(int32_t)) == cudaSuccess &&
            alloc((void**)&b->d_partial, b->part_elems * sizeof(int32_t)) == cudaSuccess &&
            alloc(&b->d_y, b->y_elems * sizeof(int32_t)) == cudaSuccess &&
            alloc((void**)&b->d_spec, b->spec_elems * sizeof(float2)) == cudaSuccess &&
            alloc((void**)&b->d_err, 16) == cudaSuccess &&
            alloc((void**)&b->d_out, n * sizeof(tm_result)) == cudaSuccess;
  if (ok && b->r_elems > 0) ok = alloc((void**)&b->d_r, b->r_elems * sizeof(float)) == cudaSuccess;
  b->part_alloc = b->part_elems;
  if (ok && (flags & TM_BATCH_PIPELINED)) {
    ok = alloc((void**)&b->d_partial2, b->part_elems * sizeof(int32_t)) == cudaSuccess &&
         cudaStreamCreateWithFlags(&b->cstream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_pfork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_pjoin, cudaEventDisableTiming) == cudaSuccess;
  }
  if (ok && (flags & TM_BATCH_HOST_INPUTS)) {
    int64_t xb = 0, tb = 0;
    b->xoff.resize(n); b->toff.resize(n);
    for (int i = 0; i < n; ++i) {
      b->xoff[i] = xb; xb += pad16(signal_bytes(b->pc[i].xdtype, b->pc[i].N)) + 16;
      b->toff[i] = tb; tb += pad16(b->pc[i].K);
    }
    ok = alloc((void**)&b->d_x, xb) == cudaSuccess && alloc((void**)&b->d_t, tb * sizeof(float)) == cudaSuccess;
  }
  b->stage_bytes = n * (sizeof(FoldQ) + sizeof(CorrQ) + sizeof(LQ) + sizeof(SlotSumJob));
  if (ok) ok = cudaMallocHost(&b->h_stage, b->stage_bytes) == cudaSuccess;
  if (ok) ok = cudaEventCreateWithFlags(&b->ev_stage, cudaEventDisableTiming) == cudaSuccess;
  if (ok && !b->lq.empty())   // the side stream of the long-FFT queries' template spectra
    ok = cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return fail(TM_ENOMEM, "device workspace allocation failed");
  }
  TM_CUDA(cudaMemset(b->d_err, 0, 16));
  TM_CUDA(cudaMemcpy(b->d_order, b->order.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (!b->direct.empty())   // the entry-by-entry folds' query list follows the order
    TM_CUDA(cudaMemcpy(b->d_order + n, b->direct.data(), b->direct.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice));
  return TM_OK;
}

tm_status batch_build(const tm_query* q, int32_t n, uint32_t flags, tm_batch_t* out) {
  if (!out) return fail(TM_EINVAL, "null output handle");
  *out = nullptr;
  tm_batch_t b = new (std::nothrow) tm_batch_s();
  if (!b) return fail(TM_ENOMEM, "host allocation");
  tm_status st = batch_plan(b, q, n, flags);
  if (st == TM_OK) st = batch_alloc(b);
  if (st == TM_OK) {
    bind_pointers(b);
    st = upload_descriptors(b, nullptr);
  }
  if (st == TM_OK) {
    const cudaError_t e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) st = cuda_fail(e, "descriptor upload");
  }
  if (st != TM_OK) {
    batch_free(b);
    return st;
  }
  *out = b;
  return TM_OK;
}

// The share starts of a fold group whose shares follow piece boundaries.
void fold_args_shares(FoldArgs& a, const tm_batch_s::FoldGroup& g) {
  a.has_cb = g.cb.empty() ? 0 : 1;
  for (size_t c = 0; c < g.cb.size(); ++c) a.cb[c] = g.cb[c];
}

tm_status batch_fold(tm_batch_t b, cudaStream_t s, int parity, bool clear_err) {
  int32_t* partial = parity ? b->d_partial2 : b->d_partial;
  int32_t* err = b->d_err + parity;
  if (clear_err) TM_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
  if (!b->lq.empty() && b->aux) {
    // the long-FFT queries' template spectra need only t: they run on a
    // side stream while the fold streams x (joined in batch_correlate)
    TM_CUDA(cudaEventRecord(b->ev_fork, s));
    TM_CUDA(cudaStreamWaitEvent(b->aux, b->ev_fork, 0));
    TM_CUDA(launch_large_template(b->d_lq, b->lq.data(), int(b->lq.size()), b->lq_maxP, b->lq_two != 0, b->aux));
    TM_CUDA(cudaEventRecord(b->ev_join, b->aux));
    b->tpl_pending = true;
  }
  for (const auto& g : b->groups) {
    if (g.W == 0) continue;
    FoldArgs a;
    a.q = b->d_fq + g.first; a.nq = g.count; a.dtype = g.dtype; a.nctas = g.nctas; a.W = g.W;
    a.partial = partial; a.err = err; a.tile = g.tile;
    fold_args_shares(a, g);
    fold_args_first_queries(a, b->fq.data() + g.first);
    TM_CUDA(launch_fold(a, g.jmax, s));
  }
  if (!b->direct.empty())
    TM_CUDA(launch_fold_direct(b->d_cq, b->d_order + b->n, int32_t(b->direct.size()), b->maxP_direct,
                               b->maxmod_direct, b->maxM_direct, b->maxHM_direct, partial, b->d_y, s));
  return TM_OK;
}

tm_status batch_correlate(tm_batch_t b, tm_result* out, cudaStream_t s, int parity, bool after_fold) {
  CorrArgs a;
  a.q = b->d_cq; a.order = b->d_order; a.nq = b->n - b->n_blocked - b->n_large;
  a.partial = parity ? b->d_partial2 : b->d_partial;
  a.y = b->d_y; a.spec = b->d_spec; a.r = b->d_r; a.tw = b->tw;
  a.out = out; a.err = b->d_err + parity;
  a.ctas = b->corr_ctas;
  // a fold kernel (not a copy) ran last on s: the slot sums and the
  // correlation may start before it ends (their template work overlaps it)
  const bool pdl = after_fold && (b->W > 0 || !b->direct.empty());
  if (!b->ssum.empty()) {
    SlotSumArgs sa;
    sa.partial = parity ? b->d_partial2 : b->d_partial;
    sa.job = b->d_ssum;
    sa.njobs = int32_t(b->ssum.size());
    sa.max_cols = b->ssum_cols;
    sa.pdl = pdl ? 1 : 0;
    TM_CUDA(launch_slot_sums(sa, s));
  }
  a.pdl = pdl ? 1 : 0;
  if (after_fold && a.nq == 1 && a.ctas == 0) {
    // one query on this launch: its descriptor goes as a kernel parameter,
    // unless a graph is being captured (later tm_batch_set_inputs calls
    // must reach the replays through the device copy)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    TM_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      a.lone = b->order[0];
      a.q1 = b->cq[a.lone];
    }
  }
  if (a.nq > 0) TM_CUDA(launch_correlate(a, b->maxP, s));
  a.pdl = 0;
  a.lone = -1;
  a.ctas = 0;
  a.first = 0;
  if (b->n_blocked > 0) {
    a.order = b->d_order + (b->n - b->n_large - b->n_blocked);
    a.nq = b->n_blocked;
    TM_CUDA(launch_correlate_blocked(a, s));
  }
  if (!b->lq.empty()) {
    if (b->tpl_pending) {   // template spectra launched beside the fold
      TM_CUDA(cudaStreamWaitEvent(s, b->ev_join, 0));
      b->tpl_pending = false;
      TM_CUDA(launch_large_signal(b->d_lq, b->lq.data(), int(b->lq.size()), b->lq_maxP, b->lq_two != 0,
                                  b->lq_maxM, out, s));
    } else {
      TM_CUDA(launch_correlate_large(b->d_lq, b->lq.data(), int(b->lq.size()), b->lq_maxP, b->lq_two != 0,
                                     b->lq_maxM, out, s));
    }
  }
  return TM_OK;
}

namespace {

// One CTA waits on an mbarrier that nothing arrives at: the bounded wait
// must give up after limit_ns and report it.
__global__ void wait_timeout_probe(uint64_t limit_ns, int32_t* gave_up) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const bool ok = mbar_wait_for(&bar, 0, limit_ns);
  if (threadIdx.x == 0) *gave_up = ok ? 0 : 1;
}

}  // namespace

}  // namespace ftm

using namespace ftm;

// ================================================================ C ABI
extern "C" {

const char* tm_version(void) { return "tm 0.1 (sm_103a)"; }
const char* tm_last_error(void) { return g_err.c_str(); }

tm_status tm_plan_create(const tm_plan_desc* desc, tm_plan_t* out) {
  if (!desc || !out) return fail(TM_EINVAL, "null argument");
  *out = nullptr;
  tm_plan_t p = new (std::nothrow) tm_plan_s();
  if (!p) return fail(TM_ENOMEM, "host allocation");
  p->d = *desc;
  tm_status st = make_plan(desc->N, desc->K, desc->xdtype, desc->mode, desc->M1, desc->M2, desc->flags, p->pc,
                           desc->M3);
  if (st != TM_OK) { delete p; return st; }
  *out = p;
  return TM_OK;
}

tm_status tm_plan_get_info(tm_plan_t p, tm_plan_info* info) {
  if (!p || !info) return fail(TM_EINVAL, "null argument");
  info->N = p->pc.N; info->K = p->pc.K; info->xdtype = p->pc.xdtype;
  info->M1 = p->pc.M[0]; info->M2 = p->pc.M[1];
  info->L1 = p->pc.L[0]; info->L2 = p->pc.L[1];
  info->M3 = p->pc.nmod == 3 ? p->pc.M[2] : 0;
  info->reserved = 0;
  info->L3 = p->pc.nmod == 3 ? p->pc.L[2] : 0;
  info->P = p->pc.P;
  info->max_cand = int32_t(std::min<int64_t>(p->pc.max_cand, INT32_MAX));
  return TM_OK;
}

tm_status tm_plan_destroy(tm_plan_t p) {
  if (!p) return TM_OK;
  batch_free(p->b);
  if (p->sw) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->sw->device);
    delete p->sw;
    cudaSetDevice(cur);
  }
  delete p;
  return TM_OK;
}

namespace {

// The slice scratch of plan p on the current device, with room for `slots`
// partial slots.
tm_status slice_ws(tm_plan_t p, int64_t slots, SliceWs** out) {
  int dev = 0;
  TM_CUDA(cudaGetDevice(&dev));
  if (p->sw && p->sw->device != dev) return fail(TM_EINVAL, "plan's slice scratch lives on another device");
  if (!p->sw) {
    SliceWs* w = new (std::nothrow) SliceWs();
    if (!w) return fail(TM_ENOMEM, "host allocation");
    w->device = dev;
    const bool ok = cudaMalloc((void**)&w->d_fq, sizeof(FoldQ)) == cudaSuccess &&
                    cudaMalloc((void**)&w->d_cq, sizeof(CorrQ)) == cudaSuccess &&
                    cudaMalloc((void**)&w->d_order, 16) == cudaSuccess &&
                    cudaMalloc((void**)&w->d_err, 16) == cudaSuccess &&
                    cudaMalloc((void**)&w->d_spec, size_t(p->pc.P) * sizeof(float2)) == cudaSuccess;
    if (!ok) {
      delete w;
      cudaGetLastError();
      return fail(TM_ENOMEM, "slice scratch");
    }
    TM_CUDA(cudaMemset(w->d_order, 0, 16));
    TM_CUDA(cudaMemset(w->d_err, 0, 16));
    p->sw = w;
  }
  const int64_t stride = pad16(p->pc.Mp[0]) + pad16(p->pc.Mp[1]);
  if (slots * stride > p->sw->part_cap) {
    cudaFree(p->sw->d_partial);
    p->sw->d_partial = nullptr;
    p->sw->part_cap = 0;
    if (cudaMalloc((void**)&p->sw->d_partial, size_t(slots * stride) * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      return fail(TM_ENOMEM, "slice partial folds");
    }
    p->sw->part_cap = slots * stride;
  }
  *out = p->sw;
  return TM_OK;
}

}  // namespace

tm_status tm_fold_slice(tm_plan_t p, const void* x, int64_t n0, int64_t len, void* y, tm_stream_t stream) {
  if (!p || !y || (len > 0 && !x)) return fail(TM_EINVAL, "null argument");
  const PlanCore& pc = p->pc;
  if (n0 < 0 || len < 0 || n0 + len > pc.N) return fail(TM_EINVAL, "slice outside [0, N)");
  const FoldGeom geo = fold_geom(pc.xdtype);
  if ((n0 * geo.bits) % 128 != 0) return fail(TM_EINVAL, "slice start must fall on a 16-byte boundary of the signal");
  if (reinterpret_cast<uintptr_t>(x) & 15) return fail(TM_EINVAL, "x must be 16-byte aligned");
  if (pc.P > kPMax) return fail(TM_EUNSUPPORTED, "slices need P <= 16384");
  if (pc.flags & TM_THM2_SAMPLING) return fail(TM_EUNSUPPORTED, "slices use the sampling of Eq. (3)");
  if (pc.nmod != 2) return fail(TM_EUNSUPPORTED, "slices use two moduli");
  if (pc.direct) return fail(TM_EUNSUPPORTED, "slices need moduli the streaming fold holds");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  TM_CUDA(cudaGetDevice(&dev));
  TM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float2* tw = nullptr;
  tm_status st = device_setup(dev, &tw);
  if (st != TM_OK) return st;
  const int64_t W = fold_bytes(pc.xdtype, len);
  const int64_t max_share = int64_t(kFoldMaxRowsPerSlot - 2) * std::min(pc.Mp[0], pc.Mp[1]) * geo.bits / 8;
  int64_t nctas = std::min<int64_t>(sms, std::max<int64_t>(1, ceil_div(W, 65536)));
  if (W > 0) nctas = std::max<int64_t>(nctas, ceil_div(W, max_share));
  SliceWs* w = nullptr;
  if ((st = slice_ws(p, nctas, &w)) != TM_OK) return st;
  FoldQ f{};
  f.x = static_cast<const uint8_t*>(x);
  f.goff = 0;
  f.nbytes = int32_t(W);
  f.Mp[0] = pc.Mp[0]; f.Mp[1] = pc.Mp[1];
  f.moff[0] = 0; f.moff[1] = int32_t(pad16(pc.Mp[0]));
  f.stride = int32_t(pad16(pc.Mp[0]) + pad16(pc.Mp[1]));
  f.nmod = 2;
  f.first_cta = 0;
  f.nslots = W > 0 ? int32_t(nctas) : 0;
  f.part = 0;
  f.e0 = n0;
  TM_CUDA(cudaMemcpyAsync(w->d_fq, &f, sizeof(f), cudaMemcpyHostToDevice, s));
  if (W > 0) {
    FoldArgs a;
    a.q = w->d_fq; a.nq = 1; a.dtype = pc.xdtype; a.nctas = int32_t(nctas); a.W = W;
    a.partial = w->d_partial; a.err = w->d_err;
    const int jmax = std::max(fold_units_per_lane(pc.Mp[0], kFoldWarps0, geo.E),
                              fold_units_per_lane(pc.Mp[1], kFoldWarps1, geo.E));
    TM_CUDA(launch_fold(a, jmax, s));
  }
  SliceFoldArgs c{};
  c.partial = w->d_partial;
  c.nslots = f.nslots;
  c.stride = f.stride;
  for (int j = 0; j < 2; ++j) { c.moff[j] = f.moff[j]; c.M[j] = pc.M[j]; c.R[j] = pc.R[j]; c.L[j] = pc.L[j]; }
  c.N = pc.N; c.K = pc.K; c.P = pc.P; c.xdtype = pc.xdtype;
  c.x = x; c.n0 = n0; c.len = len; c.nfold = fold_elems(pc.xdtype, len);
  c.y = y;
  TM_CUDA(launch_fold_slice_complete(c, s));
  return TM_OK;
}

tm_status tm_correlate_folds(tm_plan_t p, const void* y, const float* t, tm_result* out, tm_stream_t stream) {
  if (!p || !y || !t || !out) return fail(TM_EINVAL, "null argument");
  const PlanCore& pc = p->pc;
  if (pc.P > kPMax) return fail(TM_EUNSUPPORTED, "folds given: P <= 16384 only");
  if (pc.nmod != 2) return fail(TM_EUNSUPPORTED, "folds given: two moduli");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  TM_CUDA(cudaGetDevice(&dev));
  float2* tw = nullptr;
  tm_status st = device_setup(dev, &tw);
  if (st != TM_OK) return st;
  SliceWs* w = nullptr;
  if ((st = slice_ws(p, 0, &w)) != TM_OK) return st;
  CorrQ c{};
  c.x = nullptr; c.t = t; c.N = pc.N; c.K = pc.K; c.xdtype = pc.xdtype; c.nmod = 2;
  for (int j = 0; j < 2; ++j) { c.M[j] = pc.M[j]; c.R[j] = pc.R[j]; c.L[j] = pc.L[j]; }
  c.P = pc.P; c.logP = pc.logP; c.inv = pc.inv;
  c.thm2 = (pc.flags & TM_THM2_SAMPLING) ? 1 : 0;
  c.nelem16 = int32_t(fold_elems(pc.xdtype, pc.N));
  c.nslots = 0; c.stride = 0; c.part = 0; c.y_off = 0; c.spec_off = 0; c.r_off = -1;
  c.y_in = y;
  TM_CUDA(cudaMemcpyAsync(w->d_cq, &c, sizeof(c), cudaMemcpyHostToDevice, s));
  TM_CUDA(cudaMemsetAsync(w->d_err, 0, sizeof(int32_t), s));
  CorrArgs a;
  a.q = w->d_cq; a.order = w->d_order; a.nq = 1; a.partial = nullptr;
  a.y = const_cast<void*>(y); a.spec = w->d_spec; a.r = nullptr; a.tw = tw; a.out = out; a.err = w->d_err;
  TM_CUDA(launch_correlate(a, pc.P, s));
  return TM_OK;
}

tm_status tm_score_slice(tm_plan_t p, const void* x, int64_t n0, int64_t len, const float* t, const int64_t* m,
                         int32_t nm, double* out, tm_stream_t stream) {
  if (!p || !t || (nm > 0 && (!m || !out)) || (len > 0 && !x)) return fail(TM_EINVAL, "null argument");
  const PlanCore& pc = p->pc;
  if (n0 < 0 || len < 0 || n0 + len > pc.N || nm < 0) return fail(TM_EINVAL, "slice outside [0, N)");
  if (pc.xdtype == TM_BITS_PM1 && n0 % 8 != 0) return fail(TM_EINVAL, "bit-packed slices start on a byte");
  SliceScoreArgs a;
  a.x = x; a.xdtype = pc.xdtype; a.N = pc.N; a.n0 = n0; a.len = len; a.t = t; a.K = pc.K; a.m = m; a.nm = nm;
  a.out = out;
  TM_CUDA(launch_score_slice(a, reinterpret_cast<cudaStream_t>(stream)));
  return TM_OK;
}

tm_status tm_match(tm_plan_t p, const void* x, const float* t, tm_result* out, tm_stream_t stream) {
  if (!p || !x || !t || !out) return fail(TM_EINVAL, "null argument");
  tm_query q;
  q.x = x; q.t = t; q.N = p->d.N; q.K = p->d.K; q.xdtype = p->d.xdtype; q.mode = p->d.mode;
  q.M1 = p->d.M1; q.M2 = p->d.M2; q.flags = p->d.flags; q.M3 = p->d.M3; q.reserved = 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!p->b) {
    tm_status st = batch_build(&q, 1, 0, &p->b);
    if (st != TM_OK) return st;
  } else if (p->b->q[0].x != x || p->b->q[0].t != t) {
    if (reinterpret_cast<uintptr_t>(x) & 15) return fail(TM_EINVAL, "x must be 16-byte aligned");
    p->b->q[0] = q;
    bind_pointers(p->b);
    tm_status st = upload_descriptors(p->b, s);
    if (st != TM_OK) return st;
  }
  tm_status st = batch_fold(p->b, s);
  if (st != TM_OK) return st;
  return batch_correlate(p->b, out, s, 0, true);
}

tm_status tm_batch_create(const tm_query* q, int32_t n, uint32_t flags, tm_batch_t* out) {
  return batch_build(q, n, flags, out);
}

tm_status tm_batch_set_inputs(tm_batch_t b, const tm_query* q, int32_t n) {
  if (!b || !q || n != b->n) return fail(TM_EINVAL, "batch size mismatch");
  for (int i = 0; i < n; ++i) {
    if (q[i].N != b->q[i].N || q[i].K != b->q[i].K || q[i].xdtype != b->q[i].xdtype)
      return fail(TM_EINVAL, "query shapes differ from the batch");
    if (reinterpret_cast<uintptr_t>(q[i].x) & 15) return fail(TM_EINVAL, "x must be 16-byte aligned");
  }
  for (int i = 0; i < n; ++i) { b->q[i].x = q[i].x; b->q[i].t = q[i].t; }
  bind_pointers(b);
  return upload_descriptors(b, nullptr);
}

tm_status tm_batch_fold(tm_batch_t b, tm_stream_t stream) {
  if (!b) return fail(TM_EINVAL, "null batch");
  return batch_fold(b, reinterpret_cast<cudaStream_t>(stream));
}

tm_status tm_batch_correlate(tm_batch_t b, tm_result* out, tm_stream_t stream) {
  if (!b || !out) return fail(TM_EINVAL, "null argument");
  return batch_correlate(b, out, reinterpret_cast<cudaStream_t>(stream));
}

tm_status tm_batch_run(tm_batch_t b, tm_result* out, tm_stream_t stream) {
  if (!b || !out) return fail(TM_EINVAL, "null argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  tm_status st = batch_fold(b, s);
  if (st != TM_OK) return st;
  return batch_correlate(b, out, s, 0, true);
}

tm_status tm_batch_set_grid(tm_batch_t b, int32_t fold_ctas, int32_t corr_ctas) {
  if (!b) return fail(TM_EINVAL, "null batch");
  if (!b->owns_memory) return fail(TM_EINVAL, "the batch's memory belongs to a server");
  if (fold_ctas < 0 || corr_ctas < 0) return fail(TM_EINVAL, "negative CTA count");
  if (b->pending) return fail(TM_EBUSY, "a pipelined run is pending (tm_batch_pipeline_flush first)");
  TM_CUDA(cudaSetDevice(b->device));
  int32_t tiles[4] = {kFoldTile, kFoldTile, kFoldTile, kFoldTile};
  for (const auto& g : b->groups) tiles[g.dtype] = g.tile;
  const std::vector<tm_query> q = b->q;
  b->fold_cap = fold_ctas;
  b->corr_ctas = corr_ctas;
  tm_status st = batch_plan(b, q.data(), b->n, b->flags);
  if (st != TM_OK) return st;
  for (auto& g : b->groups) g.tile = tiles[g.dtype];
  if (b->part_elems > b->part_alloc) {
    // more shares than the buffers were sized for: grow them
    TM_CUDA(cudaDeviceSynchronize());
    cudaFree(b->d_partial);
    b->d_partial = nullptr;
    if (b->d_partial2) { cudaFree(b->d_partial2); b->d_partial2 = nullptr; }
    bool ok = cudaMalloc((void**)&b->d_partial, b->part_elems * sizeof(int32_t)) == cudaSuccess;
    if (ok && (b->flags & TM_BATCH_PIPELINED))
      ok = cudaMalloc((void**)&b->d_partial2, b->part_elems * sizeof(int32_t)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return fail(TM_ENOMEM, "partial fold buffers");
    }
    b->ws_bytes += (b->part_elems - b->part_alloc) * int64_t(sizeof(int32_t)) * ((b->flags & TM_BATCH_PIPELINED) ? 2 : 1);
    b->part_alloc = b->part_elems;
  }
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  bind_pointers(b);
  st = upload_descriptors(b, nullptr);
  if (st != TM_OK) return st;
  TM_CUDA(cudaStreamSynchronize(nullptr));
  return TM_OK;
}

tm_status tm_batch_run_pipelined(tm_batch_t b, tm_result* out, tm_stream_t stream, tm_event_t fold_begin,
                                 tm_event_t fold_end) {
  if (!b || !out) return fail(TM_EINVAL, "null argument");
  if (!(b->flags & TM_BATCH_PIPELINED)) return fail(TM_EINVAL, "batch was created without TM_BATCH_PIPELINED");
  if (b->n_large > 0 || b->n_blocked > 0 || !b->direct.empty())
    return fail(TM_EUNSUPPORTED, "pipelined runs need every query on the streaming fold and FFT lengths up to 16384");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int par = b->pp;
  // the correlation stream starts after the caller's earlier work
  TM_CUDA(cudaEventRecord(b->ev_pfork, s));
  TM_CUDA(cudaStreamWaitEvent(b->cstream, b->ev_pfork, 0));
  // the fold's error word was reset on the correlation stream after its
  // last reader (the previous call's); the first call after a flush or a
  // plain run resets it here
  const bool clear_here = !b->pending;
  if (clear_here) TM_CUDA(cudaMemsetAsync(b->d_err + par, 0, sizeof(int32_t), s));
  if (fold_begin) TM_CUDA(cudaEventRecord(reinterpret_cast<cudaEvent_t>(fold_begin), s));
  tm_status st = batch_fold(b, s, par, false);
  if (st != TM_OK) return st;
  if (fold_end) TM_CUDA(cudaEventRecord(reinterpret_cast<cudaEvent_t>(fold_end), s));
  if (b->pending) {
    st = batch_correlate(b, b->pending_out, b->cstream, par ^ 1);
    if (st != TM_OK) return st;
    // the next call folds into parity par ^ 1: its error word is free now
    TM_CUDA(cudaMemsetAsync(b->d_err + (par ^ 1), 0, sizeof(int32_t), b->cstream));
  }
  TM_CUDA(cudaEventRecord(b->ev_pjoin, b->cstream));
  TM_CUDA(cudaStreamWaitEvent(s, b->ev_pjoin, 0));
  b->pending = true;
  b->pending_out = out;
  b->pp = par ^ 1;
  return TM_OK;
}

tm_status tm_batch_pipeline_flush(tm_batch_t b, tm_stream_t stream) {
  if (!b) return fail(TM_EINVAL, "null batch");
  if (!b->pending) return TM_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  tm_status st = batch_correlate(b, b->pending_out, s, b->pp ^ 1);
  if (st != TM_OK) return st;
  // after its last reader: the error word is clean for the next fold of this parity
  TM_CUDA(cudaMemsetAsync(b->d_err + (b->pp ^ 1), 0, sizeof(int32_t), s));
  b->pending = false;
  b->pending_out = nullptr;
  return TM_OK;
}

tm_status tm_selftest_wait_timeout(int64_t limit_ns, int32_t* gave_up) {
  if (!gave_up) return fail(TM_EINVAL, "tm_selftest_wait_timeout: null argument");
  const int64_t lim = limit_ns < 1000 ? 1000 : limit_ns > 100000000 ? 100000000 : limit_ns;
  int32_t* d = nullptr;
  TM_CUDA(cudaMalloc(&d, sizeof(int32_t)));
  cudaError_t e = cudaMemset(d, 0xff, sizeof(int32_t));
  if (e == cudaSuccess) {
    wait_timeout_probe<<<1, 32>>>(uint64_t(lim), d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(gave_up, d, sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "tm_selftest_wait_timeout");
  return TM_OK;
}

namespace {

// Tuned stage sizes by (storage type, log2 of the group's bytes, log2 of
// the mean effective modulus), shared by all batches of the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int32_t> g_tune;

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << (l + 1)) <= v) ++l;
  return l;
}

}  // namespace

namespace {

std::map<std::tuple<int32_t, int64_t, int32_t>, std::pair<int32_t, int32_t>> g_tune_grid;

// Pipelined calls per candidate split of the SMs; keeps the fastest.
tm_status tune_grid(tm_batch_t b, cudaStream_t s, uint32_t flags, cudaEvent_t e0, cudaEvent_t e1) {
  if (!(b->flags & TM_BATCH_PIPELINED)) return fail(TM_EINVAL, "TM_TUNE_GRID needs a TM_BATCH_PIPELINED batch");
  if (b->pending) return fail(TM_EBUSY, "a pipelined run is pending (tm_batch_pipeline_flush first)");
  const auto key = std::make_tuple(b->n, b->W, b->maxP);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_grid.find(key);
    if (it != g_tune_grid.end() && !(flags & TM_TUNE_FORCE))
      return tm_batch_set_grid(b, it->second.first, it->second.second);
  }
  int sms = 0;
  TM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  std::vector<std::pair<int32_t, int32_t>> cand = {{0, 0}};
  for (int c : {16, 20, 22, 24, 28, 32, sms / 5, sms / 4, sms / 3, sms / 2}) {
    if (c < 1 || c >= sms || c > b->n) continue;
    const std::pair<int32_t, int32_t> fc(sms - c, c);
    if (std::find(cand.begin(), cand.end(), fc) == cand.end()) cand.push_back(fc);
  }
  float best = -1.f;
  std::pair<int32_t, int32_t> pick(0, 0);
  for (const auto& fc : cand) {
    tm_status st = tm_batch_set_grid(b, fc.first, fc.second);
    if (st != TM_OK) return st;
    const int reps = 6;
    for (int r = 0; r < 2 && st == TM_OK; ++r) st = tm_batch_run_pipelined(b, b->d_out, s, nullptr, nullptr);
    if (st == TM_OK) st = tm_batch_pipeline_flush(b, s);
    TM_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps && st == TM_OK; ++r) st = tm_batch_run_pipelined(b, b->d_out, s, nullptr, nullptr);
    if (st == TM_OK) st = tm_batch_pipeline_flush(b, s);
    if (st != TM_OK) return st;
    TM_CUDA(cudaEventRecord(e1, s));
    TM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    TM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (best < 0.f || ms < best) {
      best = ms;
      pick = fc;
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_grid[key] = pick;
  }
  return tm_batch_set_grid(b, pick.first, pick.second);
}

}  // namespace

tm_status tm_batch_get_grid(tm_batch_t b, int32_t* fold_ctas, int32_t* corr_ctas) {
  if (!b) return fail(TM_EINVAL, "null batch");
  if (fold_ctas) *fold_ctas = b->fold_cap;
  if (corr_ctas) *corr_ctas = b->corr_ctas;
  return TM_OK;
}

tm_status tm_batch_autotune(tm_batch_t b, tm_stream_t stream, uint32_t flags, int32_t* tiles) {
  if (!b) return fail(TM_EINVAL, "null batch");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TM_CUDA(cudaSetDevice(b->device));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TM_CUDA(cudaEventCreate(&e0));
  TM_CUDA(cudaEventCreate(&e1));
  tm_status st = TM_OK;
  for (auto& g : b->groups) {
    if (g.W == 0) continue;
    int64_t mp = 0;
    for (int32_t k = g.first; k < g.first + g.count; ++k) mp += b->fq[k].Mp[0];
    const auto key = std::make_tuple(int(g.dtype), ilog2(g.W), ilog2(std::max<int64_t>(1, mp / g.count)));
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end() && !(flags & TM_TUNE_FORCE)) {
        g.tile = it->second;
        continue;
      }
    }
    FoldArgs a;
    a.q = b->d_fq + g.first; a.nq = g.count; a.dtype = g.dtype; a.nctas = g.nctas; a.W = g.W;
    a.partial = b->d_partial; a.err = b->d_err;
    fold_args_shares(a, g);
    fold_args_first_queries(a, b->fq.data() + g.first);
    float best = 0.f;
    int32_t best_tile = kFoldTile;
    for (int32_t tile : {65536, 32768, 16384}) {
      a.tile = tile;
      cudaError_t e = launch_fold(a, g.jmax, s);   // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_fold(a, g.jmax, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "tm_batch_autotune");
        break;
      }
      if (tile == 65536 || ms < best) {
        best = ms;
        best_tile = tile;
      }
    }
    if (st != TM_OK) break;
    g.tile = best_tile;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best_tile;
  }
  if (st == TM_OK && (flags & TM_TUNE_GRID)) st = tune_grid(b, s, flags, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TM_OK) return st;
  if (tiles) {
    for (int d = 0; d < 4; ++d) tiles[d] = 0;
    for (const auto& g : b->groups)
      if (g.dtype >= 0 && g.dtype < 4) tiles[g.dtype] = g.tile;
  }
  return TM_OK;
}

tm_status tm_batch_graph_capture(tm_batch_t b, tm_result* out) {
  if (!b || !out) return fail(TM_EINVAL, "tm_batch_graph_capture: null argument");
  TM_CUDA(cudaSetDevice(b->device));
  if (!b->cap_stream) TM_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  TM_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  tm_status st = batch_fold(b, b->cap_stream);
  if (st == TM_OK) st = batch_correlate(b, out, b->cap_stream, 0, true);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
  if (st != TM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  const cudaError_t e2 = cudaGraphInstantiate(&b->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    b->gexec = nullptr;
    return cuda_fail(e2, "cudaGraphInstantiate");
  }
  return TM_OK;
}

tm_status tm_batch_graph_launch(tm_batch_t b, tm_stream_t stream) {
  if (!b || !b->gexec) return fail(TM_EINVAL, "tm_batch_graph_launch: no captured graph");
  TM_CUDA(cudaGraphLaunch(b->gexec, reinterpret_cast<cudaStream_t>(stream)));
  return TM_OK;
}

tm_status tm_batch_run_host(tm_batch_t b, const void* const* x_host, const float* const* t_host,
                            tm_result* out_host, tm_stream_t stream) {
  if (!b || !x_host || !t_host || !out_host) return fail(TM_EINVAL, "null argument");
  if (!(b->flags & TM_BATCH_HOST_INPUTS)) return fail(TM_EINVAL, "batch was created without TM_BATCH_HOST_INPUTS");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < b->n; ++i) {
    TM_CUDA(cudaMemcpyAsync(b->d_x + b->xoff[i], x_host[i], signal_bytes(b->pc[i].xdtype, b->pc[i].N),
                            cudaMemcpyHostToDevice, s));
    TM_CUDA(cudaMemcpyAsync(b->d_t + b->toff[i], t_host[i], size_t(b->pc[i].K) * sizeof(float),
                            cudaMemcpyHostToDevice, s));
  }
  tm_status st = batch_fold(b, s);
  if (st != TM_OK) return st;
  st = batch_correlate(b, b->d_out, s, 0, true);
  if (st != TM_OK) return st;
  TM_CUDA(cudaMemcpyAsync(out_host, b->d_out, size_t(b->n) * sizeof(tm_result), cudaMemcpyDeviceToHost, s));
  TM_CUDA(cudaStreamSynchronize(s));
  return TM_OK;
}

tm_status tm_batch_folds(tm_batch_t b, int32_t i, void** y, int32_t* is_float) {
  if (!b || !y || i < 0 || i >= b->n) return fail(TM_EINVAL, "bad query index");
  *y = static_cast<char*>(b->d_y) + b->cq[i].y_off * 4;
  if (is_float) *is_float = (b->pc[i].xdtype == TM_F16 || b->pc[i].xdtype == TM_F32) ? 1 : 0;
  return TM_OK;
}

tm_status tm_batch_corr(tm_batch_t b, int32_t i, float** r) {
  if (!b || !r || i < 0 || i >= b->n) return fail(TM_EINVAL, "bad query index");
  if (b->cq[i].r_off < 0) return fail(TM_EINVAL, "batch was created without TM_BATCH_KEEP_CORR");
  *r = b->d_r + b->cq[i].r_off;
  return TM_OK;
}

tm_status tm_batch_stats(tm_batch_t b, int32_t* launches, int32_t* fold_ctas, int64_t* ws) {
  if (!b) return fail(TM_EINVAL, "null batch");
  if (launches) {
    const int32_t nsm = b->n - b->n_blocked - b->n_large;   // queries of the shared-memory correlation
    const int32_t waves = nsm == 0 ? 0 : (b->corr_ctas > 0 ? int32_t(ceil_div(nsm, b->corr_ctas)) : 1);
    int32_t l = waves + (b->n_blocked > 0 ? 1 : 0) + (b->ssum.empty() ? 0 : 1);
    for (const auto& g : b->groups) l += g.W > 0 ? 1 : 0;
    l += b->direct.empty() ? 0 : (b->maxHM_direct > 0 ? 2 : 1);
    if (!b->lq.empty()) l += large_launches(b->lq_two ? 2 : 1);
    *launches = l;
  }
  if (fold_ctas) *fold_ctas = b->nctas;
  if (ws) *ws = b->ws_bytes;
  return TM_OK;
}

tm_status tm_batch_device_error(tm_batch_t b, tm_stream_t stream, int32_t* err) {
  if (!b || !err) return fail(TM_EINVAL, "null argument");
  TM_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  int32_t w[2] = {0, 0};   // pipelined batches alternate between two error words
  TM_CUDA(cudaMemcpy(w, b->d_err, sizeof(w), cudaMemcpyDeviceToHost));
  *err = w[0] | ((b->flags & TM_BATCH_PIPELINED) ? w[1] : 0);
  return TM_OK;
}

tm_status tm_batch_destroy(tm_batch_t b) {
  batch_free(b);
  return TM_OK;
}

tm_status tm_match_batch(const tm_query* q, int32_t n, tm_result* out, tm_stream_t stream) {
  tm_batch_t b = nullptr;
  tm_status st = batch_build(q, n, 0, &b);
  if (st != TM_OK) return st;
  st = tm_batch_run(b, out, stream);
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  batch_free(b);
  if (st != TM_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "tm_match_batch");
  return TM_OK;
}

int32_t tm_crt_candidates(int64_t N, int32_t M1, int32_t M2, int32_t m1, int32_t m2, int64_t* out, int32_t cap) {
  if (N < 1 || M1 < 1 || M2 < 1 || m1 < 0 || m2 < 0 || m1 >= M1 || m2 >= M2 || gcd64(M1, M2) != 1) return -1;
  const CrtSet c = crt_intersect(N, M1, M2, mod_inverse(M1, M2), m1, m2);
  std::vector<int64_t> v;
  for (int64_t j = 0; j < c.nnat && int64_t(v.size()) < int64_t(cap) + 2; ++j) v.push_back(c.m0 + j * c.step);
  for (int k = 0; k < c.nw; ++k) v.push_back(c.w[k]);
  std::sort(v.begin(), v.end());
  const int64_t total = c.nnat + c.nw;
  for (int64_t k = 0; k < std::min<int64_t>(cap, int64_t(v.size())); ++k) out[k] = v[k];
  return int32_t(std::min<int64_t>(total, INT32_MAX));
}

int64_t tm_struct_size(int32_t which) {
  switch (which) {
    case 0: return int64_t(sizeof(tm_plan_desc));
    case 1: return int64_t(sizeof(tm_query));
    case 2: return int64_t(sizeof(tm_result));
    case 3: return int64_t(sizeof(tm_serve_cfg));
    case 4: return int64_t(sizeof(tm_result_tagged));
    case 5: return int64_t(sizeof(tm_serve_stats));
    default: return 0;
  }
}

}  // extern "C"

// ================================================================ no-allocation entry point
// tm_match_noalloc: one query whose scratch lives in a fixed device array
// instead of buffers from cudaMalloc (see tm.h for who needs this).

// The scratch array. In host code its name is only a stand-in: host code
// must use the device address from cudaGetSymbolAddress (noalloc_setup).
static __device__ __align__(256) unsigned char g_tm_noalloc_scratch[TM_NOALLOC_SCRATCH_BYTES];

namespace {

// Layout of the scratch array (byte offsets, 256-aligned).
constexpr size_t kNaErr = 0;                 // int32 error word (cleared by every call)
constexpr size_t kNaOrder = 16;              // int32 processing order (one query: 0)
constexpr size_t kNaJob = 64;                // slot-sum job (used when the fold has many rows)
constexpr size_t kNaFoldQ = 256;             // FoldQ descriptor
constexpr size_t kNaCorrQ = 512;             // CorrQ descriptor
constexpr size_t kNaTw = 1024;               // twiddles W_16384^m, written once per device
constexpr size_t kNaY = kNaTw + size_t(kPMax) * sizeof(float2);      // folds [2][P] int32
constexpr size_t kNaSpec = kNaY + 2 * size_t(kPMax) * sizeof(int32_t);  // template spectrum
constexpr size_t kNaPart = kNaSpec + size_t(kPMax) * sizeof(float2);    // partial fold counts
constexpr size_t kNaPartBytes = TM_NOALLOC_SCRATCH_BYTES - kNaPart;
static_assert(sizeof(FoldQ) <= 256 && sizeof(CorrQ) <= 512 && kNaJob + sizeof(SlotSumJob) <= kNaFoldQ,
              "descriptor slots");

}  // namespace

namespace ftm_noalloc {
// Writes one call's descriptors into the scratch array. They travel as
// kernel parameters (copied by the launch itself), so no host buffer has to
// outlive the call.
__global__ void noalloc_write_descriptors(const FoldQ f, const CorrQ c, const SlotSumJob j, unsigned char* base) {
  const int tid = threadIdx.x;
  if (tid < int(sizeof(SlotSumJob) / 4))
    reinterpret_cast<int*>(base + kNaJob)[tid] = reinterpret_cast<const int*>(&j)[tid];
  if (tid < int(sizeof(FoldQ) / 4)) reinterpret_cast<int*>(base + kNaFoldQ)[tid] = reinterpret_cast<const int*>(&f)[tid];
  if (tid < int(sizeof(CorrQ) / 4)) reinterpret_cast<int*>(base + kNaCorrQ)[tid] = reinterpret_cast<const int*>(&c)[tid];
  if (tid < 4) reinterpret_cast<int*>(base + kNaOrder)[tid] = 0;   // processing order of the one query
  if (tid == 0) *reinterpret_cast<int*>(base + kNaErr) = 0;          // the previous call's error word is stale
}
static_assert(sizeof(FoldQ) % 4 == 0 && sizeof(CorrQ) % 4 == 0 && sizeof(SlotSumJob) % 4 == 0 &&
              sizeof(CorrQ) / 4 <= 256, "descriptor words");
}  // namespace ftm_noalloc

namespace {

std::mutex g_na_mu;
unsigned char* g_na_base[128] = {};   // device address of the array, per device
float2 g_na_tw_host[kPMax];           // host copy of the twiddles (static storage)
bool g_na_tw_ready = false;

// Once per device, with that device current: device address of the array,
// kernel attributes, twiddles.
tm_status noalloc_setup(int dev, unsigned char** base) {
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (dev < 0 || dev >= 128) return fail(TM_EUNSUPPORTED, "device index above 127");
  if (!g_na_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_tm_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    TM_CUDA(fold_configure());
    TM_CUDA(corr_configure());
    if (!g_na_tw_ready) {
      const double two_pi = 6.283185307179586476925286766559;
      for (int m = 0; m < kPMax; ++m) {
        const double ang = two_pi * double(m) / double(kPMax);
        g_na_tw_host[m] = make_float2(float(std::cos(ang)), float(-std::sin(ang)));
      }
      g_na_tw_ready = true;
    }
    TM_CUDA(cudaMemcpy(static_cast<unsigned char*>(p) + kNaTw, g_na_tw_host, sizeof(g_na_tw_host),
                       cudaMemcpyHostToDevice));
    g_na_base[dev] = static_cast<unsigned char*>(p);
  }
  *base = g_na_base[dev];
  return TM_OK;
}

}  // namespace

extern "C" tm_status tm_match_noalloc(const tm_plan_desc* desc, const void* x, const float* t, tm_result* out,
                                      tm_stream_t stream) {
  if (!desc || !x || !t || !out) return fail(TM_EINVAL, "null argument");
  if (reinterpret_cast<uintptr_t>(x) & 15) return fail(TM_EINVAL, "x must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(t) & 3) return fail(TM_EINVAL, "t must be 4-byte aligned");
  PlanCore p;
  tm_status st = make_plan(desc->N, desc->K, desc->xdtype, desc->mode, desc->M1, desc->M2, desc->flags, p, desc->M3);
  if (st != TM_OK) return st;
  if (p.nmod != 2) return fail(TM_EUNSUPPORTED, "the no-allocation entry point uses two moduli (use tm_match)");
  if (p.P > kPMax)
    return fail(TM_EUNSUPPORTED, "the no-allocation entry point handles FFT lengths up to 16384 (use tm_match)");
  if (p.direct)
    return fail(TM_EUNSUPPORTED, "the no-allocation entry point needs moduli the streaming fold holds (use tm_match)");
  if (signal_bytes(p.xdtype, p.N) > TM_NOALLOC_MAX_SIGNAL_BYTES)
    return fail(TM_EUNSUPPORTED, "signal larger than the " + std::to_string(TM_NOALLOC_MAX_SIGNAL_BYTES) +
                                     " bytes the no-allocation entry point accepts (use tm_match)");

  // fold geometry for one signal: equal shares, as many as the array holds
  const int64_t W = fold_bytes(p.xdtype, p.N);
  const int64_t stride = pad16(p.Mp[0]) + pad16(p.Mp[1]);
  const int64_t max_slots = int64_t(kNaPartBytes / sizeof(int32_t)) / stride;
  const int64_t rows_cap = int64_t(kFoldMaxRowsPerSlot - 2) * std::min(p.Mp[0], p.Mp[1]) * fold_geom(p.xdtype).bits / 8;
  int dev = 0, sms = 0;
  TM_CUDA(cudaGetDevice(&dev));
  TM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int64_t nctas = std::min<int64_t>(sms, std::max<int64_t>(1, ceil_div(W, 65536)));
  nctas = std::min(nctas, max_slots);
  if (W > 0 && (nctas < 1 || nctas < ceil_div(W, rows_cap)))
    return fail(TM_EUNSUPPORTED, "query needs more scratch than the " + std::to_string(TM_NOALLOC_SCRATCH_BYTES) +
                                     "-byte no-allocation array holds (use tm_match)");
  unsigned char* base = nullptr;
  st = noalloc_setup(dev, &base);
  if (st != TM_OK) return st;

  FoldQ f{};
  f.x = static_cast<const uint8_t*>(x);
  f.goff = 0;
  f.nbytes = int32_t(W);
  f.Mp[0] = p.Mp[0]; f.Mp[1] = p.Mp[1];
  f.moff[0] = 0; f.moff[1] = int32_t(pad16(p.Mp[0]));
  f.nmod = 2;
  f.stride = int32_t(stride);
  f.first_cta = 0;
  f.part = 0;
  f.nslots = 0;
  if (W > 0) {
    int32_t lo = 0, hi = int32_t(nctas) - 1;   // CTA whose share holds the last byte
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) / 2;
      if (fold_cta_begin(W, int32_t(nctas), mid) <= W - 1) lo = mid; else hi = mid - 1;
    }
    f.nslots = lo + 1;
  }
  CorrQ c{};
  c.x = x; c.t = t; c.N = p.N; c.K = p.K; c.xdtype = p.xdtype; c.nmod = 2;
  for (int j = 0; j < 2; ++j) { c.M[j] = p.M[j]; c.R[j] = p.R[j]; c.L[j] = p.L[j]; c.moff[j] = f.moff[j]; }
  c.P = p.P; c.logP = p.logP; c.inv = p.inv;
  c.thm2 = (p.flags & TM_THM2_SAMPLING) ? 1 : 0;
  c.nelem16 = int32_t(fold_elems(p.xdtype, p.N));
  c.nslots = f.nslots; c.stride = f.stride; c.part = 0;
  c.y_off = 0; c.spec_off = 0; c.r_off = -1;
  SlotSumJob job{};
  const bool ssum = f.nslots >= kSlotSumMin && f.nslots < max_slots;
  if (ssum) {   // the rows' sum in the row after them
    job.src = 0; job.dst = int64_t(f.nslots) * stride;
    job.nslots = f.nslots; job.cols = f.stride;
    job.real = (p.xdtype == TM_F16 || p.xdtype == TM_F32) ? 1 : 0;
    c.nslots = 1;
    c.part = job.dst;
  }

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int32_t* err = reinterpret_cast<int32_t*>(base + kNaErr);
  ftm_noalloc::noalloc_write_descriptors<<<1, 256, 0, s>>>(f, c, job, base);
  TM_CUDA(cudaGetLastError());
  if (W > 0) {
    FoldArgs fa;
    fa.q = reinterpret_cast<const FoldQ*>(base + kNaFoldQ);
    fa.nq = 1; fa.dtype = p.xdtype; fa.nctas = int32_t(nctas); fa.W = W;
    fa.partial = reinterpret_cast<int32_t*>(base + kNaPart);
    fa.err = err;
    const int E = fold_geom(p.xdtype).E;
    const int jmax = std::max(fold_units_per_lane(p.Mp[0], kFoldWarps0, E), fold_units_per_lane(p.Mp[1], kFoldWarps1, E));
    TM_CUDA(launch_fold(fa, jmax, s));
  }
  if (ssum) {
    SlotSumArgs sa;
    sa.partial = reinterpret_cast<int32_t*>(base + kNaPart);
    sa.job = reinterpret_cast<const SlotSumJob*>(base + kNaJob);
    sa.njobs = 1;
    sa.max_cols = job.cols;
    sa.pdl = 1;   // after the fold kernel
    TM_CUDA(launch_slot_sums(sa, s));
  }
  CorrArgs ca;
  ca.q = reinterpret_cast<const CorrQ*>(base + kNaCorrQ);
  ca.order = reinterpret_cast<const int32_t*>(base + kNaOrder);
  ca.nq = 1;
  ca.partial = reinterpret_cast<const int32_t*>(base + kNaPart);
  ca.y = base + kNaY;
  ca.spec = reinterpret_cast<float2*>(base + kNaSpec);
  ca.r = nullptr;
  ca.tw = reinterpret_cast<const float2*>(base + kNaTw);
  ca.out = out;
  ca.err = err;
  ca.pdl = 1;   // after a kernel of this call (descriptors, fold or slot sums)
  ca.lone = 0;  // the descriptor as a kernel parameter too
  ca.q1 = c;
  TM_CUDA(launch_correlate(ca, p.P, s));
  return TM_OK;
}
