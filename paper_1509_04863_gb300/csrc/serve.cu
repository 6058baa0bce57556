// Continuous-batching server (tm_serve_*), see include/tm.h.
//
// A worker thread owns the device work. Each in-flight iteration has a
// stream, a device arena (one allocation at start-up), pinned staging for
// templates, descriptors and results, and an event. The worker loop:
//   1. retire iterations whose event completed: post their results with
//      latencies to the completion queue;
//   2. for each idle stream, take pending requests in arrival order, as many
//      as fit the arena (planned on the host; the batch shrinks until its
//      buffers fit), copy their templates, upload the batch descriptors and
//      launch fold + correlation + result copy on that stream;
//   3. spin briefly while iterations are in flight, otherwise sleep on the
//      submission condition variable.
// Requests that arrive while others run join the next iteration, so work of
// consecutive iterations overlaps on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "runtime.h"

using namespace ftm;

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t tag;
  int32_t sig;
  tm_query q;      // x filled from the signal, t set per iteration
  PlanCore plan;
  std::vector<float> t;
  double t_submit;
  double t_admit = 0.0;   // taken from the queue by the worker
};

struct Signal {
  const void* x;
  int64_t N;
  int32_t dtype;
  bool owned;
};

// Fold cache: the folds over k < M_j of (signal, M1, M2), rows of `pitch`
// entries; `ev` completes when they are written; refs counts in-flight
// iterations reading them, pending is set until the writing iteration
// retires (an entry is dropped only with neither).
using CacheKey = std::tuple<int32_t, int32_t, int32_t, uint32_t>;   // signal, M1, M2, sampling / moduli flags
struct CacheEntry {
  void* y = nullptr;
  int32_t pitch = 0;
  int64_t bytes = 0;
  cudaEvent_t ev = nullptr;
  int refs = 0;
  bool pending = true;
  uint64_t last = 0;
};

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  char* arena = nullptr;
  int64_t arena_bytes = 0;
  char* h_up = nullptr;         // pinned image of the arena's uploaded head (descriptors,
  size_t h_up_cap = 0;          // order, error word, templates): one copy per iteration
  tm_result* h_out = nullptr;   // pinned results
  tm_batch_s* b = nullptr;
  std::vector<Req> reqs;
  std::vector<CacheKey> hits, made;   // fold-cache entries read / written by the iteration
  bool busy = false;
  double t_launched = 0.0;   // the iteration's last launch returned
};

}  // namespace

struct tm_server_s {
  tm_serve_cfg cfg{};
  int device = 0;
  std::vector<Slot> slots;
  std::vector<Signal> signals;
  std::mutex mu;                       // pending, signals
  std::condition_variable cv;
  std::deque<Req> pending;
  std::mutex cmu;                      // completed, stats
  std::condition_variable ccv;
  std::deque<tm_result_tagged> done;
  std::vector<double> lat;             // completed latencies (bounded)
  int64_t submitted = 0, completed = 0, failed = 0, iterations = 0, batched = 0;
  double sum_queue = 0.0, sum_host = 0.0, sum_device = 0.0;   // over completed requests
  std::map<CacheKey, CacheEntry> fcache;   // worker thread only
  int64_t fcache_bytes = 0;
  uint64_t fclock = 0;
  int64_t fc_hits = 0, fc_misses = 0;
  std::atomic<bool> stop{false};
  std::atomic<int> busy{0};            // iterations in flight
  std::thread worker;
};

namespace {

// Arena layout of a planned batch: first the part written from the host
// every iteration (descriptors, processing order, error word, templates),
// then the device-only buffers.
size_t upload_bytes(const tm_batch_s* b, int64_t t_floats) {
  const size_t n = size_t(b->n);
  return align_up(n * sizeof(FoldQ)) + align_up(n * sizeof(CorrQ)) + align_up(n * sizeof(LQ)) +
         align_up(n * sizeof(SlotSumJob)) + align_up(2 * n * sizeof(int32_t)) + align_up(16) +
         align_up(size_t(t_floats) * 4);
}

size_t batch_bytes(const tm_batch_s* b, int64_t t_floats) {
  const size_t n = size_t(b->n);
  return upload_bytes(b, t_floats) + align_up(size_t(b->part_elems) * 4) + align_up(size_t(b->y_elems) * 4) +
         align_up(size_t(b->spec_elems) * sizeof(float2)) + align_up(size_t(b->r_elems) * 4) +
         align_up(n * sizeof(tm_result));
}

void carve(tm_batch_s* b, char* base, int64_t t_floats) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = base + o;
    o += align_up(bytes);
    return p;
  };
  const size_t n = size_t(b->n);
  b->d_fq = reinterpret_cast<FoldQ*>(take(n * sizeof(FoldQ)));
  b->d_cq = reinterpret_cast<CorrQ*>(take(n * sizeof(CorrQ)));
  b->d_lq = reinterpret_cast<LQ*>(take(n * sizeof(LQ)));
  b->d_ssum = reinterpret_cast<SlotSumJob*>(take(n * sizeof(SlotSumJob)));
  b->d_order = reinterpret_cast<int32_t*>(take(2 * n * sizeof(int32_t)));
  b->d_err = reinterpret_cast<int32_t*>(take(16));
  b->d_t = reinterpret_cast<float*>(take(size_t(t_floats) * 4));
  // o == upload_bytes(b, t_floats)
  b->d_partial = reinterpret_cast<int32_t*>(take(size_t(b->part_elems) * 4));
  b->d_y = take(size_t(b->y_elems) * 4);
  b->d_spec = reinterpret_cast<float2*>(take(size_t(b->spec_elems) * sizeof(float2)));
  b->d_r = b->r_elems > 0 ? reinterpret_cast<float*>(take(size_t(b->r_elems) * 4)) : nullptr;
  b->d_out = reinterpret_cast<tm_result*>(take(n * sizeof(tm_result)));
}

void reset_batch(tm_batch_s* b) {
  tm_batch_s fresh;
  fresh.owns_memory = false;
  fresh.h_stage = b->h_stage;
  fresh.stage_bytes = b->stage_bytes;
  fresh.ev_stage = b->ev_stage;
  *b = std::move(fresh);
}

void post(tm_server_t sv, std::vector<tm_result_tagged>& out) {
  std::lock_guard<std::mutex> lk(sv->cmu);
  for (auto& r : out) {
    sv->done.push_back(r);
    if (r.status == TM_OK) {
      ++sv->completed;
      if (sv->lat.size() < (size_t(1) << 22)) sv->lat.push_back(r.latency_us);
    } else {
      ++sv->failed;
    }
  }
  sv->ccv.notify_all();
}

void fail_reqs(tm_server_t sv, std::vector<Req>& reqs, tm_status st) {
  std::vector<tm_result_tagged> out;
  const double t = now_us();
  for (auto& q : reqs) {
    tm_result_tagged r{};
    r.tag = q.tag;
    r.status = st;
    r.latency_us = t - q.t_submit;
    r.r.shift = -1;
    out.push_back(r);
  }
  reqs.clear();
  post(sv, out);
}

// Launch one iteration of `reqs` on slot `sl`; false if it could not be set up.
tm_status launch_iteration(tm_server_t sv, Slot& sl) {
  std::vector<Req>& reqs = sl.reqs;
  const int n = int(reqs.size());
  std::vector<tm_query> qs(n);
  int64_t t_floats = 0;
  std::vector<int64_t> toff(n);
  for (int i = 0; i < n; ++i) {
    toff[i] = t_floats;
    t_floats += pad16(reqs[i].q.K);
  }
  // the template pointers are only known after carving; plan with
  // placeholders (planning reads shapes only), then bind
  for (int i = 0; i < n; ++i) {
    qs[i] = reqs[i].q;
    qs[i].t = reinterpret_cast<const float*>(uintptr_t(16));
  }
  // fold cache lookups: hits skip the fold kernel
  const bool cache_on = sv->cfg.fold_cache_bytes > 0;
  std::vector<uint8_t> nofold(size_t(n), 0);
  std::vector<CacheEntry*> hit(size_t(n), nullptr);
  if (cache_on) {
    for (int i = 0; i < n; ++i) {
      if (reqs[i].plan.P > kPMax) continue;
      auto it = sv->fcache.find(CacheKey(reqs[i].sig, reqs[i].plan.M[0], reqs[i].plan.M[1], reqs[i].plan.flags & (TM_THM2_SAMPLING | TM_THREE_MODULI)));
      if (it != sv->fcache.end()) {
        nofold[i] = 1;
        hit[i] = &it->second;
      }
    }
  }
  reset_batch(sl.b);
  tm_status st = batch_plan(sl.b, qs.data(), n, 0, nofold.data());
  if (st != TM_OK) return st;
  if (batch_bytes(sl.b, t_floats) > size_t(sl.arena_bytes)) return TM_ENOMEM;
  const size_t up = upload_bytes(sl.b, t_floats);
  if (up > sl.h_up_cap) {
    // templates longer than the staging holds (long FFTs): alone, the
    // slot's staging grows (the slot is idle, nothing reads it); with
    // others, the iteration is split
    if (n > 1) return TM_ENOMEM;
    char* h = nullptr;
    if (cudaMallocHost(&h, up) != cudaSuccess) {
      cudaGetLastError();
      return TM_ENOMEM;
    }
    cudaFreeHost(sl.h_up);
    sl.h_up = h;
    sl.h_up_cap = up;
  }
  carve(sl.b, sl.arena, t_floats);
  // the host image of the arena's head, at the same offsets
  char* h = sl.h_up;
  auto at = [&](const void* d) { return h + (static_cast<const char*>(d) - sl.arena); };
  for (int i = 0; i < n; ++i) {
    sl.b->q[i].t = sl.b->d_t + toff[i];
    std::memcpy(at(sl.b->d_t + toff[i]), reqs[i].t.data(), size_t(reqs[i].q.K) * sizeof(float));
  }
  std::memcpy(at(sl.b->d_order), sl.b->order.data(), size_t(n) * sizeof(int32_t));
  if (!sl.b->direct.empty())   // the entry-by-entry folds' query list follows the order
    std::memcpy(at(sl.b->d_order + n), sl.b->direct.data(), sl.b->direct.size() * sizeof(int32_t));
  std::memset(at(sl.b->d_err), 0, 16);   // the error words start clear
  bind_pointers(sl.b);
  for (int i = 0; i < n; ++i) {
    if (!hit[i]) continue;
    sl.b->cq[i].y_core = hit[i]->y;
    sl.b->cq[i].core_pitch = hit[i]->pitch;
    TM_CUDA(cudaStreamWaitEvent(sl.s, hit[i]->ev, 0));
  }
  std::memcpy(at(sl.b->d_fq), sl.b->fq.data(), sl.b->fq.size() * sizeof(FoldQ));
  std::memcpy(at(sl.b->d_cq), sl.b->cq.data(), sl.b->cq.size() * sizeof(CorrQ));
  if (!sl.b->lq.empty()) std::memcpy(at(sl.b->d_lq), sl.b->lq.data(), sl.b->lq.size() * sizeof(LQ));
  if (!sl.b->ssum.empty())
    std::memcpy(at(sl.b->d_ssum), sl.b->ssum.data(), sl.b->ssum.size() * sizeof(SlotSumJob));
  TM_CUDA(cudaMemcpyAsync(sl.arena, h, up, cudaMemcpyHostToDevice, sl.s));
  st = batch_fold(sl.b, sl.s, 0, false);   // the copy cleared the error word
  if (st != TM_OK) return st;
  // results straight into the pinned host array (mapped: the same address
  // on the device), read once the iteration's event has completed
  st = batch_correlate(sl.b, sl.h_out, sl.s, 0, true);
  if (st != TM_OK) return st;
  TM_CUDA(cudaEventRecord(sl.ev, sl.s));
  if (cache_on) {
    sl.hits.clear();
    sl.made.clear();
    for (int i = 0; i < n; ++i) {
      if (!hit[i]) continue;
      ++hit[i]->refs;
      hit[i]->last = ++sv->fclock;
      sl.hits.emplace_back(reqs[i].sig, reqs[i].plan.M[0], reqs[i].plan.M[1], reqs[i].plan.flags & (TM_THM2_SAMPLING | TM_THREE_MODULI));
    }
    int64_t nh = 0;
    for (int i = 0; i < n; ++i) nh += hit[i] ? 1 : 0;
    {
      std::lock_guard<std::mutex> lk(sv->cmu);
      sv->fc_hits += nh;
      sv->fc_misses += n - nh;
    }
    // new entries from this iteration's folds (copied once it has run)
    for (int i = 0; i < n; ++i) {
      if (hit[i] || reqs[i].plan.P > kPMax) continue;
      const CacheKey key(reqs[i].sig, reqs[i].plan.M[0], reqs[i].plan.M[1], reqs[i].plan.flags & (TM_THM2_SAMPLING | TM_THREE_MODULI));
      if (sv->fcache.count(key)) continue;
      const int rows = reqs[i].plan.nmod;
      const int32_t pitch = std::max(std::max(reqs[i].plan.M[0], reqs[i].plan.M[1]), rows == 3 ? reqs[i].plan.M[2] : 0);
      const int64_t bytes = rows * int64_t(pitch) * 4;
      // drop least recently used entries that nothing reads or writes
      while (sv->fcache_bytes + bytes > sv->cfg.fold_cache_bytes) {
        auto victim = sv->fcache.end();
        for (auto it = sv->fcache.begin(); it != sv->fcache.end(); ++it)
          if (it->second.refs == 0 && !it->second.pending &&
              (victim == sv->fcache.end() || it->second.last < victim->second.last))
            victim = it;
        if (victim == sv->fcache.end()) break;
        cudaFreeAsync(victim->second.y, sl.s);
        cudaEventDestroy(victim->second.ev);
        sv->fcache_bytes -= victim->second.bytes;
        sv->fcache.erase(victim);
      }
      if (sv->fcache_bytes + bytes > sv->cfg.fold_cache_bytes) continue;
      CacheEntry e;
      e.pitch = pitch;
      e.bytes = bytes;
      e.last = ++sv->fclock;
      if (cudaMallocAsync(&e.y, size_t(bytes), sl.s) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      const char* src = static_cast<const char*>(sl.b->d_y) + sl.b->cq[i].y_off * 4;
      if (cudaMemcpy2DAsync(e.y, size_t(pitch) * 4, src, size_t(sl.b->cq[i].P) * 4, size_t(pitch) * 4, size_t(rows),
                            cudaMemcpyDeviceToDevice, sl.s) != cudaSuccess ||
          cudaEventCreateWithFlags(&e.ev, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventRecord(e.ev, sl.s) != cudaSuccess) {
        cudaGetLastError();
        if (e.ev) cudaEventDestroy(e.ev);
        cudaFreeAsync(e.y, sl.s);
        continue;
      }
      sv->fcache_bytes += bytes;
      sv->fcache.emplace(key, e);
      sl.made.push_back(key);
    }
  }
  return TM_OK;
}

// Take the next requests that fit the arena of `sl` (in arrival order).
void admit(tm_server_t sv, Slot& sl) {
  std::vector<Req> take;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    const size_t k = std::min<size_t>(sv->pending.size(), size_t(sv->cfg.max_batch));
    for (size_t i = 0; i < k; ++i) {
      take.push_back(std::move(sv->pending.front()));
      sv->pending.pop_front();
    }
  }
  const double t_admit = now_us();
  for (auto& r : take) r.t_admit = t_admit;
  while (!take.empty()) {
    sl.reqs = std::move(take);
    take.clear();
    const tm_status st = launch_iteration(sv, sl);
    if (st == TM_OK) {
      sl.t_launched = now_us();
      sl.busy = true;
      sv->busy.fetch_add(1);
      std::lock_guard<std::mutex> lk(sv->cmu);
      ++sv->iterations;
      sv->batched += int64_t(sl.reqs.size());
      return;
    }
    if (st == TM_ENOMEM && sl.reqs.size() > 1) {
      // too large for the arena: return the newer half to the queue front
      const size_t keep = sl.reqs.size() / 2;
      std::lock_guard<std::mutex> lk(sv->mu);
      for (size_t i = sl.reqs.size(); i-- > keep;) sv->pending.push_front(std::move(sl.reqs[i]));
      sl.reqs.resize(keep);
      take = std::move(sl.reqs);
      continue;
    }
    fail_reqs(sv, sl.reqs, st);
    return;
  }
}

// The iteration on `sl` no longer reads or writes its fold-cache entries.
void release_cache(tm_server_t sv, Slot& sl) {
  for (const auto& k : sl.hits) {
    auto it = sv->fcache.find(k);
    if (it != sv->fcache.end()) --it->second.refs;
  }
  for (const auto& k : sl.made) {
    auto it = sv->fcache.find(k);
    if (it != sv->fcache.end()) it->second.pending = false;
  }
  sl.hits.clear();
  sl.made.clear();
}

void retire(tm_server_t sv, Slot& sl) {
  release_cache(sv, sl);
  const double t = now_us();
  std::vector<tm_result_tagged> out(sl.reqs.size());
  double q = 0.0, h = 0.0;
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    out[i].tag = sl.reqs[i].tag;
    out[i].status = TM_OK;
    out[i].latency_us = t - sl.reqs[i].t_submit;
    out[i].r = sl.h_out[i];
    q += sl.reqs[i].t_admit - sl.reqs[i].t_submit;
    h += sl.t_launched - sl.reqs[i].t_admit;
  }
  {
    std::lock_guard<std::mutex> lk(sv->cmu);
    sv->sum_queue += q;
    sv->sum_host += h;
    sv->sum_device += double(sl.reqs.size()) * (t - sl.t_launched);
  }
  sl.reqs.clear();
  sl.busy = false;
  sv->busy.fetch_sub(1);
  post(sv, out);
}

void worker_main(tm_server_t sv) {
  cudaSetDevice(sv->device);
  double t_last = now_us();   // last time the worker had something to do
  while (true) {
    bool progressed = false, any_busy = false;
    for (auto& sl : sv->slots) {
      if (!sl.busy) continue;
      const cudaError_t e = cudaEventQuery(sl.ev);
      if (e == cudaSuccess) {
        retire(sv, sl);
        progressed = true;
      } else if (e != cudaErrorNotReady) {
        cudaGetLastError();
        release_cache(sv, sl);
        sl.busy = false;
        sv->busy.fetch_sub(1);
        fail_reqs(sv, sl.reqs, TM_ECUDA);
        progressed = true;
      } else {
        any_busy = true;
      }
    }
    bool have_pending;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      have_pending = !sv->pending.empty();
    }
    if (have_pending) {
      for (auto& sl : sv->slots) {
        if (sl.busy) continue;
        admit(sv, sl);
        progressed = true;
        break;
      }
    }
    if (sv->stop.load() && !have_pending && !any_busy) break;
    if (progressed || any_busy) t_last = now_us();
    if (!progressed) {
      if (any_busy || now_us() - t_last < double(sv->cfg.idle_spin_us)) {
        std::this_thread::yield();
      } else {
        std::unique_lock<std::mutex> lk(sv->mu);
        sv->cv.wait_for(lk, std::chrono::milliseconds(2),
                        [&] { return !sv->pending.empty() || sv->stop.load(); });
      }
    }
  }
}

void server_free(tm_server_t sv) {
  for (auto& sl : sv->slots) {
    if (sl.s) cudaStreamSynchronize(sl.s);
    if (sl.b) batch_free(sl.b);   // destroys the staging event, not the arena
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.s) cudaStreamDestroy(sl.s);
    cudaFree(sl.arena);
    if (sl.h_up) cudaFreeHost(sl.h_up);
    if (sl.h_out) cudaFreeHost(sl.h_out);
  }
  for (auto& kv : sv->fcache) {
    cudaFree(kv.second.y);
    if (kv.second.ev) cudaEventDestroy(kv.second.ev);
  }
  for (auto& sg : sv->signals)
    if (sg.owned) cudaFree(const_cast<void*>(sg.x));
  delete sv;
}

}  // namespace

extern "C" {

tm_status tm_serve_create(const tm_serve_cfg* cfg_in, tm_server_t* out) {
  if (!out) return fail(TM_EINVAL, "null output handle");
  *out = nullptr;
  tm_serve_cfg cfg = cfg_in ? *cfg_in : tm_serve_cfg{};
  if (cfg.n_streams <= 0) cfg.n_streams = 2;
  if (cfg.n_streams > 4) return fail(TM_EINVAL, "n_streams must be 1..4");
  if (cfg.max_batch <= 0) cfg.max_batch = 512;
  if (cfg.queue_capacity <= 0) cfg.queue_capacity = 65536;
  if (cfg.idle_spin_us < 0) return fail(TM_EINVAL, "idle_spin_us must be >= 0");
  if (cfg.flags & ~TM_SERVE_FINE_PIECES) return fail(TM_EINVAL, "unknown server flag");
  if (cfg.hbm_reserve_bytes <= 0) cfg.hbm_reserve_bytes = int64_t(4) << 30;
  tm_server_t sv = new (std::nothrow) tm_server_s();
  if (!sv) return fail(TM_ENOMEM, "host allocation");
  cudaError_t e = cudaGetDevice(&sv->device);
  if (e != cudaSuccess) { delete sv; return cuda_fail(e, "cudaGetDevice"); }
  float2* tw = nullptr;
  tm_status st = device_setup(sv->device, &tw);
  if (st != TM_OK) { delete sv; return st; }
  if (cfg.arena_bytes <= 0) {
    size_t freeb = 0, total = 0;
    e = cudaMemGetInfo(&freeb, &total);
    if (e != cudaSuccess) { delete sv; return cuda_fail(e, "cudaMemGetInfo"); }
    const int64_t usable = int64_t(freeb) - cfg.hbm_reserve_bytes;
    if (usable < (int64_t(64) << 20)) { delete sv; return fail(TM_ENOMEM, "not enough free device memory"); }
    cfg.arena_bytes = std::min<int64_t>(usable / cfg.n_streams, int64_t(8) << 30);
  }
  sv->cfg = cfg;
  sv->slots.resize(cfg.n_streams);
  // upload staging: descriptors and order for max_batch requests and
  // templates of 8192 entries on average; a larger iteration is split
  const size_t nb = size_t(cfg.max_batch);
  const size_t up_cap = align_up(nb * sizeof(FoldQ)) + align_up(nb * sizeof(CorrQ)) + align_up(nb * sizeof(LQ)) +
                        align_up(nb * sizeof(SlotSumJob)) + align_up(2 * nb * sizeof(int32_t)) + align_up(16) +
                        align_up(std::max<size_t>(nb * 8192, 65536) * sizeof(float));
  for (auto& sl : sv->slots) {
    bool ok = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&sl.arena, size_t(cfg.arena_bytes)) == cudaSuccess &&
              cudaMallocHost(&sl.h_up, up_cap) == cudaSuccess &&
              cudaMallocHost(&sl.h_out, size_t(cfg.max_batch) * sizeof(tm_result)) == cudaSuccess;
    sl.arena_bytes = cfg.arena_bytes;
    sl.h_up_cap = up_cap;
    if (ok) {
      sl.b = new (std::nothrow) tm_batch_s();
      ok = sl.b != nullptr && cudaEventCreateWithFlags(&sl.b->ev_stage, cudaEventDisableTiming) == cudaSuccess;
      if (ok) sl.b->owns_memory = false;
    }
    if (!ok) {
      cudaGetLastError();
      server_free(sv);
      return fail(TM_ENOMEM, "server allocation failed");
    }
  }
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return TM_OK;
}

tm_status tm_serve_register_signal(tm_server_t sv, const void* x, int64_t N, int32_t xdtype, uint32_t flags,
                                   int32_t* sig_id) {
  if (!sv || !x || !sig_id) return fail(TM_EINVAL, "null argument");
  if (N < 1 || xdtype < TM_I8_PM1 || xdtype > TM_F32) return fail(TM_EINVAL, "bad signal shape");
  Signal sg{x, N, xdtype, false};
  if (!(flags & TM_SERVE_SIGNAL_DEVICE)) {
    void* d = nullptr;
    const size_t bytes = size_t(signal_bytes(xdtype, N));
    TM_CUDA(cudaSetDevice(sv->device));
    TM_CUDA(cudaMalloc(&d, bytes));
    const cudaError_t e = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return cuda_fail(e, "signal upload"); }
    sg.x = d;
    sg.owned = true;
  } else if (reinterpret_cast<uintptr_t>(x) & 15) {
    return fail(TM_EINVAL, "x must be 16-byte aligned");
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->signals.push_back(sg);
  *sig_id = int32_t(sv->signals.size() - 1);
  return TM_OK;
}

namespace {

// A request record: plan, query shape, a copy of the template.
tm_status build_request(tm_server_t sv, int32_t sig_id, const float* t_host, int32_t K, int32_t mode, int32_t M1,
                        int32_t M2, uint32_t plan_flags, uint64_t tag, Req& r) {
  if (!t_host) return fail(TM_EINVAL, "null template");
  if (K < 1) return fail(TM_EINVAL, "empty template");
  if (sv->cfg.flags & TM_SERVE_FINE_PIECES) plan_flags |= TM_FINE_PIECES;
  r.tag = tag;
  r.sig = sig_id;
  Signal sg;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sig_id < 0 || sig_id >= int32_t(sv->signals.size())) return fail(TM_EINVAL, "unknown signal id");
    sg = sv->signals[sig_id];
  }
  tm_status st = make_plan(sg.N, K, sg.dtype, mode, M1, M2, plan_flags, r.plan);
  if (st != TM_OK) return st;
  r.q.x = sg.x;
  r.q.t = nullptr;
  r.q.N = sg.N;
  r.q.K = K;
  r.q.xdtype = sg.dtype;
  r.q.mode = mode;
  r.q.M1 = M1;
  r.q.M2 = M2;
  r.q.flags = plan_flags;
  r.t.assign(t_host, t_host + K);
  r.t_submit = now_us();
  return TM_OK;
}

// Queues reqs[0..n) in order while the queue has room; returns how many.
int32_t enqueue_requests(tm_server_t sv, std::vector<Req>& reqs, int32_t n) {
  int32_t k = 0;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    while (k < n && int64_t(sv->pending.size()) < sv->cfg.queue_capacity) sv->pending.push_back(std::move(reqs[k++]));
  }
  if (k > 0) {
    {
      std::lock_guard<std::mutex> lk(sv->cmu);
      sv->submitted += k;
    }
    sv->cv.notify_one();
  }
  return k;
}

}  // namespace

tm_status tm_serve_submit(tm_server_t sv, int32_t sig_id, const float* t_host, int32_t K, int32_t mode, int32_t M1,
                          int32_t M2, uint32_t plan_flags, uint64_t tag) {
  if (!sv || !t_host) return fail(TM_EINVAL, "null argument");
  std::vector<Req> r(1);
  tm_status st = build_request(sv, sig_id, t_host, K, mode, M1, M2, plan_flags, tag, r[0]);
  if (st != TM_OK) return st;
  if (enqueue_requests(sv, r, 1) == 0) return fail(TM_EAGAIN, "queue full");
  return TM_OK;
}

int32_t tm_serve_submit_many(tm_server_t sv, int32_t n, const int32_t* sig_ids, const float* const* t_host,
                             const int32_t* K, int32_t mode, uint32_t plan_flags, const uint64_t* tags) {
  if (!sv || n < 0 || (n > 0 && (!sig_ids || !t_host || !K || !tags)))
    return -int32_t(fail(TM_EINVAL, "null argument"));
  std::vector<Req> reqs(size_t(n > 0 ? n : 0));
  for (int32_t i = 0; i < n; ++i) {
    const tm_status st = build_request(sv, sig_ids[i], t_host[i], K[i], mode, 0, 0, plan_flags, tags[i], reqs[i]);
    if (st != TM_OK) {
      // the valid prefix still goes in; the caller learns where it stopped
      const int32_t k = enqueue_requests(sv, reqs, i);
      return k > 0 ? k : -int32_t(st);
    }
  }
  return enqueue_requests(sv, reqs, n);
}

int32_t tm_serve_poll(tm_server_t sv, tm_result_tagged* out, int32_t max, int64_t timeout_us) {
  if (!sv || !out || max < 1) return -int32_t(fail(TM_EINVAL, "bad poll arguments"));
  std::unique_lock<std::mutex> lk(sv->cmu);
  if (sv->done.empty() && timeout_us > 0)
    sv->ccv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !sv->done.empty(); });
  int32_t k = 0;
  while (k < max && !sv->done.empty()) {
    out[k++] = sv->done.front();
    sv->done.pop_front();
  }
  return k;
}

tm_status tm_serve_stats_get(tm_server_t sv, tm_serve_stats* st) {
  if (!sv || !st) return fail(TM_EINVAL, "null argument");
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lk(sv->cmu);
    st->submitted = sv->submitted;
    st->completed = sv->completed;
    st->failed = sv->failed;
    st->iterations = sv->iterations;
    st->mean_batch = sv->iterations ? double(sv->batched) / double(sv->iterations) : 0.0;
    st->fold_cache_hits = sv->fc_hits;
    st->fold_cache_misses = sv->fc_misses;
    const double nc = sv->completed > 0 ? double(sv->completed) : 1.0;
    st->queue_us = sv->sum_queue / nc;
    st->host_us = sv->sum_host / nc;
    st->device_us = sv->sum_device / nc;
    lat = sv->lat;
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    st->pending = int64_t(sv->pending.size());
  }
  st->in_flight = sv->busy.load();
  st->p50_us = st->p99_us = st->max_us = 0.0;
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    st->p50_us = lat[lat.size() / 2];
    st->p99_us = lat[std::min(lat.size() - 1, size_t(double(lat.size()) * 0.99))];
    st->max_us = lat.back();
  }
  return TM_OK;
}

tm_status tm_serve_destroy(tm_server_t sv) {
  if (!sv) return TM_OK;
  sv->stop.store(true);
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  server_free(sv);
  return TM_OK;
}

}  // extern "C"
