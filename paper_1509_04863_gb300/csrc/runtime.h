// Host runtime shared by the C ABI (api.cu) and the server (serve.cu):
// planning, batch layouts and launches.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "tm_internal.h"

namespace ftm {

// Error reporting: sets the calling thread's message (tm_last_error).
tm_status fail(tm_status s, const std::string& msg);
tm_status cuda_fail(cudaError_t e, const char* what);
std::string& last_error();

#define TM_CUDA(call)                                           \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return ::ftm::cuda_fail(e_, #call);  \
  } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t pad16(int64_t v) { return (v + 15) & ~int64_t(15); }

struct PlanCore {
  int64_t N = 0;
  int32_t K = 0, xdtype = 0;
  int32_t nmod = 2;                 // moduli of step 2 (3 with TM_THREE_MODULI)
  int32_t M[3] = {0, 0, 0};
  int64_t L[3] = {0, 0, 0};
  int32_t P = 0, logP = 0;
  int32_t inv = 0;                  // M1^-1 mod M2
  int32_t inv3 = 0;                 // (M1 M2)^-1 mod M3
  int32_t R[3] = {1, 1, 1}, Mp[3] = {0, 0, 0};
  int64_t max_cand = 0;
  uint32_t flags = 0;   // TM_ALLOW_AMBIG, TM_THM2_SAMPLING, TM_THREE_MODULI
  int32_t direct = 0;   // moduli too wide for the streaming fold: entry-by-entry fold
  int32_t large = 0;    // FFT longer than the blocked correlation: multi-CTA passes
};


// Algorithm 1 step 2 and the derived sizes (host only).
tm_status make_plan(int64_t N, int32_t K, int32_t xdtype, int32_t mode, int32_t M1, int32_t M2, uint32_t flags,
                    PlanCore& pc, int32_t M3 = 0);
int64_t signal_bytes(int32_t dtype, int64_t N);
int64_t fold_bytes(int32_t dtype, int64_t N);
int64_t fold_elems(int32_t dtype, int64_t N);
// Once per device: kernel attributes and the twiddle table.
tm_status device_setup(int dev, float2** tw);

}  // namespace ftm

struct tm_batch_s {
  bool owns_memory = true;   // false: device buffers belong to a server arena
  int device = 0;
  uint32_t flags = 0;
  int32_t n = 0;
  std::vector<ftm::PlanCore> pc;
  std::vector<tm_query> q;
  std::vector<ftm::FoldQ> fq;
  std::vector<ftm::CorrQ> cq;
  std::vector<int32_t> order;
  std::vector<int64_t> xoff, toff;   // device input copies (TM_BATCH_HOST_INPUTS)
  // One fold launch per signal storage type present: its queries occupy
  // fq[first, first + count) (fq is ordered by group), fold_of[i] is the
  // fq position of query i.
  struct FoldGroup {
    int32_t dtype, first, count, nctas, jmax;
    int64_t W;
    int32_t tile = ftm::kFoldTile;   // stage bytes (tm_batch_autotune may change it)
    std::vector<int64_t> cb;         // share starts on piece boundaries (real signals), else empty
  };
  std::vector<FoldGroup> groups;
  std::vector<int32_t> fold_of;
  int32_t nctas = 0;   // largest fold grid
  int64_t W = 0;       // bytes folded in total
  int32_t maxP = 0;        // largest FFT of the shared-memory correlation launch
  std::vector<int32_t> direct;   // queries folded entry by entry (fold_direct)
  int32_t maxP_direct = 0, maxmod_direct = 0, maxM_direct = 0, maxHM_direct = 0;
  std::vector<int32_t> dh, drows, dpitch;   // entry-by-entry folds: row groups, rows per group, row pitch, partial offsets
  std::vector<int64_t> dpart;
  std::vector<ftm::SlotSumJob> ssum;   // folds whose rows are summed ahead of the correlation
  std::vector<int32_t> ssum_of;        // fold descriptor -> job (-1: none)
  int32_t ssum_cols = 0;               // longest row among them
  int32_t n_blocked = 0;   // queries correlated in blocks (order[n - n_large - n_blocked, n - n_large))
  int32_t n_large = 0;     // queries on the multi-CTA path (order[n - n_large, n))
  std::vector<uint8_t> is_large;
  std::vector<ftm::LQ> lq;  // their launch descriptors, in the order of the all-SM launches
  std::vector<int32_t> lq_of;   // query -> position in lq (-1: not on that path)
  int32_t lq_maxP = 0, lq_maxM = 0, lq_two = 0;
  ftm::LQ* d_lq = nullptr;
  ftm::SlotSumJob* d_ssum = nullptr;   // the slot-sum jobs (device copy of ssum)
  int64_t y_elems = 0, spec_elems = 0, r_elems = 0, part_elems = 0;
  ftm::FoldQ* d_fq = nullptr;
  ftm::CorrQ* d_cq = nullptr;
  int32_t* d_order = nullptr;
  int32_t* d_partial = nullptr;
  void* d_y = nullptr;
  float2* d_spec = nullptr;
  float* d_r = nullptr;
  int32_t* d_err = nullptr;
  tm_result* d_out = nullptr;
  uint8_t* d_x = nullptr;
  float* d_t = nullptr;
  float2* tw = nullptr;
  // pinned staging for descriptor uploads, guarded by an event
  void* h_stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t ev_stage = nullptr;
  // long-FFT queries: their template spectra run on aux beside the fold
  // (fork on the caller's stream before the fold launches, join before
  // the signal spectra); only batches that own their memory have aux
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool tpl_pending = false;
  int64_t ws_bytes = 0;
  // tm_batch_graph_capture: the captured run and the stream it was captured on
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // launch geometry (tm_batch_set_grid): most fold CTAs (0: one per SM) and
  // most correlation CTAs at a time (0: one per query)
  int32_t fold_cap = 0, corr_ctas = 0;
  int64_t part_alloc = 0;   // int32 entries allocated for each partial buffer
  // pipelined runs (TM_BATCH_PIPELINED): a second partial buffer, the
  // correlation's stream, the fork/join events, and the run whose
  // correlation is still to come
  int32_t* d_partial2 = nullptr;
  cudaStream_t cstream = nullptr;
  cudaEvent_t ev_pfork = nullptr, ev_pjoin = nullptr;
  int32_t pp = 0;                 // partial buffer of the next fold
  bool pending = false;
  tm_result* pending_out = nullptr;
};


namespace ftm {

// Host layout of a batch (plans, fold groups, descriptors, order, sizes);
// needs the device that will run it to be current (SM count, twiddles).
// nofold (optional, n entries): queries whose folds come from elsewhere
// (CorrQ::y_core); the fold kernel does not read their signals.
tm_status batch_plan(tm_batch_s* b, const tm_query* q, int32_t n, uint32_t flags,
                     const uint8_t* nofold = nullptr);
// Device buffers from cudaMalloc (owns_memory) and pinned staging.
tm_status batch_alloc(tm_batch_s* b);
void batch_free(tm_batch_s* b);
void bind_pointers(tm_batch_s* b);
tm_status upload_descriptors(tm_batch_s* b, cudaStream_t s);
// parity: which partial buffer and error word (pipelined batches alternate)
// clear_err: reset the parity's error word on `s` first (pipelined runs
// reset it on the correlation stream instead, after its last reader)
tm_status batch_fold(tm_batch_s* b, cudaStream_t s, int parity = 0, bool clear_err = true);
// after_fold: the last operation on s is this batch's batch_fold, so the
// first correlation launch may be a programmatic dependent of its kernels
tm_status batch_correlate(tm_batch_s* b, tm_result* out, cudaStream_t s, int parity = 0, bool after_fold = false);

}  // namespace ftm
