/*
 * tm.h - C ABI of a GB300 (sm_103a) implementation of the fast template
 * matcher of Hsieh, Lu & Pei, "Fast Template Matching by Subsampled
 * Circulant Matrix" (arXiv 1509.04863).
 *
 * Problem (Sec. 1 Eq. (1), Sec. 3): given a signal x in R^N and a template
 * t in R^K, find the cyclic shift m maximising the cross-correlation
 *     (Tx)_k = sum_{i<K} t_i x_{(k+i) mod N},   0 <= k < N.
 * Method (Algorithm 1): fold x with two co-prime moduli M1, M2 into
 * y_{M}[k] = sum_{i<ceil(N/M)} x_{(k+iM) mod N}, k < M+K-1 (step 3, Eq. (2)),
 * correlate each fold with t by FFT (steps 4-6), take the argmax over
 * j < M (step 7) and intersect the candidate sets {m~ + i M mod N} (steps
 * 8-9, Thm. 4).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are CUDA device pointers, *_host host pointers.
 *    The caller owns every buffer it passes; the library never frees them.
 *  - Streams: tm_stream_t is the same type as cudaStream_t (NULL = the
 *    legacy default stream). Work is asynchronous; outputs are valid once
 *    the stream has synchronised.
 *  - Errors: every call returns a tm_status; nothing aborts or exits.
 *    tm_last_error() gives a message for the calling thread's last error.
 *  - Signals must be 16-byte aligned on the device; templates 4-byte.
 *  - Inputs must be finite. +-1 int8 signals must hold only 0x01 or 0xFF.
 */
#ifndef TM_H_
#define TM_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TM_API __attribute__((visibility("default")))
#else
#define TM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tm_stream_t;
typedef struct CUevent_st* tm_event_t;   /* the same type as cudaEvent_t */

typedef enum {
  TM_OK = 0,
  TM_EINVAL = 1,        /* invalid argument or plan (see tm_last_error) */
  TM_ENOMEM = 2,        /* device or host allocation failed */
  TM_ECUDA = 3,         /* a CUDA runtime call failed (no GPU, launch error) */
  TM_EBUSY = 4,         /* server: no free slot or memory right now */
  TM_ETIMEDOUT = 5,     /* a bounded wait (host or device) ran out */
  TM_EAGAIN = 6,        /* server: queue full, retry later */
  TM_EUNSUPPORTED = 7   /* valid request outside what this build handles */
} tm_status;

/* Signal storage. TM_BITS_PM1 packs one element per bit, least significant
 * bit first; bit 1 is +1 and bit 0 is -1. */
typedef enum { TM_I8_PM1 = 0, TM_BITS_PM1 = 1, TM_F16 = 2, TM_F32 = 3 } tm_dtype;

/* Choice of the co-prime moduli (Algorithm 1 step 2).
 *  PAPER:    M1 = K, M2 = K+1 (Sec. 3.5 proof of Thm. 5; Sec. 4).
 *  AUTO:     M1 = max(K, s), M2 = M1+1, s the least integer with s(s+1) > N,
 *            so that M1*M2 > N as step 2 requires.
 *  EXPLICIT: the caller's M1, M2 (co-prime, both >= K). */
typedef enum { TM_MODE_AUTO = 0, TM_MODE_PAPER = 1, TM_MODE_EXPLICIT = 2 } tm_mode;

/* Plan flag: accept M1*M2 <= N. The intersection of step 9 may then hold
 * several shifts; they are resolved by their exact (Tx)_m. */
#define TM_ALLOW_AMBIG 0x1u
/* Plan flag: step 3 with the second sampling matrix of Thm. 2, Phi =
 * [I_M ... I_M] on x zero-padded to a multiple of M (no wrap-around term),
 * and steps 4-6 as the circular correlation of period M with the template
 * (y extended periodically); candidate positions in the padding are
 * dropped in step 8. */
#define TM_THM2_SAMPLING 0x2u
/* Plan flag: step 2 with three pairwise co-prime moduli M1 < M2 < M3 (Thm.
 * 4: the residues determine the shift once M1 M2 M3 > N, which holds for
 * much smaller K than M1 M2 > N). PAPER: c, c+1, c+2 from the least odd
 * c >= K; AUTO: from the least odd c >= max(K, s), s(s+1)(s+2) > N;
 * EXPLICIT: M1, M2, M3 as given. Steps 3-8 run for each modulus and step 9
 * intersects the three candidate sets. FFT lengths up to 16384; no
 * slices, no Thm. 2 sampling with it. */
#define TM_THREE_MODULI 0x4u
/* Plan flag (no counterpart in the paper; real signals only): the fold of
 * step 3 cuts an fp16/fp32 signal into pieces of at least 256 KiB (at most
 * 128 per signal) instead of at least 2 MiB (at most 64), one partial row
 * of R1 M1 + R2 M2 fp32 sums per piece. A signal folded alone then spreads
 * over up to 8x more CTAs (lower latency) at the price of more partial-sum
 * traffic in large batches. The fp32 sums are added in another order, so
 * results depend on the flag; with a given flag they do not depend on the
 * rest of the batch. */
#define TM_FINE_PIECES 0x8u

/* tm_result.status values (low byte) and flag bits. */
#define TM_FOUND 0      /* |S1 ∩ S2| = 1 */
#define TM_EMPTY 1      /* |S1 ∩ S2| = 0; shift = -1 */
#define TM_RESOLVED 2   /* |S1 ∩ S2| > 1; best exact (Tx)_m, ties -> smallest m */
#define TM_RF_FULL_RESCORE 0x100  /* too many near-maximal r_j: all j rescored */
#define TM_RF_DEVICE_ERROR 0x200  /* a device-side bounded wait ran out */
#define TM_RF_SCORE_PENDING 0x400 /* tm_correlate_folds: no signal, so the member(s)
                                     of S1 ∩ S2 are unscored; shift = the first
                                     member, to be resolved by the caller */
#define TM_RF_UNCERTIFIED 0x800   /* FFT lengths above 2^18 only: more than 4096
                                     indices lay within the FFT rounding bound of
                                     the maximum and M K > 2^36, so m_j is the
                                     largest FFT value (smallest index among
                                     equal ones), not proven the exact argmax */

typedef struct {
  int64_t N;       /* signal length, 1 <= N */
  int32_t K;       /* template length, 1 <= K <= N */
  int32_t xdtype;  /* tm_dtype */
  int32_t mode;    /* tm_mode */
  int32_t M1, M2;  /* only read for TM_MODE_EXPLICIT */
  uint32_t flags;  /* TM_ALLOW_AMBIG, TM_THM2_SAMPLING, TM_THREE_MODULI */
  int32_t M3;      /* only read for TM_MODE_EXPLICIT with TM_THREE_MODULI */
  int32_t reserved;
} tm_plan_desc;

typedef struct {
  int64_t N;
  int32_t K, xdtype;
  int32_t M1, M2;  /* moduli of step 2 */
  int64_t L1, L2;  /* ceil(N/M1), ceil(N/M2): terms per fold entry (Eq. (2)) */
  int32_t P;       /* FFT length: the least power of two >= max(M1,M2)+K-1 */
  int32_t max_cand;/* bound on |S1 ∩ S2|: ceil(N/(M1*M2)) + 2 */
  int32_t M3;      /* third modulus (TM_THREE_MODULI), else 0 */
  int32_t reserved;
  int64_t L3;
} tm_plan_info;

/* One matching result (64 bytes), written to device memory. */
typedef struct {
  int64_t shift;   /* recovered m^ in [0, N), or -1 (TM_EMPTY) */
  int32_t status;  /* TM_FOUND / TM_EMPTY / TM_RESOLVED | TM_RF_* flags */
  int32_t n_cand;  /* |S1 ∩ S2| (∩ S3 with TM_THREE_MODULI) */
  int32_t m1, m2;  /* step-7 maxima m~1 < M1, m~2 < M2 */
  double r1, r2;   /* exact r_{M1}[m~1], r_{M2}[m~2] (rescored, see below) */
  double score;    /* exact (Tx)_shift, 0 when shift = -1 */
  int32_t m3;      /* TM_THREE_MODULI: m~3 < M3 and its exact r; else 0 */
  int32_t reserved;
  double r3;
} tm_result;

/* One query of a batch. */
typedef struct {
  const void* x;   /* signal storage (device, 16-byte aligned) */
  const float* t;  /* template, K floats (device) */
  int64_t N;
  int32_t K;
  int32_t xdtype;
  int32_t mode;
  int32_t M1, M2;
  uint32_t flags;
  int32_t M3;
  int32_t reserved;
} tm_query;

/* ------------------------------------------------------------------ misc */

/* Library version string. */
TM_API const char* tm_version(void);
/* Message of the calling thread's last failed call ("" if none). */
TM_API const char* tm_last_error(void);

/* ------------------------------------------------------------------ plan */

typedef struct tm_plan_s* tm_plan_t;

/* Validate a problem and choose M1, M2 (Algorithm 1 step 2) and the FFT
 * length P >= max(M)+K-1 (steps 4-5 zero-pad t and y to a common length).
 * Host only; needs no GPU. TM_EINVAL when K < 1, K > N, M_i < K, M_i > 2N,
 * gcd(M1, M2) != 1, or M1*M2 <= N without TM_ALLOW_AMBIG;
 * TM_EUNSUPPORTED when P > 2^26 (2^14 with TM_THREE_MODULI) or the byte
 * size of x exceeds 2^31-2^16. FFT lengths up to 16384 run in shared
 * memory, one CTA per query; longer ones in overlap-save blocks (a CTA per
 * query, batches of more than eight such queries) or as passes over global
 * memory on all SMs (up to 2^26; every P above 2^18). */
TM_API tm_status tm_plan_create(const tm_plan_desc* desc, tm_plan_t* out);
TM_API tm_status tm_plan_get_info(tm_plan_t plan, tm_plan_info* info);
/* Frees the plan and its device workspace. Safe on NULL. */
TM_API tm_status tm_plan_destroy(tm_plan_t plan);

/* One query, Algorithm 1 steps 3-9 on the device: out_dev receives one
 * tm_result. The plan owns a device workspace (allocated on the first call
 * on the current device); calls on one plan must not overlap on the GPU. */
TM_API tm_status tm_match(tm_plan_t plan, const void* x_dev, const float* t_dev,
                   tm_result* out_dev, tm_stream_t stream);

/* ------------------------------------------------- slices of one signal
 * A signal too large for one GPU is cut into contiguous slices [n0, n0+len),
 * one per GPU. Eq. (2) is a sum over the entries of x, so the slices'
 * extended folds add up to the signal's (exactly for +-1 signals); one sum
 * reduction brings them to one GPU, which runs steps 4-8 on the sum; the
 * exact scores of step 9 are again sums over slices. Plans of P <= 16384. */

/* Folds of the slice: y[0..P) for M1 and y[P..2P) for M2 (int32 for +-1
 * signals, float32 for real ones; entries k >= M_j+K-1 set to 0), where
 * y_j[k] = sum_{l<L_j} x_{(k + l M_j) mod N} keeps only the terms whose index
 * lies in [n0, n0+len). x: the slice's storage (entry n0 first), 16-byte
 * aligned; n0 must fall on a 16-byte boundary of the signal (n0 * bits per
 * entry a multiple of 128). Writes all 2P entries of y (caller-owned device
 * memory). Calls on one plan must not overlap on the GPU. */
TM_API tm_status tm_fold_slice(tm_plan_t plan, const void* x_dev, int64_t n0, int64_t len, void* y_dev,
                               tm_stream_t stream);
/* Steps 4-8 from complete folds y (layout of tm_fold_slice, e.g. the sum of
 * all slices' folds): one tm_result with m1, m2, r1, r2, n_cand. With one
 * member of S1 ∩ S2 it is the shift; its score, and the choice among several
 * members (step 9), need the signal: the result carries TM_RF_SCORE_PENDING,
 * shift = the first member, score = 0 (tm_crt_candidates lists the members;
 * tm_score_slice scores them). */
TM_API tm_status tm_correlate_folds(tm_plan_t plan, const void* y_dev, const float* t_dev,
                                    tm_result* out_dev, tm_stream_t stream);
/* Partial exact scores over a slice: out[c] = sum_{i<K} t_i x_{(m[c]+i) mod N}
 * over the terms whose index lies in [n0, n0+len) (fp64; exact for integer
 * data). m_dev, out_dev: nm entries of device memory. */
TM_API tm_status tm_score_slice(tm_plan_t plan, const void* x_dev, int64_t n0, int64_t len,
                                const float* t_dev, const int64_t* m_dev, int32_t nm, double* out_dev,
                                tm_stream_t stream);

/* ----------------------------------------------------------------- batch */

typedef struct tm_batch_s* tm_batch_t;

/* Batch flags. */
#define TM_BATCH_KEEP_CORR 0x1u   /* keep r_{M1}, r_{M2} for tm_batch_corr */
#define TM_BATCH_HOST_INPUTS 0x2u /* allocate device copies of x and t so that
                                     tm_batch_run_host can take host buffers */
#define TM_BATCH_PIPELINED 0x4u   /* allocate a second partial-fold buffer, a
                                     stream and events for tm_batch_run_pipelined */

/* Plan n queries (each as tm_plan_create does) and allocate one device
 * workspace for them: partial folds, folds, template spectra. The pointers
 * in q are recorded (TM_BATCH_HOST_INPUTS: ignored). Needs the GPU that
 * will run the batch to be current. */
TM_API tm_status tm_batch_create(const tm_query* q, int32_t n, uint32_t flags, tm_batch_t* out);
/* Replace the x / t pointers of every query (same shapes as at creation). */
TM_API tm_status tm_batch_set_inputs(tm_batch_t b, const tm_query* q, int32_t n);
/* Step 3 for the whole batch: one launch per signal storage type that
 * streams every signal once and writes partial column sums of both folds;
 * moduli too wide for its register-resident columns (about 2^14 and more)
 * are folded entry by entry instead (one or two more launches). Queries on
 * the all-SM path also get their template spectra (steps 4-5, which read
 * only t) here, launched on a stream private to the batch that waits for
 * `stream`'s earlier work and runs beside the fold; tm_batch_correlate
 * joins it into its own stream, so t and the descriptors must stay as they
 * are until tm_batch_correlate is enqueued. */
TM_API tm_status tm_batch_fold(tm_batch_t b, tm_stream_t stream);
/* Steps 3 (completion: wrap term, extension k >= M), 4-9 for every query:
 * one CTA per query, largest FFT first, in one launch (plus one launch for
 * the overlap-save queries, and a sequence of launches per query on the
 * all-SM path, see tm_plan_create); writes n tm_results to out_dev.
 * Must follow tm_batch_fold on the same stream (it first waits for the
 * template spectra tm_batch_fold launched on the batch's private stream). */
TM_API tm_status tm_batch_correlate(tm_batch_t b, tm_result* out_dev, tm_stream_t stream);
/* tm_batch_fold + tm_batch_correlate. */
TM_API tm_status tm_batch_run(tm_batch_t b, tm_result* out_dev, tm_stream_t stream);
/* End to end from host memory (needs TM_BATCH_HOST_INPUTS): copies each
 * x_host[i] (tm_query N/xdtype bytes) and t_host[i] (K floats) to the
 * batch's device buffers, runs the batch and copies the n results back to
 * out_host. Synchronises the stream before returning. Pinned host memory
 * gives the fastest copies. */
TM_API tm_status tm_batch_run_host(tm_batch_t b, const void* const* x_host,
                            const float* const* t_host, tm_result* out_host,
                            tm_stream_t stream);
/* Autotuner: for each storage type in the batch, time the fold launch with
 * stage rings of 3 x 64 KiB, 6 x 32 KiB and 12 x 16 KiB on the batch's own
 * inputs (a few launches each on `stream`, which it synchronises) and keep
 * the fastest for later runs and captures. Choices are cached per process
 * by (storage type, size class of the batch, size class of the effective
 * modulus); TM_TUNE_FORCE re-times. tiles (optional, 4 entries indexed by
 * tm_dtype) receives the chosen stage bytes, 0 for types not in the batch.
 * Partial folds are overwritten: run the batch again before reading them. */
#define TM_TUNE_FORCE 0x1u
/* With TM_TUNE_GRID (batches created with TM_BATCH_PIPELINED only), the
 * autotuner also times pipelined calls (tm_batch_run_pipelined into the
 * batch's own result buffer, flushed) for splits of the SMs between the fold
 * and the correlation: corr_ctas C from a fixed list of counts (16 to half
 * the SM count), fold_ctas = SMs - C, and the unsplit launch; it keeps the
 * fastest with tm_batch_set_grid (cached per process by the batch's query
 * count, bytes and largest FFT length). tm_batch_get_grid reads the choice. */
#define TM_TUNE_GRID 0x2u
TM_API tm_status tm_batch_autotune(tm_batch_t b, tm_stream_t stream, uint32_t flags, int32_t* tiles);
/* The launch geometry set by tm_batch_set_grid or the autotuner. */
TM_API tm_status tm_batch_get_grid(tm_batch_t b, int32_t* fold_ctas, int32_t* corr_ctas);
/* Record one tm_batch_run(b, out_dev) - the fold launches and the
 * correlation launches with the memsets before them - as a CUDA graph held
 * by the batch (captured on a private stream; nothing runs). Replaces an
 * earlier capture. The graph reads the query descriptors from device
 * memory, so tm_batch_set_inputs still applies to it; out_dev is fixed. */
TM_API tm_status tm_batch_graph_capture(tm_batch_t b, tm_result* out_dev);
/* Launch the captured graph on a stream: the same work as tm_batch_run in
 * one graph launch. TM_EINVAL without a capture. */
TM_API tm_status tm_batch_graph_launch(tm_batch_t b, tm_stream_t stream);
/* Launch geometry: the fold runs on at most fold_ctas CTAs (one per SM
 * when 0 or above the SM count; the batch's signals are re-split into that
 * many equal shares, which needs no new memory when fold_ctas does not
 * exceed the SM count), and the shared-memory correlation keeps at most
 * corr_ctas CTAs running at a time (0: one CTA per query, all launched at
 * once; otherwise waves of launches of corr_ctas CTAs each). With
 * fold_ctas + corr_ctas <= the SM count, the two kernels of
 * tm_batch_run_pipelined run side by side on disjoint SMs (each of their
 * CTAs takes a whole SM's shared memory). Results do not change for +-1
 * signals; for real signals the fold's fp32 sums follow the new shares.
 * Replaces a graph captured before (capture again). Not while a pipelined
 * run is pending (TM_EBUSY: flush first). */
TM_API tm_status tm_batch_set_grid(tm_batch_t b, int32_t fold_ctas, int32_t corr_ctas);
/* Pipelined runs (needs TM_BATCH_PIPELINED): call i folds the batch's
 * current inputs (step 3, on `stream`) while the correlation of call i-1's
 * folds (steps 3-9) runs beside it on a stream of the batch, into the
 * out_dev that call i-1 was given; `stream` then waits for both, so each
 * call costs about the longer of the two rather than their sum when
 * tm_batch_set_grid has split the SMs between them. Call i-1's results are
 * therefore complete once call i (or tm_batch_pipeline_flush) has finished
 * on `stream`, and the inputs (x, t) of call i-1 must stay unchanged until
 * then (its correlation reads them for the wrap-around, extension and
 * exact scores). Batches whose queries all use the shared-memory
 * correlation (P <= 16384) and the streaming fold only (TM_EUNSUPPORTED
 * otherwise). The fold alternates between two partial buffers and error
 * words, so call i's fold never overwrites what call i-1's correlation
 * reads. fold_begin / fold_end (optional, NULL to skip): events recorded on
 * `stream` just before and after this call's fold launches, so that a
 * caller can time the fold while the correlation runs beside it. */
TM_API tm_status tm_batch_run_pipelined(tm_batch_t b, tm_result* out_dev, tm_stream_t stream, tm_event_t fold_begin,
                                        tm_event_t fold_end);
/* Runs the pending correlation of the last pipelined call on `stream`
 * (nothing when none is pending). */
TM_API tm_status tm_batch_pipeline_flush(tm_batch_t b, tm_stream_t stream);
/* Device pointers to query i's folds from the last run: y[0..P) for M1,
 * y[P..2P) for M2 (and y[2P..3P) for M3 with TM_THREE_MODULI), entries
 * k < M_j+K-1 valid. int32 for +-1 signals, float32 for real signals
 * (*is_float set accordingly). */
TM_API tm_status tm_batch_folds(tm_batch_t b, int32_t i, void** y_dev, int32_t* is_float);
/* Device pointer to query i's FFT correlations from the last run (needs
 * TM_BATCH_KEEP_CORR): r[0..M1), r[P..P+M2) (and r[2P..2P+M3)), float32. */
TM_API tm_status tm_batch_corr(tm_batch_t b, int32_t i, float** r_dev);
/* Number of CUDA kernels one tm_batch_run launches, and fold CTAs. */
TM_API tm_status tm_batch_stats(tm_batch_t b, int32_t* launches_per_run, int32_t* fold_ctas,
                         int64_t* workspace_bytes);
/* Device error word of the last run (0 = none; bit 0: a bounded device-side
 * wait ran out). Synchronises the stream. Pipelined runs reset each error
 * word once the correlation that reads it has flagged its results
 * (TM_RF_DEVICE_ERROR), so for them the results carry the report. */
TM_API tm_status tm_batch_device_error(tm_batch_t b, tm_stream_t stream, int32_t* err);
TM_API tm_status tm_batch_destroy(tm_batch_t b);

/* Self-test of the library's bounded device-side waits: one CTA waits on
 * an mbarrier that nothing arrives at, with the limit limit_ns (clamped to
 * [1 us, 100 ms]); *gave_up = 1 when the wait ended at its limit (the
 * expected outcome), 0 if it completed. The kernels' own waits use the same
 * code with a 2 s limit and then set their device error word. Synchronises
 * the current device. */
TM_API tm_status tm_selftest_wait_timeout(int64_t limit_ns, int32_t* gave_up);

/* One-shot batch: create, run, destroy (synchronises the stream). */
TM_API tm_status tm_match_batch(const tm_query* q, int32_t n, tm_result* out_dev, tm_stream_t stream);

/* ---------------------------------------------------------------- server */

/* Continuous-batching server for a synchronisation-receiver style use of the
 * method (Sec. 3.5: a known code x is resident, templates arrive and their
 * shift is wanted). Signals are registered once and stay in device memory;
 * clients submit (signal, template) requests from any thread; a worker
 * thread gathers the pending requests into an iteration that fits a fixed
 * device arena (admission by memory), runs it as a batch (tm_batch_run) on
 * one of n_streams streams while further requests keep arriving, and posts
 * results with per-request latency. Results are those of tm_match. */

typedef struct tm_server_s* tm_server_t;

typedef struct {
  int32_t n_streams;          /* iterations in flight, 1..4 (0: 2) */
  int32_t max_batch;          /* requests per iteration (0: 512) */
  int32_t queue_capacity;     /* pending requests before TM_EAGAIN (0: 65536) */
  uint32_t flags;             /* TM_SERVE_FINE_PIECES or 0 */
  int64_t arena_bytes;        /* device workspace per stream (0: share of free memory) */
  int64_t hbm_reserve_bytes;  /* left free when arena_bytes is 0 (0: 4 GiB) */
  int64_t fold_cache_bytes;   /* fold cache (0: off): the folds of a resident signal
                                 over k < M_j depend only on (signal, M1, M2), so a
                                 request whose pair was folded before skips the O(N)
                                 fold and pays only steps 4-9 (Sec. 3.5: a known code,
                                 many templates). Least recently used pairs are
                                 dropped beyond this many device bytes. Requests with
                                 FFT lengths above 16384 are not cached. */
  int64_t idle_spin_us;       /* with nothing pending or in flight, the worker keeps
                                 polling the queue this long before it sleeps on a
                                 condition variable (0: it sleeps at once): a request
                                 arriving meanwhile is taken without a thread wake-up,
                                 at the cost of a busy host core */
} tm_serve_cfg;

typedef struct {
  uint64_t tag;        /* the caller's tag from tm_serve_submit */
  int32_t status;      /* TM_OK, or why the request failed (e.g. TM_ENOMEM) */
  int32_t reserved;
  double latency_us;   /* submission to result, host clock */
  tm_result r;
} tm_result_tagged;

typedef struct {
  int64_t submitted, completed, failed, iterations, pending, in_flight;
  double mean_batch;   /* requests per iteration */
  double p50_us, p99_us, max_us;   /* latency over the completed requests */
  int64_t fold_cache_hits, fold_cache_misses;   /* requests served from / missing the fold cache */
  /* Mean over the completed requests of their latency's parts, host clock:
   * queue_us from submission until the worker takes the request, host_us
   * from then until its iteration's last launch has returned (planning,
   * staging, launches), device_us from then until the worker sees the
   * iteration's completion event. */
  double queue_us, host_us, device_us;
} tm_serve_stats;

/* Server flag: every request is planned with TM_FINE_PIECES (real signals
 * folded on more CTAs when an iteration holds few requests). */
#define TM_SERVE_FINE_PIECES 0x1u

/* Signal registration flag: x is device memory to use in place (the caller
 * keeps it alive until tm_serve_destroy); otherwise x is host memory and
 * the server keeps its own device copy. */
#define TM_SERVE_SIGNAL_DEVICE 0x1u

TM_API tm_status tm_serve_create(const tm_serve_cfg* cfg, tm_server_t* out);
TM_API tm_status tm_serve_register_signal(tm_server_t s, const void* x, int64_t N, int32_t xdtype, uint32_t flags,
                                          int32_t* sig_id);
/* Copies t_host (K floats) and queues the request; TM_EAGAIN when the queue
 * is full, TM_EINVAL for an unknown signal or an invalid plan, TM_ENOMEM when
 * the request alone exceeds the arena. mode/M1/M2/plan_flags as tm_plan_desc. */
TM_API tm_status tm_serve_submit(tm_server_t s, int32_t sig_id, const float* t_host, int32_t K, int32_t mode,
                                 int32_t M1, int32_t M2, uint32_t plan_flags, uint64_t tag);
/* n requests in one call (for clients that submit at high rates: one lock
 * and one wake-up for all of them): request i is (sig_ids[i], t_host[i],
 * K[i] floats, tags[i]) with the common mode (TM_MODE_AUTO or
 * TM_MODE_PAPER) and plan_flags. Requests are queued in order while the
 * queue has room; returns how many were queued (0..n; fewer than n when the
 * queue filled: submit the rest later), or -tm_status when request 0 is
 * invalid (a later invalid request stops the call after the valid prefix,
 * which is queued and counted). Templates are copied before the call
 * returns. */
TM_API int32_t tm_serve_submit_many(tm_server_t s, int32_t n, const int32_t* sig_ids, const float* const* t_host,
                                    const int32_t* K, int32_t mode, uint32_t plan_flags, const uint64_t* tags);
/* Up to max finished results; waits up to timeout_us for the first one.
 * Returns the number written (0 on timeout) or -tm_status on error. */
TM_API int32_t tm_serve_poll(tm_server_t s, tm_result_tagged* out, int32_t max, int64_t timeout_us);
TM_API tm_status tm_serve_stats_get(tm_server_t s, tm_serve_stats* st);
/* Stops the worker after the in-flight iterations, frees everything. */
TM_API tm_status tm_serve_destroy(tm_server_t s);

/* ----------------------------------------------------------- host helper */

/* Steps 8-9 in closed form on the host: the elements of
 * S1 ∩ S2, S_i = {(m_i + l M_i) mod N : l < ceil(N/M_i)}, in ascending
 * order (up to cap of them). Returns |S1 ∩ S2|, or -1 on invalid input.
 * The device uses the same function. */
TM_API int32_t tm_crt_candidates(int64_t N, int32_t M1, int32_t M2, int32_t m1, int32_t m2,
                          int64_t* out, int32_t cap);

/* sizeof of this header's public structs as compiled into the library, for
 * bindings that lay them out themselves: which = 0 tm_plan_desc, 1
 * tm_query, 2 tm_result, 3 tm_serve_cfg, 4 tm_result_tagged, 5
 * tm_serve_stats; 0 for any other value. Host only, no device needed. */
TM_API int64_t tm_struct_size(int32_t which);

/* ------------------------------------------------- no-allocation variant */

/* The paper has no counterpart to this entry point: it is a deployment
 * variant of tm_match for callers that must not allocate GPU memory, such
 * as real-time receiver loops (cudaMalloc / cudaFree can synchronise the
 * whole device and take unbounded time), processes whose device memory is
 * already claimed by another allocator's pool, and code that may only
 * allocate at start-up.
 *
 * It runs one query (Algorithm 1 steps 3-9, the same kernels and results as
 * tm_match) with every scratch buffer carved from one fixed device array of
 * TM_NOALLOC_SCRATCH_BYTES that the library holds on every GPU it is loaded
 * on until the process exits. The caller passes x_dev, t_dev and out_dev as
 * for tm_match. Signals above TM_NOALLOC_MAX_SIGNAL_BYTES return
 * TM_EUNSUPPORTED with a message (checked before any GPU work); invalid
 * problems TM_EINVAL. The fold runs on as many shares as the array holds
 * (fewer than tm_match uses for long signals, so it can be slower). No
 * cudaMalloc, cudaFree or other allocating call is made.
 *
 * The first call on a device sets that device up (finds the array's device
 * address, configures the kernels, uploads the FFT twiddles with a
 * synchronous copy); make that first call before any stream capture. The
 * address and the twiddles are kept for the life of the process: do not
 * reset the device (cudaDeviceReset) while the process still calls this
 * entry point. Every call reuses the same array, which keeps the previous
 * call's contents: calls that overlap on the GPU (different streams, or
 * other threads) race and corrupt each other's results. Calls on one stream
 * are ordered: each call's descriptors reach the array as the arguments of
 * a small kernel launched on that stream, so no host buffer is read after
 * the call returns. */
#define TM_NOALLOC_SCRATCH_BYTES (4u << 20)
#define TM_NOALLOC_MAX_SIGNAL_BYTES (1ll << 28)
TM_API tm_status tm_match_noalloc(const tm_plan_desc* desc, const void* x_dev, const float* t_dev,
                                  tm_result* out_dev, tm_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TM_H_ */
