// Internal descriptors shared by the host runtime and the kernels.
#pragma once

#include <cstdint>

#include "../../include/tm.h"

namespace ftm {

// ---------------------------------------------------------------- limits
constexpr int kPMax = 16384;          // largest FFT length held in shared memory
constexpr int kLogPMax = 14;
constexpr int kMaxCand = 8192;        // bound on |S1 ∩ S2| accepted by the planner
constexpr int64_t kMaxQueryBytes = (int64_t(1) << 31) - (int64_t(1) << 16);

// ---------------------------------------------------------------- fold kernel (step 3)
// Each CTA streams a contiguous, equal share of the concatenation of all
// signals' 16-byte-aligned prefixes. Consumer warps 0-7 accumulate the M1
// fold, warps 8-16 the M2 fold (the odd modulus K+1 has one more 16-column
// unit per row than K), warp 17 issues bulk copies into a ring of
// shared-memory stages.
constexpr int kFoldWarps0 = 8;                       // consumer warps of modulus M1
constexpr int kFoldWarps1 = 9;                       // consumer warps of modulus M2
constexpr int kFoldConsumers = 32 * (kFoldWarps0 + kFoldWarps1);

// Consumer warps of modulus j: with two moduli 8 and 9, with three 6, 6, 5.
__host__ __device__ inline int fold_warp_first(int nmod, int j) {
  return nmod == 3 ? 6 * j : (j == 0 ? 0 : kFoldWarps0);
}
__host__ __device__ inline int fold_warp_count(int nmod, int j) {
  return nmod == 3 ? (j == 2 ? 5 : 6) : (j == 0 ? kFoldWarps0 : kFoldWarps1);
}
constexpr int kFoldThreads = kFoldConsumers + 32;    // + producer warp
// The ring of shared-memory stages: 3 x 64 KiB by default; an autotuner
// may pick 6 x 32 KiB or 12 x 16 KiB for a batch (same ring bytes).
constexpr int kFoldStages = 3;
constexpr int kFoldTile = 65536;                     // bytes per stage (default)
constexpr int kFoldRingBytes = kFoldStages * kFoldTile;
constexpr int kFoldMinTile = 16384;
constexpr int kFoldMaxStages = kFoldRingBytes / kFoldMinTile;
// A consumer's 16-bit lane counters hold twice the number of -1 entries;
// the host caps a CTA's share so that no column sees more rows than this.
constexpr int kFoldMaxRowsPerSlot = 32000;
constexpr int kFoldMaxCtas = 256;   // CTAs whose first signal a launch can carry as a parameter

// Per signal storage type: columns per consumer unit (a unit is 16 bytes of
// a row, 4 bytes for bit-packed signals), bits per element, the floor of the
// effective modulus Mp = R M, and the most units per lane a launch supports.
struct FoldGeom {
  int E;
  int bits;
  int min_mp;
  int jmax;
};
__host__ __device__ inline FoldGeom fold_geom(int dtype) {
  switch (dtype) {
    case TM_BITS_PM1: return FoldGeom{32, 1, 8192, 2};
    case TM_F16: return FoldGeom{8, 16, 4096, 8};
    case TM_F32: return FoldGeom{4, 32, 4096, 16};
    default: return FoldGeom{16, 8, 4096, 5};
  }
}

// Units per lane needed for an effective modulus Mp on `warps` warps, with
// units of E columns dealt out in chunks of 32 consecutive units per warp.
__host__ __device__ inline int fold_units_per_lane(int Mp, int warps, int E) {
  const int chunks = ((Mp + E - 1) / E + 31) / 32;
  return (chunks + warps - 1) / warps;
}

struct FoldQ {
  const uint8_t* x;   // signal bytes, 16-byte aligned
  int64_t goff;       // first byte of this signal in the flattened space
  int32_t nbytes;     // bytes folded by the kernel (multiple of 16)
  int32_t nmod;       // moduli folded (2 or 3)
  int32_t Mp[3];      // effective moduli R_j * M_j (>= fold_geom(dtype).min_mp)
  int32_t moff[3];    // offset of modulus j inside a slot (int32 units)
  int32_t stride;     // slot length (int32 units)
  int32_t first_cta;  // CTA whose share holds goff
  int32_t nslots;
  int64_t part;       // offset of this query's first slot in the partial buffer
  int64_t e0;         // element index of x[0] within its signal (a slice), else 0;
                      // the byte offset e0 * bits / 8 is a multiple of 16
  int64_t piece;      // 0: one slot per CTA share holding bytes of this signal;
                      // > 0: the signal is cut into pieces of this many bytes
                      // (a multiple of 64 KiB, fixed by the signal alone) that
                      // no CTA share splits, one slot per piece in piece order,
                      // so fp32 sums do not depend on the rest of the batch
};

struct FoldArgs {
  const FoldQ* q;     // the signals of one storage type, in byte-space order
  int32_t nq;
  int32_t dtype;      // tm_dtype shared by all of them
  int32_t nctas;
  int64_t W;          // total bytes (multiple of 16)
  int32_t* partial;   // per (slot, modulus, column): int32 counts of -1 (int8) or
                      // +1 (bits) entries, or fp32 sums (real signals)
  int32_t* err;       // device error word
  int32_t tile = kFoldTile;   // bytes per stage: 16384, 32768 or 65536
  // q0[c]: the first signal whose bytes reach CTA c's share (has_q0 set by
  // fold_args_first_queries); otherwise each CTA searches the descriptors,
  // a chain of dependent global loads ahead of its first copy
  int32_t has_q0 = 0;
  int32_t q0[kFoldMaxCtas];
  // cb[c]: start of CTA c's share (cb[nctas] = W) when the shares follow
  // piece boundaries (has_cb); otherwise equal shares (fold_cta_begin)
  int32_t has_cb = 0;
  int64_t cb[kFoldMaxCtas + 1];
};

// Start of CTA c's share of W bytes (multiple of 16). Shared by the host
// planner (slot assignment) and the kernel.
__host__ __device__ inline int64_t fold_cta_begin(int64_t W, int32_t nctas, int32_t c) {
  const int64_t units = W >> 4;
  return ((units * c) / nctas) << 4;
}

// Start of CTA c's share of a launch.
__host__ __device__ inline int64_t fold_share_begin(const FoldArgs& a, int32_t c) {
  return a.has_cb ? a.cb[c] : fold_cta_begin(a.W, a.nctas, c);
}

// Fills a.q0 from the host copy hq[0..a.nq) of the descriptors a.q points
// to (same order), when a.nctas fits; a.cb (has_cb) must be set before.
inline void fold_args_first_queries(FoldArgs& a, const FoldQ* hq) {
  a.has_q0 = 0;
  if (a.nctas <= 0 || a.nctas > kFoldMaxCtas) return;
  int i = 0;
  for (int32_t c = 0; c < a.nctas; ++c) {
    const int64_t cb = fold_share_begin(a, c);
    while (i < a.nq && hq[i].goff + hq[i].nbytes <= cb) ++i;   // shares ascend with c
    a.q0[c] = i;
  }
  a.has_q0 = 1;
}

// Piece size of a real signal of `bytes` bytes: at least 2 MiB, at most 64
// pieces, a multiple of 64 KiB (so that every stage of the fold's ring lies
// inside one piece). Depends on the signal alone.
inline int64_t fold_piece_bytes(int64_t bytes, bool fine = false) {
  const int64_t unit = 65536;
  const int64_t most = fine ? 128 : 64, least = fine ? (int64_t(256) << 10) : (int64_t(2) << 20);
  const int64_t per = ((bytes + most - 1) / most + unit - 1) / unit * unit;
  return per > least ? per : least;
}

// ---------------------------------------------------------------- correlation kernel (steps 3-9)
constexpr int kCorrThreads = 512;
constexpr int kCandCap = 128;         // near-maximal r_j rescored exactly per modulus

struct CorrQ {
  const void* x;
  const float* t;
  int64_t N;
  int32_t K;
  int32_t xdtype;
  int32_t nmod;       // 2 or 3 moduli
  int32_t M[3];
  int32_t R[3];       // fold multipliers: Mp = R * M
  int64_t L[3];       // ceil(N / M_j)
  int32_t P, logP;
  int32_t inv;        // M1^{-1} mod M2
  int32_t inv3;       // (M1 M2)^{-1} mod M3
  int32_t thm2;       // Thm. 2 sampling: no wrap-around term, periodic extension
  int32_t nelem16;    // elements covered by the fold kernel
  int32_t nslots;
  int32_t moff[3];
  int32_t stride;
  int64_t part;       // first slot in the partial buffer (int32 units)
  int64_t y_off;      // fold output [nmod][P] (int32 or float), element offset
  int64_t spec_off;   // template spectrum scratch [P] float2, element offset
  int64_t r_off;      // correlation output [2][P] float, or -1
  const void* y_in;   // complete folds [2][P] supplied by the caller (the fold
                      // completion is skipped; x may then be null: no exact score)
  int32_t direct;     // folded entry by entry into y (then given as y_in)
  int32_t dh;         // entry-by-entry fold: row groups of the first stage (0: none)
  int32_t drows;      // rows per group
  int32_t dpitch;     // columns per group row of the partial sums (max M_j, rounded up to 4)
  int64_t dpart;      // its partial sums [nmod][dh][dpitch] in the partial buffer (int32 units)
  const void* y_core; // cached folds over k < M_j (wrap-around and last entries
                      // included), row j at y_core + j core_pitch; the fold
                      // kernel skips the signal, only the extension is added
  int32_t core_pitch;
};

struct CorrArgs {
  const CorrQ* q;
  const int32_t* order;   // query processing order (largest P first)
  int32_t nq;
  const int32_t* partial;
  void* y;                // int32 or float per query (by dtype)
  float2* spec;
  float* r;               // may be null
  const float2* tw;       // twiddles W_{kPMax}^m, m < kPMax
  tm_result* out;
  int32_t* err;
  int32_t smem_bytes;     // dynamic shared memory of the launch (set by the launcher)
  int32_t ctas = 0;       // most CTAs running at a time (0: one CTA per query,
                          // all at once); more queries run as waves of launches
  int32_t first = 0;      // first position in the order (set per wave by the launcher)
  int32_t pdl = 0;        // programmatic dependent of the kernel before it in the stream
                          // (a fold or the slot sums): the template spectrum runs
                          // before that kernel has finished (one wave only)
  int32_t lone = -1;      // >= 0: a launch of this one query, whose descriptor is q1
                          // (no dependent global loads of order and descriptor ahead
                          // of its work); launchers that a graph may capture leave it -1
  CorrQ q1;
};

// Launch configuration with the programmatic stream-serialisation attribute
// when pdl is set (the kernel then calls pdl_acquire before reading what
// the kernel before it writes).
inline cudaLaunchConfig_t launch_config(dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                                        cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t c = {};
  c.gridDim = grid;
  c.blockDim = block;
  c.dynamicSmemBytes = smem;
  c.stream = s;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  c.attrs = attr;
  c.numAttrs = pdl ? 1 : 0;
  return c;
}

// ---------------------------------------------------------------- kernels' host launchers
cudaError_t launch_fold(const FoldArgs& a, int jmax, cudaStream_t s);
cudaError_t launch_correlate(const CorrArgs& a, int32_t maxP, cudaStream_t s);
// Queries with max(M)+K-1 > kPMax: blocked correlation with 2*8192-point
// FFTs; needs spectra scratch of blocked_spectra(K, max M) * 16384 complex
// and an r buffer [2][P] (r_off >= 0).
cudaError_t launch_correlate_blocked(const CorrArgs& a, cudaStream_t s);
int blocked_spectra(int K, int maxM);
constexpr int kLogPMaxBlocked = 18;   // longest FFT of the blocked correlation: 262144
// ---------------------------------------------------------------- slot sums (end of step 1)
// A signal that many fold CTAs share leaves one partial row per share (or
// per piece); a lone correlation CTA reading dozens of rows is bound by its
// own load latency. The slot-sum kernel first adds the rows of such folds
// into one row, spread over many CTAs; the correlation then reads that row.
// The sum goes to a row of its own (not row 0), so correlating the same
// fold twice sums the same rows again.
constexpr int kSlotSumMin = 8;        // folds of at least this many rows are summed ahead
constexpr int kSlotSumThreads = 512;  // 16 warps share a row's slots; 32 column quads per CTA
struct SlotSumJob {
  int64_t src;      // first row (int32 units in the partial buffer)
  int64_t dst;      // the sum row
  int32_t nslots;   // rows to add
  int32_t cols;     // row length (int32 units, multiple of 16): the slot stride
  int32_t real;     // rows hold fp32 sums (else int32 counts)
};
struct SlotSumArgs {
  int32_t* partial;
  const SlotSumJob* job;   // device array of njobs jobs
  int32_t njobs;
  int32_t max_cols;        // longest row among them
  int32_t pdl = 0;         // launched as a programmatic dependent of the fold before it
};
cudaError_t launch_slot_sums(const SlotSumArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- slices of one signal
// Completion of a slice's fold: the extended folds [2][P] of Eq. (2)
// restricted to the entries x_n with n in [n0, n0 + len), from the fold
// kernel's slots over [n0, n0 + nfold) plus the slice's own tail, wrap-around
// and extension terms.
struct SliceFoldArgs {
  const int32_t* partial;   // [nslots][stride] int32 counts or fp32 sums
  int32_t nslots, stride;
  int32_t moff[2], M[2], R[2];
  int64_t L[2];
  int64_t N;
  int32_t K, P, xdtype;
  const void* x;            // the slice's storage: element n0 first
  int64_t n0, len, nfold;
  void* y;                  // [2][P] int32 (+-1 signals) or float
};
cudaError_t launch_fold_slice_complete(const SliceFoldArgs& a, cudaStream_t s);
// Partial scores sum_{i<K} t_i x_{(m+i) mod N} over the entries in the slice,
// for each candidate m; fp64 (exact for integer data).
struct SliceScoreArgs {
  const void* x;
  int32_t xdtype;
  int64_t N, n0, len;
  const float* t;
  int32_t K;
  const int64_t* m;
  int32_t nm;
  double* out;
};
cudaError_t launch_score_slice(const SliceScoreArgs& a, cudaStream_t s);

// Step 3 entry by entry for the queries idx[0..n) of q (CorrQ::direct):
// partial sums over dh row groups into partial + q.dpart, then the complete
// folds written to y + q.y_off. maxM, maxHM: the largest M_j and dh * nmod
// (maxHM = 0: no query has a first stage, one launch).
cudaError_t launch_fold_direct(const CorrQ* q, const int32_t* idx, int32_t n, int32_t maxP, int32_t maxmod,
                               int32_t maxM, int32_t maxHM, int32_t* partial, void* y, cudaStream_t s);
// Row groups of the entry-by-entry fold for L rows: about 64 rows each for
// int8 signals (all moduli in one thread), 16 for the others.
inline int32_t direct_row_groups(int64_t L, int32_t dtype) {
  const int64_t per = dtype == TM_I8_PM1 ? 64 : 16;
  const int64_t h = (L + per - 1) / per;
  return int32_t(h < 1 ? 1 : (h > 64 ? 64 : h));
}
constexpr int kDirCols = 4;   // fold columns per thread of the first stage

// ---------------------------------------------------------------- long FFTs on all SMs (steps 4-9)
// One query whose FFT length P = 2^logP (2^14 <= P <= 2^26) runs as a
// sequence of launches over global memory: the transforms are cut into
// 8192-point contiguous row blocks and one or two strided column passes
// (dims logL[0..nsd) outermost first, each <= 2^9 points), then candidate
// collection, chunked exact rescoring, the intersection and the scores.
constexpr int kLogPMinLarge = 14;
constexpr int kLogPMaxLarge = 26;
constexpr int kLargeCap = 4096;       // candidates per modulus rescored from a list
constexpr int kLargePart = 1 << 18;   // partial dot products of all candidates
constexpr int kLargeMembers = 256;    // members scored from a list
constexpr int kLargeMPart = 1 << 16;  // partial dot products of all members
constexpr int kLargeCtas = 1216;      // grid of the rescoring and scoring launches
// Queries with P > kPMax take this path (all SMs, the batch's queries in
// the same launches) when P >= 2^kLogPLargeAlways, or when the batch holds
// at most kLargeMaxQueries queries of P > kPMax; the others (many queries of
// 2^15 or 2^16 points) take the overlap-save blocks, one CTA per query.
constexpr int kLargeMaxQueries = 8;
constexpr int kLogPLargeAlways = 17;

struct LQ {
  const void* x;
  const float* t;
  const void* y;        // complete folds [2][P] (int32 for +-1 signals, else float)
  float* r;             // correlations [2][P]
  float2* A;            // [P] signal spectrum, then the products
  float2* B;            // [P] template spectrum
  void* ws;             // large_ws_bytes() of statistics, candidates and partial sums
  int32_t* err;
  int64_t N;
  int32_t K, xdtype;
  int32_t M[2];
  int32_t inv;
  int32_t P, logP;
  int32_t thm2;
  int32_t nsd;          // strided dims (1 or 2)
  int32_t logL[2];
  int32_t qi;           // index of the query in the batch (its result slot)
  int32_t pad_;
};
size_t large_ws_bytes();
// Strided dims of a length-2^logP transform (8192-point rows innermost).
inline int large_dims(int logP, int32_t (&logL)[2]) {
  const int q = logP - 13;
  if (q <= 9) { logL[0] = q; logL[1] = 0; return 1; }
  logL[0] = (q + 1) / 2; logL[1] = q / 2;
  return 2;
}
// The launches for the n queries d_lq[0..n) on stream s (folds given in
// each q.y; h_lq: the same descriptors on the host): maxP, the longest FFT;
// two_dims, whether any has two strided dims; maxM, the largest modulus;
// results to out[q.qi]. A single query's descriptor goes by value (no
// load from memory ahead of each CTA's work).
cudaError_t launch_correlate_large(const LQ* d_lq, const LQ* h_lq, int n, int maxP, bool two_dims, int maxM,
                                   tm_result* out, cudaStream_t s);
// The same launches in two parts: the template spectra (read t only, so
// they may run on another stream beside the fold) and, once they and the
// folds are done, the signal spectra with steps 7-9.
cudaError_t launch_large_template(const LQ* d_lq, const LQ* h_lq, int n, int maxP, bool two_dims, cudaStream_t s);
cudaError_t launch_large_signal(const LQ* d_lq, const LQ* h_lq, int n, int maxP, bool two_dims, int maxM,
                                tm_result* out, cudaStream_t s);
int large_launches(int nsd);
cudaError_t large_configure();

cudaError_t fold_configure();   // one-time kernel attributes
cudaError_t corr_configure();

}  // namespace ftm
