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
// signals' 16-byte-aligned prefixes. Warps 0-7 accumulate the M1 fold,
// warps 8-15 the M2 fold, warp 16 issues bulk copies into a ring of
// shared-memory stages.
constexpr int kFoldModThreads = 256;                 // consumers per modulus
constexpr int kFoldConsumers = 2 * kFoldModThreads;  // 16 warps
constexpr int kFoldThreads = kFoldConsumers + 32;    // + producer warp
constexpr int kFoldStages = 4;
constexpr int kFoldTile = 32768;                     // bytes per stage
constexpr int kFoldJMax = 5;                         // 16-column units per consumer
constexpr int kFoldMinMp = 4096;                     // effective modulus floor
// A consumer's 16-bit lane counters hold twice the number of -1 entries;
// the host caps a CTA's share so that no column sees more rows than this.
constexpr int kFoldMaxRowsPerSlot = 32000;

struct FoldQ {
  const uint8_t* x;   // signal bytes, 16-byte aligned
  int64_t goff;       // first byte of this signal in the flattened space
  int32_t nbytes;     // bytes folded by the kernel (multiple of 16)
  int32_t Mp[2];      // effective moduli R_j * M_j >= kFoldMinMp
  int32_t moff[2];    // offset of modulus j inside a slot (int32 units)
  int32_t stride;     // slot length (int32 units)
  int32_t first_cta;  // CTA whose share holds goff
  int32_t nslots;
  int64_t part;       // offset of this query's first slot in the partial buffer
};

struct FoldArgs {
  const FoldQ* q;
  int32_t nq;
  int32_t nctas;
  int64_t W;          // total bytes (multiple of 16)
  int32_t* partial;   // int32 counts of -1 entries per (slot, modulus, column)
  int32_t* err;       // device error word
};

// Start of CTA c's share of W bytes (multiple of 16). Shared by the host
// planner (slot assignment) and the kernel.
__host__ __device__ inline int64_t fold_cta_begin(int64_t W, int32_t nctas, int32_t c) {
  const int64_t units = W >> 4;
  return ((units * c) / nctas) << 4;
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
  int32_t M[2];
  int32_t R[2];       // fold multipliers: Mp = R * M
  int64_t L[2];       // ceil(N / M_j)
  int32_t P, logP;
  int32_t inv;        // M1^{-1} mod M2
  int32_t nelem16;    // elements covered by the fold kernel
  int32_t nslots;
  int32_t moff[2];
  int32_t stride;
  int64_t part;       // first slot in the partial buffer (int32 units)
  int64_t y_off;      // fold output [2][P] (int32 or float), element offset
  int64_t spec_off;   // template spectrum scratch [P] float2, element offset
  int64_t r_off;      // correlation output [2][P] float, or -1
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
};

// ---------------------------------------------------------------- kernels' host launchers
cudaError_t launch_fold_i8(const FoldArgs& a, cudaStream_t s);
cudaError_t launch_correlate(const CorrArgs& a, int32_t maxP, cudaStream_t s);
cudaError_t fold_configure();   // one-time kernel attributes
cudaError_t corr_configure();

}  // namespace ftm
