// Device helpers: mbarriers with bounded waits, bulk global->shared copies.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ftm {

// A bounded device-side wait gives up after this many nanoseconds and the
// kernel records an error instead of spinning forever.
constexpr uint64_t kWaitTimeoutNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialisation attribute may start once every CTA of the kernel
// before it in the stream has signalled (pdl_release) or exited; it must
// call pdl_acquire before it reads what that kernel writes, which returns
// once that kernel has completed and its writes are visible. Without the
// attribute both are no-ops.
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_acquire() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the async (bulk copy) proxy.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity to complete; false once limit_ns
// have passed without it.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// Double-float accumulation on the FP32 pipes (GB300 has few FP64 units):
// a times b is exactly p + e with p = a b rounded and e = fma(a, b, -p); p
// goes into the running pair (hi, lo) through an error-free two-sum
// (Knuth), e and the sum's error into lo. With n terms the pair's error
// stays below about n 2^-47 sum |a_i b_i|, far below what fp32 folds carry.
struct DF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += e + pe;
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

// Sum of two pairs: the high parts by an error-free two-sum, the low parts
// and its error added in fp32. Symmetric in its arguments (the two-sum's
// error is unique), so both lanes of a butterfly exchange get the same pair.
__device__ __forceinline__ DF df_sum(const DF& a, const DF& b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  DF r;
  r.hi = s;
  r.lo = (a.lo + b.lo) + e;
  return r;
}

// Pair sum over a warp (butterfly; every lane ends with the same pair).
__device__ __forceinline__ DF warp_sum_df(DF a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF b;
    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
    b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
    a = df_sum(a, b);
  }
  return a;
}

// Pair sums over a block of NW warps, n at a time (red: n NW entries),
// warps added in index order; valid in thread 0 (the other threads keep
// their warp's sums). GB300's FP64 rate is a small fraction of its FP32
// rate: the reductions stay in fp32 pairs and thread 0 converts the one
// result it needs to double.
template <int NW, int n>
__device__ __forceinline__ void block_sum_df(DF (&v)[n], float2* red) {
#pragma unroll
  for (int i = 0; i < n; ++i) v[i] = warp_sum_df(v[i]);
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < n; ++i) red[n * (threadIdx.x >> 5) + i] = make_float2(v[i].hi, v[i].lo);
  __syncthreads();
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int i = 0; i < n; ++i) {
    DF s;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      DF p;
      const float2 q = red[n * w + i];
      p.hi = q.x;
      p.lo = q.y;
      s = df_sum(s, p);
    }
    v[i] = s;
  }
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, kWaitTimeoutNs);
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                          uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

}  // namespace ftm
