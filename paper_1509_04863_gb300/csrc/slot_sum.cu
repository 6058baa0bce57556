// Step 3 of Algorithm 1 (Eq. (2)), across CTA shares: the column sums the
// fold kernel leaves per share (or per piece of a real signal) added into one
// row before the correlation completes the fold.
//
// One CTA takes 32 column quads (128 columns) of one job (grid y strides over
// the jobs); its 16 warps take the rows w, w + 16, w + 32, ... of those
// columns, and warp 0 adds the 16 partial sums in warp order. The order
// depends on the number of rows alone, so fp32 sums are the same whatever
// else the batch holds; int32 counts are exact in any order.
#include "device_util.cuh"
#include "tm_internal.h"

namespace ftm {
namespace {

constexpr int kWarps = kSlotSumThreads / 32;

__device__ __forceinline__ void add4(float4& f, const int4 v) {
  f.x += __int_as_float(v.x); f.y += __int_as_float(v.y);
  f.z += __int_as_float(v.z); f.w += __int_as_float(v.w);
}
__device__ __forceinline__ void add4(uint4& c, const int4 v) {
  c.x += unsigned(v.x); c.y += unsigned(v.y); c.z += unsigned(v.z); c.w += unsigned(v.w);
}
__device__ __forceinline__ int4 bits4(const float4 f) {
  return make_int4(__float_as_int(f.x), __float_as_int(f.y), __float_as_int(f.z), __float_as_int(f.w));
}
__device__ __forceinline__ int4 bits4(const uint4 c) { return make_int4(int(c.x), int(c.y), int(c.z), int(c.w)); }

// Rows [0, nslots) of job j, columns [128 blockIdx.x, +128): sums in T
// (float4 for fp32 rows, uint4 for int32 counts: wrap-around addition).
template <class T>
__device__ __forceinline__ void sum_quads(int32_t* partial, const SlotSumJob& j, int4 (*part)[32]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int q = int(blockIdx.x) * 32 + lane;   // column quad
  const bool on = 4 * q < j.cols;
  const int4* src = reinterpret_cast<const int4*>(partial + j.src) + q;
  const int64_t step = j.cols / 4;             // quads per row
  T acc{};
  if (on) {
#pragma unroll 4
    for (int r = w; r < j.nslots; r += kWarps) add4(acc, __ldg(src + r * step));
  }
  part[w][lane] = bits4(acc);
  __syncthreads();
  if (w == 0 && on) {
    T s{};
    for (int k = 0; k < kWarps; ++k) add4(s, part[k][lane]);
    reinterpret_cast<int4*>(partial + j.dst)[q] = bits4(s);
  }
}

__global__ void __launch_bounds__(kSlotSumThreads) slot_sum_kernel(const SlotSumArgs a) {
  __shared__ int4 part[kWarps][32];
  pdl_release();   // the correlation after it may start its template work
  pdl_acquire();   // the fold's rows are complete
  for (int jb = blockIdx.y; jb < a.njobs; jb += gridDim.y) {
    const SlotSumJob j = a.job[jb];
    if (int(blockIdx.x) * 128 >= j.cols) continue;   // the whole CTA is past this job's row
    __syncthreads();                                  // part[] of the previous job read
    if (j.real) sum_quads<float4>(a.partial, j, part);
    else sum_quads<uint4>(a.partial, j, part);
  }
}

}  // namespace

cudaError_t launch_slot_sums(const SlotSumArgs& a, cudaStream_t s) {
  if (a.njobs <= 0) return cudaSuccess;
  const dim3 grid(unsigned((a.max_cols + 127) / 128), unsigned(a.njobs < 65535 ? a.njobs : 65535));
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t c = launch_config(grid, dim3(kSlotSumThreads), 0, s, a.pdl != 0, attr);
  return cudaLaunchKernelEx(&c, slot_sum_kernel, a);
}

}  // namespace ftm
