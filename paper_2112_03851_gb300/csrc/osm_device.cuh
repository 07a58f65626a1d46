// Device helpers shared by the kernel files of libosm: deterministic
// reductions, the SELL-32 row dot products, the last-block ticket and the
// wall-clock guard of the device-side loops.  Internal (each .cu file gets its
// own copy through the anonymous namespace).
#pragma once

#include <cuda_runtime.h>

#include "osm_internal.h"

namespace osm {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV values over the 256 threads of a block; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sm)[kTileSlices]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) sm[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kTileSlices; ++w) s += sm[k][w];
      v[k] = s;
    }
  }
}

// Sum of part[t0 .. t0+nt) in a fixed order by one warp (all lanes get it).
__device__ __forceinline__ double warp_sum_parts(const double* part, int64_t t0, int64_t nt) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int64_t k = lane; k < nt; k += 32) v += __ldcg(part + t0 + k);
  return warp_sum(v);
}

// One row of a SELL-32 slice: lane `lane` of the warp owning the slice at
// `off` (width w, multiple of 4).  Matrix data is streamed (evict-first);
// the gathered vector stays cached.
__device__ __forceinline__ double sell_row(const int32_t* __restrict__ cols,
                                           const double* __restrict__ vals, int64_t off, int w,
                                           int lane, const double* __restrict__ x) {
  const int4* c4 = reinterpret_cast<const int4*>(cols + off) + lane;
  const double2* v2 = reinterpret_cast<const double2*>(vals + off) + lane;
  double acc0 = 0.0, acc1 = 0.0;
  const int nq = w >> 2;
#pragma unroll 4
  for (int q = 0; q < nq; ++q) {
    const int4 c = __ldcs(c4 + q * 32);
    const double2 a = __ldcs(v2 + q * 64);
    const double2 b = __ldcs(v2 + q * 64 + 32);
    acc0 = fma(a.x, __ldg(x + c.x), acc0);
    acc1 = fma(a.y, __ldg(x + c.y), acc1);
    acc0 = fma(b.x, __ldg(x + c.z), acc0);
    acc1 = fma(b.y, __ldg(x + c.w), acc1);
  }
  return acc0 + acc1;
}

// FP32 values (mixed-precision inner solve): the value array uses the same
// quad layout as the columns, so one float4 per lane per step; FP32 FMA
// accumulation.
__device__ __forceinline__ float sell_row(const int32_t* __restrict__ cols, const float* __restrict__ vals,
                                          int64_t off, int w, int lane, const float* __restrict__ x) {
  const int4* c4 = reinterpret_cast<const int4*>(cols + off) + lane;
  const float4* v4 = reinterpret_cast<const float4*>(vals + off) + lane;
  float acc0 = 0.f, acc1 = 0.f;
  const int nq = w >> 2;
#pragma unroll 4
  for (int q = 0; q < nq; ++q) {
    const int4 c = __ldcs(c4 + q * 32);
    const float4 a = __ldcs(v4 + q * 32);
    acc0 = fmaf(a.x, __ldg(x + c.x), acc0);
    acc1 = fmaf(a.y, __ldg(x + c.y), acc1);
    acc0 = fmaf(a.z, __ldg(x + c.z), acc0);
    acc1 = fmaf(a.w, __ldg(x + c.w), acc1);
  }
  return acc0 + acc1;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// True (and the stop flag raised, status bit 2) once the call's wall-clock
// budget is used up.  Called by single threads only.
__device__ __forceinline__ bool out_of_time(DevCtl* c) {
  if (c->stop) return true;
  if (global_ns() - c->t_start_ns > c->t_limit_ns) {
    c->stop = 1;
    atomicOr(&c->status, 4);
    return true;
  }
  return false;
}

// Ticket of the last block: returns true in every thread of the block that
// finished last among `total` blocks counted on *cnt (and resets it).
__device__ __forceinline__ bool last_block(unsigned* cnt, unsigned total, bool* flag_sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned prev = atomicAdd(cnt, 1u);
    *flag_sm = (prev == total - 1);
    if (*flag_sm) *cnt = 0u;
  }
  __syncthreads();
  bool last = *flag_sm;
  if (last) __threadfence();
  return last;
}

}  // namespace
}  // namespace osm
