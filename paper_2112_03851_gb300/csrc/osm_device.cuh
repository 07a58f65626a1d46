// Device helpers shared by the kernel files of libosm: deterministic
// reductions, the SELL-32 row dot products, the last-block ticket and the
// wall-clock guard of the device-side loops.  Internal (each .cu file gets its
// own copy through the anonymous namespace).
#pragma once

#include <cuda_runtime.h>

#include "osm_internal.h"

namespace osm {
namespace {

// A double as an unevaluated pair of floats, hi + lo (hi the nearest float,
// lo the nearest float to the remainder): 48 significant bits, exact for the
// FP32 inputs of the double-float kernels.
__device__ __forceinline__ float2 df_split(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV values over the NW warps of a block; result valid in thread 0.
template <int NV, int NW = kTileSlices, int SW = kTileSlices>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sm)[SW]) {
  static_assert(NW <= SW, "shared scratch narrower than the warp count");
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
      for (int w = 0; w < NW; ++w) s += sm[k][w];
      v[k] = s;
    }
  }
}

// Sum NV doubles over the NT threads of a block with about one FP64 add per
// value: the values are staged in shared memory, 8 threads per value add
// interleaved eighths in a fixed order, and thread 0 adds the 8 partials.
// A warp butterfly costs five FP64 adds per lane and value, and FP64 is the
// scarce pipe on this GPU: in FP64-bound kernels (the FP64 SpMVs and CG
// update) the butterflies took a large share of it.  Result in thread 0.
template <int NV, int NT>
__device__ __forceinline__ void block_sum_d(double (&v)[NV], double (*sm)[NT]) {
  static_assert(NT % 8 == 0 && NV * 8 <= NT, "block too small for the staged sum");
  constexpr int kChunk = NT / 8;
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < NV; ++k) sm[k][t] = v[k];
  __syncthreads();
  double part = 0.0;
  if (t < NV * 8) {
    const int k = t >> 3, c = t & 7;
#pragma unroll 8
    for (int i = 0; i < kChunk; ++i) part += sm[k][i * 8 + c];
  }
  __syncthreads();
  if (t < NV * 8) sm[t >> 3][t & 7] = part;
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < 8; ++c) s += sm[k][c];
      v[k] = s;
    }
  }
}

// Sum of part[t0 .. t0+nt) in a fixed order by one warp (all lanes get it).
// Four independent loads per lane per step keep several L2 requests in flight.
__device__ __forceinline__ double warp_sum_parts(const double* part, int64_t t0, int64_t nt) {
  const int lane = threadIdx.x & 31;
  double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
  int64_t k = lane;
  for (; k + 96 < nt; k += 128) {
    v0 += __ldcg(part + t0 + k);
    v1 += __ldcg(part + t0 + k + 32);
    v2 += __ldcg(part + t0 + k + 64);
    v3 += __ldcg(part + t0 + k + 96);
  }
  for (; k < nt; k += 32) v0 += __ldcg(part + t0 + k);
  return warp_sum((v0 + v1) + (v2 + v3));
}

// Rows of one 256-row tile handled by the calling thread when each warp works
// RPL slices at once (blockDim = 256 / RPL): slice tile*8 + warp*RPL + k,
// row slice*32 + lane.  The slices' loads are interleaved step by step, so a
// lane keeps RPL independent streams in flight.  FP64 values use the pair
// layout (two double2 per step), FP32 values the quad layout (one float4).
template <class T, int RPL>
__device__ __forceinline__ void tile_rows(const int64_t* __restrict__ slice_off, const int32_t* __restrict__ cols,
                                          const T* __restrict__ vals, int64_t tile, const T* __restrict__ x,
                                          T (&y)[RPL], int64_t (&row)[RPL]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t off[RPL];
  int nq[RPL];
  int nqmax = 0;
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const int64_t slice = tile * kTileSlices + warp * RPL + k;
    off[k] = slice_off[slice];
    nq[k] = (int)((slice_off[slice + 1] - off[k]) >> 7);  // width / 4
    row[k] = slice * kSliceRows + lane;
    nqmax = max(nqmax, nq[k]);
  }
  T a0[RPL], a1[RPL];
#pragma unroll
  for (int k = 0; k < RPL; ++k) { a0[k] = T(0); a1[k] = T(0); }
#pragma unroll 2
  for (int q = 0; q < nqmax; ++q) {
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      if (q < nq[k]) {
        const int4 c = __ldcs(reinterpret_cast<const int4*>(cols + off[k]) + lane + q * 32);
        if constexpr (sizeof(T) == 8) {
          const double2* v2 = reinterpret_cast<const double2*>(vals + off[k]) + lane;
          const double2 a = __ldcs(v2 + q * 64);
          const double2 b = __ldcs(v2 + q * 64 + 32);
          a0[k] = fma(a.x, __ldg(x + c.x), a0[k]);
          a1[k] = fma(a.y, __ldg(x + c.y), a1[k]);
          a0[k] = fma(b.x, __ldg(x + c.z), a0[k]);
          a1[k] = fma(b.y, __ldg(x + c.w), a1[k]);
        } else {
          const float4 a = __ldcs(reinterpret_cast<const float4*>(vals + off[k]) + lane + q * 32);
          a0[k] = fmaf(a.x, __ldg(x + c.x), a0[k]);
          a1[k] = fmaf(a.y, __ldg(x + c.y), a1[k]);
          a0[k] = fmaf(a.z, __ldg(x + c.z), a0[k]);
          a1[k] = fmaf(a.w, __ldg(x + c.w), a1[k]);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < RPL; ++k) y[k] = a0[k] + a1[k];
}

// Rows of one tile with 16-bit column indices (subdomains of at most 65,536
// padded rows): the same layouts, but lane l of step q loads its four
// columns as one 8-byte uint2 at entry off + 128 q + 4 l (2 instead of 4
// bytes per nonzero).  Same per-row summation order as tile_rows.
template <class T, int RPL>
__device__ __forceinline__ void tile_rows16(const int64_t* __restrict__ slice_off, const uint16_t* __restrict__ cols,
                                            const T* __restrict__ vals, int64_t tile, const T* __restrict__ x,
                                            T (&y)[RPL], int64_t (&row)[RPL]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t off[RPL];
  int nq[RPL];
  int nqmax = 0;
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const int64_t slice = tile * kTileSlices + warp * RPL + k;
    off[k] = slice_off[slice];
    nq[k] = (int)((slice_off[slice + 1] - off[k]) >> 7);
    row[k] = slice * kSliceRows + lane;
    nqmax = max(nqmax, nq[k]);
  }
  T a0[RPL], a1[RPL];
#pragma unroll
  for (int k = 0; k < RPL; ++k) { a0[k] = T(0); a1[k] = T(0); }
#pragma unroll 2
  for (int q = 0; q < nqmax; ++q) {
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      if (q < nq[k]) {
        const uint2 c = __ldcs(reinterpret_cast<const uint2*>(cols + off[k]) + lane + q * 32);
        const unsigned c0 = c.x & 0xffffu, c1 = c.x >> 16, c2 = c.y & 0xffffu, c3 = c.y >> 16;
        if constexpr (sizeof(T) == 8) {
          const double2* v2 = reinterpret_cast<const double2*>(vals + off[k]) + lane;
          const double2 a = __ldcs(v2 + q * 64);
          const double2 b = __ldcs(v2 + q * 64 + 32);
          a0[k] = fma(a.x, __ldg(x + c0), a0[k]);
          a1[k] = fma(a.y, __ldg(x + c1), a1[k]);
          a0[k] = fma(b.x, __ldg(x + c2), a0[k]);
          a1[k] = fma(b.y, __ldg(x + c3), a1[k]);
        } else {
          const float4 a = __ldcs(reinterpret_cast<const float4*>(vals + off[k]) + lane + q * 32);
          a0[k] = fmaf(a.x, __ldg(x + c0), a0[k]);
          a1[k] = fmaf(a.y, __ldg(x + c1), a1[k]);
          a0[k] = fmaf(a.z, __ldg(x + c2), a0[k]);
          a1[k] = fmaf(a.w, __ldg(x + c3), a1[k]);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < RPL; ++k) y[k] = a0[k] + a1[k];
}

// Dispatch on the column width chosen at setup (C16: d.cols16).
template <class T, int RPL, bool C16>
__device__ __forceinline__ void tile_rows_any(const DevProblem& d, const T* __restrict__ vals, int64_t tile,
                                              const T* __restrict__ x, T (&y)[RPL], int64_t (&row)[RPL]) {
  if constexpr (C16) tile_rows16<T, RPL>(d.slice_off, d.cols16, vals, tile, x, y, row);
  else tile_rows<T, RPL>(d.slice_off, d.cols, vals, tile, x, y, row);
}

// Mean of c copies, s / c.  On a box grid of subdomains a node has 1, 2, 4
// or 8 copies: then s * 2^-k, which is bit-identical to the division and
// avoids FP64 division (a long instruction sequence on this GPU).
__device__ __forceinline__ double copy_mean(double s, int c) {
  if ((c & (c - 1)) == 0) return s * __longlong_as_double((long long)(1023 - (__ffs(c) - 1)) << 52);
  return s / (double)c;
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

// End of the SpMV kernel of a CG step, called by every thread after thread 0
// wrote the block's p.q partial: the subdomain's last block (a ticket on
// st.tcnt, no waiting) adds the subdomain's partials part0[sub_part0[s] ..
// sub_part0[s+1]) in a fixed order and stores p.q and alpha = rho / p.q (0 on
// a breakdown, p.q <= 0 or not finite) for the update kernel.
__device__ __forceinline__ void cg_alpha_ticket(const DevProblem& d, int s, bool* s_last) {
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned n = (unsigned)(d.sub_part0[s + 1] - d.sub_part0[s]);
    const unsigned t = atomicAdd(&d.st.tcnt[s], 1u);
    *s_last = t == n - 1u;
    if (*s_last) d.st.tcnt[s] = 0u;
  }
  __syncthreads();
  if (*s_last && (threadIdx.x >> 5) == 0) {
    __threadfence();
    const int64_t a0 = d.sub_part0[s];
    const double pq = warp_sum_parts(d.part0, a0, d.sub_part0[s + 1] - a0);
    if ((threadIdx.x & 31) == 0) {
      d.st.pq[s] = pq;
      d.st.alpha[s] = (pq > 0.0 && isfinite(pq)) ? d.st.rho[s] / pq : 0.0;
    }
  }
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
