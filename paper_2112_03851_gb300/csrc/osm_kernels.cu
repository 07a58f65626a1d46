// CUDA kernels of the batched optimized Schwarz iteration (Sec. 3) with
// Jacobi-preconditioned CG subdomain solves (Sec. 6), written for sm_103a.
//
// Data layout (see osm_internal.h): the rows of all subdomains are
// concatenated, each subdomain padded to a multiple of 256 rows, so that
// CTA tile t (256 threads, 8 warps) covers rows [256 t, 256 t + 256) of one
// subdomain and warp w of the tile owns SELL slice 8 t + w (32 rows, one per
// lane).  Every kernel therefore runs all subdomains, of any size, in one
// launch; converged subdomains' tiles return at once.
//
// Reductions are deterministic: each tile writes its partial sums, and one
// warp adds a subdomain's partials in a fixed order (the start-of-solve
// finaliser k_fin_init, and the last block of each subdomain in the CG
// update).  Loop conditions are set with cudaGraphSetConditional by the last
// arrival at a ticket (an atomic counter taken once per block or subdomain);
// no kernel waits on another block.
#include <cuda_runtime.h>

#include "osm_device.cuh"
#include "osm_internal.h"

namespace osm {

namespace {

// ------------------------------------------------------------------ kernels

// Transmission part of one interface entry: p_lo M_lo + p_hi M_hi + q_lo S_lo
// + q_hi S_hi (c: the subdomain's p_lo, q_lo, p_hi, q_hi; t: the entry's
// M_lo, M_hi, S_lo, S_hi).
__device__ __forceinline__ double tc_term(const double* __restrict__ c, const double* __restrict__ t) {
  return fma(c[0], t[0], fma(c[2], t[1], fma(c[1], t[2], c[3] * t[3])));
}

// Local matrix A_i = K_i + sum over faces (p M_G + q S_G) on interface rows
// (Sec. 3; zeroth-order Robin: q = 0), and its diagonal.
__global__ void k_set_robin(DevProblem d) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_irow) return;
  const double* c = d.tc + 4 * d.irow_sub[k];
  for (int32_t e = d.im_ptr[k]; e < d.im_ptr[k + 1]; ++e) {
    const double t = tc_term(c, d.im_tc + 4 * (int64_t)e);
    const double a = d.im_kval[e] + t;
    d.im_t[e] = t;
    d.vals[d.im_pos[e]] = a;
    if (d.vals32) d.vals32[d.im_pos32[e]] = (float)a;
  }
  const int32_t row = d.irow[k];
  const double di = 1.0 / (d.kdiag[row] + tc_term(c, d.irow_tdiag + 4 * (int64_t)k));
  d.dinv[row] = di;
  if (d.dinv32) d.dinv32[row] = (float)di;
  if (d.dinv32b) d.dinv32b[d.row_box[row]] = (float)di;   // box layout of the tensor form
}

// b_i = f_i + sum_j lam_ij on interface rows (other rows keep b = f).
__global__ void k_rhs_gather(DevProblem d) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k == 0) {
    d.ctl->n_active = 0;
    d.ctl->n_inner = 0;
    if (d.ctl->t_start_ns == 0ull) d.ctl->t_start_ns = global_ns();
  }
  if (k >= d.n_irow) return;
  const int32_t row = d.irow[k];
  double b = d.f[row];
  for (int32_t e = d.ilam_ptr[k]; e < d.ilam_ptr[k + 1]; ++e) b += d.lam[d.ilam[e]];
  d.b[row] = b;
}

// CG start from the warm iterate x: r = b - A x, z = D^-1 r, p = z, and the
// tile partials of ||r||^2, ||b||^2 and r.z (finalised by k_fin_init); y =
// A x is kept for the stop test of the iteration that produced x.
template <int RPL, bool C16>
__global__ void __launch_bounds__(kTileRows) k_cg_init(DevProblem d) {
  __shared__ double sm[3][kTileRows / RPL];
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int64_t t0 = d.sub_tile0[s];
  double ax[RPL];
  int64_t row[RPL];
  tile_rows_any<double, RPL, C16>(d, d.vals, tile, d.x + t0 * kTileRows, ax, row);
  double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const double b = d.b[row[k]];
    const double r = b - ax[k];
    const double z = d.dinv[row[k]] * r;
    d.y[row[k]] = ax[k];
    d.r[row[k]] = r;
    d.z[row[k]] = z;
    d.p[row[k]] = z;
    v[0] += r * r;
    v[1] += b * b;
    v[2] += r * z;
  }
  block_sum_d<3, kTileRows / RPL>(v, sm);
  if (threadIdx.x == 0) {
    d.part0[tile] = v[0];
    d.part1[tile] = v[1];
    d.part2[tile] = v[2];
  }
}

// Dot-product partial of one tile.  FP64 solve: FP64 products and sums.
// FP32 inner solve: the warp adds FP32 products of the scaled factors
// (x sc, y sc) and only the warp's sum is widened and unscaled (x isc2 =
// 1/sc^2, exact); on this GPU FP64 arithmetic is scarce, and per-row FP64
// sums made the short vector kernels ALU-bound.  Result in thread 0.
template <class T, int NV, int NW>
__device__ __forceinline__ void tile_dots(T (&v)[NV], double isc2, double (*sm)[kTileSlices], double (&out)[NV]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T t = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sm[k][warp] = (double)t * isc2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) s += sm[k][w];
      out[k] = s;
    }
  }
}

// q = A p and the tile partials of p.q on active subdomains (T = double for
// the FP64 solve, float for the mixed-precision inner solve).
template <class T, int RPL, bool C16>
__global__ void __launch_bounds__(kTileRows) k_cg_spmv(DevProblem d, CgVec<T> v) {
  __shared__ double sm[1][kTileRows / RPL];
  __shared__ bool s_last;
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  if (!d.st.active[s]) return;
  const int64_t t0 = d.sub_tile0[s];
  const T sc = sizeof(T) == 4 ? (T)d.st.sc[s] : T(1);
  T q[RPL];
  int64_t row[RPL];
  tile_rows_any<T, RPL, C16>(d, v.vals, tile, v.p + t0 * kTileRows, q, row);
  T vv[1] = {T(0)};
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    v.q[row[k]] = q[k];
    vv[0] = fma(v.p[row[k]] * sc, q[k] * sc, vv[0]);
  }
  double out[1] = {(double)vv[0]};
  block_sum_d<1, kTileRows / RPL>(out, sm);
  if (threadIdx.x == 0) d.part0[tile] = out[0] * (sizeof(T) == 4 ? d.st.isc2[s] : 1.0);
  cg_alpha_ticket(d, s, &s_last);
}

// Per-subdomain finalisers: one warp per subdomain adds the subdomain's tile
// partials in a fixed order and updates its CG scalars, so the big kernels
// carry no fences or atomics.  Launched with fin_blocks() blocks.

// CG start: rho, ||b||^2, ||r||^2, the active flag; the last block sets the
// inner loop condition.  mixed (the refinement forms): the partials are
// ||d||^2, ||b||^2, r.z with d the FP64 defect, the inner solve's reference
// norm is ||d||, and a subdomain whose defect already meets inner_rtol is not
// corrected.
__global__ void k_fin_init(DevProblem d, int mixed, unsigned long long cond, int use_cond) {
  __shared__ bool flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * kTileSlices + warp;
  // a graph that runs the subdomain solves alone (no k_rhs_gather) starts the
  // wall clock here; the ticket's fence publishes it to the last block
  if (blockIdx.x == 0 && threadIdx.x == 0 && d.ctl->t_start_ns == 0ull) d.ctl->t_start_ns = global_ns();
  if (s < d.n_sub) {
    const int64_t nt = d.sub_tile0[s + 1] - d.sub_tile0[s];      // the subdomain's 256-row tiles
    const int64_t i0 = d.sub_init0[s], ni = d.sub_init0[s + 1] - i0;   // its CG-start partials
    const double a0 = warp_sum_parts(d.part0, i0, ni);
    const double a1 = warp_sum_parts(d.part1, i0, ni);
    const double a2 = warp_sum_parts(d.part2, i0, ni);
    if (lane == 0) {
      d.st.rr[s] = a0;
      d.st.bb[s] = mixed ? a0 : a1;
      d.st.rho[s] = a2;
      d.st.beta[s] = 0.0;
      d.st.iters[s] = 0;
      d.st.status[s] = 0;
      // scale of the FP32 dot products: sc = 2^-e with 2^e ~ rms of the defect
      int e = 0;
      const double ms = a0 / (double)(nt * kTileRows);
      if (mixed && ms > 0.0 && isfinite(ms)) {
        frexp(sqrt(ms), &e);
        e = max(-120, min(120, e));
      }
      d.st.sc[s] = (float)ldexp(1.0, -e);
      d.st.isc2[s] = ldexp(1.0, 2 * e);
      const int act = !d.inst_done[d.sub_inst[s]] &&
                      (mixed ? (!(a0 <= d.ctl->tau2_outer * a1) && a2 > 0.0) : !(a0 <= d.ctl->tau2 * a1));
      d.st.active[s] = act;
      if (act) atomicAdd(&d.ctl->n_active, 1);
    }
  }
  if (last_block(&d.ctl->gcnt_i, gridDim.x, &flag) && threadIdx.x == 0) {
    const bool more = d.ctl->n_active > 0 && !out_of_time(d.ctl);
    if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
}

// End of a CG step for subdomain s, by one warp (the finishing block of
// k_cg_update_a): rho = r.z, the stop test ||r|| <= tau ||b|| (or the
// iteration cap), beta, from the partials in a fixed order (r.z and ||r||^2:
// one per update block, [ub0[s], ub0[s+1]); p.q: one per tile or tensor CTA,
// sub_part0).  A subdomain whose p.q partials (k_cg_update_a left its
// iterate alone) sum to <= 0 stops with a breakdown.
__device__ __forceinline__ void cg_step_finish(DevProblem& d, const int64_t* __restrict__ ub0, int s, int lane) {
  const int64_t b0 = ub0[s], nb = ub0[s + 1] - b0;
  const double rz = warp_sum_parts(d.part1, b0, nb);
  const double rr = warp_sum_parts(d.part2, b0, nb);
  const double pq = d.st.pq[s];   // formed by the step's SpMV kernel (cg_alpha_ticket)
  if (lane == 0) {
    const int it = d.st.iters[s] + 1;
    d.st.iters[s] = it;
    d.st.tsteps[s] += 1;
    d.st.rr[s] = rr;
    if (!(pq > 0.0) || !isfinite(pq)) {
      d.st.status[s] |= 2;
      atomicOr(&d.ctl->status, 2);
      d.st.active[s] = 0;
      atomicSub(&d.ctl->n_active, 1);
    } else if (rr <= d.ctl->tau2 * d.st.bb[s]) {
      d.st.active[s] = 0;
      atomicSub(&d.ctl->n_active, 1);
    } else if (it >= d.ctl->max_inner) {
      d.st.active[s] = 0;
      d.st.status[s] |= 1;
      atomicOr(&d.ctl->status, 1);
      atomicSub(&d.ctl->n_active, 1);
    }
    d.st.beta[s] = rz / d.st.rho[s];
    d.st.rho[s] = rz;
  }
}

// Every subdomain arrives here once per CG step (its finishing block, or the
// first block of an inactive one); the last of the n_sub arrivals counts the
// step and sets the inner loop condition.  A ticket, not a wait.
__device__ __forceinline__ void cg_step_arrive(DevProblem& d, unsigned long long cond, int use_cond) {
  __threadfence();
  const unsigned g = atomicAdd(&d.ctl->gcnt_b, 1u);
  if (g != (unsigned)d.n_sub - 1u) return;
  d.ctl->gcnt_b = 0u;
  __threadfence();
  const int n_inner = d.ctl->n_inner + 1;
  d.ctl->n_inner = n_inner;
  d.ctl->total_inner += 1;
  const bool more = atomicAdd(&d.ctl->n_active, 0) > 0 && n_inner <= d.ctl->max_inner && !out_of_time(d.ctl);
  if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
}

// p = z + beta p for subdomains still iterating.
template <class T>
__global__ void __launch_bounds__(kTileRows) k_cg_direction(DevProblem d, CgVec<T> v) {
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  if (!d.st.active[s]) return;
  const int64_t row = tile * kTileRows + threadIdx.x;
  v.p[row] = fma((T)d.st.beta[s], v.p[row], v.z[row]);
}

// FP32 inner CG of the mixed form in two kernels per step.  With t = A z,
// the direction update moves into the SpMV's epilogue:
//   p = z + beta p,   q = A p = t + beta q   (first step, beta = 0: p = z, q = t)
// and alpha = rho / (p.q) and beta are formed inside the update kernel, so
// k_cg_direction and the separate alpha and beta kernels of the textbook
// step drop out: the same vector traffic, fewer launches and one pass over
// the vectors fewer.
template <int RPL, bool C16>
__global__ void __launch_bounds__(kTileRows) k_cg_spmv_dir32(DevProblem d) {
  __shared__ double sm[1][kTileSlices];
  __shared__ bool s_last;
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  if (!d.st.active[s]) return;
  const int64_t t0 = d.sub_tile0[s];
  const double beta64 = d.st.beta[s];
  const bool first = beta64 == 0.0;   // uniform per subdomain: no read of p, q
  const float beta = (float)beta64, sc = d.st.sc[s];
  float t[RPL];
  int64_t row[RPL];
  tile_rows_any<float, RPL, C16>(d, d.vals32, tile, d.z32 + t0 * kTileRows, t, row);
  float vv[1] = {0.f};
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const float z = d.z32[row[k]];
    float p = z, q = t[k];
    if (!first) {
      p = fmaf(beta, d.p32[row[k]], z);
      q = fmaf(beta, d.q32[row[k]], t[k]);
    }
    d.p32[row[k]] = p;
    d.q32[row[k]] = q;
    vv[0] = fmaf(p * sc, q * sc, vv[0]);
  }
  double out[1];
  tile_dots<float, 1, kTileSlices / RPL>(vv, d.st.isc2[s], sm, out);
  if (threadIdx.x == 0) d.part0[tile] = out[0];
  cg_alpha_ticket(d, s, &s_last);
}

// With alpha = rho / (p.q) from the step's SpMV kernel (cg_alpha_ticket; 0
// on a breakdown, which leaves the iterate alone and makes the step's finish
// stop the subdomain): x += alpha p, r -= alpha q, z = D^-1 r, and the
// block's partials of r.z and ||r||^2; the subdomain's last block to finish
// then ends the step (cg_step_finish, cg_step_arrive).  A block covers up to
// G consecutive tiles of one subdomain (d.ub_tile0 / d.ub64_tile0; FP32: 8,
// FP64: 2, which keeps its registers, and so its occupancy, up).  Each
// thread adds its rows' r.z and r.r in row order, the block adds its
// threads' sums in a fixed order and writes one partial pair per block.
// T = double: the FP64 CG (FP64 dots, staged in shared memory: FP64 adds are
// scarce); the mixed form's FP32 update is k_cg_update32.
template <class T, int G>
__global__ void __launch_bounds__(kTileRows) k_cg_update_a(DevProblem d, CgVec<T> v, unsigned long long cond,
                                                           int use_cond) {
  __shared__ double sm[2][kTileSlices];
  __shared__ double sm64[sizeof(T) == 8 ? 2 : 1][sizeof(T) == 8 ? kTileRows : 1];
  __shared__ bool s_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ub = blockIdx.x;
  const int64_t t0 = (G == kUpdGroup ? d.ub_tile0 : d.ub64_tile0)[ub];
  const int64_t* __restrict__ ub0 = G == kUpdGroup ? d.sub_ub0 : d.sub_ub64_0;
  const int s = d.tile_sub[t0];
  const int64_t ts0 = d.sub_tile0[s];
  if (!d.st.active[s]) {
    if (t0 == ts0 && threadIdx.x == 0) cg_step_arrive(d, cond, use_cond);
    return;
  }
  const int nt = (int)min((int64_t)G, d.sub_tile0[s + 1] - t0);
  T pr[G], xr[G], qr[G], rr0[G], di[G];
#pragma unroll
  for (int j = 0; j < G; ++j) {
    if (j < nt) {
      const int64_t row = (t0 + j) * kTileRows + threadIdx.x;
      pr[j] = v.p[row];
      xr[j] = v.x[row];
      qr[j] = v.q[row];
      rr0[j] = v.r[row];
      di[j] = v.dinv[row];
    }
  }
  const T alpha = (T)d.st.alpha[s];   // formed by the step's SpMV kernel (cg_alpha_ticket)
  const T sc = sizeof(T) == 4 ? (T)d.st.sc[s] : T(1);
  T a = T(0), b = T(0);
#pragma unroll
  for (int j = 0; j < G; ++j) {
    if (j < nt) {
      const int64_t row = (t0 + j) * kTileRows + threadIdx.x;
      v.x[row] = fma(alpha, pr[j], xr[j]);
      const T r = fma(-alpha, qr[j], rr0[j]);
      const T z = di[j] * r;
      v.r[row] = r;
      v.z[row] = z;
      if constexpr (sizeof(T) == 8) {   // FP64: no scaling (FP64 multiplies are scarce)
        a = fma(r, z, a);
        b = fma(r, r, b);
      } else {
        const T rs = r * sc;
        a = fma(rs, z * sc, a);
        b = fma(rs, rs, b);
      }
    }
  }
  if constexpr (sizeof(T) == 8) {
    double vv[2] = {a, b};
    block_sum_d<2, kTileRows>(vv, sm64);
    if (threadIdx.x == 0) {
      d.part1[ub] = vv[0];
      d.part2[ub] = vv[1];
    }
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      const double isc2 = d.st.isc2[s];
      sm[0][warp] = (double)a * isc2;
      sm[1][warp] = (double)b * isc2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int w = 0; w < kTileSlices; ++w) {
        s0 += sm[0][w];
        s1 += sm[1][w];
      }
      d.part1[ub] = s0;
      d.part2[ub] = s1;
    }
  }
  // the last block of the subdomain to get here finishes its CG step
  // (replaces a separate finaliser launch per step)
  if (threadIdx.x == 0) {
    __threadfence();   // publish the partials before the ticket
    const unsigned nblk = (unsigned)(ub0[s + 1] - ub0[s]);
    const unsigned t = atomicAdd(&d.st.ucnt[s], 1u);
    s_last = t == nblk - 1u;
    if (s_last) d.st.ucnt[s] = 0u;
  }
  __syncthreads();
  if (!s_last || warp != 0) return;
  __threadfence();
  cg_step_finish(d, ub0, s, lane);
  if (lane == 0) cg_step_arrive(d, cond, use_cond);
}

// The FP32 update of the mixed form's inner CG with 16-byte accesses: the
// same arithmetic as k_cg_update_a<float, kUpdGroup> (alpha, x += alpha p,
// r -= alpha q, z = D^-1 r, scaled r.z and r.r per block, the subdomain's
// last block finishing the step), but a thread owns 4 consecutive rows per
// 1024-row half of the block's 2048 rows and moves each vector's values with
// one float4 load or store: a quarter of the load and store instructions.
__global__ void __launch_bounds__(kTileRows) k_cg_update32(DevProblem d, CgVec<float> v, unsigned long long cond,
                                                           int use_cond) {
  constexpr int G = kUpdGroup;
  constexpr int H = G * kTileRows / (4 * kTileRows);   // float4 groups per thread (2)
  __shared__ double sm[2][kTileSlices];
  __shared__ bool s_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ub = blockIdx.x;
  const int64_t t0 = d.ub_tile0[ub];
  const int s = d.tile_sub[t0];
  const int64_t ts0 = d.sub_tile0[s];
  if (!d.st.active[s]) {
    if (t0 == ts0 && threadIdx.x == 0) cg_step_arrive(d, cond, use_cond);
    return;
  }
  const int64_t nrows = min((int64_t)G, d.sub_tile0[s + 1] - t0) * kTileRows;
  const int64_t r0 = t0 * kTileRows;
  float4 pr[H], xr[H], qr[H], rr0[H], di[H];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const int64_t o = 4 * (int64_t)threadIdx.x + (int64_t)h * 4 * kTileRows;
    if (o < nrows) {
      pr[h] = *reinterpret_cast<const float4*>(v.p + r0 + o);
      xr[h] = *reinterpret_cast<const float4*>(v.x + r0 + o);
      qr[h] = *reinterpret_cast<const float4*>(v.q + r0 + o);
      rr0[h] = *reinterpret_cast<const float4*>(v.r + r0 + o);
      di[h] = *reinterpret_cast<const float4*>(v.dinv + r0 + o);
    }
  }
  const float alpha = (float)d.st.alpha[s];   // formed by the step's SpMV kernel
  const float sc = d.st.sc[s];
  float a = 0.f, b = 0.f;
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const int64_t o = 4 * (int64_t)threadIdx.x + (int64_t)h * 4 * kTileRows;
    if (o < nrows) {
      float4 x, r, z;
      x.x = fmaf(alpha, pr[h].x, xr[h].x);
      x.y = fmaf(alpha, pr[h].y, xr[h].y);
      x.z = fmaf(alpha, pr[h].z, xr[h].z);
      x.w = fmaf(alpha, pr[h].w, xr[h].w);
      r.x = fmaf(-alpha, qr[h].x, rr0[h].x);
      r.y = fmaf(-alpha, qr[h].y, rr0[h].y);
      r.z = fmaf(-alpha, qr[h].z, rr0[h].z);
      r.w = fmaf(-alpha, qr[h].w, rr0[h].w);
      z.x = di[h].x * r.x;
      z.y = di[h].y * r.y;
      z.z = di[h].z * r.z;
      z.w = di[h].w * r.w;
      *reinterpret_cast<float4*>(v.x + r0 + o) = x;
      *reinterpret_cast<float4*>(v.r + r0 + o) = r;
      *reinterpret_cast<float4*>(v.z + r0 + o) = z;
      const float rs0 = r.x * sc, rs1 = r.y * sc, rs2 = r.z * sc, rs3 = r.w * sc;
      a = fmaf(rs0, z.x * sc, a);
      a = fmaf(rs1, z.y * sc, a);
      a = fmaf(rs2, z.z * sc, a);
      a = fmaf(rs3, z.w * sc, a);
      b = fmaf(rs0, rs0, b);
      b = fmaf(rs1, rs1, b);
      b = fmaf(rs2, rs2, b);
      b = fmaf(rs3, rs3, b);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    const double isc2 = d.st.isc2[s];
    sm[0][warp] = (double)a * isc2;
    sm[1][warp] = (double)b * isc2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int w = 0; w < kTileSlices; ++w) {
      s0 += sm[0][w];
      s1 += sm[1][w];
    }
    d.part1[ub] = s0;
    d.part2[ub] = s1;
    __threadfence();   // publish the partials before the ticket
    const unsigned nblk = (unsigned)(d.sub_ub0[s + 1] - d.sub_ub0[s]);
    const unsigned t = atomicAdd(&d.st.ucnt[s], 1u);
    s_last = t == nblk - 1u;
    if (s_last) d.st.ucnt[s] = 0u;
  }
  __syncthreads();
  if (!s_last || warp != 0) return;
  __threadfence();
  cg_step_finish(d, d.sub_ub0, s, lane);
  if (lane == 0) cg_step_arrive(d, cond, use_cond);
}

// Profiling state: every subdomain active, beta = 1/2 (the full epilogue of
// k_cg_spmv_dir32 runs), unit dot scale.
__global__ void k_profile_state(DevProblem d, int stride) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.n_sub) return;
  d.st.active[s] = s % stride == 0 ? 1 : 0;
  d.st.beta[s] = 0.5;
  d.st.sc[s] = 1.f;
  d.st.isc2[s] = 1.0;
}

// Mixed precision, start of one refinement step: FP64 defect
// d = b - A u (FP64 values and accumulation), then the FP32 CG on A e = d
// from e = 0: r = d, z = D^-1 r, p = z, and the tile partials of ||d||^2,
// ||b||^2 and r.z (k_fin_init decides which subdomains are corrected); y =
// A u is kept for the stop test.
template <int RPL, bool C16>
__global__ void __launch_bounds__(kTileRows) k_cg_init_mixed(DevProblem d) {
  __shared__ double sm[3][kTileRows / RPL];
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int64_t t0 = d.sub_tile0[s];
  double ax[RPL];
  int64_t row[RPL];
  tile_rows_any<double, RPL, C16>(d, d.vals, tile, d.x + t0 * kTileRows, ax, row);
  double vv[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const double b = d.b[row[k]];
    const double dfc = b - ax[k];
    d.y[row[k]] = ax[k];
    const float r = (float)dfc;
    float z = 0.f;
    // the FP32 solve's row: the same row, or its row in the tensor form's box layout
    const int64_t rb = d.t32 ? (int64_t)d.row_box[row[k]] : row[k];
    if (rb >= 0) {
      z = (d.t32 ? d.dinv32b : d.dinv32)[rb] * r;
      d.r32[rb] = r;
      d.z32[rb] = z;   // p = z is formed by the first CG-step kernel (beta = 0)
      d.x32[rb] = 0.f;
    }
    vv[0] += dfc * dfc;
    vv[1] += b * b;
    vv[2] += (double)r * (double)z;
  }
  block_sum_d<3, kTileRows / RPL>(vv, sm);
  if (threadIdx.x == 0) {
    d.part0[tile] = vv[0];
    d.part1[tile] = vv[1];
    d.part2[tile] = vv[2];
  }
}

// Mixed precision, end of the refinement step: u += e in FP64 (e read from
// the tensor form's box layout when that is in use).
__global__ void __launch_bounds__(kTileRows) k_mixed_correct(DevProblem d) {
  const int64_t row = blockIdx.x * (int64_t)kTileRows + threadIdx.x;
  if (d.t32) {
    const int32_t rb = d.row_box[row];
    if (rb >= 0) {
      const double u = d.x[row] + (double)d.x32[rb];
      d.x[row] = u;
      if (d.ub) d.ub[rb] = u;   // the box-layout mirrors read by the tensor starts
      if (d.ub2) d.ub2[rb] = df_split(u);
    }
  } else {
    d.x[row] += (double)d.x32[row];
  }
}

// The iterate u copied into its box-layout mirrors (when a tensor start is
// switched on for a handle whose iterate is not zero).
__global__ void __launch_bounds__(kTileRows) k_box_mirror(DevProblem d) {
  const int64_t row = blockIdx.x * (int64_t)kTileRows + threadIdx.x;
  const int32_t rb = d.row_box[row];
  if (rb >= 0) {
    if (d.ub) d.ub[rb] = d.x[row];
    if (d.ub2) d.ub2[rb] = df_split(d.x[row]);
  }
}

// y32 = A32 x32 (FP32 values) on every tile: the mixed inner operator.
template <int RPL, bool C16>
__global__ void __launch_bounds__(kTileRows) k_spmv_plain32(DevProblem d, const float* __restrict__ x,
                                                            float* __restrict__ y) {
  const int64_t tile = blockIdx.x;
  const int64_t t0 = d.sub_tile0[d.tile_sub[tile]];
  float q[RPL];
  int64_t row[RPL];
  tile_rows_any<float, RPL, C16>(d, d.vals32, tile, x + t0 * kTileRows, q, row);
#pragma unroll
  for (int k = 0; k < RPL; ++k) y[row[k]] = q[k];
}

// Canonical local layout <-> the FP32 solve's rows (box rows under the tensor form).
__device__ __forceinline__ int64_t row32_of(const DevProblem& d, int64_t k) {
  const int32_t r = d.can2vec[k];
  return d.t32 ? (int64_t)d.row_box[r] : (int64_t)r;
}

__global__ void k_scatter_local32(DevProblem d, const double* __restrict__ canon, float* __restrict__ vec) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_local) return;
  vec[row32_of(d, k)] = (float)canon[k];
}

__global__ void k_gather_local32(DevProblem d, const float* __restrict__ vec, double* __restrict__ canon) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_local) return;
  canon[k] = (double)vec[row32_of(d, k)];
}

// Robin exchange on every face entry (parallel update, Sec. 3):
// lam_st <- (p_s + p_t) M u_t - lam_ts, lam_ts <- (p_s + p_t) M u_s - lam_st.
__global__ void k_exchange(DevProblem d) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= d.n_fent) return;
  const int f = d.fent_face[e];
  if (d.inst_done[d.sub_inst[d.face_s[f]]]) return;
  const int64_t eo = d.face_eo[f];
  const int32_t nf = d.face_n[f];
  const int64_t m = e - eo;
  // s is the lower side of the face: its (p_lo, q_lo) plus t's (p_hi, q_hi)
  const double* cs = d.tc + 4 * d.face_s[f];
  const double* ct = d.tc + 4 * d.face_t[f];
  const double pp = cs[0] + ct[2], qq = cs[1] + ct[3];
  double mus = 0.0, mut = 0.0, sus = 0.0, sut = 0.0;
  const int32_t k0 = d.fm_ptr[e], k1 = d.fm_ptr[e + 1];
  if (qq == 0.0) {   // zeroth-order Robin: the face mass only
#pragma unroll 4
    for (int32_t k = k0; k < k1; ++k) {
      const double mv = d.fm_val[k];
      const int32_t c = d.fm_col[k];
      mus = fma(mv, d.x[d.fent_row_s[c]], mus);
      mut = fma(mv, d.x[d.fent_row_t[c]], mut);
    }
  } else {
#pragma unroll 4
    for (int32_t k = k0; k < k1; ++k) {
      const double mv = d.fm_val[k], sv = d.fs_val[k];
      const int32_t c = d.fm_col[k];
      const double xs = d.x[d.fent_row_s[c]], xt = d.x[d.fent_row_t[c]];
      mus = fma(mv, xs, mus);
      mut = fma(mv, xt, mut);
      sus = fma(sv, xs, sus);
      sut = fma(sv, xt, sut);
    }
  }
  double* lst = d.lam + 2 * eo + m;
  double* lts = d.lam + 2 * eo + nf + m;
  const double old_st = *lst, old_ts = *lts;
  *lst = fma(pp, mut, qq * sut) - old_ts;
  *lts = fma(pp, mus, qq * sus) - old_st;
}

// Stop test, step 1, at the interface nodes (two or more copies): ubar =
// average of the copies, scattered back to every copy (w) and, on handles
// with a box layout, ubar - u for the tensor layer.  A node with one copy
// has ubar = u, so ubar - u = 0 there (dl32 stays zero) and its w is never
// read; phi is formed once per call by k_phi.
__global__ void k_average(DevProblem d) {
  const int b = blockIdx.x;
  if (d.inst_done[d.iblock_inst[b]]) return;
  for (int64_t k = d.iblock0[b] + threadIdx.x; k < d.iblock0[b + 1]; k += blockDim.x) {
    const int32_t n = d.inodes[k];
    const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
    double s = 0.0;
    for (int32_t c = c0; c < c1; ++c) s += d.x[d.cp_idx[c]];
    const double ub = copy_mean(s, c1 - c0);
    for (int32_t c = c0; c < c1; ++c) {
      const int32_t r = d.cp_idx[c];
      d.w[r] = ub;
      if (d.dl32) d.dl32[d.row_box[r]] = (float)(ub - d.x[r]);   // ubar - u for the tensor layer
    }
  }
}

// y = A x on every tile (all subdomains).
template <int RPL, bool C16>
__global__ void __launch_bounds__(kTileRows) k_spmv_plain(DevProblem d, const double* __restrict__ x,
                                                          double* __restrict__ y) {
  const int64_t tile = blockIdx.x;
  const int64_t t0 = d.sub_tile0[d.tile_sub[tile]];
  double q[RPL];
  int64_t row[RPL];
  tile_rows_any<double, RPL, C16>(d, d.vals, tile, x + t0 * kTileRows, q, row);
#pragma unroll
  for (int k = 0; k < RPL; ++k) y[row[k]] = q[k];
}

// y -= (transmission part of A_i) x on interface rows: turns A_i x into K_i x.
__global__ void k_face_correct(DevProblem d, const double* __restrict__ x, double* __restrict__ y) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_irow) return;
  double acc = 0.0;
  for (int32_t e = d.im_ptr[k]; e < d.im_ptr[k + 1]; ++e) acc = fma(d.im_t[e], x[d.im_col[e]], acc);
  const int32_t row = d.irow[k];
  y[row] -= acc;
}

// Stop test: y = A u (from the CG start) becomes K ubar = A u - T u +
// K (ubar - u); ubar - u vanishes off the interface rows, so only the
// interface-column layer of K is applied (w = ubar on every copy, x = u), and
// on interface rows the transmission part T u (face mass and face stiffness
// terms, the same entries as k_face_correct) is taken off.  Eight threads per
// row, each taking every eighth entry, so that a row's entries are read as
// contiguous runs; their sums are added in a fixed shuffle order.
constexpr int kLayerLanes = 8;
__global__ void __launch_bounds__(256) k_stop_layer(DevProblem d) {
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kLayerLanes;
  const int sub = threadIdx.x & (kLayerLanes - 1);
  double acc = 0.0;
  if (k < d.n_lrow) {
    for (int32_t e = d.li_ptr[k] + sub; e < d.li_ptr[k + 1]; e += kLayerLanes) {
      const int32_t c = d.li_col[e];
      acc = fma(d.li_val[e], d.w[c] - d.x[c], acc);
    }
    const int32_t ir = d.li_irow[k];
    if (ir >= 0)
      for (int32_t e = d.im_ptr[ir] + sub; e < d.im_ptr[ir + 1]; e += kLayerLanes)
        acc = fma(-d.im_t[e], d.x[d.im_col[e]], acc);
  }
#pragma unroll
  for (int o = kLayerLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (k < d.n_lrow && sub == 0) d.y[d.li_row[k]] += acc;
}

// Stop test, step 2, at the interface nodes: r = sum_copies f -
// sum_copies K_i ubar per node and the per-block partials of ||r||^2 (no
// tickets: the single-block k_residual_fin adds them to those of
// k_residual_rows).  A node with one copy is the single-copy row's, r = f -
// y there, and k_residual_rows streams those; a node without copies
// (Dirichlet) has r = 0.
__global__ void __launch_bounds__(256) k_residual(DevProblem d) {
  __shared__ double sm[1][256];
  const int b = blockIdx.x;
  double v[1] = {0.0};
  if (!d.inst_done[d.iblock_inst[b]]) {
    for (int64_t k = d.iblock0[b] + threadIdx.x; k < d.iblock0[b + 1]; k += blockDim.x) {
      const int32_t n = d.inodes[k];
      const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
      double ku = 0.0;
      for (int32_t c = c0; c < c1; ++c) ku += d.y[d.cp_idx[c]];
      const double r = d.fg[n] - ku;
      v[0] += r * r;
    }
  }
  block_sum_d<1, 256>(v, sm);
  if (threadIdx.x == 0) d.rpart[b] = v[0];
}

// Stop test, step 2 on the single-copy rows (every other row): r = f - y
// on the vector row itself, read as contiguous streams.  One warp per tile
// of 256 rows (8 rows per lane, no block barrier) and its partial of
// ||r||^2 per tile.  Padding rows have f = y = 0.
__global__ void __launch_bounds__(kTileRows) k_residual_rows(DevProblem d) {
  const int64_t tile = blockIdx.x * (int64_t)kTileSlices + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= d.n_tiles) return;
  if (d.inst_done[d.sub_inst[d.tile_sub[tile]]]) return;   // k_residual_fin skips the instance
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < kTileRows / 32; ++k) {
    const int64_t row = tile * kTileRows + k * 32 + lane;
    if (d.row_single[row]) {
      const double r = d.f[row] - d.y[row];
      v = fma(r, r, v);
    }
  }
  v = warp_sum(v);
  if (lane == 0) d.tpart[tile] = v;
}

// Marks the vector rows whose node has exactly one copy (setup).
__global__ void k_mark_single(DevProblem d, uint8_t* single) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < d.n_nodes;
       n += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
    if (c1 - c0 == 1) single[d.cp_idx[c0]] = 1;
  }
}

// phi = the average of the copies of every node (0 on the Dirichlet boundary,
// where a node has none), once at the end of a solve or iterate call.  An
// instance that finished earlier in the call has a frozen iterate (its
// subdomain solves add nothing and its exchange stops), so its phi is that of
// its last stop test.
__global__ void k_phi(DevProblem d) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < d.n_nodes;
       n += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
    double s = 0.0;
    for (int32_t c = c0; c < c1; ++c) s += d.x[d.cp_idx[c]];
    d.phi[n] = c0 == c1 ? 0.0 : copy_mean(s, c1 - c0);
  }
}

// Start of a solve: the assembled load f_n = sum over the copies of each
// node (constant during the solve) and the block partials of ||f||^2 that
// every stop test divides by.
__global__ void __launch_bounds__(256) k_load_nodes(DevProblem d) {
  __shared__ double sm[1][256];
  const int b = blockIdx.x;
  double v[1] = {0.0};
  for (int64_t n = d.rblock_node0[b] + threadIdx.x; n < d.rblock_node0[b + 1]; n += blockDim.x) {
    const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
    double fg = 0.0;
    for (int32_t c = c0; c < c1; ++c) fg += d.f[d.cp_idx[c]];
    d.fg[n] = fg;
    v[0] += fg * fg;
  }
  block_sum_d<1, 256>(v, sm);
  if (threadIdx.x == 0) d.rpart2[b] = v[0];
}

// Stop test, step 3 (one block): per instance, ||r|| / ||f|| from its block
// partials in a fixed order, its iteration count and whether it is done
// (reached rtol or max_outer); then counts the Schwarz iteration and sets
// the outer loop condition (any instance still running).
__global__ void __launch_bounds__(kResFinThreads) k_residual_fin(DevProblem d, unsigned long long cond, int use_cond) {
  __shared__ double sm[2][kResFinThreads / 32];
  const int n_outer = d.ctl->n_outer;
  for (int inst = 0; inst < d.n_inst; ++inst) {
    if (d.inst_done[inst]) continue;   // uniform across the block
    // ||f||^2: one partial per node block; ||r||^2: one per interface-node
    // block and one per tile of single-copy rows
    const int b0 = d.inst_rblock0[inst], nb = d.inst_rblock0[inst + 1] - b0;
    const int i0 = d.inst_iblock0[inst], ni = d.inst_iblock0[inst + 1] - i0;
    double u[2] = {0.0, 0.0}, w[2] = {0.0, 0.0};
    for (int k = threadIdx.x; k < nb; k += blockDim.x) u[1] += __ldcg(d.rpart2 + b0 + k);
    for (int k = threadIdx.x; k < ni; k += blockDim.x) u[0] += __ldcg(d.rpart + i0 + k);
    // the single-copy rows' partials, one per tile of the instance
    for (int64_t t = d.inst_tile0[inst] + threadIdx.x; t < d.inst_tile0[inst + 1]; t += blockDim.x)
      w[0] += __ldcg(d.tpart + t);
    u[0] += w[0];
    u[1] += w[1];
    block_sum<2, kResFinThreads / 32>(u, sm);
    if (threadIdx.x == 0) {
      const double rel = u[1] > 0.0 ? sqrt(u[0] / u[1]) : sqrt(u[0]);
      d.inst_relres[inst] = rel;
      d.inst_iters[inst] = n_outer + 1;
      if (d.n_inst == 1) {
        if (n_outer < d.ctl->max_outer) d.hist[n_outer] = rel;
        d.ctl->relres = rel;
      }
      if (!(rel > d.ctl->rtol) || !isfinite(rel) || n_outer + 1 >= d.ctl->max_outer) d.inst_done[inst] = 1;
    }
    __syncthreads();   // sm is reused by the next instance
  }
  if (threadIdx.x == 0) {
    d.ctl->n_outer = n_outer + 1;
    int running = 0;
    double worst = 0.0;
    for (int i = 0; i < d.n_inst; ++i) {
      running += !d.inst_done[i];
      worst = fmax(worst, d.inst_relres[i]);
    }
    if (d.n_inst > 1) d.ctl->relres = worst;
    d.ctl->running = running;
    const bool more = running > 0 && !out_of_time(d.ctl);
    if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
}

__global__ void k_scatter_local(DevProblem d, const double* __restrict__ canon, double* __restrict__ vec) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_local) return;
  vec[d.can2vec[k]] = canon[k];
}

__global__ void k_gather_local(DevProblem d, const double* __restrict__ vec, double* __restrict__ canon) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_local) return;
  canon[k] = vec[d.can2vec[k]];
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }
inline unsigned fin_blocks(const DevProblem& d) { return (unsigned)((d.n_sub + kTileSlices - 1) / kTileSlices); }

// Launch an SpMV-bearing kernel in the variant chosen at setup by the
// autotuner: RPL slices per warp (256 / RPL threads per 256-row tile) and
// 16- or 32-bit column indices (c16).
#define OSM_LAUNCH_RPL(rpl, c16, KERNEL, s, ...)                                                  \
  do {                                                                                            \
    if (c16) {                                                                                    \
      if ((rpl) == 2) KERNEL<2, true><<<(unsigned)d.n_tiles, kTileRows / 2, 0, s>>>(__VA_ARGS__); \
      else KERNEL<1, true><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(__VA_ARGS__);                \
    } else {                                                                                      \
      if ((rpl) == 2) KERNEL<2, false><<<(unsigned)d.n_tiles, kTileRows / 2, 0, s>>>(__VA_ARGS__); \
      else KERNEL<1, false><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(__VA_ARGS__);                \
    }                                                                                             \
  } while (0)

}  // namespace

cudaError_t launch_set_robin(const DevProblem& d, cudaStream_t s) {
  if (d.n_irow == 0) return cudaSuccess;
  k_set_robin<<<blocks_for(d.n_irow, 256), 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_rhs_gather(const DevProblem& d, cudaStream_t s) {
  k_rhs_gather<<<blocks_for(d.n_irow > 0 ? d.n_irow : 1, 256), 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond,
                           int defect_norm) {
  OSM_LAUNCH_RPL(d.rpl64, d.c16_64, k_cg_init, s, d);
  k_fin_init<<<fin_blocks(d), kTileRows, 0, s>>>(d, defect_norm, cond, use_cond);
  return cudaGetLastError();
}

cudaError_t launch_cg_iteration(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond) {
  const CgVec<double> v{d.x, d.r, d.z, d.p, d.q, d.dinv, d.vals};
  if (d.c16_64) {
    if (d.rpl64 == 2) k_cg_spmv<double, 2, true><<<(unsigned)d.n_tiles, kTileRows / 2, 0, s>>>(d, v);
    else k_cg_spmv<double, 1, true><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
  } else {
    if (d.rpl64 == 2) k_cg_spmv<double, 2, false><<<(unsigned)d.n_tiles, kTileRows / 2, 0, s>>>(d, v);
    else k_cg_spmv<double, 1, false><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
  }
  k_cg_update_a<double, kUpdGroup64><<<(unsigned)d.n_ublocks64, kTileRows, 0, s>>>(d, v, cond, use_cond);
  k_cg_direction<double><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
  return cudaGetLastError();
}

cudaError_t launch_cg_iteration32(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond) {
  if (d.t32) {
    const DevProblem b = fp32_view(d);
    cudaError_t e = launch_tensor_dir32(b, s);
    if (e != cudaSuccess) return e;
    const CgVec<float> v{b.x32, b.r32, b.z32, b.p32, b.q32, b.dinv32b, b.vals32};
    k_cg_update32<<<(unsigned)b.n_ublocks, kTileRows, 0, s>>>(b, v, cond, use_cond);
    return cudaGetLastError();
  }
  OSM_LAUNCH_RPL(d.rpl32, d.c16_32, k_cg_spmv_dir32, s, d);
  const CgVec<float> v{d.x32, d.r32, d.z32, d.p32, d.q32, d.dinv32, d.vals32};
  k_cg_update32<<<(unsigned)d.n_ublocks, kTileRows, 0, s>>>(d, v, cond, use_cond);
  return cudaGetLastError();
}

cudaError_t launch_cg_spmv_alone(const DevProblem& d, int fp32, cudaStream_t s) {
  if (fp32 && d.t32) return launch_tensor_dir32(fp32_view(d), s);
  if (fp32) {
    OSM_LAUNCH_RPL(d.rpl32, d.c16_32, k_cg_spmv_dir32, s, d);
  } else {
    const CgVec<double> v{d.x, d.r, d.z, d.p, d.q, d.dinv, d.vals};
    if (d.c16_64) {
      if (d.rpl64 == 2) k_cg_spmv<double, 2, true><<<(unsigned)d.n_tiles, kTileRows / 2, 0, s>>>(d, v);
      else k_cg_spmv<double, 1, true><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
    } else {
      if (d.rpl64 == 2) k_cg_spmv<double, 2, false><<<(unsigned)d.n_tiles, kTileRows / 2, 0, s>>>(d, v);
      else k_cg_spmv<double, 1, false><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_profile_state(const DevProblem& d, cudaStream_t s, int stride) {
  k_profile_state<<<blocks_for(d.n_sub, 256), 256, 0, s>>>(d, stride < 1 ? 1 : stride);
  return cudaGetLastError();
}

cudaError_t launch_mixed_correct(const DevProblem& d, cudaStream_t s) {
  k_mixed_correct<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_spmv_plain32(const DevProblem& d, const float* x, float* y, cudaStream_t s) {
  if (d.t32) return launch_tensor_apply32(d, x, y, s);
  OSM_LAUNCH_RPL(d.rpl32, d.c16_32, k_spmv_plain32, s, d, x, y);
  return cudaGetLastError();
}

cudaError_t launch_apply32(const DevProblem& d, const double* x, double* y, cudaStream_t s) {
  k_scatter_local32<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, x, d.z32);
  cudaError_t e = launch_spmv_plain32(d, d.z32, d.q32, s);
  if (e != cudaSuccess) return e;
  k_gather_local32<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, d.q32, y);
  return cudaGetLastError();
}

cudaError_t launch_exchange(const DevProblem& d, cudaStream_t s) {
  if (d.n_fent == 0) return cudaSuccess;
  k_exchange<<<blocks_for(d.n_fent, 256), 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_spmv_plain(const DevProblem& d, const double* x, double* y, cudaStream_t s) {
  OSM_LAUNCH_RPL(d.rpl64, d.c16_64, k_spmv_plain, s, d, x, y);
  return cudaGetLastError();
}

cudaError_t launch_box_mirror(const DevProblem& d, cudaStream_t s) {
  k_box_mirror<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_cg_start(const DevProblem& d, cudaStream_t s, int mixed) {
  if (mixed && d.t64i == 2) return launch_tensor_init_df(d, s);
  if (mixed && d.t64i) return launch_tensor_init64(d, s);
  if (mixed) OSM_LAUNCH_RPL(d.rpl64, d.c16_64, k_cg_init_mixed, s, d);
  else OSM_LAUNCH_RPL(d.rpl64, d.c16_64, k_cg_init, s, d);
  return cudaGetLastError();
}

cudaError_t launch_fin_init(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond,
                            int defect_norm) {
  k_fin_init<<<fin_blocks(d), kTileRows, 0, s>>>(d, defect_norm, cond, use_cond);
  return cudaGetLastError();
}

cudaError_t launch_stop_test(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond) {
  if (d.n_iblocks) k_average<<<(unsigned)d.n_iblocks, 256, 0, s>>>(d);
  if (d.dl32) {   // box layout: the transmission part in FP64, K (ubar - u) by the FP32 tensor kernel
    if (d.n_irow) k_face_correct<<<blocks_for(d.n_irow, 256), 256, 0, s>>>(d, d.x, d.y);
    cudaError_t e = launch_tensor_layer(d, s);
    if (e != cudaSuccess) return e;
  } else if (d.n_lrow) {
    k_stop_layer<<<blocks_for((int64_t)d.n_lrow * kLayerLanes, 256), 256, 0, s>>>(d);
  }
  if (d.n_iblocks) k_residual<<<(unsigned)d.n_iblocks, 256, 0, s>>>(d);
  k_residual_rows<<<(unsigned)((d.n_tiles + kTileSlices - 1) / kTileSlices), kTileRows, 0, s>>>(d);
  k_residual_fin<<<1, kResFinThreads, 0, s>>>(d, cond, use_cond);
  return cudaGetLastError();
}

cudaError_t launch_mark_single(const DevProblem& d, uint8_t* single, cudaStream_t s) {
  k_mark_single<<<kNodeBlocks, 256, 0, s>>>(d, single);
  return cudaGetLastError();
}

cudaError_t launch_phi(const DevProblem& d, cudaStream_t s) {
  k_phi<<<kNodeBlocks, 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_load_nodes(const DevProblem& d, cudaStream_t s) {
  k_load_nodes<<<(unsigned)d.n_rblocks, 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_apply(const DevProblem& d, int op, const double* x, double* y, cudaStream_t s) {
  k_scatter_local<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, x, d.w);
  OSM_LAUNCH_RPL(d.rpl64, d.c16_64, k_spmv_plain, s, d, d.w, d.y);
  if (op == 1 && d.n_irow) k_face_correct<<<blocks_for(d.n_irow, 256), 256, 0, s>>>(d, d.w, d.y);
  k_gather_local<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, d.y, y);
  return cudaGetLastError();
}

cudaError_t launch_apply_scratch(const DevProblem& d, int op, const double* x, double* y, double* w_scratch,
                                 double* y_scratch, cudaStream_t s) {
  k_scatter_local<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, x, w_scratch);
  OSM_LAUNCH_RPL(d.rpl64, d.c16_64, k_spmv_plain, s, d, w_scratch, y_scratch);
  if (op == 1 && d.n_irow) k_face_correct<<<blocks_for(d.n_irow, 256), 256, 0, s>>>(d, w_scratch, y_scratch);
  k_gather_local<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, y_scratch, y);
  return cudaGetLastError();
}

cudaError_t launch_gather_local(const DevProblem& d, const double* vec, double* canon, cudaStream_t s) {
  k_gather_local<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, vec, canon);
  return cudaGetLastError();
}

}  // namespace osm
