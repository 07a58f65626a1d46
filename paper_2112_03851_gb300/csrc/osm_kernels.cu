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
// Reductions are deterministic: each tile writes its partial sums, and the
// last tile of a subdomain to finish (atomic ticket) adds the subdomain's
// partials in a fixed order and updates that subdomain's CG scalars.  Kernels
// that steer a device-side loop do the same across the whole grid and call
// cudaGraphSetConditional from that single last block.
#include <cuda_runtime.h>

#include "osm_device.cuh"
#include "osm_internal.h"

namespace osm {

namespace {

// ------------------------------------------------------------------ kernels

// Robin matrix A_i = K_i + p_i M_Gi on interface rows, and its diagonal.
__global__ void k_set_robin(DevProblem d) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_irow) return;
  const int s = d.irow_sub[k];
  const double p = d.psub[s];
  for (int32_t e = d.im_ptr[k]; e < d.im_ptr[k + 1]; ++e) {
    const double a = d.im_kval[e] + p * d.im_val[e];
    d.vals[d.im_pos[e]] = a;
    if (d.vals32) d.vals32[d.im_pos32[e]] = (float)a;
  }
  const int32_t row = d.irow[k];
  const double di = 1.0 / (d.kdiag[row] + p * d.irow_mdiag[k]);
  d.dinv[row] = di;
  if (d.dinv32) d.dinv32[row] = (float)di;
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
// tile partials of ||r||^2, ||b||^2 and r.z (finalised by k_fin_init).
__global__ void __launch_bounds__(kTileRows) k_cg_init(DevProblem d) {
  __shared__ double sm[3][kTileSlices];
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s];
  const double* xs = d.x + t0 * kTileRows;
  const int64_t row = tile * kTileRows + threadIdx.x;
  const double ax = sell_row(d.cols, d.vals, off, w, lane, xs);
  const double b = d.b[row];
  const double r = b - ax;
  const double z = d.dinv[row] * r;
  d.r[row] = r;
  d.z[row] = z;
  d.p[row] = z;
  double v[3] = {r * r, b * b, r * z};
  block_sum<3>(v, sm);
  if (threadIdx.x == 0) {
    d.part0[tile] = v[0];
    d.part1[tile] = v[1];
    d.part2[tile] = v[2];
  }
}

// q = A p and the tile partials of p.q on active subdomains (T = double for
// the FP64 solve, float for the mixed-precision inner solve; dots in FP64).
template <class T>
__global__ void __launch_bounds__(kTileRows) k_cg_spmv(DevProblem d, CgVec<T> v) {
  __shared__ double sm[1][kTileSlices];
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  if (!d.st.active[s]) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s];
  const int64_t row = tile * kTileRows + threadIdx.x;
  const T q = sell_row(d.cols, v.vals, off, w, lane, v.p + t0 * kTileRows);
  v.q[row] = q;
  double vv[1] = {(double)v.p[row] * (double)q};
  block_sum<1>(vv, sm);
  if (threadIdx.x == 0) d.part0[tile] = vv[0];
}

// x += alpha p, r -= alpha q, z = D^-1 r, and the tile partials of r.z and
// ||r||^2 (k_fin_beta turns them into rho, the stop test and beta).
template <class T>
__global__ void __launch_bounds__(kTileRows) k_cg_update(DevProblem d, CgVec<T> v) {
  __shared__ double sm[2][kTileSlices];
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int act = d.st.active[s];
  if (act) {
    const int64_t row = tile * kTileRows + threadIdx.x;
    const T alpha = (T)d.st.alpha[s];
    const T pr = v.p[row];
    v.x[row] = fma(alpha, pr, v.x[row]);
    const T r = fma(-alpha, v.q[row], v.r[row]);
    const T z = v.dinv[row] * r;
    v.r[row] = r;
    v.z[row] = z;
    double vv[2] = {(double)r * (double)z, (double)r * (double)r};
    block_sum<2>(vv, sm);
    if (threadIdx.x == 0) {
      d.part1[tile] = vv[0];
      d.part2[tile] = vv[1];
    }
  }
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
  if (s < d.n_sub) {
    const int64_t t0 = d.sub_tile0[s], nt = d.sub_tile0[s + 1] - t0;
    const double a0 = warp_sum_parts(d.part0, t0, nt);
    const double a1 = warp_sum_parts(d.part1, t0, nt);
    const double a2 = warp_sum_parts(d.part2, t0, nt);
    if (lane == 0) {
      d.st.rr[s] = a0;
      d.st.bb[s] = mixed ? a0 : a1;
      d.st.rho[s] = a2;
      d.st.beta[s] = 0.0;
      d.st.iters[s] = 0;
      d.st.status[s] = 0;
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

// alpha = rho / (p.q), or a breakdown stop of the subdomain.
__global__ void k_fin_alpha(DevProblem d) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * kTileSlices + warp;
  if (s >= d.n_sub || !d.st.active[s]) return;
  const int64_t t0 = d.sub_tile0[s], nt = d.sub_tile0[s + 1] - t0;
  const double pq = warp_sum_parts(d.part0, t0, nt);
  if (lane == 0) {
    if (!(pq > 0.0) || !isfinite(pq)) {
      d.st.alpha[s] = 0.0;
      d.st.status[s] |= 2;
      atomicOr(&d.ctl->status, 2);
      d.st.active[s] = 0;
      atomicSub(&d.ctl->n_active, 1);
    } else {
      d.st.alpha[s] = d.st.rho[s] / pq;
    }
  }
}

// rho = r.z, the stop test ||r|| <= tau ||b|| (or the iteration cap), beta;
// the last block counts the step and sets the inner loop condition.
__global__ void k_fin_beta(DevProblem d, unsigned long long cond, int use_cond) {
  __shared__ bool flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * kTileSlices + warp;
  if (s < d.n_sub && d.st.active[s]) {
    const int64_t t0 = d.sub_tile0[s], nt = d.sub_tile0[s + 1] - t0;
    const double rz = warp_sum_parts(d.part1, t0, nt);
    const double rr = warp_sum_parts(d.part2, t0, nt);
    if (lane == 0) {
      const int it = d.st.iters[s] + 1;
      d.st.iters[s] = it;
      d.st.rr[s] = rr;
      if (rr <= d.ctl->tau2 * d.st.bb[s]) {
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
  if (last_block(&d.ctl->gcnt_b, gridDim.x, &flag) && threadIdx.x == 0) {
    const int n_inner = d.ctl->n_inner + 1;
    d.ctl->n_inner = n_inner;
    d.ctl->total_inner += 1;
    const bool more = d.ctl->n_active > 0 && n_inner <= d.ctl->max_inner && !out_of_time(d.ctl);
    if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
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

// Mixed precision, start of one refinement step: FP64 defect
// d = b - A u (FP64 values and accumulation), then the FP32 CG on A e = d
// from e = 0: r = d, z = D^-1 r, p = z.  A subdomain whose FP64 defect already
// meets the FP64 tolerance (||d|| <= inner_rtol ||b||) is not corrected; the
// FP32 solve stops at ||r|| <= mixed_inner_rtol ||d||.
__global__ void __launch_bounds__(kTileRows) k_cg_init_mixed(DevProblem d) {
  __shared__ double sm[3][kTileSlices];
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s];
  const int64_t row = tile * kTileRows + threadIdx.x;
  const double ax = sell_row(d.cols, d.vals, off, w, lane, d.x + t0 * kTileRows);
  const double b = d.b[row];
  const double dfc = b - ax;
  const float r = (float)dfc;
  const float z = d.dinv32[row] * r;
  d.r32[row] = r;
  d.z32[row] = z;
  d.p32[row] = z;
  d.x32[row] = 0.f;
  double vv[3] = {dfc * dfc, b * b, (double)r * (double)z};
  block_sum<3>(vv, sm);
  if (threadIdx.x == 0) {
    d.part0[tile] = vv[0];
    d.part1[tile] = vv[1];
    d.part2[tile] = vv[2];
  }
}

// Mixed precision, end of the refinement step: u += e in FP64.
__global__ void __launch_bounds__(kTileRows) k_mixed_correct(DevProblem d) {
  const int64_t row = blockIdx.x * (int64_t)kTileRows + threadIdx.x;
  d.x[row] += (double)d.x32[row];
}

// y32 = A32 x32 (FP32 values) on every tile: the mixed inner operator.
__global__ void __launch_bounds__(kTileRows) k_spmv_plain32(DevProblem d, const float* __restrict__ x,
                                                            float* __restrict__ y) {
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s];
  y[tile * kTileRows + threadIdx.x] = sell_row(d.cols, d.vals32, off, w, lane, x + t0 * kTileRows);
}

__global__ void k_scatter_local32(DevProblem d, const double* __restrict__ canon, float* __restrict__ vec) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_local) return;
  vec[d.can2vec[k]] = (float)canon[k];
}

__global__ void k_gather_local32(DevProblem d, const float* __restrict__ vec, double* __restrict__ canon) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_local) return;
  canon[k] = (double)vec[d.can2vec[k]];
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
  double mus = 0.0, mut = 0.0;
  for (int32_t k = d.fm_ptr[e]; k < d.fm_ptr[e + 1]; ++k) {
    const double mv = d.fm_val[k];
    const int32_t c = d.fm_col[k];
    mus = fma(mv, d.x[d.fent_row_s[c]], mus);
    mut = fma(mv, d.x[d.fent_row_t[c]], mut);
  }
  const double pp = d.psub[d.face_s[f]] + d.psub[d.face_t[f]];
  double* lst = d.lam + 2 * eo + m;
  double* lts = d.lam + 2 * eo + nf + m;
  const double old_st = *lst, old_ts = *lts;
  *lst = pp * mut - old_ts;
  *lts = pp * mus - old_st;
}

// Stop test, step 1: ubar = average of the copies of each node; phi = ubar
// on the full grid; w = ubar scattered back to every copy.
__global__ void k_average(DevProblem d) {
  const int b = blockIdx.x;
  if (d.inst_done[d.rblock_inst[b]]) return;  // a finished instance keeps its phi
  for (int64_t n = d.rblock_node0[b] + threadIdx.x; n < d.rblock_node0[b + 1]; n += blockDim.x) {
    const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
    if (c0 == c1) {
      d.phi[n] = 0.0;
      continue;
    }
    double s = 0.0;
    for (int32_t c = c0; c < c1; ++c) s += d.x[d.cp_idx[c]];
    const double ub = s / (double)(c1 - c0);
    d.phi[n] = ub;
    for (int32_t c = c0; c < c1; ++c) d.w[d.cp_idx[c]] = ub;
  }
}

// y = A x on every tile (all subdomains).
__global__ void __launch_bounds__(kTileRows) k_spmv_plain(DevProblem d, const double* __restrict__ x,
                                                          double* __restrict__ y) {
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s];
  y[tile * kTileRows + threadIdx.x] = sell_row(d.cols, d.vals, off, w, lane, x + t0 * kTileRows);
}

// y -= p_i M_Gi x on interface rows: turns A_i x into K_i x.
__global__ void k_face_correct(DevProblem d, const double* __restrict__ x, double* __restrict__ y) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_irow) return;
  const double p = d.psub[d.irow_sub[k]];
  double acc = 0.0;
  for (int32_t e = d.im_ptr[k]; e < d.im_ptr[k + 1]; ++e) acc = fma(d.im_val[e], x[d.im_col[e]], acc);
  const int32_t row = d.irow[k];
  y[row] -= p * acc;
}

// Stop test, step 2: r = sum_copies f - sum_copies K_i ubar per node and
// ||r|| / ||f|| per instance by a deterministic two-level sum.  The last
// block of an instance records its residual and whether it is done (reached
// rtol or max_outer); the last block overall counts the Schwarz iteration
// and sets the outer loop condition (any instance still running).
__global__ void __launch_bounds__(256) k_residual(DevProblem d, unsigned long long cond, int use_cond) {
  __shared__ double sm[2][kTileSlices];
  __shared__ bool flag;
  const int b = blockIdx.x;
  const int inst = d.rblock_inst[b];
  const bool live = !d.inst_done[inst];
  double v[2] = {0.0, 0.0};
  if (live) {
    for (int64_t n = d.rblock_node0[b] + threadIdx.x; n < d.rblock_node0[b + 1]; n += blockDim.x) {
      const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
      double fg = 0.0, ku = 0.0;
      for (int32_t c = c0; c < c1; ++c) {
        fg += d.f[d.cp_idx[c]];
        ku += d.y[d.cp_idx[c]];
      }
      const double r = fg - ku;
      v[0] += r * r;
      v[1] += fg * fg;
    }
  }
  block_sum<2>(v, sm);
  if (threadIdx.x == 0) {
    d.rpart[b] = v[0];
    d.rpart2[b] = v[1];
  }
  const int b0 = d.inst_rblock0[inst], nb = d.inst_rblock0[inst + 1] - b0;
  if (last_block(&d.inst_cnt[inst], (unsigned)nb, &flag) && live) {
    double u[2] = {0.0, 0.0};
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
      u[0] += __ldcg(d.rpart + b0 + k);
      u[1] += __ldcg(d.rpart2 + b0 + k);
    }
    block_sum<2>(u, sm);
    if (threadIdx.x == 0) {
      const double rel = u[1] > 0.0 ? sqrt(u[0] / u[1]) : sqrt(u[0]);
      const int n_outer = d.ctl->n_outer;
      d.inst_relres[inst] = rel;
      d.inst_iters[inst] = n_outer + 1;
      if (d.n_inst == 1) {
        if (n_outer < d.ctl->max_outer) d.hist[n_outer] = rel;
        d.ctl->relres = rel;
      }
      if (!(rel > d.ctl->rtol) || !isfinite(rel) || n_outer + 1 >= d.ctl->max_outer) d.inst_done[inst] = 1;
    }
  }
  if (last_block(&d.ctl->gcnt_r, gridDim.x, &flag) && threadIdx.x == 0) {
    d.ctl->n_outer += 1;
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
  k_cg_init<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d);
  k_fin_init<<<fin_blocks(d), kTileRows, 0, s>>>(d, defect_norm, cond, use_cond);
  return cudaGetLastError();
}

cudaError_t launch_cg_iteration(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond) {
  const CgVec<double> v{d.x, d.r, d.z, d.p, d.q, d.dinv, d.vals};
  k_cg_spmv<double><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
  k_fin_alpha<<<fin_blocks(d), kTileRows, 0, s>>>(d);
  k_cg_update<double><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
  k_fin_beta<<<fin_blocks(d), kTileRows, 0, s>>>(d, cond, use_cond);
  k_cg_direction<double><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
  return cudaGetLastError();
}

cudaError_t launch_cg_iteration32(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond) {
  const CgVec<float> v{d.x32, d.r32, d.z32, d.p32, d.q32, d.dinv32, d.vals32};
  k_cg_spmv<float><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
  k_fin_alpha<<<fin_blocks(d), kTileRows, 0, s>>>(d);
  k_cg_update<float><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
  k_fin_beta<<<fin_blocks(d), kTileRows, 0, s>>>(d, cond, use_cond);
  k_cg_direction<float><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, v);
  return cudaGetLastError();
}

cudaError_t launch_cg_init_mixed(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond) {
  k_cg_init_mixed<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d);
  k_fin_init<<<fin_blocks(d), kTileRows, 0, s>>>(d, 1, cond, use_cond);
  return cudaGetLastError();
}

cudaError_t launch_mixed_correct(const DevProblem& d, cudaStream_t s) {
  k_mixed_correct<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_spmv_plain32(const DevProblem& d, const float* x, float* y, cudaStream_t s) {
  k_spmv_plain32<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, x, y);
  return cudaGetLastError();
}

cudaError_t launch_apply32(const DevProblem& d, const double* x, double* y, cudaStream_t s) {
  k_scatter_local32<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, x, d.z32);
  k_spmv_plain32<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, d.z32, d.q32);
  k_gather_local32<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, d.q32, y);
  return cudaGetLastError();
}

cudaError_t launch_exchange(const DevProblem& d, cudaStream_t s) {
  if (d.n_fent == 0) return cudaSuccess;
  k_exchange<<<blocks_for(d.n_fent, 256), 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_spmv_plain(const DevProblem& d, const double* x, double* y, cudaStream_t s) {
  k_spmv_plain<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, x, y);
  return cudaGetLastError();
}

cudaError_t launch_residual(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond) {
  k_average<<<(unsigned)d.n_rblocks, 256, 0, s>>>(d);
  k_spmv_plain<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, d.w, d.y);
  if (d.n_irow) k_face_correct<<<blocks_for(d.n_irow, 256), 256, 0, s>>>(d, d.w, d.y);
  k_residual<<<(unsigned)d.n_rblocks, 256, 0, s>>>(d, cond, use_cond);
  return cudaGetLastError();
}

cudaError_t launch_apply(const DevProblem& d, int op, const double* x, double* y, cudaStream_t s) {
  k_scatter_local<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, x, d.w);
  k_spmv_plain<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, d.w, d.y);
  if (op == 1 && d.n_irow) k_face_correct<<<blocks_for(d.n_irow, 256), 256, 0, s>>>(d, d.w, d.y);
  k_gather_local<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, d.y, y);
  return cudaGetLastError();
}

cudaError_t launch_apply_scratch(const DevProblem& d, int op, const double* x, double* y, double* w_scratch,
                                 double* y_scratch, cudaStream_t s) {
  k_scatter_local<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, x, w_scratch);
  k_spmv_plain<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, w_scratch, y_scratch);
  if (op == 1 && d.n_irow) k_face_correct<<<blocks_for(d.n_irow, 256), 256, 0, s>>>(d, w_scratch, y_scratch);
  k_gather_local<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, y_scratch, y);
  return cudaGetLastError();
}

cudaError_t launch_gather_local(const DevProblem& d, const double* vec, double* canon, cudaStream_t s) {
  k_gather_local<<<blocks_for(d.n_local, 256), 256, 0, s>>>(d, vec, canon);
  return cudaGetLastError();
}

}  // namespace osm
