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

// ------------------------------------------------------------------ kernels

// Robin matrix A_i = K_i + p_i M_Gi on interface rows, and its diagonal.
__global__ void k_set_robin(DevProblem d) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_irow) return;
  const int s = d.irow_sub[k];
  const double p = d.psub[s];
  for (int32_t e = d.im_ptr[k]; e < d.im_ptr[k + 1]; ++e) d.vals[d.im_pos[e]] = d.im_kval[e] + p * d.im_val[e];
  const int32_t row = d.irow[k];
  d.dinv[row] = 1.0 / (d.kdiag[row] + p * d.irow_mdiag[k]);
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

// CG start from the warm iterate x: r = b - A x, z = D^-1 r, p = z;
// per subdomain rho = r.z, ||b||^2, ||r||^2 and the active flag.
__global__ void __launch_bounds__(kTileRows) k_cg_init(DevProblem d, unsigned long long cond, int use_cond) {
  __shared__ double sm[3][kTileSlices];
  __shared__ bool flag;
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s], nt = d.sub_tile0[s + 1] - t0;
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
  if (last_block(&d.st.cnt_i[s], (unsigned)nt, &flag)) {
    if (warp == 0) {
      const double rr = warp_sum_parts(d.part0, t0, nt);
      const double bb = warp_sum_parts(d.part1, t0, nt);
      const double rz = warp_sum_parts(d.part2, t0, nt);
      if (lane == 0) {
        d.st.rr[s] = rr;
        d.st.bb[s] = bb;
        d.st.rho[s] = rz;
        d.st.beta[s] = 0.0;
        d.st.iters[s] = 0;
        d.st.status[s] = 0;
        const int act = !(rr <= d.ctl->tau2 * bb);
        d.st.active[s] = act;
        if (act) atomicAdd(&d.ctl->n_active, 1);
      }
    }
  }
  if (use_cond && last_block(&d.ctl->gcnt_i, gridDim.x, &flag)) {
    if (threadIdx.x == 0)
      cudaGraphSetConditional(cond, (atomicAdd(&d.ctl->n_active, 0) > 0 && !out_of_time(d.ctl)) ? 1u : 0u);
  }
}

// q = A p and alpha = rho / (p.q) per active subdomain.
__global__ void __launch_bounds__(kTileRows) k_cg_spmv(DevProblem d) {
  __shared__ double sm[1][kTileSlices];
  __shared__ bool flag;
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  if (!d.st.active[s]) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s], nt = d.sub_tile0[s + 1] - t0;
  const int64_t row = tile * kTileRows + threadIdx.x;
  const double q = sell_row(d.cols, d.vals, off, w, lane, d.p + t0 * kTileRows);
  d.q[row] = q;
  double v[1] = {d.p[row] * q};
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) d.part0[tile] = v[0];
  if (last_block(&d.st.cnt_a[s], (unsigned)nt, &flag) && warp == 0) {
    const double pq = warp_sum_parts(d.part0, t0, nt);
    if (lane == 0) {
      if (!(pq > 0.0) || !isfinite(pq)) {  // breakdown: stop this subdomain
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
}

// x += alpha p, r -= alpha q, z = D^-1 r; then rho, ||r||^2, the stop test
// ||r|| <= tau ||b|| and beta per subdomain.
__global__ void __launch_bounds__(kTileRows) k_cg_update(DevProblem d, unsigned long long cond, int use_cond) {
  __shared__ double sm[2][kTileSlices];
  __shared__ bool flag;
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int act = d.st.active[s];
  if (act) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t0 = d.sub_tile0[s], nt = d.sub_tile0[s + 1] - t0;
    const int64_t row = tile * kTileRows + threadIdx.x;
    const double alpha = d.st.alpha[s];
    const double pr = d.p[row];
    d.x[row] = fma(alpha, pr, d.x[row]);
    const double r = fma(-alpha, d.q[row], d.r[row]);
    const double z = d.dinv[row] * r;
    d.r[row] = r;
    d.z[row] = z;
    double v[2] = {r * z, r * r};
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) {
      d.part1[tile] = v[0];
      d.part2[tile] = v[1];
    }
    if (last_block(&d.st.cnt_b[s], (unsigned)nt, &flag) && warp == 0) {
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
  }
  if (last_block(&d.ctl->gcnt_b, gridDim.x, &flag)) {
    if (threadIdx.x == 0) {
      const int n_inner = d.ctl->n_inner + 1;
      d.ctl->n_inner = n_inner;
      d.ctl->total_inner += 1;
      const bool more = atomicAdd(&d.ctl->n_active, 0) > 0 && n_inner <= d.ctl->max_inner &&
                        !out_of_time(d.ctl);
      if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
    }
  }
}

// p = z + beta p for subdomains still iterating.
__global__ void __launch_bounds__(kTileRows) k_cg_direction(DevProblem d) {
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  if (!d.st.active[s]) return;
  const int64_t row = tile * kTileRows + threadIdx.x;
  d.p[row] = fma(d.st.beta[s], d.p[row], d.z[row]);
}

// Robin exchange on every face entry (parallel update, Sec. 3):
// lam_st <- (p_s + p_t) M u_t - lam_ts, lam_ts <- (p_s + p_t) M u_s - lam_st.
__global__ void k_exchange(DevProblem d) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= d.n_fent) return;
  const int f = d.fent_face[e];
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
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= d.n_nodes) return;
  const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
  if (c0 == c1) { d.phi[n] = 0.0; return; }
  double s = 0.0;
  for (int32_t c = c0; c < c1; ++c) s += d.x[d.cp_idx[c]];
  const double ub = s / (double)(c1 - c0);
  d.phi[n] = ub;
  for (int32_t c = c0; c < c1; ++c) d.w[d.cp_idx[c]] = ub;
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

// Stop test, step 2: r = sum_copies f - sum_copies K_i ubar per node,
// ||r|| / ||f|| by a deterministic two-level sum; the last block records the
// residual, counts the Schwarz iteration and sets the outer loop condition.
__global__ void __launch_bounds__(256) k_residual(DevProblem d, unsigned long long cond, int use_cond) {
  __shared__ double sm[2][kTileSlices];
  __shared__ bool flag;
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (n < d.n_nodes) {
    const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
    double fg = 0.0, ku = 0.0;
    for (int32_t c = c0; c < c1; ++c) {
      fg += d.f[d.cp_idx[c]];
      ku += d.y[d.cp_idx[c]];
    }
    const double r = fg - ku;
    v[0] = r * r;
    v[1] = fg * fg;
  }
  block_sum<2>(v, sm);
  if (threadIdx.x == 0) {
    d.rpart[blockIdx.x] = v[0];
    d.rpart2[blockIdx.x] = v[1];
  }
  if (last_block(&d.ctl->gcnt_r, gridDim.x, &flag)) {
    double u[2] = {0.0, 0.0};
    for (int64_t k = threadIdx.x; k < (int64_t)gridDim.x; k += blockDim.x) {
      u[0] += __ldcg(d.rpart + k);
      u[1] += __ldcg(d.rpart2 + k);
    }
    block_sum<2>(u, sm);
    if (threadIdx.x == 0) {
      const double rel = u[1] > 0.0 ? sqrt(u[0] / u[1]) : sqrt(u[0]);
      const int n_outer = d.ctl->n_outer;
      if (n_outer < d.ctl->max_outer) d.hist[n_outer] = rel;
      d.ctl->n_outer = n_outer + 1;
      d.ctl->relres = rel;
      if (use_cond) {
        const bool more = (rel > d.ctl->rtol) && (n_outer + 1 < d.ctl->max_outer) && isfinite(rel) &&
                          !out_of_time(d.ctl);
        cudaGraphSetConditional(cond, more ? 1u : 0u);
      }
    }
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

cudaError_t launch_cg_init(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond) {
  k_cg_init<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, cond, use_cond);
  return cudaGetLastError();
}

cudaError_t launch_cg_iteration(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond) {
  k_cg_spmv<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d);
  k_cg_update<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, cond, use_cond);
  k_cg_direction<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d);
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
  k_average<<<blocks_for(d.n_nodes, 256), 256, 0, s>>>(d);
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
