// Batched evaluation of Robin parameters: the stochastic search of Sec. 4
// needs the Schwarz iteration (Sec. 3) run for a population of candidate p
// values.  Here up to 32 candidates run as one batched solve that shares the
// subdomain stiffness matrices K_i:
//
//   A_k = K_i + p_k M_Gi,   lam_ij,k <- 2 p_k M_Gij u_j,k - lam_ji,k,
//
// each candidate with its own iterate, Robin data, CG scalars per subdomain,
// convergence mask and stop test.
//
// Layout: every vector holds the 32 candidates of a row contiguously
// ([row][32]), so the 32 lanes of a warp are the 32 candidates.  A warp owns
// one SELL-32 slice and walks its 32 rows; each matrix entry is loaded once
// (the same address in all lanes, a broadcast) and applied to all candidates,
// and every gather of x reads one contiguous 256-byte row of candidates.  The
// stored SELL values are K_i (the caller sets p = 0 before the batched run);
// the Robin term p_k M_Gi is added per candidate on interface rows.
#include <cuda_runtime.h>

#include "osm_device.cuh"
#include "osm_internal.h"

namespace osm {
namespace {

constexpr int W = kSampleWidth;

// sum over the 8 warps of a block of a per-lane value; result in warp 0
template <int NV>
__device__ __forceinline__ void lane_block_sum(double (&v)[NV], double (*sm)[kTileSlices][W]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) sm[i][warp][lane] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kTileSlices; ++w) s += sm[i][w][lane];
      v[i] = s;
    }
  }
}

// sum over tiles t0 .. t0+nt of part[t][lane] in a fixed order
__device__ __forceinline__ double lane_sum_tiles(const double* part, int64_t t0, int64_t nt, int lane) {
  double s = 0.0;
  for (int64_t j = 0; j < nt; ++j) s += __ldcg(part + (t0 + j) * W + lane);
  return s;
}

// Rows of the batched SpMM: lane k returns (K x_k)[row] (+ p_k (M_G x_k)[row]
// on interface rows when ROBIN).  Xs: subdomain base of X, Xg: X itself.
// FP64 reads the FP64 values (pair layout), FP32 the FP32 values (quad
// layout); every matrix load is a broadcast shared by the 32 candidates.
// NR consecutive rows rl .. rl+NR-1 of the slice at `off` (all of width w)
// at once: NR independent load -> gather -> FMA chains per step keep NR
// times more requests in flight than a row-at-a-time walk, which left the
// batched SpMM latency-bound.
template <class T, int NR, bool ROBIN = true>
__device__ __forceinline__ void mp_rows(const DevProblem& d, const DevSample& m, int64_t off, int rl, int w,
                                        const T* __restrict__ Xs, const T* __restrict__ Xg, int64_t row0,
                                        double pk, int k, T (&out)[NR]) {
  T acc0[NR], acc1[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { acc0[r] = T(0); acc1[r] = T(0); }
  const int nq = w >> 2;
#pragma unroll 2
  for (int q = 0; q < nq; ++q) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int4 c = __ldg(reinterpret_cast<const int4*>(d.cols + off) + rl + r + q * 32);
      if constexpr (sizeof(T) == 8) {
        const double2* v2 = reinterpret_cast<const double2*>(d.vals + off) + rl + r;
        const double2 a = __ldg(v2 + q * 64);
        const double2 b = __ldg(v2 + q * 64 + 32);
        acc0[r] = fma(a.x, Xs[(int64_t)c.x * W + k], acc0[r]);
        acc1[r] = fma(a.y, Xs[(int64_t)c.y * W + k], acc1[r]);
        acc0[r] = fma(b.x, Xs[(int64_t)c.z * W + k], acc0[r]);
        acc1[r] = fma(b.y, Xs[(int64_t)c.w * W + k], acc1[r]);
      } else {
        const float4 a = __ldg(reinterpret_cast<const float4*>(d.vals32 + off) + rl + r + q * 32);
        acc0[r] = fmaf(a.x, Xs[(int64_t)c.x * W + k], acc0[r]);
        acc1[r] = fmaf(a.y, Xs[(int64_t)c.y * W + k], acc1[r]);
        acc0[r] = fmaf(a.z, Xs[(int64_t)c.z * W + k], acc0[r]);
        acc1[r] = fmaf(a.w, Xs[(int64_t)c.w * W + k], acc1[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    T acc = acc0[r] + acc1[r];
    const int32_t ir = ROBIN ? m.row_irow[row0 + r] : -1;
    if (ir >= 0) {
      T f = T(0);
      for (int32_t e = d.im_ptr[ir]; e < d.im_ptr[ir + 1]; ++e)
        f = fma((T)d.im_val[e], Xg[(int64_t)d.im_col[e] * W + k], f);
      acc = fma((T)pk, f, acc);
    }
    out[r] = acc;
  }
}

__device__ __forceinline__ double mp_dinv(const DevProblem& d, const DevSample& m, int64_t row, double pk) {
  const int32_t ir = m.row_irow[row];
  if (ir < 0) return d.dinv[row];
  return 1.0 / (d.kdiag[row] + pk * d.irow_mdiag[ir]);
}

// Dot-product term of the FP32 inner solve: products of the factors scaled
// by sc (a power of two per subdomain and candidate, set from the defect) are
// summed in FP32 over the slice's rows; the caller widens and unscales once.
template <class T>
struct MpDot {
  T acc = T(0);
  __device__ __forceinline__ void add(T a, T b, T sc) { acc = fma(a * sc, b * sc, acc); }
};

// b_k = f on every row, for every candidate (start of a batched run).
__global__ void k_mp_bcast_f(DevProblem d, DevSample m, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  m.b[i] = d.f[i / W];
}

// Robin right-hand sides on interface rows: b_k = f + sum_j lam_ij,k.
__global__ void k_mp_rhs_gather(DevProblem d, DevSample m) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int k = threadIdx.x & 31;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.ctl->n_active = 0;
    d.ctl->n_inner = 0;
    if (d.ctl->t_start_ns == 0ull) d.ctl->t_start_ns = global_ns();
  }
  if (gw >= d.n_irow) return;
  const int32_t row = d.irow[gw];
  double b = d.f[row];
  for (int32_t e = d.ilam_ptr[gw]; e < d.ilam_ptr[gw + 1]; ++e) b += m.lam[(int64_t)d.ilam[e] * W + k];
  m.b[(int64_t)row * W + k] = b;
}

// CG start for every candidate: r = b - A_k x, z = D_k^-1 r, p = z.
__global__ void __launch_bounds__(kTileRows) k_mp_cg_init(DevProblem d, DevSample m) {
  __shared__ double sm[3][kTileSlices][W];
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s];
  const double* Xs = m.x + t0 * kTileRows * W;
  const double pk = m.psamp[k];
  double v[3] = {0.0, 0.0, 0.0};
  for (int rl = 0; rl < kSliceRows; rl += 4) {
    double ax4[4];
    mp_rows<double, 4>(d, m, off, rl, w, Xs, m.x, slice * kSliceRows + rl, pk, k, ax4);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t row = slice * kSliceRows + rl + j;
      const int64_t idx = row * W + k;
      const double b = m.b[idx];
      const double r = b - ax4[j];
      const double z = mp_dinv(d, m, row, pk) * r;
      m.r[idx] = r;
      m.z[idx] = z;
      m.pd[idx] = z;
      v[0] += r * r;
      v[1] += b * b;
      v[2] += r * z;
    }
  }
  lane_block_sum<3>(v, sm);
  if (warp == 0) {
    m.part0[tile * W + k] = v[0];
    m.part1[tile * W + k] = v[1];
    m.part2[tile * W + k] = v[2];
  }
}

// q_k = A_k p_k and the tile partials of p.q per (subdomain, candidate)
// still iterating (T = double: FP64 batch; float: the inner solve of the
// mixed batch).
template <class T>
__global__ void __launch_bounds__(kTileRows) k_mp_cg_spmv(DevProblem d, DevSample m, MpVec<T> v) {
  __shared__ double sm[1][kTileSlices][W];
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int64_t sk = (int64_t)s * W + k;
  const int act = m.active[sk];
  if (!__any_sync(0xffffffffu, act)) return;  // same answer in every warp of the block
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s];
  const T* Xs = v.pd + t0 * kTileRows * W;
  const double pk = m.psamp[k];
  const T sc = sizeof(T) == 4 ? (T)m.sc[sk] : T(1);
  MpDot<T> pq;
  // only the candidates still iterating on this subdomain gather and compute:
  // a finished candidate's lane requests no sectors of the candidate rows
  // (the host sorts candidates by p, so the lanes still running tend to be
  // neighbours and share sectors)
  if (act) {
    constexpr int NR = 4;
    for (int rl = 0; rl < kSliceRows; rl += NR) {
      const int64_t row0 = slice * kSliceRows + rl;
      T q[NR];
      mp_rows<T, NR>(d, m, off, rl, w, Xs, v.pd, row0, pk, k, q);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int64_t idx = (row0 + r) * W + k;
        v.q[idx] = q[r];
        pq.add(v.pd[idx], q[r], sc);
      }
    }
  }
  double acc[1] = {(double)pq.acc * (sizeof(T) == 4 ? m.isc2[sk] : 1.0)};
  lane_block_sum<1>(acc, sm);
  if (warp == 0) m.part0[tile * W + k] = acc[0];
}

// x += alpha p, r -= alpha q, z = D_k^-1 r and the tile partials of r.z and
// ||r||^2 per (subdomain, candidate).
template <class T>
__global__ void __launch_bounds__(kTileRows) k_mp_cg_update(DevProblem d, DevSample m, MpVec<T> v) {
  __shared__ double sm[2][kTileSlices][W];
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int64_t sk = (int64_t)s * W + k;
  const int act = m.active[sk];
  if (__any_sync(0xffffffffu, act)) {
    const T alpha = (T)m.alpha[sk];
    const double pk = m.psamp[k];
    const T sc = sizeof(T) == 4 ? (T)m.sc[sk] : T(1);
    MpDot<T> rz, rr;
    const int64_t slice = tile * kTileSlices + warp;
#pragma unroll 4
    for (int rl = 0; rl < kSliceRows; ++rl) {
      const int64_t row = slice * kSliceRows + rl;
      const int64_t idx = row * W + k;
      if (act) {
        v.x[idx] = fma(alpha, v.pd[idx], v.x[idx]);
        const T r = fma(-alpha, v.q[idx], v.r[idx]);
        const T z = (T)mp_dinv(d, m, row, pk) * r;
        v.r[idx] = r;
        v.z[idx] = z;
        rz.add(r, z, sc);
        rr.add(r, r, sc);
      }
    }
    const double un = sizeof(T) == 4 ? m.isc2[sk] : 1.0;
    double acc[2] = {(double)rz.acc * un, (double)rr.acc * un};
    lane_block_sum<2>(acc, sm);
    if (warp == 0) {
      m.part1[tile * W + k] = acc[0];
      m.part2[tile * W + k] = acc[1];
    }
  }
}

// Mixed batch, start of a refinement step: FP64 defect d_k = b_k - A_k x_k,
// then the FP32 CG on A_k e = d_k from e = 0 (r = d, z = D_k^-1 r, p = z)
// and the tile partials of ||d||^2, ||b||^2 and r.z.
__global__ void __launch_bounds__(kTileRows) k_mp_cg_init_mixed(DevProblem d, DevSample m) {
  __shared__ double sm[3][kTileSlices][W];
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s];
  const double* Xs = m.x + t0 * kTileRows * W;
  const double pk = m.psamp[k];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int rl = 0; rl < kSliceRows; rl += 4) {
    double ax4[4];
    mp_rows<double, 4>(d, m, off, rl, w, Xs, m.x, slice * kSliceRows + rl, pk, k, ax4);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t row = slice * kSliceRows + rl + j;
      const int64_t idx = row * W + k;
      const double b = m.b[idx];
      const double dfc = b - ax4[j];
      const float r = (float)dfc;
      const float z = (float)mp_dinv(d, m, row, pk) * r;
      m.x32[idx] = 0.f;
      m.r32[idx] = r;
      m.z32[idx] = z;
      m.pd32[idx] = z;
      acc[0] += dfc * dfc;
      acc[1] += b * b;
      acc[2] += (double)r * (double)z;
    }
  }
  lane_block_sum<3>(acc, sm);
  if (warp == 0) {
    m.part0[tile * W + k] = acc[0];
    m.part1[tile * W + k] = acc[1];
    m.part2[tile * W + k] = acc[2];
  }
}

// Mixed batch, end of the refinement step: x_k += e_k in FP64.
__global__ void k_mp_mixed_correct(DevSample m, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) m.x[i] += (double)m.x32[i];
}

// Per-subdomain finalisers, one warp per subdomain and one lane per
// candidate: the tile partials are added in a fixed order.

// mixed (the refinement forms): the partials are ||d||^2, ||b||^2, r.z with
// d the defect; the inner solve's reference norm is ||d|| and a candidate
// whose defect meets inner_rtol on this subdomain is not corrected.
__global__ void k_mp_fin_init(DevProblem d, DevSample m, int mixed, unsigned long long cond, int use_cond) {
  __shared__ bool flag;
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int s = blockIdx.x * kTileSlices + warp;
  if (s < d.n_sub) {
    const int64_t t0 = d.sub_tile0[s], nt = d.sub_tile0[s + 1] - t0;
    const double rr = lane_sum_tiles(m.part0, t0, nt, k);
    const double bb = lane_sum_tiles(m.part1, t0, nt, k);
    const double rz = lane_sum_tiles(m.part2, t0, nt, k);
    const int64_t sk = (int64_t)s * W + k;
    m.rr[sk] = rr;
    m.bb[sk] = mixed ? rr : bb;
    m.rho[sk] = rz;
    m.beta[sk] = 0.0;
    m.iters[sk] = 0;
    // scale of the FP32 dot products: sc = 2^-e with 2^e ~ rms of the defect
    int e = 0;
    const double ms = rr / (double)(nt * kTileRows);
    if (mixed && ms > 0.0 && isfinite(ms)) {
      frexp(sqrt(ms), &e);
      e = max(-120, min(120, e));
    }
    m.sc[sk] = (float)ldexp(1.0, -e);
    m.isc2[sk] = ldexp(1.0, 2 * e);
    const int act = !m.done[k] && (mixed ? (!(rr <= d.ctl->tau2_outer * bb) && rz > 0.0) : !(rr <= d.ctl->tau2 * bb));
    m.active[sk] = act;
    const unsigned bal = __ballot_sync(0xffffffffu, act);
    if (k == 0 && bal) atomicAdd(&d.ctl->n_active, __popc(bal));
  }
  if (last_block(&d.ctl->gcnt_i, gridDim.x, &flag) && threadIdx.x == 0) {
    const bool more = d.ctl->n_active > 0 && !out_of_time(d.ctl);
    if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
  }
}

__global__ void k_mp_fin_alpha(DevProblem d, DevSample m) {
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int s = blockIdx.x * kTileSlices + warp;
  if (s >= d.n_sub) return;
  const int64_t sk = (int64_t)s * W + k;
  if (!m.active[sk]) return;
  const int64_t t0 = d.sub_tile0[s], nt = d.sub_tile0[s + 1] - t0;
  const double pq = lane_sum_tiles(m.part0, t0, nt, k);
  if (!(pq > 0.0) || !isfinite(pq)) {
    m.alpha[sk] = 0.0;
    m.active[sk] = 0;
    atomicOr(&d.ctl->status, 2);
    atomicSub(&d.ctl->n_active, 1);
  } else {
    m.alpha[sk] = m.rho[sk] / pq;
  }
}

__global__ void k_mp_fin_beta(DevProblem d, DevSample m, unsigned long long cond, int use_cond) {
  __shared__ bool flag;
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int s = blockIdx.x * kTileSlices + warp;
  if (s < d.n_sub) {
    const int64_t sk = (int64_t)s * W + k;
    if (m.active[sk]) {
      const int64_t t0 = d.sub_tile0[s], nt = d.sub_tile0[s + 1] - t0;
      const double rz = lane_sum_tiles(m.part1, t0, nt, k);
      const double rr = lane_sum_tiles(m.part2, t0, nt, k);
      const int it = m.iters[sk] + 1;
      m.iters[sk] = it;
      m.rr[sk] = rr;
      if (rr <= d.ctl->tau2 * m.bb[sk]) {
        m.active[sk] = 0;
        atomicSub(&d.ctl->n_active, 1);
      } else if (it >= d.ctl->max_inner) {
        m.active[sk] = 0;
        atomicOr(&d.ctl->status, 1);
        atomicSub(&d.ctl->n_active, 1);
      }
      m.beta[sk] = rz / m.rho[sk];
      m.rho[sk] = rz;
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

// p = z + beta p for the (subdomain, candidate) pairs still iterating.
template <class T>
__global__ void __launch_bounds__(kTileRows) k_mp_cg_direction(DevProblem d, DevSample m, MpVec<T> v) {
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int64_t sk = (int64_t)s * W + k;
  if (!m.active[sk]) return;
  const T beta = (T)m.beta[sk];
  const int64_t slice = tile * kTileSlices + warp;
#pragma unroll 4
  for (int rl = 0; rl < kSliceRows; ++rl) {
    const int64_t idx = (slice * kSliceRows + rl) * W + k;
    v.pd[idx] = fma(beta, v.pd[idx], v.z[idx]);
  }
}

// Robin exchange for every candidate still running (warp per face entry).
__global__ void k_mp_exchange(DevProblem d, DevSample m) {
  const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int k = threadIdx.x & 31;
  if (e >= d.n_fent || m.done[k]) return;
  const int f = d.fent_face[e];
  const int64_t eo = d.face_eo[f];
  const int32_t nf = d.face_n[f];
  const int64_t mm = e - eo;
  double mus = 0.0, mut = 0.0;
  for (int32_t j = d.fm_ptr[e]; j < d.fm_ptr[e + 1]; ++j) {
    const double mv = d.fm_val[j];
    const int32_t c = d.fm_col[j];
    mus = fma(mv, m.x[(int64_t)d.fent_row_s[c] * W + k], mus);
    mut = fma(mv, m.x[(int64_t)d.fent_row_t[c] * W + k], mut);
  }
  const double pp = 2.0 * m.psamp[k];
  double* lst = m.lam + (2 * eo + mm) * W + k;
  double* lts = m.lam + (2 * eo + nf + mm) * W + k;
  const double old_st = *lst, old_ts = *lts;
  *lst = pp * mut - old_ts;
  *lts = pp * mus - old_st;
}

// ubar_k = mean of the copies of every node, scattered back to the copies.
__global__ void k_mp_average(DevProblem d, DevSample m) {
  const int k = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t n = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; n < d.n_nodes; n += nw) {
    const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
    if (c0 == c1) continue;
    double s = 0.0;
    for (int32_t c = c0; c < c1; ++c) s += m.x[(int64_t)d.cp_idx[c] * W + k];
    const double ub = copy_mean(s, c1 - c0);
    for (int32_t c = c0; c < c1; ++c) m.w[(int64_t)d.cp_idx[c] * W + k] = ub;
  }
}

// y_k = K w_k (Neumann stiffness, no Robin term) on every tile.
__global__ void __launch_bounds__(kTileRows) k_mp_spmv_k(DevProblem d, DevSample m) {
  const int64_t tile = blockIdx.x;
  const int s = d.tile_sub[tile];
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int64_t slice = tile * kTileSlices + warp;
  const int64_t off = d.slice_off[slice];
  const int w = (int)((d.slice_off[slice + 1] - off) >> 5);
  const int64_t t0 = d.sub_tile0[s];
  const double* Xs = m.w + t0 * kTileRows * W;
  for (int rl = 0; rl < kSliceRows; rl += 4) {
    double y4[4];
    mp_rows<double, 4, false>(d, m, off, rl, w, Xs, m.w, slice * kSliceRows + rl, 0.0, k, y4);
#pragma unroll
    for (int j = 0; j < 4; ++j) m.y[(slice * kSliceRows + rl + j) * W + k] = y4[j];
  }
}

// Stop test per candidate: ||sum_copies f - sum_copies K_i ubar_k|| / ||f||;
// the last block records it, marks converged candidates and steers the loop.
__global__ void __launch_bounds__(256) k_mp_residual(DevProblem d, DevSample m, unsigned long long cond,
                                                     int use_cond) {
  __shared__ double sm[2][kTileSlices][W];
  __shared__ bool flag;
  const int warp = threadIdx.x >> 5, k = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  double v[2] = {0.0, 0.0};
  for (int64_t n = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; n < d.n_nodes; n += nw) {
    const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
    double fg = 0.0, ku = 0.0;
    for (int32_t c = c0; c < c1; ++c) {
      fg += d.f[d.cp_idx[c]];
      ku += m.y[(int64_t)d.cp_idx[c] * W + k];
    }
    const double r = fg - ku;
    v[0] += r * r;
    v[1] += fg * fg;
  }
  lane_block_sum<2>(v, sm);
  if (warp == 0) {
    m.rpart[blockIdx.x * W + k] = v[0];
    m.rpart2[blockIdx.x * W + k] = v[1];
  }
  if (last_block(&d.ctl->gcnt_r, gridDim.x, &flag) && warp == 0) {
    double rr = 0.0, ff = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      rr += __ldcg(m.rpart + (int64_t)b * W + k);
      ff += __ldcg(m.rpart2 + (int64_t)b * W + k);
    }
    const double rel = ff > 0.0 ? sqrt(rr / ff) : sqrt(rr);
    const int n_outer = d.ctl->n_outer + 1;
    const bool live = !m.done[k];
    if (live) {
      m.relres[k] = rel;
      m.outer_iters[k] = n_outer;
      if (rel <= d.ctl->rtol || !isfinite(rel) || n_outer >= d.ctl->max_outer) m.done[k] = 1;
    }
    // race: once a candidate reaches rtol, no candidate still running can
    // need fewer iterations, so all stop here (each keeps this residual)
    const unsigned won = __ballot_sync(0xffffffffu, live && rel <= d.ctl->rtol);
    if (d.ctl->race && won) m.done[k] = 1;
    const unsigned running = __ballot_sync(0xffffffffu, !m.done[k]);
    if (k == 0) {
      d.ctl->n_outer = n_outer;
      const bool more = running != 0u && !out_of_time(d.ctl);
      if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
      d.ctl->n_active = (int)__popc(running);  // host-loop mode reads it as "candidates running"
    }
  }
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }
inline unsigned fin_blocks(const DevProblem& d) { return (unsigned)((d.n_sub + kTileSlices - 1) / kTileSlices); }

}  // namespace

cudaError_t launch_mp_start(const DevProblem& d, const DevSample& m, cudaStream_t s) {
  const int64_t n = d.n_tiles * (int64_t)kTileRows * W;
  k_mp_bcast_f<<<blocks_for(n, 256), 256, 0, s>>>(d, m, n);
  return cudaGetLastError();
}

cudaError_t launch_mp_rhs_init(const DevProblem& d, const DevSample& m, cudaStream_t s, unsigned long long cond,
                               int use_cond, int fp32, int refine) {
  k_mp_rhs_gather<<<blocks_for((d.n_irow > 0 ? d.n_irow : 1) * (int64_t)32, 256), 256, 0, s>>>(d, m);
  if (fp32) k_mp_cg_init_mixed<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, m);
  else k_mp_cg_init<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, m);
  k_mp_fin_init<<<fin_blocks(d), kTileRows, 0, s>>>(d, m, refine, cond, use_cond);
  return cudaGetLastError();
}

template <class T>
static void mp_cg_iteration(const DevProblem& d, const DevSample& m, MpVec<T> v, cudaStream_t s,
                            unsigned long long cond, int use_cond) {
  k_mp_cg_spmv<T><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, m, v);
  k_mp_fin_alpha<<<fin_blocks(d), kTileRows, 0, s>>>(d, m);
  k_mp_cg_update<T><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, m, v);
  k_mp_fin_beta<<<fin_blocks(d), kTileRows, 0, s>>>(d, m, cond, use_cond);
  k_mp_cg_direction<T><<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, m, v);
}

cudaError_t launch_mp_cg_iteration(const DevProblem& d, const DevSample& m, cudaStream_t s,
                                   unsigned long long cond, int use_cond, int mixed) {
  if (mixed) mp_cg_iteration<float>(d, m, MpVec<float>{m.x32, m.r32, m.z32, m.pd32, m.q32}, s, cond, use_cond);
  else mp_cg_iteration<double>(d, m, MpVec<double>{m.x, m.r, m.z, m.pd, m.q}, s, cond, use_cond);
  return cudaGetLastError();
}

cudaError_t launch_mp_exchange_residual(const DevProblem& d, const DevSample& m, cudaStream_t s,
                                        unsigned long long cond, int use_cond, int mixed) {
  if (mixed) {
    const int64_t n = d.n_tiles * (int64_t)kTileRows * W;
    k_mp_mixed_correct<<<blocks_for(n, 256), 256, 0, s>>>(m, n);
  }
  if (d.n_fent) k_mp_exchange<<<blocks_for(d.n_fent * (int64_t)32, 256), 256, 0, s>>>(d, m);
  k_mp_average<<<kNodeBlocks, 256, 0, s>>>(d, m);
  k_mp_spmv_k<<<(unsigned)d.n_tiles, kTileRows, 0, s>>>(d, m);
  k_mp_residual<<<kNodeBlocks, 256, 0, s>>>(d, m, cond, use_cond);
  return cudaGetLastError();
}

}  // namespace osm
