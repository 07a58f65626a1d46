// Adjoint gradient of a surface-gravity misfit (not in the paper; the
// forward model is the gravimetry problem of Sec. 2 solved by the Schwarz
// method of Sec. 3).
//
// With the load f = 4 pi G F drho (F: per-element constant density to nodal
// load, entries int_e phi_a) and K phi = f, the misfit
//     J = 1/2 sum_s (g_s - g_obs,s)^2,   g = B phi,
// (B: d/dz of the Q2 interpolant at each station) has the gradient
//     dJ/d drho = 4 pi G F^T w,   K w = B^T (B phi - g_obs),
// where w comes from one more Schwarz solve with the same subdomain
// machinery (K is symmetric).  For a general output L(phi) the same adjoint
// solve with K w = dL/dphi gives dL/d drho = 4 pi G F^T w.
//
// Everything here is node- or element-centric, so every sum has a fixed
// order and no atomics are needed.
#include <cuda_runtime.h>

#include "osm_device.cuh"
#include "osm_internal.h"

namespace osm {
namespace {

// 1-D weight int phi_a over element e (length h) of the node at 1-D index i
// in that element: h/6 at either end, 4h/6 at the mid node.
__device__ __forceinline__ double w1d(int i, int e, double h) {
  const int a = i - 2 * e;
  return a == 1 ? h * (4.0 / 6.0) : h * (1.0 / 6.0);
}

// f_i = 4 pi G sum over the (at most 8) elements of subdomain i around the
// row's node of drho_e * wx * wy * wz.  Writes the load and b = f.
__global__ void k_load_from_density(DevProblem d, DevAdjoint a, const double* __restrict__ drho) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= d.n_tiles * (int64_t)kTileRows) return;
  const int32_t node = a.row_node[row];
  double f = 0.0;
  if (node >= 0) {
    const int s = d.tile_sub[row / kTileRows];
    const int32_t* box = a.sub_box + 6 * s;
    const int i = node % a.NX, j = (node / a.NX) % a.NY, k = node / (a.NX * a.NY);
    int ex_lo = (i % 2 == 0) ? i / 2 - 1 : (i - 1) / 2, ex_hi = (i % 2 == 0) ? i / 2 : (i - 1) / 2;
    int ey_lo = (j % 2 == 0) ? j / 2 - 1 : (j - 1) / 2, ey_hi = (j % 2 == 0) ? j / 2 : (j - 1) / 2;
    int ez_lo = (k % 2 == 0) ? k / 2 - 1 : (k - 1) / 2, ez_hi = (k % 2 == 0) ? k / 2 : (k - 1) / 2;
    ex_lo = max(ex_lo, box[0]); ex_hi = min(ex_hi, box[1] - 1);
    ey_lo = max(ey_lo, box[2]); ey_hi = min(ey_hi, box[3] - 1);
    ez_lo = max(ez_lo, box[4]); ez_hi = min(ez_hi, box[5] - 1);
    for (int ez = ez_lo; ez <= ez_hi; ++ez) {
      const double wz = w1d(k, ez, a.zc[ez + 1] - a.zc[ez]);
      for (int ey = ey_lo; ey <= ey_hi; ++ey) {
        const double wy = w1d(j, ey, a.yc[ey + 1] - a.yc[ey]);
        for (int ex = ex_lo; ex <= ex_hi; ++ex) {
          const double wx = w1d(i, ex, a.xc[ex + 1] - a.xc[ex]);
          const double rho = drho[ex + (int64_t)a.nx * (ey + (int64_t)a.ny * ez)];
          f += rho * (wx * wy * wz);
        }
      }
    }
    f *= 4.0 * kPi * kGravity;
  }
  d.f[row] = f;
  d.b[row] = f;
}

// g_s = sum_a B_sa phi_a; res_s = g_s - g_obs,s (g_obs may be null).
__global__ void k_station_values(DevAdjoint a, const double* __restrict__ phi, const double* __restrict__ g_obs) {
  const int64_t st = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (st >= a.n_st) return;
  double g = 0.0;
  for (int q = 0; q < 27; ++q) g = fma(a.st_w[st * 27 + q], phi[a.st_node[st * 27 + q]], g);
  a.g[st] = g;
  a.res[st] = g_obs ? g - g_obs[st] : 0.0;
}

// J = 1/2 sum_s res_s^2 in one block (fixed order).
__global__ void k_misfit(DevAdjoint a, double* J) {
  __shared__ double sm[1][kTileSlices];
  double v[1] = {0.0};
  for (int64_t st = threadIdx.x; st < a.n_st; st += blockDim.x) v[0] += a.res[st] * a.res[st];
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) *J = 0.5 * v[0];
}

// Nodal adjoint load v = B^T res (v zeroed before): one thread adds every
// station's 27 contributions in station order, which fixes the summation
// order; stations are few (thousands), so this is a small serial pass.
__global__ void k_stations_transpose(DevAdjoint a) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int64_t st = 0; st < a.n_st; ++st)
    for (int q = 0; q < 27; ++q) a.v_nodes[a.st_node[st * 27 + q]] += a.st_w[st * 27 + q] * a.res[st];
}

// Subdomain loads from a nodal vector: every copy of node n receives v_n / c_n
// (c_n copies), so that sum_i R_i^T f_i = v on the unknowns.
__global__ void k_nodal_load(DevProblem d, const double* __restrict__ v) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < d.n_nodes; n += stride) {
    const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
    if (c0 == c1) continue;
    const double share = v[n] / (double)(c1 - c0);
    for (int32_t c = c0; c < c1; ++c) {
      d.f[d.cp_idx[c]] = share;
      d.b[d.cp_idx[c]] = share;
    }
  }
}

// dL/d drho_e = 4 pi G sum over the 27 nodes of e of w_a wx wy wz.
__global__ void k_density_gradient(DevAdjoint a, const double* __restrict__ w, double* __restrict__ grad) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ne = (int64_t)a.nx * a.ny * a.nz;
  if (e >= ne) return;
  const int ex = (int)(e % a.nx), ey = (int)((e / a.nx) % a.ny), ez = (int)(e / ((int64_t)a.nx * a.ny));
  const double hx = a.xc[ex + 1] - a.xc[ex], hy = a.yc[ey + 1] - a.yc[ey], hz = a.zc[ez + 1] - a.zc[ez];
  const double w1[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
  double acc = 0.0;
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int q = 0; q < 3; ++q) {
        const int64_t node = (2 * ex + q) + (int64_t)a.NX * ((2 * ey + b) + (int64_t)a.NY * (2 * ez + c));
        acc = fma(w[node], (w1[q] * hx) * (w1[b] * hy) * (w1[c] * hz), acc);
      }
  grad[e] = 4.0 * kPi * kGravity * acc;
}

// ---- reverse-mode Schwarz (derivative of the N-iteration misfit w.r.t. p)
//
// The forward iteration (symmetric p, exact local solves) is
//   u^n = A(p)^-1 (f + G lam^{n-1}),  lam^n = 2 p E u^n - P lam^{n-1},
//   J_N = 1/2 ||B S u^N - g_obs||^2,
// with G the Robin-data gather into the right-hand sides, E the face mass
// from the sending side, P the swap of the two sides of a face and S the
// average of the copies.  Its adjoint runs n = N .. 1 with
//   ubar^N = S^T B^T r,  ubar^n = 2 p E^T lambar^n (n < N),
//   bbar^n = A^-1 ubar^n,  lambar^{n-1} = G^T bbar^n - P^T lambar^n,
//   dJ_N/dp = sum_n [ lambar^n . 2 E u^n  -  bbar^n . M_G u^n ].

// out[c] = v_n / c_n on every copy c of node n (the transpose of the average).
__global__ void k_nodal_split(DevProblem d, const double* __restrict__ v, double* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < d.n_nodes; n += stride) {
    const int32_t c0 = d.cp_ptr[n], c1 = d.cp_ptr[n + 1];
    for (int32_t c = c0; c < c1; ++c) out[d.cp_idx[c]] = v[n] / (double)(c1 - c0);
  }
}

// mu = M_face lam on both sides of every face (face layout).
__global__ void k_face_mass_lam(DevProblem d, const double* __restrict__ lam, double* __restrict__ mu) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= d.n_fent) return;
  const int f = d.fent_face[e];
  const int64_t eo = d.face_eo[f];
  const int32_t nf = d.face_n[f];
  double ast = 0.0, ats = 0.0;
  for (int32_t k = d.fm_ptr[e]; k < d.fm_ptr[e + 1]; ++k) {
    const int64_t c = d.fm_col[k] - eo;
    ast = fma(d.fm_val[k], lam[2 * eo + c], ast);
    ats = fma(d.fm_val[k], lam[2 * eo + nf + c], ats);
  }
  mu[2 * eo + (e - eo)] = ast;
  mu[2 * eo + nf + (e - eo)] = ats;
}

// ubar = p2 E^T lambar on the interface rows (zero elsewhere, set before):
// a row sends to the face slot opposite to the one it receives.
__global__ void k_exchange_transpose(DevProblem d, const int32_t* __restrict__ partner, const double* __restrict__ mu,
                                     double p2, double* __restrict__ ub) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= d.n_irow) return;
  double acc = 0.0;
  for (int32_t e = d.ilam_ptr[k]; e < d.ilam_ptr[k + 1]; ++e) acc += mu[partner[e]];
  ub[d.irow[k]] = p2 * acc;
}

// Block partials of lambar . 2 E u (face entries) and of -bbar . M_G u
// (interface rows); a single-block kernel adds them in order.
__global__ void k_dp_terms(DevProblem d, const double* __restrict__ lam, const double* __restrict__ u,
                           const double* __restrict__ bbar, double* __restrict__ part) {
  __shared__ double sm[1][kTileSlices];
  double v[1] = {0.0};
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < d.n_fent) {
    const int f = d.fent_face[i];
    const int64_t eo = d.face_eo[f];
    const int32_t nf = d.face_n[f];
    double mus = 0.0, mut = 0.0;
    for (int32_t k = d.fm_ptr[i]; k < d.fm_ptr[i + 1]; ++k) {
      const int32_t c = d.fm_col[k];
      mus = fma(d.fm_val[k], u[d.fent_row_s[c]], mus);
      mut = fma(d.fm_val[k], u[d.fent_row_t[c]], mut);
    }
    v[0] = 2.0 * (lam[2 * eo + (i - eo)] * mut + lam[2 * eo + nf + (i - eo)] * mus);
  }
  const int64_t j = i - d.n_fent;
  if (j >= 0 && j < d.n_irow) {
    double mu = 0.0;
    for (int32_t e = d.im_ptr[j]; e < d.im_ptr[j + 1]; ++e) mu = fma(d.im_val[e], u[d.im_col[e]], mu);
    v[0] = -bbar[d.irow[j]] * mu;
  }
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__global__ void k_sum_parts(const double* __restrict__ part, int64_t n, double* __restrict__ out) {
  __shared__ double sm[1][kTileSlices];
  double v[1] = {0.0};
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) v[0] += part[k];
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) *out = v[0];
}

// lambar^{n-1} = G^T bbar - P^T lambar^n on every face entry.
__global__ void k_lambar_step(DevProblem d, const double* __restrict__ bbar, const double* __restrict__ lam_old,
                              double* __restrict__ lam_new) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= d.n_fent) return;
  const int f = d.fent_face[e];
  const int64_t eo = d.face_eo[f];
  const int32_t nf = d.face_n[f];
  const int64_t m = e - eo;
  lam_new[2 * eo + m] = bbar[d.fent_row_s[e]] - lam_old[2 * eo + nf + m];
  lam_new[2 * eo + nf + m] = bbar[d.fent_row_t[e]] - lam_old[2 * eo + m];
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_load_from_density(const DevProblem& d, const DevAdjoint& a, const double* drho, cudaStream_t s) {
  k_load_from_density<<<blocks_for(d.n_tiles * (int64_t)kTileRows, 256), 256, 0, s>>>(d, a, drho);
  return cudaGetLastError();
}

cudaError_t launch_station_values(const DevProblem& d, const DevAdjoint& a, const double* phi, const double* g_obs,
                                  cudaStream_t s) {
  (void)d;
  if (a.n_st == 0) return cudaSuccess;
  k_station_values<<<blocks_for(a.n_st, 256), 256, 0, s>>>(a, phi, g_obs);
  return cudaGetLastError();
}

cudaError_t launch_misfit(const DevAdjoint& a, double* J_dev, cudaStream_t s) {
  k_misfit<<<1, 256, 0, s>>>(a, J_dev);
  return cudaGetLastError();
}

cudaError_t launch_stations_transpose(const DevProblem& d, const DevAdjoint& a, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.v_nodes, 0, sizeof(double) * d.n_nodes, s);
  if (e != cudaSuccess) return e;
  k_stations_transpose<<<1, 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_nodal_load(const DevProblem& d, const DevAdjoint& a, const double* v_nodes, cudaStream_t s) {
  (void)a;
  k_nodal_load<<<kNodeBlocks, 256, 0, s>>>(d, v_nodes);
  return cudaGetLastError();
}

cudaError_t launch_density_gradient(const DevProblem& d, const DevAdjoint& a, const double* w_nodes, double* grad,
                                    cudaStream_t s) {
  (void)d;
  const int64_t ne = (int64_t)a.nx * a.ny * a.nz;
  k_density_gradient<<<blocks_for(ne, 256), 256, 0, s>>>(a, w_nodes, grad);
  return cudaGetLastError();
}

cudaError_t launch_nodal_split(const DevProblem& d, const double* v, double* out, cudaStream_t s) {
  k_nodal_split<<<kNodeBlocks, 256, 0, s>>>(d, v, out);
  return cudaGetLastError();
}

cudaError_t launch_exchange_adjoint(const DevProblem& d, const int32_t* partner, const double* lam, double* mu,
                                    double p2, double* ub, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ub, 0, sizeof(double) * d.n_tiles * kTileRows, s);
  if (e != cudaSuccess || d.n_fent == 0) return e;
  k_face_mass_lam<<<blocks_for(d.n_fent, 256), 256, 0, s>>>(d, lam, mu);
  if (d.n_irow) k_exchange_transpose<<<blocks_for(d.n_irow, 256), 256, 0, s>>>(d, partner, mu, p2, ub);
  return cudaGetLastError();
}

cudaError_t launch_dp_terms(const DevProblem& d, const double* lam, const double* u, const double* bbar, double* part,
                            double* out, cudaStream_t s) {
  const int64_t n = d.n_fent + d.n_irow;
  const unsigned nb = blocks_for(n > 0 ? n : 1, 256);
  k_dp_terms<<<nb, 256, 0, s>>>(d, lam, u, bbar, part);
  k_sum_parts<<<1, 256, 0, s>>>(part, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_lambar_step(const DevProblem& d, const double* bbar, const double* lam_old, double* lam_new,
                               cudaStream_t s) {
  if (d.n_fent == 0) return cudaSuccess;
  k_lambar_step<<<blocks_for(d.n_fent, 256), 256, 0, s>>>(d, bbar, lam_old, lam_new);
  return cudaGetLastError();
}

}  // namespace osm
