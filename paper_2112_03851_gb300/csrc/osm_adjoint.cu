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

}  // namespace osm
