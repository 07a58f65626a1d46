// Matrix-free FP32 subdomain operator of the mixed inner solve.
//
// On an axis-aligned tensor-product mesh the Q2 Neumann stiffness of a box of
// elements is exactly
//     K_i = Kx (x) My (x) Mz + Mx (x) Ky (x) Mz + Mx (x) My (x) Kz
// with Kx, Mx the assembled 1-D Q2 stiffness and mass along x (banded: node a
// couples with a-2 .. a+2), and the Robin term of a face, p M_G = p E (x) My
// (x) Mz for a face normal to x (E: the unit entry at the face's end node),
// folds into the 1-D stiffness: (Kx + p E) (x) My (x) Mz.  So
//     A_i = K~x (x) My (x) Mz + Mx (x) K~y (x) Mz + Mx (x) My (x) K~z
// for the zeroth-order transmission condition of Sec. 3 (q = 0; the second-
// order term q S_G does not factor this way and keeps the SELL matrix).
//
// The kernel applies A_i by sum factorisation without reading any matrix.
// A CTA owns 256 consecutive (x, y) columns of one subdomain box and marches
// along z.  Every input plane is staged in shared memory with two rows of
// halo in y; the y pass forms My z and Ky z, the x pass the plane's two
// partial products P = (K~x (x) My + Mx (x) K~y) z and Q = (Mx (x) My) z, and
// each thread keeps P and Q of the last five planes in registers, so that
// output plane k = sum_c Mz(k, c) P(k+c-2) + K~z(k, c) Q(k+c-2).  About 36
// FMAs and two staged loads per row replace the 62 values and column indices
// (8 bytes each) the SELL SpMV streams from HBM.
//
// Layout ("box layout"): subdomain s's box node (i, j, k) -- Dirichlet nodes
// of the outer boundary included, held at zero -- is row box_voff[s] + i +
// bnx (j + bny k).  Rows on the outer boundary are written as zero.
#include <cuda_runtime.h>

#include "osm_device.cuh"
#include "osm_internal.h"

namespace osm {

namespace {

constexpr int kTxPlane = kTileRows + 6 * kTensorMaxNx;   // staged input plane: CTA rows + 4 halo rows
constexpr int kTxRows = kTileRows + 2 * kTensorMaxNx;    // y-pass outputs: the CTA's rows, all x
constexpr int kTxPre = (kTxPlane + kTileRows - 1) / kTileRows;
constexpr int kTxY = (kTxRows + kTileRows - 1) / kTileRows;
constexpr int kTxMaxRows = kTileRows / 3 + 2;   // rows 256 columns can touch (boxes are >= 3 nodes wide)
constexpr int kTxStages = 4;                     // input planes in flight
constexpr int kTxRowsP = 640;                    // >= (256 / nx + 2) (nx + 4) for 3 <= nx <= 128
constexpr int kTxMaxZ = 128;                     // output planes per CTA (z chunks are at most this long)

// FP32 bands of every subdomain: the mass as it is, the stiffness with the
// transmission term p of each interface side added at that side's end node
// (a subdomain uses p_lo on the faces where it is the lower side -- its +x,
// +y, +z sides -- and p_hi on its -x, -y, -z sides).  One block per subdomain.
__global__ void k_tensor_coef(DevProblem d) {
  const int s = blockIdx.x;
  const int* dims = d.box_dims + kBoxDims * s;
  const int nx = dims[0], ny = dims[1], nz = dims[2], fm = dims[3];
  const double* c = d.tc + 4 * s;
  const int64_t b0 = (int64_t)d.box_band0[s] * 5;
  const int n5 = 5 * (nx + ny + nz);
  for (int t = threadIdx.x; t < n5; t += blockDim.x) {
    double kv = d.band_k[b0 + t];
    const double mv = d.band_m[b0 + t];
    if (t % 5 == 2) {   // diagonal entry of band node t / 5
      const int node = t / 5;
      const int ax = node < nx ? 0 : (node < nx + ny ? 1 : 2);
      const int pos = ax == 0 ? node : (ax == 1 ? node - nx : node - nx - ny);
      const int len = ax == 0 ? nx : (ax == 1 ? ny : nz);
      if (pos == 0 && ((fm >> (8 + 2 * ax)) & 1)) kv += c[2];
      if (pos == len - 1 && ((fm >> (9 + 2 * ax)) & 1)) kv += c[0];
    }
    d.cK32[b0 + t] = (float)kv;
    d.cM32[b0 + t] = (float)mv;
  }
}

// Asynchronous 4-byte global -> shared copy (LDGSTS); src_bytes = 0 fills
// the destination with zero (halo rows outside the box).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// MODE 0: one step of the FP32 inner CG (the tensor counterpart of
// k_cg_spmv_dir32): t = A z, then p = z + beta p, q = t + beta q (first step
// beta = 0: p = z, q = t) and the CTA's partial of p.q (scaled FP32 dots as in
// the SELL kernel) into part0[cta]; the subdomain's last CTA (a ticket, no
// waiting) adds the partials in a fixed order and stores p.q and alpha = r.z
// / p.q for the update kernel.  MODE 1: y = A x (x, y in the box layout).
// A CTA covers 256 (x, y) columns of one box and one chunk of its z range
// (box_dims: the chunk length and the number of column blocks), marching
// over the chunk's planes and the two halo planes on either side.  The input
// planes stream through kTxStages shared-memory stages filled by
// asynchronous copies issued kTxStages - 1 planes ahead, together with the
// old p and q of the output plane they complete.  The plane loop is unrolled
// by five, so the five-plane rings of the partial products live in fixed
// registers.
template <int MODE>
__global__ void __launch_bounds__(kTileRows, 3) k_tensor32(DevProblem d, const float* __restrict__ xin,
                                                           float* __restrict__ yout) {
  __shared__ __align__(16) float S[kTxStages][kTxPlane];
  __shared__ float PQ[MODE == 0 ? kTxStages : 1][2][MODE == 0 ? kTileRows : 1];   // old p, q of an output plane
  __shared__ float TM[kTxRowsP], TK[kTxRowsP];   // y-pass rows, two zero columns either side
  __shared__ float CY[kTxMaxRows][10];           // y bands of the CTA's rows: M then K~
  __shared__ float CZ[kTxMaxZ][10];              // z bands of the chunk's output planes
  __shared__ double red[kTileSlices];
  __shared__ bool s_last;
  const int cta = blockIdx.x;
  const int s = d.cta_sub[cta];
  if (MODE == 0 && !d.st.active[s]) return;
  const int* dims = d.box_dims + kBoxDims * s;
  const int nx = dims[0], ny = dims[1], nz = dims[2], fm = dims[3], zc = dims[4], ncb = dims[5];
  const int nxy = nx * ny, nxp = nx + 4;
  const int64_t voff = d.box_voff[s];
  const int local = (int)(cta - d.sub_cta0[s]);
  const int c0 = (local % ncb) * kTileRows;
  const int k0 = (local / ncb) * zc, k1 = min(nz, k0 + zc);   // output planes [k0, k1)
  const int col = c0 + (int)threadIdx.x;
  const bool valid = col < nxy;
  const int jlo = c0 / nx, jhi = min(ny - 1, (c0 + kTileRows - 1) / nx);
  const int nrow = jhi - jlo + 1, nload = (nrow + 4) * nx, ntr = nrow * nx;
  const int j = valid ? col / nx : jlo, i = valid ? col - j * nx : 0;
  const int64_t bx = (int64_t)d.box_band0[s] * 5, by = bx + 5 * (int64_t)nx, bz = by + 5 * (int64_t)ny;
  const float* __restrict__ cK = d.cK32;
  const float* __restrict__ cM = d.cM32;
  for (int t = threadIdx.x; t < 5 * nrow; t += kTileRows) {
    CY[t / 5][t % 5] = cM[by + 5 * (int64_t)jlo + t];
    CY[t / 5][5 + t % 5] = cK[by + 5 * (int64_t)jlo + t];
  }
  for (int t = threadIdx.x; t < 5 * (k1 - k0); t += kTileRows) {
    CZ[t / 5][t % 5] = cM[bz + 5 * (int64_t)k0 + t];
    CZ[t / 5][5 + t % 5] = cK[bz + 5 * (int64_t)k0 + t];
  }
  for (int t = threadIdx.x; t < 4 * nrow; t += kTileRows) {   // the zero columns of TM, TK
    const int r = t >> 2, c = t & 3;
    const int at = r * nxp + (c < 2 ? c : nx + c);
    TM[at] = 0.f;
    TK[at] = 0.f;
  }
  float kx[5], mx[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    kx[a] = cK[bx + 5 * i + a];
    mx[a] = cM[bx + 5 * i + a];
  }
  // column on the outer boundary (x or y side): its rows are Dirichlet
  const bool dcol = ((fm & 1) && i == 0) || ((fm & 2) && i == nx - 1) || ((fm & 4) && j == 0) ||
                    ((fm & 8) && j == ny - 1);
  // plane-relative offsets of this thread's staged values (the same in every
  // plane); -1: a halo row outside the box, staged as zero
  int goff[kTxPre];
#pragma unroll
  for (int m = 0; m < kTxPre; ++m) {
    const int idx = (int)threadIdx.x + m * kTileRows;
    goff[m] = -2;   // beyond the staged region: no copy
    if (idx < nload) {
      const int r = idx / nx, jj = jlo - 2 + r;
      goff[m] = (jj >= 0 && jj < ny) ? (idx - r * nx) + nx * jj : -1;
    }
  }
  // y-pass slots: output row (in the CTA's rows) and padded TM index
  int yrow[kTxY], ypad[kTxY];
#pragma unroll
  for (int m = 0; m < kTxY; ++m) {
    const int idx = (int)threadIdx.x + m * kTileRows;
    yrow[m] = idx < ntr ? idx / nx : -1;
    ypad[m] = yrow[m] >= 0 ? yrow[m] * nxp + 2 + (idx - yrow[m] * nx) : 0;
  }
  const int xbase = (j - jlo) * nxp + i;   // TM index of this column's neighbour i - 2
  const int zown = (j - jlo + 2) * nx + i;  // this column in the staged plane
  const float* __restrict__ src = MODE == 0 ? d.z32 : xin;
  float beta = 0.f, sc = 1.f;
  bool first = true;
  if (MODE == 0) {
    const double b64 = d.st.beta[s];
    first = b64 == 0.0;
    beta = (float)b64;
    sc = d.st.sc[s];
  }
  // copies into stage st of input plane kk and (CG step) of the old p, q of
  // output plane kk - 2, which is produced when plane kk is consumed; one
  // commit group per plane, empty outside the box, so that the group count
  // stays uniform
  auto issue = [&](int kk, int st) {
    if (kk >= 0 && kk < nz) {
      const float* pl = src + voff + (int64_t)nxy * kk;
#pragma unroll
      for (int m = 0; m < kTxPre; ++m)
        if (goff[m] >= -1) cp_async4(&S[st][threadIdx.x + m * kTileRows], pl + max(goff[m], 0), goff[m] >= 0);
    }
    if (MODE == 0 && !first && valid && kk - 2 >= k0 && kk - 2 < k1) {
      const int64_t row = voff + col + (int64_t)nxy * (kk - 2);
      cp_async4(&PQ[st][0][threadIdx.x], d.p32 + row, true);
      cp_async4(&PQ[st][1][threadIdx.x], d.q32 + row, true);
    }
    cp_async_commit();
  };
  float ph[5], qh[5], zh[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) { ph[c] = 0.f; qh[c] = 0.f; zh[c] = 0.f; }
  float vv = 0.f;
#pragma unroll
  for (int st = 0; st < kTxStages - 1; ++st) issue(k0 - 2 + st, st);
  int st = 0;
  for (int kb = k0 - 2; kb < k1 + 2; kb += 5) {
#pragma unroll
    for (int u = 0; u < 5; ++u) {
      const int kk = kb + u;
      if (kk < k1 + 2) {   // uniform across the CTA
        // plane kk + stages - 1 into the stage freed at the end of the last plane
        issue(kk + kTxStages - 1, st == 0 ? kTxStages - 1 : st - 1);
        cp_async_wait<kTxStages - 1>();   // this thread's copies of plane kk have landed
        __syncthreads();                  // ... and every other thread's
        const bool pin = kk >= 0 && kk < nz;
        float zc_own = 0.f;
        if (pin) {
          // y pass: My z and K~y z on the CTA's rows, every x
#pragma unroll
          for (int m = 0; m < kTxY; ++m) {
            if (yrow[m] >= 0) {
              const int idx = (int)threadIdx.x + m * kTileRows;
              const float* cy = CY[yrow[m]];
              float sm = 0.f, sk = 0.f;
#pragma unroll
              for (int b = 0; b < 5; ++b) {
                const float v = S[st][idx + b * nx];
                sm = fmaf(cy[b], v, sm);
                sk = fmaf(cy[5 + b], v, sk);
              }
              TM[ypad[m]] = sm;
              TK[ypad[m]] = sk;
            }
          }
          if (valid) zc_own = S[st][zown];
        }
        __syncthreads();   // TM, TK complete; stage st is free for the next issue
        // x pass for this thread's column: P = K~x (My z) + Mx (K~y z), Q = Mx (My z)
        float P = 0.f, Q = 0.f;
        if (pin && valid) {
#pragma unroll
          for (int a = 0; a < 5; ++a) {
            const float tm = TM[xbase + a], tk = TK[xbase + a];
            P = fmaf(kx[a], tm, fmaf(mx[a], tk, P));
            Q = fmaf(mx[a], tm, Q);
          }
        }
        // ring slot u holds plane kk; slot (u + 1 + c) % 5 holds plane kk - 4 + c
        ph[u] = P;
        qh[u] = Q;
        zh[u] = zc_own;
        const int k = kk - 2;   // output plane: its neighbours k-2 .. k+2 are in the rings
        if (k >= k0 && valid) {
          const float* cz = CZ[k - k0];
          float t = 0.f;
#pragma unroll
          for (int c = 0; c < 5; ++c) t = fmaf(cz[c], ph[(u + 1 + c) % 5], fmaf(cz[5 + c], qh[(u + 1 + c) % 5], t));
          if (dcol || ((fm & 16) && k == 0) || ((fm & 32) && k == nz - 1)) t = 0.f;
          const int64_t row = voff + col + (int64_t)nxy * k;
          if (MODE == 0) {
            const float z = zh[(u + 3) % 5];
            float p = z, q = t;
            if (!first) {   // this thread's own staged values: no barrier needed
              p = fmaf(beta, PQ[st][0][threadIdx.x], z);
              q = fmaf(beta, PQ[st][1][threadIdx.x], t);
            }
            d.p32[row] = p;
            d.q32[row] = q;
            vv = fmaf(p * sc, q * sc, vv);
          } else {
            yout[row] = t;
          }
        }
        st = st + 1 == kTxStages ? 0 : st + 1;
      }
    }
  }
  cp_async_wait<0>();   // no copy outlives the CTA
  if (MODE == 0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vv += __shfl_xor_sync(0xffffffffu, vv, o);
    if (lane == 0) red[warp] = (double)vv * d.st.isc2[s];
    __syncthreads();
    if (threadIdx.x == 0) {
      double acc = 0.0;
#pragma unroll
      for (int w = 0; w < kTileSlices; ++w) acc += red[w];
      d.part0[cta] = acc;
      // the subdomain's last CTA forms p.q and alpha (a ticket, not a wait)
      __threadfence();
      const unsigned nct = (unsigned)(d.sub_cta0[s + 1] - d.sub_cta0[s]);
      const unsigned t = atomicAdd(&d.st.tcnt[s], 1u);
      s_last = t == nct - 1u;
      if (s_last) d.st.tcnt[s] = 0u;
    }
    __syncthreads();
    if (s_last && warp == 0) {
      __threadfence();
      const int64_t a0 = d.sub_cta0[s];
      const double pq = warp_sum_parts(d.part0, a0, d.sub_cta0[s + 1] - a0);
      if (lane == 0) {
        d.st.pq[s] = pq;
        d.st.alpha[s] = (pq > 0.0 && isfinite(pq)) ? d.st.rho[s] / pq : 0.0;
      }
    }
  }
}

}  // namespace

DevProblem fp32_view(const DevProblem& d) {
  if (!d.t32) return d;
  DevProblem v = d;
  v.tile_sub = d.box_tile_sub;
  v.sub_tile0 = d.box_sub_tile0;
  v.n_tiles = d.box_n_tiles;
  v.ub_tile0 = d.box_ub_tile0;
  v.sub_ub0 = d.box_sub_ub0;
  v.n_ublocks = d.box_n_ublocks;
  v.alpha_ready = 1;   // the tensor kernel's last CTA per subdomain forms p.q and alpha
  v.sub_part0 = d.sub_cta0;
  return v;
}

cudaError_t launch_tensor_coef(const DevProblem& d, cudaStream_t s) {
  if (!d.box_dims || d.n_sub == 0) return cudaSuccess;
  k_tensor_coef<<<(unsigned)d.n_sub, 128, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_tensor_dir32(const DevProblem& d, cudaStream_t s) {
  k_tensor32<0><<<(unsigned)d.n_cta32, kTileRows, 0, s>>>(d, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_tensor_apply32(const DevProblem& d, const float* x, float* y, cudaStream_t s) {
  k_tensor32<1><<<(unsigned)d.n_cta32, kTileRows, 0, s>>>(d, x, y);
  return cudaGetLastError();
}

}  // namespace osm
