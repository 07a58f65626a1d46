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

#include <type_traits>

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

// FP32 (and FP64) bands of every subdomain: the mass as it is, the stiffness with the
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
    d.cKp32[b0 + t] = (float)d.band_k[b0 + t];   // plain stiffness (stop-test layer)
    if (d.cK64) {
      d.cK64[b0 + t] = kv;
      d.cM64[b0 + t] = mv;
    }
    if (d.cKdf) {
      d.cKdf[b0 + t] = df_split(kv);
      d.cMdf[b0 + t] = df_split(mv);
    }
  }
}

// Asynchronous 4- or 8-byte global -> shared copy (LDGSTS); src_bytes = 0
// fills the destination with zero (halo rows outside the box).
template <class T>
__device__ __forceinline__ void cp_async(T* dst, const T* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Fused multiply-add in the kernel's own precision (fmaf for float: no
// detour through double).
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// Double-float number: the unevaluated sum hi + lo of two floats.  A sum of
// products is formed by compensated dot-product summation (Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005),
// algorithm Dot2, extended to double-float factors): every product a b is
// split without error into p + e by one FMA (e = fma(a.hi, b.hi, -p)), the
// cross terms a.hi b.lo + a.lo b.hi join e, p enters the running hi by an
// error-free two-sum, and all error terms gather in lo.  Inside a sum the
// pair is unnormalised; fin_t renormalises it (|lo| <= ulp(hi) / 2) before it
// is stored or multiplied again.  The result carries about 48 significant
// bits, in FP32 arithmetic only.
struct __align__(8) Df {
  float hi, lo;
  Df() = default;
  __device__ constexpr Df(float h, float l = 0.f) : hi(h), lo(l) {}
};
__device__ __forceinline__ Df fma_t(Df a, Df b, Df acc) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);                  // a.hi b.hi = p + e exactly
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));       // a.lo b.lo is below the pair's precision
  const float s = acc.hi + p;                      // two-sum: acc.hi + p = s + err exactly
  const float bv = s - acc.hi;
  const float err = (acc.hi - (s - bv)) + (p - bv);
  return Df(s, acc.lo + (err + e));
}
__device__ __forceinline__ float fin_t(float v) { return v; }
__device__ __forceinline__ double fin_t(double v) { return v; }
__device__ __forceinline__ Df fin_t(Df v) {   // fast two-sum (|hi| >= |lo|)
  const float h = v.hi + v.lo;
  return Df(h, v.lo - (h - v.hi));
}
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(Df v) { return (double)v.hi + (double)v.lo; }

// Modes of the tensor kernel.
constexpr int kTxCgStep = 0;   // FP32: one step of the inner CG (t = A z and the direction epilogue)
constexpr int kTxApply = 1;    // FP32: y = A x
constexpr int kTxInit = 2;     // FP64 or double-float: the refinement's defect d = b - A u and the FP32 CG start
constexpr int kTxLayer = 3;    // FP32: y += K (ubar - u) for the stop test (plain stiffness K)

// Dynamic shared memory of the tensor kernel (element type T): the staged
// input planes, the old p and q (CG step), the two y-pass rows, the y and z
// bands, and the block reduction.
template <class T, int MODE>
struct TxSmem {
  static constexpr size_t S = 0;
  static constexpr size_t PQ = S + sizeof(T) * kTxStages * kTxPlane;
  static constexpr size_t TM = PQ + (MODE == kTxCgStep ? sizeof(float) * kTxStages * 2 * kTileRows : 0);
  static constexpr size_t TK = TM + sizeof(T) * kTxRowsP;
  static constexpr size_t CY = TK + sizeof(T) * kTxRowsP;
  static constexpr size_t CZ = CY + sizeof(T) * kTxMaxRows * 10;
  static constexpr size_t RED = (CZ + sizeof(T) * kTxMaxZ * 10 + 15) / 16 * 16;
  static constexpr size_t BYTES = RED + sizeof(double) * 3 * kTileSlices + 16;
};

// kTxCgStep: one step of the FP32 inner CG (the tensor counterpart of
// k_cg_spmv_dir32): t = A z, then p = z + beta p, q = t + beta q (first step
// beta = 0: p = z, q = t) and the CTA's partial of p.q (scaled FP32 dots as in
// the SELL kernel) into part0[cta]; the subdomain's last CTA (a ticket, no
// waiting) adds the partials in a fixed order and stores p.q and alpha = r.z
// / p.q for the update kernel.
// kTxApply: y = A x (x, y in the box layout).
// kTxLayer: the stop test's interface correction.  The difference of the
// averaged and the local iterate, ubar - u, is nonzero on interface nodes
// only and small; K (ubar - u) with the plain stiffness K (no transmission
// term) in FP32 is added to y = A u - T u (FP64, vector rows) to give K ubar.
// Its FP32 rounding, ~1e-7 of |K| |ubar - u|, is far below the residual it
// enters.
// kTxInit (T = double): the mixed form's refinement step starts here when
// the tensor form is in use: with u in the box layout (ub), t = A u in FP64,
// and for every unknown (vector row `row`) y[row] = t, the defect d = b - t,
// r = d and z = D^-1 r in FP32 for the inner CG (x = 0), and the CTA's
// partials of ||d||^2, ||b||^2 and r.z (k_fin_init adds them).
// A CTA covers 256 (x, y) columns of one box and one chunk of its z range
// (box_dims: the chunk length and the number of column blocks), marching
// over the chunk's planes and the two halo planes on either side.  The input
// planes stream through kTxStages shared-memory stages filled by
// asynchronous copies issued kTxStages - 1 planes ahead, together with the
// old p and q of the output plane they complete (CG step).  The plane loop is
// unrolled by five, so the five-plane rings of the partial products live in
// fixed registers.
template <class T, int MODE>
__global__ void __launch_bounds__(kTileRows, sizeof(T) == 4 ? 3 : 2)
    k_tensor(DevProblem d, const T* __restrict__ xin, T* __restrict__ yout) {
  using L = TxSmem<T, MODE>;
  extern __shared__ __align__(16) unsigned char smem[];
  T (*S)[kTxPlane] = reinterpret_cast<T (*)[kTxPlane]>(smem + L::S);
  float (*PQ)[2][kTileRows] = reinterpret_cast<float (*)[2][kTileRows]>(smem + L::PQ);
  T* TM = reinterpret_cast<T*>(smem + L::TM);   // y-pass rows, two zero columns either side
  T* TK = reinterpret_cast<T*>(smem + L::TK);
  T (*CY)[10] = reinterpret_cast<T (*)[10]>(smem + L::CY);   // y bands of the CTA's rows: M then K~
  T (*CZ)[10] = reinterpret_cast<T (*)[10]>(smem + L::CZ);   // z bands of the chunk's output planes
  double (*red)[kTileSlices] = reinterpret_cast<double (*)[kTileSlices]>(smem + L::RED);
  bool* s_last = reinterpret_cast<bool*>(smem + L::RED + sizeof(double) * 3 * kTileSlices);
  const int cta = blockIdx.x;
  const int s = d.cta_sub[cta];
  if (MODE == kTxCgStep && !d.st.active[s]) return;
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
  const T* __restrict__ cK;
  const T* __restrict__ cM;
  if constexpr (MODE == kTxLayer) {
    cK = d.cKp32;
    cM = d.cM32;
  } else if constexpr (sizeof(T) == 4) {
    cK = d.cK32;
    cM = d.cM32;
  } else if constexpr (std::is_same<T, Df>::value) {
    cK = reinterpret_cast<const Df*>(d.cKdf);
    cM = reinterpret_cast<const Df*>(d.cMdf);
  } else {
    cK = d.cK64;
    cM = d.cM64;
  }
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
    TM[at] = T(0);
    TK[at] = T(0);
  }
  T kx[5], mx[5];
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
  const int xbase = (j - jlo) * nxp + i;    // TM index of this column's neighbour i - 2
  const int zown = (j - jlo + 2) * nx + i;  // this column in the staged plane
  const T* __restrict__ src;
  if constexpr (MODE == kTxCgStep) src = d.z32;
  else if constexpr (MODE == kTxInit && std::is_same<T, Df>::value) src = reinterpret_cast<const Df*>(d.ub2);
  else if constexpr (MODE == kTxInit) src = reinterpret_cast<const T*>(d.ub);
  else if constexpr (MODE == kTxLayer) src = d.dl32;
  else src = xin;
  float beta = 0.f, sc = 1.f;
  bool first = true;
  if (MODE == kTxCgStep) {
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
      const T* pl = src + voff + (int64_t)nxy * kk;
#pragma unroll
      for (int m = 0; m < kTxPre; ++m)
        if (goff[m] >= -1) cp_async(&S[st][threadIdx.x + m * kTileRows], pl + max(goff[m], 0), goff[m] >= 0);
    }
    if (MODE == kTxCgStep && !first && valid && kk - 2 >= k0 && kk - 2 < k1) {
      const int64_t row = voff + col + (int64_t)nxy * (kk - 2);
      cp_async(&PQ[st][0][threadIdx.x], d.p32 + row, true);
      cp_async(&PQ[st][1][threadIdx.x], d.q32 + row, true);
    }
    cp_async_commit();
  };
  T ph[5], qh[5], zh[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) { ph[c] = T(0); qh[c] = T(0); zh[c] = T(0); }
  float vv = 0.f;                    // CG step: p.q
  double v0 = 0.0, v1 = 0.0, v2 = 0.0;   // init: ||d||^2, ||b||^2, r.z
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
        T zc_own = T(0);
        if (pin) {
          // y pass: My z and K~y z on the CTA's rows, every x
#pragma unroll
          for (int m = 0; m < kTxY; ++m) {
            if (yrow[m] >= 0) {
              const int idx = (int)threadIdx.x + m * kTileRows;
              const T* cy = CY[yrow[m]];
              T sm = T(0), sk = T(0);
#pragma unroll
              for (int b = 0; b < 5; ++b) {
                const T v = S[st][idx + b * nx];
                sm = fma_t(cy[b], v, sm);
                sk = fma_t(cy[5 + b], v, sk);
              }
              TM[ypad[m]] = fin_t(sm);
              TK[ypad[m]] = fin_t(sk);
            }
          }
          if (MODE == kTxCgStep && valid) zc_own = S[st][zown];
        }
        __syncthreads();   // TM, TK complete; stage st is free for the next issue
        // x pass for this thread's column: P = K~x (My z) + Mx (K~y z), Q = Mx (My z)
        T P = T(0), Q = T(0);
        if (pin && valid) {
#pragma unroll
          for (int a = 0; a < 5; ++a) {
            const T tm = TM[xbase + a], tk = TK[xbase + a];
            P = fma_t(kx[a], tm, fma_t(mx[a], tk, P));
            Q = fma_t(mx[a], tm, Q);
          }
        }
        // ring slot u holds plane kk; slot (u + 1 + c) % 5 holds plane kk - 4 + c
        ph[u] = fin_t(P);
        qh[u] = fin_t(Q);
        zh[u] = zc_own;
        const int k = kk - 2;   // output plane: its neighbours k-2 .. k+2 are in the rings
        if (k >= k0 && valid) {
          const T* cz = CZ[k - k0];
          T t = T(0);
#pragma unroll
          for (int c = 0; c < 5; ++c) t = fma_t(cz[c], ph[(u + 1 + c) % 5], fma_t(cz[5 + c], qh[(u + 1 + c) % 5], t));
          const bool dir = dcol || ((fm & 16) && k == 0) || ((fm & 32) && k == nz - 1);
          const int64_t row = voff + col + (int64_t)nxy * k;
          if constexpr (MODE == kTxCgStep) {
            if (dir) t = 0.f;
            const float z = zh[(u + 3) % 5];
            float p = z, q = t;
            if (!first) {   // this thread's own staged values: no barrier needed
              p = fmaf(beta, PQ[st][0][threadIdx.x], z);
              q = fmaf(beta, PQ[st][1][threadIdx.x], t);
            }
            d.p32[row] = p;
            d.q32[row] = q;
            vv = fmaf(p * sc, q * sc, vv);
          } else if constexpr (MODE == kTxInit) {
            const int32_t vr = d.box_vec[row];   // the unknown's vector row (-1: Dirichlet)
            if (!dir && vr >= 0) {
              const double b = d.b[vr];
              const double tv = to_double(t);
              const double dfc = b - tv;
              d.y[vr] = tv;
              const float r = (float)dfc;
              const float z = d.dinv32b[row] * r;
              d.r32[row] = r;
              d.z32[row] = z;   // p = z is formed by the first CG-step kernel (beta = 0)
              d.x32[row] = 0.f;
              v0 = fma(dfc, dfc, v0);
              v1 = fma(b, b, v1);
              v2 += (double)r * (double)z;
            }
          } else if constexpr (MODE == kTxLayer) {
            const int32_t vr = d.box_vec[row];
            if (!dir && vr >= 0) d.y[vr] += (double)t;
          } else {
            yout[row] = dir ? T(0) : t;
          }
        }
        st = st + 1 == kTxStages ? 0 : st + 1;
      }
    }
  }
  cp_async_wait<0>();   // no copy outlives the CTA
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (MODE == kTxCgStep) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vv += __shfl_xor_sync(0xffffffffu, vv, o);
    if (lane == 0) red[0][warp] = (double)vv * d.st.isc2[s];
    __syncthreads();
    if (threadIdx.x == 0) {
      double acc = 0.0;
#pragma unroll
      for (int w = 0; w < kTileSlices; ++w) acc += red[0][w];
      d.part0[cta] = acc;
      // the subdomain's last CTA forms p.q and alpha (a ticket, not a wait)
      __threadfence();
      const unsigned nct = (unsigned)(d.sub_cta0[s + 1] - d.sub_cta0[s]);
      const unsigned tk = atomicAdd(&d.st.tcnt[s], 1u);
      *s_last = tk == nct - 1u;
      if (*s_last) d.st.tcnt[s] = 0u;
    }
    __syncthreads();
    if (*s_last && warp == 0) {
      __threadfence();
      const int64_t a0 = d.sub_cta0[s];
      const double pq = warp_sum_parts(d.part0, a0, d.sub_cta0[s + 1] - a0);
      if (lane == 0) {
        d.st.pq[s] = pq;
        d.st.alpha[s] = (pq > 0.0 && isfinite(pq)) ? d.st.rho[s] / pq : 0.0;
      }
    }
  } else if constexpr (MODE == kTxInit) {
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    if (lane == 0) {
      red[0][warp] = v0;
      red[1][warp] = v1;
      red[2][warp] = v2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double acc = 0.0;
#pragma unroll
      for (int w = 0; w < kTileSlices; ++w) acc += red[threadIdx.x][w];
      (threadIdx.x == 0 ? d.part0 : threadIdx.x == 1 ? d.part1 : d.part2)[cta] = acc;
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
  v.sub_part0 = d.sub_cta0;
  return v;
}

cudaError_t launch_tensor_coef(const DevProblem& d, cudaStream_t s) {
  if (!d.box_dims || d.n_sub == 0) return cudaSuccess;
  k_tensor_coef<<<(unsigned)d.n_sub, 128, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t tensor_kernel_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_tensor<float, kTxCgStep>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TxSmem<float, kTxCgStep>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tensor<float, kTxApply>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TxSmem<float, kTxApply>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tensor<double, kTxInit>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TxSmem<double, kTxInit>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tensor<Df, kTxInit>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TxSmem<Df, kTxInit>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tensor<float, kTxLayer>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TxSmem<float, kTxLayer>::BYTES);
  return e;
}

cudaError_t launch_tensor_dir32(const DevProblem& d, cudaStream_t s) {
  k_tensor<float, kTxCgStep><<<(unsigned)d.n_cta32, kTileRows, TxSmem<float, kTxCgStep>::BYTES, s>>>(d, nullptr,
                                                                                                    nullptr);
  return cudaGetLastError();
}

cudaError_t launch_tensor_apply32(const DevProblem& d, const float* x, float* y, cudaStream_t s) {
  k_tensor<float, kTxApply><<<(unsigned)d.n_cta32, kTileRows, TxSmem<float, kTxApply>::BYTES, s>>>(d, x, y);
  return cudaGetLastError();
}

cudaError_t launch_tensor_layer(const DevProblem& d, cudaStream_t s) {
  k_tensor<float, kTxLayer><<<(unsigned)d.n_cta32, kTileRows, TxSmem<float, kTxLayer>::BYTES, s>>>(d, nullptr,
                                                                                                   nullptr);
  return cudaGetLastError();
}

cudaError_t launch_tensor_init_df(const DevProblem& d, cudaStream_t s) {
  k_tensor<Df, kTxInit><<<(unsigned)d.n_cta32, kTileRows, TxSmem<Df, kTxInit>::BYTES, s>>>(d, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_tensor_init64(const DevProblem& d, cudaStream_t s) {
  k_tensor<double, kTxInit><<<(unsigned)d.n_cta32, kTileRows, TxSmem<double, kTxInit>::BYTES, s>>>(d, nullptr,
                                                                                                  nullptr);
  return cudaGetLastError();
}

}  // namespace osm
