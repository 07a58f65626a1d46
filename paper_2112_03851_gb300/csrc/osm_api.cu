// C ABI of libosm (include/osm.h): handle lifetime, upload of the host-built
// problem, and the solve driver.
//
// The whole Schwarz solve is one CUDA graph with two nested device-side
// while loops (conditional graph nodes), so no host round trip happens
// inside a solve:
//
//   while (relres > rtol && n < max_outer) {          // Schwarz iteration
//     b_i = f_i + sum_j lam_ij                          // Robin RHS
//     CG start on every subdomain (warm)                // r, z, p, active flags
//     while (any subdomain active) { q = A p; alpha; x, r, z update; beta; p }
//     lam exchange                                      // Sec. 3
//     ubar, r = f - K ubar, relres                      // stop test
//   }
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "osm_internal.h"

using namespace osm;

// z-chunk lengths the autotuner tries for the tensor kernel (the last one
// leaves every box of up to 128 planes whole).
constexpr int kZChunks[4] = {8, 16, 32, 128};
constexpr int kTailStride = 8;   // z-chunk tuning: the tail state keeps one subdomain in 8 active

struct osm_ctx {
  HostProblem hp;
  osm_opts opts;
  cudaStream_t stream = nullptr;
  int device = 0;
  DevProblem d{};
  std::vector<void*> allocs;
  size_t dev_bytes = 0;
  std::string err;
  double setup_seconds = 0.0;
  // graph
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  DevCtl* ctl_host = nullptr;   // pinned mirror
  std::vector<double> psub_host;
  std::vector<double> tc_host;  // 4 per subdomain: p_lo, q_lo, p_hi, q_hi
  bool tc_general = false;      // second-order or unsymmetric coefficients in use
  // batched p evaluation (allocated on the first osm_sample_p call)
  bool mp_ready = false;
  DevSample mp{};
  cudaGraph_t mp_graph = nullptr;
  cudaGraphExec_t mp_exec = nullptr;
  int last_kind = 0;            // 0: single solve / iterate, 1: batched p evaluation
  double tune_ms[2][4] = {};  // [fp64, fp32][2 c16 + rpl - 1]
  // tensor-product FP32 operator (mixed handles whose boxes fit the kernel)
  bool have_box = false;
  int fp32_tuned = 1;           // 1: SELL, 2: tensor product (autotuner or opts.fp32_operator)
  int init_tuned = 0;           // the mixed refinement step's start: 0 SELL, 1 FP64 tensor, 2 double-float tensor
  double tune_init_ms[3] = {};  // autotuner timings of those three
  int zchunk = kZChunks[1];     // z planes per CTA of the tensor kernel (autotuned)
  double tune_tensor_ms = 0.0;
  double tune_zchunk_ms[4] = {};
  double tune_zchunk_tail_ms[4] = {};   // the same with one subdomain in kTailStride active
  // adjoint gradient (allocated on first use)
  bool adj_ready = false;
  DevAdjoint adj{};
  double* J_dev = nullptr;
  // reverse-mode Schwarz: partner slot of every received Robin datum, and a
  // graph that only runs the subdomain solves
  int32_t* ilam_partner = nullptr;
  cudaGraph_t ls_graph = nullptr;
  cudaGraphExec_t ls_exec = nullptr;
};

namespace {

osm_status fail(osm_ctx* h, osm_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

#define OSM_CUDA(h, call)                                                                       \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(h, e_ == cudaErrorMemoryAllocation ? OSM_E_NOMEM : OSM_E_CUDA,                \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

template <class T>
cudaError_t dalloc(osm_ctx* h, T** p, size_t n) {
  size_t bytes = (n ? n : 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess) {
    h->allocs.push_back(*p);
    h->dev_bytes += bytes;
    e = cudaMemsetAsync(*p, 0, bytes, h->stream);
  }
  return e;
}

template <class T>
cudaError_t upload(osm_ctx* h, T** p, const std::vector<T>& v) {
  cudaError_t e = dalloc(h, p, v.size());
  if (e == cudaSuccess && !v.empty())
    e = cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream);
  return e;
}

cudaError_t set_zchunk(osm_ctx* h, int zc);

osm_status upload_problem(osm_ctx* h) {
  HostProblem& hp = h->hp;
  DevProblem& d = h->d;
  const size_t nv = hp.vec_rows, ns = hp.nsub;
  int32_t *cols, *tile_sub;
  int64_t *slice_off, *sub_tile0;
  OSM_CUDA(h, upload(h, &slice_off, hp.slice_off));
  OSM_CUDA(h, upload(h, &cols, hp.cols));
  OSM_CUDA(h, upload(h, &d.vals, hp.vals));
  OSM_CUDA(h, upload(h, &tile_sub, hp.tile_sub));
  std::vector<int64_t> st0(ns + 1);
  for (size_t s = 0; s < ns; ++s) st0[s] = hp.sub[s].tile0;
  st0[ns] = hp.n_tiles;
  OSM_CUDA(h, upload(h, &sub_tile0, st0));
  d.slice_off = slice_off; d.cols = cols; d.tile_sub = tile_sub; d.sub_tile0 = sub_tile0;
  // blocks of the FP32 CG update: runs of up to kUpdGroup tiles within a subdomain
  for (int g : {kUpdGroup, kUpdGroup64}) {
    std::vector<int64_t> ub, sub_ub0(ns + 1, 0);
    for (size_t si = 0; si < ns; ++si) {
      const int64_t a0 = st0[si], a1 = st0[si + 1];
      sub_ub0[si] = (int64_t)ub.size();
      for (int64_t t = a0; t < a1; t += g) ub.push_back(t);
    }
    sub_ub0[ns] = (int64_t)ub.size();
    int64_t *dub, *dsub;
    OSM_CUDA(h, upload(h, &dub, ub));
    OSM_CUDA(h, upload(h, &dsub, sub_ub0));
    (g == kUpdGroup ? d.ub_tile0 : d.ub64_tile0) = dub;
    (g == kUpdGroup ? d.sub_ub0 : d.sub_ub64_0) = dsub;
    (g == kUpdGroup ? d.n_ublocks : d.n_ublocks64) = (int64_t)ub.size();
  }
  // 16-bit column indices for the single-path SpMVs when every subdomain fits
  // (the batched p evaluation keeps reading the 32-bit ones)
  int64_t max_pad = 0;
  for (const SubInfo& S : hp.sub) max_pad = std::max<int64_t>(max_pad, S.npad);
  if (h->opts.index16 && max_pad <= 65536) {
    std::vector<uint16_t> c16(hp.cols.size());
    for (size_t k = 0; k < c16.size(); ++k) c16[k] = (uint16_t)hp.cols[k];
    uint16_t* dc16;
    OSM_CUDA(h, upload(h, &dc16, c16));
    d.cols16 = dc16;
  }
  d.n_tiles = hp.n_tiles;
  d.n_sub = hp.nsub;
  for (double** v : {&d.x, &d.r, &d.z, &d.p, &d.q, &d.w, &d.y}) OSM_CUDA(h, dalloc(h, v, nv));
  OSM_CUDA(h, upload(h, &d.f, hp.f));
  OSM_CUDA(h, upload(h, &d.b, hp.f));       // b = f off the interface rows
  OSM_CUDA(h, upload(h, &d.dinv, hp.dinv0));
  double* kd;
  OSM_CUDA(h, upload(h, &kd, hp.kdiag));
  d.kdiag = kd;
  OSM_CUDA(h, dalloc(h, &d.psub, ns));
  DevSubState& st = d.st;
  for (double** v : {&st.rho, &st.alpha, &st.beta, &st.bb, &st.rr}) OSM_CUDA(h, dalloc(h, v, ns));
  for (int32_t** v : {&st.active, &st.iters, &st.status, &st.tsteps}) OSM_CUDA(h, dalloc(h, v, ns));
  OSM_CUDA(h, dalloc(h, &st.ucnt, ns));
  OSM_CUDA(h, dalloc(h, &st.tcnt, ns));
  OSM_CUDA(h, dalloc(h, &st.pq, ns));
  OSM_CUDA(h, dalloc(h, &st.sc, ns));
  OSM_CUDA(h, dalloc(h, &st.isc2, ns));
  // the tensor form of the FP32 operator (mixed handles): box layout tables
  if (h->opts.prec == OSM_MIXED && h->opts.fp32_operator != 1 && !hp.row_boxidx.empty()) {
    build_box_layout(hp, kZChunks[0]);   // the smallest chunk: the most CTAs
    h->have_box = hp.box_max_nx <= kTensorMaxNx && hp.box_rows < ((int64_t)1 << 31);
  }
  const size_t nparts = h->have_box ? (size_t)std::max({hp.n_tiles, hp.box_tiles, hp.box_ctas}) : (size_t)hp.n_tiles;
  for (double** v : {&d.part0, &d.part1, &d.part2}) OSM_CUDA(h, dalloc(h, v, nparts));
  d.sub_part0 = sub_tile0;
  d.sub_init0 = sub_tile0;
  // interface rows
  d.n_irow = (int32_t)hp.irow.size();
  int32_t *irow, *irow_sub, *ilam_ptr, *ilam, *im_ptr, *im_col;
  double *irow_mdiag, *im_val, *im_kval;
  int64_t* im_pos;
  OSM_CUDA(h, upload(h, &irow, hp.irow));
  OSM_CUDA(h, upload(h, &irow_sub, hp.irow_sub));
  OSM_CUDA(h, upload(h, &irow_mdiag, hp.irow_mdiag));
  OSM_CUDA(h, upload(h, &ilam_ptr, hp.ilam_ptr));
  OSM_CUDA(h, upload(h, &ilam, hp.ilam));
  OSM_CUDA(h, upload(h, &im_ptr, hp.im_ptr));
  OSM_CUDA(h, upload(h, &im_col, hp.im_col));
  OSM_CUDA(h, upload(h, &im_val, hp.im_val));
  OSM_CUDA(h, upload(h, &im_pos, hp.im_pos));
  OSM_CUDA(h, upload(h, &im_kval, hp.im_kval));
  d.irow = irow; d.irow_sub = irow_sub; d.irow_mdiag = irow_mdiag; d.ilam_ptr = ilam_ptr;
  d.ilam = ilam; d.im_ptr = im_ptr; d.im_col = im_col; d.im_val = im_val; d.im_pos = im_pos;
  d.im_kval = im_kval;
  double *im_tc, *irow_tdiag;
  OSM_CUDA(h, upload(h, &im_tc, hp.im_tc));
  OSM_CUDA(h, upload(h, &irow_tdiag, hp.irow_tdiag));
  d.im_tc = im_tc; d.irow_tdiag = irow_tdiag;
  OSM_CUDA(h, dalloc(h, &d.tc, 4 * ns));
  OSM_CUDA(h, dalloc(h, &d.im_t, hp.im_col.size()));
  // faces
  d.n_fent = hp.n_fent;
  int32_t *fent_face, *fent_row_s, *fent_row_t, *fm_ptr, *fm_col, *face_s, *face_t, *face_n;
  double* fm_val;
  int64_t* face_eo;
  OSM_CUDA(h, upload(h, &fent_face, hp.fent_face));
  OSM_CUDA(h, upload(h, &fent_row_s, hp.fent_row_s));
  OSM_CUDA(h, upload(h, &fent_row_t, hp.fent_row_t));
  OSM_CUDA(h, upload(h, &fm_ptr, hp.fm_ptr));
  OSM_CUDA(h, upload(h, &fm_col, hp.fm_col));
  OSM_CUDA(h, upload(h, &fm_val, hp.fm_val));
  double* fs_val;
  OSM_CUDA(h, upload(h, &fs_val, hp.fs_val));
  d.fs_val = fs_val;
  OSM_CUDA(h, upload(h, &face_s, hp.face_s));
  OSM_CUDA(h, upload(h, &face_t, hp.face_t));
  OSM_CUDA(h, upload(h, &face_n, hp.face_n));
  OSM_CUDA(h, upload(h, &face_eo, hp.face_eo));
  d.fent_face = fent_face; d.fent_row_s = fent_row_s; d.fent_row_t = fent_row_t; d.fm_ptr = fm_ptr;
  d.fm_col = fm_col; d.fm_val = fm_val; d.face_s = face_s; d.face_t = face_t; d.face_n = face_n;
  d.face_eo = face_eo;
  OSM_CUDA(h, dalloc(h, &d.lam, 2 * (size_t)hp.n_fent));
  // interface-column layer of K_i (stop test)
  d.n_lrow = (int32_t)hp.li_row.size();
  int32_t *li_row, *li_ptr, *li_col, *li_irow;
  double* li_val;
  OSM_CUDA(h, upload(h, &li_irow, hp.li_irow));
  d.li_irow = li_irow;
  OSM_CUDA(h, upload(h, &li_row, hp.li_row));
  OSM_CUDA(h, upload(h, &li_ptr, hp.li_ptr));
  OSM_CUDA(h, upload(h, &li_col, hp.li_col));
  OSM_CUDA(h, upload(h, &li_val, hp.li_val));
  d.li_row = li_row; d.li_ptr = li_ptr; d.li_col = li_col; d.li_val = li_val;
  // copies, outputs, stop test
  d.n_nodes = hp.n_nodes;
  int32_t *cp_ptr, *cp_idx, *can2vec;
  OSM_CUDA(h, upload(h, &cp_ptr, hp.cp_ptr));
  OSM_CUDA(h, upload(h, &cp_idx, hp.cp_idx));
  OSM_CUDA(h, upload(h, &can2vec, hp.can2vec));
  d.cp_ptr = cp_ptr; d.cp_idx = cp_idx; d.can2vec = can2vec;
  d.n_local = hp.n_local;
  OSM_CUDA(h, dalloc(h, &d.phi, hp.n_nodes));
  d.n_rblocks = (int64_t)hp.rblock_inst.size();
  d.n_inst = hp.n_inst;
  int32_t *sub_inst, *rblock_inst, *inst_rblock0;
  int64_t* rblock_node0;
  OSM_CUDA(h, upload(h, &sub_inst, hp.sub_inst));
  OSM_CUDA(h, upload(h, &rblock_inst, hp.rblock_inst));
  OSM_CUDA(h, upload(h, &inst_rblock0, hp.inst_rblock0));
  OSM_CUDA(h, upload(h, &rblock_node0, hp.rblock_node0));
  d.sub_inst = sub_inst; d.rblock_inst = rblock_inst; d.inst_rblock0 = inst_rblock0; d.rblock_node0 = rblock_node0;
  OSM_CUDA(h, dalloc(h, &d.inst_done, hp.n_inst));
  OSM_CUDA(h, dalloc(h, &d.inst_iters, hp.n_inst));
  OSM_CUDA(h, dalloc(h, &d.inst_relres, hp.n_inst));
  // interface nodes (two or more copies) of each instance and their blocks
  {
    std::vector<int32_t> inodes, iblock_inst, inst_iblock0(hp.n_inst + 1, 0);
    std::vector<int64_t> iblock0;
    for (int i = 0; i < hp.n_inst; ++i) {
      inst_iblock0[i] = (int32_t)iblock_inst.size();
      const size_t first = inodes.size();
      for (int64_t n = hp.rblock_node0[hp.inst_rblock0[i]]; n < hp.rblock_node0[hp.inst_rblock0[i + 1]]; ++n)
        if (hp.cp_ptr[n + 1] - hp.cp_ptr[n] >= 2) inodes.push_back((int32_t)n);
      for (size_t k = first; k < inodes.size(); k += 256) {
        iblock0.push_back((int64_t)k);
        iblock_inst.push_back(i);
      }
    }
    inst_iblock0[hp.n_inst] = (int32_t)iblock_inst.size();
    iblock0.push_back((int64_t)inodes.size());
    d.n_iblocks = (int64_t)iblock_inst.size();
    int32_t *din, *dii, *dib;
    int64_t* di0;
    OSM_CUDA(h, upload(h, &din, inodes));
    OSM_CUDA(h, upload(h, &di0, iblock0));
    OSM_CUDA(h, upload(h, &dii, iblock_inst));
    OSM_CUDA(h, upload(h, &dib, inst_iblock0));
    d.inodes = din; d.iblock0 = di0; d.iblock_inst = dii; d.inst_iblock0 = dib;
  }
  OSM_CUDA(h, dalloc(h, &d.rpart, std::max<int64_t>(1, d.n_iblocks)));
  OSM_CUDA(h, dalloc(h, &d.rpart2, d.n_rblocks));
  // the stop test's row-wise part: single-copy row flags, per-tile partials,
  // and each instance's tile range (its subdomains are consecutive)
  OSM_CUDA(h, dalloc(h, &d.tpart, hp.n_tiles));
  {
    std::vector<int64_t> it0(hp.n_inst + 1, hp.n_tiles);
    for (int s = hp.nsub - 1; s >= 0; --s) it0[hp.sub_inst[s]] = hp.sub[s].tile0;
    int64_t* dit0;
    OSM_CUDA(h, upload(h, &dit0, it0));
    d.inst_tile0 = dit0;
    uint8_t* single;
    OSM_CUDA(h, dalloc(h, &single, nv));
    OSM_CUDA(h, launch_mark_single(d, single, h->stream));
    d.row_single = single;
  }
  OSM_CUDA(h, dalloc(h, &d.fg, hp.n_nodes));
  OSM_CUDA(h, dalloc(h, &d.hist, h->opts.max_outer > 0 ? h->opts.max_outer : 1));
  OSM_CUDA(h, dalloc(h, &d.ctl, 1));
  OSM_CUDA(h, cudaMallocHost((void**)&h->ctl_host, sizeof(DevCtl)));
  if (h->opts.prec == OSM_MIXED) {
    OSM_CUDA(h, upload(h, &d.vals32, hp.vals32));
    int64_t* ip32;
    OSM_CUDA(h, upload(h, &ip32, hp.im_pos32));
    d.im_pos32 = ip32;
    const size_t nv32 = h->have_box ? std::max<size_t>(nv, (size_t)hp.box_rows) : nv;
    for (float** v : {&d.x32, &d.r32, &d.z32, &d.p32, &d.q32}) OSM_CUDA(h, dalloc(h, v, nv32));
    std::vector<float> di32(hp.dinv0.begin(), hp.dinv0.end());
    OSM_CUDA(h, upload(h, &d.dinv32, di32));
    if (h->have_box) {
      int32_t *row_box, *box_dims, *box_band0, *box_tile_sub, *cta_sub;
      int64_t *box_voff, *box_sub_tile0, *box_ub_tile0, *sub_cta0;
      OSM_CUDA(h, upload(h, &row_box, hp.row_box));
      OSM_CUDA(h, upload(h, &box_voff, hp.box_voff));
      OSM_CUDA(h, upload(h, &box_dims, hp.box_dims));
      std::vector<int32_t> band0(ns);
      for (size_t s = 0; s < ns; ++s) band0[s] = hp.sub[s].band0;
      OSM_CUDA(h, upload(h, &box_band0, band0));
      OSM_CUDA(h, upload(h, &box_tile_sub, hp.box_tile_sub));
      OSM_CUDA(h, upload(h, &box_sub_tile0, hp.box_sub_tile0));
      OSM_CUDA(h, upload(h, &box_ub_tile0, hp.box_ub_tile0));
      int64_t* box_sub_ub0;
      OSM_CUDA(h, upload(h, &box_sub_ub0, hp.box_sub_ub0));
      d.box_sub_ub0 = box_sub_ub0;
      OSM_CUDA(h, upload(h, &cta_sub, hp.box_cta_sub));
      OSM_CUDA(h, upload(h, &sub_cta0, hp.box_sub_cta0));
      d.row_box = row_box; d.box_voff = box_voff; d.box_dims = box_dims; d.box_band0 = box_band0;
      d.box_tile_sub = box_tile_sub; d.box_sub_tile0 = box_sub_tile0; d.box_ub_tile0 = box_ub_tile0;
      d.cta_sub = cta_sub; d.sub_cta0 = sub_cta0;
      d.box_n_tiles = hp.box_tiles;
      d.box_n_ublocks = (int64_t)hp.box_ub_tile0.size();
      d.n_cta32 = hp.box_ctas;
      if (h->opts.tensor_zchunk > 0) h->zchunk = h->opts.tensor_zchunk;
      OSM_CUDA(h, set_zchunk(h, h->zchunk));
      double *bk, *bm;
      OSM_CUDA(h, upload(h, &bk, hp.band_k));
      OSM_CUDA(h, upload(h, &bm, hp.band_m));
      d.band_k = bk; d.band_m = bm;
      OSM_CUDA(h, dalloc(h, &d.cK32, hp.band_k.size()));
      OSM_CUDA(h, dalloc(h, &d.cM32, hp.band_m.size()));
      int32_t* box_vec;
      OSM_CUDA(h, upload(h, &box_vec, hp.box_vec));
      d.box_vec = box_vec;
      OSM_CUDA(h, dalloc(h, &d.ub, hp.box_rows));
      OSM_CUDA(h, dalloc(h, &d.ub2, hp.box_rows));
      OSM_CUDA(h, dalloc(h, &d.cKdf, hp.band_k.size()));
      OSM_CUDA(h, dalloc(h, &d.cMdf, hp.band_m.size()));
      OSM_CUDA(h, dalloc(h, &d.cK64, hp.band_k.size()));
      OSM_CUDA(h, dalloc(h, &d.cKp32, hp.band_k.size()));
      OSM_CUDA(h, dalloc(h, &d.dl32, hp.box_rows));
      OSM_CUDA(h, dalloc(h, &d.cM64, hp.band_m.size()));
      OSM_CUDA(h, tensor_kernel_setup());
      std::vector<float> dib(hp.box_rows, 0.f);
      for (int64_t r = 0; r < hp.vec_rows; ++r)
        if (hp.row_box[r] >= 0) dib[hp.row_box[r]] = (float)hp.dinv0[r];
      OSM_CUDA(h, upload(h, &d.dinv32b, dib));
    }
  }
  return OSM_OK;
}

// Uploads the handle's transmission coefficients (tc_host: p_lo, q_lo, p_hi,
// q_hi per subdomain; psub_host: the Robin parameter of the zeroth-order
// symmetric form, used by the batched p evaluation and the p-derivative) and
// forms the local matrices and Jacobi diagonals.
osm_status select_fp32_operator(osm_ctx* h);

// CTA tables of the tensor kernel for z chunks of about `zc` planes, into the
// device arrays sized for the smallest chunk.
cudaError_t set_zchunk(osm_ctx* h, int zc) {
  HostProblem& hp = h->hp;
  box_cta_tables(hp, zc);
  h->zchunk = zc;
  cudaError_t e = cudaMemcpyAsync((void*)h->d.box_dims, hp.box_dims.data(), sizeof(int32_t) * hp.box_dims.size(),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void*)h->d.cta_sub, hp.box_cta_sub.data(), sizeof(int32_t) * hp.box_cta_sub.size(),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void*)h->d.sub_cta0, hp.box_sub_cta0.data(), sizeof(int64_t) * hp.box_sub_cta0.size(),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // the host tables change on the next call
  h->d.n_cta32 = hp.box_ctas;
  return e;
}

osm_status apply_robin(osm_ctx* h) {
  OSM_CUDA(h, cudaMemcpyAsync(h->d.psub, h->psub_host.data(), sizeof(double) * h->hp.nsub,
                              cudaMemcpyHostToDevice, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(h->d.tc, h->tc_host.data(), sizeof(double) * 4 * h->hp.nsub,
                              cudaMemcpyHostToDevice, h->stream));
  OSM_CUDA(h, launch_set_robin(h->d, h->stream));
  if (h->have_box) OSM_CUDA(h, launch_tensor_coef(h->d, h->stream));
  return select_fp32_operator(h);
}

void drop_graphs(osm_ctx* h) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->mp_exec) cudaGraphExecDestroy(h->mp_exec);
  if (h->mp_graph) cudaGraphDestroy(h->mp_graph);
  if (h->ls_exec) cudaGraphExecDestroy(h->ls_exec);
  if (h->ls_graph) cudaGraphDestroy(h->ls_graph);
  h->exec = nullptr; h->graph = nullptr;
  h->mp_exec = nullptr; h->mp_graph = nullptr;
  h->ls_exec = nullptr; h->ls_graph = nullptr;
}

// The FP32 inner solve runs the tensor-product operator when it was chosen
// and every transmission coefficient q is zero (the tensor form folds p M_G
// only); otherwise the SELL matrix.  A change of layout rebuilds the solve
// graphs (they hold the kernel arguments) and clears the FP32 vectors, whose
// rows mean different nodes in the two layouts.
osm_status select_fp32_operator(osm_ctx* h) {
  bool q_zero = true;
  for (size_t s = 0; s < h->tc_host.size() / 4; ++s)
    if (h->tc_host[4 * s + 1] != 0.0 || h->tc_host[4 * s + 3] != 0.0) q_zero = false;
  const int want = (h->have_box && h->fp32_tuned == 2 && q_zero) ? 1 : 0;
  const int want_init = want ? h->init_tuned : 0;
  if (want == h->d.t32 && want_init == h->d.t64i) return OSM_OK;
  const bool layout_change = want != h->d.t32;
  const bool mirror = want_init && !h->d.t64i;
  h->d.t32 = want;
  h->d.t64i = want_init;
  if (mirror) OSM_CUDA(h, launch_box_mirror(h->d, h->stream));   // ub from the current iterate
  h->d.sub_init0 = want_init ? h->d.sub_cta0 : h->d.sub_tile0;
  drop_graphs(h);
  if (!layout_change) return OSM_OK;
  const size_t n32 = std::max<size_t>((size_t)h->hp.vec_rows, (size_t)h->hp.box_rows);
  for (float* v : {h->d.x32, h->d.r32, h->d.z32, h->d.p32, h->d.q32})
    OSM_CUDA(h, cudaMemsetAsync(v, 0, sizeof(float) * n32, h->stream));
  return OSM_OK;
}

// Zeroth-order symmetric Robin condition with parameter p_sub[s] in
// subdomain s (tc = (p, 0, p, 0)).
void set_oo0(osm_ctx* h, const std::vector<double>& p_sub) {
  h->psub_host = p_sub;
  h->tc_host.assign(4 * p_sub.size(), 0.0);
  for (size_t s = 0; s < p_sub.size(); ++s) {
    h->tc_host[4 * s + 0] = p_sub[s];
    h->tc_host[4 * s + 2] = p_sub[s];
  }
  h->tc_general = false;
}

osm_status mp_alloc(osm_ctx* h) {
  if (h->mp_ready) return OSM_OK;
  const HostProblem& hp = h->hp;
  DevSample& m = h->mp;
  const size_t W = kSampleWidth, nv = hp.vec_rows, ns = hp.nsub;
  for (double** v : {&m.x, &m.r, &m.z, &m.pd, &m.q, &m.b, &m.w, &m.y}) OSM_CUDA(h, dalloc(h, v, nv * W));
  OSM_CUDA(h, dalloc(h, &m.lam, 2 * (size_t)hp.n_fent * W));
  for (double** v : {&m.part0, &m.part1, &m.part2}) OSM_CUDA(h, dalloc(h, v, hp.n_tiles * W));
  for (double** v : {&m.rho, &m.alpha, &m.beta, &m.bb, &m.rr}) OSM_CUDA(h, dalloc(h, v, ns * W));
  OSM_CUDA(h, dalloc(h, &m.sc, ns * W));
  OSM_CUDA(h, dalloc(h, &m.isc2, ns * W));
  for (int32_t** v : {&m.active, &m.iters}) OSM_CUDA(h, dalloc(h, v, ns * W));
  OSM_CUDA(h, dalloc(h, &m.psamp, W));
  OSM_CUDA(h, dalloc(h, &m.done, W));
  OSM_CUDA(h, dalloc(h, &m.outer_iters, W));
  OSM_CUDA(h, dalloc(h, &m.relres, W));
  OSM_CUDA(h, dalloc(h, &m.rpart, (size_t)kNodeBlocks * W));
  OSM_CUDA(h, dalloc(h, &m.rpart2, (size_t)kNodeBlocks * W));
  if (h->opts.prec == OSM_MIXED)
    for (float** v : {&m.x32, &m.r32, &m.z32, &m.pd32, &m.q32}) OSM_CUDA(h, dalloc(h, v, nv * W));
  std::vector<int32_t> row_irow(nv, -1);
  for (size_t k = 0; k < hp.irow.size(); ++k) row_irow[hp.irow[k]] = (int32_t)k;
  int32_t* ri;
  OSM_CUDA(h, upload(h, &ri, row_irow));
  m.row_irow = ri;
  h->mp_ready = true;
  return OSM_OK;
}

osm_status run_iterations(osm_ctx* h, double rtol, int max_outer);
osm_status reset_state(osm_ctx* h);

osm_status adj_alloc(osm_ctx* h) {
  if (h->adj_ready) return OSM_OK;
  const HostProblem& hp = h->hp;
  DevAdjoint& a = h->adj;
  double *xc, *yc, *zc;
  OSM_CUDA(h, upload(h, &xc, hp.xc));
  OSM_CUDA(h, upload(h, &yc, hp.yc));
  OSM_CUDA(h, upload(h, &zc, hp.zc));
  a.xc = xc; a.yc = yc; a.zc = zc;
  a.nx = hp.nx; a.ny = hp.ny; a.nz = hp.nz; a.NX = hp.NX; a.NY = hp.NY; a.NZ = hp.NZ;
  std::vector<int32_t> box(6 * hp.nsub);
  for (int s = 0; s < hp.nsub; ++s) {
    const SubInfo& S = hp.sub[s];
    int32_t* b = &box[6 * s];
    b[0] = S.ex0; b[1] = S.ex1; b[2] = S.ey0; b[3] = S.ey1; b[4] = S.ez0; b[5] = S.ez1;
  }
  int32_t *sb, *rn;
  OSM_CUDA(h, upload(h, &sb, box));
  a.sub_box = sb;
  std::vector<int32_t> row_node(hp.vec_rows, -1);
  for (int64_t n = 0; n < hp.n_nodes; ++n)
    for (int32_t c = hp.cp_ptr[n]; c < hp.cp_ptr[n + 1]; ++c) row_node[hp.cp_idx[c]] = (int32_t)n;
  OSM_CUDA(h, upload(h, &rn, row_node));
  a.row_node = rn;
  OSM_CUDA(h, dalloc(h, &a.jpart, kNodeBlocks));
  OSM_CUDA(h, dalloc(h, &a.f_save, hp.vec_rows));
  OSM_CUDA(h, dalloc(h, &a.v_nodes, hp.n_nodes));
  OSM_CUDA(h, dalloc(h, &h->J_dev, 1));
  h->adj_ready = true;
  return OSM_OK;
}

// Adjoint solve K w = v (v nodal, device) and dL/d drho = 4 pi G F^T w into
// grad; the handle's load is restored afterwards.
osm_status adjoint_solve(osm_ctx* h, double rtol, const double* v_nodes, double* grad, int32_t* iters,
                         double* relres) {
  DevAdjoint& a = h->adj;
  const size_t nv = h->hp.vec_rows;
  OSM_CUDA(h, cudaMemcpyAsync(a.f_save, h->d.f, sizeof(double) * nv, cudaMemcpyDeviceToDevice, h->stream));
  OSM_CUDA(h, launch_nodal_load(h->d, a, v_nodes, h->stream));
  osm_status st = reset_state(h);
  if (st == OSM_OK) st = run_iterations(h, rtol, h->opts.max_outer);
  cudaError_t e = cudaSuccess;
  if (st == OSM_OK) e = launch_density_gradient(h->d, a, h->d.phi, grad, h->stream);
  // restore the density load (b = f off the interface rows)
  cudaError_t e2 = cudaMemcpyAsync(h->d.f, a.f_save, sizeof(double) * nv, cudaMemcpyDeviceToDevice, h->stream);
  if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(h->d.b, a.f_save, sizeof(double) * nv, cudaMemcpyDeviceToDevice, h->stream);
  if (st != OSM_OK) return st;
  OSM_CUDA(h, e);
  OSM_CUDA(h, e2);
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (iters) *iters = h->ctl_host->n_outer;
  if (relres) *relres = h->ctl_host->relres;
  return OSM_OK;
}

// Q2 Lagrange basis on [0,1] (nodes 0, 1/2, 1) and its derivative.
static void lagrange_q2(double s, double* L, double* dL) {
  L[0] = (1.0 - s) * (1.0 - 2.0 * s);
  L[1] = 4.0 * s * (1.0 - s);
  L[2] = s * (2.0 * s - 1.0);
  dL[0] = 4.0 * s - 3.0;
  dL[1] = 4.0 - 8.0 * s;
  dL[2] = 4.0 * s - 1.0;
}

// element index containing coordinate v (the last element for v = c[n])
static int locate(const std::vector<double>& c, double v) {
  const int n = (int)c.size() - 1;
  int e = (int)(std::upper_bound(c.begin(), c.end(), v) - c.begin()) - 1;
  return std::min(std::max(e, 0), n - 1);
}

osm_status build_mp_graph(osm_ctx* h) {
  if (h->mp_exec) return OSM_OK;
  cudaStream_t cs = h->cap_stream;
  cudaGraph_t g = nullptr;
  OSM_CUDA(h, cudaGraphCreate(&g, 0));
  h->mp_graph = g;
  cudaGraphConditionalHandle c_out, c_in;
  OSM_CUDA(h, cudaGraphConditionalHandleCreate(&c_out, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams po{};
  po.type = cudaGraphNodeTypeConditional;
  po.conditional.handle = c_out;
  po.conditional.type = cudaGraphCondTypeWhile;
  po.conditional.size = 1;
  cudaGraphNode_t n_out;
  OSM_CUDA(h, cudaGraphAddNode(&n_out, g, nullptr, nullptr, 0, &po));
  cudaGraph_t body = po.conditional.phGraph_out[0];
  OSM_CUDA(h, cudaGraphConditionalHandleCreate(&c_in, body, 0, 0));
  OSM_CUDA(h, cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const int mixed = h->opts.prec == OSM_MIXED, refine = h->opts.prec != OSM_FP64;
  cudaError_t e = launch_mp_rhs_init(h->d, h->mp, cs, c_in, 1, mixed, refine);
  cudaGraphNodeParams pi{};
  cudaGraphNode_t n_in = nullptr;
  if (e == cudaSuccess) {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (e == cudaSuccess) {
      pi.type = cudaGraphNodeTypeConditional;
      pi.conditional.handle = c_in;
      pi.conditional.type = cudaGraphCondTypeWhile;
      pi.conditional.size = 1;
      e = cudaGraphAddNode(&n_in, body, deps, nullptr, ndeps, &pi);
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &n_in, nullptr, 1, cudaStreamSetCaptureDependencies);
  }
  if (e == cudaSuccess) e = launch_mp_exchange_residual(h->d, h->mp, cs, c_out, 1, mixed);
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
  OSM_CUDA(h, e);
  OSM_CUDA(h, e2);
  cudaGraph_t ibody = pi.conditional.phGraph_out[0];
  OSM_CUDA(h, cudaStreamBeginCaptureToGraph(cs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  e = launch_mp_cg_iteration(h->d, h->mp, cs, c_in, 1, mixed);
  e2 = cudaStreamEndCapture(cs, &captured);
  OSM_CUDA(h, e);
  OSM_CUDA(h, e2);
  OSM_CUDA(h, cudaGraphInstantiate(&h->mp_exec, g, 0));
  return OSM_OK;
}

// Autotuner: times the CG step's SpMV-bearing kernel of each precision, in
// every variant, on this handle's own matrices and keeps the fastest:
//  FP64: k_cg_spmv<double> with one or two SELL slices per warp and 32- or
//        (if stored) 16-bit column indices;
//  FP32 (mixed): k_cg_spmv_dir32 in the same four variants and, when the
//        handle's boxes fit it, the tensor-product kernel.
// 16-bit columns cut the bytes, but unpacking them costs integer issue slots,
// which the FP64 SpMV (near the FP64 FMA limit) may not have to spare.  The
// kernels run in the profiling state (every subdomain active) on the
// handle's current vectors (zero at setup); the variant chosen for the CG
// step also serves the CG start and the stop test of that precision.
osm_status autotune_spmv(osm_ctx* h) {
  const int fixed = h->opts.autotune == 2 ? 2 : 1;
  const int have16 = h->d.cols16 != nullptr;
  const bool mixed = h->opts.prec == OSM_MIXED;
  h->d.rpl64 = fixed;
  h->d.rpl32 = mixed ? fixed : 0;
  h->d.c16_64 = have16;
  h->d.c16_32 = have16 && mixed;
  h->fp32_tuned = (mixed && h->have_box && h->opts.fp32_operator == 2) ? 2 : 1;
  h->init_tuned = (mixed && h->have_box && h->opts.fp64_start >= 2) ? h->opts.fp64_start - 1 : 0;
  if (h->opts.autotune != 1) return select_fp32_operator(h);
  h->d.t32 = 0;   // the SELL variants first (vectors are zero: no layout to clear)
  OSM_CUDA(h, launch_profile_state(h->d, h->stream));
  cudaEvent_t e0, e1;
  OSM_CUDA(h, cudaEventCreate(&e0));
  OSM_CUDA(h, cudaEventCreate(&e1));
  cudaError_t e = cudaSuccess;
  auto time_kernel = [&](int fp32, double* out) {
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = launch_cg_spmv_alone(h->d, fp32, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = launch_cg_spmv_alone(h->d, fp32, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    *out = ms / 5.0;
  };
  double best_sell32 = 1e300;
  for (int prec = 0; prec < (mixed ? 2 : 1) && e == cudaSuccess; ++prec) {
    int best_rpl = 1, best_c16 = 0;
    double best_ms = 1e300;
    int32_t& rpl_ref = prec == 0 ? h->d.rpl64 : h->d.rpl32;
    int32_t& c16_ref = prec == 0 ? h->d.c16_64 : h->d.c16_32;
    for (int c16 = 0; c16 <= have16 && e == cudaSuccess; ++c16)
      for (int rpl = 1; rpl <= 2 && e == cudaSuccess; ++rpl) {
        rpl_ref = rpl;
        c16_ref = c16;
        double ms = 0.0;
        time_kernel(prec, &ms);
        h->tune_ms[prec][2 * c16 + rpl - 1] = ms;
        if (ms < best_ms) {
          best_ms = ms;
          best_rpl = rpl;
          best_c16 = c16;
        }
      }
    rpl_ref = best_rpl;
    c16_ref = best_c16;
    if (prec == 1) best_sell32 = best_ms;
  }
  if (e == cudaSuccess && mixed && h->have_box) {
    // the tensor kernel with every z-chunk length, timed with every subdomain
    // active and with one in kTailStride (the tail of an inner solve, where a
    // CTA's march along z, not the work, sets the time); the smallest sum
    // stays
    h->d.t32 = 1;
    int best_zc = h->zchunk;
    double best_t = 1e300, best_sum = 1e300;
    for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
      e = set_zchunk(h, kZChunks[c]);
      if (e == cudaSuccess) time_kernel(1, &h->tune_zchunk_ms[c]);
      if (e == cudaSuccess) e = launch_profile_state(h->d, h->stream, kTailStride);
      if (e == cudaSuccess) time_kernel(1, &h->tune_zchunk_tail_ms[c]);
      if (e == cudaSuccess) e = launch_profile_state(h->d, h->stream);
      const double sum = h->tune_zchunk_ms[c] + h->tune_zchunk_tail_ms[c];
      if (sum < best_sum) {
        best_sum = sum;
        best_t = h->tune_zchunk_ms[c];
        best_zc = kZChunks[c];
      }
    }
    if (h->opts.tensor_zchunk > 0) best_zc = h->opts.tensor_zchunk;   // forced (timings still reported)
    if (e == cudaSuccess) e = set_zchunk(h, best_zc);
    h->tune_tensor_ms = best_t;
    // the mixed refinement step's start: SELL SpMV, FP64 or double-float
    // tensor kernel (the partial tables follow the kernel); the fastest serves
    // whenever the tensor layout is in use
    for (int t = 0; t < 3 && e == cudaSuccess; ++t) {
      h->d.t64i = t;
      h->d.sub_init0 = t ? h->d.sub_cta0 : h->d.sub_tile0;
      for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = launch_cg_start(h->d, h->stream, 1);
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
      for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = launch_cg_start(h->d, h->stream, 1);
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      h->tune_init_ms[t] = ms / 5.0;
    }
    if (h->opts.fp64_start > 0) {
      h->init_tuned = h->opts.fp64_start - 1;
    } else {
      h->init_tuned = 0;
      for (int t = 1; t < 3; ++t)
        if (h->tune_init_ms[t] < h->tune_init_ms[h->init_tuned]) h->init_tuned = t;
    }
    h->d.t64i = 0;
    h->d.sub_init0 = h->d.sub_tile0;
    h->d.t32 = 0;
    if (e == cudaSuccess && h->opts.fp32_operator == 0 && best_t < best_sell32) h->fp32_tuned = 2;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  OSM_CUDA(h, e);
  // the tensor kernel's profiling run wrote its layout's p, q: start clean
  if (h->have_box) {
    const size_t n32 = std::max<size_t>((size_t)h->hp.vec_rows, (size_t)h->hp.box_rows);
    for (float* v : {h->d.p32, h->d.q32}) OSM_CUDA(h, cudaMemsetAsync(v, 0, sizeof(float) * n32, h->stream));
  }
  return select_fp32_operator(h);
}

// Graph of the subdomain solves alone (x = A_i^-1 b_i from the current x):
// CG start, then the device-side CG loop.
osm_status build_lsolve_graph(osm_ctx* h) {
  if (h->ls_exec) return OSM_OK;
  cudaStream_t cs = h->cap_stream;
  OSM_CUDA(h, cudaGraphCreate(&h->ls_graph, 0));
  cudaGraphConditionalHandle c_in;
  OSM_CUDA(h, cudaGraphConditionalHandleCreate(&c_in, h->ls_graph, 0, 0));
  OSM_CUDA(h, cudaStreamBeginCaptureToGraph(cs, h->ls_graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_cg_init(h->d, cs, c_in, 1, 0);
  cudaGraphNodeParams pi{};
  cudaGraphNode_t n_in = nullptr;
  if (e == cudaSuccess) {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (e == cudaSuccess) {
      pi.type = cudaGraphNodeTypeConditional;
      pi.conditional.handle = c_in;
      pi.conditional.type = cudaGraphCondTypeWhile;
      pi.conditional.size = 1;
      e = cudaGraphAddNode(&n_in, h->ls_graph, deps, nullptr, ndeps, &pi);
    }
  }
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
  OSM_CUDA(h, e);
  OSM_CUDA(h, e2);
  OSM_CUDA(h, cudaStreamBeginCaptureToGraph(cs, pi.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
  e = launch_cg_iteration(h->d, cs, c_in, 1);
  e2 = cudaStreamEndCapture(cs, &captured);
  OSM_CUDA(h, e);
  OSM_CUDA(h, e2);
  OSM_CUDA(h, cudaGraphInstantiate(&h->ls_exec, h->ls_graph, 0));
  return OSM_OK;
}

// Adds a conditional WHILE node after the work captured so far on cs (whose
// capture target is `graph`) and makes it the capture's only dependency.
cudaError_t add_while_after_capture(cudaStream_t cs, cudaGraph_t graph, cudaGraphConditionalHandle c,
                                    cudaGraphNodeParams* p, cudaGraphNode_t* node) {
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  *p = cudaGraphNodeParams{};
  p->type = cudaGraphNodeTypeConditional;
  p->conditional.handle = c;
  p->conditional.type = cudaGraphCondTypeWhile;
  p->conditional.size = 1;
  e = cudaGraphAddNode(node, graph, deps, nullptr, ndeps, p);
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, node, nullptr, 1, cudaStreamSetCaptureDependencies);
  return e;
}

// The solve graph:
//   RHS gather, CG start                                  (first iteration)
//   while (running) {                                      // Schwarz iteration
//     CG finaliser; while (any subdomain active) CG step   // subdomain solves
//     [u += e]; Robin exchange                             // Sec. 3
//     RHS gather, CG start of the next iteration (r = b - A u, y = A u)
//     stop test on y: K ubar = y - T u + K (ubar - u)      // Sec. 6
//   }
// The next iteration's CG start comes before the stop test so that its
// product A u serves the stop test too: one SpMV over the FP64 matrices per
// Schwarz iteration instead of two.
osm_status build_graph(osm_ctx* h) {
  if (h->exec) return OSM_OK;
  cudaStream_t cs = h->cap_stream;
  cudaGraph_t g = nullptr;
  OSM_CUDA(h, cudaGraphCreate(&g, 0));
  h->graph = g;
  const bool mixed = h->opts.prec == OSM_MIXED;
  const int refine = h->opts.prec == OSM_FP64_REFINE;
  cudaGraphConditionalHandle c_out, c_in;
  OSM_CUDA(h, cudaGraphConditionalHandleCreate(&c_out, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams po{}, pi{};
  cudaGraphNode_t n_out = nullptr, n_in = nullptr;
  cudaGraph_t captured = nullptr;
  // first iteration's RHS and CG start, then the outer loop
  OSM_CUDA(h, cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_rhs_gather(h->d, cs);
  if (e == cudaSuccess) e = launch_cg_start(h->d, cs, mixed);
  if (e == cudaSuccess) e = add_while_after_capture(cs, g, c_out, &po, &n_out);
  cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
  OSM_CUDA(h, e);
  OSM_CUDA(h, e2);
  cudaGraph_t body = po.conditional.phGraph_out[0];
  OSM_CUDA(h, cudaGraphConditionalHandleCreate(&c_in, body, 0, 0));
  // outer body
  OSM_CUDA(h, cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  e = launch_fin_init(h->d, cs, c_in, 1, mixed ? 1 : refine);
  if (e == cudaSuccess) e = add_while_after_capture(cs, body, c_in, &pi, &n_in);
  if (e == cudaSuccess && mixed) e = launch_mixed_correct(h->d, cs);
  if (e == cudaSuccess) e = launch_exchange(h->d, cs);
  if (e == cudaSuccess) e = launch_rhs_gather(h->d, cs);
  if (e == cudaSuccess) e = launch_cg_start(h->d, cs, mixed);
  if (e == cudaSuccess) e = launch_stop_test(h->d, cs, c_out, 1);
  e2 = cudaStreamEndCapture(cs, &captured);
  OSM_CUDA(h, e);
  OSM_CUDA(h, e2);
  // inner body: one CG iteration on every active subdomain
  cudaGraph_t ibody = pi.conditional.phGraph_out[0];
  OSM_CUDA(h, cudaStreamBeginCaptureToGraph(cs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  e = mixed ? launch_cg_iteration32(h->d, cs, c_in, 1) : launch_cg_iteration(h->d, cs, c_in, 1);
  e2 = cudaStreamEndCapture(cs, &captured);
  OSM_CUDA(h, e);
  OSM_CUDA(h, e2);
  OSM_CUDA(h, cudaGraphInstantiate(&h->exec, g, 0));
  return OSM_OK;
}

void ctl_reset(osm_ctx* h, double rtol, int max_outer) {
  DevCtl& c = *h->ctl_host;
  memset(&c, 0, sizeof(c));
  c.rtol = rtol;
  const bool mixed = h->opts.prec != OSM_FP64;  // OSM_MIXED and OSM_FP64_REFINE
  c.tau2 = mixed ? h->opts.mixed_inner_rtol * h->opts.mixed_inner_rtol : h->opts.inner_rtol * h->opts.inner_rtol;
  c.tau2_outer = h->opts.inner_rtol * h->opts.inner_rtol;
  c.max_outer = max_outer;
  c.max_inner = h->opts.max_inner;
  c.relres = INFINITY;
  c.t_start_ns = 0ull;
  c.t_limit_ns = (unsigned long long)h->opts.max_seconds * 1000000000ull;
}

// Stop tolerances below which a solve that would start its refinement steps
// with the double-float tensor kernel uses the FP64 one instead: the
// double-float defect's rounding (about 2^-48 |A| |u| per row, 1e-11 to 1e-10
// of ||f|| on these meshes) would blur a tighter stop test.
constexpr double kDfStartMinRtol = 1e-9;

// Run Schwarz iterations until relres <= rtol or max_outer iterations.
osm_status run_iterations(osm_ctx* h, double rtol, int max_outer) {
  if (h->opts.prec == OSM_MIXED && h->d.t32) {
    const int start = (h->init_tuned == 2 && rtol > 0.0 && rtol < kDfStartMinRtol) ? 1 : h->init_tuned;
    if (start != h->d.t64i) {   // both box mirrors are kept current: only the graphs change
      h->d.t64i = start;
      drop_graphs(h);
    }
  }
  ctl_reset(h, rtol, max_outer);
  h->ctl_host->running = h->hp.n_inst;
  OSM_CUDA(h, cudaMemsetAsync(h->d.inst_done, 0, sizeof(int32_t) * h->hp.n_inst, h->stream));
  OSM_CUDA(h, cudaMemsetAsync(h->d.inst_iters, 0, sizeof(int32_t) * h->hp.n_inst, h->stream));
  OSM_CUDA(h, cudaMemsetAsync(h->d.st.tsteps, 0, sizeof(int32_t) * h->hp.nsub, h->stream));
  OSM_CUDA(h, cudaMemsetAsync(h->d.inst_relres, 0, sizeof(double) * h->hp.n_inst, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(h->d.ctl, h->ctl_host, sizeof(DevCtl), cudaMemcpyHostToDevice, h->stream));
  OSM_CUDA(h, launch_load_nodes(h->d, h->stream));
  if (h->opts.use_graph) {
    osm_status st = build_graph(h);
    if (st != OSM_OK) return st;
    OSM_CUDA(h, cudaGraphLaunch(h->exec, h->stream));
  } else {
    // the same launch sequence as the graph (build_graph), driven from the host
    const bool mixed = h->opts.prec == OSM_MIXED;
    OSM_CUDA(h, launch_rhs_gather(h->d, h->stream));
    OSM_CUDA(h, launch_cg_start(h->d, h->stream, mixed));
    for (int n = 0; n < max_outer; ++n) {
      OSM_CUDA(h, launch_fin_init(h->d, h->stream, 0, 0, mixed ? 1 : h->opts.prec == OSM_FP64_REFINE));
      for (int it = 0; it <= h->opts.max_inner; ++it) {
        OSM_CUDA(h, cudaMemcpyAsync(h->ctl_host, h->d.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
        OSM_CUDA(h, cudaStreamSynchronize(h->stream));
        if (h->ctl_host->n_active == 0 || h->ctl_host->stop) break;
        OSM_CUDA(h, mixed ? launch_cg_iteration32(h->d, h->stream, 0, 0) : launch_cg_iteration(h->d, h->stream, 0, 0));
      }
      if (mixed) OSM_CUDA(h, launch_mixed_correct(h->d, h->stream));
      OSM_CUDA(h, launch_exchange(h->d, h->stream));
      OSM_CUDA(h, launch_rhs_gather(h->d, h->stream));
      OSM_CUDA(h, launch_cg_start(h->d, h->stream, mixed));
      OSM_CUDA(h, launch_stop_test(h->d, h->stream, 0, 0));
      OSM_CUDA(h, cudaMemcpyAsync(h->ctl_host, h->d.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
      OSM_CUDA(h, cudaStreamSynchronize(h->stream));
      if (h->ctl_host->running == 0 || h->ctl_host->stop) break;
    }
  }
  OSM_CUDA(h, launch_phi(h->d, h->stream));   // phi = ubar of the final iterate of every instance
  OSM_CUDA(h, cudaMemcpyAsync(h->ctl_host, h->d.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

// One batch of at most kSampleWidth candidates; the SELL values must hold K.
osm_status run_sample_batch(osm_ctx* h, int nb, const double* p, double rtol, int max_outer, int race,
                            int32_t* iters, double* relres) {
  const int W = kSampleWidth;
  DevSample& m = h->mp;
  std::vector<double> ps(W, 1.0), rel(W, INFINITY);
  std::vector<int32_t> done(W, 1), it(W, 0);
  for (int k = 0; k < nb; ++k) { ps[k] = p[k]; done[k] = 0; }
  OSM_CUDA(h, cudaMemcpyAsync(m.psamp, ps.data(), sizeof(double) * W, cudaMemcpyHostToDevice, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(m.done, done.data(), sizeof(int32_t) * W, cudaMemcpyHostToDevice, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(m.outer_iters, it.data(), sizeof(int32_t) * W, cudaMemcpyHostToDevice, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(m.relres, rel.data(), sizeof(double) * W, cudaMemcpyHostToDevice, h->stream));
  OSM_CUDA(h, cudaMemsetAsync(m.x, 0, sizeof(double) * h->hp.vec_rows * W, h->stream));
  if (h->hp.n_fent) OSM_CUDA(h, cudaMemsetAsync(m.lam, 0, sizeof(double) * 2 * h->hp.n_fent * W, h->stream));
  OSM_CUDA(h, launch_mp_start(h->d, m, h->stream));
  ctl_reset(h, rtol, max_outer);  // the candidates run the handle's precision mode
  h->ctl_host->race = race;
  const int mixed = h->opts.prec == OSM_MIXED, refine = h->opts.prec != OSM_FP64;
  OSM_CUDA(h, cudaMemcpyAsync(h->d.ctl, h->ctl_host, sizeof(DevCtl), cudaMemcpyHostToDevice, h->stream));
  if (h->opts.use_graph) {
    osm_status st = build_mp_graph(h);
    if (st != OSM_OK) return st;
    OSM_CUDA(h, cudaGraphLaunch(h->mp_exec, h->stream));
  } else {
    for (int n = 0; n < max_outer; ++n) {
      OSM_CUDA(h, launch_mp_rhs_init(h->d, m, h->stream, 0, 0, mixed, refine));
      for (int k = 0; k <= h->opts.max_inner; ++k) {
        OSM_CUDA(h, cudaMemcpyAsync(h->ctl_host, h->d.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
        OSM_CUDA(h, cudaStreamSynchronize(h->stream));
        if (h->ctl_host->n_active == 0 || h->ctl_host->stop) break;
        OSM_CUDA(h, launch_mp_cg_iteration(h->d, m, h->stream, 0, 0, mixed));
      }
      OSM_CUDA(h, launch_mp_exchange_residual(h->d, m, h->stream, 0, 0, mixed));
      OSM_CUDA(h, cudaMemcpyAsync(h->ctl_host, h->d.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
      OSM_CUDA(h, cudaStreamSynchronize(h->stream));
      if (h->ctl_host->n_active == 0 || h->ctl_host->stop) break;
    }
  }
  OSM_CUDA(h, cudaMemcpyAsync(it.data(), m.outer_iters, sizeof(int32_t) * W, cudaMemcpyDeviceToHost, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(rel.data(), m.relres, sizeof(double) * W, cudaMemcpyDeviceToHost, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(h->ctl_host, h->d.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k < nb; ++k) {
    iters[k] = it[k];
    relres[k] = rel[k];
  }
  return OSM_OK;
}

osm_status reset_state(osm_ctx* h) {
  OSM_CUDA(h, cudaMemsetAsync(h->d.x, 0, sizeof(double) * h->hp.vec_rows, h->stream));
  if (h->d.ub) OSM_CUDA(h, cudaMemsetAsync(h->d.ub, 0, sizeof(double) * h->hp.box_rows, h->stream));
  if (h->d.ub2) OSM_CUDA(h, cudaMemsetAsync(h->d.ub2, 0, sizeof(float2) * h->hp.box_rows, h->stream));
  if (h->hp.n_fent) OSM_CUDA(h, cudaMemsetAsync(h->d.lam, 0, sizeof(double) * 2 * h->hp.n_fent, h->stream));
  return OSM_OK;
}

}  // namespace

namespace osm {

const DevProblem* handle_problem(osm_handle h, cudaStream_t* stream, int64_t* vec_rows, int* device) {
  if (!h) return nullptr;
  if (stream) *stream = h->stream;
  if (vec_rows) *vec_rows = h->hp.vec_rows;
  if (device) *device = h->device;
  return &h->d;
}

void handle_set_error(osm_handle h, const char* msg) {
  if (h) h->err = msg;
}

}  // namespace osm

extern "C" {

void osm_default_opts(osm_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->prec = OSM_FP64;
  o->inner_rtol = 1e-10;
  o->mixed_inner_rtol = 1e-5;
  o->max_outer = 10000;
  o->max_inner = 20000;
  o->use_graph = 1;
  o->max_seconds = 900;
  o->autotune = 1;
  o->index16 = 1;
}

const char* osm_status_string(osm_status s) {
  switch (s) {
    case OSM_OK: return "ok";
    case OSM_E_ARG: return "invalid argument";
    case OSM_E_CUDA: return "CUDA error";
    case OSM_E_NOMEM: return "out of memory";
    case OSM_E_NOCONV: return "iteration cap reached";
    case OSM_E_BREAKDOWN: return "CG breakdown";
    case OSM_E_STATE: return "invalid state";
    case OSM_E_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* osm_last_error(osm_handle h) { return h ? h->err.c_str() : "null handle"; }

osm_status osm_setup(const osm_mesh* mesh, const double* drho, const osm_decomp* dec, const osm_opts* opts,
                     void* cuda_stream, osm_handle* out) {
  if (!out) return OSM_E_ARG;
  *out = nullptr;
  if (!mesh || !dec || !drho) return OSM_E_ARG;
  osm_ctx* h = new (std::nothrow) osm_ctx();
  if (!h) return OSM_E_NOMEM;
  if (opts) h->opts = *opts; else osm_default_opts(&h->opts);
  if (!(h->opts.inner_rtol > 0.0) || h->opts.max_outer < 1 || h->opts.max_inner < 1 || h->opts.max_seconds < 1 ||
      h->opts.fp32_operator < 0 || h->opts.fp32_operator > 2 || h->opts.fp64_start < 0 || h->opts.fp64_start > 3 ||
      (h->opts.tensor_zchunk != 0 && (h->opts.tensor_zchunk < kZChunks[0] || h->opts.tensor_zchunk > kZChunks[3]))) {
    delete h;
    return OSM_E_ARG;
  }
  h->stream = (cudaStream_t)cuda_stream;
  auto t0 = std::chrono::steady_clock::now();
  if (h->opts.prec != OSM_FP64 && h->opts.prec != OSM_MIXED && h->opts.prec != OSM_FP64_REFINE) {
    delete h;
    return OSM_E_ARG;
  }
  if (h->opts.prec != OSM_FP64 && !(h->opts.mixed_inner_rtol > 0.0 && h->opts.mixed_inner_rtol < 1.0)) {
    delete h;
    return OSM_E_ARG;
  }
  std::string msg = build_host_problem(*mesh, drho, *dec, h->hp, h->opts.prec == OSM_MIXED);
  if (!msg.empty()) {
    *out = h;  // keep the handle so the caller can read the message
    h->err = msg;
    return OSM_E_ARG;
  }
  *out = h;
  OSM_CUDA(h, cudaGetDevice(&h->device));
  OSM_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  osm_status st = upload_problem(h);
  if (st != OSM_OK) return st;
  set_oo0(h, std::vector<double>(h->hp.nsub, 1.0));
  st = apply_robin(h);
  if (st != OSM_OK) return st;
  st = autotune_spmv(h);
  if (st != OSM_OK) return st;
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // host copies of the large arrays are not needed any more (the layer's row
  // list stays: its length counts launches)
  std::vector<int32_t>().swap(h->hp.cols);
  std::vector<double>().swap(h->hp.vals);
  std::vector<float>().swap(h->hp.vals32);
  std::vector<int32_t>().swap(h->hp.li_col);
  std::vector<double>().swap(h->hp.li_val);
  return OSM_OK;
}

osm_status osm_info(osm_handle h, osm_info_t* o) {
  if (!h || !o) return OSM_E_ARG;
  o->n_sub = h->hp.nsub;
  o->n_face = h->hp.nface;
  o->n_nodes = h->hp.n_nodes;
  o->n_dofs = h->hp.n_dofs;
  o->n_local = h->hp.n_local;
  o->n_face_vals = 2 * h->hp.n_fent;
  o->nnz = h->hp.nnz;
  o->sell_entries = h->hp.sell_entries;
  o->n_slices = h->hp.n_slices;
  o->vec_rows = h->hp.vec_rows;
  o->device_bytes = (int64_t)h->dev_bytes;
  o->setup_seconds = h->setup_seconds;
  o->spmv_variant_fp64 = h->d.rpl64;
  o->spmv_variant_fp32 = h->d.rpl32;
  for (int v = 0; v < 2; ++v) {
    o->spmv_ms_fp64[v] = h->tune_ms[0][v];
    o->spmv_ms_fp32[v] = h->tune_ms[1][v];
    o->spmv_ms16_fp64[v] = h->tune_ms[0][2 + v];
    o->spmv_ms16_fp32[v] = h->tune_ms[1][2 + v];
  }
  o->col_bytes_fp64 = h->d.c16_64 ? 2 : 4;
  o->col_bytes_fp32 = h->opts.prec == OSM_MIXED ? (h->d.c16_32 ? 2 : 4) : 0;
  o->fp32_operator = h->opts.prec == OSM_MIXED ? (h->d.t32 ? 2 : 1) : 0;
  o->fp32_operator_tuned = h->opts.prec == OSM_MIXED ? h->fp32_tuned : 0;
  o->tensor_ms_fp32 = h->tune_tensor_ms;
  o->tensor_zchunk = h->have_box ? h->zchunk : 0;
  o->fp64_start = h->opts.prec == OSM_MIXED ? (h->d.t32 ? h->init_tuned : 0) + 1 : 0;
  for (int t = 0; t < 3; ++t) o->start_ms[t] = h->tune_init_ms[t];
  for (int c = 0; c < 4; ++c) o->tensor_ms_zchunk[c] = h->tune_zchunk_ms[c];
  for (int c = 0; c < 4; ++c) o->tensor_ms_zchunk_tail[c] = h->tune_zchunk_tail_ms[c];
  o->box_rows = h->have_box ? h->hp.box_rows : 0;
  return OSM_OK;
}

osm_status osm_set_density(osm_handle h, const double* drho) {
  if (!h || !drho) return OSM_E_ARG;
  if (h->hp.n_inst > 1) return fail(h, OSM_E_STATE, "osm_set_density needs a single-problem handle");
  for (int64_t e = 0; e < (int64_t)h->hp.nx * h->hp.ny * h->hp.nz; ++e)
    if (!std::isfinite(drho[e])) return fail(h, OSM_E_ARG, "density must be finite");
  build_load(h->hp, drho, h->hp.f);
  OSM_CUDA(h, cudaMemcpyAsync(h->d.f, h->hp.f.data(), sizeof(double) * h->hp.vec_rows, cudaMemcpyHostToDevice, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(h->d.b, h->hp.f.data(), sizeof(double) * h->hp.vec_rows, cudaMemcpyHostToDevice, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

osm_status osm_set_robin(osm_handle h, double p) {
  if (!h) return OSM_E_ARG;
  if (!(p > 0.0) || !std::isfinite(p)) return fail(h, OSM_E_ARG, "Robin parameter must be positive and finite");
  set_oo0(h, std::vector<double>(h->hp.nsub, p));
  return apply_robin(h);
}

osm_status osm_set_transmission(osm_handle h, double p_lo, double q_lo, double p_hi, double q_hi) {
  if (!h) return OSM_E_ARG;
  for (double p : {p_lo, p_hi})
    if (!(p > 0.0) || !std::isfinite(p)) return fail(h, OSM_E_ARG, "transmission p must be positive and finite");
  for (double q : {q_lo, q_hi})
    if (!(q >= 0.0) || !std::isfinite(q)) return fail(h, OSM_E_ARG, "transmission q must be >= 0 and finite");
  const int ns = h->hp.nsub;
  h->tc_host.resize(4 * (size_t)ns);
  for (int s = 0; s < ns; ++s) {
    h->tc_host[4 * s + 0] = p_lo;
    h->tc_host[4 * s + 1] = q_lo;
    h->tc_host[4 * s + 2] = p_hi;
    h->tc_host[4 * s + 3] = q_hi;
  }
  // psub is read only by the zeroth-order symmetric paths (osm_grad_p checks tc_general)
  h->psub_host.assign(ns, p_lo);
  h->tc_general = !(q_lo == 0.0 && q_hi == 0.0 && p_lo == p_hi);
  return apply_robin(h);
}

osm_status osm_set_robin_sub(osm_handle h, const double* p_sub) {
  if (!h || !p_sub) return OSM_E_ARG;
  for (int s = 0; s < h->hp.nsub; ++s)
    if (!(p_sub[s] > 0.0) || !std::isfinite(p_sub[s]))
      return fail(h, OSM_E_ARG, "Robin parameters must be positive and finite");
  set_oo0(h, std::vector<double>(p_sub, p_sub + h->hp.nsub));
  return apply_robin(h);
}

static osm_status finish_status(osm_ctx* h, bool stop_test, double rtol) {
  const DevCtl& c = *h->ctl_host;
  if (c.status & 4) return fail(h, OSM_E_TIMEOUT, "solve exceeded opts.max_seconds; stopped on the device");
  if (c.status & 2) return fail(h, OSM_E_BREAKDOWN, "CG breakdown in a subdomain solve");
  if (stop_test && !(c.relres <= rtol)) return fail(h, OSM_E_NOCONV, "Schwarz iteration cap reached");
  if (c.status & 1) {
    h->err = "a subdomain CG reached max_inner";
  }
  return OSM_OK;
}

osm_status osm_solve(osm_handle h, double rtol, double* phi, int32_t* iters, double* relres) {
  if (!h) return OSM_E_ARG;
  if (!(rtol > 0.0)) return fail(h, OSM_E_ARG, "rtol must be positive");
  h->err.clear();
  osm_status st = reset_state(h);
  if (st != OSM_OK) return st;
  h->last_kind = 0;
  st = run_iterations(h, rtol, h->opts.max_outer);
  if (st != OSM_OK) return st;
  if (phi) {
    OSM_CUDA(h, cudaMemcpyAsync(phi, h->d.phi, sizeof(double) * h->hp.n_nodes, cudaMemcpyDeviceToDevice, h->stream));
    OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  if (iters) *iters = h->ctl_host->n_outer;
  if (relres) *relres = h->ctl_host->relres;
  return finish_status(h, true, rtol);
}

osm_status osm_setup_batch(int32_t n_inst, const osm_mesh* meshes, const double* const* drho, const osm_decomp* decs,
                           const osm_opts* opts, void* cuda_stream, osm_handle* out) {
  if (!out) return OSM_E_ARG;
  *out = nullptr;
  if (n_inst < 1 || !meshes || !drho || !decs) return OSM_E_ARG;
  osm_ctx* h = new (std::nothrow) osm_ctx();
  if (!h) return OSM_E_NOMEM;
  if (opts) h->opts = *opts; else osm_default_opts(&h->opts);
  *out = h;
  if (!(h->opts.inner_rtol > 0.0) || h->opts.max_outer < 1 || h->opts.max_inner < 1 || h->opts.max_seconds < 1 ||
      (h->opts.prec != OSM_FP64 && h->opts.prec != OSM_MIXED && h->opts.prec != OSM_FP64_REFINE) ||
      (h->opts.prec != OSM_FP64 && !(h->opts.mixed_inner_rtol > 0.0 && h->opts.mixed_inner_rtol < 1.0)) ||
      h->opts.fp32_operator < 0 || h->opts.fp32_operator > 2 || h->opts.fp64_start < 0 || h->opts.fp64_start > 3 ||
      (h->opts.tensor_zchunk != 0 && (h->opts.tensor_zchunk < kZChunks[0] || h->opts.tensor_zchunk > kZChunks[3])))
    return fail(h, OSM_E_ARG, "osm_setup_batch: bad options");
  h->stream = (cudaStream_t)cuda_stream;
  auto t0 = std::chrono::steady_clock::now();
  std::vector<HostProblem> parts(n_inst);
  std::string msg;
  for (int32_t i = 0; i < n_inst && msg.empty(); ++i) {
    if (!drho[i]) msg = "null density";
    else msg = build_host_problem(meshes[i], drho[i], decs[i], parts[i], h->opts.prec == OSM_MIXED);
    if (!msg.empty()) msg = "instance " + std::to_string(i) + ": " + msg;
  }
  if (msg.empty()) msg = merge_problems(parts, h->hp);
  if (!msg.empty()) return fail(h, OSM_E_ARG, msg);
  OSM_CUDA(h, cudaGetDevice(&h->device));
  OSM_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  osm_status st = upload_problem(h);
  if (st != OSM_OK) return st;
  set_oo0(h, std::vector<double>(h->hp.nsub, 1.0));
  st = apply_robin(h);
  if (st != OSM_OK) return st;
  st = autotune_spmv(h);
  if (st != OSM_OK) return st;
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  std::vector<int32_t>().swap(h->hp.cols);
  std::vector<double>().swap(h->hp.vals);
  std::vector<float>().swap(h->hp.vals32);
  std::vector<int32_t>().swap(h->hp.li_col);
  std::vector<double>().swap(h->hp.li_val);
  return OSM_OK;
}

osm_status osm_batch_info(osm_handle h, int32_t* n_inst, int64_t* node_offsets) {
  if (!h || !n_inst) return OSM_E_ARG;
  *n_inst = h->hp.n_inst;
  if (node_offsets)
    for (int i = 0; i <= h->hp.n_inst; ++i) node_offsets[i] = h->hp.inst_node0[i];
  return OSM_OK;
}

osm_status osm_set_robin_inst(osm_handle h, const double* p_inst) {
  if (!h || !p_inst) return OSM_E_ARG;
  for (int i = 0; i < h->hp.n_inst; ++i)
    if (!(p_inst[i] > 0.0) || !std::isfinite(p_inst[i]))
      return fail(h, OSM_E_ARG, "Robin parameters must be positive and finite");
  std::vector<double> ps(h->hp.nsub);
  for (int s = 0; s < h->hp.nsub; ++s) ps[s] = p_inst[h->hp.sub_inst[s]];
  set_oo0(h, ps);
  return apply_robin(h);
}

osm_status osm_solve_batch(osm_handle h, double rtol, double* phi, int32_t* iters, double* relres) {
  if (!h) return OSM_E_ARG;
  if (!(rtol > 0.0)) return fail(h, OSM_E_ARG, "rtol must be positive");
  h->err.clear();
  osm_status st = reset_state(h);
  if (st != OSM_OK) return st;
  h->last_kind = 0;
  st = run_iterations(h, rtol, h->opts.max_outer);
  if (st != OSM_OK) return st;
  const int n = h->hp.n_inst;
  std::vector<int32_t> it(n);
  std::vector<double> rel(n);
  OSM_CUDA(h, cudaMemcpyAsync(it.data(), h->d.inst_iters, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(rel.data(), h->d.inst_relres, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  if (phi)
    OSM_CUDA(h, cudaMemcpyAsync(phi, h->d.phi, sizeof(double) * h->hp.n_nodes, cudaMemcpyDeviceToDevice, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  bool all = true;
  for (int i = 0; i < n; ++i) {
    if (iters) iters[i] = it[i];
    if (relres) relres[i] = rel[i];
    all = all && rel[i] <= rtol;
  }
  const DevCtl& c = *h->ctl_host;
  if (c.status & 4) return fail(h, OSM_E_TIMEOUT, "solve exceeded opts.max_seconds; stopped on the device");
  if (c.status & 2) return fail(h, OSM_E_BREAKDOWN, "CG breakdown in a subdomain solve");
  if (!all) return fail(h, OSM_E_NOCONV, "an instance reached max_outer");
  return OSM_OK;
}

osm_status osm_reset(osm_handle h) {
  if (!h) return OSM_E_ARG;
  osm_status st = reset_state(h);
  if (st != OSM_OK) return st;
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

osm_status osm_iterate(osm_handle h, int32_t n, double* hist) {
  if (!h) return OSM_E_ARG;
  if (n < 0 || n > h->opts.max_outer) return fail(h, OSM_E_ARG, "n must be in [0, max_outer]");
  if (n == 0) return OSM_OK;
  h->err.clear();
  h->last_kind = 0;
  osm_status st = run_iterations(h, -1.0, n);
  if (st != OSM_OK) return st;
  if (hist) OSM_CUDA(h, cudaMemcpy(hist, h->d.hist, sizeof(double) * n, cudaMemcpyDeviceToHost));
  return finish_status(h, false, 0.0);
}

osm_status osm_apply(osm_handle h, int32_t op, const double* x, double* y) {
  if (!h || !x || !y || op < 0 || op > 2) return OSM_E_ARG;
  if (op == 2) {
    if (h->opts.prec != OSM_MIXED) return fail(h, OSM_E_STATE, "op 2 needs a handle set up with OSM_MIXED");
    OSM_CUDA(h, launch_apply32(h->d, x, y, h->stream));
    OSM_CUDA(h, cudaStreamSynchronize(h->stream));
    return OSM_OK;
  }
  OSM_CUDA(h, launch_apply(h->d, op, x, y, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

osm_status osm_get_local(osm_handle h, double* u) {
  if (!h || !u) return OSM_E_ARG;
  OSM_CUDA(h, launch_gather_local(h->d, h->d.x, u, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

osm_status osm_get_lambda(osm_handle h, double* lam) {
  if (!h || !lam) return OSM_E_ARG;
  if (h->hp.n_fent)
    OSM_CUDA(h, cudaMemcpyAsync(lam, h->d.lam, sizeof(double) * 2 * h->hp.n_fent, cudaMemcpyDeviceToDevice, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

osm_status osm_set_lambda(osm_handle h, const double* lam) {
  if (!h || !lam) return OSM_E_ARG;
  if (h->hp.n_fent)
    OSM_CUDA(h, cudaMemcpyAsync(h->d.lam, lam, sizeof(double) * 2 * h->hp.n_fent, cudaMemcpyDeviceToDevice, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

osm_status osm_stats(osm_handle h, osm_stats_t* o) {
  if (!h || !o) return OSM_E_ARG;
  const DevCtl& c = *h->ctl_host;
  o->n_outer = c.n_outer;
  o->n_cg_steps = c.total_inner;
  // Kernel launches of the last call, counted from the launch sequence.
  const int mixed = h->opts.prec == OSM_MIXED;
  const int faces = h->hp.n_fent ? 1 : 0;
  if (h->last_kind == 1) {
    // batched p evaluation: per Schwarz iteration RHS gather, CG start, its
    // finaliser, FP64 correction (mixed), exchange (if any face), average,
    // K ubar, residual; per batched CG step SpMM, alpha, update, beta,
    // direction; plus the start of the batch
    const int64_t per_outer = 3 + mixed + faces + 3;
    o->n_launches = 1 + per_outer * c.n_outer + 5 * (int64_t)c.total_inner;
  } else {
    // solve: once the nodal load, the first RHS gather and CG start, and at
    // the end phi; per Schwarz iteration the CG finaliser, FP64 correction
    // (mixed), exchange (if any face), the next RHS gather and CG start,
    // average, interface layer (if any; on the tensor form the transmission
    // correction and the FP32 tensor kernel), residual partials of the
    // interface nodes and of the single-copy rows, residual finaliser; per CG
    // step SpMV (+ direction epilogue in FP32) and update (+ the step's
    // finish), plus the FP64 direction
    const int64_t layer = h->d.dl32 ? 1 + (h->hp.irow.empty() ? 0 : 1) : (h->hp.li_row.empty() ? 0 : 1);
    const int64_t per_outer = 1 + mixed + faces + 2 + 1 + layer + 3;
    o->n_launches = 4 + per_outer * c.n_outer + (mixed ? 2 : 3) * (int64_t)c.total_inner;
  }
  o->relres = c.relres;
  o->status = c.status;
  o->reserved = 0;
  // rows the CG-step kernels processed: each subdomain's CG steps times its
  // local unknowns, and times the rows its CG-step kernels sweep (the box
  // layout's tiles on the FP32 tensor-product form, the padded SELL rows
  // otherwise)
  o->sub_row_steps = 0;
  o->op_row_steps = 0;
  if (h->last_kind == 0) {
    const int ns = h->hp.nsub;
    std::vector<int32_t> steps(ns);
    OSM_CUDA(h, cudaMemcpy(steps.data(), h->d.st.tsteps, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost));
    const bool box = h->opts.prec == OSM_MIXED && h->d.t32;
    for (int s = 0; s < ns; ++s) {
      const SubInfo& S = h->hp.sub[s];
      const int64_t op = box ? (h->hp.box_sub_tile0[s + 1] - h->hp.box_sub_tile0[s]) * kTileRows : S.npad;
      o->sub_row_steps += (int64_t)steps[s] * S.n;
      o->op_row_steps += (int64_t)steps[s] * op;
    }
  }
  return OSM_OK;
}

osm_status osm_inner_iters(osm_handle h, int32_t* iters) {
  if (!h || !iters) return OSM_E_ARG;
  OSM_CUDA(h, cudaMemcpy(iters, h->d.st.iters, sizeof(int32_t) * h->hp.nsub, cudaMemcpyDeviceToHost));
  return OSM_OK;
}

osm_status osm_sample_p(osm_handle h, int32_t n_p, const double* p_host, double rtol, int32_t max_outer,
                        int32_t* iters_host, double* relres_host, int32_t* best_idx) {
  return osm_sample_p_ex(h, n_p, p_host, rtol, max_outer, 0, iters_host, relres_host, best_idx);
}

osm_status osm_sample_p_ex(osm_handle h, int32_t n_p, const double* p_host, double rtol, int32_t max_outer,
                           int32_t flags, int32_t* iters_host, double* relres_host, int32_t* best_idx) {
  if (!h) return OSM_E_ARG;
  if (flags & ~OSM_SAMPLE_RACE) return fail(h, OSM_E_ARG, "osm_sample_p_ex: unknown flags");
  const int race = (flags & OSM_SAMPLE_RACE) != 0;
  if (h->hp.n_inst > 1) return fail(h, OSM_E_STATE, "osm_sample_p needs a single-problem handle");
  if (n_p < 1 || !p_host || !iters_host || !relres_host || !best_idx || !(rtol > 0.0) || max_outer < 1)
    return fail(h, OSM_E_ARG, "osm_sample_p: bad arguments");
  for (int32_t k = 0; k < n_p; ++k)
    if (!(p_host[k] > 0.0) || !std::isfinite(p_host[k]))
      return fail(h, OSM_E_ARG, "osm_sample_p: every p must be positive and finite");
  h->err.clear();
  osm_status st = mp_alloc(h);
  if (st != OSM_OK) return st;
  // the batched run needs the plain stiffness K_i in the SELL values
  OSM_CUDA(h, cudaMemsetAsync(h->d.psub, 0, sizeof(double) * h->hp.nsub, h->stream));
  OSM_CUDA(h, cudaMemsetAsync(h->d.tc, 0, sizeof(double) * 4 * h->hp.nsub, h->stream));
  OSM_CUDA(h, launch_set_robin(h->d, h->stream));
  // candidates run in order of p (a candidate's run does not depend on its
  // batch companions): lanes of similar p finish their CG at similar steps,
  // so the lanes still running share cache sectors of the candidate rows
  std::vector<int32_t> order(n_p);
  for (int32_t k = 0; k < n_p; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return p_host[a] < p_host[b]; });
  std::vector<double> ps(n_p), rel_s(n_p);
  std::vector<int32_t> it_s(n_p);
  for (int32_t k = 0; k < n_p; ++k) ps[k] = p_host[order[k]];
  int status_or = 0;
  int cap = max_outer;   // race: later batches cannot beat the best count so far
  for (int32_t b0 = 0; b0 < n_p && st == OSM_OK; b0 += kSampleWidth) {
    const int nb = std::min<int32_t>(kSampleWidth, n_p - b0);
    st = run_sample_batch(h, nb, ps.data() + b0, rtol, cap, race, it_s.data() + b0, rel_s.data() + b0);
    status_or |= h->ctl_host->status;
    if (race)
      for (int k = b0; k < b0 + nb; ++k)
        if (rel_s[k] <= rtol) cap = std::min<int>(cap, it_s[k]);
  }
  for (int32_t k = 0; k < n_p; ++k) {
    iters_host[order[k]] = it_s[k];
    relres_host[order[k]] = rel_s[k];
  }
  h->last_kind = 1;
  osm_status st2 = apply_robin(h);  // back to the handle's own p
  if (st != OSM_OK) return st;
  if (st2 != OSM_OK) return st2;
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  int best = -1;
  for (int32_t k = 0; k < n_p; ++k) {
    if (!(relres_host[k] <= rtol)) continue;
    if (best < 0 || iters_host[k] < iters_host[best] ||
        (iters_host[k] == iters_host[best] &&
         (relres_host[k] < relres_host[best] || (relres_host[k] == relres_host[best] && p_host[k] < p_host[best]))))
      best = k;
  }
  *best_idx = best;
  if (status_or & 4) return fail(h, OSM_E_TIMEOUT, "osm_sample_p exceeded opts.max_seconds");
  if (status_or & 2) return fail(h, OSM_E_BREAKDOWN, "CG breakdown in a candidate's subdomain solve");
  if (best < 0) return fail(h, OSM_E_NOCONV, "no candidate reached rtol within max_outer");
  return OSM_OK;
}

osm_status osm_log_uniform_p(uint64_t seed, int32_t n, double lo, double hi, double* p_host) {
  if (n < 0 || !p_host || !(lo > 0.0) || !(hi >= lo)) return OSM_E_ARG;
  uint64_t state = seed;
  const double llo = std::log(lo), lhi = std::log(hi);
  for (int32_t i = 0; i < n; ++i) {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const double u = (double)(z >> 11) * 0x1.0p-53;
    p_host[i] = std::exp(llo + u * (lhi - llo));
  }
  return OSM_OK;
}

osm_status osm_set_density_dev(osm_handle h, const double* drho) {
  if (!h || !drho) return OSM_E_ARG;
  if (h->hp.n_inst > 1) return fail(h, OSM_E_STATE, "osm_set_density_dev needs a single-problem handle");
  osm_status st = adj_alloc(h);
  if (st != OSM_OK) return st;
  OSM_CUDA(h, launch_load_from_density(h->d, h->adj, drho, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

osm_status osm_set_stations(osm_handle h, int32_t n_st, const double* xyz) {
  if (!h || n_st < 1 || !xyz) return OSM_E_ARG;
  if (h->hp.n_inst > 1) return fail(h, OSM_E_STATE, "osm_set_stations needs a single-problem handle");
  const HostProblem& hp = h->hp;
  std::vector<int32_t> node(27 * (size_t)n_st);
  std::vector<double> w(27 * (size_t)n_st);
  for (int32_t st = 0; st < n_st; ++st) {
    const double x = xyz[3 * st], y = xyz[3 * st + 1], z = xyz[3 * st + 2];
    if (!(x >= hp.xc.front() && x <= hp.xc.back() && y >= hp.yc.front() && y <= hp.yc.back() &&
          z >= hp.zc.front() && z <= hp.zc.back()))
      return fail(h, OSM_E_ARG, "osm_set_stations: a station lies outside the mesh");
    const int ex = locate(hp.xc, x), ey = locate(hp.yc, y), ez = locate(hp.zc, z);
    const double hx = hp.xc[ex + 1] - hp.xc[ex], hy = hp.yc[ey + 1] - hp.yc[ey], hz = hp.zc[ez + 1] - hp.zc[ez];
    double Lx[3], dLx[3], Ly[3], dLy[3], Lz[3], dLz[3];
    lagrange_q2((x - hp.xc[ex]) / hx, Lx, dLx);
    lagrange_q2((y - hp.yc[ey]) / hy, Ly, dLy);
    lagrange_q2((z - hp.zc[ez]) / hz, Lz, dLz);
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          const int q = a + 3 * b + 9 * c;
          node[27 * (size_t)st + q] = (2 * ex + a) + hp.NX * ((2 * ey + b) + hp.NY * (2 * ez + c));
          w[27 * (size_t)st + q] = Lx[a] * Ly[b] * dLz[c] / hz;
        }
  }
  osm_status s2 = adj_alloc(h);
  if (s2 != OSM_OK) return s2;
  DevAdjoint& a = h->adj;
  if (a.n_st != n_st) {
    int32_t* sn;
    double* sw;
    OSM_CUDA(h, upload(h, &sn, node));
    OSM_CUDA(h, upload(h, &sw, w));
    a.st_node = sn;
    a.st_w = sw;
    OSM_CUDA(h, dalloc(h, &a.g, n_st));
    OSM_CUDA(h, dalloc(h, &a.res, n_st));
    a.n_st = n_st;
  } else {
    OSM_CUDA(h, cudaMemcpyAsync((void*)a.st_node, node.data(), sizeof(int32_t) * node.size(), cudaMemcpyHostToDevice,
                                h->stream));
    OSM_CUDA(h, cudaMemcpyAsync((void*)a.st_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, h->stream));
  }
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

osm_status osm_gravity(osm_handle h, const double* phi, double* g) {
  if (!h || !phi || !g) return OSM_E_ARG;
  if (!h->adj_ready || h->adj.n_st == 0) return fail(h, OSM_E_STATE, "osm_gravity: call osm_set_stations first");
  OSM_CUDA(h, launch_station_values(h->d, h->adj, phi, nullptr, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(g, h->adj.g, sizeof(double) * h->adj.n_st, cudaMemcpyDeviceToDevice, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

osm_status osm_potential_vjp(osm_handle h, double rtol, const double* v, double* grad) {
  if (!h || !v || !grad || !(rtol > 0.0)) return OSM_E_ARG;
  if (h->hp.n_inst > 1) return fail(h, OSM_E_STATE, "osm_potential_vjp needs a single-problem handle");
  h->err.clear();
  osm_status st = adj_alloc(h);
  if (st != OSM_OK) return st;
  h->last_kind = 0;
  st = adjoint_solve(h, rtol, v, grad, nullptr, nullptr);
  if (st != OSM_OK) return st;
  return finish_status(h, true, rtol);
}

osm_status osm_grad(osm_handle h, double rtol, const double* g_obs, double* J, double* dJ_drho, double* dJ_dp) {
  if (!h || !g_obs || !J || !dJ_drho || !(rtol > 0.0)) return OSM_E_ARG;
  if (!h->adj_ready || h->adj.n_st == 0) return fail(h, OSM_E_STATE, "osm_grad: call osm_set_stations first");
  h->err.clear();
  h->last_kind = 0;
  // forward solve
  osm_status st = reset_state(h);
  if (st == OSM_OK) st = run_iterations(h, rtol, h->opts.max_outer);
  if (st != OSM_OK) return st;
  st = finish_status(h, true, rtol);
  if (st != OSM_OK) return st;
  // misfit and its nodal adjoint load
  DevAdjoint& a = h->adj;
  OSM_CUDA(h, launch_station_values(h->d, a, h->d.phi, g_obs, h->stream));
  OSM_CUDA(h, launch_misfit(a, h->J_dev, h->stream));
  OSM_CUDA(h, launch_stations_transpose(h->d, a, h->stream));
  OSM_CUDA(h, cudaMemcpyAsync(J, h->J_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  // adjoint Schwarz solve and the density gradient
  st = adjoint_solve(h, rtol, a.v_nodes, dJ_drho, nullptr, nullptr);
  if (st != OSM_OK) return st;
  // the converged discrete solution does not depend on p (the Schwarz fixed
  // point is the Galerkin solution for every p > 0)
  if (dJ_dp) *dJ_dp = 0.0;
  return finish_status(h, true, rtol);
}

osm_status osm_grad_p(osm_handle h, int32_t n_iter, const double* g_obs, double* J, double* dJ_dp) {
  if (!h || n_iter < 1 || !g_obs || !J || !dJ_dp) return OSM_E_ARG;
  if (h->hp.n_inst > 1) return fail(h, OSM_E_STATE, "osm_grad_p needs a single-problem handle");
  if (h->opts.prec != OSM_FP64) return fail(h, OSM_E_STATE, "osm_grad_p needs an OSM_FP64 handle");
  if (!h->adj_ready || h->adj.n_st == 0) return fail(h, OSM_E_STATE, "osm_grad_p: call osm_set_stations first");
  if (n_iter > h->opts.max_outer) return fail(h, OSM_E_ARG, "osm_grad_p: n_iter exceeds max_outer");
  if (h->tc_general) return fail(h, OSM_E_STATE, "osm_grad_p needs the zeroth-order symmetric Robin condition");
  for (double q : h->psub_host)
    if (q != h->psub_host[0]) return fail(h, OSM_E_STATE, "osm_grad_p needs one Robin parameter for all subdomains");
  h->err.clear();
  const double p = h->psub_host[0];
  const size_t nv = h->hp.vec_rows, nl = 2 * (size_t)(h->hp.n_fent ? h->hp.n_fent : 1);
  if (!h->ilam_partner) {
    std::vector<int32_t> partner_of(nl, 0);
    for (int f = 0; f < h->hp.nface; ++f) {
      const int64_t eo = h->hp.face_eo[f];
      const int32_t nf = h->hp.face_n[f];
      for (int32_t m = 0; m < nf; ++m) {
        partner_of[2 * eo + m] = (int32_t)(2 * eo + nf + m);
        partner_of[2 * eo + nf + m] = (int32_t)(2 * eo + m);
      }
    }
    std::vector<int32_t> partner(h->hp.ilam.size());
    for (size_t e = 0; e < partner.size(); ++e) partner[e] = partner_of[h->hp.ilam[e]];
    OSM_CUDA(h, upload(h, &h->ilam_partner, partner));
  }
  osm_status st = build_lsolve_graph(h);
  if (st != OSM_OK) return st;
  // temporaries of this call
  double *uhist = nullptr, *lam_a = nullptr, *lam_b = nullptr, *mu = nullptr, *ub = nullptr, *part = nullptr,
         *dps = nullptr;
  const int64_t nparts = (h->hp.n_fent + (int64_t)h->hp.irow.size() + 255) / 256 + 1;
  auto cleanup = [&]() {
    for (double* q : {uhist, lam_a, lam_b, mu, ub, part, dps}) if (q) cudaFree(q);
  };
  cudaError_t e = cudaMalloc((void**)&uhist, sizeof(double) * nv * (size_t)n_iter);
  if (e == cudaSuccess) e = cudaMalloc((void**)&lam_a, sizeof(double) * nl);
  if (e == cudaSuccess) e = cudaMalloc((void**)&lam_b, sizeof(double) * nl);
  if (e == cudaSuccess) e = cudaMalloc((void**)&mu, sizeof(double) * nl);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ub, sizeof(double) * nv);
  if (e == cudaSuccess) e = cudaMalloc((void**)&part, sizeof(double) * nparts);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dps, sizeof(double) * n_iter);
  if (e != cudaSuccess) {
    cleanup();
    return fail(h, e == cudaErrorMemoryAllocation ? OSM_E_NOMEM : OSM_E_CUDA, cudaGetErrorString(e));
  }
  // forward: exactly n_iter Schwarz iterations from zero, keeping every iterate
  h->last_kind = 0;
  st = reset_state(h);
  for (int n = 0; n < n_iter && st == OSM_OK; ++n) {
    st = run_iterations(h, -1.0, 1);
    if (st == OSM_OK && (h->ctl_host->status & 6)) st = fail(h, OSM_E_BREAKDOWN, "forward Schwarz iteration failed");
    if (st == OSM_OK) {
      e = cudaMemcpyAsync(uhist + (size_t)n * nv, h->d.x, sizeof(double) * nv, cudaMemcpyDeviceToDevice, h->stream);
      if (e != cudaSuccess) st = fail(h, OSM_E_CUDA, cudaGetErrorString(e));
    }
  }
  // misfit of the averaged last iterate and ubar^N = S^T B^T r
  DevAdjoint& a = h->adj;
  if (st == OSM_OK) {
    e = launch_station_values(h->d, a, h->d.phi, g_obs, h->stream);
    if (e == cudaSuccess) e = launch_misfit(a, h->J_dev, h->stream);
    if (e == cudaSuccess) e = launch_stations_transpose(h->d, a, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(J, h->J_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ub, 0, sizeof(double) * nv, h->stream);
    if (e == cudaSuccess) e = launch_nodal_split(h->d, a.v_nodes, ub, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(lam_a, 0, sizeof(double) * nl, h->stream);
    if (e != cudaSuccess) st = fail(h, OSM_E_CUDA, cudaGetErrorString(e));
  }
  // backward sweep (bstatus: loop status of every adjoint local solve)
  std::vector<int32_t> bstatus(n_iter, 0);
  for (int n = n_iter - 1; n >= 0 && st == OSM_OK; --n) {
    const double* un = uhist + (size_t)n * nv;
    if (n < n_iter - 1) e = launch_exchange_adjoint(h->d, h->ilam_partner, lam_a, mu, 2.0 * p, ub, h->stream);
    // bbar^n = A^-1 ubar^n
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d.b, ub, sizeof(double) * nv, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d.x, 0, sizeof(double) * nv, h->stream);
    // the tensor starts read u from its box-layout mirrors: zero them too
    if (e == cudaSuccess && h->d.ub) e = cudaMemsetAsync(h->d.ub, 0, sizeof(double) * h->hp.box_rows, h->stream);
    if (e == cudaSuccess && h->d.ub2) e = cudaMemsetAsync(h->d.ub2, 0, sizeof(float2) * h->hp.box_rows, h->stream);
    if (e != cudaSuccess) { st = fail(h, OSM_E_CUDA, cudaGetErrorString(e)); break; }
    ctl_reset(h, -1.0, 1);
    OSM_CUDA(h, cudaMemcpyAsync(h->d.ctl, h->ctl_host, sizeof(DevCtl), cudaMemcpyHostToDevice, h->stream));
    // the forward pass left the instance marked done; the subdomain solves must run
    OSM_CUDA(h, cudaMemsetAsync(h->d.inst_done, 0, sizeof(int32_t) * h->hp.n_inst, h->stream));
    e = cudaGraphLaunch(h->ls_exec, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&bstatus[n], &h->d.ctl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = launch_dp_terms(h->d, lam_a, un, h->d.x, part, dps + n, h->stream);
    if (e == cudaSuccess) e = launch_lambar_step(h->d, h->d.x, lam_a, lam_b, h->stream);
    if (e != cudaSuccess) { st = fail(h, OSM_E_CUDA, cudaGetErrorString(e)); break; }
    std::swap(lam_a, lam_b);
  }
  std::vector<double> terms(n_iter, 0.0);
  if (st == OSM_OK) {
    e = cudaMemcpyAsync(terms.data(), dps, sizeof(double) * n_iter, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->ctl_host, h->d.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) st = fail(h, OSM_E_CUDA, cudaGetErrorString(e));
    int any = 0;
    for (int32_t b : bstatus) any |= b;
    if (st == OSM_OK && (any & 4)) st = fail(h, OSM_E_TIMEOUT, "osm_grad_p: adjoint solves exceeded opts.max_seconds");
    if (st == OSM_OK && (any & 2)) st = fail(h, OSM_E_BREAKDOWN, "osm_grad_p: CG breakdown in an adjoint solve");
  }
  // restore the handle: b = f off the interface, zero iterates
  cudaMemcpyAsync(h->d.b, h->d.f, sizeof(double) * nv, cudaMemcpyDeviceToDevice, h->stream);
  osm_status st2 = reset_state(h);
  cudaStreamSynchronize(h->stream);
  cleanup();
  if (st != OSM_OK) return st;
  if (st2 != OSM_OK) return st2;
  double sum = 0.0;
  for (int n = 0; n < n_iter; ++n) sum += terms[n];
  *dJ_dp = sum;
  return OSM_OK;
}

// Local system of one subdomain unpacked from the SELL arrays plus the
// transmission entries: p * M (tc == nullptr) or the split form with tc.
static osm_status host_local_system(const osm_mesh* mesh, const double* drho, const osm_decomp* dec, double p,
                                    const double* tc, int32_t sub, int64_t* n, int64_t* nnz, int64_t* rowptr,
                                    int32_t* col, double* val, double* f) {
  if (!mesh || !drho || !dec || !n || !nnz) return OSM_E_ARG;
  HostProblem hp;
  if (!build_host_problem(*mesh, drho, *dec, hp).empty()) return OSM_E_ARG;
  if (sub < 0 || sub >= hp.nsub) return OSM_E_ARG;
  const SubInfo& S = hp.sub[sub];
  // vector row -> canonical index of this subdomain
  std::vector<int32_t> v2c(S.npad, -1);
  for (int32_t q = 0; q < S.n; ++q) v2c[hp.can2vec[S.canon_off + q] - S.voff] = q;
  std::vector<std::vector<std::pair<int32_t, double>>> rows(S.n);
  for (int32_t r = 0; r < S.n; ++r) {
    const int64_t sl = S.slice0 + r / kSliceRows;
    const int lane = r % kSliceRows;
    const int64_t off = hp.slice_off[sl];
    const int w = (int)((hp.slice_off[sl + 1] - off) / kSliceRows);
    auto& row = rows[v2c[r]];
    for (int j = 0; j < w; ++j) {
      const int32_t c = hp.cols[off + (int64_t)(j / 4) * 128 + lane * 4 + (j % 4)];
      const double v = hp.vals[off + (int64_t)(j / 2) * 64 + lane * 2 + (j % 2)];
      row.push_back({v2c[c], v});
    }
  }
  for (size_t k = 0; k < hp.irow.size(); ++k) {
    if (hp.irow_sub[k] != sub) continue;
    auto& row = rows[v2c[hp.irow[k] - S.voff]];
    for (int32_t e = hp.im_ptr[k]; e < hp.im_ptr[k + 1]; ++e) {
      const double* t = hp.im_tc.data() + 4 * (size_t)e;
      const double a = tc ? tc[0] * t[0] + tc[2] * t[1] + tc[1] * t[2] + tc[3] * t[3] : p * hp.im_val[e];
      row.push_back({v2c[hp.im_col[e] - S.voff], a});
    }
  }
  int64_t total = 0;
  for (auto& row : rows) {  // merge duplicates (padding adds zero to the diagonal)
    std::sort(row.begin(), row.end(),
              [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) { return a.first < b.first; });
    size_t o = 0;
    for (size_t i = 0; i < row.size(); ++i) {
      if (o > 0 && row[o - 1].first == row[i].first) row[o - 1].second += row[i].second;
      else row[o++] = row[i];
    }
    row.resize(o);
    total += (int64_t)o;
  }
  *n = S.n;
  *nnz = total;
  if (!rowptr) return OSM_OK;
  if (!col || !val || !f) return OSM_E_ARG;
  rowptr[0] = 0;
  for (int32_t q = 0; q < S.n; ++q) {
    int64_t o = rowptr[q];
    for (auto& e : rows[q]) { col[o] = e.first; val[o] = e.second; ++o; }
    rowptr[q + 1] = o;
    f[q] = hp.f[hp.can2vec[S.canon_off + q]];
  }
  return OSM_OK;
}

osm_status osm_host_local_system(const osm_mesh* mesh, const double* drho, const osm_decomp* dec, double p,
                                 int32_t sub, int64_t* n, int64_t* nnz, int64_t* rowptr, int32_t* col,
                                 double* val, double* f) {
  return host_local_system(mesh, drho, dec, p, nullptr, sub, n, nnz, rowptr, col, val, f);
}

osm_status osm_host_local_system_tc(const osm_mesh* mesh, const double* drho, const osm_decomp* dec,
                                    const double* tc, int32_t sub, int64_t* n, int64_t* nnz, int64_t* rowptr,
                                    int32_t* col, double* val, double* f) {
  if (!tc) return OSM_E_ARG;
  return host_local_system(mesh, drho, dec, 0.0, tc, sub, n, nnz, rowptr, col, val, f);
}

osm_status osm_host_face_stiffness(const osm_mesh* mesh, const double* drho, const osm_decomp* dec, int32_t face,
                                   double* val) {
  if (!mesh || !drho || !dec || !val) return OSM_E_ARG;
  HostProblem hp;
  if (!build_host_problem(*mesh, drho, *dec, hp).empty()) return OSM_E_ARG;
  if (face < 0 || face >= hp.nface) return OSM_E_ARG;
  const int64_t eo = hp.face_eo[face];
  const int32_t nf = hp.face_n[face];
  for (int32_t k = hp.fm_ptr[eo]; k < hp.fm_ptr[eo + nf]; ++k) val[k - hp.fm_ptr[eo]] = hp.fs_val[k];
  return OSM_OK;
}

osm_status osm_host_face_system(const osm_mesh* mesh, const double* drho, const osm_decomp* dec, int32_t face,
                                int64_t* n, int64_t* nnz, int32_t* node, int64_t* rowptr, int32_t* col,
                                double* val) {
  if (!mesh || !drho || !dec || !n || !nnz) return OSM_E_ARG;
  HostProblem hp;
  if (!build_host_problem(*mesh, drho, *dec, hp).empty()) return OSM_E_ARG;
  if (face < 0 || face >= hp.nface) return OSM_E_ARG;
  const int64_t eo = hp.face_eo[face];
  const int32_t nf = hp.face_n[face];
  *n = nf;
  *nnz = hp.fm_ptr[eo + nf] - hp.fm_ptr[eo];
  if (!rowptr) return OSM_OK;
  if (!node || !col || !val) return OSM_E_ARG;
  // node index from the s-side vector row via the copies map
  std::vector<int32_t> row2node(hp.vec_rows, -1);
  for (int64_t nd = 0; nd < hp.n_nodes; ++nd)
    for (int32_t c = hp.cp_ptr[nd]; c < hp.cp_ptr[nd + 1]; ++c) row2node[hp.cp_idx[c]] = (int32_t)nd;
  rowptr[0] = 0;
  for (int32_t m = 0; m < nf; ++m) {
    node[m] = row2node[hp.fent_row_s[eo + m]];
    int64_t o = rowptr[m];
    for (int32_t k = hp.fm_ptr[eo + m]; k < hp.fm_ptr[eo + m + 1]; ++k) {
      col[o] = (int32_t)(hp.fm_col[k] - eo);
      val[o] = hp.fm_val[k];
      ++o;
    }
    rowptr[m + 1] = o;
  }
  return OSM_OK;
}

osm_status osm_profile_spmv(osm_handle h, int32_t prec, int32_t reps, double* ms) {
  if (!h || !ms || reps < 1 || prec < 0 || prec > 4) return OSM_E_ARG;
  if ((prec == 1 || prec == 2 || prec == 4) && h->opts.prec != OSM_MIXED)
    return fail(h, OSM_E_STATE, "prec 1, 2 and 4 need an OSM_MIXED handle");
  if (prec >= 2) OSM_CUDA(h, launch_profile_state(h->d, h->stream));
  auto launch = [&]() {
    switch (prec) {
      case 0: return launch_spmv_plain(h->d, h->d.w, h->d.y, h->stream);
      case 1: return launch_spmv_plain32(h->d, h->d.z32, h->d.q32, h->stream);
      case 2: return launch_cg_spmv_alone(h->d, 1, h->stream);
      case 4: return launch_cg_start(h->d, h->stream, 1);
      default: return launch_cg_spmv_alone(h->d, 0, h->stream);
    }
  };
  cudaEvent_t e0, e1;
  OSM_CUDA(h, cudaEventCreate(&e0));
  OSM_CUDA(h, cudaEventCreate(&e1));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 20 && e == cudaSuccess; ++i) e = launch();  // bring clocks up
  std::vector<double> trial;
  for (int t = 0; t < 5 && e == cudaSuccess; ++t) {
    e = cudaEventRecord(e0, h->stream);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float tm = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&tm, e0, e1);
    trial.push_back((double)tm / reps);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  OSM_CUDA(h, e);
  std::sort(trial.begin(), trial.end());
  *ms = trial[trial.size() / 2];
  return OSM_OK;
}

void osm_destroy(osm_handle h) {
  if (!h) return;
  drop_graphs(h);
  cudaStreamSynchronize(h->stream);
  for (void* p : h->allocs) cudaFree(p);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

}  // extern "C"
