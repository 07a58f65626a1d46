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
  d.n_tiles = hp.n_tiles;
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
  for (int32_t** v : {&st.active, &st.iters, &st.status}) OSM_CUDA(h, dalloc(h, v, ns));
  for (unsigned** v : {&st.cnt_a, &st.cnt_b, &st.cnt_i}) OSM_CUDA(h, dalloc(h, v, ns));
  for (double** v : {&d.part0, &d.part1, &d.part2}) OSM_CUDA(h, dalloc(h, v, hp.n_tiles));
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
  OSM_CUDA(h, upload(h, &face_s, hp.face_s));
  OSM_CUDA(h, upload(h, &face_t, hp.face_t));
  OSM_CUDA(h, upload(h, &face_n, hp.face_n));
  OSM_CUDA(h, upload(h, &face_eo, hp.face_eo));
  d.fent_face = fent_face; d.fent_row_s = fent_row_s; d.fent_row_t = fent_row_t; d.fm_ptr = fm_ptr;
  d.fm_col = fm_col; d.fm_val = fm_val; d.face_s = face_s; d.face_t = face_t; d.face_n = face_n;
  d.face_eo = face_eo;
  OSM_CUDA(h, dalloc(h, &d.lam, 2 * (size_t)hp.n_fent));
  // copies, outputs, stop test
  d.n_nodes = hp.n_nodes;
  int32_t *cp_ptr, *cp_idx, *can2vec;
  OSM_CUDA(h, upload(h, &cp_ptr, hp.cp_ptr));
  OSM_CUDA(h, upload(h, &cp_idx, hp.cp_idx));
  OSM_CUDA(h, upload(h, &can2vec, hp.can2vec));
  d.cp_ptr = cp_ptr; d.cp_idx = cp_idx; d.can2vec = can2vec;
  d.n_local = hp.n_local;
  OSM_CUDA(h, dalloc(h, &d.phi, hp.n_nodes));
  d.n_rblocks = (hp.n_nodes + 255) / 256;
  OSM_CUDA(h, dalloc(h, &d.rpart, d.n_rblocks));
  OSM_CUDA(h, dalloc(h, &d.rpart2, d.n_rblocks));
  OSM_CUDA(h, dalloc(h, &d.hist, h->opts.max_outer > 0 ? h->opts.max_outer : 1));
  OSM_CUDA(h, dalloc(h, &d.ctl, 1));
  OSM_CUDA(h, cudaMallocHost((void**)&h->ctl_host, sizeof(DevCtl)));
  return OSM_OK;
}

osm_status apply_robin(osm_ctx* h) {
  OSM_CUDA(h, cudaMemcpyAsync(h->d.psub, h->psub_host.data(), sizeof(double) * h->hp.nsub,
                              cudaMemcpyHostToDevice, h->stream));
  OSM_CUDA(h, launch_set_robin(h->d, h->stream));
  return OSM_OK;
}

osm_status build_graph(osm_ctx* h) {
  if (h->exec) return OSM_OK;
  cudaStream_t cs = h->cap_stream;
  cudaGraph_t g = nullptr;
  OSM_CUDA(h, cudaGraphCreate(&g, 0));
  h->graph = g;
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
  // outer body: RHS, CG start, [inner loop], exchange, stop test
  OSM_CUDA(h, cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_rhs_gather(h->d, cs);
  if (e == cudaSuccess) e = launch_cg_init(h->d, cs, c_in, 1);
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
  if (e == cudaSuccess) e = launch_exchange(h->d, cs);
  if (e == cudaSuccess) e = launch_residual(h->d, cs, c_out, 1);
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
  OSM_CUDA(h, e);
  OSM_CUDA(h, e2);
  // inner body: one CG iteration on every active subdomain
  cudaGraph_t ibody = pi.conditional.phGraph_out[0];
  OSM_CUDA(h, cudaStreamBeginCaptureToGraph(cs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  e = launch_cg_iteration(h->d, cs, c_in, 1);
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
  c.tau2 = h->opts.inner_rtol * h->opts.inner_rtol;
  c.max_outer = max_outer;
  c.max_inner = h->opts.max_inner;
  c.relres = INFINITY;
  c.t_start_ns = 0ull;
  c.t_limit_ns = (unsigned long long)h->opts.max_seconds * 1000000000ull;
}

// Run Schwarz iterations until relres <= rtol or max_outer iterations.
osm_status run_iterations(osm_ctx* h, double rtol, int max_outer) {
  ctl_reset(h, rtol, max_outer);
  OSM_CUDA(h, cudaMemcpyAsync(h->d.ctl, h->ctl_host, sizeof(DevCtl), cudaMemcpyHostToDevice, h->stream));
  if (h->opts.use_graph) {
    osm_status st = build_graph(h);
    if (st != OSM_OK) return st;
    OSM_CUDA(h, cudaGraphLaunch(h->exec, h->stream));
  } else {
    for (int n = 0; n < max_outer; ++n) {
      OSM_CUDA(h, launch_rhs_gather(h->d, h->stream));
      OSM_CUDA(h, launch_cg_init(h->d, h->stream, 0, 0));
      for (int it = 0; it <= h->opts.max_inner; ++it) {
        OSM_CUDA(h, cudaMemcpyAsync(h->ctl_host, h->d.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
        OSM_CUDA(h, cudaStreamSynchronize(h->stream));
        if (h->ctl_host->n_active == 0 || h->ctl_host->stop) break;
        OSM_CUDA(h, launch_cg_iteration(h->d, h->stream, 0, 0));
      }
      OSM_CUDA(h, launch_exchange(h->d, h->stream));
      OSM_CUDA(h, launch_residual(h->d, h->stream, 0, 0));
      OSM_CUDA(h, cudaMemcpyAsync(h->ctl_host, h->d.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
      OSM_CUDA(h, cudaStreamSynchronize(h->stream));
      if (!(h->ctl_host->relres > rtol) || !std::isfinite(h->ctl_host->relres) || h->ctl_host->stop) break;
    }
  }
  OSM_CUDA(h, cudaMemcpyAsync(h->ctl_host, h->d.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  return OSM_OK;
}

osm_status reset_state(osm_ctx* h) {
  OSM_CUDA(h, cudaMemsetAsync(h->d.x, 0, sizeof(double) * h->hp.vec_rows, h->stream));
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
  if (!(h->opts.inner_rtol > 0.0) || h->opts.max_outer < 1 || h->opts.max_inner < 1 || h->opts.max_seconds < 1) {
    delete h;
    return OSM_E_ARG;
  }
  h->stream = (cudaStream_t)cuda_stream;
  auto t0 = std::chrono::steady_clock::now();
  std::string msg = build_host_problem(*mesh, drho, *dec, h->hp);
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
  h->psub_host.assign(h->hp.nsub, 1.0);
  st = apply_robin(h);
  if (st != OSM_OK) return st;
  OSM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // host copies of the large arrays are not needed any more
  std::vector<int32_t>().swap(h->hp.cols);
  std::vector<double>().swap(h->hp.vals);
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
  return OSM_OK;
}

osm_status osm_set_density(osm_handle h, const double* drho) {
  if (!h || !drho) return OSM_E_ARG;
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
  h->psub_host.assign(h->hp.nsub, p);
  return apply_robin(h);
}

osm_status osm_set_robin_sub(osm_handle h, const double* p_sub) {
  if (!h || !p_sub) return OSM_E_ARG;
  for (int s = 0; s < h->hp.nsub; ++s)
    if (!(p_sub[s] > 0.0) || !std::isfinite(p_sub[s]))
      return fail(h, OSM_E_ARG, "Robin parameters must be positive and finite");
  h->psub_host.assign(p_sub, p_sub + h->hp.nsub);
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
  osm_status st = run_iterations(h, -1.0, n);
  if (st != OSM_OK) return st;
  if (hist) OSM_CUDA(h, cudaMemcpy(hist, h->d.hist, sizeof(double) * n, cudaMemcpyDeviceToHost));
  return finish_status(h, false, 0.0);
}

osm_status osm_apply(osm_handle h, int32_t op, const double* x, double* y) {
  if (!h || !x || !y || (op != 0 && op != 1)) return OSM_E_ARG;
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
  // per Schwarz iteration: RHS gather, CG start, exchange (if any face),
  // average, SpMV, face correction (if any interface), residual;
  // per batched CG step: SpMV+dot, update, direction
  const int64_t per_outer = 2 + (h->hp.n_fent ? 1 : 0) + 3 + (h->hp.irow.empty() ? 0 : 1);
  o->n_launches = per_outer * c.n_outer + 3 * (int64_t)c.total_inner;
  o->relres = c.relres;
  o->status = c.status;
  o->reserved = 0;
  return OSM_OK;
}

osm_status osm_inner_iters(osm_handle h, int32_t* iters) {
  if (!h || !iters) return OSM_E_ARG;
  OSM_CUDA(h, cudaMemcpy(iters, h->d.st.iters, sizeof(int32_t) * h->hp.nsub, cudaMemcpyDeviceToHost));
  return OSM_OK;
}

osm_status osm_sample_p(osm_handle h, int32_t n_p, const double* p_host, double rtol, int32_t max_outer,
                        int32_t* iters_host, double* relres_host, int32_t* best_idx) {
  (void)n_p; (void)p_host; (void)rtol; (void)max_outer; (void)iters_host; (void)relres_host; (void)best_idx;
  return fail(h, OSM_E_STATE, "osm_sample_p is not available in this build");
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

osm_status osm_host_local_system(const osm_mesh* mesh, const double* drho, const osm_decomp* dec, double p,
                                 int32_t sub, int64_t* n, int64_t* nnz, int64_t* rowptr, int32_t* col,
                                 double* val, double* f) {
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
    for (int32_t e = hp.im_ptr[k]; e < hp.im_ptr[k + 1]; ++e)
      row.push_back({v2c[hp.im_col[e] - S.voff], p * hp.im_val[e]});
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

osm_status osm_profile_spmv(osm_handle h, int32_t reps, double* ms) {
  if (!h || !ms || reps < 1) return OSM_E_ARG;
  cudaEvent_t e0, e1;
  OSM_CUDA(h, cudaEventCreate(&e0));
  OSM_CUDA(h, cudaEventCreate(&e1));
  // x -> y on the residual work vectors (w, y): the solver's iterates are untouched
  cudaError_t e = launch_spmv_plain(h->d, h->d.w, h->d.y, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch_spmv_plain(h->d, h->d.w, h->d.y, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  OSM_CUDA(h, e);
  *ms = (double)t / reps;
  return OSM_OK;
}

void osm_destroy(osm_handle h) {
  if (!h) return;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  cudaStreamSynchronize(h->stream);
  for (void* p : h->allocs) cudaFree(p);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

}  // extern "C"
