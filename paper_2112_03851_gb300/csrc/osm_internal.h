// Internal declarations of libosm: host-side problem description, device
// buffers and kernel launchers.  Not part of the public ABI (include/osm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/osm.h"

namespace osm {

// Rows of one SELL slice (one warp, one lane per row) and rows per CTA tile.
constexpr int kSliceRows = 32;
constexpr int kTileRows = 256;
constexpr int kTileSlices = kTileRows / kSliceRows;
// Tiles per block of the CG update (all of one subdomain): FP32 and FP64.
constexpr int kUpdGroup = 8;
constexpr int kUpdGroup64 = 2;
// Threads of the one-block stop-test finaliser.
constexpr int kResFinThreads = 1024;
// SELL row widths are padded to a multiple of 4 so that every lane can load
// four column indices (int4) and two value pairs (double2) per step.
constexpr int kWidthQuantum = 4;
// Widest subdomain box (nodes along x) the tensor-product kernel stages in
// shared memory; wider handles keep the SELL operator for the FP32 solve.
constexpr int kTensorMaxNx = 128;
// Entries per subdomain of the box table: bnx, bny, bnz, face mask, z-chunk
// length, column blocks, z chunks, unused.
constexpr int kBoxDims = 8;

constexpr double kPi = 3.14159265358979323846;
constexpr double kGravity = 6.672e-11;  // Sec. 2

// ---------------------------------------------------------------- host side

// One subdomain's element box and its place in the device arrays.
struct SubInfo {
  int ex0, ex1, ey0, ey1, ez0, ez1;   // element ranges
  int i0, i1, j0, j1, k0, k1;         // node box (inclusive)
  int32_t n;                          // unknowns
  int32_t npad;                       // rows padded to kTileRows
  int64_t voff;                       // first vector row
  int64_t canon_off;                  // first canonical-layout index
  int64_t tile0;                      // first tile
  int64_t slice0;                     // first slice
  bool iface[6];                      // -x, +x, -y, +y, -z, +z side is an interface
  int32_t band0 = 0;                  // first node of its 1-D bands (x, then y, then z)
  int32_t fmask = 0;                  // bits 0-5: side -x .. +z on the outer (Dirichlet)
                                      // boundary; bits 8-13: side is an interface
};

// Everything the host builds before upload.
struct HostProblem {
  int nx, ny, nz, NX, NY, NZ;
  int sx, sy, sz, nsub;
  std::vector<double> xc, yc, zc;
  std::vector<SubInfo> sub;
  int64_t n_nodes = 0, n_dofs = 0, n_local = 0, vec_rows = 0, n_tiles = 0, n_slices = 0;
  int64_t nnz = 0, sell_entries = 0;

  // SELL-32 storage of K_i (p = 0); slice s holds 32 rows x width w entries
  // at [slice_off[s], slice_off[s+1]), laid out so that lane l of step q
  // reads cols[off + 128 q + 4 l .. +3] and vals[off + 128 q + 4 l .. +3] as
  // two double2 at off + 64 (2q) + 2 l and off + 64 (2q+1) + 2 l.
  std::vector<int64_t> slice_off;
  std::vector<int32_t> cols;          // subdomain-local row index (internal order)
  std::vector<double> vals;
  std::vector<float> vals32;          // FP32 copy in the column (quad) layout, mixed mode only

  std::vector<int32_t> tile_sub;      // tile -> subdomain
  std::vector<int32_t> row_sub;       // not stored on device; per vector row
  std::vector<int32_t> can2vec;       // canonical local index -> vector row
  std::vector<double> f;              // load per vector row
  std::vector<double> kdiag;          // diag(K_i) per vector row
  std::vector<double> dinv0;          // 1 / diag(K_i) (padding rows: 0)

  // Interface rows: rows of subdomain i lying on a face with a neighbour.
  std::vector<int32_t> irow;          // vector row
  std::vector<int32_t> irow_sub;      // its subdomain
  std::vector<double> irow_mdiag;     // diag(M_Gi) on that row
  std::vector<int32_t> ilam_ptr;      // -> lam indices of data received at this row
  std::vector<int32_t> ilam;
  std::vector<int32_t> im_ptr;        // -> entries of M_Gi in this row
  std::vector<int32_t> im_col;        // vector row of the column
  std::vector<double> im_val;         // M_Gi value
  std::vector<int64_t> im_pos;        // position of the entry in the SELL value array
  std::vector<double> im_kval;        // K_i value at that position
  std::vector<int64_t> im_pos32;      // position in the FP32 value array
  // Second-order / unsymmetric transmission: the same entries split by the
  // side of the face (lower: this subdomain has the smaller coordinate along
  // the face normal) into face mass and face tangential stiffness parts.
  std::vector<double> im_tc;          // 4 per entry: M_lo, M_hi, S_lo, S_hi
  std::vector<double> irow_tdiag;     // 4 per interface row: their diagonals

  // Faces (canonical face layout) and their mass matrices.
  int nface = 0;
  std::vector<int32_t> face_s, face_t, face_n;
  std::vector<int64_t> face_eo;       // first face entry (lam offset is 2*eo)
  int64_t n_fent = 0;
  std::vector<int32_t> fent_face;     // entry -> face
  std::vector<int32_t> fent_row_s, fent_row_t;  // vector rows on the two sides
  std::vector<int32_t> fm_ptr;        // face mass CSR over entries
  std::vector<int32_t> fm_col;        // global entry index
  std::vector<double> fm_val;
  std::vector<double> fs_val;         // face tangential stiffness, same CSR

  // Tensor-product form of the subdomain operators (mixed handles): the
  // assembled 1-D Q2 stiffness and mass of every subdomain along x, y and z,
  // 5 band entries per node (neighbours a-2 .. a+2), and the box index
  // (i + bnx (j + bny k), box-local) of every vector row (-1: padding row).
  std::vector<double> band_k, band_m;
  std::vector<int32_t> row_boxidx;
  // Box layout of the FP32 inner solve (build_box_layout): subdomain s's box
  // node (i, j, k) at row box_voff[s] + i + bnx (j + bny k), each subdomain
  // padded to whole 256-row tiles; the tensor kernel runs one CTA per 256
  // (x, y) columns of a box.
  std::vector<int64_t> box_voff;
  std::vector<int32_t> box_dims;      // kBoxDims per subdomain (see kBoxDims)
  std::vector<int32_t> box_tile_sub;
  std::vector<int64_t> box_sub_tile0; // n_sub + 1
  std::vector<int64_t> box_ub_tile0;  // FP32 update blocks (kUpdGroup tiles of one subdomain)
  std::vector<int64_t> box_sub_ub0;   // n_sub + 1: first update block of each subdomain
  std::vector<int32_t> box_cta_sub;
  std::vector<int64_t> box_sub_cta0;  // n_sub + 1
  std::vector<int32_t> row_box;       // vector row -> box row (-1: padding)
  std::vector<int32_t> box_vec;       // box row -> vector row (-1: Dirichlet node or padding)
  int64_t box_rows = 0, box_tiles = 0, box_ctas = 0;
  int32_t box_max_nx = 0;

  // Interface-column layer of the Neumann matrices: for every row of K_i
  // with entries in columns that are interface rows of the same subdomain,
  // those entries (CSR over the rows li_row, ascending).  The stop test forms
  // K_i ubar_i = A_i u_i - T_i u_i + K_i (ubar_i - u_i), and ubar_i - u_i
  // vanishes off the interface rows.
  std::vector<int32_t> li_row, li_ptr, li_col;
  std::vector<double> li_val;
  std::vector<int32_t> li_irow;       // per layer row: its interface-row index, or -1

  // Copies of each node of the full grid (vector rows, subdomain order).
  std::vector<int32_t> cp_ptr;        // n_nodes + 1
  std::vector<int32_t> cp_idx;

  // Independent problems (instances) solved together: instance i owns
  // subdomains [inst_sub0[i], inst_sub0[i+1]) and nodes [inst_node0[i],
  // inst_node0[i+1]) of the concatenated node grids.  A single problem is
  // one instance.
  int n_inst = 1;
  std::vector<int32_t> sub_inst;      // subdomain -> instance
  std::vector<int32_t> inst_sub0;     // n_inst + 1
  std::vector<int64_t> inst_node0;    // n_inst + 1
  // Blocks of the node-wise stop-test kernels: block b covers nodes
  // [rblock_node0[b], rblock_node0[b+1]) of instance rblock_inst[b].
  std::vector<int32_t> rblock_inst;
  std::vector<int64_t> rblock_node0;
  std::vector<int32_t> inst_rblock0;  // n_inst + 1: first residual block of each instance
};

// Concatenate independently built problems into one batched problem.
std::string merge_problems(std::vector<HostProblem>& parts, HostProblem& out);
// Fill the instance / residual-block tables of a single problem.
void single_instance_tables(HostProblem& hp);

// Build everything on the host.  Returns an empty string on success, else
// the reason of the failure.
std::string build_host_problem(const osm_mesh& mesh, const double* drho, const osm_decomp& dec,
                               HostProblem& hp, bool want_fp32 = false);

// Box layout tables of the tensor-product FP32 operator (from sub, band0,
// row_boxidx and tile_sub); the tensor kernel's CTAs split each box's z
// range into chunks of about zchunk planes.
void build_box_layout(HostProblem& hp, int zchunk);
// Only the CTA tables (box_dims chunk entries, box_cta_sub, box_sub_cta0)
// for another z-chunk length.
void box_cta_tables(HostProblem& hp, int zchunk);

// Rebuild the load vector (per vector row) for a new density.
void build_load(const HostProblem& hp, const double* drho, std::vector<double>& f);

// ------------------------------------------------------------- device side

// Per-subdomain CG scalars and status (device arrays of n_sub entries).
struct DevSubState {
  double* rho;      // r.z
  double* alpha;
  double* beta;
  double* bb;       // ||b||^2
  double* rr;       // ||r||^2
  int32_t* active;  // 1 while the subdomain's CG runs
  int32_t* iters;   // CG iterations of the current solve
  int32_t* tsteps;  // CG steps of the subdomain summed over the current call's Schwarz iterations
  int32_t* status;  // 0 ok, 1 cap reached, 2 breakdown
  unsigned* ucnt;   // per-subdomain ticket of the CG update's blocks (reset by the last)
  unsigned* tcnt;   // per-subdomain ticket of the tensor kernel's CTAs (reset by the last)
  double* pq;       // p.q of the current CG step (set by the tensor kernel's last CTA)
  float* sc;        // FP32 inner solve: power of two applied to both factors
                    // of every FP32 dot product (keeps r*r out of underflow)
  double* isc2;     // 1 / sc^2, undoes that scaling on the warp partials
};

// Loop-control block living in device memory.
struct DevCtl {
  double rtol;            // Schwarz stop
  double tau2;            // inner_rtol^2
  int32_t max_outer;
  int32_t max_inner;
  int32_t n_outer;        // Schwarz iterations done
  int32_t n_inner;        // CG iterations of the current subdomain solve
  int32_t n_active;       // subdomains still iterating
  int32_t status;         // OR of subdomain statuses seen in this solve
  int32_t total_inner;    // batched CG steps summed over the Schwarz iterations
  int32_t race;           // batched p evaluation: stop every candidate when the first converges
  double relres;          // last stop-test value
  double tau2_outer;      // mixed mode: FP64 local tolerance^2 that skips a correction
  unsigned long long t_start_ns;  // %globaltimer at the first kernel of the call
  unsigned long long t_limit_ns;  // wall-clock budget of the call
  int32_t stop;           // set once the budget is exhausted: both loops end
  int32_t running;        // instances not yet done after the last stop test
  unsigned gcnt_b;        // global last-block counters
  unsigned gcnt_i;
  unsigned gcnt_r;
  unsigned pad;
};

struct DevProblem {
  // SELL
  const int64_t* slice_off;
  const int32_t* cols;
  const uint16_t* cols16;     // 16-bit copy of cols (subdomains <= 65,536 padded rows), or null
  int32_t c16_64, c16_32;     // 1: the FP64 / FP32 SpMVs read cols16 (chosen by the autotuner)
  const int64_t* ub_tile0;    // first tile of each FP32-update block (kUpdGroup tiles, one subdomain)
  int64_t n_ublocks;
  const int64_t* ub64_tile0;  // ... of each FP64-update block (kUpdGroup64 tiles)
  int64_t n_ublocks64;
  const int64_t* sub_ub0;     // n_sub + 1: first FP32-update block of each subdomain
  const int64_t* sub_ub64_0;  // n_sub + 1: first FP64-update block of each subdomain
  double* vals;
  const int32_t* tile_sub;
  const int64_t* sub_tile0;   // n_sub + 1
  int64_t n_tiles;
  int32_t n_sub;
  int32_t rpl64, rpl32;       // SpMV variant (slices per warp) chosen by the autotuner
  // vectors (vec_rows each)
  double *x, *r, *z, *p, *q, *b, *f, *dinv, *w, *y;
  // per subdomain
  double* psub;
  DevSubState st;
  // per tile partials
  double *part0, *part1, *part2;
  // interface rows
  int32_t n_irow;
  const int32_t *irow, *irow_sub, *ilam_ptr, *ilam, *im_ptr, *im_col;
  const double *irow_mdiag, *im_val, *im_kval;
  const double *im_tc, *irow_tdiag;     // split face terms (HostProblem)
  double* tc;                           // 4 per subdomain: p_lo, q_lo, p_hi, q_hi
  double* im_t;                         // transmission part of each entry (set by k_set_robin)
  const int64_t* im_pos;
  const double* kdiag;
  // faces
  int64_t n_fent;
  const int32_t *fent_face, *fent_row_s, *fent_row_t, *fm_ptr, *fm_col;
  const double* fm_val;
  const double* fs_val;
  const int32_t *face_s, *face_t, *face_n;
  const int64_t* face_eo;
  double* lam;
  // interface-column layer of K_i (HostProblem li_*)
  int32_t n_lrow;
  const int32_t *li_row, *li_ptr, *li_col, *li_irow;
  const double* li_val;
  // copies
  int64_t n_nodes;
  const int32_t *cp_ptr, *cp_idx;
  double* phi;          // internal full-grid output
  double* rpart;        // stop-test partials of ||r||^2 (per residual block)
  double* rpart2;       // ... of ||f||^2 (written once per solve by k_load_nodes)
  double* tpart;        // stop-test partials of ||r||^2 over the single-copy rows, one per tile
  // interface nodes (two or more copies) of every instance in node order, in
  // blocks of up to 256 of one instance: [iblock0[b], iblock0[b+1]) of
  // inodes, instance iblock_inst[b]; inst_iblock0 (n_inst + 1) is each
  // instance's first block.  The per-iteration averaging and the interface
  // part of the residual run over these (rpart: one partial per block).
  const int32_t* inodes;
  const int64_t* iblock0;
  const int32_t *iblock_inst, *inst_iblock0;
  int64_t n_iblocks;
  const uint8_t* row_single;  // 1: the vector row's node has no other copy (subdomain interior)
  const int64_t* inst_tile0;  // n_inst + 1: first tile of each instance
  double* fg;           // assembled load per node (full grid), set per solve
  int64_t n_rblocks;
  double* hist;         // residual history (max_outer)
  // instances
  int32_t n_inst;
  const int32_t *sub_inst, *rblock_inst, *inst_rblock0;
  const int64_t* rblock_node0;
  int32_t* inst_done;   // instance converged (or out of iterations) in this solve
  int32_t* inst_iters;  // Schwarz iterations of each instance
  double* inst_relres;  // last stop-test value of each instance
  // mixed precision (null in FP64 mode)
  float* vals32;
  const int64_t* im_pos32;
  float *x32, *r32, *z32, *p32, *q32, *dinv32;
  // Range table of the p.q partials of the CG step's SpMV kernel (sub_tile0
  // for the SELL kernels; sub_cta0 for the tensor kernel).
  const int64_t* sub_part0;
  // FP32 inner solve on the tensor-product operator in the box layout (t32 =
  // 1; else the FP32 SELL operator in the vector-row layout).  The x32 .. q32
  // vectors then hold box rows, dinv32b is the box-layout Jacobi diagonal.
  int32_t t32;
  const int32_t* row_box;
  const int64_t* box_voff;
  const int32_t* box_dims;
  const int32_t* box_band0;
  const int32_t* box_tile_sub;
  const int64_t* box_sub_tile0;
  const int64_t* box_ub_tile0;
  const int64_t* box_sub_ub0;
  int64_t box_n_tiles, box_n_ublocks, n_cta32;
  const int32_t* cta_sub;
  const int64_t* sub_cta0;
  const double *band_k, *band_m;        // plain 1-D bands (5 per band node)
  float *cK32, *cM32;                   // FP32 bands, stiffness with the Robin terms folded in
  float* dinv32b;
  // tensor-product start of the mixed form's refinement step (only with t32;
  // t64i = 1: FP64 arithmetic, 2: double-float arithmetic): the iterate u
  // mirrored in the box layout (ub; ub2 the same as (hi, lo) float pairs),
  // the vector row of every box row (box_vec, -1: Dirichlet or padding), the
  // bands in FP64 and as float pairs
  int32_t t64i;
  double* ub;
  float2* ub2;
  const int32_t* box_vec;
  double *cK64, *cM64;
  float2 *cKdf, *cMdf;
  // stop test on the tensor form (handles with a box layout): ubar - u in the
  // box layout (FP32, written by k_average) and the plain FP32 stiffness bands
  float *dl32, *cKp32;
  // partial range table of the CG start's ||r||^2, ||b||^2, r.z partials
  // (sub_tile0 for the SELL kernels, sub_cta0 for the tensor start)
  const int64_t* sub_init0;
  DevCtl* ctl;
  const int32_t* can2vec;
  int64_t n_local;
};

// Batched evaluation of Robin parameters (osm_sample_p): up to
// kSampleWidth candidates run as one Schwarz solve.  Every vector holds the
// candidates' values of a row contiguously ([row][kSampleWidth]) so that a
// warp's 32 lanes are the 32 candidates.
constexpr int kSampleWidth = 32;
constexpr int kNodeBlocks = 1024;   // blocks of the node-wise kernels (grid-stride)

struct DevSample {
  double* psamp;                        // [kSampleWidth]
  double *x, *r, *z, *pd, *q, *b, *w, *y;  // [vec_rows][kSampleWidth]
  double* lam;                          // [2 n_fent][kSampleWidth]
  double *part0, *part1, *part2;        // [n_tiles][kSampleWidth]
  double *rho, *alpha, *beta, *bb, *rr; // [n_sub][kSampleWidth]
  float* sc;                            // [n_sub][kSampleWidth]: FP32 dot scale (power of two)
  double* isc2;                         // [n_sub][kSampleWidth]: 1 / sc^2
  int32_t *active, *iters;              // [n_sub][kSampleWidth]
  int32_t* done;                        // [kSampleWidth]
  int32_t* outer_iters;                 // [kSampleWidth]
  double* relres;                       // [kSampleWidth]
  double *rpart, *rpart2;               // [kNodeBlocks][kSampleWidth]
  const int32_t* row_irow;              // [vec_rows]: interface-row index or -1
  // mixed batch (null otherwise): FP32 correction e, r, z, p, q
  float *x32, *r32, *z32, *pd32, *q32;  // [vec_rows][kSampleWidth]
};

// CG vectors of the batched evaluation in one precision.
template <class T>
struct MpVec {
  T *x, *r, *z, *pd, *q;
};

// Adjoint gradient data (osm_adjoint.cu): device copies of the mesh and the
// subdomain element boxes, the row -> node map, and the station operator B
// (one row per station: 27 node ids and weights of d/dz of the Q2
// interpolant of the station's element).
struct DevAdjoint {
  const double *xc, *yc, *zc;
  int32_t nx, ny, nz, NX, NY, NZ;
  const int32_t* sub_box;     // [n_sub][6]: ex0, ex1, ey0, ey1, ez0, ez1
  const int32_t* row_node;    // [vec_rows]: full-grid node or -1
  int32_t n_st;
  const int32_t* st_node;     // [n_st][27]
  const double* st_w;         // [n_st][27]
  double *g, *res;            // [n_st]: B phi, B phi - g_obs
  double* jpart;              // [kNodeBlocks]
  double* f_save;             // [vec_rows]: the density load while an adjoint load is in place
  double* v_nodes;            // [n_nodes]: nodal adjoint load
};

// CG vectors of one precision.
template <class T>
struct CgVec {
  T *x, *r, *z, *p, *q;
  const T* dinv;
  const T* vals;
};

// Kernel launchers (osm_kernels.cu).  All enqueue on `s` and return the
// launch error.  `cond` / `use_cond` name the graph conditional to drive.
cudaError_t launch_set_robin(const DevProblem& d, cudaStream_t s);
cudaError_t launch_rhs_gather(const DevProblem& d, cudaStream_t s);
cudaError_t launch_cg_init(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond,
                           int defect_norm = 0);
cudaError_t launch_cg_iteration(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond);
// The CG-step SpMV kernel alone (fp32: k_cg_spmv_dir32, else k_cg_spmv<double>)
// and the state that makes it run on every subdomain (profiling only).
cudaError_t launch_cg_spmv_alone(const DevProblem& d, int fp32, cudaStream_t s);
// CG state for timing a CG step alone: every stride-th subdomain active
// (stride 1: all), beta = 0.5, unit dot-product scaling.
cudaError_t launch_profile_state(const DevProblem& d, cudaStream_t s, int stride = 1);
// Assembled nodal load and ||f||^2 partials for the stop test (once per solve).
cudaError_t launch_load_nodes(const DevProblem& d, cudaStream_t s);
cudaError_t launch_cg_iteration32(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond);
cudaError_t launch_mixed_correct(const DevProblem& d, cudaStream_t s);
cudaError_t launch_apply32(const DevProblem& d, const double* x, double* y, cudaStream_t s);
cudaError_t launch_spmv_plain32(const DevProblem& d, const float* x, float* y, cudaStream_t s);
cudaError_t launch_exchange(const DevProblem& d, cudaStream_t s);
// tensor-product FP32 operator (osm_tensor.cu)
cudaError_t launch_tensor_coef(const DevProblem& d, cudaStream_t s);
cudaError_t launch_tensor_dir32(const DevProblem& d, cudaStream_t s);
cudaError_t launch_tensor_apply32(const DevProblem& d, const float* x, float* y, cudaStream_t s);
cudaError_t launch_tensor_init64(const DevProblem& d, cudaStream_t s);
// setup: flag the vector rows whose node has one copy; end of a call: phi
cudaError_t launch_mark_single(const DevProblem& d, uint8_t* single, cudaStream_t s);
cudaError_t launch_phi(const DevProblem& d, cudaStream_t s);
cudaError_t launch_tensor_init_df(const DevProblem& d, cudaStream_t s);
cudaError_t launch_box_mirror(const DevProblem& d, cudaStream_t s);
cudaError_t launch_tensor_layer(const DevProblem& d, cudaStream_t s);
// Shared-memory limits of the tensor kernels (once per process and device).
cudaError_t tensor_kernel_setup();
// The DevProblem seen by the FP32 CG kernels: the box layout's tile tables
// when the tensor operator is in use, else d itself.
DevProblem fp32_view(const DevProblem& d);
// adjoint gradient (osm_adjoint.cu)
cudaError_t launch_load_from_density(const DevProblem& d, const DevAdjoint& a, const double* drho, cudaStream_t s);
cudaError_t launch_station_values(const DevProblem& d, const DevAdjoint& a, const double* phi, const double* g_obs,
                                  cudaStream_t s);
cudaError_t launch_misfit(const DevAdjoint& a, double* J_dev, cudaStream_t s);
cudaError_t launch_stations_transpose(const DevProblem& d, const DevAdjoint& a, cudaStream_t s);
cudaError_t launch_nodal_load(const DevProblem& d, const DevAdjoint& a, const double* v_nodes, cudaStream_t s);
cudaError_t launch_density_gradient(const DevProblem& d, const DevAdjoint& a, const double* w_nodes, double* grad,
                                    cudaStream_t s);
cudaError_t launch_nodal_split(const DevProblem& d, const double* v, double* out, cudaStream_t s);
cudaError_t launch_exchange_adjoint(const DevProblem& d, const int32_t* partner, const double* lam, double* mu,
                                    double p2, double* ub, cudaStream_t s);
cudaError_t launch_dp_terms(const DevProblem& d, const double* lam, const double* u, const double* bbar, double* part,
                            double* out, cudaStream_t s);
cudaError_t launch_lambar_step(const DevProblem& d, const double* bbar, const double* lam_old, double* lam_new,
                               cudaStream_t s);
// batched p evaluation (osm_sample.cu)
cudaError_t launch_mp_start(const DevProblem& d, const DevSample& m, cudaStream_t s);
cudaError_t launch_mp_rhs_init(const DevProblem& d, const DevSample& m, cudaStream_t s, unsigned long long cond,
                               int use_cond, int fp32, int refine);
cudaError_t launch_mp_cg_iteration(const DevProblem& d, const DevSample& m, cudaStream_t s,
                                   unsigned long long cond, int use_cond, int mixed);
cudaError_t launch_mp_exchange_residual(const DevProblem& d, const DevSample& m, cudaStream_t s,
                                        unsigned long long cond, int use_cond, int mixed);
// CG start of the next Schwarz iteration (the SpMV kernel only: r = b - A u
// or the FP64 defect, y = A u kept for the stop test) and its finaliser.
cudaError_t launch_cg_start(const DevProblem& d, cudaStream_t s, int mixed);
cudaError_t launch_fin_init(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond,
                            int defect_norm);
// Stop test after launch_cg_start: ubar, K ubar = y - T u + K (ubar - u), the
// relative residual, the outer loop condition.
cudaError_t launch_stop_test(const DevProblem& d, cudaStream_t s, unsigned long long cond, int use_cond);
cudaError_t launch_apply(const DevProblem& d, int op, const double* x, double* y, cudaStream_t s);
cudaError_t launch_gather_local(const DevProblem& d, const double* vec, double* canon, cudaStream_t s);
cudaError_t launch_spmv_plain(const DevProblem& d, const double* x, double* y, cudaStream_t s);
// launch_apply with caller-chosen scratch vectors (vec_rows doubles each;
// w_scratch must be zero on every padding row).
cudaError_t launch_apply_scratch(const DevProblem& d, int op, const double* x, double* y, double* w_scratch,
                                 double* y_scratch, cudaStream_t s);

// Access to a handle's device problem for entry points defined outside
// osm_api.cu.  Returns nullptr for a null handle.
const DevProblem* handle_problem(osm_handle h, cudaStream_t* stream, int64_t* vec_rows, int* device);
void handle_set_error(osm_handle h, const char* msg);

}  // namespace osm
