/*
 * osm.h -- C ABI of the GB300 optimized-Schwarz gravimetry library (libosm.so).
 *
 * The library solves the gravimetry Poisson problem of Sec. 2,
 *     -Laplace(Phi) = 4 pi G drho   in a box,  Phi = 0 on its boundary,
 * discretised by Q2 (27-node triquadratic) hexahedral finite elements
 * ("high order finite elements", Sec. 6), with the non-overlapping optimized
 * Schwarz method of Sec. 3 using the zeroth-order Robin transmission operator
 * A = p ("oo0"; second-order and unsymmetric operators: osm_set_transmission):
 * every iteration solves all subdomain problems
 *     (K_i + p_i M_Gi) u_i = f_i + sum_j lam_ij
 * by Jacobi-preconditioned CG (Sec. 6), all subdomains batched in the same
 * kernels, then exchanges the interface Robin data
 *     lam_ij <- (p_i + p_j) M_Gij u_j - lam_ji
 * and evaluates the global relative residual ||f - K ubar|| / ||f|| of the
 * averaged interface values (the stop test of Sec. 6).  Sec. 4's stochastic
 * search over p is served by osm_sample_p, which runs many p values as one
 * batched Schwarz run.
 *
 * Conventions shared by every entry point
 *  - Host pointers ("host") are read during the call only; the caller keeps
 *    ownership.  Device pointers ("device") must be cudaMalloc'ed memory on
 *    the device that was current at osm_setup; the caller owns them too.
 *  - All device work is enqueued on the CUDA stream given to osm_setup.
 *    Entry points that return results on the host synchronise that stream.
 *  - Element-indexed arrays are x-fastest: e = ex + nx (ey + ny ez).
 *    Node-indexed arrays cover the full (2nx+1)(2ny+1)(2nz+1) Q2 node grid,
 *    x-fastest, Dirichlet nodes included (their value is 0).
 *  - Subdomain s = a + sx (b + sy c) owns elements [cx[a], cx[a+1]) x
 *    [cy[b], cy[b+1]) x [cz[c], cz[c+1]).  Its unknowns are the nodes of its
 *    closed element box that are not on the outer boundary; interface nodes
 *    are duplicated in every subdomain that touches them.
 *  - "Canonical local layout": the unknowns of subdomain 0, then 1, ...,
 *    each subdomain's unknowns in ascending node index.
 *  - "Canonical face layout": interface faces ordered x-normal faces first
 *    (loops c, b, a with a fastest), then y-normal, then z-normal; face f
 *    between s < t holds 2 n_f values: the datum received by s from t for its
 *    n_f non-Dirichlet nodes in ascending node index, then the datum received
 *    by t from s in the same node order.
 *  - Every function returns an osm_status; on failure the handle's
 *    osm_last_error() text says why.  No entry point aborts the process.
 */
#ifndef OSM_H
#define OSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct osm_ctx *osm_handle;   /* opaque, owned by the library */

typedef enum {
    OSM_OK = 0,
    OSM_E_ARG = 1,        /* invalid argument (sizes, p <= 0, null pointer) */
    OSM_E_CUDA = 2,       /* a CUDA runtime call failed */
    OSM_E_NOMEM = 3,      /* device or host allocation failed */
    OSM_E_NOCONV = 4,     /* iteration cap reached; outputs are still written */
    OSM_E_BREAKDOWN = 5,  /* CG breakdown (p.Ap <= 0 or non-finite) */
    OSM_E_STATE = 6,      /* call not valid in the handle's current state */
    OSM_E_TIMEOUT = 7     /* a bounded device wait gave up */
} osm_status;

typedef enum {
    OSM_FP64 = 0,   /* every step in FP64 */
    OSM_MIXED = 1,  /* per Schwarz iteration and subdomain: FP64 defect d = b - A u, one
                       FP32 CG solve of A e = d from e = 0 (FP32 matrix values, FP32
                       vectors and accumulation; dot products of power-of-two-scaled
                       factors summed in FP32 per warp and in FP64 across warps and
                       tiles) to ||r|| <= mixed_inner_rtol ||d||, then u += e in FP64;
                       the Robin exchange and the stop test stay FP64 */
    OSM_FP64_REFINE = 2 /* the OSM_MIXED algorithm in FP64: FP64 CG warm-started from u_i,
                           stopped at ||r|| <= mixed_inner_rtol times its initial residual
                           (the defect), subdomains whose defect meets inner_rtol skipped */
} osm_precision;

typedef struct {
    int32_t nx, ny, nz;            /* elements per direction, >= 1 */
    const double *xc, *yc, *zc;    /* host; nx+1, ny+1, nz+1 strictly increasing
                                      vertex coordinates (axis-aligned tensor mesh,
                                      so graded meshes are allowed) */
} osm_mesh;

typedef struct {
    int32_t sx, sy, sz;            /* subdomains per direction, >= 1 */
    const int32_t *cx, *cy, *cz;   /* host; s+1 element-index cuts, 0 = c[0] < ... < c[s] = n */
} osm_decomp;

typedef struct {
    osm_precision prec;
    double inner_rtol;      /* FP64 subdomain CG stop ||b_i - A_i u_i|| <= inner_rtol ||b_i||
                               (Sec. 6 uses 1e-10) */
    double mixed_inner_rtol;/* OSM_MIXED / OSM_FP64_REFINE: CG stop on each correction,
                               relative to the FP64 defect, in (0, 1) (default 1e-5; the
                               fastest on the 64^3 layered benchmark was 0.4-0.5: fewer CG
                               steps for more Schwarz iterations) */
    int32_t max_outer;      /* Schwarz iteration cap (default 10000) */
    int32_t max_inner;      /* CG iteration cap per subdomain solve (default 20000) */
    int32_t use_graph;      /* 1 (default): the whole solve runs as one CUDA graph with
                               device-side while loops; 0: host-driven loop (debugging) */
    int32_t max_seconds;    /* device wall-clock limit of one solve (default 900): past it
                               both loops stop and the call returns OSM_E_TIMEOUT */
    int32_t autotune;       /* 1 (default): at setup, time the SpMV kernel variants (one or
                               two SELL slices per warp, 32- or 16-bit columns) on this
                               handle's matrices and keep the fastest per precision; 0: one
                               slice per warp; 2: two slices per warp (no timing) */
    int32_t index16;        /* 1 (default): when every subdomain has at most 65,536 padded
                               rows, also store the column indices in 16 bits (FP64: 10
                               instead of 12 bytes per nonzero, FP32: 6 instead of 8); the
                               autotuner picks the width per precision (with autotune != 1
                               the 16-bit ones are used); 0: always 32 bits */
    int32_t fp32_operator;  /* OSM_MIXED: the operator of the FP32 inner CG.  0 (default):
                               chosen by the autotuner (timing both CG-step kernels);
                               1: the FP32 SELL matrix; 2: the tensor-product form
                               K_i = Kx (x) My (x) Mz + Mx (x) Ky (x) Mz + Mx (x) My (x) Kz of
                               the assembled 1-D Q2 operators, applied matrix-free by sum
                               factorisation, with the Robin term p M_G folded into the
                               1-D stiffness at interface ends.  The tensor form holds for
                               zeroth-order transmission (q = 0) only: with q != 0 the
                               handle uses the SELL matrix.  Boxes wider than 128 nodes
                               along x also keep the SELL matrix. */
    int32_t fp64_start;     /* OSM_MIXED with the tensor form: the kernel of each
                               refinement step's defect d = b - A u.  0 (default):
                               chosen by the autotuner; 1: the FP64 SELL SpMV; 2: the
                               tensor-product kernel in FP64 on a box-layout copy of u;
                               3: the same in double-float arithmetic (pairs of floats,
                               about 48 significant bits, compensated sums: the FP32
                               pipe instead of the FP64 one).  The double-float defect's
                               rounding, about 2^-48 |A| |u| per row, stays some 100x
                               below a stop tolerance of 1e-8 on these meshes; use 1 or
                               2 for tolerances below about 1e-10. */
    int32_t tensor_zchunk;  /* tensor form: z planes per CTA of the tensor-product kernels
                               (a box's z range is cut into chunks of nearly equal length
                               up to this).  0 (default): chosen by the autotuner among
                               8, 16, 32 and 128; 8 .. 128: that length. */
} osm_opts;

typedef struct {
    int32_t n_sub, n_face;
    int64_t n_nodes;        /* full node grid */
    int64_t n_dofs;         /* global unknowns (interior nodes) */
    int64_t n_local;        /* sum of subdomain unknowns (canonical local layout length) */
    int64_t n_face_vals;    /* canonical face layout length (2 * sum n_f) */
    int64_t nnz;            /* sum of subdomain matrix nonzeros (algorithmic) */
    int64_t sell_entries;   /* stored SELL entries (nonzeros + padding) */
    int64_t n_slices;       /* SELL slices of 32 rows */
    int64_t vec_rows;       /* padded device vector length */
    int64_t device_bytes;   /* device memory held by the handle */
    double setup_seconds;   /* host assembly + upload wall time */
    int32_t spmv_variant_fp64;   /* SELL slices per warp chosen for the FP64 SpMV */
    int32_t spmv_variant_fp32;   /* ... for the FP32 SpMV (0 without OSM_MIXED) */
    double spmv_ms_fp64[2];      /* autotuner timings of the FP64 variants, one / two slices per
                                    warp, 32-bit columns (ms, 0 if not run) */
    double spmv_ms_fp32[2];
    double spmv_ms16_fp64[2];    /* the same with 16-bit columns (0 if not stored or not run) */
    double spmv_ms16_fp32[2];
    int32_t col_bytes_fp64;      /* bytes per column index read by the FP64 SpMVs (2 or 4) */
    int32_t col_bytes_fp32;      /* ... by the FP32 SpMVs (0 without OSM_MIXED) */
    int32_t fp32_operator;       /* operator of the FP32 inner CG in use: 1 SELL, 2 tensor
                                    product (0 without OSM_MIXED) */
    int32_t fp32_operator_tuned; /* the autotuner's (or opts.fp32_operator's) choice, used
                                    whenever the transmission condition allows it */
    double tensor_ms_fp32;       /* autotuner timing of the tensor-product CG-step kernel in its
                                    chosen shape (ms, 0 if not run) */
    int32_t tensor_zchunk;       /* z planes per CTA of the tensor kernel (0: no tensor form);
                                    2^20 leaves every subdomain box whole */
    int32_t reserved_i;
    double tensor_ms_zchunk[4];  /* autotuner timings with z chunks of 8, 16, 32 and 128 planes
                                    (ms, 0 if not run) */
    int32_t fp64_start;          /* OSM_MIXED: kernel of each refinement step's defect
                                    d = b - A u: 1 the FP64 SELL SpMV, 2 the FP64 tensor-
                                    product kernel, 3 its double-float form (osm_opts
                                    fp64_start; chosen by the autotuner with the tensor
                                    form); 0 otherwise */
    int32_t reserved_j;
    double start_ms[3];          /* autotuner timings of that step: SELL, FP64 tensor,
                                    double-float tensor (ms, 0 if not run) */
    int64_t box_rows;            /* rows of the box layout of the tensor form (0 if none) */
    double tensor_ms_zchunk_tail[4];  /* the same timings with one subdomain in eight active (the
                                    tail of an inner solve); the autotuner keeps the z chunk
                                    with the smallest sum of both */
} osm_info_t;

typedef struct {
    int32_t n_outer;        /* Schwarz iterations of the last solve / iterate call */
    int32_t n_cg_steps;     /* batched CG iterations summed over those Schwarz iterations */
    int64_t n_launches;     /* kernels the call launched on the GPU */
    double relres;          /* last stop-test value */
    int32_t status;         /* bit 0: a subdomain CG hit max_inner; bit 1: CG breakdown */
    int32_t reserved;
    int64_t sub_row_steps;  /* osm_solve / osm_iterate: sum over subdomains of (CG steps of the
                               call) x (its local unknowns); 0 after osm_sample_p */
    int64_t op_row_steps;   /* the same with the rows the CG-step kernels sweep per step: the
                               box layout's rows (tiles of 256) on the FP32 tensor-product form,
                               the padded SELL rows otherwise */
} osm_stats_t;

/* Fill *o with the defaults listed in osm_opts. */
void osm_default_opts(osm_opts *o);

/*
 * Assemble every subdomain system on the host from the closed-form Q2
 * tensor-product element matrices, pack it for the GPU and upload it.
 * drho: host, nx*ny*nz per-element constant density anomalies (kg/m^3);
 * the load is 4 pi G drho with G = 6.672e-11 (Sec. 2).  opts may be NULL
 * (defaults).  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * The Robin parameter starts at p = 1 for every subdomain; call osm_set_robin.
 * Errors: OSM_E_ARG for bad sizes or non-increasing coordinates/cuts,
 * OSM_E_NOMEM / OSM_E_CUDA on allocation or upload failure.  When a handle
 * was created before the failure, *out is still set so that
 * osm_last_error() can be read; the caller then calls osm_destroy on it.
 */
osm_status osm_setup(const osm_mesh *mesh, const double *drho, const osm_decomp *dec,
                     const osm_opts *opts, void *cuda_stream, osm_handle *out);

/* Sizes and memory of a handle. */
osm_status osm_info(osm_handle h, osm_info_t *out);

/* Replace the density (host array, nx*ny*nz); rebuilds the load only. */
osm_status osm_set_density(osm_handle h, const double *drho);

/* Robin parameter p > 0 on every subdomain (Sec. 3, A = p).  OSM_E_ARG if
 * p <= 0 or not finite. */
osm_status osm_set_robin(osm_handle h, double p);

/* One Robin parameter per subdomain (host, n_sub values, all > 0): the
 * unsymmetric form where subdomain i uses p_i and the exchange uses p_i + p_j. */
osm_status osm_set_robin_sub(osm_handle h, const double *p_sub);

/*
 * Second-order and unsymmetric transmission conditions (Sec. 3, Table 1).
 * The operator of a subdomain on a face is A = p + q (-d^2/dtau^2), Fourier
 * symbol p + q k^2, with weak form p M_G + q S_G (S_G: the face's tangential
 * Q2 stiffness).  On every interface face the subdomain on the lower side
 * (smaller coordinate along the face normal) uses (p_lo, q_lo) and the one
 * on the upper side (p_hi, q_hi); the exchange becomes
 *   lam_ij <- (p_i + p_j) M_Gij u_j + (q_i + q_j) S_Gij u_j - lam_ji.
 * p_lo = p_hi, q = 0 is osm_set_robin.  Needs p > 0 and q >= 0, finite
 * (A_i stays SPD), else OSM_E_ARG.  osm_sample_p still evaluates zeroth-order
 * symmetric candidates and restores these coefficients afterwards;
 * osm_grad_p returns OSM_E_STATE while q != 0 or p_lo != p_hi.
 */
osm_status osm_set_transmission(osm_handle h, double p_lo, double q_lo, double p_hi, double q_hi);

/*
 * Full Schwarz solve from u = 0, lam = 0 until ||f - K ubar|| <= rtol ||f||.
 * phi: device, n_nodes doubles (may be NULL): the averaged solution ubar on
 * the full node grid.  iters / relres: host (may be NULL): Schwarz iterations
 * done and the final relative residual.  Returns OSM_E_NOCONV when max_outer
 * is reached (outputs written) and OSM_E_BREAKDOWN on a CG breakdown.
 */
osm_status osm_solve(osm_handle h, double rtol, double *phi, int32_t *iters, double *relres);

/*
 * Batched stochastic evaluation of Robin parameters (Sec. 4): the n_p
 * candidate values p_host[k] > 0 (host) run the Schwarz solve of osm_solve,
 * in the handle's precision mode (OSM_FP64, OSM_MIXED with the FP32 inner
 * solve, or OSM_FP64_REFINE), in batches of up to 32 candidates that share the subdomain
 * stiffness matrices K_i (one pass over K_i serves every candidate of the
 * batch), each from u = 0 with its own iterate, Robin data, subdomain CG
 * scalars and convergence mask, until its own relative residual reaches rtol
 * or max_outer iterations pass.  iters_host / relres_host (host, n_p each)
 * receive each candidate's Schwarz iteration count and final relative
 * residual; best_idx (host) the fastest-converging candidate: fewest
 * iterations among those that reached rtol, ties to the lower residual, then
 * the smaller p; -1 if none converged (the call then returns OSM_E_NOCONV
 * with the outputs written).  A candidate's result does not depend on the
 * other candidates of its batch.  The first call allocates the batch buffers
 * (about 8 x 32 vectors); the handle's own Robin parameters are restored
 * before the call returns.
 */
osm_status osm_sample_p(osm_handle h, int32_t n_p, const double *p_host, double rtol,
                        int32_t max_outer, int32_t *iters_host, double *relres_host,
                        int32_t *best_idx);

/*
 * osm_sample_p with flags.  OSM_SAMPLE_RACE: the search wants the fastest-
 * converging p (fewest Schwarz iterations, Sec. 4), so a batch stops at the
 * iteration where its first candidate reaches rtol -- no candidate still
 * running can need fewer -- and a later batch of 32 stops at the best count
 * found so far.  The winner and every candidate converging at the same
 * iteration get exactly their osm_sample_p results; the others report the
 * iteration and the residual at which they were stopped (relres > rtol).
 * Unknown flags: OSM_E_ARG.
 */
#define OSM_SAMPLE_RACE 1
osm_status osm_sample_p_ex(osm_handle h, int32_t n_p, const double *p_host, double rtol, int32_t max_outer,
                           int32_t flags, int32_t *iters_host, double *relres_host, int32_t *best_idx);

/* ----------------------------------------------------------------------
 * Adjoint gradient of a surface-gravity misfit.  The paper's forward model
 * (Sec. 2, solved as in Sec. 3) is differentiated; the paper itself has no
 * gradient.  With f = 4 pi G F drho (F_ae = int_e phi_a) and K phi = f:
 *   g = B phi (B: d/dz of the Q2 interpolant of the element holding each
 *   station), J = 1/2 sum_s (g_s - g_obs,s)^2,
 *   dJ/d drho = 4 pi G F^T w with K w = B^T (g - g_obs),
 * w computed by one more Schwarz solve with the same p and precision.
 * ---------------------------------------------------------------------- */

/* Replace the density from a device array (nx*ny*nz, x-fastest); the load
 * is assembled on the GPU (node-centric, fixed summation order). */
osm_status osm_set_density_dev(osm_handle h, const double *drho);

/* Stations (host, n_st x 3 coordinates inside the mesh).  A station on an
 * element boundary belongs to the element on its upper side in that
 * direction, except on the upper mesh boundary (e.g. surface stations at the
 * top face), where it belongs to the element below. */
osm_status osm_set_stations(osm_handle h, int32_t n_st, const double *xyz);

/* g = B phi for a full-grid field phi (device), g device (n_st). */
osm_status osm_gravity(osm_handle h, const double *phi, double *g);

/* Vector-Jacobian product of phi(drho): given v = dL/dphi (device, full node
 * grid; Dirichlet entries ignored), solve K w = v by the Schwarz method to
 * rtol and write dL/d drho = 4 pi G F^T w (device, nx*ny*nz).  The handle's
 * load is kept; its iterates are overwritten. */
osm_status osm_potential_vjp(osm_handle h, double rtol, const double *v, double *dL_drho);

/* Forward solve, misfit and adjoint gradient: J (host), dJ_drho (device,
 * nx*ny*nz), dJ_dp (host, may be NULL).  g_obs: device, n_st.  The
 * converged solution is the Galerkin solution for every p > 0, so the exact
 * dJ/dp of the converged map is 0; *dJ_dp receives that value. */
osm_status osm_grad(osm_handle h, double rtol, const double *g_obs, double *J, double *dJ_drho,
                    double *dJ_dp);

/* Derivative of the truncated iteration with respect to p.  J_N(p) is the
 * misfit of the averaged iterate after exactly n_iter Schwarz iterations
 * from zero (each subdomain solve to opts.inner_rtol); dJ_N/dp is computed
 * by reverse-mode (adjoint) Schwarz: the iterates are kept, then n_iter
 * backward steps each apply one adjoint subdomain solve, so the cost is
 * about one more Schwarz solve.  OSM_FP64 single-problem handles with one p
 * for all subdomains; stations must be set.  g_obs: device (n_st); J, dJ_dp:
 * host.  The handle's iterates are reset to zero afterwards; the call
 * allocates n_iter iterate copies for its duration. */
osm_status osm_grad_p(osm_handle h, int32_t n_iter, const double *g_obs, double *J, double *dJ_dp);

/* SplitMix64 (Steele, Lea & Flood 2014) log-uniform samples in [lo, hi]:
 * p = exp(log lo + u (log hi - log lo)), u = (x >> 11) * 2^-53, x the k-th
 * output after seeding the state with `seed`.  p_host: host, n values. */
osm_status osm_log_uniform_p(uint64_t seed, int32_t n, double lo, double hi, double *p_host);

/* ----------------------------------------------------------------------
 * Independent problems in one handle: every instance (its own mesh,
 * density, decomposition and Robin parameter) runs the Schwarz solve of
 * osm_solve; all instances' subdomains share every kernel launch of one
 * CUDA graph, and an instance that has converged is frozen while the others
 * continue.  Instance i's nodes occupy [off[i], off[i+1]) of node-indexed
 * arrays (osm_batch_info), each instance's grid x-fastest as usual.
 * Gradient, stations, osm_set_density* and osm_sample_p need a single-problem
 * handle (OSM_E_STATE otherwise).
 * ---------------------------------------------------------------------- */

/* meshes, decs: host arrays of n_inst descriptors; drho: host array of n_inst
 * host pointers (nx*ny*nz each).  Same errors and *out rule as osm_setup. */
osm_status osm_setup_batch(int32_t n_inst, const osm_mesh *meshes, const double *const *drho,
                           const osm_decomp *decs, const osm_opts *opts, void *cuda_stream,
                           osm_handle *out);

/* n_inst (host) and, if node_offsets != NULL, the n_inst + 1 node offsets. */
osm_status osm_batch_info(osm_handle h, int32_t *n_inst, int64_t *node_offsets);

/* One Robin parameter per instance (host, n_inst values > 0). */
osm_status osm_set_robin_inst(osm_handle h, const double *p_inst);

/* Solve every instance from zero to its own relative residual rtol.  phi:
 * device, total node count (may be NULL); iters / relres: host, n_inst each
 * (may be NULL).  OSM_E_NOCONV if an instance reached max_outer. */
osm_status osm_solve_batch(osm_handle h, double rtol, double *phi, int32_t *iters, double *relres);

/* ----------------------------------------------------------------------
 * Step-level entry points (used by the parity tests; same conventions).
 * ---------------------------------------------------------------------- */

/* y = A x per subdomain with x, y in the canonical local layout (device,
 * n_local doubles each).  op 0: A_i = K_i + p_i M_Gi (the Robin matrix);
 * op 1: A_i = K_i (Neumann stiffness); op 2 (OSM_MIXED handles only, else
 * OSM_E_STATE): the FP32 Robin matrix of the mixed inner solve applied to x
 * rounded to FP32, with FP32 accumulation, returned widened to FP64.  This
 * call uses the inner solve's work vectors. */
osm_status osm_apply(osm_handle h, int32_t op, const double *x, double *y);

/* Zero the subdomain iterates u_i and the Robin data lam. */
osm_status osm_reset(osm_handle h);

/* n Schwarz iterations continuing from the current state, no stop test
 * other than the caps.  relres_hist: host, n doubles (may be NULL), the
 * stop-test residual after each iteration. */
osm_status osm_iterate(osm_handle h, int32_t n, double *relres_hist);

/* Copy the subdomain iterates u_i out in the canonical local layout (device). */
osm_status osm_get_local(osm_handle h, double *u);

/* Copy the Robin data out / in, canonical face layout (device). */
osm_status osm_get_lambda(osm_handle h, double *lam);
osm_status osm_set_lambda(osm_handle h, const double *lam);

/* Counters of the last osm_solve / osm_iterate call (host). */
osm_status osm_stats(osm_handle h, osm_stats_t *out);

/* CG iteration counts of the last subdomain solves (host, n_sub values). */
osm_status osm_inner_iters(osm_handle h, int32_t *iters);

/*
 * Host-only checks of the packing (no GPU needed).  Both assemble and pack
 * the problem exactly as osm_setup does and then unpack one piece of it.
 *
 * osm_host_local_system: subdomain `sub`'s Robin matrix A_i = K_i + p M_Gi
 * (unpacked from the SELL arrays) and load f_i, in its canonical local
 * numbering, as CSR with ascending columns.  Call once with rowptr == NULL
 * to get *n and *nnz, then with rowptr[n+1], col[nnz], val[nnz], f[n] (host).
 *
 * osm_host_face_system: interface face `face` (canonical face order): the
 * node index of each of its n_f nodes and its face mass M_Gst as CSR over
 * the face nodes.  Same two-call protocol: node[n], rowptr[n+1], col[nnz],
 * val[nnz] (host).
 */
osm_status osm_host_local_system(const osm_mesh *mesh, const double *drho, const osm_decomp *dec,
                                 double p, int32_t sub, int64_t *n, int64_t *nnz, int64_t *rowptr,
                                 int32_t *col, double *val, double *f);
osm_status osm_host_face_system(const osm_mesh *mesh, const double *drho, const osm_decomp *dec,
                                int32_t face, int64_t *n, int64_t *nnz, int32_t *node,
                                int64_t *rowptr, int32_t *col, double *val);

/*
 * osm_host_local_system_tc: as osm_host_local_system with the transmission
 * coefficients tc = {p_lo, q_lo, p_hi, q_hi} of osm_set_transmission (host,
 * 4 values).  osm_host_face_stiffness: the tangential stiffness S_G of face
 * `face`, nnz values (host) in the CSR order of osm_host_face_system.
 */
osm_status osm_host_local_system_tc(const osm_mesh *mesh, const double *drho, const osm_decomp *dec,
                                    const double *tc, int32_t sub, int64_t *n, int64_t *nnz, int64_t *rowptr,
                                    int32_t *col, double *val, double *f);
osm_status osm_host_face_stiffness(const osm_mesh *mesh, const double *drho, const osm_decomp *dec, int32_t face,
                                   double *val);

/* Time one operator kernel alone over every subdomain.
 *   prec 0: the plain FP64 SELL operator y = A x (the SpMV of the FP64 paths);
 *   prec 1: the plain FP32 operator of the mixed inner solve (SELL, or the
 *           tensor-product kernel when osm_info fp32_operator is 2);
 *   prec 2: the FP32 CG-step kernel (k_cg_spmv_dir32 or its tensor-product
 *           counterpart: the operator plus the p, q direction epilogue and
 *           the p.q partials);
 *   prec 3: the FP64 CG-step kernel k_cg_spmv<double> (SpMV of p, p.q);
 *   prec 4: the start of a mixed refinement step (the FP64 defect d = b - A u
 *           with the FP32 CG start; SELL or tensor-product, osm_info
 *           fp64_start).
 * 1, 2 and 4 need an OSM_MIXED handle (else OSM_E_STATE).  After 20 untimed
 * launches, 5 trials of `reps` back-to-back launches are timed with CUDA
 * events on the handle's stream; *ms receives the median time per launch in
 * milliseconds (host).  0 and 1 use the work vectors only; 2, 3 and 4
 * overwrite the CG vectors and scalars (2 and 3 mark every subdomain
 * active), so call them between solves (the next osm_solve starts afresh). */
osm_status osm_profile_spmv(osm_handle h, int32_t prec, int32_t reps, double *ms);

/*
 * y = A x exactly as osm_apply computes it, but without any device
 * allocation for the call.  The paper has no counterpart.  It serves callers
 * that cannot call cudaMalloc where they need the operator: plug-ins whose
 * device memory is reserved and capped by a host framework's own allocator
 * (a cudaMalloc of their own bypasses it and can fail), and callers with a
 * memory budget fixed at start-up.  Besides x and y (canonical local layout,
 * device, n_local doubles each) the call uses only a fixed 8 MiB scratch
 * array inside the library image, which every GPU that loads the library
 * holds until the process exits.  Limit: the handle's padded vector length
 * (osm_info vec_rows) must be at most 524288; larger problems get OSM_E_ARG
 * with an explanation.  The first call on a device looks up the scratch
 * array's device address, so make it before any stream capture.  All calls
 * share the scratch: calls that overlap on the GPU race.
 * op 0: A_i = K_i + p_i M_Gi; op 1: A_i = K_i.  Synchronises the stream.
 */
osm_status osm_apply_noalloc(osm_handle h, int32_t op, const double *x, double *y);

/* Static description of a status code. */
const char *osm_status_string(osm_status s);

/* Text of the last error on this handle ("" if none); valid until the next call. */
const char *osm_last_error(osm_handle h);

/* Free every device and host resource of the handle (NULL is ignored). */
void osm_destroy(osm_handle h);

#ifdef __cplusplus
}
#endif

#endif /* OSM_H */
