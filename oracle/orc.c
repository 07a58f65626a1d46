/*
 * Oracle for the optimized Schwarz gravimetry solver: plain, slow FP64 CPU
 * code.  TEST INFRASTRUCTURE ONLY -- it is called by the test suite, by the
 * smoke check and by the CPU-baseline leg of the benchmark, never by the
 * product path, and it shares no code with the CUDA library.
 *
 * What it computes (paper sections / equations it follows):
 *   - Sec. 2: the gravimetry Poisson problem  -Laplace(Phi) = 4 pi G drho  with
 *     homogeneous Dirichlet data on the outer boundary (Sec. 3 states the
 *     method for this boundary condition).
 *   - "High order finite elements" on hexahedra (Sec. 6): Q2 (27-node
 *     triquadratic) Lagrange elements.  Element matrices are computed here
 *     by 3x3x3 Gauss quadrature of the Lagrange basis gradients, which is
 *     exact for Q2 on axis-aligned boxes.
 *   - Sec. 6: diagonal (Jacobi) preconditioned CG with a relative residual
 *     stop, CSR storage.
 *   - Sec. 3, the two-subdomain Robin iteration (operators A = p, the
 *     zeroth-order "oo0" condition), generalised to a box grid of
 *     subdomains with parallel (Jacobi-type) updates.  The discrete form is:
 *        (K_i + p_i M_Gi) u_i = f_i + sum_j lam_ij
 *        lam_ij <- (p_i + p_j) M_Gij u_j - lam_ji
 *     where lam_ij is the weak Robin datum on face G_ij received by i from j.
 *     Second-order ("oo2") and unsymmetric conditions (Sec. 3, Table 1):
 *     the operator of subdomain s on a face is p_s + q_s (-d^2/dtau^2)
 *     (Fourier symbol p_s + q_s k^2), whose weak form is p_s M + q_s S with
 *     S the face's tangential Q2 stiffness; then
 *        (K_i + sum_faces (p_i M_Gij + q_i S_Gij)) u_i = f_i + sum_j lam_ij
 *        lam_ij <- (p_i + p_j) M_Gij u_j + (q_i + q_j) S_Gij u_j - lam_ji.
 *     In the unsymmetric form the lower side of every face (smaller
 *     coordinate along its normal) takes (p1, q1), the upper side (p2, q2).
 *   - Sec. 6 stop test: global relative residual ||f - K ubar|| / ||f||
 *     with ubar the average of the subdomain copies at interface nodes.
 *
 * Node grid: (2nx+1)(2ny+1)(2nz+1) nodes, x fastest.  Element e = (ex,ey,ez)
 * covers node indices 2ex..2ex+2 in x (likewise y, z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_G 6.672e-11

/* ------------------------------------------------------------------------ */
/* 1-D Q2 Lagrange basis on [0,1], nodes 0, 1/2, 1.                          */
/* ------------------------------------------------------------------------ */
void orc_basis_1d(double s, double phi[3], double dphi[3])
{
    phi[0] = (1.0 - s) * (1.0 - 2.0 * s);
    phi[1] = 4.0 * s * (1.0 - s);
    phi[2] = s * (2.0 * s - 1.0);
    dphi[0] = 4.0 * s - 3.0;
    dphi[1] = 4.0 - 8.0 * s;
    dphi[2] = 4.0 * s - 1.0;
}

/* Three-point Gauss-Legendre rule on [0,1] (exact to degree 5). */
static void gauss3(double pt[3], double wt[3])
{
    double d = 0.5 * sqrt(0.6);
    pt[0] = 0.5 - d; pt[1] = 0.5; pt[2] = 0.5 + d;
    wt[0] = 5.0 / 18.0; wt[1] = 8.0 / 18.0; wt[2] = 5.0 / 18.0;
}

/*
 * Element stiffness K[27*27], mass M[27*27] and basis integrals w[27] of the
 * box element hx x hy x hz, local node I = a + 3b + 9c.  Plain quadrature:
 * K_IJ = int grad(phi_I).grad(phi_J), M_IJ = int phi_I phi_J, w_I = int phi_I.
 */
void orc_element(double hx, double hy, double hz, double *K, double *M, double *w)
{
    double pt[3], wt[3];
    gauss3(pt, wt);
    memset(K, 0, sizeof(double) * 729);
    memset(M, 0, sizeof(double) * 729);
    memset(w, 0, sizeof(double) * 27);
    for (int qc = 0; qc < 3; ++qc)
    for (int qb = 0; qb < 3; ++qb)
    for (int qa = 0; qa < 3; ++qa) {
        double W = wt[qa] * wt[qb] * wt[qc] * hx * hy * hz;
        double fx[3], dx[3], fy[3], dy[3], fz[3], dz[3];
        orc_basis_1d(pt[qa], fx, dx);
        orc_basis_1d(pt[qb], fy, dy);
        orc_basis_1d(pt[qc], fz, dz);
        double val[27], gx[27], gy[27], gz[27];
        for (int c = 0; c < 3; ++c)
        for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
            int I = a + 3 * b + 9 * c;
            val[I] = fx[a] * fy[b] * fz[c];
            gx[I] = dx[a] / hx * fy[b] * fz[c];
            gy[I] = fx[a] * dy[b] / hy * fz[c];
            gz[I] = fx[a] * fy[b] * dz[c] / hz;
        }
        for (int I = 0; I < 27; ++I) {
            w[I] += W * val[I];
            for (int J = 0; J < 27; ++J) {
                K[I * 27 + J] += W * (gx[I] * gx[J] + gy[I] * gy[J] + gz[I] * gz[J]);
                M[I * 27 + J] += W * val[I] * val[J];
            }
        }
    }
}

/* 2-D Q2 face mass M[9*9] of an ha x hb rectangle, local node a + 3b. */
void orc_face_element(double ha, double hb, double *M)
{
    double pt[3], wt[3];
    gauss3(pt, wt);
    memset(M, 0, sizeof(double) * 81);
    for (int qb = 0; qb < 3; ++qb)
    for (int qa = 0; qa < 3; ++qa) {
        double W = wt[qa] * wt[qb] * ha * hb;
        double fa[3], da[3], fb[3], db[3];
        orc_basis_1d(pt[qa], fa, da);
        orc_basis_1d(pt[qb], fb, db);
        for (int I = 0; I < 9; ++I)
            for (int J = 0; J < 9; ++J)
                M[I * 9 + J] += W * fa[I % 3] * fb[I / 3] * fa[J % 3] * fb[J / 3];
    }
}

/* 2-D Q2 tangential stiffness S[9*9] of an ha x hb rectangle, local node
 * a + 3b: S_IJ = int grad_t(phi_I) . grad_t(phi_J) over the face (the weak
 * form of -d^2/dtau^2 in the second-order transmission operator, Sec. 3). */
void orc_face_stiffness(double ha, double hb, double *S)
{
    double pt[3], wt[3];
    gauss3(pt, wt);
    memset(S, 0, sizeof(double) * 81);
    for (int qb = 0; qb < 3; ++qb)
    for (int qa = 0; qa < 3; ++qa) {
        double W = wt[qa] * wt[qb] * ha * hb;
        double fa[3], da[3], fb[3], db[3];
        orc_basis_1d(pt[qa], fa, da);
        orc_basis_1d(pt[qb], fb, db);
        for (int I = 0; I < 9; ++I)
            for (int J = 0; J < 9; ++J) {
                double ga_i = da[I % 3] / ha * fb[I / 3], gb_i = fa[I % 3] * db[I / 3] / hb;
                double ga_j = da[J % 3] / ha * fb[J / 3], gb_j = fa[J % 3] * db[J / 3] / hb;
                S[I * 9 + J] += W * (ga_i * ga_j + gb_i * gb_j);
            }
    }
}

/* Physical Gauss points of every element: pts[(e*27 + q)*3 + d], q = qa+3qb+9qc. */
void orc_gauss_points(int nx, int ny, int nz, const double *xc, const double *yc,
                      const double *zc, double *pts)
{
    double pt[3], wt[3];
    gauss3(pt, wt);
    for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
    for (int ex = 0; ex < nx; ++ex) {
        int64_t e = ex + (int64_t)nx * (ey + (int64_t)ny * ez);
        for (int q = 0; q < 27; ++q) {
            double *o = pts + (e * 27 + q) * 3;
            o[0] = xc[ex] + pt[q % 3] * (xc[ex + 1] - xc[ex]);
            o[1] = yc[ey] + pt[(q / 3) % 3] * (yc[ey + 1] - yc[ey]);
            o[2] = zc[ez] + pt[q / 9] * (zc[ez + 1] - zc[ez]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Element matrix cache (many elements share their size).                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n, cap;
    double *h;      /* 3 per entry */
    double *K, *M, *w;
} emat_cache;

static const double *cache_get(emat_cache *c, double hx, double hy, double hz, int which)
{
    int i;
    for (i = 0; i < c->n; ++i)
        if (c->h[3 * i] == hx && c->h[3 * i + 1] == hy && c->h[3 * i + 2] == hz)
            break;
    if (i == c->n) {
        if (c->n == c->cap) {
            c->cap = c->cap ? 2 * c->cap : 16;
            c->h = realloc(c->h, sizeof(double) * 3 * c->cap);
            c->K = realloc(c->K, sizeof(double) * 729 * c->cap);
            c->M = realloc(c->M, sizeof(double) * 729 * c->cap);
            c->w = realloc(c->w, sizeof(double) * 27 * c->cap);
        }
        c->h[3 * i] = hx; c->h[3 * i + 1] = hy; c->h[3 * i + 2] = hz;
        orc_element(hx, hy, hz, c->K + 729 * i, c->M + 729 * i, c->w + 27 * i);
        c->n++;
    }
    return which == 0 ? c->K + 729 * i : which == 1 ? c->M + 729 * i : c->w + 27 * i;
}

static void cache_free(emat_cache *c) { free(c->h); free(c->K); free(c->M); free(c->w); }

/* ------------------------------------------------------------------------ */
/* Box systems: stiffness over a box of elements, CSR over its unknowns.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    double *xc, *yc, *zc;
    int NX, NY, NZ;         /* node grid */
} geom;

typedef struct {
    int64_t n;              /* unknowns */
    int64_t *rp;            /* n+1 */
    int32_t *ci;
    double *v;
    int32_t *gnode;         /* full-grid node id (x fastest) per unknown */
    int32_t *boxmap;        /* box node -> unknown index or -1 */
    int i0, i1, j0, j1, k0, k1;
} box_sys;

static int on_bnd(const geom *g, int i, int j, int k)
{
    return i == 0 || j == 0 || k == 0 || i == g->NX - 1 || j == g->NY - 1 || k == g->NZ - 1;
}

/* 1-D neighbour half-width: a vertex (even index) touches +-2, a mid node +-1. */
static int reach(int i) { return (i % 2 == 0) ? 2 : 1; }

static int64_t find_col(const box_sys *S, int64_t row, int32_t col)
{
    int64_t lo = S->rp[row], hi = S->rp[row + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (S->ci[mid] == col) return mid;
        if (S->ci[mid] < col) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/*
 * Pattern and stiffness of the elements [ex0,ex1) x [ey0,ey1) x [ez0,ez1).
 * Unknowns are the box nodes, minus outer-boundary nodes unless keep_bnd.
 * Two nodes are coupled when they share an element of the box.
 */
static int build_box(const geom *g, emat_cache *cache, int ex0, int ex1, int ey0, int ey1,
                     int ez0, int ez1, int keep_bnd, box_sys *S)
{
    S->i0 = 2 * ex0; S->i1 = 2 * ex1; S->j0 = 2 * ey0; S->j1 = 2 * ey1;
    S->k0 = 2 * ez0; S->k1 = 2 * ez1;
    int bx = S->i1 - S->i0 + 1, by = S->j1 - S->j0 + 1, bz = S->k1 - S->k0 + 1;
    int64_t nbox = (int64_t)bx * by * bz;
    S->boxmap = malloc(sizeof(int32_t) * nbox);
    int64_t n = 0;
    for (int k = S->k0; k <= S->k1; ++k)
    for (int j = S->j0; j <= S->j1; ++j)
    for (int i = S->i0; i <= S->i1; ++i) {
        int64_t bi = (i - S->i0) + (int64_t)bx * ((j - S->j0) + (int64_t)by * (k - S->k0));
        S->boxmap[bi] = (keep_bnd || !on_bnd(g, i, j, k)) ? (int32_t)(n++) : -1;
    }
    S->n = n;
    S->gnode = malloc(sizeof(int32_t) * (n ? n : 1));
    S->rp = malloc(sizeof(int64_t) * (n + 1));
    /* count */
    S->rp[0] = 0;
    int64_t r = 0;
    for (int k = S->k0; k <= S->k1; ++k)
    for (int j = S->j0; j <= S->j1; ++j)
    for (int i = S->i0; i <= S->i1; ++i) {
        int64_t bi = (i - S->i0) + (int64_t)bx * ((j - S->j0) + (int64_t)by * (k - S->k0));
        if (S->boxmap[bi] < 0) continue;
        int64_t cnt = 0;
        for (int kk = k - reach(k); kk <= k + reach(k); ++kk)
        for (int jj = j - reach(j); jj <= j + reach(j); ++jj)
        for (int ii = i - reach(i); ii <= i + reach(i); ++ii) {
            if (ii < S->i0 || ii > S->i1 || jj < S->j0 || jj > S->j1 || kk < S->k0 || kk > S->k1) continue;
            int64_t bj = (ii - S->i0) + (int64_t)bx * ((jj - S->j0) + (int64_t)by * (kk - S->k0));
            if (S->boxmap[bj] >= 0) cnt++;
        }
        S->gnode[r] = i + g->NX * (j + g->NY * k);
        S->rp[r + 1] = S->rp[r] + cnt;
        r++;
    }
    int64_t nnz = S->rp[n];
    S->ci = malloc(sizeof(int32_t) * (nnz ? nnz : 1));
    S->v = calloc(nnz ? nnz : 1, sizeof(double));
    r = 0;
    for (int k = S->k0; k <= S->k1; ++k)
    for (int j = S->j0; j <= S->j1; ++j)
    for (int i = S->i0; i <= S->i1; ++i) {
        int64_t bi = (i - S->i0) + (int64_t)bx * ((j - S->j0) + (int64_t)by * (k - S->k0));
        if (S->boxmap[bi] < 0) continue;
        int64_t pos = S->rp[r];
        for (int kk = k - reach(k); kk <= k + reach(k); ++kk)
        for (int jj = j - reach(j); jj <= j + reach(j); ++jj)
        for (int ii = i - reach(i); ii <= i + reach(i); ++ii) {
            if (ii < S->i0 || ii > S->i1 || jj < S->j0 || jj > S->j1 || kk < S->k0 || kk > S->k1) continue;
            int64_t bj = (ii - S->i0) + (int64_t)bx * ((jj - S->j0) + (int64_t)by * (kk - S->k0));
            if (S->boxmap[bj] >= 0) S->ci[pos++] = S->boxmap[bj];
        }
        r++;
    }
    /* element loop: scatter 27x27 stiffness blocks */
    for (int ez = ez0; ez < ez1; ++ez)
    for (int ey = ey0; ey < ey1; ++ey)
    for (int ex = ex0; ex < ex1; ++ex) {
        const double *Ke = cache_get(cache, g->xc[ex + 1] - g->xc[ex], g->yc[ey + 1] - g->yc[ey],
                                     g->zc[ez + 1] - g->zc[ez], 0);
        int32_t loc[27];
        for (int I = 0; I < 27; ++I) {
            int i = 2 * ex + I % 3, j = 2 * ey + (I / 3) % 3, k = 2 * ez + I / 9;
            int64_t bi = (i - S->i0) + (int64_t)bx * ((j - S->j0) + (int64_t)by * (k - S->k0));
            loc[I] = S->boxmap[bi];
        }
        for (int I = 0; I < 27; ++I) {
            if (loc[I] < 0) continue;
            for (int J = 0; J < 27; ++J) {
                if (loc[J] < 0) continue;
                int64_t pos = find_col(S, loc[I], loc[J]);
                if (pos < 0) return -1;   /* pattern bug */
                S->v[pos] += Ke[I * 27 + J];
            }
        }
    }
    return 0;
}

static void box_free(box_sys *S)
{
    free(S->rp); free(S->ci); free(S->v); free(S->gnode); free(S->boxmap);
    memset(S, 0, sizeof(*S));
}

static int64_t box_index(const box_sys *S, int i, int j, int k)
{
    if (i < S->i0 || i > S->i1 || j < S->j0 || j > S->j1 || k < S->k0 || k > S->k1) return -1;
    int bx = S->i1 - S->i0 + 1, by = S->j1 - S->j0 + 1;
    return S->boxmap[(i - S->i0) + (int64_t)bx * ((j - S->j0) + (int64_t)by * (k - S->k0))];
}

/* Load of per-element constant density: f_I += 4 pi G drho_e int phi_I. */
static void box_load_const(const geom *g, emat_cache *cache, const box_sys *S, int ex0, int ex1,
                           int ey0, int ey1, int ez0, int ez1, const double *drho, double *f)
{
    memset(f, 0, sizeof(double) * S->n);
    for (int ez = ez0; ez < ez1; ++ez)
    for (int ey = ey0; ey < ey1; ++ey)
    for (int ex = ex0; ex < ex1; ++ex) {
        double rho = drho[ex + (int64_t)g->nx * (ey + (int64_t)g->ny * ez)];
        if (rho == 0.0) continue;
        const double *we = cache_get(cache, g->xc[ex + 1] - g->xc[ex], g->yc[ey + 1] - g->yc[ey],
                                     g->zc[ez + 1] - g->zc[ez], 2);
        for (int I = 0; I < 27; ++I) {
            int64_t l = box_index(S, 2 * ex + I % 3, 2 * ey + (I / 3) % 3, 2 * ez + I / 9);
            if (l >= 0) f[l] += 4.0 * ORC_PI * ORC_G * rho * we[I];
        }
    }
}

static void geom_init(geom *g, int nx, int ny, int nz, const double *xc, const double *yc, const double *zc)
{
    g->nx = nx; g->ny = ny; g->nz = nz;
    g->xc = malloc(sizeof(double) * (nx + 1)); memcpy(g->xc, xc, sizeof(double) * (nx + 1));
    g->yc = malloc(sizeof(double) * (ny + 1)); memcpy(g->yc, yc, sizeof(double) * (ny + 1));
    g->zc = malloc(sizeof(double) * (nz + 1)); memcpy(g->zc, zc, sizeof(double) * (nz + 1));
    g->NX = 2 * nx + 1; g->NY = 2 * ny + 1; g->NZ = 2 * nz + 1;
}

static void geom_free(geom *g) { free(g->xc); free(g->yc); free(g->zc); }

/* ------------------------------------------------------------------------ */
/* Global system (exported for tests)                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    geom g;
    box_sys S;
    double *f;
} orc_global;

/* Assemble K (and the constant-density load if drho != NULL) on the whole mesh.
 * keep_bnd = 0 eliminates the Dirichlet nodes; 1 keeps every node. */
orc_global *orc_global_create(int nx, int ny, int nz, const double *xc, const double *yc,
                              const double *zc, const double *drho, int keep_bnd)
{
    orc_global *G = calloc(1, sizeof(orc_global));
    geom_init(&G->g, nx, ny, nz, xc, yc, zc);
    emat_cache cache = {0};
    if (build_box(&G->g, &cache, 0, nx, 0, ny, 0, nz, keep_bnd, &G->S) != 0) {
        cache_free(&cache); return NULL;
    }
    G->f = calloc(G->S.n ? G->S.n : 1, sizeof(double));
    if (drho) box_load_const(&G->g, &cache, &G->S, 0, nx, 0, ny, 0, nz, drho, G->f);
    cache_free(&cache);
    return G;
}

int64_t orc_global_n(const orc_global *G) { return G->S.n; }
int64_t orc_global_nnz(const orc_global *G) { return G->S.rp[G->S.n]; }

/* Copy out CSR arrays, load and the node id of each unknown. */
void orc_global_export(const orc_global *G, int64_t *rp, int32_t *ci, double *v, double *f, int32_t *gnode)
{
    int64_t n = G->S.n, nnz = G->S.rp[n];
    if (rp) memcpy(rp, G->S.rp, sizeof(int64_t) * (n + 1));
    if (ci) memcpy(ci, G->S.ci, sizeof(int32_t) * nnz);
    if (v) memcpy(v, G->S.v, sizeof(double) * nnz);
    if (f) memcpy(f, G->f, sizeof(double) * n);
    if (gnode) memcpy(gnode, G->S.gnode, sizeof(int32_t) * n);
}

/* Load from a general source sampled at the Gauss points (fq[e*27+q]):
 * f_I = sum_e sum_q W_q fq phi_I(q).  Used for manufactured solutions. */
void orc_global_load_gauss(const orc_global *G, const double *fq, double *f)
{
    const geom *g = &G->g;
    double pt[3], wt[3];
    gauss3(pt, wt);
    memset(f, 0, sizeof(double) * G->S.n);
    for (int ez = 0; ez < g->nz; ++ez)
    for (int ey = 0; ey < g->ny; ++ey)
    for (int ex = 0; ex < g->nx; ++ex) {
        int64_t e = ex + (int64_t)g->nx * (ey + (int64_t)g->ny * ez);
        double hx = g->xc[ex + 1] - g->xc[ex], hy = g->yc[ey + 1] - g->yc[ey], hz = g->zc[ez + 1] - g->zc[ez];
        for (int q = 0; q < 27; ++q) {
            int qa = q % 3, qb = (q / 3) % 3, qc = q / 9;
            double W = wt[qa] * wt[qb] * wt[qc] * hx * hy * hz * fq[e * 27 + q];
            double fx[3], dx[3], fy[3], dy[3], fz[3], dz[3];
            orc_basis_1d(pt[qa], fx, dx); orc_basis_1d(pt[qb], fy, dy); orc_basis_1d(pt[qc], fz, dz);
            for (int I = 0; I < 27; ++I) {
                int64_t l = box_index(&G->S, 2 * ex + I % 3, 2 * ey + (I / 3) % 3, 2 * ez + I / 9);
                if (l >= 0) f[l] += W * fx[I % 3] * fy[(I / 3) % 3] * fz[I / 9];
            }
        }
    }
}

void orc_global_destroy(orc_global *G)
{
    if (!G) return;
    box_free(&G->S); free(G->f); geom_free(&G->g); free(G);
}

/* ------------------------------------------------------------------------ */
/* CSR kernels and Jacobi PCG (Sec. 6)                                      */
/* ------------------------------------------------------------------------ */
void orc_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *x, double *y)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
        y[i] = s;
    }
}

static void spmv_serial(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/*
 * Jacobi PCG on A x = b from the initial guess in x.  Stops when
 * ||b - A x||_2 <= tol ||b||_2 (recursive residual), checked before the first
 * iteration and after each one.  Returns the iteration count, or -1 on a
 * breakdown (p.Ap <= 0 or not finite), or -2 when maxit is reached.
 * parallel != 0 uses the OpenMP SpMV (row sums are unchanged).
 */
static int pcg_impl(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *b,
                    double *x, double tol, int maxit, double *relres, int parallel)
{
    double *r = malloc(sizeof(double) * (n ? n : 1)), *z = malloc(sizeof(double) * (n ? n : 1));
    double *p = malloc(sizeof(double) * (n ? n : 1)), *q = malloc(sizeof(double) * (n ? n : 1));
    double *dinv = malloc(sizeof(double) * (n ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) if (ci[k] == i) d = v[k];
        dinv[i] = 1.0 / d;
    }
    if (parallel) orc_spmv(n, rp, ci, v, x, q); else spmv_serial(n, rp, ci, v, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    double bb = dot(n, b, b), rr = dot(n, r, r);
    int it = 0, status = 0;
    if (!(rr <= tol * tol * bb)) {
        for (int64_t i = 0; i < n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
        double rho = dot(n, r, z);
        for (;;) {
            if (it >= maxit) { status = -2; break; }
            if (parallel) orc_spmv(n, rp, ci, v, p, q); else spmv_serial(n, rp, ci, v, p, q);
            double pq = dot(n, p, q);
            if (!(pq > 0.0) || !isfinite(pq)) { status = -1; break; }
            double alpha = rho / pq;
            for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
            ++it;
            rr = dot(n, r, r);
            if (rr <= tol * tol * bb) break;
            for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
            double rho_new = dot(n, r, z);
            double beta = rho_new / rho;
            rho = rho_new;
            for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
    }
    if (relres) *relres = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
    free(r); free(z); free(p); free(q); free(dinv);
    return status ? status : it;
}

int orc_pcg(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *b,
            double *x, double tol, int maxit, double *relres)
{
    return pcg_impl(n, rp, ci, v, b, x, tol, maxit, relres, 1);
}

/* ------------------------------------------------------------------------ */
/* Sequential (Jacobi-type) optimized Schwarz, Sec. 3                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int s, t;               /* the two subdomains, s < t */
    int axis;               /* normal direction 0/1/2 */
    int64_t n;              /* face unknowns */
    int32_t *loc_s, *loc_t; /* local unknown index on each side */
    int64_t *rp; int32_t *ci; double *m;   /* face mass, face-node CSR */
    double *sv;                /* face tangential stiffness, same CSR */
    double ps, qs, pt, qt;     /* transmission coefficients of side s and side t */
    double *lam_st, *lam_ts;   /* Robin data received by s (from t) and by t (from s) */
} orc_face;

typedef struct {
    box_sys S;              /* A_s = K_s + p_s M_Gs in S.v */
    double *f, *b, *u;
    double p;
    int ex0, ex1, ey0, ey1, ez0, ez1;
    int last_iters;
    double last_relres;
} orc_sub;

typedef struct {
    geom g;
    int sx, sy, sz, nsub, nface;
    orc_sub *sub;
    orc_face *face;
    box_sys KG;             /* global stiffness (Dirichlet eliminated) */
    double *fG, fnorm;
    int32_t *gunk;          /* full-grid node -> global unknown or -1 */
    double *ubar, *work;
    int32_t *ncopy;
    int status;             /* worst local PCG status of the last iteration */
} orc_sz;

/*
 * Face between subdomains s and t, normal to `axis`, at node plane `plane`;
 * in-plane node ranges [a0,a1] x [b0,b1] of the two tangential directions.
 */
static void face_build(orc_sz *Z, orc_face *F, int s, int t, int axis, int plane,
                       int a0, int a1, int b0, int b1)
{
    const geom *g = &Z->g;
    F->s = s; F->t = t; F->axis = axis;
    int na = a1 - a0 + 1, nb = b1 - b0 + 1;
    int32_t *fmap = malloc(sizeof(int32_t) * na * nb);
    int64_t n = 0;
    /* tangential directions: axis 0 -> (y,z), 1 -> (x,z), 2 -> (x,y) */
    for (int b = b0; b <= b1; ++b)
    for (int a = a0; a <= a1; ++a) {
        int i, j, k;
        if (axis == 0) { i = plane; j = a; k = b; }
        else if (axis == 1) { i = a; j = plane; k = b; }
        else { i = a; j = b; k = plane; }
        fmap[(a - a0) + na * (b - b0)] = on_bnd(g, i, j, k) ? -1 : (int32_t)(n++);
    }
    F->n = n;
    F->loc_s = malloc(sizeof(int32_t) * (n ? n : 1));
    F->loc_t = malloc(sizeof(int32_t) * (n ? n : 1));
    F->lam_st = calloc(n ? n : 1, sizeof(double));
    F->lam_ts = calloc(n ? n : 1, sizeof(double));
    F->rp = malloc(sizeof(int64_t) * (n + 1));
    F->rp[0] = 0;
    int64_t r = 0;
    for (int b = b0; b <= b1; ++b)
    for (int a = a0; a <= a1; ++a) {
        if (fmap[(a - a0) + na * (b - b0)] < 0) continue;
        int i, j, k;
        if (axis == 0) { i = plane; j = a; k = b; }
        else if (axis == 1) { i = a; j = plane; k = b; }
        else { i = a; j = b; k = plane; }
        F->loc_s[r] = (int32_t)box_index(&Z->sub[s].S, i, j, k);
        F->loc_t[r] = (int32_t)box_index(&Z->sub[t].S, i, j, k);
        int64_t cnt = 0;
        for (int bb = b - reach(b); bb <= b + reach(b); ++bb)
        for (int aa = a - reach(a); aa <= a + reach(a); ++aa)
            if (aa >= a0 && aa <= a1 && bb >= b0 && bb <= b1 && fmap[(aa - a0) + na * (bb - b0)] >= 0) cnt++;
        F->rp[r + 1] = F->rp[r] + cnt;
        r++;
    }
    F->ci = malloc(sizeof(int32_t) * (F->rp[n] ? F->rp[n] : 1));
    F->m = calloc(F->rp[n] ? F->rp[n] : 1, sizeof(double));
    F->sv = calloc(F->rp[n] ? F->rp[n] : 1, sizeof(double));
    r = 0;
    for (int b = b0; b <= b1; ++b)
    for (int a = a0; a <= a1; ++a) {
        if (fmap[(a - a0) + na * (b - b0)] < 0) continue;
        int64_t pos = F->rp[r];
        for (int bb = b - reach(b); bb <= b + reach(b); ++bb)
        for (int aa = a - reach(a); aa <= a + reach(a); ++aa)
            if (aa >= a0 && aa <= a1 && bb >= b0 && bb <= b1 && fmap[(aa - a0) + na * (bb - b0)] >= 0)
                F->ci[pos++] = fmap[(aa - a0) + na * (bb - b0)];
        r++;
    }
    /* face-element loop (2-D elements of the face) */
    const double *ca = axis == 0 ? g->yc : g->xc;
    const double *cb = axis == 2 ? g->yc : g->zc;
    for (int eb = b0 / 2; eb < b1 / 2; ++eb)
    for (int ea = a0 / 2; ea < a1 / 2; ++ea) {
        double Mf[81], Sf[81];
        orc_face_element(ca[ea + 1] - ca[ea], cb[eb + 1] - cb[eb], Mf);
        orc_face_stiffness(ca[ea + 1] - ca[ea], cb[eb + 1] - cb[eb], Sf);
        int32_t loc[9];
        for (int I = 0; I < 9; ++I) {
            int a = 2 * ea + I % 3, b = 2 * eb + I / 3;
            loc[I] = fmap[(a - a0) + na * (b - b0)];
        }
        for (int I = 0; I < 9; ++I) {
            if (loc[I] < 0) continue;
            for (int J = 0; J < 9; ++J) {
                if (loc[J] < 0) continue;
                int64_t pos = -1;
                for (int64_t k = F->rp[loc[I]]; k < F->rp[loc[I] + 1]; ++k)
                    if (F->ci[k] == loc[J]) pos = k;
                F->m[pos] += Mf[I * 9 + J];
                F->sv[pos] += Sf[I * 9 + J];
            }
        }
    }
    free(fmap);
}

/* Add the weak transmission operator p M_face + q S_face of side `which`
 * (0 = s, 1 = t) into that side's local matrix. */
static void face_add_robin(orc_sz *Z, const orc_face *F, int which)
{
    orc_sub *U = &Z->sub[which ? F->t : F->s];
    const int32_t *loc = which ? F->loc_t : F->loc_s;
    const double p = which ? F->pt : F->ps, q = which ? F->qt : F->qs;
    for (int64_t r = 0; r < F->n; ++r)
        for (int64_t k = F->rp[r]; k < F->rp[r + 1]; ++k) {
            int64_t pos = find_col(&U->S, loc[r], loc[F->ci[k]]);
            U->S.v[pos] += p * F->m[k] + q * F->sv[k];
        }
}

/* face apply: y = M_face x|face and ys = S_face x|face */
static void face_apply(const orc_face *F, const double *u, const int32_t *loc, double *y, double *ys)
{
    for (int64_t r = 0; r < F->n; ++r) {
        double acc = 0.0, accs = 0.0;
        for (int64_t k = F->rp[r]; k < F->rp[r + 1]; ++k) {
            acc += F->m[k] * u[loc[F->ci[k]]];
            accs += F->sv[k] * u[loc[F->ci[k]]];
        }
        y[r] = acc;
        ys[r] = accs;
    }
}

/*
 * Build the decomposition.  cx/cy/cz are element-index cuts (s+1 entries,
 * first 0, last n).  Transmission coefficients: with tc == NULL subdomain s
 * uses the Robin parameter p_sub[s] on all its faces (q = 0); otherwise every
 * face uses tc = {p_lo, q_lo, p_hi, q_hi}: (p_lo, q_lo) in the condition of
 * the subdomain on the lower side of the face (smaller coordinate along the
 * normal), (p_hi, q_hi) in that of the upper side.
 */
static orc_sz *sz_create(int nx, int ny, int nz, const double *xc, const double *yc, const double *zc,
                         const double *drho, int sx, int sy, int sz, const int32_t *cx,
                         const int32_t *cy, const int32_t *cz, const double *p_sub, const double *tc)
{
    orc_sz *Z = calloc(1, sizeof(orc_sz));
    geom_init(&Z->g, nx, ny, nz, xc, yc, zc);
    Z->sx = sx; Z->sy = sy; Z->sz = sz; Z->nsub = sx * sy * sz;
    Z->sub = calloc(Z->nsub, sizeof(orc_sub));
    emat_cache cache = {0};
    int bad = 0;
    #pragma omp parallel for schedule(dynamic) reduction(|:bad)
    for (int s = 0; s < Z->nsub; ++s) {
        emat_cache lc = {0};
        int a = s % sx, b = (s / sx) % sy, c = s / (sx * sy);
        orc_sub *U = &Z->sub[s];
        U->ex0 = cx[a]; U->ex1 = cx[a + 1]; U->ey0 = cy[b]; U->ey1 = cy[b + 1];
        U->ez0 = cz[c]; U->ez1 = cz[c + 1];
        U->p = p_sub ? p_sub[s] : 0.0;
        if (build_box(&Z->g, &lc, U->ex0, U->ex1, U->ey0, U->ey1, U->ez0, U->ez1, 0, &U->S)) bad |= 1;
        int64_t n = U->S.n ? U->S.n : 1;
        U->f = calloc(n, sizeof(double)); U->b = calloc(n, sizeof(double)); U->u = calloc(n, sizeof(double));
        box_load_const(&Z->g, &lc, &U->S, U->ex0, U->ex1, U->ey0, U->ey1, U->ez0, U->ez1, drho, U->f);
        cache_free(&lc);
    }
    if (bad) { cache_free(&cache); return NULL; }
    /* faces: x-normal, then y-normal, then z-normal */
    int maxf = (sx - 1) * sy * sz + sx * (sy - 1) * sz + sx * sy * (sz - 1);
    Z->face = calloc(maxf ? maxf : 1, sizeof(orc_face));
    int nf = 0;
    for (int c = 0; c < sz; ++c) for (int b = 0; b < sy; ++b) for (int a = 0; a + 1 < sx; ++a) {
        int s = a + sx * (b + sy * c), t = s + 1;
        face_build(Z, &Z->face[nf++], s, t, 0, 2 * cx[a + 1], 2 * cy[b], 2 * cy[b + 1], 2 * cz[c], 2 * cz[c + 1]);
    }
    for (int c = 0; c < sz; ++c) for (int b = 0; b + 1 < sy; ++b) for (int a = 0; a < sx; ++a) {
        int s = a + sx * (b + sy * c), t = s + sx;
        face_build(Z, &Z->face[nf++], s, t, 1, 2 * cy[b + 1], 2 * cx[a], 2 * cx[a + 1], 2 * cz[c], 2 * cz[c + 1]);
    }
    for (int c = 0; c + 1 < sz; ++c) for (int b = 0; b < sy; ++b) for (int a = 0; a < sx; ++a) {
        int s = a + sx * (b + sy * c), t = s + sx * sy;
        face_build(Z, &Z->face[nf++], s, t, 2, 2 * cz[c + 1], 2 * cx[a], 2 * cx[a + 1], 2 * cy[b], 2 * cy[b + 1]);
    }
    Z->nface = nf;
    for (int f = 0; f < nf; ++f) {
        orc_face *F = &Z->face[f];
        if (tc) { F->ps = tc[0]; F->qs = tc[1]; F->pt = tc[2]; F->qt = tc[3]; }
        else { F->ps = Z->sub[F->s].p; F->qs = 0.0; F->pt = Z->sub[F->t].p; F->qt = 0.0; }
        face_add_robin(Z, F, 0);
        face_add_robin(Z, F, 1);
    }
    /* global system for the stop test */
    if (build_box(&Z->g, &cache, 0, nx, 0, ny, 0, nz, 0, &Z->KG)) { cache_free(&cache); return NULL; }
    Z->fG = calloc(Z->KG.n ? Z->KG.n : 1, sizeof(double));
    box_load_const(&Z->g, &cache, &Z->KG, 0, nx, 0, ny, 0, nz, drho, Z->fG);
    cache_free(&cache);
    Z->fnorm = sqrt(dot(Z->KG.n, Z->fG, Z->fG));
    int64_t nn = (int64_t)Z->g.NX * Z->g.NY * Z->g.NZ;
    Z->gunk = malloc(sizeof(int32_t) * nn);
    for (int64_t i = 0; i < nn; ++i) Z->gunk[i] = -1;
    for (int64_t r = 0; r < Z->KG.n; ++r) Z->gunk[Z->KG.gnode[r]] = (int32_t)r;
    Z->ubar = calloc(Z->KG.n ? Z->KG.n : 1, sizeof(double));
    Z->work = calloc(Z->KG.n ? Z->KG.n : 1, sizeof(double));
    Z->ncopy = calloc(Z->KG.n ? Z->KG.n : 1, sizeof(int32_t));
    for (int s = 0; s < Z->nsub; ++s)
        for (int64_t r = 0; r < Z->sub[s].S.n; ++r) Z->ncopy[Z->gunk[Z->sub[s].S.gnode[r]]]++;
    return Z;
}

orc_sz *orc_sz_create(int nx, int ny, int nz, const double *xc, const double *yc, const double *zc,
                      const double *drho, int sx, int sy, int sz, const int32_t *cx,
                      const int32_t *cy, const int32_t *cz, const double *p_sub)
{
    return sz_create(nx, ny, nz, xc, yc, zc, drho, sx, sy, sz, cx, cy, cz, p_sub, NULL);
}

orc_sz *orc_sz_create_tc(int nx, int ny, int nz, const double *xc, const double *yc, const double *zc,
                         const double *drho, int sx, int sy, int sz, const int32_t *cx,
                         const int32_t *cy, const int32_t *cz, const double *tc)
{
    return sz_create(nx, ny, nz, xc, yc, zc, drho, sx, sy, sz, cx, cy, cz, NULL, tc);
}

int orc_sz_nsub(const orc_sz *Z) { return Z->nsub; }
int orc_sz_nface(const orc_sz *Z) { return Z->nface; }
int64_t orc_sz_global_n(const orc_sz *Z) { return Z->KG.n; }
int64_t orc_sz_sub_n(const orc_sz *Z, int s) { return Z->sub[s].S.n; }
int64_t orc_sz_sub_nnz(const orc_sz *Z, int s) { return Z->sub[s].S.rp[Z->sub[s].S.n]; }
int orc_sz_status(const orc_sz *Z) { return Z->status; }

void orc_sz_face_info(const orc_sz *Z, int f, int32_t *s, int32_t *t, int32_t *axis, int64_t *n)
{
    *s = Z->face[f].s; *t = Z->face[f].t; *axis = Z->face[f].axis; *n = Z->face[f].n;
}

/* side 0: data received by s (lam_st); side 1: received by t (lam_ts). */
void orc_sz_get_lambda(const orc_sz *Z, int f, int side, double *out)
{
    const orc_face *F = &Z->face[f];
    memcpy(out, side ? F->lam_ts : F->lam_st, sizeof(double) * F->n);
}

void orc_sz_set_lambda(orc_sz *Z, int f, int side, const double *in)
{
    orc_face *F = &Z->face[f];
    memcpy(side ? F->lam_ts : F->lam_st, in, sizeof(double) * F->n);
}

/* Face node full-grid ids (side-independent) and face mass CSR export. */
void orc_sz_face_export(const orc_sz *Z, int f, int32_t *gnode, int64_t *rp, int32_t *ci, double *m)
{
    const orc_face *F = &Z->face[f];
    for (int64_t r = 0; r < F->n; ++r) gnode[r] = Z->sub[F->s].S.gnode[F->loc_s[r]];
    if (rp) memcpy(rp, F->rp, sizeof(int64_t) * (F->n + 1));
    if (ci) memcpy(ci, F->ci, sizeof(int32_t) * F->rp[F->n]);
    if (m) memcpy(m, F->m, sizeof(double) * F->rp[F->n]);
}

/* Face tangential stiffness values (same CSR as the face mass). */
void orc_sz_face_stiffness_export(const orc_sz *Z, int f, double *sv)
{
    const orc_face *F = &Z->face[f];
    memcpy(sv, F->sv, sizeof(double) * F->rp[F->n]);
}

/* Local system export: A_s = K_s + p_s M_Gs (CSR), f_s, node ids. */
void orc_sz_sub_export(const orc_sz *Z, int s, int64_t *rp, int32_t *ci, double *v, double *f,
                       int32_t *gnode, double *u)
{
    const orc_sub *U = &Z->sub[s];
    int64_t n = U->S.n, nnz = U->S.rp[n];
    if (rp) memcpy(rp, U->S.rp, sizeof(int64_t) * (n + 1));
    if (ci) memcpy(ci, U->S.ci, sizeof(int32_t) * nnz);
    if (v) memcpy(v, U->S.v, sizeof(double) * nnz);
    if (f) memcpy(f, U->f, sizeof(double) * n);
    if (gnode) memcpy(gnode, U->S.gnode, sizeof(int32_t) * n);
    if (u) memcpy(u, U->u, sizeof(double) * n);
}

void orc_sz_set_rhs(orc_sz *Z, int s, const double *f)
{
    memcpy(Z->sub[s].f, f, sizeof(double) * Z->sub[s].S.n);
}

void orc_sz_set_global_rhs(orc_sz *Z, const double *fG)
{
    memcpy(Z->fG, fG, sizeof(double) * Z->KG.n);
    Z->fnorm = sqrt(dot(Z->KG.n, Z->fG, Z->fG));
}

/*
 * One Schwarz iteration: b_s = f_s + sum lam; local Jacobi PCG from the
 * previous u_s to tol (relative to ||b_s||); then the parallel exchange
 *   lam_st <- (p_s + p_t) M u_t + (q_s + q_t) S u_t - lam_ts,
 *   lam_ts <- (p_s + p_t) M u_s + (q_s + q_t) S u_s - lam_st
 * (the weak normal flux of the neighbour, -lam + (p M + q S) u, plus the
 * receiving side's own transmission operator applied to the neighbour's
 * trace).
 * Local PCG iteration counts are written to iters_sub (may be NULL).
 */
void orc_sz_iterate(orc_sz *Z, double tol, int maxit, int32_t *iters_sub)
{
    for (int s = 0; s < Z->nsub; ++s) memcpy(Z->sub[s].b, Z->sub[s].f, sizeof(double) * Z->sub[s].S.n);
    for (int f = 0; f < Z->nface; ++f) {
        orc_face *F = &Z->face[f];
        for (int64_t r = 0; r < F->n; ++r) {
            Z->sub[F->s].b[F->loc_s[r]] += F->lam_st[r];
            Z->sub[F->t].b[F->loc_t[r]] += F->lam_ts[r];
        }
    }
    int worst = 0;
    #pragma omp parallel for schedule(dynamic) reduction(min:worst)
    for (int s = 0; s < Z->nsub; ++s) {
        orc_sub *U = &Z->sub[s];
        int it = pcg_impl(U->S.n, U->S.rp, U->S.ci, U->S.v, U->b, U->u, tol, maxit, &U->last_relres, 0);
        U->last_iters = it;
        if (it < worst) worst = it;
    }
    Z->status = worst;
    if (iters_sub) for (int s = 0; s < Z->nsub; ++s) iters_sub[s] = Z->sub[s].last_iters;
    for (int f = 0; f < Z->nface; ++f) {
        orc_face *F = &Z->face[f];
        int64_t nb = F->n ? F->n : 1;
        double *mu_t = malloc(sizeof(double) * nb), *su_t = malloc(sizeof(double) * nb);
        double *mu_s = malloc(sizeof(double) * nb), *su_s = malloc(sizeof(double) * nb);
        face_apply(F, Z->sub[F->t].u, F->loc_t, mu_t, su_t);
        face_apply(F, Z->sub[F->s].u, F->loc_s, mu_s, su_s);
        double pp = F->ps + F->pt, qq = F->qs + F->qt;
        for (int64_t r = 0; r < F->n; ++r) {
            double new_st = pp * mu_t[r] + qq * su_t[r] - F->lam_ts[r];
            double new_ts = pp * mu_s[r] + qq * su_s[r] - F->lam_st[r];
            F->lam_st[r] = new_st;
            F->lam_ts[r] = new_ts;
        }
        free(mu_t); free(su_t); free(mu_s); free(su_s);
    }
}

/*
 * Stop test: ubar = average of the subdomain copies, r = f - K ubar,
 * returns ||r|| / ||f|| (||r|| if f = 0).  phi (full node grid, may be NULL)
 * receives ubar with zeros on the outer boundary.
 */
double orc_sz_residual(orc_sz *Z, double *phi)
{
    memset(Z->ubar, 0, sizeof(double) * Z->KG.n);
    for (int s = 0; s < Z->nsub; ++s)
        for (int64_t r = 0; r < Z->sub[s].S.n; ++r)
            Z->ubar[Z->gunk[Z->sub[s].S.gnode[r]]] += Z->sub[s].u[r];
    for (int64_t i = 0; i < Z->KG.n; ++i) Z->ubar[i] /= (double)Z->ncopy[i];
    orc_spmv(Z->KG.n, Z->KG.rp, Z->KG.ci, Z->KG.v, Z->ubar, Z->work);
    double rr = 0.0;
    for (int64_t i = 0; i < Z->KG.n; ++i) { double d = Z->fG[i] - Z->work[i]; rr += d * d; }
    if (phi) {
        int64_t nn = (int64_t)Z->g.NX * Z->g.NY * Z->g.NZ;
        for (int64_t i = 0; i < nn; ++i) phi[i] = Z->gunk[i] >= 0 ? Z->ubar[Z->gunk[i]] : 0.0;
    }
    return Z->fnorm > 0.0 ? sqrt(rr) / Z->fnorm : sqrt(rr);
}

/* Full solve from u = 0, lam = 0.  Returns the number of Schwarz iterations
 * done; relres receives the last stop-test value; hist (may be NULL, length
 * max_outer) the residual after each iteration. */
int orc_sz_solve(orc_sz *Z, double tol, int max_inner, double rtol, int max_outer,
                 double *phi, double *relres, double *hist)
{
    for (int s = 0; s < Z->nsub; ++s) memset(Z->sub[s].u, 0, sizeof(double) * Z->sub[s].S.n);
    for (int f = 0; f < Z->nface; ++f) {
        memset(Z->face[f].lam_st, 0, sizeof(double) * Z->face[f].n);
        memset(Z->face[f].lam_ts, 0, sizeof(double) * Z->face[f].n);
    }
    int n = 0;
    double rel = INFINITY;
    while (n < max_outer) {
        orc_sz_iterate(Z, tol, max_inner, NULL);
        ++n;
        rel = orc_sz_residual(Z, phi);
        if (hist) hist[n - 1] = rel;
        if (rel <= rtol) break;
    }
    if (relres) *relres = rel;
    return n;
}

void orc_sz_destroy(orc_sz *Z)
{
    if (!Z) return;
    for (int s = 0; s < Z->nsub; ++s) {
        box_free(&Z->sub[s].S); free(Z->sub[s].f); free(Z->sub[s].b); free(Z->sub[s].u);
    }
    for (int f = 0; f < Z->nface; ++f) {
        orc_face *F = &Z->face[f];
        free(F->loc_s); free(F->loc_t); free(F->rp); free(F->ci); free(F->m); free(F->sv);
        free(F->lam_st); free(F->lam_ts);
    }
    free(Z->sub); free(Z->face);
    box_free(&Z->KG); free(Z->fG); free(Z->gunk); free(Z->ubar); free(Z->work); free(Z->ncopy);
    geom_free(&Z->g);
    free(Z);
}
