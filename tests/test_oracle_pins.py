"""Pins of the FP64 oracle against closed forms, textbook special cases and
the paper's own statements -- never against the oracle itself.

* Q2 1-D matrices and tensor-product structure (closed form textbook values).
* Q2 exactness: a solution inside the Q2 space is reproduced exactly.
* Convergence order on a smooth manufactured solution.
* PCG against a dense LAPACK solve on tiny meshes.
* Sphere potential (Sec. 2): Phi = G M / r outside, 2 pi G rho (R^2 - r^2/3)
  inside, with the exterior closed form imposed on the box boundary.
* Sec. 3: the converged Schwarz iterate equals the monolithic solve.
* Sec. 3: Robin contraction factor (p - D)/(p + D) per iteration of a
  Fourier mode, D the Dirichlet-to-Neumann symbol (k coth k for a slab of
  width 1, -> |k|), and convergence in two iterations when p = D.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import gen
import oracle

# Textbook 1-D Q2 matrices on an element of length h (nodes 0, h/2, h).
K1 = np.array([[7.0, -8.0, 1.0], [-8.0, 16.0, -8.0], [1.0, -8.0, 7.0]]) / 3.0
M1 = np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]]) / 30.0
W1 = np.array([1.0, 4.0, 1.0]) / 6.0


def k1(h): return K1 / h
def m1(h): return M1 * h


def test_basis_is_lagrange():
    for node, s in enumerate((0.0, 0.5, 1.0)):
        phi, _ = oracle.basis_1d(s)
        e = np.zeros(3)
        e[node] = 1.0
        assert np.allclose(phi, e, atol=1e-15)
    for s in np.linspace(0, 1, 7):
        phi, dphi = oracle.basis_1d(s)
        assert abs(phi.sum() - 1.0) < 1e-14 and abs(dphi.sum()) < 1e-13


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.3, 1.7, 0.05)])
def test_element_matrices_closed_form(h):
    hx, hy, hz = h
    K, M, w = oracle.element(hx, hy, hz)
    # node I = a + 3b + 9c: x fastest -> kron(z, kron(y, x))
    Kref = (np.kron(m1(hz), np.kron(m1(hy), k1(hx))) + np.kron(m1(hz), np.kron(k1(hy), m1(hx)))
            + np.kron(k1(hz), np.kron(m1(hy), m1(hx))))
    Mref = np.kron(m1(hz), np.kron(m1(hy), m1(hx)))
    wref = np.kron(W1 * hz, np.kron(W1 * hy, W1 * hx))
    scale = np.abs(Kref).max()
    assert np.abs(K - Kref).max() < 1e-13 * scale
    assert np.abs(M - Mref).max() < 1e-15 * max(1.0, np.abs(Mref).max())
    assert np.abs(w - wref).max() < 1e-15
    # invariants: constants are in the kernel of K, mass integrates 1 exactly
    assert np.abs(K.sum(axis=1)).max() < 1e-12 * scale
    assert abs(M.sum() - hx * hy * hz) < 1e-14
    assert abs(w.sum() - hx * hy * hz) < 1e-14
    assert np.allclose(K, K.T, atol=1e-14 * scale) and np.allclose(M, M.T)


def test_face_mass_closed_form():
    M = oracle.face_element(0.7, 0.2)
    assert np.abs(M - np.kron(m1(0.2), m1(0.7))).max() < 1e-15
    assert abs(M.sum() - 0.14) < 1e-15


def _graded(n, length, r):
    return gen.graded_coords(n, length, r)


def test_q2_exactness_on_graded_mesh():
    """Phi* = x(1-x) y(1-y) z(1-z) lies in the Q2 space and vanishes on the
    boundary; with the exact (Gauss) load of f = -Lap Phi*, the Galerkin
    solution equals Phi* at every node (Galerkin orthogonality)."""
    xc = np.linspace(0, 1, 5)
    yc = np.array([0.0, 0.1, 0.45, 0.5, 1.0])
    zc = _graded(4, 1.0, 1.3)
    G = oracle.GlobalSystem(xc, yc, zc)
    pts = oracle.gauss_points(xc, yc, zc)
    X, Y, Z = pts[..., 0], pts[..., 1], pts[..., 2]
    a, b, c = X * (1 - X), Y * (1 - Y), Z * (1 - Z)
    fq = 2.0 * (b * c + a * c + a * b)
    f = G.load_gauss(fq)
    u, it, rel = G.solve(f, tol=1e-14)
    nodes = _node_coords(xc, yc, zc)[G.gnode]
    exact = np.prod(nodes * (1 - nodes), axis=1)
    assert np.abs(u - exact).max() < 1e-12 * np.abs(exact).max()


def _node_coords(xc, yc, zc):
    def fine(c):
        out = np.empty(2 * len(c) - 1)
        out[0::2] = c
        out[1::2] = 0.5 * (c[:-1] + c[1:])
        return out
    fx, fy, fz = fine(xc), fine(yc), fine(zc)
    Z, Y, X = np.meshgrid(fz, fy, fx, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def test_manufactured_sine_convergence_order():
    """Phi = sin(pi x) sin(pi y) sin(pi z): the nodal error of Q2 decreases
    at least at order 3 under refinement."""
    errs = []
    for n in (4, 8, 16):
        xc = np.linspace(0, 1, n + 1)
        G = oracle.GlobalSystem(xc, xc, xc)
        pts = oracle.gauss_points(xc, xc, xc)
        s = np.sin(np.pi * pts)
        fq = 3 * np.pi ** 2 * s[..., 0] * s[..., 1] * s[..., 2]
        u, _, _ = G.solve(G.load_gauss(fq), tol=1e-14)
        nodes = _node_coords(xc, xc, xc)[G.gnode]
        exact = np.prod(np.sin(np.pi * nodes), axis=1)
        errs.append(np.abs(u - exact).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 3.0, (errs, orders)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_pcg_matches_dense_solve(n):
    prob = gen.layered_problem(n=n, s=1, seed=3, n_spheres=2)
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    A = G.to_scipy().toarray()
    assert np.allclose(A, A.T, rtol=0, atol=1e-14 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    u, _, _ = G.solve(tol=1e-14)
    ref = np.linalg.solve(A, G.f)
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)


def test_load_is_4piG_rho_times_volume():
    prob = gen.layered_problem(n=4, s=1, seed=1, n_spheres=3)
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho, keep_boundary=True)
    vol = 1.0 / 4 ** 3
    assert abs(G.f.sum() - 4 * np.pi * gen.G_NEWTON * prob.drho.sum() * vol) < 1e-12 * np.abs(G.f).sum()


def _sphere_fraction_density(n, R, rho, sub=8):
    """Per-element density rho * (volume fraction inside the sphere), by
    midpoint sub-sampling of each element (sub^3 points)."""
    t = (np.arange(n * sub) + 0.5) / (n * sub)
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    inside = ((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2 <= R * R).astype(np.float64)
    frac = inside.reshape(n, sub, n, sub, n, sub).mean(axis=(1, 3, 5))
    return rho * frac.ravel()


def _sphere_dirichlet_error(n, R=0.2, rho=300.0):
    """Free-space sphere (Sec. 2): impose Phi = G M / r on the box boundary
    and compare the interior with the closed forms G M / r outside and
    2 pi G rho (R^2 - r^2 / 3) inside."""
    xc = np.linspace(0, 1, n + 1)
    drho = _sphere_fraction_density(n, R, rho)
    G = oracle.GlobalSystem(xc, xc, xc, drho, keep_boundary=True)
    Gm = gen.G_NEWTON * (4.0 / 3.0) * np.pi * R ** 3 * rho
    nodes = _node_coords(xc, xc, xc)
    r = np.linalg.norm(nodes - 0.5, axis=1)
    on_b = np.any((nodes == 0.0) | (nodes == 1.0), axis=1)[G.gnode]
    A = G.to_scipy().tocsr()
    gB = Gm / r[G.gnode][on_b]
    I = np.where(~on_b)[0]
    B = np.where(on_b)[0]
    AII = A[I][:, I]
    rhs = G.f[I] - A[I][:, B] @ gB
    u, it, rel = oracle.pcg(AII.indptr, AII.indices, AII.data, rhs, tol=1e-13)
    rI = r[G.gnode][I]
    outside = rI > R + 0.1
    inside = rI < R - 0.08
    ext = Gm / rI[outside]
    inn = 2 * np.pi * gen.G_NEWTON * rho * (R ** 2 - rI[inside] ** 2 / 3.0)
    e_out = np.abs(u[outside] - ext).max() / ext.max()
    e_in = np.abs(u[inside] - inn).max() / inn.max()
    return e_out, e_in


def test_sphere_closed_form_and_refinement():
    res = [_sphere_dirichlet_error(n) for n in (8, 16, 32)]
    e_out = np.array([r[0] for r in res])
    e_in = np.array([r[1] for r in res])
    # discretisation error of the sphere (Q2 + piecewise-constant density)
    # shrinks monotonically under refinement and is small on the finest mesh
    # (measured: exterior ~h^3, interior ~h^2, the density's jump at r = R)
    assert np.all(e_out[:-1] / e_out[1:] > 3.0) and np.all(e_in[:-1] / e_in[1:] > 3.0), res
    assert e_out[-1] < 5e-4 and e_in[-1] < 1e-2, res


def test_schwarz_converges_to_monolithic_sphere():
    prob = gen.sphere_problem(16, 2, 10.0)
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    ref, _, _ = G.solve(tol=1e-14)
    S = oracle.Schwarz.from_problem(prob)
    phi, n, rel, hist = S.solve(inner_rtol=1e-12, rtol=1e-11)
    assert rel <= 1e-11
    refg = G.to_grid(ref)
    assert np.linalg.norm(phi - refg) <= 1e-10 * np.linalg.norm(refg)
    # Schwarz contraction: residual history is eventually monotone
    assert np.all(np.diff(hist[5:]) < 0)


def test_schwarz_uneven_graded_matches_monolithic():
    prob = gen.regional_problem(nx=12, ny=10, nz=8, sx=3, sy=2, sz=2, p=2.0, seed=4,
                                lx=10.0, ly=8.0, lz=3.0)
    assert len(set(np.diff(prob.cx))) > 1  # genuinely uneven
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    ref, _, _ = G.solve(tol=1e-14)
    S = oracle.Schwarz.from_problem(prob)
    phi, n, rel, _ = S.solve(inner_rtol=1e-13, rtol=1e-11, max_outer=3000)
    assert rel <= 1e-11
    refg = G.to_grid(ref)
    assert np.linalg.norm(phi - refg) <= 1e-9 * np.linalg.norm(refg)


def test_symmetry_of_sphere_solution():
    """Sphere at (0.5, 0.5, 0.6) on a symmetric mesh and decomposition:
    Phi is invariant under x -> 1-x, y -> 1-y and x <-> y."""
    prob = gen.sphere_problem(16, 2, 10.0)
    S = oracle.Schwarz.from_problem(prob)
    phi, n, rel, _ = S.solve(inner_rtol=1e-12, rtol=1e-10)
    P = phi.reshape(33, 33, 33)  # [z, y, x]
    scale = np.abs(P).max()
    assert np.abs(P - P[:, :, ::-1]).max() < 1e-9 * scale
    assert np.abs(P - P[:, ::-1, :]).max() < 1e-9 * scale
    assert np.abs(P - P.transpose(0, 2, 1)).max() < 1e-9 * scale
    # qualitative: positive potential, maximum near the sphere centre
    k, j, i = np.unravel_index(np.argmax(P), P.shape)
    assert P.max() > 0 and abs(i - 16) <= 1 and abs(j - 16) <= 1 and abs(k - 19) <= 3


def _two_slab(m, p0, p1):
    xc = np.linspace(0, 2, 2 * m + 1)
    yc = np.linspace(0, 1, m + 1)
    S = oracle.Schwarz(xc, yc, yc, np.zeros(2 * m ** 3), [0, m, 2 * m], [0, m], [0, m], [p0, p1])
    A, _, g, _ = S.sub_export(0)
    gf, Mf = S.face_export(0)
    A, Mf = A.toarray(), Mf.toarray()
    loc = {x: i for i, x in enumerate(g)}
    fi = np.array([loc[x] for x in gf])
    K = A.copy()
    K[np.ix_(fi, fi)] -= p0 * Mf
    ii = np.setdiff1d(np.arange(len(g)), fi)
    Sch = K[np.ix_(fi, fi)] - K[np.ix_(fi, ii)] @ np.linalg.solve(K[np.ix_(ii, ii)], K[np.ix_(ii, fi)])
    D, V = sla.eigh(Sch, Mf)
    return S, Mf, D, V


def test_dtn_symbol_is_k_coth_k():
    """Lowest Steklov eigenvalues of a unit-width slab approach k coth(k),
    k = pi sqrt(m^2 + n^2), at the Q2 rate (about h^4)."""
    ks = sorted(np.pi * np.hypot(a, b) for a in range(1, 5) for b in range(1, 5))
    cont = np.array([k / np.tanh(k) for k in ks[:4]])
    errs = []
    for m in (4, 8):
        _, _, D, _ = _two_slab(m, 1.0, 1.0)
        errs.append(np.abs(D[:4] - cont) / cont)
    assert errs[1].max() < 3e-3
    assert np.all(errs[0] / errs[1] > 8.0)


@pytest.mark.parametrize("p0,p1", [(3.0, 3.0), (1.5, 9.0)])
def test_robin_contraction_factor(p0, p1):
    """Sec. 3: each Schwarz iteration multiplies a DtN eigenmode of the
    interface data by (p_j - D)/(p_i + D); two iterations give the Fourier
    rate (p0 - D)(p1 - D)/((p0 + D)(p1 + D))."""
    S, Mf, D, V = _two_slab(4, p0, p1)
    for mode in (0, 3):
        g = V[:, mode]
        d = D[mode]
        S.set_lambda(0, 0, Mf @ g)       # datum received by subdomain 0
        S.set_lambda(0, 1, np.zeros_like(g))
        S.iterate(inner_rtol=1e-15)
        l_st, l_ts = S.get_lambda(0, 0), S.get_lambda(0, 1)
        f1 = (p1 - d) / (p0 + d)
        assert np.abs(l_st).max() < 1e-12 * np.abs(Mf @ g).max()
        assert np.abs(l_ts - f1 * (Mf @ g)).max() < 1e-10 * np.abs(Mf @ g).max()
        S.iterate(inner_rtol=1e-15)
        rate = (p0 - d) * (p1 - d) / ((p0 + d) * (p1 + d))
        assert np.abs(S.get_lambda(0, 0) - rate * (Mf @ g)).max() < 1e-10 * np.abs(Mf @ g).max()


def test_optimal_p_converges_in_two_iterations():
    """Sec. 3: with the exact DtN symbol as transmission operator the
    algorithm converges in two iterations; for one mode, p = D does it."""
    _, _, D, V = _two_slab(4, 1.0, 1.0)
    d = D[0]
    S, Mf, _, _ = _two_slab(4, d, d)
    g = V[:, 0]
    S.set_lambda(0, 0, Mf @ g)
    S.set_lambda(0, 1, 0.7 * (Mf @ g))
    S.iterate(inner_rtol=1e-15)
    S.iterate(inner_rtol=1e-15)
    for side in (0, 1):
        assert np.abs(S.get_lambda(0, side)).max() < 1e-10 * np.abs(Mf @ g).max()


def _assembled_1d_mass(c):
    """Assembled 1-D Q2 mass over the elements with vertex coordinates c."""
    n = len(c) - 1
    M = np.zeros((2 * n + 1, 2 * n + 1))
    for e in range(n):
        M[2 * e:2 * e + 3, 2 * e:2 * e + 3] += m1(c[e + 1] - c[e])
    return M


def test_face_mass_matches_tensor_product_on_graded_uneven_mesh():
    """Every interface face mass equals the Kronecker product of assembled
    1-D Q2 masses of its two tangential directions (non-square, graded face
    elements), restricted to the face's non-Dirichlet nodes."""
    prob = gen.regional_problem(nx=12, ny=10, nz=8, sx=3, sy=2, sz=2, p=2.0, seed=4,
                                lx=10.0, ly=8.0, lz=3.0)
    S = oracle.Schwarz.from_problem(prob)
    NX, NY = 2 * prob.nx + 1, 2 * prob.ny + 1
    cuts = (prob.cx, prob.cy, prob.cz)
    coords = (prob.xc, prob.yc, prob.zc)
    for f in range(S.nface):
        s, t, axis, n = S.face_info(f)
        g, Mf = S.face_export(f)
        ijk = np.stack([g % NX, (g // NX) % NY, g // (NX * NY)], axis=1)
        tang = [d for d in range(3) if d != axis]
        sub_idx = (s % 3, (s // 3) % 2, s // 6)
        blocks = []
        for d in tang:
            lo, hi = cuts[d][sub_idx[d]], cuts[d][sub_idx[d] + 1]
            blocks.append((2 * lo, _assembled_1d_mass(coords[d][lo:hi + 1])))
        (oa, Ma), (ob, Mb) = blocks
        a = ijk[:, tang[0]] - oa
        b = ijk[:, tang[1]] - ob
        ref = Mb[np.ix_(b, b)] * Ma[np.ix_(a, a)]
        assert np.abs(Mf.toarray() - ref).max() <= 1e-14 * np.abs(ref).max(), f


# ------------------------------------------------------------- gradient ----

def test_station_operator_is_exact_on_q2_fields():
    """B applied to the interpolant of phi = x(1-x) y(1-y) z^2 (in Q2) gives
    d phi/dz = 2 z x(1-x) y(1-y) exactly, at surface and interior stations."""
    xc = np.linspace(0, 1, 5)
    yc = np.array([0.0, 0.2, 0.5, 0.7, 1.0])
    zc = gen.graded_coords(4, 1.0, 1.2)
    G = oracle.GlobalSystem(xc, yc, zc, keep_boundary=True)
    rng = np.random.default_rng(2)
    st = np.concatenate([gen.surface_stations(5), rng.uniform(0.05, 0.95, size=(10, 3))])
    B = oracle.station_matrix(G, st)
    nodes = _node_coords(xc, yc, zc)[G.gnode]
    X, Y, Z = nodes.T
    phi = X * (1 - X) * Y * (1 - Y) * Z ** 2
    exact = 2 * st[:, 2] * st[:, 0] * (1 - st[:, 0]) * st[:, 1] * (1 - st[:, 1])
    assert np.abs(B @ phi - exact).max() < 1e-13


def test_load_matrix_columns_integrate_the_element():
    prob = gen.regional_problem(nx=4, ny=3, nz=5, sx=1, sy=1, sz=1, seed=1, lx=2.0, ly=1.0, lz=1.5)
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, keep_boundary=True)
    F = oracle.load_matrix(G)
    hx, hy, hz = np.diff(prob.xc), np.diff(prob.yc), np.diff(prob.zc)
    vol = (hz[:, None, None] * hy[None, :, None] * hx[None, None, :]).ravel()
    assert np.allclose(np.asarray(F.sum(axis=0)).ravel(), 4 * np.pi * gen.G_NEWTON * vol, rtol=1e-14)
    G2 = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    F2 = oracle.load_matrix(G2)
    assert np.allclose(F2 @ prob.drho, G2.f, rtol=1e-12, atol=1e-30)


def test_misfit_gradient_matches_central_differences():
    """J is exactly quadratic in drho, so the central difference with any h
    equals the directional derivative; 50 seeded unit directions."""
    prob = gen.layered_problem(n=8, s=1, seed=5, n_spheres=3)
    st = gen.surface_stations(8)
    M = oracle.Misfit(prob.xc, prob.yc, prob.zc, st)
    rng = np.random.default_rng(9)
    g_obs = M.gravity(prob.drho + rng.normal(0, 20, prob.drho.size))
    J, grad = M.value_and_grad(prob.drho, g_obs)
    h = 1e-2
    for _ in range(50):
        d = rng.standard_normal(prob.drho.size)
        d /= np.linalg.norm(d)
        Jp = 0.5 * np.sum((M.gravity(prob.drho + h * d) - g_obs) ** 2)
        Jm = 0.5 * np.sum((M.gravity(prob.drho - h * d) - g_obs) ** 2)
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - grad @ d) <= 1e-5 * np.linalg.norm(grad)
