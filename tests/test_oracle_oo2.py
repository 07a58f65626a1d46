"""Pins of the oracle's second-order (oo2) and unsymmetric transmission
conditions (Sec. 3, Table 1) against closed forms and the separable
two-subdomain analysis -- never against the oracle itself.

* The face tangential stiffness is the Q2 weak form of -d^2/dtau^2: the
  Kronecker closed form of the textbook 1-D matrices per face element, and
  the exact energy integral of a Q2 function on an assembled face.
* On a slab pair the interface problem separates: every Dirichlet-to-Neumann
  eigenmode g of the face is also an eigenmode of the tangential pencil
  (S g = mu M g), and one Schwarz iteration multiplies it by
  (p2 + q2 mu - D) / (p1 + q1 mu + D): the Fourier rate of Sec. 3 with the
  operator symbol p + q k^2.  With p + q mu = D on two modes, both vanish in
  two iterations (a zeroth-order condition can do that for one mode only).
* The fixed point does not depend on (p, q): oo2 Schwarz converges to the
  monolithic solution.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import gen
import oracle

K1 = np.array([[7.0, -8.0, 1.0], [-8.0, 16.0, -8.0], [1.0, -8.0, 7.0]]) / 3.0
M1 = np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]]) / 30.0


@pytest.mark.parametrize("ha,hb", [(1.0, 1.0), (0.3, 2.5)])
def test_face_stiffness_closed_form(ha, hb):
    """S = M1(hb) (x) K1(ha) + K1(hb) (x) M1(ha), local node a + 3b."""
    S = oracle.face_stiffness(ha, hb)
    ref = np.kron(M1 * hb, K1 / ha) + np.kron(K1 / hb, M1 * ha)
    assert np.abs(S - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(S.sum(axis=1)).max() < 1e-13 * np.abs(ref).max()   # constants in the kernel


def test_assembled_face_stiffness_energy_is_exact():
    """v = a(1-a) b(1-b) (in Q2, zero on the face rim) on the interface of a
    unit cube split at x = 1/2: v^T S v = int |grad_t v|^2 = 2 (1/3)(1/30)
    = 1/45 and v^T M v = int v^2 = 1/900, on a graded face mesh."""
    m = 4
    xc = np.linspace(0.0, 1.0, m + 1)
    yc = np.array([0.0, 0.1, 0.35, 0.7, 1.0])
    zc = np.array([0.0, 0.25, 0.45, 0.8, 1.0])
    Z = oracle.Schwarz(xc, yc, zc, np.zeros(m ** 3), [0, 2, 4], [0, 4], [0, 4], tc=(1.0, 0.5, 2.0, 0.25))
    g, Mf = Z.face_export(0)
    Sf = Z.face_stiffness_export(0)
    NX, NY = 2 * m + 1, 2 * m + 1
    j = (g // NX) % NY
    k = g // (NX * NY)
    # node coordinates: element vertices and midpoints
    ny_ = np.concatenate([[yc[0]], np.ravel(np.column_stack([(yc[:-1] + yc[1:]) / 2, yc[1:]]))])
    nz_ = np.concatenate([[zc[0]], np.ravel(np.column_stack([(zc[:-1] + zc[1:]) / 2, zc[1:]]))])
    a, b = ny_[j], nz_[k]
    v = a * (1 - a) * b * (1 - b)
    assert abs(v @ (Sf @ v) - 1.0 / 45.0) < 1e-13
    assert abs(v @ (Mf @ v) - 1.0 / 900.0) < 1e-14


def _two_slab(m, tc):
    """Slab pair [0,1] | [1,2] x [0,1]^2, oo2 coefficients tc; returns the
    oracle, face M and S, and the Dirichlet-to-Neumann eigenpairs of the
    face (generalised to M) from the Schur complement of subdomain 0's K."""
    xc = np.linspace(0, 2, 2 * m + 1)
    yc = np.linspace(0, 1, m + 1)
    Z = oracle.Schwarz(xc, yc, yc, np.zeros(2 * m ** 3), [0, m, 2 * m], [0, m], [0, m], tc=tc)
    A, _, g, _ = Z.sub_export(0)
    gf, Mf = Z.face_export(0)
    Sf = Z.face_stiffness_export(0).toarray()
    A, Mf = A.toarray(), Mf.toarray()
    loc = {x: i for i, x in enumerate(g)}
    fi = np.array([loc[x] for x in gf])
    K = A.copy()
    K[np.ix_(fi, fi)] -= tc[0] * Mf + tc[1] * Sf     # subdomain 0 is the lower side
    ii = np.setdiff1d(np.arange(len(g)), fi)
    Sch = K[np.ix_(fi, fi)] - K[np.ix_(fi, ii)] @ np.linalg.solve(K[np.ix_(ii, ii)], K[np.ix_(ii, fi)])
    D, V = sla.eigh(Sch, Mf)
    return Z, Mf, Sf, D, V


@pytest.mark.parametrize("tc", [(0.7, 0.3, 0.7, 0.3), (1.2, 0.05, 0.2, 0.9)])
def test_oo2_contraction_factor(tc):
    p1, q1, p2, q2 = tc
    _, Mf, Sf, D, V = _two_slab(4, tc)
    for mode in (0, 3, 8):
        Z = _two_slab(4, tc)[0]          # fresh state (u = 0) for every mode
        g, d = V[:, mode], D[mode]
        mu = g @ Sf @ g / (g @ Mf @ g)
        # separability: the DtN mode is a tangential eigenmode
        assert np.abs(Sf @ g - mu * (Mf @ g)).max() < 1e-9 * np.abs(Sf @ g).max()
        lam = Mf @ g
        Z.set_lambda(0, 0, lam)
        Z.set_lambda(0, 1, np.zeros_like(g))
        Z.iterate(inner_rtol=1e-15)
        f1 = (p2 + q2 * mu - d) / (p1 + q1 * mu + d)
        assert np.abs(Z.get_lambda(0, 0)).max() < 1e-12 * np.abs(lam).max()
        assert np.abs(Z.get_lambda(0, 1) - f1 * lam).max() < 1e-10 * np.abs(lam).max()
        Z.iterate(inner_rtol=1e-15)
        rate = (p1 + q1 * mu - d) * (p2 + q2 * mu - d) / ((p1 + q1 * mu + d) * (p2 + q2 * mu + d))
        assert np.abs(Z.get_lambda(0, 0) - rate * lam).max() < 1e-10 * np.abs(lam).max()


def test_oo2_matched_on_two_modes_kills_both_in_two_iterations():
    """p + q mu = D on modes 0 and 3 (two conditions, two unknowns)."""
    _, Mf, Sf, D, V = _two_slab(4, (1.0, 0.1, 1.0, 0.1))
    ga, gb = V[:, 0], V[:, 3]
    mua, mub = (g @ Sf @ g / (g @ Mf @ g) for g in (ga, gb))
    q = (D[3] - D[0]) / (mub - mua)
    p = D[0] - q * mua
    assert p > 0 and q > 0
    Z, Mf, _, _, _ = _two_slab(4, (p, q, p, q))
    lam = Mf @ (ga + 0.5 * gb)
    Z.set_lambda(0, 0, lam)
    Z.set_lambda(0, 1, 0.7 * lam)
    Z.iterate(inner_rtol=1e-15)
    Z.iterate(inner_rtol=1e-15)
    for side in (0, 1):
        assert np.abs(Z.get_lambda(0, side)).max() < 1e-10 * np.abs(lam).max()
    # the same p alone (q = 0) leaves mode 3 alive
    Z0, Mf0, _, _, _ = _two_slab(4, (p, 0.0, p, 0.0))
    Z0.set_lambda(0, 0, lam)
    Z0.set_lambda(0, 1, 0.7 * lam)
    Z0.iterate(inner_rtol=1e-15)
    Z0.iterate(inner_rtol=1e-15)
    assert np.abs(Z0.get_lambda(0, 0)).max() > 1e-3 * np.abs(lam).max()


@pytest.mark.parametrize("tc", [(2.0, 0.05, 2.0, 0.05), (6.0, 0.02, 1.0, 0.1)])
def test_oo2_fixed_point_is_the_monolithic_solution(tc):
    prob = gen.regional_problem(nx=12, ny=10, nz=8, sx=3, sy=2, sz=2, p=2.0, seed=4,
                                lx=10.0, ly=8.0, lz=3.0)
    Z = oracle.Schwarz.from_problem(prob, tc=tc)
    phi, n, rel, _ = Z.solve(inner_rtol=1e-13, rtol=1e-11, max_outer=3000)
    assert rel <= 1e-11
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    ref, _, _ = G.solve(tol=1e-14)
    ref = G.to_grid(ref)
    assert np.linalg.norm(phi - ref) <= 1e-9 * np.linalg.norm(ref)
