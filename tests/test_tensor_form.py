"""The identity the tensor-product FP32 operator rests on, checked on the
CPU against the oracle's assembled subdomain matrices: on a tensor-product
mesh, a subdomain's Q2 Robin matrix (Sec. 3, zeroth-order condition) is
    A_i = K~x (x) My (x) Mz + Mx (x) K~y (x) Mz + Mx (x) My (x) K~z
with Kx, Mx the assembled 1-D Q2 stiffness and mass over the subdomain's
elements along x (textbook element matrices) and K~ = K + p at each end node
that lies on an interface; outer-boundary (Dirichlet) nodes removed."""
import numpy as np
import pytest

import gen
import oracle


def _k1(h):
    return np.array([[7.0, -8.0, 1.0], [-8.0, 16.0, -8.0], [1.0, -8.0, 7.0]]) / (3.0 * h)


def _m1(h):
    return np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]]) * h / 30.0


def _factors(coords, cuts, idx, n_nodes, p_lo_end, p_hi_end):
    e0, e1 = cuts[idx], cuts[idx + 1]
    n = 2 * (e1 - e0) + 1
    K, M = np.zeros((n, n)), np.zeros((n, n))
    for e in range(e0, e1):
        h, a = coords[e + 1] - coords[e], 2 * (e - e0)
        K[a:a + 3, a:a + 3] += _k1(h)
        M[a:a + 3, a:a + 3] += _m1(h)
    if idx > 0:
        K[0, 0] += p_lo_end
    if idx < len(cuts) - 2:
        K[-1, -1] += p_hi_end
    keep = np.array([0 < 2 * e0 + t < n_nodes - 1 for t in range(n)])
    return K, M, keep


def _tensor_matrix(prob, a, b, c, p_hi, p_lo):
    """A_i of subdomain (a, b, c); the subdomain uses p_hi on its -x, -y, -z
    sides (where it is the upper side of the face) and p_lo on its +x, +y, +z
    sides."""
    Kx, Mx, kx = _factors(prob.xc, prob.cx, a, 2 * prob.nx + 1, p_hi, p_lo)
    Ky, My, ky = _factors(prob.yc, prob.cy, b, 2 * prob.ny + 1, p_hi, p_lo)
    Kz, Mz, kz = _factors(prob.zc, prob.cz, c, 2 * prob.nz + 1, p_hi, p_lo)
    A = np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Kz, np.kron(My, Mx))
    keep = np.kron(kz, np.kron(ky, kx)).astype(bool)
    return A[np.ix_(keep, keep)]


@pytest.mark.parametrize("case", ["sphere8", "uneven_graded"])
@pytest.mark.parametrize("tc", [(3.3, 3.3), (2.0, 0.7)])
def test_kronecker_form_equals_assembled_robin_matrix(case, tc):
    if case == "sphere8":
        prob = gen.sphere_problem(8, 2, 1.0)
    else:
        prob = gen.regional_problem(nx=9, ny=7, nz=6, sx=3, sy=2, sz=2, p=2.0, seed=4, lx=10.0, ly=8.0, lz=3.0)
    p_lo, p_hi = tc
    S = oracle.Schwarz(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, tc=(p_lo, 0.0, p_hi, 0.0))
    sx, sy = len(prob.cx) - 1, len(prob.cy) - 1
    for s in range(S.nsub):
        a, b, c = s % sx, (s // sx) % sy, s // (sx * sy)
        A = S.sub_export(s)[0].toarray()
        T = _tensor_matrix(prob, a, b, c, p_hi, p_lo)
        assert T.shape == A.shape
        assert np.abs(T - A).max() <= 1e-12 * np.abs(A).max(), s


def test_second_order_term_does_not_fold():
    """With q != 0 the face stiffness q S_G = q E (x) (Ky (x) Mz + My (x) Kz) is
    not of the folded form: the assembled matrix differs from the zeroth-order
    Kronecker form by more than rounding (why the tensor kernel keeps q = 0)."""
    prob = gen.sphere_problem(6, 2, 1.0)
    S = oracle.Schwarz(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, tc=(2.0, 0.1, 2.0, 0.1))
    A = S.sub_export(0)[0].toarray()
    T = _tensor_matrix(prob, 0, 0, 0, 2.0, 2.0)
    assert np.abs(T - A).max() > 1e-6 * np.abs(A).max()
