"""The tensor-product (matrix-free) FP32 operator of the mixed inner solve.

On a tensor-product mesh a subdomain's Q2 Robin matrix is
    A_i = K~x (x) My (x) Mz + Mx (x) K~y (x) Mz + Mx (x) My (x) K~z,
K~ the assembled 1-D stiffness with p added at interface ends.  The kernel
applies it by sum factorisation in FP32.  Checks:
* op 2 (FP32 operator) against the oracle's assembled A_i: each output is a
  nested sum of at most 17 FP32 roundings over products of three FP32-rounded
  1-D coefficients, so |y32 - A x| <= ~20 * 2^-24 (B |x|) with
  B = |K~x| (x) |My| (x) |Mz| + |Mx| (x) |K~y| (x) |Mz| + |Mx| (x) |My| (x) |K~z|
  (B >= |A| entrywise); tested at 1e-5 (B |x|)_row.  B is built here from the
  textbook 1-D Q2 element matrices (the same closed forms that pin the
  oracle's quadrature).
* mixed solves on the tensor operator match the FP64 oracle to 1e-8 and the
  SELL operator's solves;
* a second-order condition (q != 0) falls back to the SELL matrix and back;
* batched instances give their single solves bit for bit.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osm(cuda_ok):
    from paper_2112_03851_gb300 import build
    build.build()
    import paper_2112_03851_gb300 as pkg
    pkg.load()
    return pkg


def small_uneven():
    return gen.regional_problem(nx=12, ny=10, nz=8, sx=3, sy=2, sz=2, p=2.0, seed=4,
                                lx=10.0, ly=8.0, lz=3.0)


def _k1(h):
    return np.array([[7.0, -8.0, 1.0], [-8.0, 16.0, -8.0], [1.0, -8.0, 7.0]]) / (3.0 * h)


def _m1(h):
    return np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]]) * h / 30.0


def _band(c, e0, e1):
    n = 2 * (e1 - e0) + 1
    K, M = np.zeros((n, n)), np.zeros((n, n))
    for e in range(e0, e1):
        h, a = c[e + 1] - c[e], 2 * (e - e0)
        K[a:a + 3, a:a + 3] += _k1(h)
        M[a:a + 3, a:a + 3] += _m1(h)
    return K, M


def _axis_factors(coords, cuts, idx, n_nodes, p):
    """|K~|, |M| of one subdomain along one axis (K~: p added at interface
    ends) and the mask of its non-Dirichlet nodes."""
    K, M = _band(coords, cuts[idx], cuts[idx + 1])
    if idx > 0:
        K[0, 0] += p
    if idx < len(cuts) - 2:
        K[-1, -1] += p
    lo = 2 * cuts[idx]
    keep = np.array([0 < lo + t < n_nodes - 1 for t in range(K.shape[0])])
    return np.abs(K), np.abs(M), keep


def _bound_matrices(prob, p):
    """Per subdomain (canonical order): B (the bound matrix above) restricted
    to the subdomain's unknowns."""
    sx, sy, sz = len(prob.cx) - 1, len(prob.cy) - 1, len(prob.cz) - 1
    out = []
    for c in range(sz):
        for b in range(sy):
            for a in range(sx):
                Kx, Mx, kx = _axis_factors(prob.xc, prob.cx, a, 2 * prob.nx + 1, p)
                Ky, My, ky = _axis_factors(prob.yc, prob.cy, b, 2 * prob.ny + 1, p)
                Kz, Mz, kz = _axis_factors(prob.zc, prob.cz, c, 2 * prob.nz + 1, p)
                B = np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Kz, np.kron(My, Mx))
                keep = np.kron(kz, np.kron(ky, kx)).astype(bool)
                out.append(B[np.ix_(keep, keep)])
    return out


@pytest.mark.parametrize("case", ["sphere16", "uneven"])
def test_tensor_operator_within_fp32_bound(osm, case):
    import torch
    prob = gen.sphere_problem(16, 2, 10.0) if case == "sphere16" else small_uneven()
    p = 3.3
    S = oracle.Schwarz(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, p)
    sol = osm.Solver.from_problem(prob, p=p, prec="mixed", fp32_operator=2)
    assert sol.info["fp32_operator"] == 2 and sol.info["box_rows"] > 0
    rng = np.random.default_rng(3)
    x = rng.standard_normal(sol.info["n_local"])
    y32 = sol.apply(torch.from_numpy(x).cuda(), op=2).cpu().numpy()
    bounds = _bound_matrices(prob, p)
    off = 0
    for s in range(S.nsub):
        A, _, _, _ = S.sub_export(s)
        n = A.shape[0]
        xs = x[off:off + n]
        B = bounds[s]
        assert B.shape == A.shape
        assert np.all(B >= np.abs(A.toarray()) - 1e-12 * np.abs(A).max())   # B bounds |A|
        ref = A @ xs
        assert np.all(np.abs(y32[off:off + n] - ref) <= 1e-5 * (B @ np.abs(xs))), s
        off += n


def _mono(prob):
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    ref, _, _ = G.solve(tol=1e-14)
    return G.to_grid(ref)


@pytest.mark.parametrize("case", ["sphere16", "uneven"])
def test_tensor_mixed_solve_matches_oracle_and_sell(osm, case):
    """Mixed solves on the SELL FP32 matrix, on the tensor form with the
    SELL FP64 defect, and on the tensor form with the FP64 tensor defect
    (u mirrored in the box layout) all reach the oracle's solution."""
    prob = gen.sphere_problem(16, 2, 10.0) if case == "sphere16" else small_uneven()
    ref = _mono(prob)
    phis = {}
    for op, start in ((1, 0), (2, 1), (2, 2)):
        sol = osm.Solver.from_problem(prob, prec="mixed", mixed_inner_rtol=0.3, inner_rtol=1e-13, max_outer=4000,
                                      fp32_operator=op, fp64_start=start)
        assert sol.info["fp32_operator"] == op
        assert sol.info["fp64_start"] == (start if op == 2 else 1)
        phi, n, rel = sol.solve(rtol=1e-10)
        assert rel <= 1e-10
        phis[(op, start)] = phi.cpu().numpy()
        assert np.linalg.norm(phis[(op, start)] - ref) <= 1e-8 * np.linalg.norm(ref), (op, start)
    for key in ((2, 1), (2, 2)):
        assert np.linalg.norm(phis[(1, 0)] - phis[key]) <= 1e-8 * np.linalg.norm(ref), key


def test_second_order_condition_falls_back_to_sell(osm):
    prob = small_uneven()
    sol = osm.Solver.from_problem(prob, p=2.0, prec="mixed", mixed_inner_rtol=0.3, inner_rtol=1e-13,
                                  max_outer=4000, fp32_operator=2)
    assert sol.info["fp32_operator"] == 2
    ref = _mono(prob)
    tc = (2.0, 0.05, 1.5, 0.08)
    sol.set_transmission(*tc)
    info = osm._lib.OsmInfo()
    osm.load().osm_info(sol._h, osm._lib.C.byref(info))
    assert info.fp32_operator == 1 and info.fp32_operator_tuned == 2
    assert sol.info["fp32_operator"] == 1 and sol.info["fp64_start"] == 1   # the binding's view follows too
    phi, n, rel = sol.solve(rtol=1e-10)
    assert rel <= 1e-10 and np.linalg.norm(phi.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    # unsymmetric zeroth order (q = 0) is back on the tensor form
    sol.set_transmission(2.0, 0.0, 1.5, 0.0)
    osm.load().osm_info(sol._h, osm._lib.C.byref(info))
    assert info.fp32_operator == 2
    phi2, n2, rel2 = sol.solve(rtol=1e-10)
    assert rel2 <= 1e-10 and np.linalg.norm(phi2.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)


def test_tensor_batch_equals_single_solves(osm):
    probs = [gen.sphere_problem(8, 2, 4.0), small_uneven(), gen.sphere_problem(6, 1, 3.0)]
    kw = dict(prec="mixed", inner_rtol=1e-13, max_outer=3000, fp32_operator=2, fp64_start=2, mixed_inner_rtol=0.3)
    bs = osm.BatchSolver(probs, **kw)
    assert bs.info["fp32_operator"] == 2 and bs.info["fp64_start"] == 2
    phi, iters, rel = bs.solve(rtol=1e-10)
    assert np.all(rel <= 1e-10)
    for i, q in enumerate(probs):
        one = osm.Solver.from_problem(q, **kw)
        ph1, n1, r1 = one.solve(rtol=1e-10)
        assert iters[i] == n1 and rel[i] == r1, (i, iters[i], n1)
        assert bool((bs.instance_phi(phi, i) == ph1).all()), i


def test_bad_fp32_operator_is_rejected(osm):
    with pytest.raises(osm.OsmError):
        osm.Solver.from_problem(gen.sphere_problem(4, 2, 1.0), prec="mixed", fp32_operator=3)


@pytest.mark.parametrize("case", ["sphere16", "uneven"])
def test_double_float_start_tracks_the_fp64_start(osm, case):
    """The refinement start in double-float arithmetic (fp64_start 3) against
    the FP64 one (2), everything else equal: the defects differ by their
    rounding (about 2^-48 |A| |u| against 2^-53), far below the FP32 inner
    solve's, so the first stop test agrees to rounding and the Schwarz
    residual histories stay close; a solve to
    1e-9 with it reaches the oracle's solution like the FP64 start does; a
    tighter stop tolerance falls back to the FP64 start and still gets
    there."""
    prob = gen.sphere_problem(16, 2, 10.0) if case == "sphere16" else small_uneven()
    ref = _mono(prob)
    kw = dict(prec="mixed", mixed_inner_rtol=0.3, inner_rtol=1e-13, max_outer=4000, fp32_operator=2)
    hist, phis = {}, {}
    for start in (2, 3):
        sol = osm.Solver.from_problem(prob, fp64_start=start, **kw)
        assert sol.info["fp64_start"] == start
        hist[start] = np.asarray(sol.iterate(30))
        phi, n, rel = sol.solve(rtol=1e-9)
        assert rel <= 1e-9
        phis[start] = phi.cpu().numpy()
        assert np.linalg.norm(phis[start] - ref) <= 1e-8 * np.linalg.norm(ref), start
        if start == 3:   # below 1e-9 the FP64 start serves
            phi, n, rel = sol.solve(rtol=1e-11)
            assert rel <= 1e-11
            assert np.linalg.norm(phi.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)
            assert sol.info["fp64_start"] == 3
    # the first stop test sees the same iterate in both runs (the first
    # defect, b - A 0, is exact): only the start's rounding of A u differs
    assert abs(hist[3][0] - hist[2][0]) <= 1e-12 * hist[2][0], (hist[3][0], hist[2][0])
    # afterwards the FP32 inner CG turns any rounding difference in its input
    # into a different (equally valid) trajectory: the histories stay close
    assert np.all(np.abs(hist[3] - hist[2]) <= 1e-3 * hist[2]), np.max(np.abs(hist[3] - hist[2]) / hist[2])
    assert np.linalg.norm(phis[3] - phis[2]) <= 1e-8 * np.linalg.norm(ref)
