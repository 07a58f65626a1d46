"""Mixed precision (FP32 subdomain CG inside FP64 refinement) against the
FP64 oracle.

Tolerances:
* FP32 operator (osm_apply op 2): x and the values are rounded to FP32 and a
  row of at most 125 terms is accumulated in FP32 FMA, so
  |y32 - y| <= (n + 2) 2^-24 (|A| |x|)_row with n <= 125; tested at
  1e-5 (|A| |x|)_row (> 127 * 2^-24 = 7.6e-6).
* Solves: the refinement's defect, exchange and stop test are FP64, so the
  mixed solution must match the FP64 oracle to a relative L2 error of 1e-8
  (the target for the mixed form) when solved to a global residual of 1e-10.
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


@pytest.mark.parametrize("case", ["sphere16", "uneven"])
def test_fp32_operator_within_fp32_bound(osm, case):
    import torch
    prob = gen.sphere_problem(16, 2, 10.0) if case == "sphere16" else small_uneven()
    p = 3.3
    S = oracle.Schwarz(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, p)
    sol = osm.Solver.from_problem(prob, p=p, prec="mixed", fp32_operator=1)   # the FP32 SELL matrix
    rng = np.random.default_rng(3)
    x = rng.standard_normal(sol.info["n_local"])
    xt = torch.from_numpy(x).cuda()
    y32 = sol.apply(xt, op=2).cpu().numpy()
    y64 = sol.apply(xt, op=0).cpu().numpy()
    off = 0
    for s in range(S.nsub):
        A, _, _, _ = S.sub_export(s)
        n = A.shape[0]
        xs = x[off:off + n]
        bound = abs(A) @ np.abs(xs)
        ref = A @ xs
        assert np.all(np.abs(y32[off:off + n] - ref) <= 1e-5 * bound), s
        assert np.all(np.abs(y64[off:off + n] - ref) <= 1e-13 * bound), s
        # genuinely FP32: not bitwise the FP64 result
        off += n
    assert np.abs(y32 - y64).max() > 0.0


def _mono(prob):
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    ref, _, _ = G.solve(tol=1e-14)
    return G, G.to_grid(ref)


@pytest.mark.parametrize("fp32_op", [1, 2])
@pytest.mark.parametrize("case", ["sphere16", "uneven"])
def test_mixed_solve_matches_fp64_oracle(osm, case, fp32_op):
    prob = gen.sphere_problem(16, 2, 10.0) if case == "sphere16" else small_uneven()
    G, ref = _mono(prob)
    # the FP64 local tolerance (inner_rtol) caps the reachable global residual:
    # a subdomain whose defect is below inner_rtol ||b_i|| is not corrected
    sol = osm.Solver.from_problem(prob, prec="mixed", mixed_inner_rtol=1e-5, inner_rtol=1e-13,
                                  max_outer=3000, fp32_operator=fp32_op)
    assert sol.info["fp32_operator"] == fp32_op
    phi, n, rel = sol.solve(rtol=1e-10)
    phi = phi.cpu().numpy()
    assert rel <= 1e-10
    assert G.residual(phi) <= 1.01e-10
    err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    assert err <= 1e-8, err


@pytest.mark.parametrize("tin", [0.5, 0.4, 0.3, 1e-1, 1e-3])
def test_refinement_forms_reach_fp64_accuracy(osm, tin):
    """Loose inner tolerances (relative to each Schwarz iteration's defect)
    in FP32 (mixed, on both FP32 operators) and FP64 (fp64_refine) still
    reach the FP64 stop test and the oracle's solution; 0.3 - 0.5 are the
    benchmark tuner's candidates."""
    prob = gen.sphere_problem(16, 2, 10.0)
    G, ref = _mono(prob)
    for prec, op in (("mixed", 1), ("mixed", 2), ("fp64_refine", 0)):
        sol = osm.Solver.from_problem(prob, prec=prec, mixed_inner_rtol=tin, inner_rtol=1e-13, max_outer=4000,
                                      fp32_operator=op)
        phi, n, rel = sol.solve(rtol=1e-10)
        phi = phi.cpu().numpy()
        assert rel <= 1e-10 and G.residual(phi) <= 1.01e-10
        assert np.linalg.norm(phi - ref) <= 1e-8 * np.linalg.norm(ref), prec


def test_mixed_and_fp64_agree_and_mixed_is_cheaper(osm):
    """Same workload in both precisions: both reach the FP64 residual, agree
    with each other to 1e-8, and the mixed form moves fewer matrix bytes per
    CG step (8 B per nonzero instead of 12)."""
    prob = gen.layered_problem(24, 2, p=8.0, seed=1)
    a = osm.Solver.from_problem(prob, prec="fp64")
    b = osm.Solver.from_problem(prob, prec="mixed")
    pa, na, ra = a.solve(rtol=1e-9)
    pb, nb, rb = b.solve(rtol=1e-9)
    assert ra <= 1e-9 and rb <= 1e-9
    pa, pb = pa.cpu().numpy(), pb.cpu().numpy()
    assert np.linalg.norm(pa - pb) <= 1e-8 * np.linalg.norm(pa)
    assert abs(na - nb) <= max(3, 0.1 * na)


def test_mixed_layered64_full_size_residual_and_error(osm):
    """64^3 layered workload in mixed precision at inner tolerance 0.4,
    certified by the oracle's own assembled K (||f - K phi|| <= 1e-8 ||f||)
    and within 1e-8 relative L2 of the oracle's monolithic solve."""
    prob = gen.workload("layered64")
    sol = osm.Solver.from_problem(prob, p=20.0, prec="mixed", mixed_inner_rtol=0.4)
    phi, n, rel = sol.solve(rtol=1e-8)
    assert rel <= 1e-8
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    phi = phi.cpu().numpy()
    assert G.residual(phi) <= 1.001e-8
    ref, _, _ = G.solve(tol=1e-13)
    ref = G.to_grid(ref)
    assert np.linalg.norm(phi - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("case", ["sphere16", "uneven"])
def test_16bit_columns_give_identical_results(osm, case):
    """The SpMVs with 16-bit column indices read the same entries in the same
    order as with 32-bit ones: the FP32 and FP64 operators and a whole mixed
    solve are bit-identical."""
    import torch
    prob = gen.sphere_problem(16, 2, 10.0) if case == "sphere16" else small_uneven()
    a = osm.Solver.from_problem(prob, p=3.3, prec="mixed", index16=1, autotune=0, inner_rtol=1e-12)
    b = osm.Solver.from_problem(prob, p=3.3, prec="mixed", index16=0, autotune=0, inner_rtol=1e-12)
    assert a.info["col_bytes_fp64"] == 2 and a.info["col_bytes_fp32"] == 2
    assert b.info["col_bytes_fp64"] == 4 and b.info["col_bytes_fp32"] == 4
    x = torch.from_numpy(np.random.default_rng(5).standard_normal(a.info["n_local"])).cuda()
    for op in (0, 1, 2):
        assert bool((a.apply(x, op=op) == b.apply(x, op=op)).all()), op
    pa, na, ra = a.solve(rtol=1e-10)
    pb, nb, rb = b.solve(rtol=1e-10)
    assert na == nb and ra == rb and bool((pa == pb).all())


def test_32bit_columns_for_large_subdomains(osm):
    """A subdomain of more than 65,536 padded rows keeps 32-bit indices."""
    prob = gen.sphere_problem(26, 1, 10.0)            # one subdomain, 51^3 = 132,651 unknowns
    sol = osm.Solver.from_problem(prob, prec="mixed", index16=1, inner_rtol=1e-12)
    assert sol.info["col_bytes_fp64"] == 4 and sol.info["col_bytes_fp32"] == 4
    phi, n, rel = sol.solve(rtol=1e-9)
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    assert G.residual(phi.cpu().numpy()) <= 1.001e-9


def test_regional_full_size_mixed_residual_and_error(osm):
    """The regional workload at full size (128 x 128 x 48 graded Q2, 6.18M
    unknowns, 192 uneven subdomains from jittered cuts) in the launch
    configuration the benchmark times: mixed precision, the benchmark's p, the
    inner tolerances its tuner chooses from, to 1e-8.  The oracle's own
    assembled K certifies ||f - K phi|| <= rtol ||f||, and every solution is
    within 1e-8 relative L2 of the oracle's monolithic solve."""
    prob = gen.workload("regional")
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    ref, _, _ = G.solve(tol=1e-13)
    ref = G.to_grid(ref)
    for tin in (0.3, 0.4, 0.5):
        sol = osm.Solver.from_problem(prob, p=1.6664, prec="mixed", mixed_inner_rtol=tin, max_outer=5000)
        phi, n, rel = sol.solve(rtol=1e-8)
        assert rel <= 1e-8
        phi = phi.cpu().numpy()
        assert G.residual(phi) <= 1.001e-8, tin
        assert np.linalg.norm(phi - ref) <= 1e-8 * np.linalg.norm(ref), tin
        sol.close()
