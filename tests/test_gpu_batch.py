"""Independent problems solved together in one handle (one CUDA graph per
solve): every instance must give exactly its own single-problem solve --
same Schwarz iteration count, same residual, same solution -- and the
oracle's monolithic solution, while converged instances stay frozen."""
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


def _instances():
    a = gen.sphere_problem(8, 2, 4.0)
    b = gen.layered_problem(10, 2, p=6.0, seed=3, n_spheres=4)
    b.cz = np.array([0, 10], dtype=np.int32)           # 2 x 2 x 1
    c = gen.regional_problem(nx=12, ny=10, nz=8, sx=3, sy=2, sz=2, p=2.0, seed=4, lx=10.0, ly=8.0, lz=3.0)
    d = gen.sphere_problem(6, 1, 3.0)                  # one subdomain: converges in one iteration
    return [a, b, c, d]


@pytest.mark.parametrize("prec, fp32_op, start",
                         [("fp64", 0, 0), ("mixed", 1, 0), ("mixed", 2, 1), ("mixed", 2, 2), ("mixed", 2, 3)])
def test_batch_equals_single_solves(osm, prec, fp32_op, start):
    probs = _instances()
    # the FP32 operator and the refinement's FP64 start are pinned: the
    # autotuner could pick differently for the batch and for a single instance
    kw = dict(prec=prec, inner_rtol=1e-13, max_outer=3000, fp32_operator=fp32_op, fp64_start=start)
    bs = osm.BatchSolver(probs, **kw)
    rt = 1e-9 if start == 3 else 1e-10   # the double-float start serves stop tolerances >= 1e-9
    phi, iters, rel = bs.solve(rtol=rt)
    assert np.all(rel <= rt)
    for i, q in enumerate(probs):
        one = osm.Solver.from_problem(q, **kw)
        ph1, n1, r1 = one.solve(rtol=rt)
        assert iters[i] == n1 and rel[i] == r1, (i, iters[i], n1, rel[i], r1)
        pi = bs.instance_phi(phi, i)
        assert bool((pi == ph1).all()), i
        G = oracle.GlobalSystem(q.xc, q.yc, q.zc, q.drho)
        ref, _, _ = G.solve(tol=1e-14)
        ref = G.to_grid(ref)
        tol = 1e-10 if prec == "fp64" else 1e-8
        assert np.linalg.norm(pi.cpu().numpy() - ref) <= tol * np.linalg.norm(ref), i
    # the single-subdomain instance finishes first (one iteration in FP64, a
    # few refinement steps in mixed precision) and stays frozen at its count
    assert iters[3] == (1 if prec == "fp64" else iters[3]) and iters[3] < 5 and iters.max() > 10


def test_batch_uneven_sizes_mixed_residuals(osm):
    """A smaller version of the uneven-batch workload: instances with
    n ~ U{6..12}, 2x2x2 subdomains each, own density and own p, mixed
    precision to 1e-8; each instance certified by the oracle's own K."""
    probs = gen.batch_instances(n_inst=8, lo=6, hi=12, seed=1)
    bs = osm.BatchSolver(probs, prec="mixed", max_outer=3000)
    phi, iters, rel = bs.solve(rtol=1e-8)
    assert np.all(rel <= 1e-8)
    assert len(set(iters.tolist())) > 1                # instances converge at different iterations
    for i, q in enumerate(probs):
        G = oracle.GlobalSystem(q.xc, q.yc, q.zc, q.drho)
        assert G.residual(bs.instance_phi(phi, i).cpu().numpy()) <= 1.001e-8, i


def test_batch_rejects_single_problem_calls(osm):
    bs = osm.BatchSolver(_instances()[:2])
    with pytest.raises(osm.OsmError):
        bs.sample_p(np.array([1.0, 2.0]))
    with pytest.raises(osm.OsmError):
        bs.set_stations(gen.surface_stations(4))
