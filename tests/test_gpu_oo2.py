"""Second-order and unsymmetric transmission conditions (Sec. 3, Table 1) on
the GPU against the oracle: the first Schwarz iterations element by element,
full solves (iteration counts +-1, solution = monolithic oracle), mixed
precision, argument checks and the interplay with the batched p evaluation
and the p-derivative."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

TC_SYM = (2.0, 0.05, 2.0, 0.05)
TC_UNSYM = (6.0, 0.02, 1.0, 0.1)


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


def _mono(prob):
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    ref, _, _ = G.solve(tol=1e-14)
    return G, G.to_grid(ref)


@pytest.mark.parametrize("tc", [TC_SYM, TC_UNSYM])
def test_first_iterations_match_oracle(osm, tc):
    prob = small_uneven()
    S = oracle.Schwarz.from_problem(prob, tc=tc)
    sol = osm.Solver.from_problem(prob, tc=tc, inner_rtol=1e-12, use_graph=False)
    sol.reset()
    for it in range(3):
        S.iterate(inner_rtol=1e-12)
        _, rel_ref = S.residual()
        hist = sol.iterate(1)
        u = sol.get_local().cpu().numpy()
        u_ref = np.concatenate([S.sub_export(s)[3] for s in range(S.nsub)])
        assert np.linalg.norm(u - u_ref) <= 1e-10 * np.linalg.norm(u_ref), it
        lam = sol.get_lambda().cpu().numpy()
        lam_ref = np.concatenate([np.concatenate([S.get_lambda(f, 0), S.get_lambda(f, 1)])
                                  for f in range(S.nface)])
        assert np.linalg.norm(lam - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref), it
        assert abs(hist[0] - rel_ref) <= 1e-8 * rel_ref, (hist[0], rel_ref)


@pytest.mark.parametrize("tc", [TC_SYM, TC_UNSYM])
def test_solve_matches_oracle(osm, tc):
    prob = small_uneven()
    _, ref = _mono(prob)
    S = oracle.Schwarz.from_problem(prob, tc=tc)
    _, n_ref, _, _ = S.solve(inner_rtol=1e-12, rtol=1e-10, max_outer=3000)
    sol = osm.Solver.from_problem(prob, tc=tc, inner_rtol=1e-12, max_outer=3000)
    phi, n, rel = sol.solve(rtol=1e-10)
    assert rel <= 1e-10 and abs(n - n_ref) <= 1, (n, n_ref)
    phi = phi.cpu().numpy()
    assert np.linalg.norm(phi - ref) <= 1e-9 * np.linalg.norm(ref)


def test_mixed_precision_with_second_order_conditions(osm):
    prob = small_uneven()
    G, ref = _mono(prob)
    sol = osm.Solver.from_problem(prob, tc=TC_UNSYM, prec="mixed", mixed_inner_rtol=0.3,
                                  inner_rtol=1e-13, max_outer=3000)
    phi, n, rel = sol.solve(rtol=1e-9)
    assert rel <= 1e-9
    phi = phi.cpu().numpy()
    assert G.residual(phi) <= 1.001e-9
    assert np.linalg.norm(phi - ref) <= 1e-7 * np.linalg.norm(ref)


def test_set_transmission_rejects_bad_coefficients(osm):
    sol = osm.Solver.from_problem(gen.sphere_problem(4, 2, 1.0))
    for bad in [(0.0, 0.1, 1.0, 0.1), (1.0, -0.1, 1.0, 0.1), (1.0, 0.1, float("nan"), 0.1),
                (1.0, 0.1, 1.0, float("inf"))]:
        with pytest.raises(osm.OsmError):
            sol.set_transmission(*bad)


def test_zeroth_order_transmission_equals_set_robin(osm):
    """(p, 0, p, 0) is the Robin condition: same iteration count, residual
    to rounding."""
    prob = small_uneven()
    a = osm.Solver.from_problem(prob, p=3.0, inner_rtol=1e-12)
    b = osm.Solver.from_problem(prob, tc=(3.0, 0.0, 3.0, 0.0), inner_rtol=1e-12)
    pa, na, ra = a.solve(rtol=1e-10)
    pb, nb, rb = b.solve(rtol=1e-10)
    assert abs(na - nb) <= 1
    assert np.linalg.norm((pa - pb).cpu().numpy()) <= 1e-10 * np.linalg.norm(pa.cpu().numpy())


def test_sampling_restores_second_order_handle(osm):
    prob = gen.sphere_problem(8, 2, 4.0)
    sol = osm.Solver.from_problem(prob, tc=(4.0, 0.01, 3.0, 0.02), inner_rtol=1e-10, max_outer=400)
    phi0, n0, r0 = sol.solve(rtol=1e-8)
    sol.sample_p(np.array([2.0, 8.0]), rtol=1e-8, max_outer=400)
    phi1, n1, r1 = sol.solve(rtol=1e-8)
    assert n1 == n0 and r1 == r0 and bool((phi1 == phi0).all())


def test_grad_p_needs_zeroth_order_symmetric(osm):
    prob = gen.sphere_problem(6, 2, 4.0)
    sol = osm.Solver.from_problem(prob, tc=TC_SYM, inner_rtol=1e-10)
    sol.set_stations(gen.surface_stations(4))
    import torch
    g_obs = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(osm.OsmError):
        sol.grad_p(g_obs, n_iter=3)


def test_slab_decomposition_matches_oracle(osm):
    """x-slab decomposition of a thin box (the paper's partition, Sec. 6) with
    unsymmetric second-order conditions: iteration count and solution."""
    prob = gen.slab_problem(nx=24, ny=12, nz=4, n_slabs=6, seed=2)
    _, ref = _mono(prob)
    tc = (0.9, 0.6, 0.3, 1.4)
    S = oracle.Schwarz.from_problem(prob, tc=tc)
    _, n_ref, _, _ = S.solve(inner_rtol=1e-12, rtol=1e-8, max_outer=2000)
    sol = osm.Solver.from_problem(prob, tc=tc, inner_rtol=1e-12, max_outer=2000)
    phi, n, rel = sol.solve(rtol=1e-8)
    assert rel <= 1e-8 and abs(n - n_ref) <= 1, (n, n_ref)
    assert np.linalg.norm(phi.cpu().numpy() - ref) <= 1e-7 * np.linalg.norm(ref)


def test_batch_instances_with_second_order_conditions(osm):
    """osm_set_transmission on a batch handle applies to every instance: each
    instance gives exactly its single-problem oo2 solve."""
    probs = [small_uneven(), gen.slab_problem(nx=24, ny=12, nz=4, n_slabs=6, seed=2)]
    tc = (0.9, 0.6, 0.3, 1.4)
    bs = osm.BatchSolver(probs, inner_rtol=1e-12, max_outer=3000)
    bs.set_transmission(*tc)
    phi, iters, rel = bs.solve(rtol=1e-9)
    for i, q in enumerate(probs):
        one = osm.Solver.from_problem(q, tc=tc, inner_rtol=1e-12, max_outer=3000)
        ph1, n1, r1 = one.solve(rtol=1e-9)
        assert iters[i] == n1 and rel[i] == r1, (i, iters[i], n1)
        assert bool((bs.instance_phi(phi, i) == ph1).all()), i
