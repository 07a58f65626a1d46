"""Batched stochastic evaluation of Robin parameters (osm_sample_p, Sec. 4)
against independent single-p solves and the oracle's Schwarz iteration
counts.

Each candidate runs the same FP64 algorithm as osm_solve, with its own state,
so its Schwarz iteration count must equal the single solve's (rounding can
move a residual across the threshold: +-1) and the oracle's (+-1), and its
final residual must agree with the single solve's to the stop tolerance.
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


@pytest.mark.parametrize("case", ["sphere8", "uneven"])
def test_sample_matches_single_solves_and_oracle(osm, case):
    prob = gen.sphere_problem(8, 2, 4.0) if case == "sphere8" else small_uneven()
    ps = gen.log_uniform_p(0, 6, 0.5, 40.0)
    rtol = 1e-9
    sol = osm.Solver.from_problem(prob, inner_rtol=1e-11, max_outer=600)
    iters, rel, best = sol.sample_p(ps, rtol=rtol, max_outer=600)
    for k, p in enumerate(ps):
        sol.set_robin(float(p))
        _, n1, r1 = sol.solve(rtol=rtol, allow_noconv=True)
        assert abs(int(iters[k]) - n1) <= 1, (k, p, iters[k], n1)
        if n1 == iters[k]:  # same iterate up to summation order
            assert abs(rel[k] - r1) <= 1e-4 * r1 + 1e-300
    for k in (0, 3):
        S = oracle.Schwarz.from_problem(prob, p=float(ps[k]))
        _, n_ref, _, _ = S.solve(inner_rtol=1e-11, rtol=rtol, max_outer=600)
        assert abs(int(iters[k]) - n_ref) <= 1, (k, iters[k], n_ref)
    conv = [k for k in range(len(ps)) if rel[k] <= rtol]
    exp = min(conv, key=lambda k: (iters[k], rel[k], ps[k]))
    assert best == exp


def test_sample_batches_beyond_32_and_restores_handle(osm):
    prob = gen.sphere_problem(8, 2, 4.0)
    sol = osm.Solver.from_problem(prob, inner_rtol=1e-10, max_outer=400)
    phi0, n0, r0 = sol.solve(rtol=1e-8)
    ps = gen.log_uniform_p(7, 40, 0.5, 40.0)
    iters, rel, best = sol.sample_p(ps, rtol=1e-8, max_outer=400)
    # the last 8 candidates ran in a second batch: compare with a batch of their own
    it2, rel2, _ = sol.sample_p(ps[32:], rtol=1e-8, max_outer=400)
    assert np.array_equal(iters[32:], it2) and np.array_equal(rel[32:], rel2)
    # batching does not change a candidate's run: the same p in two batch positions
    it3, rel3, _ = sol.sample_p(np.array([ps[3], ps[35], ps[3]]), rtol=1e-8, max_outer=400)
    assert it3[0] == it3[2] == iters[3] and it3[1] == iters[35]
    assert rel3[0] == rel3[2] == rel[3]
    # the handle's own p (4.0) is back in place: bit-identical solve
    phi1, n1, r1 = sol.solve(rtol=1e-8)
    assert n1 == n0 and r1 == r0 and bool((phi1 == phi0).all())


def test_sample_reports_non_converging_candidates(osm):
    prob = gen.sphere_problem(8, 2, 4.0)
    sol = osm.Solver.from_problem(prob, inner_rtol=1e-10)
    iters, rel, best = sol.sample_p(np.array([1e-3, 4.0, 1e4]), rtol=1e-8, max_outer=300)
    assert iters[0] == 300 and rel[0] > 1e-8      # far too small p: stalls
    assert iters[2] == 300 and rel[2] > 1e-8      # far too large p: stalls
    assert rel[1] <= 1e-8 and iters[1] < 300 and best == 1


def test_sample_rejects_bad_p(osm):
    prob = gen.sphere_problem(4, 2, 4.0)
    sol = osm.Solver.from_problem(prob)
    for bad in ([1.0, -2.0], [float("nan")], []):
        with pytest.raises(osm.OsmError):
            sol.sample_p(np.array(bad, dtype=np.float64))


@pytest.mark.parametrize("prec", ["mixed", "fp64_refine"])
def test_sample_in_refinement_modes_matches_single_solves(osm, prec):
    """On a mixed (FP32 inner) or FP64-refinement handle every candidate runs
    that handle's algorithm: same Schwarz iteration count as a single solve
    (+-1 for rounding of the reductions) and a residual at rtol."""
    prob = small_uneven()
    ps = gen.log_uniform_p(3, 5, 0.5, 20.0)
    # the batched evaluation's FP32 inner solve reads the SELL matrix: the
    # single solves it is compared with use it too
    sol = osm.Solver.from_problem(prob, prec=prec, mixed_inner_rtol=0.3, inner_rtol=1e-12, max_outer=1500,
                                  fp32_operator=1)
    iters, rel, best = sol.sample_p(ps, rtol=1e-9, max_outer=1500)
    for k, p in enumerate(ps):
        sol.set_robin(float(p))
        _, n1, r1 = sol.solve(rtol=1e-9, allow_noconv=True)
        assert abs(int(iters[k]) - n1) <= max(1, n1 // 50), (k, p, iters[k], n1)
        if rel[k] <= 1e-9:
            assert r1 <= 1e-9
    assert best >= 0 and rel[best] <= 1e-9


def test_cma_es_search_with_batched_evaluation(osm):
    """CMA-ES (Sec. 4) over log p with the measured Schwarz iteration count as
    the cost, each generation one batched run: it must reach a p at least as
    good as the best of a log-uniform sample of the same budget's first
    generation."""
    from paper_2112_03851_gb300 import search
    prob = gen.sphere_problem(8, 2, 4.0)
    sol = osm.Solver.from_problem(prob, inner_rtol=1e-10, max_outer=400)
    p_best, res = search.search_p(sol, p0=1.0, sigma0=1.5, popsize=16, generations=4, rtol=1e-8, max_outer=400)
    iters, rel, _ = sol.sample_p(np.array([p_best]), rtol=1e-8, max_outer=400)
    ps = gen.log_uniform_p(11, 16, 0.1, 100.0)
    it_s, rel_s, best_s = sol.sample_p(ps, rtol=1e-8, max_outer=400)
    assert rel[0] <= 1e-8 and iters[0] <= it_s[best_s]
    assert res.evaluations == 16 * res.iterations


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_race_mode_finds_the_same_winner(osm, prec):
    """OSM_SAMPLE_RACE stops a batch at its first convergence: the winner
    (and every candidate converging at the same iteration) keeps exactly its
    full-run iteration count and residual; the others stop at or before the
    winner's count with a residual above rtol.  Across batches of 32, a later
    batch is capped at the best count so far."""
    prob = gen.sphere_problem(8, 2, 4.0)
    sol = osm.Solver.from_problem(prob, prec=prec, inner_rtol=1e-10, mixed_inner_rtol=0.3, max_outer=400)
    ps = gen.log_uniform_p(21, 40, 0.5, 40.0)
    it_full, rel_full, best_full = sol.sample_p(ps, rtol=1e-8, max_outer=400)
    it_race, rel_race, best_race = sol.sample_p(ps, rtol=1e-8, max_outer=400, race=True)
    assert best_race == best_full
    assert it_race[best_race] == it_full[best_full] and rel_race[best_race] == rel_full[best_full]
    for k in range(len(ps)):
        if rel_race[k] <= 1e-8:
            # a candidate reported converged ran its full course
            assert it_race[k] == it_full[k] and rel_race[k] == rel_full[k], k
        else:
            # a stopped one stopped no later than its own full run ended
            assert it_race[k] <= it_full[k] and not (rel_full[k] <= 1e-8 and it_full[k] <= it_race[k]), k
    # nobody needed fewer iterations than the winner
    assert it_full.min() >= 0 and all(it_full[k] >= it_full[best_full] for k in range(len(ps)) if rel_full[k] <= 1e-8)
    # unknown flags are rejected before anything runs
    one, it1, rel1, b1 = np.ones(1), np.zeros(1, dtype=np.int32), np.zeros(1), np.zeros(1, dtype=np.int32)
    st = osm.load().osm_sample_p_ex(sol._h, 1, osm._lib._ptr(one), 1e-8, 10, 4, osm._lib._ptr(it1),
                                    osm._lib._ptr(rel1), osm._lib._ptr(b1))
    assert st == osm._lib.OSM_E_ARG
