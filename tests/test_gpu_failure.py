"""Failure detection on the GPU without a GPU fault.
* The device wall-clock guard of the solve's device-side loops: a solve that
  outlives opts.max_seconds stops on the device, returns OSM_E_TIMEOUT, and
  leaves the handle and the CUDA context usable.
* CG breakdown: non-finite Robin data injected from the host make a
  subdomain's p.q non-finite; its CG stops with the breakdown status bit,
  the call returns OSM_E_BREAKDOWN, and the handle solves again after a
  reset."""
import time

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osm(cuda_ok):
    from paper_2112_03851_gb300 import build
    build.build()
    import paper_2112_03851_gb300 as pkg
    pkg.load()
    return pkg


@pytest.mark.parametrize("use_graph", [1, 0])
def test_wall_clock_guard_stops_a_long_solve(osm, use_graph):
    import torch
    prob = gen.workload("layered64")                 # an FP64 solve takes several seconds
    sol = osm.Solver.from_problem(prob, p=20.0, max_seconds=1, use_graph=use_graph)
    t0 = time.perf_counter()
    with pytest.raises(osm.OsmError) as err:
        sol.solve(rtol=1e-8)
    elapsed = time.perf_counter() - t0
    assert err.value.status == osm._lib.OSM_E_TIMEOUT
    assert elapsed < 3.5, elapsed                    # stopped soon after the 1 s limit
    st = sol.stats()
    assert st["status"] & 4 and 0 < st["n_outer"] < 151
    # the context and the handle still work: the operator equals a fresh handle's
    x = torch.from_numpy(np.random.default_rng(2).standard_normal(sol.info["n_local"])).cuda()
    ref = osm.Solver.from_problem(prob, p=20.0)
    assert torch.equal(sol.apply(x), ref.apply(x))


@pytest.mark.parametrize("use_graph", [1, 0])
def test_cg_breakdown_is_reported_and_the_handle_recovers(osm, use_graph):
    import torch

    import oracle
    prob = gen.sphere_problem(8, 2, 4.0)
    sol = osm.Solver.from_problem(prob, inner_rtol=1e-12, max_outer=2000, use_graph=use_graph)
    lam = torch.zeros(sol.info["n_face_vals"], dtype=torch.float64, device="cuda")
    lam[0] = float("nan")                           # one Robin datum of the first face
    sol.reset()
    sol.set_lambda(lam)
    with pytest.raises(osm.OsmError) as err:
        sol.iterate(1)
    assert err.value.status == osm._lib.OSM_E_BREAKDOWN
    st = sol.stats()
    assert st["status"] & 2 and st["n_outer"] == 1
    # the handle and the context still work: reset, then a full solve
    sol.reset()
    phi, n, rel = sol.solve(rtol=1e-10)
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    ref, _, _ = G.solve(tol=1e-14)
    ref = G.to_grid(ref)
    assert rel <= 1e-10 and sol.stats()["status"] == 0
    assert np.linalg.norm(phi.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
