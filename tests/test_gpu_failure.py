"""Failure detection on the GPU without a GPU fault: the device wall-clock
guard of the solve's device-side loops.  A solve that outlives
opts.max_seconds stops on the device, returns OSM_E_TIMEOUT, and leaves the
handle and the CUDA context usable."""
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
