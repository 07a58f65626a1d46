"""osm_apply_noalloc: the subdomain operator for callers that cannot allocate
device memory where they need it (a plug-in under a host framework's own,
capped allocator; a caller whose memory budget is fixed at start-up).  It
must give osm_apply's result, through the C ABI, using only the library's
fixed scratch array -- also on a second call in a row, into a caller's
preallocated output, and after another handle with a different layout has
used the same scratch -- and must allocate no device memory.

This file is collected last so that a failure here cannot hide the other
tests' results in a run that stops at the first failure.
"""
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


def _check_pair(torch, sol, x, op):
    y_ref = sol.apply(x, op=op)
    y = sol.apply_noalloc(x, op=op)
    scale = float(y_ref.abs().max())
    # same SELL kernels on the same data: the SpMV tolerance of the parity tests
    assert float((y - y_ref).abs().max()) <= 1e-13 * scale
    return y


def test_noalloc_matches_apply_twice_and_across_handles(osm):
    import torch
    rng = np.random.default_rng(5)
    a = osm.Solver.from_problem(gen.sphere_problem(16, 2, 10.0), p=3.0)
    b = osm.Solver.from_problem(gen.regional_problem(nx=12, ny=10, nz=8, sx=3, sy=2, sz=2, p=2.0,
                                                     seed=4, lx=10.0, ly=8.0, lz=3.0), p=2.0)
    for sol in (a, b, a):
        n = sol.info["n_local"]
        for op in (0, 1):
            x1 = torch.from_numpy(rng.standard_normal(n)).cuda()
            x2 = torch.from_numpy(rng.standard_normal(n) * 1e3).cuda()
            _check_pair(torch, sol, x1, op)
            _check_pair(torch, sol, x2, op)   # second call in a row, new data


def test_noalloc_rejects_problems_beyond_its_scratch(osm):
    import torch
    prob = gen.layered_problem(48, 3, p=10.0, seed=0)   # about 0.9M padded rows > 2^19
    sol = osm.Solver.from_problem(prob)
    assert sol.info["vec_rows"] > (1 << 19)
    x = torch.zeros(sol.info["n_local"], dtype=torch.float64, device="cuda")
    with pytest.raises(osm.OsmError, match="scratch"):
        sol.apply_noalloc(x)


def test_noalloc_into_preallocated_output_allocates_nothing(osm):
    """The form a capped-allocator caller uses: x and y are its own tensors.
    After one warm call, further calls leave the library's device memory,
    torch's allocator and the device's free memory unchanged."""
    import torch
    rng = np.random.default_rng(11)
    sol = osm.Solver.from_problem(gen.sphere_problem(16, 2, 10.0), p=3.0)
    n = sol.info["n_local"]
    xs = [torch.from_numpy(rng.standard_normal(n)).cuda() for _ in range(3)]
    refs = [sol.apply(x, op=0) for x in xs]
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    outs = [torch.empty_like(y) for _ in xs]       # results are copied out: no temporaries in the loop
    sol.apply_noalloc(xs[0], y=y)                  # warm: device address of the scratch looked up
    torch.cuda.synchronize()
    lib_bytes = sol.info["device_bytes"]
    torch_bytes = torch.cuda.memory_allocated()
    torch_reserved = torch.cuda.memory_reserved()
    free0, _ = torch.cuda.mem_get_info()
    for x, o in zip(xs, outs):
        out = sol.apply_noalloc(x, y=y)
        assert out.data_ptr() == y.data_ptr()
        o.copy_(y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    info = osm._lib.OsmInfo()
    osm._lib.load().osm_info(sol._h, osm._lib.C.byref(info))
    assert info.device_bytes == lib_bytes
    assert torch.cuda.memory_allocated() == torch_bytes
    assert torch.cuda.memory_reserved() == torch_reserved
    assert free1 >= free0
    for o, ref in zip(outs, refs):
        assert float((o - ref).abs().max()) <= 1e-13 * float(ref.abs().max())
