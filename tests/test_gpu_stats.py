"""osm_stats counts the rows the CG-step kernels processed (the bench's
solve-level HBM fraction is built on it).  On a symmetric 2 x 2 x 2
decomposition every subdomain has the same unknowns, SELL rows and box rows,
so one Schwarz iteration must give (sum of the subdomains' CG steps) x (rows
of one subdomain)."""
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec, op", [("fp64", None), ("mixed", 1), ("mixed", 2)])
def test_row_step_counters(prec, op):
    import paper_2112_03851_gb300 as pkg
    prob = gen.sphere_problem(16, 2, 10.0)
    opts = {} if op is None else {"fp32_operator": op}
    sol = pkg.Solver.from_problem(prob, prec=prec, mixed_inner_rtol=0.4, max_outer=500, **opts)
    i = sol.info
    sol.iterate(1)
    st = sol.stats()
    steps = int(sol.inner_iters().sum())
    assert steps > 0
    assert st["sub_row_steps"] == steps * (i["n_local"] // 8)
    box = prec == "mixed" and i["fp32_operator"] == 2
    assert box == (op == 2)
    assert st["op_row_steps"] == steps * ((i["box_rows"] if box else i["vec_rows"]) // 8)
    # a whole solve: summed over its Schwarz iterations, between the batched
    # step count and n_sub times it
    sol.solve(1e-8)
    st = sol.stats()
    total = st["sub_row_steps"] // (i["n_local"] // 8)
    assert st["n_cg_steps"] <= total <= 8 * st["n_cg_steps"]
    assert st["op_row_steps"] == total * ((i["box_rows"] if box else i["vec_rows"]) // 8)
