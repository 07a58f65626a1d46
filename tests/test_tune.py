"""Inner-tolerance autotuner (host logic, no GPU): the cache key follows the
mesh, cuts, p and rtol, and a cached choice is reused without timing."""
import json

import gen
from paper_2112_03851_gb300 import tune


def test_problem_key_follows_what_the_balance_depends_on():
    a = gen.sphere_problem(4, 2, 1.0)
    b = gen.sphere_problem(4, 2, 1.0)
    assert tune.problem_key(a, 2.0, 1e-8) == tune.problem_key(b, 2.0, 1e-8)
    assert tune.problem_key(a, 2.0, 1e-8) != tune.problem_key(a, 3.0, 1e-8)
    assert tune.problem_key(a, 2.0, 1e-8) != tune.problem_key(a, 2.0, 1e-9)
    c = gen.sphere_problem(4, 1, 1.0)
    assert tune.problem_key(a, 2.0, 1e-8) != tune.problem_key(c, 2.0, 1e-8)


def test_cached_choice_is_reused(tmp_path, monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "test-gpu")
    path = tmp_path / "cache.json"
    rec = {"best": 0.3, "candidates": [0.3, 0.4], "ms": {"0.3": 1.0, "0.4": 2.0},
           "schwarz_iterations": {"0.3": 10, "0.4": 12}, "gpu": "test-gpu"}
    path.write_text(json.dumps({"k|test-gpu": rec}))

    def never(tol):
        raise AssertionError("a cached choice must not build solvers")
    best, out = tune.tune_inner_rtol(never, "k", candidates=(0.3, 0.4), cache=str(path))
    assert best == 0.3 and out["cached"]
