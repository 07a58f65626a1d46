"""Host-side helpers of bench.py (no GPU): rooflines and the per-kernel source
hash that keys the committed ncu traffic."""
import json
from pathlib import Path

import bench


class _FakeSolver:
    info = {"nnz": 129_600_000, "n_local": 2_197_000, "n_slices": 70_000, "col_bytes_fp64": 4, "col_bytes_fp32": 2,
            "vec_rows": 2_200_000, "box_rows": 0, "fp32_operator": 1}

    def spmv_bytes(self, prec=0):
        vb = 8 if prec in (0, 3) else 4
        cb = self.info["col_bytes_fp64"] if prec in (0, 3) else self.info["col_bytes_fp32"]
        extra = 12 * self.info["n_local"] if prec == 2 else 0
        return self.info["nnz"] * (vb + cb) + self.info["n_slices"] * 8 + self.info["n_local"] * 2 * vb + extra

    def profile_spmv(self, reps=20, prec=0):
        return 0.25


def test_alu_roofline_counts_one_fma_per_nonzero():
    r = bench._roofline_alu(_FakeSolver(), 0.2592)
    assert r["bound"] == "alu" and r["unit"] == "GFLOP/s"
    assert abs(r["achieved"] - 1000.0) < 0.1 and abs(r["frac"] - 1000.0 / bench.FP64_FMA_PEAK_GFLOPS) < 1e-4


def test_hbm_roofline_fields():
    r = bench._roofline(_FakeSolver(), 3, "k")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["ms_per_launch"] == 0.25
    assert r["algorithmic_bytes"] == _FakeSolver().spmv_bytes(3)
    assert abs(r["achieved"] - r["algorithmic_bytes"] / 0.25e-3 / 1e9) < 0.1
    assert r["traffic"] is None                      # another launch size than the committed capture


def test_traffic_key_matches_the_committed_capture():
    """The committed ncu traffic of the bench workload's kernels is keyed to
    their current source and launch size: editing a kernel (or a helper it
    calls), or another workload, drops it."""
    d = json.loads(Path(bench.TRAFFIC_FILE).read_text())
    for name, e in d["entries"].items():
        assert e["kernel_hash"] == bench._kernel_hash(e["kernel"]), name
        assert bench._traffic_per_launch(name, e["rows"]) == e["dram_bytes_read"] + e["dram_bytes_write"]
        assert bench._traffic_per_launch(name, e["rows"] + 256) is None


def test_solve_level_fraction_counts_the_rows_processed():
    """bytes per solve = (CG-step bytes per row) x (rows the CG-step kernels
    processed) [+ the mixed tensor form's per-iteration start]; the fraction
    is those bytes over the solve time against the copy bandwidth."""
    sol = _FakeSolver()
    m = {"op_row_steps": 1_000_000_000, "schwarz_iterations": 100, "ms_per_step": 1000.0}
    r = bench._solve_hbm(sol, "fp64", m)
    per_row = sol.spmv_bytes(3) / sol.info["vec_rows"] + bench.UPD64_BYTES_PER_ROW + bench.DIR64_BYTES_PER_ROW
    assert r["bytes_per_solve"] == int(per_row * 1e9)
    peak, _ = bench._peaks()
    assert abs(r["frac"] - r["bytes_per_solve"] / 1.0 / 1e9 / peak) < 1e-4
    sol.info = dict(sol.info, fp32_operator=2, box_rows=2_300_000)
    sol.spmv_bytes = lambda prec=0: sol.info["box_rows"] * (8 + (12 if prec == 2 else 0))
    r = bench._solve_hbm(sol, "mixed", m)
    want = (20 + bench.UPD32_BYTES_PER_ROW) * 1e9 + bench.MIXED_OUTER_BYTES_PER_ROW * 2_300_000 * 100
    assert abs(r["bytes_per_solve"] - want) <= 1 and "tensor" in r["counted"]


def test_double_float_start_roofline_counts_fp32_operations():
    """The double-float refinement start is reported against the measured
    FP32 rate: DF_OPS_PER_ROW FP32 operations per box row (12 per compensated
    multiply-add, 3 per renormalisation of the four intermediate sums)."""
    assert bench.DF_OPS_PER_ROW == 35 * 12 + 4 * 3
    sol = _FakeSolver()
    sol.info = dict(sol.info, fp32_operator=2, fp64_start=3, box_rows=1_000_000)
    r = bench._roofline_fp64_start(sol)
    assert r["bound"] == "alu" and r["unit"] == "G FP32 ops/s" and r["peak"] == bench.FP32_OPS_PEAK_G
    want = bench.DF_OPS_PER_ROW * 1e6 / 0.25e-3 / 1e9
    assert abs(r["achieved"] - want) < 0.1 and abs(r["frac"] - want / bench.FP32_OPS_PEAK_G) < 1e-4
