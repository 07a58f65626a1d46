"""Benchmark: DOF/s of the optimized Schwarz gravimetry solve on one GB300.

One step = one full Schwarz solve (Robin RHS, batched subdomain Jacobi-PCG,
Robin exchange, global residual -- every step of the hot path) from u = 0
to a relative residual of 1e-8 on the regional workload: a 100 x 100 x 30
box, Q2 on 128 x 128 x 48 elements graded in z, 192 subdomains of uneven
size from jittered cuts (6,177,375 unknowns), Gaussian-random-field density
plus a basin.  The headline is the mixed form (FP32 subdomain CG inside FP64
refinement); the FP64 form (the paper's setting) and the FP64 refinement
form are sub-lines with their own, stated step counts (each solve takes
10-60 s).  The subdomain matrices and vectors (about 9 GB) are larger than
L2, so no flush is needed between steps.  Every line states the relative L2
error of its solution against the FP64 oracle's monolithic solve (PCG to
1e-13), computed on the host cores while the GPU is timed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun with N > 1 every rank solves
its own replica of the workload (the solve does not shard: replicas only);
the value is the units of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF/s solved to 1e-8 rel residual, mixed vs FP64; SpMV GB/s vs HBM peak"
WORKLOAD = "regional"
P_ROBIN = 20.0
# Robin parameter per workload, chosen by the batched evaluation of sampled p
# (Sec. 4; osm_sample_p race mode, fewest Schwarz iterations).  regional: 16
# log-uniform p in [0.8, 3] (SplitMix64 seed 0), mixed form, winner 1.6664
# at 660 iterations; layered64: 20 from the sweeps of the 64^3 workload.
P_FOR = {"layered64": 20.0, "regional": 1.6664, "regional_mid": 1.6664, "layered160": 40.0, "layered48": 10.0}
RTOL = 1e-8
INNER_RTOL = 1e-10
MIXED_INNER_RTOL = 0.4
FALLBACK_HBM = 6800.0
SUB_WARMUP, SUB_STEPS = 1, 2     # the FP64 and FP64-refinement sub-lines
E2E_STEPS = 5                    # end-to-end solves through the public API (headline)
ORACLE_TOL = 1e-13               # the oracle's monolithic PCG
ORACLE_WAIT_S = 1500.0           # longest wait for the oracle after the GPU work


def _is_slab(name):
    return name.startswith("slab")


def _rtol_for(name):
    # Table 2 runs the slab partitions to a residual of 1e-6
    return 1e-6 if _is_slab(name) else RTOL


def _tc_for(prob, name):
    """Transmission coefficients of a workload: the slab partitions use the
    unsymmetric second-order condition optimised by CMA-ES on the Fourier
    rate over the interface's frequency band (Sec. 4-6): from the lowest
    Dirichlet mode of the 250 x 15 face to pi over the tangential node
    spacing.  Others: None (zeroth-order Robin, P_FOR)."""
    if not _is_slab(name):
        return None
    from paper_2112_03851_gb300 import search
    ly, lz = prob.yc[-1] - prob.yc[0], prob.zc[-1] - prob.zc[0]
    h = min(float((prob.yc[1:] - prob.yc[:-1]).min()), float((prob.zc[1:] - prob.zc[:-1]).min()))
    tc, rho, band = search.transmission_for_faces(ly, lz, h, "oo2_unsym", seed=0, max_iter=2000)
    return tc, float(rho), band


def _workload_desc(prob, p, name=WORKLOAD, tc=None):
    if name == "regional":
        dens = ("Gaussian random field (l=5, sigma=100) + basin -250, 100x100x30 box graded 1.05 in z, "
                "uneven jittered cuts")
    elif _is_slab(name):
        dens = ("250x250x15 box, slabs along x (Sec. 6 partition), layered crust + buried crater "
                "(breccia lens -250, central uplift +200, peak ring +100) + N(0,10^2) noise")
    else:
        dens = "unit cube, 3 density layers + 20 random spheres"
    cond = (f"oo2 unsymmetric (p_lo, q_lo, p_hi, q_hi) = ({', '.join(f'{v:.4g}' for v in tc[0])}), "
            f"Fourier rho_max {tc[1]:.4f} on k in [{tc[2][0]:.4g}, {tc[2][1]:.4g}]" if tc else f"Robin p={p:g}")
    return (f"{name}: Q2 {prob.nx}x{prob.ny}x{prob.nz} elements ({prob.n_dofs:,} unknowns), "
            f"{len(prob.cx)-1}x{len(prob.cy)-1}x{len(prob.cz)-1} subdomains, {dens} (seed 0), {cond}, "
            f"Schwarz to {_rtol_for(name):g}")


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def _definitions(text):
    """name -> source text of every function defined at column 0 (from its
    template line to the closing brace at column 0)."""
    import re
    lines = text.split("\n")
    out = {}
    for i, ln in enumerate(lines):
        m = re.match(r"(?:__global__|__device__)[^(]*?\b(\w+)\(", re.sub(r"__launch_bounds__\([^)]*\)", "", ln))
        if not m:
            continue
        start = i
        while start > 0 and lines[start - 1].startswith("template"):
            start -= 1
        end = next(j for j in range(i, len(lines)) if lines[j] == "}")
        out[m.group(1)] = "\n".join(lines[start:end + 1])
    return out


def _kernel_hash(kernel):
    """Hash of one kernel's source.  SELL kernels: their definition and,
    transitively, the device helpers they call (osm_kernels.cu,
    osm_device.cuh).  The tensor-product kernel (one template for all its
    modes): osm_tensor.cu with osm_device.cuh."""
    import re
    csrc = os.path.join(ROOT, "paper_2112_03851_gb300", "csrc")
    if kernel.startswith("k_tensor"):
        h = hashlib.sha256()
        for name in ("osm_tensor.cu", "osm_device.cuh"):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(f.read())
        return h.hexdigest()[:16]
    defs = {}
    for name in ("osm_device.cuh", "osm_kernels.cu"):
        with open(os.path.join(csrc, name)) as f:
            defs.update(_definitions(f.read()))
    seen, todo = [], [kernel]
    while todo:
        k = todo.pop()
        if k in seen or k not in defs:
            continue
        seen.append(k)
        todo += [n for n in re.findall(r"\b(\w+)\s*[<(]", defs[k]) if n in defs and n != k]
    h = hashlib.sha256()
    for k in sorted(seen):
        h.update(defs[k].encode())
    return h.hexdigest()[:16]


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_regional.json")


def _traffic_per_launch(entry, rows):
    """DRAM bytes (read + write) of one launch of a kernel from the committed
    ncu capture on the bench workload (profiles/traffic_regional.json), if it
    was taken on the current kernel source and a launch of the same size
    (rows: box rows for the tensor kernels, vector rows for SELL); else
    None."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        e = d["entries"][entry]
        if e.get("kernel_hash") != _kernel_hash(e["kernel"]) or int(e["rows"]) != int(rows):
            return None
        return int(e["dram_bytes_read"]) + int(e["dram_bytes_write"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_over_ranks(ms_local, units_local, device=None):
    """Whole-job throughput of independent replicas: every rank processed
    units_local in ms_local; the job takes the slowest rank's time (all-reduce
    MAX) and processed the sum of the units (all-reduce SUM).  Returns
    (value per second, slowest ms).  Works on any torch.distributed backend
    (NCCL on the GPUs, gloo in the CPU tests); single process without one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units_local / (ms_local / 1e3), ms_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) / 1e3), float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_baseline(prob, p, n_outer_needed, name=WORKLOAD, budget_s=20.0):
    """The oracle's sequential Schwarz (OpenMP over subdomains) on the same
    workload: time a bounded number of Schwarz iterations, scale to the
    iterations the solve needs."""
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    threads = int(os.environ["OMP_NUM_THREADS"])
    import oracle
    t0 = time.perf_counter()
    S = oracle.Schwarz.from_problem(prob, p=p)
    setup = time.perf_counter() - t0
    done, t_iter = 0, 0.0
    while done < n_outer_needed and (t_iter < budget_s or done == 0):
        t = time.perf_counter()
        S.iterate(inner_rtol=INNER_RTOL)
        t_iter += time.perf_counter() - t
        done += 1
    per_iter = t_iter / done
    value = prob.n_dofs / (per_iter * n_outer_needed)
    return {"value": value, "unit": "DOF/s", "cores": threads, "kind": "oracle",
            "sample": (f"{done} of {n_outer_needed} Schwarz iterations of the FP64 oracle on {name} "
                       f"({per_iter:.2f} s each, OpenMP over subdomains; setup {setup:.1f} s excluded), "
                       f"solve time extrapolated to {n_outer_needed} iterations")}


def run_reference(args):
    """The reference arm: the FP64 oracle (the paper's method in plain C on
    the host cores) on the bench workload.  Each step is one of its Schwarz
    iterations (subdomain PCG to 1e-10, Sec. 6, OpenMP over subdomains);
    DOF/s = unknowns / (mean step time x the oracle's own iteration count to
    1e-8, tests/golden/<workload>_iterations.json)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import gen
    name = args.workload or WORKLOAD
    prob = gen.workload(name)
    p_robin = P_FOR.get(name, P_ROBIN)
    n_outer = _reference_iterations(name)
    threads = int(os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1)))
    import oracle
    S = oracle.Schwarz.from_problem(prob, p=p_robin)
    for _ in range(args.warmup):
        S.iterate(inner_rtol=INNER_RTOL)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        S.iterate(inner_rtol=INNER_RTOL)
        times.append(time.perf_counter() - t)
    per_iter = sum(times) / len(times)
    value = prob.n_dofs / (per_iter * n_outer)
    sample = (f"each step: one Schwarz iteration of the FP64 oracle on {name} (OpenMP over subdomains, after "
              f"{args.warmup} warm-up iterations); DOF/s = unknowns / (mean step time x {n_outer} oracle "
              f"iterations to {RTOL:g})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_iter * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": _workload_desc(prob, p_robin, name)},
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _reference_iterations(name=WORKLOAD):
    """The FP64 oracle's Schwarz iteration count to 1e-8 on a workload, from
    the committed record written by tests/golden/make_iterations.py."""
    path = os.path.join(ROOT, "tests", "golden", f"{name}_iterations.json")
    try:
        with open(path) as f:
            return int(json.load(f)["schwarz_iterations"])
    except Exception:
        return 150


def _measure(sol, prob, warmup, steps, e2e_steps, ws, local, barrier, use_graph_note, rtol=RTOL):
    """Warm-up, the timed region (CUDA events, clocks sampled) and, if
    e2e_steps > 0, the end-to-end run through the public API from host
    buffers."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    phi = torch.zeros(sol.info["n_nodes"], dtype=torch.float64, device="cuda")
    for _ in range(max(warmup, 1)):
        sol.solve(rtol, phi=phi)
    st = sol.stats()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    rel = None
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            _, it, rel = sol.solve(rtol, phi=phi)
            launches += sol.stats()["n_launches"]
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1) / steps
    value, ms_max = aggregate_over_ranks(ms, prob.n_dofs, device="cuda")
    out = {
        "value": value, "ms_per_step": ms_max, "steps": steps, "warmup": max(warmup, 1), "relres": rel,
        "schwarz_iterations": st["n_outer"], "cg_steps_per_solve": st["n_cg_steps"],
        "launches_per_step": int(st["n_launches"]), "gpu_launches": int(launches),
        "op_row_steps": int(st["op_row_steps"]), "sub_row_steps": int(st["sub_row_steps"]),
        "clocks": clk.summary(), "launch_mode": use_graph_note,
        "_phi": phi.cpu().numpy(),
    }
    if e2e_steps > 0:
        # end to end through the public API: every step copies the density
        # from pinned host memory to the device, assembles the load there
        # (osm_set_density_dev), solves, and copies the solution back to
        # pinned host memory
        phi_host = torch.empty(sol.info["n_nodes"], dtype=torch.float64, pin_memory=True)
        drho_host = torch.from_numpy(np.ascontiguousarray(prob.drho, dtype=np.float64)).pin_memory()
        drho_dev = torch.empty(drho_host.shape, dtype=torch.float64, device="cuda")
        drho_dev.copy_(drho_host)
        sol.set_density_dev(drho_dev)        # first call allocates the device assembly data
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            drho_dev.copy_(drho_host, non_blocking=True)
            sol.set_density_dev(drho_dev)
            sol.solve(rtol, phi=phi)
            phi_host.copy_(phi, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        e2e_value, _ = aggregate_over_ranks(e2e_s * 1e3, prob.n_dofs, device="cuda")
        out["e2e"] = {"value": e2e_value, "unit": "DOF/s", "steps": e2e_steps,
                      "h2d_bytes_per_step": int(drho_host.numel()) * 8,     # the density, one FP64 per element
                      "d2h_bytes_per_step": sol.info["n_nodes"] * 8}        # phi
    return out


def _oracle_job(name, path, threads):
    """The oracle's monolithic FP64 solve of a workload (Jacobi-PCG to
    ORACLE_TOL), run in a spawned process on the host cores while the GPU
    is timed; writes the full-grid solution (.npy) and its record (.json)."""
    os.environ["OMP_NUM_THREADS"] = str(threads)
    import numpy as np

    import gen
    import oracle
    t0 = time.perf_counter()
    prob = gen.workload(name)
    G = oracle.GlobalSystem(prob.xc, prob.yc, prob.zc, prob.drho)
    t_asm = time.perf_counter() - t0
    x, it, rel = G.solve(tol=ORACLE_TOL)
    np.save(path, G.to_grid(x))
    with open(path + ".json", "w") as f:
        json.dump({"pcg_iterations": int(it), "relres": float(rel), "assembly_s": round(t_asm, 1),
                   "seconds": round(time.perf_counter() - t0, 1), "threads": threads}, f)


class OracleSolution:
    """The oracle's solution of the bench workload, computed concurrently."""

    def __init__(self, name):
        import multiprocessing as mp
        self.dir = tempfile.mkdtemp(prefix="osm_oracle_")
        self.path = os.path.join(self.dir, "phi.npy")
        cores = os.cpu_count() or 1
        self.threads = max(1, cores - 2)        # leave the bench's host thread and the clock sampler a core
        self.t0 = time.perf_counter()
        self.proc = mp.get_context("spawn").Process(target=_oracle_job, args=(name, self.path, self.threads),
                                                    daemon=True)
        self.proc.start()
        self.phi = None
        self.record = None

    def wait(self, limit_s):
        self.proc.join(timeout=max(1.0, limit_s - (time.perf_counter() - self.t0)))
        if self.proc.is_alive():
            self.proc.terminate()
            self.proc.join(timeout=10)
            self.record = {"error": f"oracle solve not finished within {limit_s:.0f} s"}
            return False
        try:
            import numpy as np
            self.phi = np.load(self.path)
            with open(self.path + ".json") as f:
                self.record = json.load(f)
        except Exception as e:          # the child failed
            self.record = {"error": f"oracle solve failed: {e!r} (exit code {self.proc.exitcode})"}
            return False
        return True

    def rel_l2(self, phi):
        import numpy as np
        if self.phi is None:
            return None
        return float(np.linalg.norm(phi - self.phi) / np.linalg.norm(self.phi))

    def close(self):
        import shutil
        if self.proc.is_alive():
            self.proc.terminate()
        shutil.rmtree(self.dir, ignore_errors=True)


FP64_FMA_PEAK_GFLOPS = 1256.0   # measured FP64 FMA throughput (profiles/peaks.md)


def _roofline_alu(sol, ms):
    """The FP64 CG-step SpMV against the FP64 FMA pipe: two flops per nonzero
    (one DFMA) in `ms` per launch."""
    achieved = 2.0 * sol.info["nnz"] / (ms / 1e3) / 1e9
    return {"bound": "alu", "achieved": round(achieved, 1), "peak": FP64_FMA_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": round(achieved / FP64_FMA_PEAK_GFLOPS, 4),
            "peak_kind": "measured FP64 FMA probe (152 SMs x 2 DFMA/clk x 2.07 GHz = 1.26 TFLOP/s nominal)"}


def _roofline(sol, prec, name):
    """Roofline of a CG-step kernel timed alone with every subdomain active
    (prec 2: the FP32 CG step, tensor-product or SELL; 3: k_cg_spmv<double>):
    algorithmic bytes per launch over the CUDA-event time, against the
    measured copy bandwidth."""
    ms = sol.profile_spmv(20, prec=prec)
    nbytes = sol.spmv_bytes(prec)
    peak, kind = _peaks()
    achieved = nbytes / (ms / 1e3) / 1e9
    tensor = prec == 2 and sol.info.get("fp32_operator") == 2
    if tensor:
        traffic = _traffic_per_launch("k_tensor_cg_step", sol.info["box_rows"])
    elif prec == 3:
        traffic = _traffic_per_launch("k_cg_spmv_double", sol.info["vec_rows"])
    else:
        traffic = None
    out = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
           "frac": round(achieved / peak, 4), "traffic": traffic,
           "kernel": name, "peak_kind": f"{kind} hbm_gbs (copy), burst (kernel timed alone)",
           "ms_per_launch": round(ms, 5), "algorithmic_bytes": nbytes}
    if not tensor:
        out["col_bytes"] = sol.info["col_bytes_fp64" if prec in (0, 3) else "col_bytes_fp32"]
    return out


# FP64 multiply-adds per box row of the tensor-product operator's sum
# factorisation: 5-tap bands, y pass 2 x 5, x pass 3 x 5, z pass 2 x 5.
TENSOR_FMA_PER_ROW = 35


# FP32 operations per box row of the double-float sum factorisation: 12 per
# compensated multiply-add (product split by one FMA, two cross-term FMAs, a
# two-sum and the error gathering) and 3 per renormalisation of the four
# intermediate sums (My z, K~y z, P, Q).
DF_OPS_PER_ROW = TENSOR_FMA_PER_ROW * 12 + 4 * 3
FP32_OPS_PEAK_G = 73300.0 / 2   # measured FP32 FMA rate (profiles/peaks.md) in G lane operations per second


def _roofline_fp64_start(sol):
    """The mixed refinement step's start (prec 4) timed alone: on the tensor
    form in FP64 it is bound by the FP64 FMA pipe (2 flops per multiply-add,
    TENSOR_FMA_PER_ROW per box row, against the measured FP64 FMA rate); in
    double-float arithmetic by FP32 issue (DF_OPS_PER_ROW FP32 operations per
    box row against the measured FP32 FMA rate); on SELL it is the FP64 SpMV
    (HBM)."""
    ms = sol.profile_spmv(20, prec=4)
    if sol.info.get("fp64_start") == 3:
        ops = float(DF_OPS_PER_ROW) * sol.info["box_rows"]
        achieved = ops / (ms / 1e3) / 1e9
        return {"bound": "alu", "achieved": round(achieved, 1), "peak": FP32_OPS_PEAK_G, "unit": "G FP32 ops/s",
                "frac": round(achieved / FP32_OPS_PEAK_G, 4),
                "traffic": _traffic_per_launch("k_tensor_df_start", sol.info["box_rows"]),
                "kernel": "k_tensor<Df, 2> (double-float tensor-product defect d = b - A u and FP32 CG start)",
                "peak_kind": "measured FP32 FMA probe (152 SMs x 128 FFMA/clk x 2.07 GHz = 40.3 T lane ops/s "
                             "nominal)", "ms_per_launch": round(ms, 5), "algorithmic_fp32_ops": ops}
    if sol.info.get("fp64_start") == 2:
        flops = 2.0 * TENSOR_FMA_PER_ROW * sol.info["box_rows"]
        achieved = flops / (ms / 1e3) / 1e9
        return {"bound": "alu", "achieved": round(achieved, 1), "peak": FP64_FMA_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": round(achieved / FP64_FMA_PEAK_GFLOPS, 4),
                "traffic": _traffic_per_launch("k_tensor_fp64_start", sol.info["box_rows"]),
                "kernel": "k_tensor<double, 2> (FP64 tensor-product defect d = b - A u and FP32 CG start)",
                "peak_kind": "measured FP64 FMA probe (152 SMs x 2 DFMA/clk x 2.07 GHz = 1.26 TFLOP/s nominal)",
                "ms_per_launch": round(ms, 5), "algorithmic_flops": flops}
    nbytes = sol.spmv_bytes(0)
    peak, kind = _peaks()
    achieved = nbytes / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None,
            "kernel": "k_cg_init_mixed (FP64 SELL defect d = b - A u and FP32 CG start)",
            "peak_kind": f"{kind} hbm_gbs (copy), burst (kernel timed alone)", "ms_per_launch": round(ms, 5),
            "algorithmic_bytes": nbytes}


# Algorithmic bytes per row of the CG-step kernels, per CG step of a
# subdomain: the FP32 update (k_cg_update32) reads p, x, q, r and D^-1 and
# writes x, r and z (4 B each); the FP64 update (k_cg_update_a) the same in
# 8 B, and the FP64 direction (k_cg_direction) reads z and p and writes p.
UPD32_BYTES_PER_ROW = 32
UPD64_BYTES_PER_ROW = 64
DIR64_BYTES_PER_ROW = 24
# Per Schwarz iteration of the mixed form on the tensor-product form, per box
# row: the start reads u (8 B, FP64 or a float pair), b, D^-1 (FP32) and the
# box-to-vector map and writes y, r, z and x (FP32); the correction reads x
# and u and writes u and its two box mirrors (FP64 and float pairs).
MIXED_OUTER_BYTES_PER_ROW = 44 + 36


def _solve_hbm(sol, prec, m):
    """Solve-level HBM fraction: algorithmic bytes of one solve over its
    measured time.  Counted: the CG-step kernels at the rows they actually
    processed (osm_stats op_row_steps: each subdomain's CG steps times the
    rows its kernels sweep) and, for the mixed form on the tensor-product
    operator, the FP64 start and correction once per Schwarz iteration.  Not
    counted: the exchange, the averaging and the stop test (interface rows
    and a few vector sweeps per Schwarz iteration), so this is a lower bound."""
    i = sol.info
    rows = m["op_row_steps"]
    if prec == "mixed" and i.get("fp32_operator") == 2:
        per_row = sol.spmv_bytes(2) / i["box_rows"] + UPD32_BYTES_PER_ROW
        outer = MIXED_OUTER_BYTES_PER_ROW * i["box_rows"] * m["schwarz_iterations"]
        counted = "tensor CG step + FP32 update at the rows processed; FP64 start + correction per Schwarz iteration"
    elif prec == "mixed":
        per_row = sol.spmv_bytes(2) / i["vec_rows"] + UPD32_BYTES_PER_ROW
        outer = 0
        counted = "SELL FP32 CG step + FP32 update at the rows processed"
    else:
        per_row = sol.spmv_bytes(3) / i["vec_rows"] + UPD64_BYTES_PER_ROW + DIR64_BYTES_PER_ROW
        outer = 0
        counted = "SELL FP64 CG step (SpMV, update, direction) at the rows processed"
    nbytes = per_row * rows + outer
    peak, kind = _peaks()
    achieved = nbytes / (m["ms_per_step"] / 1e3) / 1e9
    return {"bytes_per_solve": int(nbytes), "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "op_row_steps": rows, "counted": counted,
            "peak_kind": f"{kind} hbm_gbs (copy)", "note": "lower bound: per-iteration exchange, averaging and "
            "stop-test kernels not counted"}


def _spmv_roofline_sell32(sol):
    """The FP32 SELL CG-step SpMV (k_cg_spmv_dir32) from the autotuner's
    timing of its fastest variant (CUDA events, timed alone, every subdomain
    active): the metric's 'SpMV GB/s' on this workload, also when the solve
    itself runs the tensor-product operator."""
    i = sol.info
    ms_all = [m for m in list(i["spmv_ms_fp32"]) + list(i["spmv_ms16_fp32"]) if m > 0]
    if not ms_all:
        return None
    ms = min(ms_all)
    k = (list(i["spmv_ms_fp32"]) + list(i["spmv_ms16_fp32"])).index(ms)
    cb = 2 if k >= 2 else 4
    nbytes = i["nnz"] * (4 + cb) + i["n_slices"] * 8 + i["n_local"] * 8 + 12 * i["n_local"]
    peak, kind = _peaks()
    achieved = nbytes / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "kernel": "k_cg_spmv_dir32 (batched SELL-32 FP32 SpMV of the CG "
            "step + direction epilogue, fastest variant, every subdomain active)",
            "peak_kind": f"{kind} hbm_gbs (copy), burst (kernel timed alone)", "ms_per_launch": round(ms, 5),
            "algorithmic_bytes": nbytes, "col_bytes": cb, "source": "autotuner timing at setup"}


def run_ours(args):
    import torch

    import gen
    ws, rank, local = _dist()
    name = args.workload or WORKLOAD
    single = name not in ("batch64", "sample32", "grad48")
    # the oracle's monolithic solve runs on the host cores while the GPU is
    # timed (a spawned process: no CUDA state is inherited)
    orc = None
    if single and rank == 0 and ws == 1 and not args.no_oracle and not _is_slab(name):
        orc = OracleSolution(name)
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2112_03851_gb300 as pkg
    try:
        pkg.load()
    except ImportError:
        from paper_2112_03851_gb300 import build as b
        b.build()
        pkg.load()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    if name == "batch64":
        return run_batch(args, pkg, ws, rank, local, barrier)
    if name == "sample32":
        return run_sample(args, pkg, ws, rank, local, barrier)
    if name == "grad48":
        return run_grad(args, pkg, ws, rank, local, barrier)
    prob = gen.workload(name)
    p_robin = P_FOR.get(name, P_ROBIN)
    tc = _tc_for(prob, name)
    rtol = _rtol_for(name)
    use_graph = 0 if args.launch == "host" else 1
    note = "one CUDA graph per solve" if use_graph else "host-driven launches (profiling mode)"
    res = {}
    precs = ["mixed", "fp64", "fp64_refine"] if args.prec == "both" else [args.prec]
    head = precs[0]
    # the mixed form's inner tolerance, tuned on this workload and GPU (cached)
    tin, tune_rec = MIXED_INNER_RTOL, None
    if "mixed" in precs and not args.no_tune:
        from paper_2112_03851_gb300 import tune

        def make(t):
            return pkg.Solver.from_problem(prob, p=p_robin, tc=tc[0] if tc else None, inner_rtol=INNER_RTOL,
                                           max_outer=5000, prec="mixed", mixed_inner_rtol=t, use_graph=use_graph)
        tin, tune_rec = tune.tune_inner_rtol(make, tune.problem_key(prob, p_robin, rtol), rtol=rtol)
        torch.cuda.empty_cache()
    for prec in precs:
        sol = pkg.Solver.from_problem(prob, p=p_robin, tc=tc[0] if tc else None, inner_rtol=INNER_RTOL,
                                      max_outer=5000, prec=prec, mixed_inner_rtol=tin,
                                      use_graph=use_graph)
        if prec == head:
            r = _measure(sol, prob, args.warmup, args.steps, min(args.steps, E2E_STEPS), ws, local, barrier, note,
                         rtol)
        else:
            r = _measure(sol, prob, SUB_WARMUP, SUB_STEPS, 0, ws, local, barrier, note, rtol)
        r["setup_s"] = round(sol.info["setup_seconds"], 2)
        res[prec] = r
        if prec == "mixed":
            r["fp32_operator"] = {1: "SELL-32 matrix", 2: "tensor-product (matrix-free)"}.get(sol.info["fp32_operator"])
            r["fp64_start"] = {1: "FP64 SELL SpMV", 2: "FP64 tensor-product kernel",
                               3: "double-float tensor-product kernel (~48-bit)"}.get(sol.info["fp64_start"])
            r["roofline_dominant"] = (_roofline(sol, 2, "k_tensor32 (tensor-product FP32 operator of the CG step + "
                                                       "direction epilogue, every subdomain active)")
                                      if sol.info["fp32_operator"] == 2 else
                                      _roofline(sol, 2, "k_cg_spmv_dir32 (batched SELL-32 FP32 SpMV of the CG step "
                                                       "+ direction epilogue, every subdomain active)"))
            r["spmv_roofline"] = _spmv_roofline_sell32(sol)
            r["roofline_fp64_start"] = _roofline_fp64_start(sol)
        else:
            r["roofline_dominant"] = _roofline(sol, 3, "k_cg_spmv<double> (batched SELL-32 FP64 SpMV of the CG "
                                                       "step, every subdomain active)")
            r["roofline_alu"] = _roofline_alu(sol, r["roofline_dominant"]["ms_per_launch"])
        r["solve_hbm"] = _solve_hbm(sol, prec, r)
        del sol
        torch.cuda.empty_cache()
    h = res[head]
    line = {"metric": METRIC, "value": h["value"], "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner CG + f64 refinement" if head == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": _workload_desc(prob, p_robin, name, tc),
                       "precision": (f"mixed: FP32 subdomain CG to {tin:g} of the defect "
                                     f"({h.get('fp32_operator')} operator), defect by the {h.get('fp64_start')}, "
                                     f"exchange and stop test in FP64" if head == "mixed" else "FP64"),
                       "l2": "inputs larger than L2 (several GB of subdomain matrices and vectors), no flush",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                       "launch": h["launch_mode"]},
            "gpu_launches": h["gpu_launches"], "schwarz_iterations": h["schwarz_iterations"],
            "cg_steps_per_solve": h["cg_steps_per_solve"], "relres": h["relres"],
            "setup_s": h["setup_s"], "e2e": h["e2e"], "clocks": h["clocks"],
            "roofline": h["roofline_dominant"], "solve_hbm": h["solve_hbm"]}
    if "spmv_roofline" in h:
        line["spmv_roofline"] = h["spmv_roofline"]
        line["roofline_fp64_start"] = h["roofline_fp64_start"]
    if tune_rec is not None:
        line["inner_rtol_tuning"] = tune_rec
    keys = ("value", "ms_per_step", "steps", "warmup", "schwarz_iterations", "cg_steps_per_solve", "relres",
            "gpu_launches", "clocks", "setup_s")
    if "fp64" in res and head != "fp64":
        f = res["fp64"]
        line["fp64"] = {k: f[k] for k in keys}
        line["fp64"]["precision"] = f"FP64, subdomain PCG to {INNER_RTOL:g} of ||b_i|| every iteration (Sec. 6)"
        line["fp64"]["roofline"] = f["roofline_dominant"]
        line["fp64"]["roofline_alu"] = f["roofline_alu"]
        line["fp64"]["solve_hbm"] = f["solve_hbm"]
        line["mixed_speedup_vs_fp64"] = round(h["value"] / f["value"], 3)
        line["mixed_vs_fp64_rel_l2"] = float(
            __import__("numpy").linalg.norm(h["_phi"] - f["_phi"]) / __import__("numpy").linalg.norm(f["_phi"]))
    if "fp64_refine" in res:
        f = res["fp64_refine"]
        line["fp64_refine"] = {k: f[k] for k in keys}
        line["fp64_refine"]["precision"] = (f"FP64, the mixed form's algorithm: subdomain CG to "
                                            f"{tin:g} of each iteration's defect")
        line["fp64_refine"]["roofline"] = f["roofline_dominant"]
        line["fp64_refine"]["solve_hbm"] = f["solve_hbm"]
        if head == "mixed":
            line["mixed_speedup_vs_fp64_refine"] = round(h["value"] / f["value"], 3)
    # error of every result against the FP64 oracle's monolithic solve
    if orc is not None:
        ok = orc.wait(ORACLE_WAIT_S)
        line["oracle"] = {"solve": f"monolithic Jacobi-PCG to {ORACLE_TOL:g} relative residual, FP64, "
                                   f"{orc.threads} host threads", **(orc.record or {})}
        for prec, r in res.items():
            err = orc.rel_l2(r["_phi"]) if ok else None
            tgt = line if prec == head else line.get(prec)
            if tgt is not None:
                tgt["rel_l2_vs_oracle"] = err
        orc.close()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not _is_slab(name):
        n_outer = res["fp64"]["schwarz_iterations"] if "fp64" in res else _reference_iterations(name)
        line["cpu_baseline"] = _cpu_baseline(prob, p_robin, n_outer, name)
    if _is_slab(name):
        line["cpu_baseline"] = None   # one oracle Schwarz iteration of a 19.5M-node slab run takes far too long
        line["table2_iterations"] = {"slab32": 41, "slab64": 45, "slab128": 92}[name]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args, pkg, ws, rank, local, barrier):
    """64 independent unit-cube problems (n ~ U{24..40}, 2x2x2 subdomains,
    own layered density and own log-uniform p in [2, 50]) in one handle."""
    import torch

    import gen
    probs = gen.batch_instances(64, 24, 40, seed=0)
    prec = "mixed" if args.prec == "both" else args.prec
    bs = pkg.BatchSolver(probs, prec=prec, inner_rtol=INNER_RTOL, mixed_inner_rtol=MIXED_INNER_RTOL,
                         max_outer=5000)
    dofs = sum(q.n_dofs for q in probs)
    phi = torch.zeros(bs.info["n_nodes"], dtype=torch.float64, device="cuda")
    for _ in range(max(args.warmup, 1)):
        bs.solve(RTOL, phi=phi)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        launches = 0
        for _ in range(args.steps):
            _, iters, rel = bs.solve(RTOL, phi=phi)
            launches += bs.stats()["n_launches"]
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_local = ev0.elapsed_time(ev1) / args.steps
    value, ms = aggregate_over_ranks(ms_local, dofs, device="cuda")
    line = {"metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 inner CG + f64 refinement" if prec == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": f"batch64: 64 unit-cube problems, n ~ U{{24..40}} Q2 elements per side "
                                   f"({dofs:,} unknowns in total), 2x2x2 subdomains each, own layered density "
                                   f"and own p ~ logU[2, 50], all in one CUDA graph per solve",
                       "precision": prec},
            "gpu_launches": int(launches), "schwarz_iterations_min_max": [int(iters.min()), int(iters.max())],
            "relres_max": float(rel.max()), "setup_s": round(bs.info["setup_seconds"], 2),
            "clocks": clk.summary(),
            "roofline": _roofline(bs, 2 if prec == "mixed" else 3, "CG-step SELL-32 SpMV kernel, 512 subdomains")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_sample(args, pkg, ws, rank, local, barrier):
    """Batched p evaluation (Sec. 4): 32 candidates p ~ logU[0.5, 200]
    (SplitMix64, seed 0) on layered64, every candidate its own Schwarz run to
    1e-8 (at most 400 iterations), one batched solve sharing the matrices."""
    import numpy as np
    import torch

    import gen
    prob = gen.workload(WORKLOAD)
    prec = "mixed" if args.prec == "both" else args.prec
    sol = pkg.Solver.from_problem(prob, p=P_ROBIN, inner_rtol=INNER_RTOL, mixed_inner_rtol=MIXED_INNER_RTOL,
                                  max_outer=5000, prec=prec)
    ps = gen.log_uniform_p(0, 32, 0.5, 200.0)
    max_outer = 400
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # context: one full run, every candidate to rtol or the cap
    torch.cuda.synchronize()
    ev0.record(stream)
    it_full, rel_full, best_full = sol.sample_p(ps, rtol=RTOL, max_outer=max_outer)
    ev1.record(stream)
    torch.cuda.synchronize()
    full_ms = ev0.elapsed_time(ev1)
    # timed: race mode (the batch stops when its first candidate converges)
    for _ in range(max(args.warmup, 1)):
        sol.sample_p(ps, rtol=RTOL, max_outer=max_outer, race=True)
    launches = 0
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            iters, rel, best = sol.sample_p(ps, rtol=RTOL, max_outer=max_outer, race=True)
            launches += sol.stats()["n_launches"]
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_local = ev0.elapsed_time(ev1) / args.steps
    st = sol.stats()
    # DOF/s: unknowns x candidates solved per second (a candidate that hits
    # the cap counts as evaluated; its run is part of the search)
    value, ms = aggregate_over_ranks(ms_local, prob.n_dofs * len(ps), device="cuda")
    conv = rel <= RTOL
    line = {"metric": "candidate-DOF/s of the batched p evaluation (32 candidates x unknowns / s)",
            "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner CG + f64 refinement" if prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": f"sample32: {_workload_desc(prob, 0.0)}; 32 p ~ logU[0.5, 200] (SplitMix64 "
                                   f"seed 0) in one batched solve, race mode: the batch stops when its first "
                                   f"candidate reaches {RTOL:g} (cap {max_outer} iterations)",
                       "precision": prec},
            "gpu_launches": int(launches), "best_p": float(ps[best]), "best_iterations": int(iters[best]),
            "converged": int(conv.sum()), "iterations": [int(v) for v in iters],
            "cg_steps": st["n_cg_steps"], "clocks": clk.summary(),
            "full_run": {"ms": full_ms, "best_p": float(ps[best_full]), "converged": int((rel_full <= RTOL).sum()),
                         "iterations": [int(v) for v in it_full],
                         "note": "every candidate to rtol or the cap, same batch, untimed warm-up-free single run"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_grad(args, pkg, ws, rank, local, barrier):
    """Adjoint gradient (config-4 shape): layered48 (48^3 Q2, 3x3x3), 64 x 64
    surface stations, J = 1/2 ||g_z - g_obs||^2 with g_obs from the density
    plus N(0, 20^2) per element; one forward solve, one adjoint solve and the
    element gradient per step."""
    import numpy as np
    import torch

    import gen
    prob = gen.workload("layered48")
    prec = "mixed" if args.prec == "both" else args.prec
    sol = pkg.Solver.from_problem(prob, p=P_FOR["layered48"], inner_rtol=INNER_RTOL,
                                  mixed_inner_rtol=MIXED_INNER_RTOL, max_outer=5000, prec=prec)
    st_xyz = gen.surface_stations(64)
    sol.set_stations(st_xyz)
    rng = np.random.default_rng(0)
    drho_obs = prob.drho + rng.normal(0.0, 20.0, size=prob.drho.shape)
    drho_obs_t = torch.from_numpy(drho_obs).cuda()
    drho_t = torch.from_numpy(prob.drho).cuda()
    sol.set_density_dev(drho_obs_t)
    phi_obs, _, _ = sol.solve(RTOL)
    g_obs = sol.gravity(phi_obs).clone()
    sol.set_density_dev(drho_t)
    for _ in range(max(args.warmup, 1)):
        J, dJ, _ = sol.grad(g_obs, rtol=RTOL)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            J, dJ, _ = sol.grad(g_obs, rtol=RTOL)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_local = ev0.elapsed_time(ev1) / args.steps
    value, ms = aggregate_over_ranks(ms_local, 1.0, device="cuda")
    line = {"metric": "adjoint gradients per second (forward solve + adjoint solve + dJ/d drho)",
            "value": value, "unit": "gradients/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner CG + f64 refinement" if prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": f"grad48: {_workload_desc(prob, P_FOR['layered48'], 'layered48')}; "
                                   f"64x64 stations on the top face, g_obs from drho + N(0, 20^2)",
                       "precision": prec},
            "J": float(J), "grad_norm": float(torch.linalg.norm(dJ)), "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def profile_iteration(args):
    """One Schwarz iteration of a workload (a few dozen to a few hundred
    kernel launches) after args.warm_iterations untimed ones, in the
    precision and launch mode given, between cudaProfilerStart and
    cudaProfilerStop (ncu --profile-from-start off captures just that
    iteration)."""
    import torch

    import gen
    import paper_2112_03851_gb300 as pkg
    torch.cuda.set_device(0)
    name = args.workload or WORKLOAD
    prob = gen.workload(name)
    prec = "mixed" if args.prec == "both" else args.prec
    sol = pkg.Solver.from_problem(prob, p=P_FOR.get(name, P_ROBIN), inner_rtol=INNER_RTOL, max_outer=5000, prec=prec,
                                  mixed_inner_rtol=MIXED_INNER_RTOL,
                                  use_graph=0 if args.launch == "host" else 1)
    sol.reset()
    if args.warm_iterations:
        sol.iterate(args.warm_iterations)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    hist = sol.iterate(1)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    st = sol.stats()
    print(json.dumps({"profile_iteration": name, "prec": prec, "warm_iterations": args.warm_iterations,
                      "relres": float(hist[0]), "fp32_operator": sol.info.get("fp32_operator"),
                      "fp64_start": sol.info.get("fp64_start"), **st}), flush=True)
    return 0


def profile_kernel(args):
    """The kernel osm_profile_spmv times for `--profile-kernel PREC` (2: the
    FP32 CG step, 3: the FP64 CG-step SpMV, 4: the FP64 start of a mixed
    refinement step) on a workload: 20 untimed and 5 timed launches with
    every subdomain active, between cudaProfilerStart and cudaProfilerStop."""
    import torch

    import gen
    import paper_2112_03851_gb300 as pkg
    torch.cuda.set_device(0)
    name = args.workload or WORKLOAD
    prob = gen.workload(name)
    prec = "fp64" if args.profile_kernel == 3 else "mixed"
    sol = pkg.Solver.from_problem(prob, p=P_FOR.get(name, P_ROBIN), inner_rtol=INNER_RTOL, max_outer=5000, prec=prec,
                                  mixed_inner_rtol=MIXED_INNER_RTOL)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    ms = sol.profile_spmv(1, prec=args.profile_kernel)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    i = sol.info
    print(json.dumps({"profile_kernel": args.profile_kernel, "workload": name, "ms": ms, "box_rows": i.get("box_rows"),
                      "vec_rows": i["vec_rows"], "fp32_operator": i.get("fp32_operator"),
                      "fp64_start": i.get("fp64_start")}), flush=True)
    return 0


def profile_sample(args):
    """Two Schwarz iterations of a 32-candidate batched p evaluation."""
    import torch

    import gen
    import paper_2112_03851_gb300 as pkg
    torch.cuda.set_device(0)
    prob = gen.workload(args.workload or WORKLOAD)
    prec = "fp64" if args.prec == "both" else args.prec
    sol = pkg.Solver.from_problem(prob, p=P_ROBIN, inner_rtol=INNER_RTOL, max_outer=5000, prec=prec,
                                  mixed_inner_rtol=MIXED_INNER_RTOL, use_graph=0 if args.launch == "host" else 1)
    ps = gen.log_uniform_p(0, 32, 0.5, 200.0)
    iters, rel, best = sol.sample_p(ps, rtol=RTOL, max_outer=2)
    print(json.dumps({"profile_sample": args.workload or WORKLOAD, "relres_min": float(rel.min()),
                      **sol.stats()}), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the mixed inner tolerance at its default instead of tuning it")
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip the oracle's monolithic solve (the error of each line against it)")
    ap.add_argument("--prec", choices=("both", "mixed", "fp64"), default="both")
    ap.add_argument("--workload", default=None,
                    help="another workload: layered48, regional, layered160, slab32/64/128, batch64 "
                         "(independent problems), sample32 (batched p evaluation), grad48 (adjoint gradient)")
    ap.add_argument("--launch", choices=("graph", "host"), default="graph",
                    help="host: launch the same kernels one by one (for ncu, which cannot attribute "
                         "kernels inside graphs with conditional nodes)")
    ap.add_argument("--profile-iteration", action="store_true",
                    help="set up the workload, run --warm-iterations untimed Schwarz iterations, then one inside a "
                         "cudaProfilerStart/Stop range, and exit (for ncu captures)")
    ap.add_argument("--warm-iterations", type=int, default=0)
    ap.add_argument("--profile-kernel", type=int, choices=(2, 3, 4), default=None,
                    help="set up the workload and launch the kernel osm_profile_spmv times for this prec inside a "
                         "cudaProfilerStart/Stop range (for ncu captures)")
    ap.add_argument("--profile-sample", action="store_true",
                    help="set up the workload, run two Schwarz iterations of a 32-candidate p batch and exit")
    args = ap.parse_args(argv)
    if args.profile_iteration:
        return profile_iteration(args)
    if args.profile_kernel is not None:
        return profile_kernel(args)
    if args.profile_sample:
        return profile_sample(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
