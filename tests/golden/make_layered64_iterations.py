"""Write layered64_iterations.json: the FP64 oracle's Schwarz iteration count
(sequential Jacobi-type Schwarz, Sec. 3) on the 64^3 layered workload with
4x4x4 subdomains, Robin p = 20, subdomain PCG 1e-10 (Sec. 6), stop at a global
relative residual of 1e-8.  Calls only the oracle and the input generators.

    python tests/golden/make_layered64_iterations.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gen  # noqa: E402
import oracle  # noqa: E402

P, INNER, RTOL = 20.0, 1e-10, 1e-8


def main():
    prob = gen.workload("layered64")
    S = oracle.Schwarz.from_problem(prob, p=P)
    t = time.time()
    _, n, rel, hist = S.solve(inner_rtol=INNER, rtol=RTOL, max_outer=2000)
    out = {"workload": "layered64", "p": P, "inner_rtol": INNER, "rtol": RTOL,
           "schwarz_iterations": int(n), "final_relres": rel,
           "residual_history_every_10": [float(x) for x in hist[::10]],
           "oracle_seconds": round(time.time() - t, 1)}
    with open(os.path.join(HERE, "layered64_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out["schwarz_iterations"], rel)


if __name__ == "__main__":
    main()
