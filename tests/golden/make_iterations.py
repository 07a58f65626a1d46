"""Write <workload>_iterations.json: the FP64 oracle's Schwarz iteration count
(sequential Jacobi-type Schwarz, Sec. 3) on a bench workload with its Robin
parameter, subdomain PCG 1e-10 (Sec. 6), stop at a global relative residual
of 1e-8.  Calls only the oracle and the input generators.

    python tests/golden/make_iterations.py layered64 20
    python tests/golden/make_iterations.py regional 1.6664
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gen  # noqa: E402
import oracle  # noqa: E402

INNER, RTOL = 1e-10, 1e-8


def main(name, p):
    prob = gen.workload(name)
    S = oracle.Schwarz.from_problem(prob, p=p)
    t = time.time()
    _, n, rel, hist = S.solve(inner_rtol=INNER, rtol=RTOL, max_outer=5000)
    out = {"workload": name, "p": p, "inner_rtol": INNER, "rtol": RTOL,
           "schwarz_iterations": int(n), "final_relres": rel,
           "residual_history_every_10": [float(x) for x in hist[::10]],
           "oracle_seconds": round(time.time() - t, 1)}
    with open(os.path.join(HERE, f"{name}_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out["schwarz_iterations"], rel)


if __name__ == "__main__":
    main(sys.argv[1], float(sys.argv[2]))
