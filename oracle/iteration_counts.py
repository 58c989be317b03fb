"""Record how many GMRES(30) steps the oracle needs on the benchmark workloads.

Writes tests/golden/oracle_iteration_counts.json.  The benchmark's CPU arm
times a bounded sample of oracle GMRES steps and scales it by this count to a
whole solve; the count comes from the oracle alone (this script imports
nothing but the oracle and the input generators).

Usage: python -m oracle.iteration_counts [workload ...]   (default: zb_2p1)
"""

import json
import os
import sys
import time

import workloads as W
from oracle import mesh as OM, operator as OOP, solvers as OS

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                   "oracle_iteration_counts.json")
RTOL, RESTART = 1e-8, 30


def count(name):
    w = getattr(W, name)()
    om = OM.Mesh(w.d, w.n_el, w.lo, w.hi, w.bc)
    b = OOP.rhs(om, w.m, w.V, w.psi0)
    t0 = time.time()
    r = OS.gmres(lambda v: OOP.apply(om, w.m, w.V, v), b, restart=RESTART, rtol=RTOL, maxiter=20000)
    return {"workload": w.name, "iters": r.iters, "restarts": r.restarts, "converged": bool(r.converged),
            "rel_resid_true": r.rel_resid_true, "rtol": RTOL, "restart": RESTART,
            "oracle_seconds": time.time() - t0}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for n in names:
        data[n] = count(n)
        print(n, data[n], flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["zb_2p1"])
