"""Store a seeded sample of the oracle's discrete solution of a full-size workload.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Writes
tests/golden/<workload>_solution_sample.json: the oracle's own restarted
GMRES(30) solution of D_w22 Psi_u = -D_w21 Psi_0 (Sec. 2.1, Eq. 11;
Algorithm 1 step 6) at a seeded set of unknown nodes, every spinor component,
plus the solution's 2-norm.  The solve runs to a relative residual of 1e-13,
so the stored values pin the discrete solution (to about cond(A) x 1e-13),
not an iterate.  The script imports nothing but the oracle and the input
generators; no stored value comes from anywhere else.

For the 3+1 Klein workload (names klein_3p1_seed<k>) the stored values come
from the exact 1+1 reduction solved by sparse LU instead (see klein_3p1_reduced).

Usage: python -m oracle.solution_sample [workload ...]   (default: zb_2p1)
"""

import json
import os
import sys
import time

import numpy as np

import workloads as W
from oracle import mesh as OM, operator as OOP, solvers as OS

GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")
RTOL, RESTART, NSAMPLE, SAMPLE_SEED = 1e-13, 30, 2048, 2103


def sample(name):
    w = getattr(W, name)()
    om = OM.Mesh(w.d, w.n_el, w.lo, w.hi, w.bc)
    b = OOP.rhs(om, w.m, w.V, w.psi0)
    t0 = time.time()
    r = OS.gmres(lambda v: OOP.apply(om, w.m, w.V, v), b, restart=RESTART, rtol=RTOL, maxiter=40000)
    nc = w.ncomp
    n_nodes = r.x.size // nc
    nodes = np.sort(np.random.default_rng(SAMPLE_SEED).choice(n_nodes, NSAMPLE, replace=False))
    vals = r.x.reshape(n_nodes, nc)[nodes]
    return {"workload": w.name, "rtol": RTOL, "restart": RESTART, "iters": r.iters,
            "converged": bool(r.converged), "rel_resid_true": r.rel_resid_true,
            "oracle_seconds": time.time() - t0, "ncomp": nc, "n_unknown_nodes": int(n_nodes),
            "norm": float(np.linalg.norm(r.x)), "nodes": [int(k) for k in nodes],
            "re": [[float(v.real) for v in row] for row in vals],
            "im": [[float(v.imag) for v in row] for row in vals]}


def klein_3p1_reduced(seed):
    """The 3+1 Klein workload of the given seed through its exact 1+1 reduction.

    Its packet and step potential depend on x only and y, z are periodic, so the
    component pairs (psi_1, psi_4) and (psi_2, psi_3) of the 3+1 solution each
    solve the 1+1 system on the x-t mesh (the cross-dimension reduction pinned in
    tests/test_oracle_operator.py).  Stored: the exact discrete solution (sparse
    LU) at a seeded sample of 3+1 unknown nodes, its 3+1 norm, and the oracle's
    GMRES(30) step count to 1e-8 on the stacked pair system, which equals the
    count on the 3+1 system (same Krylov spaces, inner products scaled by the
    number of y-z columns)."""
    w = W.klein_3p1(seed=seed)
    n, nt = w.n_el[0], w.n_el[3]
    m1 = OM.Mesh(1, [n, 1, 1, nt], [w.lo[0], 0, 0, w.lo[3]], [w.hi[0], 1, 1, w.hi[3]], [W.DIRICHLET, 0, 0])
    Vx = w.V.reshape(w.n_el[2], w.n_el[1], n)[0, 0, :]
    pz = w.psi0[0, 0]                                   # (n - 1, 4), the same on every (z, y)
    Dw = OOP.assemble(m1, w.m, Vx)
    A, b14 = OOP.split(m1, Dw, pz[:, [0, 3]])
    _, b23 = OOP.split(m1, Dw, pz[:, [1, 2]])
    s14 = OS.sparse_solve(A, b14).reshape(nt, n - 1, 2)
    s23 = OS.sparse_solve(A, b23).reshape(nt, n - 1, 2)
    ref = np.zeros((nt, n - 1, 4), dtype=np.complex128)
    ref[..., 0], ref[..., 3] = s14[..., 0], s14[..., 1]
    ref[..., 1], ref[..., 2] = s23[..., 0], s23[..., 1]
    ny, nz = w.n_el[1], w.n_el[2]
    n_nodes = nt * nz * ny * (n - 1)
    nodes = np.sort(np.random.default_rng(SAMPLE_SEED).choice(n_nodes, NSAMPLE, replace=False))
    it, ix = nodes // (nz * ny * (n - 1)), nodes % (n - 1)
    vals = ref[it, ix]
    half = b14.size
    stacked = lambda v: np.concatenate([A @ v[:half], A @ v[half:]])   # noqa: E731
    t0 = time.time()
    r = OS.gmres(stacked, np.concatenate([b14, b23]), restart=RESTART, rtol=1e-8, maxiter=40000)
    return {"workload": w.name, "seed": seed, "p0": w.extra["p0"], "solver": "sparse LU of the 1+1 reduction",
            "gmres30_iters_rtol_1e-8": r.iters, "gmres30_converged": bool(r.converged),
            "gmres30_seconds": time.time() - t0, "ncomp": 4, "n_unknown_nodes": int(n_nodes),
            "norm": float(np.sqrt(ny * nz) * np.linalg.norm(ref)), "nodes": [int(k) for k in nodes],
            "re": [[float(v.real) for v in row] for row in vals],
            "im": [[float(v.imag) for v in row] for row in vals]}


def main(names):
    for n in names:
        if n.startswith("klein_3p1_seed"):
            data = klein_3p1_reduced(int(n[len("klein_3p1_seed"):]))
            out = os.path.join(GOLDEN, "%s_solution_sample.json" % n)
            with open(out, "w") as f:
                json.dump(data, f, separators=(",", ":"))
            print(n, {k: data[k] for k in ("gmres30_iters_rtol_1e-8", "norm", "p0")}, flush=True)
            continue
        data = sample(n)
        out = os.path.join(GOLDEN, "%s_solution_sample.json" % n)
        with open(out, "w") as f:
            json.dump(data, f, separators=(",", ":"))
        print(n, {k: data[k] for k in ("iters", "rel_resid_true", "oracle_seconds", "norm")}, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["zb_2p1"])
