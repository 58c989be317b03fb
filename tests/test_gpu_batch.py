"""GPU parity of dst_solve_batch (many independent meshes in one call).

Small meshes (at most opts.batch_cta_max unknowns) are solved one CTA each in
a persistent kernel; larger ones by concurrent single-mesh solves on worker
streams.  Both paths run the mixed-precision refinement, so each solution is
checked against the oracle's exact discrete solution (sparse LU) at the
mixed-precision tolerance (solve to rel. residual 1e-12, rel. L2 <= 1e-8), and
the worker path is checked to be the single-mesh solve itself (bitwise).
"""
import numpy as np
import pytest

import workloads as W
from _helpers import oracle_mesh, rel_l2

pytestmark = pytest.mark.gpu
P, O, D = W.PERIODIC, W.OPEN, W.DIRICHLET


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def B():
    from paper_2103_14588_gb300 import binding
    return binding


def _x_only(w, seed):
    """Give the workload a random potential that depends on x only (the batch's requirement)."""
    rng = np.random.default_rng(seed)
    vx = rng.uniform(-1.0, 2.0, w.n_el[0])
    w.V = np.tile(vx, w.n_el[1] * w.n_el[2]) if w.d > 1 else vx
    return w


def _meshes():
    ws = [W.random_mesh(1, [40, 1, 1, 25], [P], seed=11, with_potential=False),
          _x_only(W.random_mesh(1, [20, 1, 1, 9], [D], seed=12), 1),
          _x_only(W.random_mesh(1, [33, 1, 1, 17], [D], seed=13), 2),
          W.random_mesh(2, [12, 10, 1, 14], [P, P], seed=14, with_potential=False),
          _x_only(W.random_mesh(2, [9, 7, 1, 33], [D, P], seed=15), 3),
          _x_only(W.random_mesh(2, [11, 8, 1, 9], [D, D], seed=16), 4)]
    return ws


def _lu(w):
    from oracle import operator as OOP, solvers as OS
    om = oracle_mesh(w)
    A, b = OOP.split(om, OOP.assemble(om, w.m, w.V), w.psi0)
    return OS.sparse_solve(A, b)


@pytest.mark.parametrize("cta_max", [1 << 30, 0])
def test_batch_matches_lu(torch, B, cta_max):
    """All meshes through the persistent kernel (cta_max large) or all through the
    concurrent single-mesh solves (cta_max 0)."""
    ws = _meshes()
    meshes = [B.Mesh.from_workload(w) for w in ws]
    try:
        psis = [torch.full((m.n_unknowns,), float("nan"), dtype=torch.complex128, device="cuda") for m in meshes]
        rc, sts = B.dst_solve_batch([m.handle for m in meshes],
                                    {"rtol": 1e-12, "max_iters": 100000, "batch_cta_max": cta_max}, psis)
        torch.cuda.synchronize()
        assert rc == 0
        for w, p, st in zip(ws, psis, sts):
            assert st["status"] == 0 and st["rel_resid_true"] <= 1e-12 and st["refinements"] >= 2
            assert rel_l2(p.cpu().numpy(), _lu(w)) <= 1e-8
    finally:
        for m in meshes:
            m.close()


def test_batch_mixed_paths_and_single_solves(torch, B):
    """Automatic split (the two smallest meshes go to the persistent kernel, the rest
    to worker streams): worker-path results are the single-mesh solves bit for bit,
    persistent-path results agree with them to the solve tolerance."""
    ws = _meshes()
    meshes = [B.Mesh.from_workload(w) for w in ws]
    try:
        cta_max = sorted(m.n_unknowns for m in meshes)[1]
        opts = {"rtol": 1e-11, "max_iters": 100000}
        psis = [torch.zeros(m.n_unknowns, dtype=torch.complex128, device="cuda") for m in meshes]
        rc, sts = B.dst_solve_batch([m.handle for m in meshes], dict(opts, batch_cta_max=cta_max), psis)
        assert rc == 0 and all(s["status"] == 0 for s in sts)
        for m, p in zip(meshes, psis):
            q = torch.zeros_like(p)
            st = B.dst_solve(m.handle, dict(opts, mixed_precision=1), q)
            torch.cuda.synchronize()
            assert st["status"] == 0
            if m.n_unknowns > cta_max:
                assert torch.equal(p, q)
            else:
                assert rel_l2(p.cpu().numpy(), q.cpu().numpy()) <= 1e-8
    finally:
        for m in meshes:
            m.close()


@pytest.mark.parametrize("cta_max", [1 << 30, 0])
def test_batch_iteration_cap(torch, B, cta_max):
    ws = _meshes()[:3]
    meshes = [B.Mesh.from_workload(w) for w in ws]
    try:
        psis = [torch.zeros(m.n_unknowns, dtype=torch.complex128, device="cuda") for m in meshes]
        rc, sts = B.dst_solve_batch([m.handle for m in meshes],
                                    {"rtol": 1e-14, "max_iters": 7, "batch_cta_max": cta_max}, psis)
        assert rc in (0, 1)
        for s in sts:
            assert s["status"] == 1 and 1 <= s["iters"] <= 7
    finally:
        for m in meshes:
            m.close()


def test_batch_rejects_unsupported(torch, B):
    w1 = W.random_mesh(1, [8, 1, 1, 4], [P], seed=1, with_potential=False)
    w3 = W.random_mesh(3, [4, 4, 4, 3], [P, P, P], seed=2, with_potential=False)
    wg = W.random_mesh(2, [6, 5, 1, 3], [P, P], seed=3)            # potential varies along y
    m1, m3, mg = (B.Mesh.from_workload(w) for w in (w1, w3, wg))
    try:
        def run(ms, **o):
            ps = [torch.zeros(m.n_unknowns, dtype=torch.complex128, device="cuda") for m in ms]
            return B.dst_solve_batch([m.handle for m in ms], dict({"rtol": 1e-8}, **o), ps)
        for ms, o in (([m1, m3], {}), ([mg], {}), ([m1], {"restart": 33}), ([m1], {"method": 1})):
            with pytest.raises(B.DstError) as e:
                run(ms, **o)
            assert e.value.code == B.DST_ERR_ARG
        # the same mesh twice
        p = torch.zeros(m1.n_unknowns, dtype=torch.complex128, device="cuda")
        with pytest.raises(B.DstError) as e:
            B.dst_solve_batch([m1.handle, m1.handle], {"rtol": 1e-8}, [p, p.clone()])
        assert e.value.code == B.DST_ERR_ARG
        # no initial data
        bare = B.Mesh(1, [8, 1, 1, 4], [0, 0, 0, 0], [1, 1, 1, 1], [P, P, P])
        try:
            with pytest.raises(B.DstError) as e:
                run([bare])
            assert e.value.code == B.DST_ERR_STATE
        finally:
            bare.close()
    finally:
        for m in (m1, m3, mg):
            m.close()


def test_batch_repeated_calls_identical(torch, B):
    """Three calls in a row (fresh worker threads each time, whose capture streams are
    released when they exit) give the same solutions bit for bit."""
    ws = _meshes()[3:]
    meshes = [B.Mesh.from_workload(w) for w in ws]
    try:
        runs = []
        for _ in range(3):
            psis = [torch.zeros(m.n_unknowns, dtype=torch.complex128, device="cuda") for m in meshes]
            rc, sts = B.dst_solve_batch([m.handle for m in meshes],
                                        {"rtol": 1e-11, "max_iters": 100000, "batch_cta_max": 0}, psis)
            torch.cuda.synchronize()
            assert rc == 0 and all(s["status"] == 0 for s in sts)
            runs.append(psis)
        for r in runs[1:]:
            assert all(torch.equal(a, b) for a, b in zip(r, runs[0]))
    finally:
        for m in meshes:
            m.close()
