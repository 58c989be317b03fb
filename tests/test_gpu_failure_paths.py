"""Failure paths of dst_solve, reached on a healthy GPU through the testing hooks.

Nothing here faults, traps or hangs the GPU:

* A bulk-copy wait of the projection that gives up.  With the wait limit set
  to 0 tries every wait of the bulk-copy fed projection gives up at once; the
  kernel stops consuming, waits with the standard limit for the copies it has
  in flight, and flags the step.  The solve must return DST_ERR_CUDA naming
  the wait, and the same mesh must solve normally once the limit is restored.
  The bulk-copy fed kernels serve mixed solves on an FP32-stored basis from
  1,000,000 unknowns: the 3+1 Klein workload at 32^3 x 32 (4,063,232) is the case.
* A workspace allocation that fails: DST_ERR_OOM, then a normal solve.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_bulk_copy_wait_timeout_reports_cuda_error():
    import torch
    from paper_2103_14588_gb300 import binding as B
    w = W.klein_3p1(n=32, nt=32, p0=1.05)
    with B.Mesh.from_workload(w) as mesh:
        assert mesh.n_unknowns >= 1000000
        psi = torch.zeros(mesh.n_unknowns, dtype=torch.complex128, device="cuda")
        opts = {"restart": 30, "rtol": 1e-8, "max_iters": 30, "mixed_precision": 1}
        B.dst_testing_set(B.DST_TEST_WAIT_LIMIT, 0)
        try:
            with pytest.raises(B.DstError) as e:
                B.dst_solve(mesh.handle, opts, psi)
        finally:
            B.dst_testing_set(B.DST_TEST_WAIT_LIMIT, -1)
        assert e.value.code == B.DST_ERR_CUDA
        assert "bulk-copy wait" in str(e.value)
        torch.cuda.synchronize()
        st = B.dst_solve(mesh.handle, opts, psi)
        torch.cuda.synchronize()
        assert st["status"] in (B.DST_OK, B.DST_NOT_CONVERGED) and st["iters"] == 30
        assert np.isfinite(st["rel_resid_true"]) and st["rel_resid_true"] < 1.0


def test_workspace_allocation_failure_leaves_mesh_usable():
    import torch
    from paper_2103_14588_gb300 import binding as B
    w = W.random_mesh(2, [8, 6, 1, 5], [W.PERIODIC, W.DIRICHLET], seed=3)
    with B.Mesh.from_workload(w) as mesh:
        psi = torch.zeros(mesh.n_unknowns, dtype=torch.complex128, device="cuda")
        B.dst_testing_set(B.DST_TEST_FAIL_ALLOC, 1)
        try:
            with pytest.raises(B.DstError) as e:
                B.dst_solve(mesh.handle, {"rtol": 1e-10}, psi)
        finally:
            B.dst_testing_set(B.DST_TEST_FAIL_ALLOC, 0)
        assert e.value.code == B.DST_ERR_OOM
        st = B.dst_solve(mesh.handle, {"rtol": 1e-10, "max_iters": 5000}, psi)
        torch.cuda.synchronize()
        assert st["status"] == B.DST_OK and st["rel_resid_true"] <= 1e-10


def test_testing_hooks_reject_bad_values():
    from paper_2103_14588_gb300 import binding as B
    for hook, value in ((B.DST_TEST_WAIT_LIMIT, -2), (B.DST_TEST_FAIL_ALLOC, -1), (99, 0)):
        with pytest.raises(B.DstError) as e:
            B.dst_testing_set(hook, value)
        assert e.value.code == B.DST_ERR_ARG
