"""GPU parity of the Arnoldi kernels (projection h = V^H w, update w -= V h).

FP64 sums of n products: error <= n eps sum|terms| in the worst case; with
the deterministic blocked order the observed error is ~sqrt(n) eps.  Bound
used: |dh| <= 1e-12 * ||V_j|| ||w||, elementwise |dw| <= 1e-13 max|w|.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def B():
    from paper_2103_14588_gb300 import binding
    return binding


@pytest.mark.parametrize("n,nvec", [(1, 1), (7, 3), (1023, 8), (1025, 9), (300001, 31), (2_000_003, 64)])
def test_project_and_update(torch, B, n, nvec):
    V = W.random_complex(n * nvec, 1).reshape(nvec, n)
    w = W.random_complex(n, 2)
    Vd = torch.from_numpy(V.ravel()).cuda()
    wd = torch.from_numpy(w).cuda()
    hd = torch.zeros(nvec, dtype=torch.complex128, device="cuda")
    B.dst_arnoldi_project(n, nvec, Vd, wd, hd)
    h = hd.cpu().numpy()
    ref = V.conj() @ w
    scale = np.linalg.norm(V, axis=1) * np.linalg.norm(w)
    assert np.all(np.abs(h - ref) <= 1e-12 * scale)
    # deterministic: a second call gives bit-identical results
    hd2 = torch.zeros_like(hd)
    B.dst_arnoldi_project(n, nvec, Vd, wd, hd2)
    assert torch.equal(hd, hd2)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.dst_arnoldi_update(n, nvec, Vd, hd, wd, nrm)
    wn = wd.cpu().numpy()
    wref = w - V.T @ h
    assert np.abs(wn - wref).max() <= 1e-13 * max(np.abs(w).max(), np.abs(V.T @ h).max())
    assert abs(nrm.item() - np.vdot(wref, wref).real) <= 1e-12 * np.vdot(wref, wref).real


def test_project_rejects_too_many_vectors(torch, B):
    lib = B.library()
    x = torch.zeros(4, dtype=torch.complex128, device="cuda")
    assert lib.dst_arnoldi_project(4, 65, x.data_ptr(), x.data_ptr(), x.data_ptr(), None) == B.DST_ERR_ARG
    assert lib.dst_arnoldi_project(0, 1, x.data_ptr(), x.data_ptr(), x.data_ptr(), None) == B.DST_ERR_ARG
