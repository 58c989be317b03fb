"""Accuracy of the Gram-Schmidt kernels of the mixed solve on an FP32-stored basis.

The mixed-precision GMRES stores its Krylov basis in FP32 and computes the
projection h = V^H w and the update w - V h with exact FP32 products and
anchored compensated sums (FP64 across warps and CTAs).  The anchor of each
partial sum is a power of two above four times a bound the thread knows in
advance (sum |w| over its entries, as |v| <= 1), so the error scales with
||v_j|| ||w||: measured about 2^-40 of it for unit basis vectors (far below
FP32's 2^-24 per term, short of FP64).  Checked here at 2^-36 ||v_j|| ||w||
(a regression that lost ten bits fails) against an FP64 evaluation of the same
stored values (each product of two FP32 numbers is exact in FP64; the FP64 sums
err by ~n 2^-53 of sum |v| |w|, far below the bound), for the register-fed and
the bulk-copy fed projection, at sizes on both sides of the 1,000,000-entry
switch between them in the solver (each kernel is called directly at every size).  The update: the result is w - V h
rounded to FP32 once, so it is checked at half an FP32 ulp of the exact value
plus 2^-36 of the anchor scale (max |w component| + sum_j |h_j|_1).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("n,nvec", [(1769472, 21), (4063232, 9), (6 * 2048 + 2, 3)])
@pytest.mark.parametrize("mode", [0, 1])
def test_projection_error_bound(n, nvec, mode):
    import torch
    from paper_2103_14588_gb300 import binding as B
    lib = B.library()
    gen = torch.Generator(device="cuda").manual_seed(n + nvec + mode)
    V = torch.randn(nvec, n, dtype=torch.complex128, device="cuda", generator=gen)
    V = (V / torch.linalg.vector_norm(V, dim=1, keepdim=True)).to(torch.complex64).contiguous()
    w = (torch.randn(n, dtype=torch.complex128, device="cuda", generator=gen) * 3.0).to(torch.complex64)
    h = torch.full((nvec,), complex("nan+nanj"), dtype=torch.complex128, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.dst_testing_fp32_arnoldi(mode, n, nvec, _ptr(V), _ptr(w), _ptr(h), None, st) == 0
    V64, w64 = V.to(torch.complex128), w.to(torch.complex128)
    ref = (V64.conj() * w64).sum(dim=1)
    scale = torch.linalg.vector_norm(V64, dim=1) * torch.linalg.vector_norm(w64)
    torch.cuda.synchronize()
    err = (h - ref).abs()
    assert torch.all(torch.isfinite(h.real)) and torch.all(torch.isfinite(h.imag))
    print("max |dh| / (||v|| ||w||) = 2^%.1f" % float(torch.log2((err / scale).max())))
    assert torch.all(err <= 2.0 ** -36 * scale), (err / scale).max().item()


@pytest.mark.parametrize("n,nvec", [(1769472, 21), (4063232, 9)])
def test_update_error_bound(n, nvec):
    import torch
    from paper_2103_14588_gb300 import binding as B
    lib = B.library()
    gen = torch.Generator(device="cuda").manual_seed(n + 3 * nvec)
    V = torch.randn(nvec, n, dtype=torch.complex128, device="cuda", generator=gen)
    V = (V / torch.linalg.vector_norm(V, dim=1, keepdim=True)).to(torch.complex64).contiguous()
    w = torch.randn(n, dtype=torch.complex128, device="cuda", generator=gen).to(torch.complex64)
    h = torch.randn(nvec, dtype=torch.complex128, device="cuda", generator=gen) * 1e-3 * np.sqrt(n)
    V64, w64 = V.to(torch.complex128), w.to(torch.complex128)
    exact = w64 - (h[:, None] * V64).sum(dim=0)
    wmax = torch.maximum(w64.real.abs(), w64.imag.abs())
    bound = wmax + (h.real.abs() + h.imag.abs()).sum()
    nrm2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.dst_testing_fp32_arnoldi(2, n, nvec, _ptr(V), _ptr(w), _ptr(h), _ptr(nrm2), st) == 0
    torch.cuda.synchronize()
    got = w.to(torch.complex128)
    half_ulp = 2.0 ** -24 * torch.maximum(exact.real.abs(), exact.imag.abs())
    assert torch.all((got - exact).abs() <= 1.5 * half_ulp + 2.0 ** -36 * bound)
    stored = float((got.abs() ** 2).sum())
    assert abs(float(nrm2[0]) - stored) <= 1e-10 * stored


@pytest.mark.parametrize("n,nvec", [(4063232, 9), (6 * 2048 + 2, 3), (4063232, 30)])
def test_bulk_copy_update_equals_register_update(n, nvec):
    """The update fed by bulk copies (mode 3, the solver's from 1M unknowns) does the
    register-fed update's arithmetic per entry: the same stored w bit for bit, and
    the same ||w||^2 up to the order of the FP64 partial sums."""
    import torch
    from paper_2103_14588_gb300 import binding as B
    lib = B.library()
    gen = torch.Generator(device="cuda").manual_seed(5 * n + nvec)
    V = torch.randn(nvec, n, dtype=torch.complex128, device="cuda", generator=gen)
    V = (V / torch.linalg.vector_norm(V, dim=1, keepdim=True)).to(torch.complex64).contiguous()
    w = torch.randn(n, dtype=torch.complex128, device="cuda", generator=gen).to(torch.complex64)
    h = torch.randn(nvec, dtype=torch.complex128, device="cuda", generator=gen) * 1e-3 * np.sqrt(n)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    w_reg, w_tma = w.clone(), w.clone()
    n_reg = torch.zeros(1, dtype=torch.float64, device="cuda")
    n_tma = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert lib.dst_testing_fp32_arnoldi(2, n, nvec, _ptr(V), _ptr(w_reg), _ptr(h), _ptr(n_reg), st) == 0
    assert lib.dst_testing_fp32_arnoldi(3, n, nvec, _ptr(V), _ptr(w_tma), _ptr(h), _ptr(n_tma), st) == 0
    torch.cuda.synchronize()
    assert torch.equal(w_tma, w_reg)
    assert abs(float(n_tma[0]) - float(n_reg[0])) <= 1e-13 * float(n_reg[0])


@pytest.mark.parametrize("n,nvec", [(4063232, 30), (6 * 2048 + 2, 3), (1769472, 17)])
def test_bulk_copy_combine_equals_register_combine(n, nvec):
    """x += V y at the end of a cycle, fed by bulk copies (mode 5, the solver's from 1M
    unknowns) against the register-fed combine (mode 4): the same FP64 x bit for bit."""
    import torch
    from paper_2103_14588_gb300 import binding as B
    lib = B.library()
    gen = torch.Generator(device="cuda").manual_seed(11 * n + nvec)
    V = torch.randn(nvec, n, dtype=torch.complex128, device="cuda", generator=gen)
    V = (V / torch.linalg.vector_norm(V, dim=1, keepdim=True)).to(torch.complex64).contiguous()
    x = torch.randn(n, dtype=torch.complex128, device="cuda", generator=gen)
    y = torch.randn(nvec, dtype=torch.complex128, device="cuda", generator=gen)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x_reg, x_tma = x.clone(), x.clone()
    assert lib.dst_testing_fp32_arnoldi(4, n, nvec, _ptr(V), _ptr(x_reg), _ptr(y), None, st) == 0
    assert lib.dst_testing_fp32_arnoldi(5, n, nvec, _ptr(V), _ptr(x_tma), _ptr(y), None, st) == 0
    torch.cuda.synchronize()
    assert torch.equal(x_tma, x_reg)
    ref = x + (y[:, None] * V.to(torch.complex128)).sum(dim=0)
    assert (x_reg - ref).abs().max().item() <= 1e-12 * ref.abs().max().item()
