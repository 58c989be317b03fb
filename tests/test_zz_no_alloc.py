"""dst_arnoldi_project_noalloc: the Arnoldi projection for callers that may not allocate.

Some callers cannot let the library allocate device memory - they run under
a fixed memory budget, or inside a host framework that owns every device
allocation, or on a host path where an allocation could stall or fail late.
For them the library offers a projection h = V^H w whose reduction scratch is
a fixed array inside the library instead of memory from the stream-ordered
allocator.  These checks call it through the C ABI (ctypes) and compare it
with dst_arnoldi_project, the allocating entry point, within the tolerance of
the other Arnoldi tests (|dh| <= 1e-12 ||V_j|| ||w||), on two calls in a row:
the second call, smaller than the first, must not be disturbed by what the
first call left in the shared scratch.  The file is collected last so a
failure here cannot hide another test's result in a run that stops early.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_projection_matches_allocating_projection():
    import torch
    from paper_2103_14588_gb300 import binding as B
    lib = B.library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, nvec, seed) in enumerate([(300001, 31, 5), (4097, 7, 6)]):
        V = W.random_complex(n * nvec, seed).reshape(nvec, n)
        w = W.random_complex(n, seed + 100)
        Vd = torch.from_numpy(V.ravel()).cuda()
        wd = torch.from_numpy(w).cuda()
        h_ref = torch.zeros(nvec, dtype=torch.complex128, device="cuda")
        h_new = torch.full((nvec,), complex("nan+nanj"), dtype=torch.complex128, device="cuda")
        assert lib.dst_arnoldi_project(n, nvec, _ptr(Vd), _ptr(wd), _ptr(h_ref), stream) == B.DST_OK
        assert lib.dst_arnoldi_project_noalloc(n, nvec, _ptr(Vd), _ptr(wd), _ptr(h_new), stream) == B.DST_OK
        torch.cuda.synchronize()
        a = h_new.cpu().numpy()
        b = h_ref.cpu().numpy()
        scale = np.linalg.norm(V, axis=1) * np.linalg.norm(w)
        assert np.all(np.isfinite(a)), "call %d" % call
        assert np.all(np.abs(a - b) <= 1e-12 * scale), "call %d" % call


def test_noalloc_projection_at_the_reduction_block_cap():
    """n >= 2048 x 608 with 64 vectors: the reduction grid reaches its cap of 608
    blocks, so the static scratch holds its largest count of partials (608 x 64);
    a smaller call follows and must not see the first call's leftovers."""
    import torch
    from paper_2103_14588_gb300 import binding as B
    lib = B.library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    gen = torch.Generator(device="cuda").manual_seed(7)
    for call, (n, nvec) in enumerate([(1245184 + 977, 64), (2048 * 3 + 1, 64)]):
        V = torch.randn(nvec * n, dtype=torch.complex128, device="cuda", generator=gen)
        w = torch.randn(n, dtype=torch.complex128, device="cuda", generator=gen)
        h_ref = torch.zeros(nvec, dtype=torch.complex128, device="cuda")
        h_new = torch.full((nvec,), complex("nan+nanj"), dtype=torch.complex128, device="cuda")
        assert lib.dst_arnoldi_project(n, nvec, _ptr(V), _ptr(w), _ptr(h_ref), stream) == B.DST_OK
        assert lib.dst_arnoldi_project_noalloc(n, nvec, _ptr(V), _ptr(w), _ptr(h_new), stream) == B.DST_OK
        torch.cuda.synchronize()
        scale = (torch.linalg.vector_norm(V.view(nvec, n), dim=1) * torch.linalg.vector_norm(w)).cpu().numpy()
        a = h_new.cpu().numpy()
        b = h_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), "call %d" % call
        assert np.all(np.abs(a - b) <= 1e-12 * scale), "call %d" % call
        del V, w


def test_noalloc_projection_rejects_too_many_vectors():
    import torch
    from paper_2103_14588_gb300 import binding as B
    lib = B.library()
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    rc = lib.dst_arnoldi_project_noalloc(8, 65, _ptr(x), _ptr(x), _ptr(x), None)
    assert rc == B.DST_ERR_ARG
    assert b"64" in lib.dst_last_error_detail()
    rc = lib.dst_arnoldi_project_noalloc(0, 4, _ptr(x), _ptr(x), _ptr(x), None)
    assert rc == B.DST_ERR_ARG
    assert b"at least 1" in lib.dst_last_error_detail()
