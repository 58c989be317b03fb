"""The C ABI library loads and exports every call include/diracst.h declares.

Runs without a GPU: no call here launches device work.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "diracst.h")).read()
    return sorted(set(re.findall(r"DST_API\s+(?:const\s+char\s*\*|int)\s*(dst_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def B():
    lib = os.path.join(ROOT, "paper_2103_14588_gb300", "lib", "libdiracst.so")
    if not os.path.exists(lib):
        import __graft_entry__
        __graft_entry__.build()
    from paper_2103_14588_gb300 import binding
    return binding


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("dst_create_mesh", "dst_destroy_mesh", "dst_set_mass", "dst_set_potential",
                 "dst_set_initial_data", "dst_build_rhs", "dst_apply_operator", "dst_solve"):
        assert must in names


def test_every_declared_symbol_is_exported(B):
    lib = ctypes.CDLL(B.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(B.EXPORTED)


def test_status_strings(B):
    assert B.dst_status_string(0) == "ok"
    assert "invalid" in B.dst_status_string(-1)
    assert B.dst_status_string(12345) == "unknown status"


def test_argument_errors_without_device(B):
    # invalid dimension / sizes are rejected before any CUDA call
    with pytest.raises(B.DstError) as e:
        B.dst_create_mesh(4, [4, 1, 1, 4], [0, 0, 0, 0], [1, 1, 1, 1], [0, 0, 0])
    assert e.value.code == B.DST_ERR_ARG
    with pytest.raises(B.DstError) as e:
        B.dst_create_mesh(1, [4, 1, 1, 0], [0, 0, 0, 0], [1, 1, 1, 1], [0, 0, 0])
    assert e.value.code == B.DST_ERR_ARG
    with pytest.raises(B.DstError) as e:
        B.dst_create_mesh(1, [1, 1, 1, 3], [0, 0, 0, 0], [1, 1, 1, 1], [B.DST_BC_DIRICHLET, 0, 0])
    assert e.value.code == B.DST_ERR_ARG
    with pytest.raises(B.DstError) as e:
        B.dst_create_mesh(2, [4, 4, 1, 3], [0, 0, 0, 0], [1, -1, 1, 1], [0, 0, 0])
    assert e.value.code == B.DST_ERR_ARG
    lib = B.library()
    assert lib.dst_solve(None, None, None, None, None) == B.DST_ERR_ARG
    assert lib.dst_apply_operator(None, 0, None, None, None) == B.DST_ERR_ARG
    assert lib.dst_arnoldi_project(0, 1, None, None, None, None) == B.DST_ERR_ARG
    assert lib.dst_destroy_mesh(None) == B.DST_OK


def test_every_call_rejects_missing_arguments_without_device(B):
    """Each entry point checks its pointers and sizes before any CUDA call."""
    import ctypes
    lib = B.library()
    ARG = B.DST_ERR_ARG
    assert lib.dst_mesh_sizes(None, None, None, None) == ARG
    assert lib.dst_set_mass(None, 1.0) == ARG
    assert lib.dst_set_potential(None, None) == ARG
    assert lib.dst_set_initial_data(None, None) == ARG
    assert lib.dst_build_rhs(None, None, None) == ARG
    assert lib.dst_arnoldi_update(0, 1, None, None, None, None, None) == ARG
    assert lib.dst_arnoldi_project_noalloc(0, 1, None, None, None, None) == ARG
    assert lib.dst_observables(None, None, 0.0, None, None) == ARG
    assert lib.dst_default_solve_opts(None) == ARG
    assert lib.dst_solve_batch(0, None, None, None, None, None) == ARG
    assert lib.dst_tune_apply(None, None) == ARG
    assert lib.dst_set_apply_variant(None, 0, 0) == ARG
    v, c = ctypes.c_int(), ctypes.c_int()
    assert lib.dst_get_apply_variant(None, 0, ctypes.byref(v), ctypes.byref(c)) == ARG


def test_mesh_wrapper_checks_potential_length(B):
    """The C library reads nel_x * nel_y * nel_z potential values; the wrapper refuses
    another length before it creates a mesh."""
    import numpy as np
    with pytest.raises(ValueError):
        B.Mesh(2, [4, 3, 1, 2], [0, 0, 0, 0], [1, 1, 1, 1], [0, 0, 0], V=np.zeros(11))
    with pytest.raises(ValueError):
        B.Mesh(1, [8, 1, 1, 2], [0, 0, 0, 0], [1, 1, 1, 1], [0, 0, 0], V=np.zeros(9))


def test_default_opts(B):
    o = B.dst_default_solve_opts()
    assert o.restart == 30 and o.rtol == 1e-8 and o.mixed_precision == 0 and o.use_initial_guess == 0
    assert o.mixed_ortho == 2 and o.method == 0 and o.inner_cycles == 1 and o.ortho == 0


def test_product_package_does_not_use_oracle():
    pkg = os.path.join(ROOT, "paper_2103_14588_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
                assert "oracle/" not in txt, f
