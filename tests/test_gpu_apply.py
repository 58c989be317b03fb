"""GPU parity of the operator apply and the right-hand side against the oracle.

Tolerances.  Every output of y = A x is a short sum (at most 3^(d+1) nodes x
NC components x (d+2) spin terms, < 600 terms) of O(1)-coefficient products.
The kernel sums them in sum-factorised order, the oracle element by element,
so the two differ by rounding only: at most ~K eps sum|terms| with K ~ 50.
FP64 (eps = 1.1e-16): max |dy| <= 1e-12 max|y|, rel L2 <= 1e-13.
FP32 (eps = 6.0e-8), oracle fed the same FP32-rounded x: max |dy| <= 5e-5 max|y|,
rel L2 <= 1e-5.
"""
import numpy as np
import pytest

import workloads as W
from _helpers import max_rel, oracle_mesh, rel_l2

pytestmark = pytest.mark.gpu

P, O, D = W.PERIODIC, W.OPEN, W.DIRICHLET
TOL = {"f64": (1e-12, 1e-13), "f32": (5e-5, 1e-5)}


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def B():
    from paper_2103_14588_gb300 import binding
    return binding


def _potential(d, n_el, kind, seed):
    nel = [n_el[k] if k < d else 1 for k in range(3)]
    rng = np.random.default_rng(seed)
    if kind == "none":
        return None
    if kind == "xonly":
        vx = rng.uniform(-1, 2, nel[0])
        return np.tile(vx, nel[1] * nel[2])
    return rng.uniform(-1, 2, nel[0] * nel[1] * nel[2])


def _run_apply(torch, B, w, prec, seed):
    from oracle import operator as OOP
    om = oracle_mesh(w)
    n = om.n_unknowns
    x = W.random_complex(n, seed)
    if prec == "f32":
        x = x.astype(np.complex64).astype(np.complex128)
    with B.Mesh.from_workload(w) as mesh:
        assert mesh.n_unknowns == n
        dt = torch.complex128 if prec == "f64" else torch.complex64
        xd = torch.from_numpy(x).to(dt).cuda()
        yd = torch.full_like(xd, float("nan"))
        B.dst_apply_operator(mesh.handle, B.DST_FP64 if prec == "f64" else B.DST_FP32, xd, yd)
        torch.cuda.synchronize()
        y = yd.cpu().numpy().astype(np.complex128)
    ref = OOP.apply(om, w.m, w.V, x)
    return y, ref


CASES = [
    (1, [300, 1, 1, 70], [P]), (1, [300, 1, 1, 70], [O]), (1, [300, 1, 1, 70], [D]),
    (2, [70, 19, 1, 35], [P, P]), (2, [70, 19, 1, 35], [O, P]), (2, [70, 19, 1, 35], [D, O]),
    (3, [35, 9, 6, 17], [O, P, P]), (3, [35, 9, 6, 17], [P, D, O]),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("vkind", ["none", "xonly", "general"])
@pytest.mark.parametrize("d,n_el,bc", CASES)
def test_apply_parity(torch, B, d, n_el, bc, vkind, prec):
    if d == 1 and vkind == "general":
        pytest.skip("every 1+1 potential depends on x only")
    w = W.random_mesh(d, n_el, bc, seed=100 + d)
    w.V = _potential(d, n_el, vkind, seed=7 + d)
    y, ref = _run_apply(torch, B, w, prec, seed=3)
    assert np.all(np.isfinite(y))
    tmax, tl2 = TOL[prec]
    assert max_rel(y, ref) <= tmax
    assert rel_l2(y, ref) <= tl2


EDGE = [
    (1, [1, 1, 1, 1], [P]), (1, [2, 1, 1, 3], [P]), (1, [1, 1, 1, 2], [O]), (1, [2, 1, 1, 2], [D]),
    (2, [1, 2, 1, 1], [P, P]), (2, [3, 2, 1, 2], [D, D]), (2, [33, 9, 1, 17], [O, O]),
    (3, [1, 1, 1, 1], [P, P, P]), (3, [2, 2, 2, 2], [O, O, O]), (3, [17, 5, 5, 9], [D, P, O]),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("d,n_el,bc", EDGE)
def test_apply_edge_sizes(torch, B, d, n_el, bc, prec):
    w = W.random_mesh(d, n_el, bc, seed=5)
    y, ref = _run_apply(torch, B, w, prec, seed=9)
    tmax, tl2 = TOL[prec]
    assert max_rel(y, ref) <= tmax and rel_l2(y, ref) <= tl2


@pytest.mark.parametrize("vkind", ["none", "xonly", "general"])
@pytest.mark.parametrize("d,n_el,bc", CASES + EDGE)
def test_rhs_parity(torch, B, d, n_el, bc, vkind):
    from oracle import operator as OOP
    if d == 1 and vkind == "general":
        pytest.skip("every 1+1 potential depends on x only")
    w = W.random_mesh(d, n_el, bc, seed=40 + d)
    w.V = _potential(d, n_el, vkind, seed=3)
    om = oracle_mesh(w)
    with B.Mesh.from_workload(w) as mesh:
        b = torch.full((mesh.n_unknowns,), float("nan"), dtype=torch.complex128, device="cuda")
        B.dst_build_rhs(mesh.handle, b)
        torch.cuda.synchronize()
        got = b.cpu().numpy()
    ref = OOP.rhs(om, w.m, w.V, w.psi0)
    assert max_rel(got, ref) <= 1e-12 and rel_l2(got, ref) <= 1e-13


def _sample_nodes(om, count, seed):
    nt, nz, ny, nx = om.unknown_shape[:4]
    rng = np.random.default_rng(seed)
    t = np.concatenate([rng.integers(0, nt, count), [0, 0, nt - 1, nt - 1, nt // 2]])
    z = np.concatenate([rng.integers(0, nz, count), [0, nz - 1, 0, nz - 1, nz // 2]])
    y = np.concatenate([rng.integers(0, ny, count), [0, ny - 1, ny - 1, 0, 0]])
    x = np.concatenate([rng.integers(0, nx, count), [0, nx - 1, 0, nx - 1, nx - 1]])
    return ((t * nz + z) * ny + y) * nx + x


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("which", ["zb_2p1", "klein_3p1"])
def test_apply_full_size_sampled(torch, B, which, prec):
    """Full workload sizes, launched exactly as the bench launches them; sampled rows."""
    from oracle import operator as OOP
    w = W.zb_2p1() if which == "zb_2p1" else W.klein_3p1(p0=1.05)
    om = oracle_mesh(w)
    n = om.n_unknowns
    x = W.random_complex(n, 17)
    if prec == "f32":
        x = x.astype(np.complex64).astype(np.complex128)
    with B.Mesh.from_workload(w) as mesh:
        dt = torch.complex128 if prec == "f64" else torch.complex64
        xd = torch.from_numpy(x).to(dt).cuda()
        yd = torch.empty_like(xd)
        B.dst_apply_operator(mesh.handle, B.DST_FP64 if prec == "f64" else B.DST_FP32, xd, yd)
        torch.cuda.synchronize()
        nodes = _sample_nodes(om, 1500, seed=2)
        idx = (nodes[:, None] * om.nc + np.arange(om.nc)).ravel()
        got = yd[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
        assert bool(torch.isfinite(torch.view_as_real(yd)).all())
    ref = OOP.apply_rows(om, w.m, w.V, x, nodes).ravel()
    tmax, tl2 = TOL[prec]
    assert max_rel(got, ref) <= tmax and rel_l2(got, ref) <= tl2


def test_apply_rejects_bad_arguments(torch, B):
    w = W.random_mesh(1, [8, 1, 1, 4], [P], seed=1)
    lib = B.library()
    with B.Mesh.from_workload(w) as mesh:
        x = torch.zeros(mesh.n_unknowns, dtype=torch.complex128, device="cuda")
        y = torch.zeros_like(x)
        assert lib.dst_apply_operator(mesh.handle, 7, x.data_ptr(), y.data_ptr(), None) == B.DST_ERR_ARG
        assert lib.dst_apply_operator(mesh.handle, 0, x.data_ptr(), x.data_ptr(), None) == B.DST_ERR_ARG
        with pytest.raises(TypeError):
            B.dst_apply_operator(mesh.handle, B.DST_FP64, x.to(torch.complex64), y)


# ---- tile shapes of the autotuner ------------------------------------------------

@pytest.mark.parametrize("d,n_el,bc,pot", [(1, [300, 1, 1, 45], [O], "xonly"), (1, [64, 1, 1, 7], [P], "none"),
                                           (1, [257, 1, 1, 33], [D], "xonly"),
                                           (2, [37, 21, 1, 11], [P, D], "none"), (2, [19, 17, 1, 9], [O, P], "xonly"),
                                           (2, [40, 24, 1, 13], [D, D], "none"),
                                           (3, [10, 9, 7, 6], [P, D, P], "xonly"), (3, [9, 6, 11, 5], [D, P, P], "none"),
                                           (3, [17, 12, 9, 19], [D, P, P], "xonly"),
                                           (3, [6, 5, 4, 3], [O, P, P], "xonly")])
def test_tile_variants_bitwise_equal(torch, B, d, n_el, bc, pot):
    """Every tile shape computes each output from the same neighbours in the same
    order.  FP64 applies agree bit for bit with shape 0; FP32 ones to rounding (the
    compiler may fuse a multiply-add differently in another instantiation).  3+1
    shape 1 is the z-column kernel (meshes without open axes; with an open axis it
    falls back to shape 0)."""
    w = W.random_mesh(d, n_el, bc, seed=5, with_potential=False)
    w.V = _potential(d, n_el, pot, 6)
    with B.Mesh.from_workload(w) as mesh:
        n = mesh.n_unknowns
        for prec, dt in ((B.DST_FP64, torch.complex128), (B.DST_FP32, torch.complex64)):
            v0, count = B.dst_get_apply_variant(mesh.handle, prec)
            assert count == (2 if d == 3 else 3)
            x = torch.from_numpy(W.random_complex(n, 7)).to(dt).cuda()
            ys = []
            for v in range(count):
                B.dst_set_apply_variant(mesh.handle, prec, v)
                assert B.dst_get_apply_variant(mesh.handle, prec) == (v, count)
                y = torch.full_like(x, float("nan"))
                B.dst_apply_operator(mesh.handle, prec, x, y)
                torch.cuda.synchronize()
                ys.append(y)
            for y in ys[1:]:
                if prec == B.DST_FP64:
                    assert torch.equal(y, ys[0])
                else:
                    assert (y - ys[0]).abs().max().item() <= 1e-6 * ys[0].abs().max().item()


def test_tune_apply_and_errors(torch, B):
    w2 = W.random_mesh(2, [33, 20, 1, 12], [P, P], seed=8, with_potential=False)
    w3 = W.random_mesh(3, [5, 4, 4, 3], [P, P, P], seed=9, with_potential=False)
    with B.Mesh.from_workload(w2) as m2, B.Mesh.from_workload(w3) as m3:
        B.dst_tune_apply(m2.handle)
        for prec in (B.DST_FP64, B.DST_FP32):
            v, c = B.dst_get_apply_variant(m2.handle, prec)
            assert c == 3 and 0 <= v < 3
            v3, c3 = B.dst_get_apply_variant(m3.handle, prec)
            assert c3 == 2 and v3 in (0, 1)
        for args in ((m2.handle, 7, 0), (m2.handle, B.DST_FP32, 3), (m2.handle, B.DST_FP32, -1),
                     (m3.handle, B.DST_FP64, 2)):
            with pytest.raises(B.DstError) as e:
                B.dst_set_apply_variant(*args)
            assert e.value.code == B.DST_ERR_ARG


@pytest.mark.parametrize("d,n_el,bc,kind", [(1, [40, 1, 1, 6], [P], "xonly"), (2, [12, 10, 1, 5], [P, D], "general")])
def test_rejected_setters_keep_the_operator(torch, B, d, n_el, bc, kind):
    """A potential or a mass that the library rejects (a non-finite value) leaves
    the operator as it was, for the x-only and for the general potential kernel;
    a valid change afterwards still takes effect."""
    w = W.random_mesh(d, n_el, bc, seed=21, with_potential=False)
    w.V = _potential(d, n_el, kind, 22)
    with B.Mesh.from_workload(w) as mesh:
        x = torch.from_numpy(W.random_complex(mesh.n_unknowns, 23)).cuda()

        def apply():
            y = torch.full_like(x, float("nan"))
            B.dst_apply_operator(mesh.handle, B.DST_FP64, x, y)
            torch.cuda.synchronize()
            return y

        y0 = apply()
        bad = np.array(w.V, dtype=np.float64)
        bad[-1] = np.nan
        with pytest.raises(B.DstError) as e:
            B.dst_set_potential(mesh.handle, bad)
        assert e.value.code == B.DST_ERR_ARG
        with pytest.raises(B.DstError) as e:
            B.dst_set_mass(mesh.handle, float("inf"))
        assert e.value.code == B.DST_ERR_ARG
        assert torch.equal(apply(), y0)
        B.dst_set_mass(mesh.handle, w.m + 0.5)
        assert not torch.equal(apply(), y0)
