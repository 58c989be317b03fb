"""GPU parity of dst_set_boundary_data: prescribed (nonzero) Dirichlet wall values.

Sec. 2.1, Eq. 2 prescribes Psi on the boundary, and the split of Eq. 11 moves
known spinors to the right-hand side.  Two checks against the oracle
(operator.split with boundary=..., pinned on the CPU):

* the right-hand side b = -D_w21 Psi_known with wall values on every layer,
  element by element (FP64, same tolerance as the plain right-hand side);
* the oracle's own pin on the GPU: wall values and initial layer taken from an
  open-axis solution on the same mesh make the Dirichlet solve return that
  solution at every interior node (FP64 solve to rtol 1e-13, rel. L2 <= 1e-10).
"""
import numpy as np
import pytest

import workloads as W
from _helpers import max_rel, rel_l2

pytestmark = pytest.mark.gpu
P, O, D = W.PERIODIC, W.OPEN, W.DIRICHLET

CASES = [
    (1, [14, 1, 1, 5], [D]),
    (2, [10, 4, 1, 5], [D, P]),
    (2, [9, 7, 1, 4], [D, D]),
    (3, [6, 4, 5, 3], [D, P, D]),
]


def _mesh(d, n_el, bc):
    from oracle import mesh as OM
    lo, hi = [-1.0, 0.0, -0.5, 0.0], [1.5, 1.0, 0.75, 0.8]
    return OM.Mesh(d, n_el, lo, hi, bc), lo, hi


@pytest.mark.parametrize("d,n_el,bc", CASES)
def test_rhs_with_wall_values(d, n_el, bc):
    import torch
    from oracle import operator as OOP
    from paper_2103_14588_gb300 import binding as B
    om, lo, hi = _mesh(d, n_el, bc)
    rng = np.random.default_rng(70 + d)
    V = rng.uniform(-0.5, 1.0, om.nel[0] * om.nel[1] * om.nel[2])
    psi0 = rng.standard_normal(om.spatial_shape) + 1j * rng.standard_normal(om.spatial_shape)
    walls = rng.standard_normal(om.geo_shape) + 1j * rng.standard_normal(om.geo_shape)
    _, ref = OOP.split(om, OOP.assemble(om, 0.8, V), psi0, boundary=walls)
    with B.Mesh(d, n_el, lo, hi, bc, m=0.8, V=V, psi0=psi0) as mesh:
        assert mesh.wall_grid_shape() == om.geo_shape
        mesh.set_boundary_data(walls)
        b = torch.full((mesh.n_unknowns,), float("nan"), dtype=torch.complex128, device="cuda")
        B.dst_build_rhs(mesh.handle, b)
        torch.cuda.synchronize()
        got = b.cpu().numpy()
        # cleared again: the homogeneous right-hand side
        mesh.set_boundary_data(None)
        B.dst_build_rhs(mesh.handle, b)
        torch.cuda.synchronize()
        got0 = b.cpu().numpy()
    assert max_rel(got, ref) <= 1e-12 and rel_l2(got, ref) <= 1e-13
    _, ref0 = OOP.split(om, OOP.assemble(om, 0.8, V), psi0)
    assert max_rel(got0, ref0) <= 1e-12


@pytest.mark.parametrize("d,nel", [(1, (14, 1, 1)), (2, (10, 4, 1))])
def test_wall_values_from_an_open_solution(d, nel):
    """The oracle pin of tests/test_oracle_operator.py, solved on the GPU."""
    import torch
    from oracle import mesh as OM, operator as OOP, solvers as OS
    from paper_2103_14588_gb300 import binding as B
    nt = 5
    rng = np.random.default_rng(40 + d)
    lo, hi = [-1.0, 0.0, 0.0, 0.0], [1.5, 1.0, 1.0, 0.8]
    rest = [P] if d == 2 else []
    mo = OM.Mesh(d, list(nel) + [nt], lo, hi, [O] + rest)
    md = OM.Mesh(d, list(nel) + [nt], lo, hi, [D] + rest)
    V = rng.uniform(-0.5, 1.0, nel[0] * nel[1] * nel[2])
    psi0_open = rng.standard_normal(mo.spatial_shape) + 1j * rng.standard_normal(mo.spatial_shape)
    Ao, bo = OOP.split(mo, OOP.assemble(mo, 0.8, V), psi0_open)
    xo = OS.dense_solve(Ao, bo)
    go = mo.to_geo(xo)
    go[0] = mo.layer_to_geo(psi0_open)
    inner = tuple(slice(md.u0[k], md.u0[k] + md.nu[k]) for k in (2, 1, 0))
    psi0_d = go[0][inner]
    want = md.from_geo(go).ravel()
    with B.Mesh(d, list(nel) + [nt], lo, hi, [D] + rest, m=0.8, V=V, psi0=psi0_d) as mesh:
        mesh.set_boundary_data(go)
        psi = torch.zeros(mesh.n_unknowns, dtype=torch.complex128, device="cuda")
        st = B.dst_solve(mesh.handle, {"restart": 30, "rtol": 1e-13, "max_iters": 20000}, psi)
        torch.cuda.synchronize()
        got = psi.cpu().numpy()
    assert st["status"] == 0, st
    assert rel_l2(got, want) <= 1e-10


def test_boundary_data_needs_a_dirichlet_axis():
    from paper_2103_14588_gb300 import binding as B
    with B.Mesh(2, [4, 4, 1, 3], [0, 0, 0, 0], [1, 1, 1, 1], [P, O]) as mesh:
        with pytest.raises(B.DstError) as e:
            mesh.set_boundary_data(np.zeros(mesh.wall_grid_shape(), dtype=complex))
        assert e.value.code == B.DST_ERR_ARG
        assert "Dirichlet" in str(e.value)
