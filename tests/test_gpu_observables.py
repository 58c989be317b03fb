"""GPU observables (charge, share right of x0, first moments per time layer) against the oracle.

Parity: random solutions on small meshes of every dimension and boundary kind;
the sums are deterministic FP64 over at most 10^5 terms, so the relative
difference from the oracle's trapezoid sums is at rounding level (<= 1e-12).
Full size: the mixed-precision solve of the 2+1 Zitterbewegung workload, its
<x>(t), <y>(t) and charge against the exact spectral evolution of the same
initial data (oracle.exact.evolve_fft on the same periodic grid).  The gap
is the method's second-order discretisation error at h = 1/6 (measured: 1.0e-3
in <x>, 1.1e-4 in <y>, 0.2 % charge drift; the 1+1 pin of the oracle shows
2.3e-3 at h = 1/4), bounded here by 3e-3, 1e-3 and 0.5 %.
"""
import numpy as np
import pytest

import workloads as W
from _helpers import oracle_mesh

pytestmark = pytest.mark.gpu
P, O, D = W.PERIODIC, W.OPEN, W.DIRICHLET


def _gpu_obs(torch, B, w, psi_np, x0):
    with B.Mesh.from_workload(w) as mesh:
        psi = torch.from_numpy(np.ascontiguousarray(psi_np).ravel()).cuda()
        nt = w.n_el[3]
        out = torch.full((nt, 5), float("nan"), dtype=torch.float64, device="cuda")
        B.dst_observables(mesh.handle, psi, x0, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("d,n_el,bc", [(1, [37, 1, 1, 6], [O]), (2, [11, 9, 1, 5], [D, P]), (2, [8, 7, 1, 3], [P, O]),
                                       (3, [6, 5, 4, 3], [O, P, D])])
def test_observables_parity(d, n_el, bc):
    import torch
    from oracle import observables as OB
    from paper_2103_14588_gb300 import binding as B
    w = W.random_mesh(d, n_el, bc, seed=d + 30)
    om = oracle_mesh(w)
    psi = W.random_complex(om.n_unknowns, 4).reshape(om.unknown_shape)
    x0 = 0.1
    got = _gpu_obs(torch, B, w, psi, x0)
    Q = OB.charge(om, psi)
    assert np.allclose(got[:, 0], Q, rtol=1e-12, atol=0)
    T = np.array([OB.transmission(om, psi[n], x0)[0] for n in range(om.nt)])
    assert np.allclose(got[:, 1] / got[:, 0], T, rtol=1e-12, atol=1e-14)
    for k in range(d):
        assert np.allclose(got[:, 2 + k] / got[:, 0], OB.mean_position(om, psi, k), rtol=1e-11, atol=1e-13)
    for k in range(d, 3):
        assert np.all(got[:, 2 + k] == 0.0)


def test_zitterbewegung_2p1_full_size():
    import torch
    from oracle import exact as EX, observables as OB
    from paper_2103_14588_gb300 import binding as B
    w = W.zb_2p1()
    om = oracle_mesh(w)
    with B.Mesh.from_workload(w) as mesh:
        psi = torch.zeros(mesh.n_unknowns, dtype=torch.complex128, device="cuda")
        st = B.dst_solve(mesh.handle, {"restart": 30, "rtol": 1e-10, "max_iters": 20000, "mixed_precision": 1}, psi)
        assert st["status"] == 0
        out = torch.zeros((96, 5), dtype=torch.float64, device="cuda")
        B.dst_observables(mesh.handle, psi, 0.0, out)
        torch.cuda.synchronize()
        obs = out.cpu().numpy()
    ts = om.time_coords()[1:]
    ex = EX.evolve_fft(w.psi0, 2, [16.0, 16.0], w.m, ts)
    q_ex = OB.charge(om, ex)
    x_ex = OB.mean_position(om, ex, 0)
    y_ex = OB.mean_position(om, ex, 1)
    q = obs[:, 0]
    x_fem, y_fem = obs[:, 2] / q, obs[:, 3] / q
    assert np.all(np.isfinite(obs))
    assert np.abs(q / q_ex - 1).max() < 5e-3
    assert np.abs(x_fem - x_ex).max() < 3e-3
    assert np.abs(y_fem - y_ex).max() < 1e-3
    # the trembling is there: <x> rises and falls (not a monotone drift)
    assert x_ex.max() - x_ex[0] > 0.05 and np.any(np.diff(x_fem) < 0)


# ---- energy per layer (dst_energy) ------------------------------------------------
# FP64 FFTs (Stockham, O(log n) roundings per entry) against numpy's FFT in the
# oracle: relative difference at rounding level, <= 1e-11 of the largest |E|.

@pytest.mark.parametrize("d,n_el", [(1, [24, 1, 1, 5]), (1, [15, 1, 1, 3]), (2, [12, 10, 1, 4]), (2, [9, 14, 1, 3]),
                                    (3, [6, 5, 4, 3]), (3, [8, 6, 10, 2])])
def test_energy_parity(d, n_el):
    import torch
    from oracle import observables as OB
    from paper_2103_14588_gb300 import binding as B
    w = W.random_mesh(d, n_el, [P] * d, seed=d + 50, with_potential=False)
    om = oracle_mesh(w)
    rng = np.random.default_rng(d + 60)
    psi = rng.standard_normal(om.unknown_shape) + 1j * rng.standard_normal(om.unknown_shape)
    ref = OB.energy(om, psi, w.m)
    with B.Mesh.from_workload(w) as mesh:
        pd = torch.from_numpy(np.ascontiguousarray(psi).ravel()).cuda()
        out = torch.full((om.nt,), float("nan"), dtype=torch.float64, device="cuda")
        B.dst_energy(mesh.handle, pd, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-11 * np.abs(ref).max()), (got, ref)


def test_energy_of_the_plane_wave_solution():
    """The 64 x 64 plane wave u_+(k) e^{ikx}: the FEM solution's energy per layer is the
    exact E(k) x |u|^2 x length to the method's O(h^2) accuracy, and equals the oracle's."""
    import torch
    from oracle import observables as OB
    from paper_2103_14588_gb300 import binding as B
    w = W.plane_wave_1p1(n=64)
    om = oracle_mesh(w)
    with B.Mesh.from_workload(w) as mesh:
        psi = torch.zeros(mesh.n_unknowns, dtype=torch.complex128, device="cuda")
        st = B.dst_solve(mesh.handle, {"restart": 30, "rtol": 1e-12, "max_iters": 20000}, psi)
        out = torch.zeros(om.nt, dtype=torch.float64, device="cuda")
        B.dst_energy(mesh.handle, psi, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        x = psi.cpu().numpy().reshape(om.unknown_shape)
    assert st["status"] == 0
    ref = OB.energy(om, x, w.m)
    assert np.all(np.abs(got - ref) <= 1e-11 * np.abs(ref).max())
    E = np.sqrt(1.0 + 1.0)
    assert np.all(np.abs(got / (E * 2 * np.pi) - 1.0) <= 2e-3)


def test_energy_needs_periodic_axes():
    import torch
    from paper_2103_14588_gb300 import binding as B
    w = W.random_mesh(2, [6, 5, 1, 3], [P, D], seed=1)
    with B.Mesh.from_workload(w) as mesh:
        psi = torch.zeros(mesh.n_unknowns, dtype=torch.complex128, device="cuda")
        out = torch.zeros(3, dtype=torch.float64, device="cuda")
        with pytest.raises(B.DstError) as e:
            B.dst_energy(mesh.handle, psi, out)
        assert e.value.code == B.DST_ERR_ARG
