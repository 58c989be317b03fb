"""Inputs are what their docstrings claim: positive/negative-energy spinors,
unit norms, the splitmix64 reference outputs, the step potential."""
import numpy as np
import pytest

import workloads as W
from oracle import dirac


def test_splitmix64_reference_values():
    # published reference stream for seed 1234567 (splitmix64.c test vector)
    s = 1234567
    outs = []
    for _ in range(3):
        s, z = W.splitmix64(s)
        outs.append(z)
    assert outs == [6457827717110365317, 3203168211198807973, 9817491932198370423]


@pytest.mark.parametrize("d", [1, 2, 3])
def test_spinors_are_energy_eigenvectors(d):
    p = [0.7, -1.2, 0.4][:d]
    m = 1.3
    H = dirac.hamiltonian_symbol(d, p, m)
    E = np.sqrt(np.dot(p, p) + m * m)
    up, um = W.spinor_pm(d, p, m)
    assert np.allclose(H @ up, E * up) and np.allclose(H @ um, -E * um)
    assert np.isclose(np.linalg.norm(up), 1) and np.isclose(np.linalg.norm(um), 1)
    assert abs(np.vdot(up, um)) < 1e-14


def test_zb_packet_norm_and_shape():
    w = W.zb_2p1(n=32, nt=8)
    h = 16.0 / 32
    assert np.isclose(np.sum(np.abs(w.psi0) ** 2) * h * h, 1.0)
    assert w.psi0.shape == (1, 32, 32, 2)
    assert 0 <= w.extra["phi"] < 2 * np.pi


def test_klein_potential_step():
    w = W.klein_3p1(n=8, nt=4, p0=1.05)
    V = w.V.reshape(8, 8, 8)
    assert np.all(V[:, :, :4] == 0.0) and np.all(V[:, :, 4:] == 2.5)
    assert w.psi0.shape == (8, 8, 7, 4)


def test_sommerfeld_potential_and_packet():
    """The 1+1 Sommerfeld workload samples Eq. 23 at the element centroids and
    starts a positive-energy packet far from the Dirichlet walls."""
    from oracle import exact as EX, mesh as OM
    w = W.sommerfeld_1p1(n=64, nt=8, L=0.25)
    om = OM.Mesh(w.d, w.n_el, w.lo, w.hi, w.bc)
    assert np.allclose(w.V, EX.sommerfeld(om.element_centroids(0), 2.5, 0.0, 0.25), rtol=0, atol=1e-15)
    assert w.psi0.shape == (1, 1, 63, 2)
    dens = np.sum(np.abs(w.psi0) ** 2, axis=-1).ravel()
    assert dens[0] < 1e-6 * dens.max() and dens[-1] < 1e-20 * dens.max()


def test_batch_instances_draws():
    """The batched-solve instance set is a pure function of the seed, and its draws
    stay in the stated ranges (dimension, element counts, mass, momentum, barrier)."""
    a = W.batch_instances(40, 4)
    b = W.batch_instances(40, 4)
    c = W.batch_instances(40, 5)
    assert [w.name for w in a] == [w.name for w in b]
    assert any(x.name != y.name for x, y in zip(a, c))
    assert {w.d for w in a} == {1, 2}
    for w in a:
        lo, hi = (32, 256) if w.d == 1 else (16, 48)
        axes = [w.n_el[0], w.n_el[3]] + ([w.n_el[1]] if w.d == 2 else [])
        assert all(lo <= k <= hi for k in axes)
        assert 0.5 <= w.m <= 2.0 and -4.0 <= w.extra["p0"] <= 4.0 and 0.0 <= w.extra["V0"] <= 3.0
        assert w.V.shape == (w.n_el[0] * (w.n_el[1] if w.d == 2 else 1),)
        assert np.all(w.V[: w.n_el[0] // 2 - 1] == 0.0) and np.all(w.V[w.n_el[0] // 2 + 1: w.n_el[0]] == w.extra["V0"])
        dens = np.sum(np.abs(w.psi0) ** 2)
        h = np.prod([(w.hi[k] - w.lo[k]) / w.n_el[k] for k in range(w.d)])
        assert abs(dens * h - 1.0) < 1e-12


def test_every_generator_sizes_its_data():
    """Each generator's potential has one value per spatial element (x fastest) and
    its psi0 one spinor per unknown spatial node: the lengths the C library reads."""
    P, O, D = W.PERIODIC, W.OPEN, W.DIRICHLET
    ws = [W.plane_wave_1p1(n=16), W.zb_2p1(n=8, nt=4), W.klein_3p1(n=6, nt=3),
          W.sommerfeld_1p1(n=32, nt=8, L=0.25), W.random_mesh(2, [5, 4, 1, 3], [O, D], seed=1),
          W.random_mesh(3, [3, 4, 5, 2], [P, O, D], seed=2)]
    ws += W.batch_instances(count=6, seed=3, n1=(8, 16), n2=(6, 8))
    for w in ws:
        nel = [w.n_el[k] if k < w.d else 1 for k in range(3)]
        if w.V is not None:
            assert np.size(w.V) == nel[0] * nel[1] * nel[2], w.name
        nu = [1, 1, 1]
        for k in range(w.d):
            nu[k] = {P: nel[k], O: nel[k] + 1, D: nel[k] - 1}[w.bc[k]]
        assert np.size(w.psi0) == nu[0] * nu[1] * nu[2] * (2 if w.d < 3 else 4), w.name
