"""Physics pins of the oracle: what the paper and the mathematics fix.

* Plane wave (Sec. 4.1, Appendix B): second-order L2 convergence of the
  discrete solution to the exact plane wave on periodic meshes.
* Charge self-convergence (Sec. 4.1, energy-loss study; the paper reports a
  ratio 4.091): successive differences shrink by ~4 per halving of h.
* Zitterbewegung (Sec. 4.2, Eqs. 18-20, initial data Eq. 19): the discrete
  <x(t)> follows the exact spectral evolution, and oscillates at ~2E.
* Klein step (Sec. 4.3, Eqs. 23-25): Eq. 24 (as read) equals direct
  integration of the stationary equation; the discrete T from Eq. 25 matches
  the momentum-averaged step transmission.
"""
import numpy as np
import pytest

from oracle import exact as EX, mesh as M, observables as OB, operator as OP, solvers as SO


def _u_plus(k, m):
    E = np.sqrt(k * k + m * m)
    return np.array([E + m, k]) / np.sqrt(2 * E * (E + m))


def _plane_wave_error(n, k=1.0, m=1.0):
    me = M.Mesh(1, [n, 1, 1, n], [0, 0, 0, 0], [2 * np.pi, 1, 1, 1], [M.PERIODIC] * 3)
    u0 = _u_plus(k, m)
    x = me.node_coords(0)
    A, b = OP.split(me, OP.assemble(me, m, None), np.exp(1j * k * x)[:, None] * u0)
    sol = SO.sparse_solve(A, b)
    ex = EX.plane_wave(me, [k], u0, m).ravel()
    return np.linalg.norm(sol - ex) / np.linalg.norm(ex)


def test_plane_wave_exact_solves_pde():
    # exp(ikx - iEt) u_+ satisfies i d_t psi = (alpha p + beta m) psi (finite differences)
    me = M.Mesh(1, [8, 1, 1, 4], [0, 0, 0, 0], [2 * np.pi, 1, 1, 1], [0, 0, 0])
    k, m, dt = 1.0, 1.0, 1e-6
    u0 = _u_plus(k, m)
    a = EX.plane_wave(me, [k], u0, m, times=[0.3 - dt, 0.3 + dt])
    dpsi = (a[1] - a[0]) / (2 * dt)
    E = np.sqrt(k * k + m * m)
    mid = EX.plane_wave(me, [k], u0, m, times=[0.3])[0]
    assert np.allclose(1j * dpsi, E * mid, atol=1e-7)


def test_plane_wave_second_order():
    e = [_plane_wave_error(n) for n in (16, 32, 64)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 3.7 < r1 < 4.3 and 3.7 < r2 < 4.3
    assert e[2] < 1e-4


def test_charge_self_convergence():
    k, m = 1.0, 1.0
    u0 = _u_plus(k, m)
    dq = {}
    for n in (16, 32, 64, 128):
        me = M.Mesh(1, [n, 1, 1, n], [0, 0, 0, 0], [2 * np.pi, 1, 1, 1], [M.PERIODIC] * 3)
        x = me.node_coords(0)
        A, b = OP.split(me, OP.assemble(me, m, None), np.exp(1j * k * x)[:, None] * u0)
        s = SO.sparse_solve(A, b).reshape(me.unknown_shape)
        Q = np.concatenate([[2 * np.pi], OB.charge(me, s)])
        dq[n] = (Q - Q[0])[:: n // 16]
    r = np.linalg.norm(dq[32] - dq[64]) / np.linalg.norm(dq[64] - dq[128])
    assert 3.8 < r < 4.2


def test_evolve_fft_single_mode_and_norm():
    me = M.Mesh(2, [8, 6, 1, 3], [0, 0, 0, 0], [2.0, 3.0, 1, 1], [0, 0, 0])
    kx, ky, m = 2 * np.pi / 2.0, 2 * np.pi * 2 / 3.0, 0.8
    u0 = np.array([0.2 + 0.3j, 1.0])
    X, Y = me.node_coords(0), me.node_coords(1)
    psi0 = np.exp(1j * (kx * X[None, :] + ky * Y[:, None]))[None, :, :, None] * u0
    ts = [0.1, 0.7]
    a = EX.evolve_fft(psi0, 2, [2.0, 3.0], m, ts)
    b = EX.plane_wave(me, [kx, ky], u0, m, times=ts)
    assert np.allclose(a, b, atol=1e-12)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(psi0.shape) + 1j * rng.standard_normal(psi0.shape)
    c = EX.evolve_fft(r, 2, [2.0, 3.0], m, [1.3])[0]
    assert np.isclose(np.sum(np.abs(c) ** 2), np.sum(np.abs(r) ** 2))


def test_zitterbewegung():
    m = 1.0
    nx, nt, tf, half = 160, 200, 20.0, 20.0
    me = M.Mesh(1, [nx, 1, 1, nt], [-half, 0, 0, 0], [half, 1, 1, tf], [M.PERIODIC] * 3)
    x = me.node_coords(0)
    psi0 = (1 / (32 * np.pi)) ** 0.25 * np.exp(-x ** 2 / 16)[:, None] * np.array([1.0, 1.0])
    assert np.isclose(OB.charge(me, psi0[None, None, None])[0], 1.0)
    A, b = OP.split(me, OP.assemble(me, m, None), psi0)
    sol = SO.sparse_solve(A, b).reshape(me.unknown_shape)
    ts = me.time_coords()[1:]
    ex = EX.evolve_fft(psi0[None, None], 1, [2 * half], m, ts)
    x_fem = OB.mean_position(me, sol)
    x_ex = OB.mean_position(me, ex)
    assert np.abs(x_fem - x_ex).max() < 5e-3
    # dominant angular frequency of <x> minus its linear drift, from the exact
    # evolution over a long window, is 2E averaged over |phi(p)|^2 (E ~ m = 1)
    tl = np.linspace(0, 60, 1201)
    xl = OB.mean_position(me, EX.evolve_fft(psi0[None, None], 1, [2 * half], m, tl))
    res = xl - np.polyval(np.polyfit(tl, xl, 1), tl)
    om = np.linspace(1.0, 4.0, 3001)
    power = [abs(np.sum(res * np.exp(-1j * w * tl))) for w in om]
    w_peak = om[int(np.argmax(power))]
    assert abs(w_peak - EX.zb_frequency([0.0], m)) / 2.0 < 0.06
    # and the discrete solution oscillates at the same frequency
    resf = x_fem - np.polyval(np.polyfit(ts, x_fem, 1), ts)
    powf = [abs(np.sum(resf * np.exp(-1j * w * ts))) for w in om]
    assert abs(om[int(np.argmax(powf))] - w_peak) < 0.15


@pytest.mark.parametrize("p0", [0.5, 1.05, 4.0, 6.0])
@pytest.mark.parametrize("L", [1e-3, 0.3])
def test_klein_formula_matches_transfer(p0, L):
    V0, m = 2.5, 1.0
    E = np.sqrt(p0 * p0 + m * m)
    T_ode, R_ode = EX.klein_T_transfer(E, lambda x: EX.sommerfeld(x, V0, 0.0, L), V0,
                                       -40 * L - 2, 40 * L + 2, m)
    assert abs(T_ode + R_ode - 1) < 1e-8
    assert abs(EX.klein_T_formula(p0, V0, L, m) - T_ode) < 1e-7


def test_klein_matching_textbook_step():
    # textbook sharp step: T = 4 kappa / (1 + kappa)^2, kappa = (q/k)(E + m)/(E - V0 + m)
    V0, m = 2.5, 1.0
    for p0 in (0.5, 1.05, 4.0):
        E = np.sqrt(p0 * p0 + m * m)
        k = p0
        eps = E - V0
        q = np.sign(eps) * np.sqrt(eps * eps - m * m)
        kap = (q / k) * (E + m) / (eps + m)
        T, R = EX.klein_T_matching(E, V0, m)
        assert abs(T - 4 * kap / (1 + kap) ** 2) < 1e-12 and abs(T + R - 1) < 1e-12
    # no propagating transmitted wave: total reflection
    assert EX.klein_T_matching(np.sqrt(2.0 ** 2 + 1), V0, m) == (0.0, 1.0)


def test_klein_fem_transmission():
    V0, m, p0, sig = 2.5, 1.0, 1.05, 4.0
    half, nx, nt, tf, xc = 40.0, 320, 160, 40.0, -16.0
    me = M.Mesh(1, [nx, 1, 1, nt], [-half, 0, 0, 0], [half, 1, 1, tf], [M.OPEN, 0, 0])
    x = me.node_coords(0)
    psi0 = np.exp(-(x - xc) ** 2 / (4 * sig ** 2) + 1j * p0 * x)[:, None] * _u_plus(p0, m)
    Ve = np.where(me.element_centroids(0) >= 0, V0, 0.0)
    A, b = OP.split(me, OP.assemble(me, m, Ve), psi0)
    sol = SO.sparse_solve(A, b).reshape(me.unknown_shape)
    T, R = OB.transmission(me, sol[-1], 0.0)
    ps = np.linspace(p0 - 5 / (2 * sig), p0 + 5 / (2 * sig), 801)
    w = np.exp(-2 * sig ** 2 * (ps - p0) ** 2)
    Tp = np.array([EX.klein_T_matching(np.sqrt(p * p + m * m), V0, m)[0] for p in ps])
    T_avg = np.sum(w * Tp) / np.sum(w)
    assert abs(T - T_avg) < 0.015
    assert abs(T + R - 1) < 1e-12
