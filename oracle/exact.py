"""Continuum solutions and closed forms the discrete method is checked against.

* ``plane_wave``: Psi(x, t) = exp(i k.x) exp(-i H(k) t) u_0, the exact free
  solution for plane-wave data (the plane-wave construction of Appendix B).
* ``evolve_fft``: exact free evolution of periodic data by Fourier transform,
  Psi(p, t) = exp(-i H(p) t) Psi(p, 0) (Appendix B's route: transform, assign
  the +/-E time dependence of the two energy projections, transform back).
  exp(-i H t) = cos(E t) I - i sin(E t) H / E because H(p)^2 = E^2 I.
* Klein step (Sec. 4.3): ``klein_T_matching`` solves the stationary 1+1
  equation across a sharp step by continuity of Psi and takes the ratio of
  probability currents (the textbook definition); ``klein_T_transfer``
  integrates the stationary equation through any V(x) (e.g. the Sommerfeld
  profile of Eq. 23) and takes the same current ratio; ``klein_T_formula`` is
  Eq. 24 as read here (see its docstring).
* ``zb_frequency``: the Zitterbewegung angular frequency 2E of the
  oscillating term of Eq. 18.

Pinned by tests/test_oracle_physics.py: the plane wave satisfies the PDE;
evolve_fft agrees with plane_wave on single modes and conserves the norm;
matching agrees with the transfer integration for a steep step and with the
textbook step formula; Eq. 24 (as read) agrees with the transfer integration.
"""

import numpy as np
from scipy.integrate import solve_ivp

from .dirac import hamiltonian_symbol, ncomp, SIGMA_X, SIGMA_Z


def _expmH(d, p, m, t):
    H = hamiltonian_symbol(d, p, m)
    E = np.sqrt(sum(pk * pk for pk in p) + m * m)
    return np.cos(E * t) * np.eye(ncomp(d)) - 1j * np.sin(E * t) * H / E


def plane_wave(mesh, k, u0, m, times=None):
    """Exact plane wave on the unknown nodes of ``mesh``: shape (len(times), nz, ny, nx, NC).

    k: momentum per spatial axis; u0: spinor at t = 0; m: mass.  times defaults
    to the unknown layers t_1..t_N.
    """
    d = mesh.d
    k = list(k) + [0.0] * (3 - len(k))
    if times is None:
        times = mesh.time_coords()[1:]
    X = mesh.node_coords(0)
    Y = mesh.node_coords(1) if d >= 2 else np.zeros(1)
    Z = mesh.node_coords(2) if d >= 3 else np.zeros(1)
    phase = np.exp(1j * (k[0] * X[None, None, :] + k[1] * Y[None, :, None] + k[2] * Z[:, None, None]))
    out = np.zeros((len(times),) + mesh.spatial_shape, dtype=np.complex128)
    for n, t in enumerate(times):
        u = _expmH(d, k[:d], m, t) @ np.asarray(u0, dtype=np.complex128)
        out[n] = phase[..., None] * u
    return out


def evolve_fft(psi0, d, lengths, m, times):
    """Exact free evolution of periodic samples psi0[z, y, x, c] (the mesh layout).

    d: spatial dimension; lengths: periodic box lengths (L_x, L_y, L_z) of the
    first d axes (unused axes have length-1 array axes).  Returns
    (len(times), nz, ny, nx, NC).
    """
    from .dirac import alphas_beta
    psi0 = np.asarray(psi0, dtype=np.complex128)
    shape = psi0.shape[:3]                              # (nz, ny, nx)
    p = []
    for k in range(d):
        n = shape[2 - k]
        pk = 2 * np.pi * np.fft.fftfreq(n, d=lengths[k] / n)
        sh = [1, 1, 1]
        sh[2 - k] = n
        p.append(pk.reshape(sh))
    E = np.sqrt(sum(pk ** 2 for pk in p) + m * m) * np.ones(shape)
    F = np.fft.fftn(psi0, axes=(0, 1, 2))
    al, be = alphas_beta(d)
    HF = np.einsum("ab,zyxb->zyxa", be * m, F)
    for k in range(d):
        HF = HF + p[k][..., None] * np.einsum("ab,zyxb->zyxa", al[k], F)
    out = np.zeros((len(times),) + psi0.shape, dtype=np.complex128)
    for n, t in enumerate(times):
        G = np.cos(E * t)[..., None] * F - 1j * (np.sin(E * t) / E)[..., None] * HF
        out[n] = np.fft.ifftn(G, axes=(0, 1, 2))
    return out


# ---------------------------------------------------------------- Klein step

def _current(u):
    """Probability current psi^dagger alpha psi of a 1+1 spinor (alpha = sigma_x)."""
    return float(np.real(np.conj(u) @ (SIGMA_X @ u)))


def _spinor_1p1(eps, q, m):
    """Eigenvector of sigma_x q + sigma_z m with eigenvalue eps (unnormalised)."""
    if abs(eps + m) > 1e-12:
        return np.array([eps + m, q], dtype=np.complex128)
    return np.array([q, eps - m], dtype=np.complex128)


def _transmitted_momentum(eps, m):
    """Momentum of the right-moving (group velocity q/eps > 0) or decaying wave at energy eps."""
    if eps * eps > m * m:
        return np.sign(eps) * np.sqrt(eps * eps - m * m) + 0j
    return 1j * np.sqrt(m * m - eps * eps)


def klein_T_matching(E, V0, m=1.0):
    """Transmission through the sharp step V = 0 (x < 0), V0 (x > 0) in 1+1."""
    k = np.sqrt(E * E - m * m)
    u_in = _spinor_1p1(E, k, m)
    u_rf = _spinor_1p1(E, -k, m)
    q = _transmitted_momentum(E - V0, m)
    u_tr = _spinor_1p1(E - V0, q, m)
    # u_in + r u_rf = t u_tr
    M = np.stack([u_rf, -u_tr], axis=1)
    r, t = np.linalg.solve(M, -u_in)
    if abs(q.imag) > 0:
        return 0.0, 1.0
    T = abs(t) ** 2 * _current(u_tr) / _current(u_in)
    R = -abs(r) ** 2 * _current(u_rf) / _current(u_in)
    return T, R


def klein_T_transfer(E, Vfun, V0, x_left, x_right, m=1.0):
    """Transmission through V(x) by integrating E psi = (-i sigma_x d_x + sigma_z m + V) psi.

    Starts at x_right with the pure right-moving wave of energy E - V0, integrates
    psi' = i sigma_x (E - V - sigma_z m) psi to x_left (V ~ 0 there), splits
    into incident + reflected waves and returns (T, R) as current ratios.
    """
    q = _transmitted_momentum(E - V0, m)
    if abs(q.imag) > 0:
        return 0.0, 1.0
    u_tr = _spinor_1p1(E - V0, q, m)

    def rhs(x, y):
        A = 1j * SIGMA_X @ ((E - Vfun(x)) * np.eye(2) - SIGMA_Z * m)
        return A @ y

    psi_r = u_tr * np.exp(1j * q * x_right)
    sol = solve_ivp(rhs, (x_right, x_left), psi_r, method="DOP853", rtol=1e-11, atol=1e-13)
    psi_l = sol.y[:, -1]
    k = np.sqrt(E * E - m * m)
    u_in = _spinor_1p1(E, k, m) * np.exp(1j * k * x_left)
    u_rf = _spinor_1p1(E, -k, m) * np.exp(-1j * k * x_left)
    A, B = np.linalg.solve(np.stack([u_in, u_rf], axis=1), psi_l)
    j_in = abs(A) ** 2 * _current(_spinor_1p1(E, k, m))
    T = _current(u_tr) / j_in
    R = -abs(B) ** 2 * _current(_spinor_1p1(E, -k, m)) / j_in
    return T, R


def klein_T_formula(p0, V0, L, m=1.0):
    """Eq. 24 as read here, for incident momentum p0.

    The printed formula lacks a closing parenthesis and names
    p = sqrt((E - V0)^2 - 1) (transmitted) and p' = -sqrt(E^2 - 1) (incident),
    E = sqrt(p0^2 + 1).  Reading (masses kept):
        T = | sinh(pi p L) sinh(pi p' L) /
              ( sinh(pi (V0 + p + p') L / 2) sinh(pi (V0 - p - p') L / 2) ) |
    with p = -q, q the transmitted momentum signed by the transmitted group
    velocity (q / (E - V0) > 0).  In the Klein zone E < V0 - m this is the
    printed p = +sqrt(...); above the step (E > V0 + m) it is -sqrt(...).
    T = 0 where the transmitted wave does not propagate (|E - V0| < m).
    """
    E = np.sqrt(p0 * p0 + m * m)
    eps = E - V0
    if eps * eps <= m * m:
        return 0.0
    q = np.sign(eps) * np.sqrt(eps * eps - m * m)
    p = -q
    pp = -np.sqrt(E * E - m * m)
    num = np.sinh(np.pi * p * L) * np.sinh(np.pi * pp * L)
    den = np.sinh(np.pi * (V0 + p + pp) * L / 2) * np.sinh(np.pi * (V0 - p - pp) * L / 2)
    return float(abs(num / den))


def sommerfeld(x, V0, x0, L):
    """Sommerfeld smooth step, Eq. 23: V(x) = V0/2 [1 + tanh((x - x0)/L)]."""
    return 0.5 * V0 * (1.0 + np.tanh((np.asarray(x) - x0) / L))


def zb_frequency(p, m):
    """Angular frequency 2E of the oscillating term of Eq. 18 (hbar = c = 1)."""
    return 2.0 * np.sqrt(float(np.dot(p, p)) + m * m)
