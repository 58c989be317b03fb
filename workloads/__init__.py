"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module only *generates inputs*: mesh descriptions, initial spinor data,
potentials and random vectors.  It holds none of the discretisation's
arithmetic (no element matrices, no operator, no solver) and imports neither
the oracle nor the product library.

Workloads (element counts as (x, y, z, t); every input is synthetic):

* ``plane_wave_1p1``  1+1, 64 x 64 on [0, 2 pi] x [0, 1], periodic x, m = 1,
  k = 1, Psi_0 = u_+(k) exp(i k x).  Deterministic.
* ``zb_2p1``          2+1, 96^2 x 96 on [-8, 8]^2 x [0, 4], periodic x, y,
  m = 1; Gaussian packet sigma = 0.5 (position spread of |Psi|^2), central
  momentum (2, 0), (u_+ + e^{i phi} u_-)/sqrt 2 with phi drawn from the seed
  (splitmix64, seed 20210326), unit discrete norm.
* ``klein_3p1``       3+1, 48^3 x 48 on [-6, 6]^3 x [0, 3], x homogeneous
  Dirichlet (the packet's density at x = +-6 is ~1e-14 and it does not reach
  the walls before t = 3; with open, natural ends unpreconditioned GMRES(30)
  stagnates on this system), y, z periodic, m = 1, step V = 2.5 for element
  centroids x >= 0 (0 otherwise);
  packet Gaussian in x (sigma 0.5, centre -2), uniform in y and z, momentum
  p0 x^ with p0 ~ U[1, 3] from the seed (or fixed), positive-energy spinor.

The spinors u_+/u_- are the closed-form eigenvectors of the free Dirac
Hamiltonian in the representation used throughout (1+1 and 2+1:
alpha = (sigma_x, sigma_y), beta = sigma_z; 3+1: Dirac representation).
"""

import numpy as np

PERIODIC, OPEN, DIRICHLET = 0, 1, 2
MASK64 = (1 << 64) - 1


def splitmix64(state):
    """One step of splitmix64 (Steele, Lea & Flood 2014): returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def uniform01(seed, n):
    """n doubles in [0, 1) from splitmix64 seeded with ``seed`` (top 53 bits)."""
    s, out = seed & MASK64, []
    for _ in range(n):
        s, z = splitmix64(s)
        out.append((z >> 11) * (1.0 / (1 << 53)))
    return out


def random_complex(n, seed, dtype=np.complex128):
    """Standard complex normal vector (numpy PCG64 generator)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return v.astype(dtype)


def node_coords(n_el, lo, hi, bc):
    """Coordinates of the unknown nodes along one spatial axis."""
    h = (hi - lo) / n_el
    if bc == PERIODIC:
        idx = np.arange(n_el)
    elif bc == OPEN:
        idx = np.arange(n_el + 1)
    else:
        idx = np.arange(1, n_el)
    return lo + h * idx


def element_centroids(n_el, lo, hi):
    h = (hi - lo) / n_el
    return lo + h * (np.arange(n_el) + 0.5)


def spinor_pm(d, p, m):
    """(u_+, u_-) unit eigenvectors of H(p) with eigenvalues +E and -E."""
    p = list(p) + [0.0] * (3 - len(p))
    px, py, pz = p
    E = np.sqrt(px * px + py * py + pz * pz + m * m)
    nrm = np.sqrt(2 * E * (E + m))
    if d in (1, 2):
        pc = px + 1j * py
        up = np.array([E + m, pc]) / nrm
        um = np.array([-np.conj(pc), E + m]) / nrm
        return up, um
    # 3+1, Dirac representation, spin up: (E + m) chi, sigma.p chi
    up = np.array([E + m, 0.0, pz, px + 1j * py]) / nrm
    um = np.array([-pz, -(px + 1j * py), E + m, 0.0]) / nrm
    return up, um


class Workload:
    """A mesh description plus physical inputs for one solve."""

    def __init__(self, name, d, n_el, lo, hi, bc, m, V, psi0, extra=None):
        self.name = name
        self.d = d
        self.n_el = list(n_el)
        self.lo = list(lo)
        self.hi = list(hi)
        self.bc = list(bc)
        self.m = float(m)
        self.V = V            # None or float64 array, one value per spatial element (x fastest)
        self.psi0 = psi0      # complex128 (nz, ny, nx, NC) on the unknown spatial nodes
        self.extra = extra or {}

    @property
    def ncomp(self):
        return 2 if self.d < 3 else 4

    def mesh_args(self):
        return self.d, self.n_el, self.lo, self.hi, self.bc


def _grid(d, n_el, lo, hi, bc):
    xs = [node_coords(n_el[k], lo[k], hi[k], bc[k]) if k < d else np.zeros(1) for k in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return X, Y, Z


def _unit_norm(psi, d, n_el, lo, hi):
    vol = np.prod([(hi[k] - lo[k]) / n_el[k] for k in range(d)])
    return psi / np.sqrt(np.sum(np.abs(psi) ** 2) * vol)


def plane_wave_1p1(n=64, k=1.0, m=1.0):
    n_el, lo, hi, bc = [n, 1, 1, n], [0, 0, 0, 0], [2 * np.pi, 1, 1, 1], [PERIODIC] * 3
    X, _, _ = _grid(1, n_el, lo, hi, bc)
    up, _ = spinor_pm(1, [k], m)
    psi0 = np.exp(1j * k * X)[..., None] * up
    return Workload("plane_wave_1p1_%dx%d" % (n, n), 1, n_el, lo, hi, bc, m, None, psi0,
                    {"k": k})


def zb_2p1(n=96, nt=96, seed=20210326, sigma=0.5, p0=(2.0, 0.0), m=1.0):
    n_el, lo, hi, bc = [n, n, 1, nt], [-8.0, -8.0, 0, 0], [8.0, 8.0, 1, 4.0], [PERIODIC] * 3
    X, Y, _ = _grid(2, n_el, lo, hi, bc)
    phi = 2 * np.pi * uniform01(seed, 1)[0]
    up, um = spinor_pm(2, p0, m)
    env = np.exp(-(X ** 2 + Y ** 2) / (4 * sigma ** 2) + 1j * (p0[0] * X + p0[1] * Y))
    psi0 = env[..., None] * ((up + np.exp(1j * phi) * um) / np.sqrt(2))
    psi0 = _unit_norm(psi0, 2, n_el, lo, hi)
    return Workload("zb_2p1_%dx%dx%d" % (n, n, nt), 2, n_el, lo, hi, bc, m, None, psi0,
                    {"phi": phi, "sigma": sigma, "p0": p0, "seed": seed})


def klein_3p1(n=48, nt=48, seed=1, p0=None, V0=2.5, sigma=0.5, xc=-2.0, m=1.0):
    n_el = [n, n, n, nt]
    lo, hi = [-6.0, -6.0, -6.0, 0.0], [6.0, 6.0, 6.0, 3.0]
    bc = [DIRICHLET, PERIODIC, PERIODIC]
    if p0 is None:
        p0 = 1.0 + 2.0 * uniform01(seed, 1)[0]
    X, _, _ = _grid(3, n_el, lo, hi, bc)
    up, _ = spinor_pm(3, [p0], m)
    env = np.exp(-(X - xc) ** 2 / (4 * sigma ** 2) + 1j * p0 * X)
    psi0 = _unit_norm(env[..., None] * up, 3, n_el, lo, hi)
    cx = element_centroids(n, lo[0], hi[0])
    V = np.broadcast_to(np.where(cx >= 0.0, V0, 0.0)[None, None, :], (n, n, n)).ravel().copy()
    return Workload("klein_3p1_%dx%dx%dx%d" % (n, n, n, nt), 3, n_el, lo, hi, bc, m, V, psi0,
                    {"p0": p0, "V0": V0, "seed": seed})


def sommerfeld_1p1(n=256, nt=256, L=0.001, V0=2.5, p0=1.05, sigma=4.0, xc=-16.0, half=40.0, tf=40.0, m=1.0):
    """1+1 Klein scattering at the Sommerfeld smooth step of Sec. 4.3, Eq. 23:
    V(x) = V0 / 2 (1 + tanh(x / L)) sampled at the element centroids; a
    positive-energy Gaussian packet (width sigma, centre xc, momentum p0) on
    [-half, half] x [0, tf] with homogeneous Dirichlet walls far from the packet."""
    n_el, lo, hi = [n, 1, 1, nt], [-half, 0, 0, 0], [half, 1, 1, tf]
    bc = [DIRICHLET, PERIODIC, PERIODIC]
    X, _, _ = _grid(1, n_el, lo, hi, bc)
    up, _ = spinor_pm(1, [p0], m)
    psi0 = np.exp(-(X - xc) ** 2 / (4 * sigma ** 2) + 1j * p0 * X)[..., None] * up
    cx = element_centroids(n, lo[0], hi[0])
    V = 0.5 * V0 * (1.0 + np.tanh(cx / L))
    return Workload("sommerfeld_1p1_%dx%d_L%g" % (n, nt, L), 1, n_el, lo, hi, bc, m, V, psi0,
                    {"p0": p0, "V0": V0, "L": L, "sigma": sigma})


def batch_instances(count=64, seed=4, n1=(32, 256), n2=(16, 48)):
    """Independent solves for the batched solver: each instance is 1+1 or 2+1
    (probability 1/2 each), with element counts per axis (time included) drawn
    uniformly from n1 (1+1) or n2 (2+1), mass U[0.5, 2], momentum U[-4, 4] along
    x, a barrier of height U[0, 3] over x >= 0 (x-only potential), and a
    positive-energy Gaussian packet of width 0.1 L at x = -L/4 on
    [-L/2, L/2]^d x [0, L/2], L = 20, homogeneous Dirichlet in x, periodic in y.
    All draws come from splitmix64(seed)."""
    u = uniform01(seed, 8 * count)
    out = []
    L = 20.0
    for i in range(count):
        r = u[8 * i: 8 * i + 8]
        d = 1 if r[0] < 0.5 else 2
        lo_n, hi_n = n1 if d == 1 else n2
        pick = lambda x: int(lo_n + min(int(x * (hi_n - lo_n + 1)), hi_n - lo_n))
        nx, ny, nt = pick(r[1]), pick(r[2]), pick(r[3])
        m = 0.5 + 1.5 * r[4]
        p0 = -4.0 + 8.0 * r[5]
        V0 = 3.0 * r[6]
        n_el = [nx, ny if d == 2 else 1, 1, nt]
        lo = [-L / 2, -L / 2 if d == 2 else 0.0, 0.0, 0.0]
        hi = [L / 2, L / 2 if d == 2 else 1.0, 1.0, L / 2]
        bc = [DIRICHLET, PERIODIC, PERIODIC]
        X, Y, _ = _grid(d, n_el, lo, hi, bc)
        pv = [p0] + ([0.0] if d == 2 else [])
        up, _ = spinor_pm(d, pv, m)
        sig = 0.1 * L
        env = np.exp(-((X + L / 4) ** 2) / (4 * sig ** 2) + 1j * p0 * X)
        psi0 = _unit_norm(env[..., None] * up, d, n_el, lo, hi)
        cx = element_centroids(nx, lo[0], hi[0])
        vx = np.where(cx >= 0.0, V0, 0.0)
        V = np.tile(vx, n_el[1]) if d == 2 else vx
        out.append(Workload("batch%03d_%dp1_%s" % (i, d, "x".join(str(k) for k in n_el[:d] + [nt])), d, n_el,
                            lo, hi, bc, m, V, psi0, {"p0": p0, "V0": V0}))
    return out


def random_mesh(d, n_el, bc, seed, with_potential=True, m=0.9):
    """Small random-data workload for parity tests (random psi0 and V)."""
    rng = np.random.default_rng(seed)
    lo = [-1.0, -0.5, 0.25, 0.0]
    hi = [1.0, 1.25, 1.5, 0.75]
    n_el = list(n_el)
    bc = list(bc) + [PERIODIC] * (3 - len(bc))
    nu = []
    for k in range(3):
        if k >= d:
            nu.append(1)
        elif bc[k] == PERIODIC:
            nu.append(n_el[k])
        elif bc[k] == OPEN:
            nu.append(n_el[k] + 1)
        else:
            nu.append(n_el[k] - 1)
    nc = 2 if d < 3 else 4
    shape = (nu[2], nu[1], nu[0], nc)
    psi0 = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    nsp = int(np.prod([n_el[k] if k < d else 1 for k in range(3)]))
    V = rng.uniform(-1.0, 2.0, nsp) if with_potential else None
    return Workload("random_%dp1" % d, d, n_el, lo, hi, bc, m, V, psi0)
