"""Pins of the oracle's per-layer observables (charge, mean position, transmitted
share) to results that do not depend on the oracle's own code.

The observables integrate |psi|^2 over one time layer with the nodal (trapezoid)
rule of the Q1 mesh: weight h per node, h/2 at the two end nodes of an open
axis, the end nodes of a Dirichlet axis (psi = 0 there) left out.  The pins:
* the trapezoid rule is exact for trigonometric polynomials of degree below the
  node count on a periodic axis, for linear functions on an open axis and for
  piecewise-linear functions with kinks at nodes, so the charge of such
  densities equals their integral in closed form; on a product mesh it is the
  product of the one-axis integrals;
* a density carried by one node has its mean position at that node, whose
  coordinate is fixed by the axis type (Dirichlet unknown i sits at lo + (i+1) h);
* a density on two nodes on either side of x0 splits into shares given by the
  two nodes' weights, and a node at x0 itself counts half to each side.
A dropped half weight, an end node counted on a Dirichlet axis, a coordinate
off by one node, or the axes of a 3+1 mesh taken in the wrong order fail one
of them.
"""
import numpy as np
import pytest

from oracle import observables as OB
from oracle.mesh import DIRICHLET, OPEN, PERIODIC, Mesh

LO, HI = [-1.5, 0.25, -2.0, 0.0], [2.5, 1.75, 1.0, 1.0]


def _mesh(d, n_el, bc):
    """Mesh with the given spatial element counts and two time elements."""
    nel = list(n_el) + [1] * (3 - len(n_el))
    return Mesh(d, nel + [2], LO, HI, list(bc) + [PERIODIC] * (3 - len(bc)))


def _layers(mesh, rho_axes, nlayers=2):
    """psi layers whose density is the product of per-axis nodal densities, split
    unevenly over the spinor components (the observables sum |psi_c|^2)."""
    rho = np.ones((mesh.nu[2], mesh.nu[1], mesh.nu[0]))
    for k, r in enumerate(rho_axes):
        shape = [1, 1, 1]
        shape[2 - k] = -1
        rho = rho * np.asarray(r, dtype=float).reshape(shape)
    frac = np.linspace(0.2, 0.8, mesh.nc)
    frac = frac / frac.sum()
    psi = np.sqrt(rho[..., None] * frac) * np.exp(1j * np.arange(mesh.nc))
    return np.stack([psi * (1 + 0.5 * n) for n in range(nlayers)])     # layer n scales rho by (1 + n/2)^2


def _node_x(lo, hi, nel, bc):
    """Coordinates of an axis' unknown nodes, from the axis type alone."""
    h = (hi - lo) / nel
    if bc == PERIODIC:
        return lo + h * np.arange(nel)
    if bc == OPEN:
        return lo + h * np.arange(nel + 1)
    return lo + h * np.arange(1, nel)


def _exact_density(kind, lo, hi, x):
    """(nodal density, its integral over [lo, hi]) for which the trapezoid rule is exact."""
    L = hi - lo
    if kind == "trig":                       # periodic axis: 1 + cos(2 pi 3 (x - lo) / L) / 2
        return 1 + 0.5 * np.cos(2 * np.pi * 3 * (x - lo) / L), L
    if kind == "linear":                     # open axis: 2 + (x - lo) / L
        return 2 + (x - lo) / L, 2 * L + L / 2
    xm = lo + L * 0.75                       # Dirichlet axis: hat of height 3, zero at both ends
    return np.where(x <= xm, 3 * (x - lo) / (xm - lo), 3 * (hi - x) / (hi - xm)), 1.5 * L


KIND = {PERIODIC: "trig", OPEN: "linear", DIRICHLET: "hat"}


@pytest.mark.parametrize("d,n_el,bc", [(1, [16], [PERIODIC]), (1, [12], [OPEN]), (1, [8], [DIRICHLET]),
                                       (2, [16, 10], [PERIODIC, OPEN]), (2, [12, 8], [OPEN, DIRICHLET]),
                                       (3, [8, 12, 16], [DIRICHLET, OPEN, PERIODIC])])
def test_charge_exact_quadrature(d, n_el, bc):
    mesh = _mesh(d, n_el, bc)
    rhos, total = [], 1.0
    for k in range(d):
        x = _node_x(LO[k], HI[k], n_el[k], bc[k])
        np.testing.assert_allclose(mesh.node_coords(k), x, rtol=0, atol=1e-15)
        r, integral = _exact_density(KIND[bc[k]], LO[k], HI[k], x)
        rhos.append(r)
        total *= integral
    Q = OB.charge(mesh, _layers(mesh, rhos))
    np.testing.assert_allclose(Q, [total, total * 2.25], rtol=1e-13)


@pytest.mark.parametrize("bc", [PERIODIC, OPEN, DIRICHLET])
def test_mean_position_of_one_node(bc):
    """3+1 mesh, every axis of type bc: a density on the single node (i, j, l) has
    <x_k> at that node's coordinate on each axis k."""
    n_el = [6, 8, 10]
    mesh = _mesh(3, n_el, [bc] * 3)
    idx = [1, mesh.nu[1] - 2, mesh.nu[2] // 2]
    rhos = []
    for k in range(3):
        r = np.zeros(mesh.nu[k])
        r[idx[k]] = 1.0
        rhos.append(r)
    psi = _layers(mesh, rhos, nlayers=1)
    for k in range(3):
        expect = _node_x(LO[k], HI[k], n_el[k], bc)[idx[k]]
        assert OB.mean_position(mesh, psi, k)[0] == pytest.approx(expect, abs=1e-13)


def test_mean_position_symmetric_density():
    """Open axis, density symmetric about the middle node: <x> is the midpoint,
    the half weights of the end nodes included."""
    mesh = _mesh(1, [10], [OPEN])
    x = mesh.node_coords(0)
    r = 1 + (x - 0.5) ** 2
    psi = _layers(mesh, [r], nlayers=1)
    assert OB.mean_position(mesh, psi, 0)[0] == pytest.approx(0.5, abs=1e-14)
    # the end nodes carry half weight: a density on both end nodes, 1 on the left and 3 on the right
    r = np.zeros_like(x)
    r[0], r[-1], r[4] = 1.0, 3.0, 1.0
    psi = _layers(mesh, [r], nlayers=1)
    num = 0.5 * 1.0 * x[0] + 0.5 * 3.0 * x[-1] + 1.0 * x[4]
    den = 0.5 * 1.0 + 0.5 * 3.0 + 1.0
    assert OB.mean_position(mesh, psi, 0)[0] == pytest.approx(num / den, abs=1e-14)


def test_transmission_shares():
    mesh = _mesh(1, [10], [OPEN])          # nodes -1.5, -1.1, ..., 2.5 (h = 0.4)
    x = mesh.node_coords(0)
    r = np.zeros_like(x)
    r[0], r[7] = 2.0, 1.0                  # end node (half weight) left of x0, an interior node right of it
    psi = _layers(mesh, [r], nlayers=1)[0]
    T, R = OB.transmission(mesh, psi, 0.0)
    assert T == pytest.approx(1.0 / (1.0 + 0.5 * 2.0), abs=1e-14) and T + R == pytest.approx(1.0, abs=1e-15)
    # a node exactly at x0 counts half to each side
    r = np.zeros_like(x)
    r[5] = 1.0                             # x[5] = 0.5
    T, _ = OB.transmission(mesh, _layers(mesh, [r], nlayers=1)[0], x[5])
    assert T == pytest.approx(0.5, abs=1e-15)
    # Dirichlet axis: unknown 0 sits at lo + h, so x0 between lo and lo + h leaves it on the right
    mesh = _mesh(1, [10], [DIRICHLET])
    r = np.zeros(mesh.nu[0])
    r[0] = 1.0
    T, _ = OB.transmission(mesh, _layers(mesh, [r], nlayers=1)[0], LO[0] + 0.2)
    assert T == pytest.approx(1.0, abs=1e-15)


def _plane(mesh, j, u):
    """u e^{i p.x} on the unknown nodes, p_k = 2 pi j_k / L_k (a mode of the periodic grid)."""
    p = np.array([2 * np.pi * j[k] / (mesh.hi[k] - mesh.lo[k]) for k in range(mesh.d)])
    phase = np.zeros((mesh.nu[2], mesh.nu[1], mesh.nu[0]))
    for k in range(mesh.d):
        shape = [1, 1, 1]
        shape[2 - k] = -1
        phase = phase + p[k] * mesh.node_coords(k).reshape(shape)
    return np.exp(1j * phase)[..., None] * u, p


@pytest.mark.parametrize("d,n_el,j", [(1, [16], [3]), (2, [12, 10], [2, -3]), (3, [8, 6, 10], [1, 2, -2])])
def test_energy_of_plane_waves(d, n_el, j):
    """A periodic-grid plane wave u_+-(p) e^{i p.x} has energy +-E(p) x volume, E = sqrt(p^2 + m^2);
    a superposition of two modes has the sum of the parts (the modes are orthogonal)."""
    import workloads as W
    m = 1.3
    mesh = _mesh(d, n_el, [PERIODIC] * d)
    vol = np.prod([mesh.hi[k] - mesh.lo[k] for k in range(d)])
    psi_p, p = _plane(mesh, j, 1.0)
    up, um = W.spinor_pm(d, p, m)
    E = np.sqrt(p @ p + m * m)
    for u, sign in ((up, 1.0), (um, -1.0)):
        psi, _ = _plane(mesh, j, u)
        assert OB.energy(mesh, psi[None], m)[0] == pytest.approx(sign * E * vol, rel=1e-12)
    j2 = [-x + 1 for x in j]
    psi2, p2 = _plane(mesh, j2, 1.0)
    up2, um2 = W.spinor_pm(d, p2, m)
    E2 = np.sqrt(p2 @ p2 + m * m)
    a, c = 0.6 - 0.2j, 0.5j
    mix = a * _plane(mesh, j, up)[0] + c * _plane(mesh, j2, um2)[0]
    expect = (abs(a) ** 2 * E - abs(c) ** 2 * E2) * vol
    assert OB.energy(mesh, mix[None], m)[0] == pytest.approx(expect, rel=1e-12)
