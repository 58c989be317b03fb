"""Observables of a discrete solution, by trapezoidal sums over spatial nodes.

* ``charge``: Q(t) = int ||psi(x, t)||^2 dx per time layer (the conserved
  quantity monitored in Sec. 4.1's energy-loss study, read here as the
  charge; the paper does not define its E(t)).
* ``energy``: int psi^dagger H psi dx per layer with H applied spectrally
  (periodic meshes only), the other reading of Sec. 4.1's E(t).
* ``mean_position``: <x(t)> = int x ||psi||^2 dx / int ||psi||^2 dx
  (Sec. 4.2, Eq. 20, normalised).
* ``transmission``: T and R of Sec. 4.3, Eq. 25 - the fraction of
  int ||psi(x, t_f)||^2 dx lying on either side of x0.

Trapezoid weights per axis: periodic axes weight every node by h; open axes
halve the two end nodes; Dirichlet axes hold interior nodes only (the ends are
zero) and weight them by h.

Pinned by tests/test_oracle_observables.py: the charge of densities for
which the trapezoid rule is exact equals their closed-form integral; a
one-node density has its mean position at that node on every axis of a 3+1
mesh; transmitted shares follow the node weights (a node at x0 counting
half); a periodic-grid plane wave u_+-(p) e^{i p.x} has energy +-E(p) times
the volume, and a superposition of modes the sum of its parts.  The charge
self-convergence and Zitterbewegung tests (tests/test_oracle_physics.py) use
charge and mean_position on FEM solutions.
"""

import numpy as np

from .mesh import OPEN


def axis_weights(mesh, k):
    w = np.full(mesh.nu[k], mesh.h[k] if k < mesh.d else 1.0)
    if k < mesh.d and mesh.bc[k] == OPEN:
        w[0] *= 0.5
        w[-1] *= 0.5
    return w


def _weights(mesh):
    wx, wy, wz = (axis_weights(mesh, k) for k in range(3))
    return wz[:, None, None] * wy[None, :, None] * wx[None, None, :]


def density(psi_layers):
    """||psi||^2 summed over spinor components; input (..., NC)."""
    return np.sum(np.abs(psi_layers) ** 2, axis=-1)


def charge(mesh, psi_layers):
    """Q per layer; psi_layers (n_layers, nz, ny, nx, NC)."""
    w = _weights(mesh)
    return np.einsum("nzyx,zyx->n", density(psi_layers), w)


def mean_position(mesh, psi_layers, k=0):
    """<x_k> per layer."""
    w = _weights(mesh)
    c = mesh.node_coords(k)
    shape = [1, 1, 1]
    shape[2 - k] = -1
    xk = c.reshape(shape)
    rho = density(psi_layers)
    return np.einsum("nzyx,zyx->n", rho, w * xk) / np.einsum("nzyx,zyx->n", rho, w)


def transmission(mesh, psi_layer, x0):
    """(T, R): shares of int ||psi||^2 at x > x0 and x < x0 (node at x0 split in half)."""
    rho = density(psi_layer[None])[0]
    w = _weights(mesh)
    x = mesh.node_coords(0)[None, None, :]
    tot = np.sum(rho * w)
    side = np.where(x > x0 + 1e-12, 1.0, np.where(x < x0 - 1e-12, 0.0, 0.5))
    T = np.sum(rho * w * side) / tot
    return T, 1.0 - T


def energy(mesh, psi_layers, m):
    """int psi^dagger H psi dx per layer, H = alpha.p + beta m applied by FFT (periodic axes)."""
    from .dirac import alphas_beta
    d = mesh.d
    al, be = alphas_beta(d)
    out = []
    for psi in psi_layers:
        F = np.fft.fftn(psi, axes=(0, 1, 2))
        ks = []
        for k in range(3):
            n = mesh.nu[k]
            ks.append(2 * np.pi * np.fft.fftfreq(n, d=mesh.h[k]) if k < d else np.zeros(1))
        pz, py, px = np.meshgrid(ks[2], ks[1], ks[0], indexing="ij")
        p = [px, py, pz]
        HF = np.einsum("ab,zyxb->zyxa", be * m, F)
        for k in range(d):
            HF = HF + p[k][..., None] * np.einsum("ab,zyxb->zyxa", al[k], F)
        Hpsi = np.fft.ifftn(HF, axes=(0, 1, 2))
        out.append(np.real(np.sum(np.conj(psi) * Hpsi) * np.prod([mesh.h[k] for k in range(d)])))
    return np.array(out)
