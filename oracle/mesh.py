"""Structured spacetime mesh: geometry, node numbering, known/unknown split.

Algorithm 1 step 1 (build the global mesh) and the known/unknown partition of
Sec. 2.1 (Eqs. 8-11): the spinors on the t = 0 layer are known (the K values
Psi_1..Psi_K of Eq. 8); every node of every later time layer, including the
final one, is unknown.

Spatial boundary per axis (the paper states Psi = Psi_0 on the boundary in
Eq. 2 but Algorithm 1 removes only the t = 0 layer; readings):
* PERIODIC  (0): nodes 0..n_el-1, element e joins nodes e and (e+1) mod n_el.
* OPEN      (1): nodes 0..n_el, natural (no condition) at both ends.
* DIRICHLET (2): nodes 0..n_el, the two end nodes are known and zero at all
  times (homogeneous), so only nodes 1..n_el-1 are unknowns.

Arrays are indexed [t][z][y][x][c] (x fastest, spinor component innermost);
axes a mesh does not have keep length one.  "Geometric" arrays hold all mesh
nodes including t = 0 and Dirichlet end nodes; "unknown" arrays hold only the
unknowns, time layers 1..N_t.
"""

import numpy as np

from .dirac import ncomp

PERIODIC, OPEN, DIRICHLET = 0, 1, 2


class Mesh:
    """Uniform structured Q1 mesh over [lo, hi] per axis (x, y, z, t)."""

    def __init__(self, d, n_el, lo, hi, bc):
        if d not in (1, 2, 3):
            raise ValueError("d must be 1, 2 or 3")
        self.d = d
        self.nc = ncomp(d)
        self.nel = [int(n_el[k]) if k < d else 1 for k in range(3)]
        self.nt = int(n_el[3])
        self.lo = [float(lo[k]) if k < d else 0.0 for k in range(3)]
        self.hi = [float(hi[k]) if k < d else 1.0 for k in range(3)]
        self.t_lo, self.t_hi = float(lo[3]), float(hi[3])
        self.bc = [int(bc[k]) if k < d else PERIODIC for k in range(3)]
        for k in range(d):
            if self.nel[k] < 1 or (self.bc[k] == DIRICHLET and self.nel[k] < 2):
                raise ValueError("too few elements on axis %d" % k)
        if self.nt < 1:
            raise ValueError("need at least one time element")
        self.h = [(self.hi[k] - self.lo[k]) / self.nel[k] for k in range(3)]
        self.ht = (self.t_hi - self.t_lo) / self.nt
        # geometric nodes per axis and the unknown sub-range [u0, u0 + nu)
        self.ngeo, self.u0, self.nu = [], [], []
        for k in range(3):
            if k >= d:
                self.ngeo.append(1); self.u0.append(0); self.nu.append(1)
            elif self.bc[k] == PERIODIC:
                self.ngeo.append(self.nel[k]); self.u0.append(0); self.nu.append(self.nel[k])
            elif self.bc[k] == OPEN:
                self.ngeo.append(self.nel[k] + 1); self.u0.append(0); self.nu.append(self.nel[k] + 1)
            else:
                self.ngeo.append(self.nel[k] + 1); self.u0.append(1); self.nu.append(self.nel[k] - 1)

    # ---- sizes -----------------------------------------------------------
    @property
    def unknown_shape(self):
        """(N_t, nz, ny, nx, NC) of the unknown vector."""
        return (self.nt, self.nu[2], self.nu[1], self.nu[0], self.nc)

    @property
    def geo_shape(self):
        """(N_t + 1, gz, gy, gx, NC) of the geometric node array."""
        return (self.nt + 1, self.ngeo[2], self.ngeo[1], self.ngeo[0], self.nc)

    @property
    def n_spatial_nodes(self):
        return self.nu[0] * self.nu[1] * self.nu[2]

    @property
    def n_unknowns(self):
        return self.nt * self.n_spatial_nodes * self.nc

    @property
    def spatial_shape(self):
        """(nz, ny, nx, NC): one time layer of unknowns, also the psi0 layout."""
        return (self.nu[2], self.nu[1], self.nu[0], self.nc)

    # ---- geometry --------------------------------------------------------
    def node_coords(self, k):
        """Coordinates of the unknown nodes along spatial axis k."""
        return self.lo[k] + self.h[k] * (self.u0[k] + np.arange(self.nu[k]))

    def time_coords(self):
        """Times of layers 0..N_t (layer 0 is the initial data)."""
        return self.t_lo + self.ht * np.arange(self.nt + 1)

    def element_centroids(self, k):
        """Centroid coordinate of each element along spatial axis k."""
        return self.lo[k] + self.h[k] * (np.arange(self.nel[k]) + 0.5)

    # ---- connectivity ----------------------------------------------------
    def elem_node(self, k, e, a):
        """Geometric node index along spatial axis k of local node a of element e."""
        g = np.asarray(e) + a
        if self.bc[k] == PERIODIC:
            return g % self.ngeo[k]
        return g

    def to_geo(self, u):
        """Unknown array (N_t, nz, ny, nx, NC) -> geometric array with zero t=0 and ends."""
        g = np.zeros(self.geo_shape, dtype=np.complex128)
        g[1:, self.u0[2]:self.u0[2] + self.nu[2], self.u0[1]:self.u0[1] + self.nu[1],
          self.u0[0]:self.u0[0] + self.nu[0], :] = u.reshape(self.unknown_shape)
        return g

    def from_geo(self, g):
        """Geometric array -> the unknown entries (rows of D_w22)."""
        return g[1:, self.u0[2]:self.u0[2] + self.nu[2], self.u0[1]:self.u0[1] + self.nu[1],
                 self.u0[0]:self.u0[0] + self.nu[0], :].copy()

    def layer_to_geo(self, psi0):
        """Initial data on the unknown spatial nodes -> a t = 0 geometric layer."""
        g = np.zeros(self.geo_shape[1:], dtype=np.complex128)
        g[self.u0[2]:self.u0[2] + self.nu[2], self.u0[1]:self.u0[1] + self.nu[1],
          self.u0[0]:self.u0[0] + self.nu[0], :] = np.asarray(psi0).reshape(self.spatial_shape)
        return g

    def unknown_mask_geo(self):
        """Boolean geometric array (without the component axis): True at unknowns."""
        msk = np.zeros(self.geo_shape[:4], dtype=bool)
        msk[1:, self.u0[2]:self.u0[2] + self.nu[2], self.u0[1]:self.u0[1] + self.nu[1],
            self.u0[0]:self.u0[0] + self.nu[0]] = True
        return msk
