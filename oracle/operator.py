"""The discretised spacetime Dirac operator: assembly, known/unknown split, apply.

Sec. 2.1 (Eqs. 6-12) and Sec. 2.2: the weak form gives the block matrix D_w
(Eq. 7), assembled element by element as the sum of element stiffness
matrices (Sec. 2.2).  The t = 0 spinors are known (Eq. 8); removing their rows
and moving their columns to the right-hand side gives
    D_w22 Psi_unknown = - D_w21 Psi_0          (Eq. 11, Algorithm 1 steps 3-5),
so the hot-path operator is A = D_w22 and the right-hand side b = -D_w21 Psi_0.

Three routes, all from the same element operator (oracle.element):
* ``assemble`` + ``split``: Algorithm 1 literally (sparse D_w over every mesh
  node, then the sub-matrices D_w22 / D_w21).  Small meshes.
* ``apply`` / ``rhs``: matrix-free, element by element - gather the 2^(d+1)
  local spinors, multiply by the dense element operator, scatter-add.
* ``apply_rows``: the same sum evaluated one output node at a time, for
  sampling outputs of meshes too large for a full oracle apply.

Potential V: one value per spatial element (sampled at its centroid), constant
in time, entering the element operator as -V_e D^0 (x) I (Hamiltonian form).

Nonzero Dirichlet values (``split(..., boundary=...)``) move to the
right-hand side with the t = 0 layer; the paper's Eq. 2 prescribes the
boundary values, and every workload here uses zero.

Pinned by tests/test_oracle_operator.py: the exact discrete Fourier reduction
of a periodic mesh (symbols h(2 + cos th)/3 and i sin th), exact reduction of
2+1 / 3+1 with data uniform in y (and z) to 1+1, equality of the three routes,
identical LU solutions of the Hamiltonian and appendix forms, and Dirichlet
data taken from an open-axis solution reproducing that solution inside.
"""

import numpy as np
import scipy.sparse as sp

from .element import element_operator, local_bits
from .mesh import Mesh  # noqa: F401  (type used by callers)


def _spatial_elements(mesh):
    """Flat lists (ez, ey, ex) of all spatial elements, x fastest."""
    ez, ey, ex = np.meshgrid(np.arange(mesh.nel[2]), np.arange(mesh.nel[1]),
                             np.arange(mesh.nel[0]), indexing="ij")
    return ez.ravel(), ey.ravel(), ex.ravel()


def _geo_flat(mesh, t, z, y, x):
    g = mesh.ngeo
    return ((np.asarray(t) * g[2] + z) * g[1] + y) * g[0] + x


def _local_geo_index(mesh, et, ez, ey, ex):
    """(nE, nloc) flat geometric node index of every local node of each element."""
    d = mesh.d
    cols = []
    for l in range(2 ** (d + 1)):
        b = local_bits(l, d)                      # [a_x, (a_y), (a_z), a_t]
        ax = b[0]
        ay = b[1] if d >= 2 else 0
        az = b[2] if d >= 3 else 0
        at = b[d]
        cols.append(_geo_flat(mesh, et + at, mesh.elem_node(2, ez, az),
                              mesh.elem_node(1, ey, ay), mesh.elem_node(0, ex, ax)))
    return np.stack(cols, axis=1)


def _potential(mesh, V):
    if V is None:
        return np.zeros(mesh.nel[0] * mesh.nel[1] * mesh.nel[2])
    V = np.asarray(V, dtype=np.float64).ravel()
    if V.size != mesh.nel[0] * mesh.nel[1] * mesh.nel[2]:
        raise ValueError("V needs one value per spatial element")
    return V


def _apply_slabs(mesh, m, V, Xgeo, slabs, form):
    """Element-by-element y = sum_e A_e x over the time slabs listed (geometric)."""
    nc = mesh.nc
    A0, AV = element_operator(mesh.d, mesh.h, mesh.ht, m, form)
    ez, ey, ex = _spatial_elements(mesh)
    Ve = _potential(mesh, V)
    X = Xgeo.reshape(-1, nc)
    Y = np.zeros_like(X)
    nloc = 2 ** (mesh.d + 1)
    for et in slabs:
        idx = _local_geo_index(mesh, et, ez, ey, ex)                # (nE, nloc)
        G = X[idx].reshape(idx.shape[0], nloc * nc)                # gather
        out = G @ A0.T + Ve[:, None] * (G @ AV.T)                  # local matvec
        np.add.at(Y, idx.reshape(-1), out.reshape(-1, nc))         # scatter-add
    return Y.reshape(Xgeo.shape)


def apply(mesh, m, V, x, form="hamiltonian"):
    """y = A x with A = D_w22: x, y flat complex vectors of the unknowns."""
    Xg = mesh.to_geo(np.asarray(x, dtype=np.complex128))
    Yg = _apply_slabs(mesh, m, V, Xg, range(mesh.nt), form)
    return mesh.from_geo(Yg).ravel()


def rhs(mesh, m, V, psi0, form="hamiltonian"):
    """b = -D_w21 Psi_0: only the first time slab couples layer 0 to the unknowns."""
    Xg = np.zeros(mesh.geo_shape, dtype=np.complex128)
    Xg[0] = mesh.layer_to_geo(psi0)
    Yg = _apply_slabs(mesh, m, V, Xg, [0], form)
    Yg[0] = 0.0
    Yg[2:] = 0.0
    return -mesh.from_geo(Yg).ravel()


def apply_rows(mesh, m, V, x, nodes, form="hamiltonian"):
    """Rows of y = A x at selected unknown nodes, each summed element by element.

    nodes: flat indices into the unknown node grid (N_t, nz, ny, nx) (no
    component).  Returns (len(nodes), NC) complex.
    """
    d, nc = mesh.d, mesh.nc
    nodes = np.asarray(nodes, dtype=np.int64)
    Xg = mesh.to_geo(np.asarray(x, dtype=np.complex128)).reshape(-1, nc)
    A0, AV = element_operator(d, mesh.h, mesh.ht, m, form)
    Ve = _potential(mesh, V)
    nt, nz, ny, nx = mesh.unknown_shape[:4]
    ix = nodes % nx
    iy = (nodes // nx) % ny
    iz = (nodes // (nx * ny)) % nz
    it = nodes // (nx * ny * nz)
    gt = it + 1
    gz, gy, gx = iz + mesh.u0[2], iy + mesh.u0[1], ix + mesh.u0[0]
    out = np.zeros((nodes.size, nc), dtype=np.complex128)
    nloc = 2 ** (d + 1)
    for lrow in range(nloc):                     # position of the row node in the element
        b = local_bits(lrow, d)
        a = [b[0], b[1] if d >= 2 else 0, b[2] if d >= 3 else 0]
        et = gt - b[d]
        ok = (et >= 0) & (et < mesh.nt)
        esp = []
        for k, gk in enumerate((gx, gy, gz)):
            e = gk - a[k]
            if k < d and mesh.bc[k] == 0:        # periodic: always an element
                e = e % mesh.nel[k]
            elif k < d:
                ok &= (e >= 0) & (e < mesh.nel[k])
            esp.append(e)
        if not ok.any():
            continue
        sel = np.nonzero(ok)[0]
        ex_, ey_, ez_ = esp[0][sel], esp[1][sel], esp[2][sel]
        idx = _local_geo_index(mesh, et[sel], ez_, ey_, ex_)
        G = Xg[idx].reshape(sel.size, nloc * nc)
        eflat = (ez_ * mesh.nel[1] + ey_) * mesh.nel[0] + ex_
        rows = slice(lrow * nc, (lrow + 1) * nc)
        out[sel] += G @ A0[rows].T + Ve[eflat][:, None] * (G @ AV[rows].T)
    return out


def assemble(mesh, m, V, form="hamiltonian"):
    """Sparse D_w over every geometric node (Eq. 7, Algorithm 1 step 3)."""
    nc = mesh.nc
    A0, AV = element_operator(mesh.d, mesh.h, mesh.ht, m, form)
    ez, ey, ex = _spatial_elements(mesh)
    Ve = _potential(mesh, V)
    rows, cols, vals = [], [], []
    for et in range(mesh.nt):
        idx = _local_geo_index(mesh, et, ez, ey, ex)
        dof = (idx[:, :, None] * nc + np.arange(nc)).reshape(idx.shape[0], -1)  # (nE, nloc*nc)
        blk = A0[None, :, :] + Ve[:, None, None] * AV[None, :, :]
        rows.append(np.broadcast_to(dof[:, :, None], blk.shape).ravel())
        cols.append(np.broadcast_to(dof[:, None, :], blk.shape).ravel())
        vals.append(blk.ravel())
    n = int(np.prod(mesh.geo_shape))
    Dw = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(n, n)).tocsr()
    Dw.sum_duplicates()
    return Dw


def dirichlet_end_mask(mesh):
    """Boolean spatial geometric array (gz, gy, gx): True at the end nodes of Dirichlet axes."""
    msk = np.zeros(mesh.geo_shape[1:4], dtype=bool)
    for k in range(mesh.d):
        if mesh.bc[k] == 2:                                   # DIRICHLET
            sl = [slice(None)] * 3
            for end in (0, mesh.ngeo[k] - 1):
                sl[2 - k] = end
                msk[tuple(sl)] = True
    return msk


def split(mesh, Dw, psi0, boundary=None):
    """Eq. 11: return (D_w22, b = -D_w21 Psi_known).

    Psi_known is the t = 0 layer (psi0 on its unknown spatial nodes) and the
    end nodes of Dirichlet axes on every layer, zero unless ``boundary`` (a
    geometric array of shape mesh.geo_shape) gives their spinors; its other
    entries are ignored.  Prescribed Dirichlet values thus enter only the
    right-hand side, like the initial data."""
    nc = mesh.nc
    unk = np.repeat(mesh.unknown_mask_geo().ravel(), nc)
    known_vals = np.zeros(mesh.geo_shape, dtype=np.complex128)
    known_vals[0] = mesh.layer_to_geo(psi0)
    if boundary is not None:
        ends = dirichlet_end_mask(mesh)
        known_vals[:, ends] = np.asarray(boundary, dtype=np.complex128).reshape(mesh.geo_shape)[:, ends]
    known_vals = known_vals.ravel()[~unk]
    D22 = Dw[unk][:, unk].tocsr()
    D21 = Dw[unk][:, ~unk].tocsr()
    return D22, -(D21 @ known_vals)
