"""Preconditioners for flexible GMRES on A Psi_u = b (test infrastructure).

The paper's conclusion asks for a preconditioner (suggesting a time-additive
Schwarz method) and specifies none.  These are the non-learned candidates,
each returning a callable v -> M v for ``solvers.fgmres``:

* ``node_block_jacobi``: at every unknown spacetime node, the inverse of the
  NC x NC diagonal block of D_w22 (point Jacobi for spinors).
* ``time_slab_schwarz``: restricted additive Schwarz over time slabs of S
  layers, each slab extended by ``overlap`` layers on both sides and solved
  exactly by sparse LU, its result kept on the slab's own layers only;
  overlap 0 is time-slab block Jacobi.

The unknown vector is ordered [t][z][y][x][c] (time slowest), so a time
layer is a contiguous run of ``per`` = n_spatial_nodes * NC entries and a
node a run of NC entries.

Only ``tests/`` imports this module.  Pinned by tests/test_oracle_precond.py:
each preconditioner is the exact inverse of a matrix that is block diagonal
in its own blocks, and one slab covering all layers inverts A.
"""

import numpy as np
import scipy.sparse.linalg as spla


def node_block_jacobi(nc, A):
    """v -> blockdiag(A_ii)^-1 v over consecutive NC x NC diagonal blocks of A."""
    A = A.tocsr()
    n = A.shape[0]
    if n % nc:
        raise ValueError("size is not a multiple of NC")
    nb = n // nc
    blocks = np.zeros((nb, nc, nc), dtype=np.complex128)
    for i in range(nb):
        blocks[i] = A[i * nc:(i + 1) * nc, i * nc:(i + 1) * nc].toarray()
    inv = np.linalg.inv(blocks)

    def apply(v):
        return np.einsum("bij,bj->bi", inv, np.asarray(v, dtype=np.complex128).reshape(nb, nc)).ravel()
    return apply


def time_slab_schwarz(A, nt, per, S, overlap=0):
    """Restricted additive Schwarz over time slabs of S layers (``per`` unknowns per layer)."""
    A = A.tocsr()
    if A.shape[0] != nt * per or S < 1 or overlap < 0:
        raise ValueError("bad slab layout")
    slabs = []
    for s0 in range(0, nt, S):
        lo = max(0, s0 - overlap) * per
        hi = min(nt, s0 + S + overlap) * per
        own = (s0 * per, min(nt, s0 + S) * per)
        slabs.append((lo, hi, own, spla.splu(A[lo:hi, lo:hi].tocsc())))

    def apply(v):
        v = np.asarray(v, dtype=np.complex128)
        z = np.zeros_like(v)
        for lo, hi, own, lu in slabs:
            zs = lu.solve(v[lo:hi])
            z[own[0]:own[1]] = zs[own[0] - lo:own[1] - lo]
        return z
    return apply
