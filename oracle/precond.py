"""Preconditioners for flexible GMRES on A Psi_u = b (test infrastructure).

The paper's conclusion (Sec. 5) asks for a preconditioner (suggesting a time-additive
Schwarz method) and specifies none.  These are the non-learned candidates,
each returning a callable v -> M v for ``solvers.fgmres``:

* ``node_block_jacobi``: at every unknown spacetime node, the inverse of the
  NC x NC diagonal block of D_w22 (point Jacobi for spinors).
* ``time_slab_schwarz``: restricted additive Schwarz over time slabs of S
  layers, each slab extended by ``overlap`` layers on both sides and solved
  exactly by sparse LU, its result kept on the slab's own layers only;
  overlap 0 is time-slab block Jacobi.
* ``crank_nicolson_sweep``: a time-marching preconditioner built from the
  structure of Eq. 7's discretisation.  Row t of D_w22 tests against the hat
  function of time node t, which is the sum of its halves on the elements
  (t-1, t) and (t, t+1).  Testing each time element against a constant
  instead gives Crank-Nicolson: the block lower-bidiagonal
      B[t, t] = i M_s + (h_t/2) K_s,   B[t, t-1] = -i M_s + (h_t/2) K_s,
  with M_s the spatial mass matrix and K_s the spatial part of the operator
  (for a time-independent operator, D_w22[t, t+-1] = +-(i/2) M_s +
  (h_t/6) K_s on interior layers).  Averaging adjacent element rows,
  S = (I + U) / 2 (U the shift to the next layer; the last layer, whose test
  function is a half hat, keeps 1/2 only), reproduces the time-derivative
  terms of D_w22 exactly and its spatial terms up to (h_t/12) K_s times the
  second difference in time (and h_t/12 K_s (x_N - x_{N-1}) on the last
  layer).  The preconditioner is M = B^-1 S^-1: a backward sweep for S
  (s_{N-1} = 2 v_{N-1}, s_t = 2 v_t - s_{t+1}) and a forward Crank-Nicolson
  march for B (x_0 = Bd^-1 s_0, x_t = Bd^-1 (s_t - Bl x_{t-1})), one spatial
  solve with the LU factors of Bd per layer.

The unknown vector is ordered [t][z][y][x][c] (time slowest), so a time
layer is a contiguous run of ``per`` = n_spatial_nodes * NC entries and a
node a run of NC entries.

Only ``tests/`` imports this module.  Pinned by tests/test_oracle_precond.py:
each Jacobi / Schwarz preconditioner is the exact inverse of a matrix that
is block diagonal in its own blocks, and one slab covering all layers
inverts A; for the Crank-Nicolson sweep, the extracted M_s is the real
symmetric positive definite mass matrix (its entries sum to the domain
volume times NC), h_t K_s is Hermitian, S B agrees with D_w22 on every row but
the last for data linear in time, and M inverts S B.
"""

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
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


def crank_nicolson_sweep(A, nt, per):
    """(apply, S, B, M_s, h_t K_s): v -> B^-1 S^-1 v for a time-independent D_w22
    with ``nt`` >= 3 layers of ``per`` unknowns; M_s and K_s are taken from
    layer 1's couplings to layers 0 and 2."""
    A = A.tocsr()
    if nt < 3 or A.shape[0] != nt * per:
        raise ValueError("needs at least three time layers")

    def block(t, u):
        return A[t * per:(t + 1) * per, u * per:(u + 1) * per]

    up, down = block(1, 2), block(1, 0)
    Ms = (-1j * (up - down)).real.tocsr()                  # (i/2) M_s - (-(i/2) M_s) = i M_s
    htK = (3.0 * (up + down)).tocsr()                       # 2 (h_t/6) K_s * 3 = h_t K_s
    Bd = (1j * Ms + 0.5 * htK).tocsr()
    Bl = (-1j * Ms + 0.5 * htK).tocsr()
    # block (t, t) = Bd, block (t, t - 1) = Bl; S: block (t, t) = (t, t + 1) = I / 2
    lower = sp.eye(nt, k=-1, format="csr")
    B = (sp.kron(sp.eye(nt, format="csr"), Bd) + sp.kron(lower, Bl)).astype(np.complex128)
    S = (0.5 * sp.kron(sp.eye(nt, format="csr") + sp.eye(nt, k=1, format="csr"), sp.eye(per, format="csr")))
    B, S = B.tocsc(), S.astype(np.complex128).tocsc()
    # one factorisation of the layer matrix Bd serves every layer of the march
    if per <= 4096:
        lu = sla.lu_factor(Bd.toarray())
        solve_Bd = lambda r: sla.lu_solve(lu, r)                      # noqa: E731
    else:
        slu = spla.splu(Bd.tocsc())
        solve_Bd = slu.solve

    def apply(v):
        V = np.asarray(v, dtype=np.complex128).reshape(nt, per)
        s_ = np.empty_like(V)                         # S^-1: backward over the layers
        s_[-1] = 2.0 * V[-1]
        for t in range(nt - 2, -1, -1):
            s_[t] = 2.0 * V[t] - s_[t + 1]
        x = np.empty_like(V)                          # B^-1: the forward Crank-Nicolson march
        x[0] = solve_Bd(s_[0])
        for t in range(1, nt):
            x[t] = solve_Bd(s_[t] - Bl @ x[t - 1])
        return x.ravel()
    return apply, S, B, Ms, htK
