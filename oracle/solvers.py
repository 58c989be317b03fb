"""Linear solvers for A Psi_u = b (Algorithm 1 step 6).

* ``gmres``: restarted GMRES(m) of Saad & Schultz (1986), the Krylov solver
  the paper uses (Sec. 2.2, last paragraph): Arnoldi with modified
  Gram-Schmidt, complex Givens rotations on the Hessenberg matrix, the
  least-squares residual |g_{j+1}| as the stopping estimate, a true residual
  b - A x at every restart.  A new Arnoldi vector of norm below 1e-14 times
  ||A v_j|| ends the solve (lucky breakdown: the Krylov space is invariant).
  Unpreconditioned, x_0 = 0 unless given (the paper states neither restart
  length nor preconditioner: read as PETSc-like defaults, restart chosen by
  the caller).
* ``fgmres``: flexible GMRES(m) of Saad (1993, SIAM J. Sci. Comput. 14),
  right-preconditioned: each Arnoldi direction v_j is preconditioned to
  z_j = M_j(v_j) by a preconditioner that may change from step to step (a
  nonlinear one included), w = A z_j is orthogonalised against V, and the
  iterate is x_0 + Z_k y_k with y_k the least-squares solution of the same
  Hessenberg problem as GMRES.  The relation A Z_k = V_{k+1} Hbar_k keeps
  |g_{k+1}| equal to the true residual norm of that iterate.  The paper's
  conclusion asks for a preconditioner; this is the Krylov method for one.
* ``bicgstab``: van der Vorst's BiCGSTAB (1992), the other Krylov solver of
  Sec. 4.1's tables, in complex arithmetic (inner products conjugate the
  first argument), x_0 = 0 unless given, shadow residual = initial residual.
* ``dense_solve``: LU with partial pivoting (LAPACK getrf/getrs) of the
  assembled D_w22 - the exact discrete solution on tiny meshes.
* ``sparse_solve``: sparse LU (SuperLU) of the assembled D_w22 for the
  physics checks on medium meshes.

Pinned by tests/test_oracle_solvers.py: GMRES with restart >= n equals the
dense LU solution; restarted GMRES reaches the same solution; breakdown on an
exact Krylov solve; iteration cap status; BiCGSTAB reaches the LU solution;
FGMRES with the identity is GMRES, with the exact inverse converges in one
step, with a fixed linear M gives M times the GMRES solution of A M, and with
a preconditioner that changes every step its implicit residual equals the
true residual of x_0 + Z y.
"""

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


class GmresResult:
    def __init__(self, x, iters, restarts, converged, rel_resid_true, history, breakdown):
        self.x = x
        self.iters = iters
        self.restarts = restarts
        self.converged = converged
        self.rel_resid_true = rel_resid_true
        self.history = history          # implicit |g_{j+1}| / ||b|| after each iteration
        self.breakdown = breakdown


def givens(a, b):
    """Complex rotation (c real, s complex) with [[c, s], [-conj(s), c]] [a, b]^T = [r, 0]^T."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, 1.0 + 0.0j
    rho = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    c = abs(a) / rho
    s = (a / abs(a)) * np.conj(b) / rho
    return c, s


def gmres(A, b, x0=None, restart=30, rtol=1e-10, maxiter=100000):
    """Restarted GMRES(restart) for a callable A on complex vectors."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return GmresResult(np.zeros(n, dtype=np.complex128), 0, 0, True, 0.0, [], False)
    history = []
    total = 0
    restarts = 0
    breakdown = False
    m = restart
    r = b - A(x)
    beta = np.linalg.norm(r)
    while True:
        if beta <= rtol * bnorm or total >= maxiter:
            break
        V = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(m):
            w = A(V[j])
            wnorm0 = np.linalg.norm(w)
            total += 1
            for i in range(j + 1):                        # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            for i in range(j):                            # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if hn <= 1e-14 * wnorm0:                      # invariant subspace: exact solution
                breakdown = True
                break
            V[j + 1] = w / hn
            if abs(g[j + 1]) <= rtol * bnorm or total >= maxiter:
                break
        y = sla.solve_triangular(H[:k, :k], g[:k], lower=False)
        x = x + V[:k].T @ y
        restarts += 1
        r = b - A(x)
        beta = np.linalg.norm(r)
        if breakdown:
            break
    rel = beta / bnorm
    return GmresResult(x, total, restarts, rel <= rtol, rel, history, breakdown)


def fgmres(A, b, M=None, x0=None, restart=30, rtol=1e-10, maxiter=100000):
    """Flexible restarted GMRES(restart) for callables A and M (M None: identity).

    M is called once per Arnoldi step on the unit vector v_j and may return a
    different linear (or nonlinear) image each time."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return GmresResult(np.zeros(n, dtype=np.complex128), 0, 0, True, 0.0, [], False)
    if M is None:
        M = lambda v: v
    history = []
    total = 0
    restarts = 0
    breakdown = False
    m = restart
    r = b - A(x)
    beta = np.linalg.norm(r)
    while True:
        if beta <= rtol * bnorm or total >= maxiter:
            break
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(m):
            Z[j] = np.asarray(M(V[j]), dtype=np.complex128)
            w = A(Z[j])
            wnorm0 = np.linalg.norm(w)
            total += 1
            for i in range(j + 1):                        # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            for i in range(j):                            # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if hn <= 1e-14 * wnorm0:                      # A z_j lies in span(V): exact solution
                breakdown = True
                break
            V[j + 1] = w / hn
            if abs(g[j + 1]) <= rtol * bnorm or total >= maxiter:
                break
        y = sla.solve_triangular(H[:k, :k], g[:k], lower=False)
        x = x + Z[:k].T @ y
        restarts += 1
        r = b - A(x)
        beta = np.linalg.norm(r)
        if breakdown:
            break
    rel = beta / bnorm
    return GmresResult(x, total, restarts, rel <= rtol, rel, history, breakdown)


def bicgstab(A, b, x0=None, rtol=1e-10, maxiter=100000):
    """BiCGSTAB for a callable A; returns (x, iterations, rel. true residual, converged)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, True
    r = b - A(x)
    rhat = r.copy()
    rho = alpha = omega = 1.0 + 0.0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    while np.linalg.norm(r) > rtol * bnorm and it < maxiter:
        rho_new = np.vdot(rhat, r)
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
        v = A(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        t = A(s)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        it += 1
    rel = np.linalg.norm(b - A(x)) / bnorm
    return x, it, rel, rel <= rtol


def dense_solve(D22, b):
    """Exact discrete solution by LU with partial pivoting (dense)."""
    M = D22.toarray() if hasattr(D22, "toarray") else np.asarray(D22)
    lu, piv = sla.lu_factor(M)
    return sla.lu_solve((lu, piv), b)


def sparse_solve(D22, b):
    """Exact discrete solution by sparse LU (SuperLU)."""
    return spla.splu(D22.tocsc()).solve(np.asarray(b, dtype=np.complex128))
