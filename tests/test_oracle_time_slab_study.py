"""Time-slab Schwarz preconditioning (the time-additive Schwarz idea the paper's
conclusion proposes), studied on the CPU with the oracle's assembly.

Right-preconditioned restarted GMRES(30) on the 32 x 32 plane-wave system, with
slab solves done exactly by sparse LU: thin slabs (one time layer) stall, wide
slabs converge in a handful of steps.  This is the measurement behind the
decision not to build a GPU version: thin slabs do not precondition, and a wide
slab is itself a hard inner solve.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from _helpers import oracle_mesh


def _gmres_right(Aop, b, M, m=30, rtol=1e-8, maxit=600):
    """Right-preconditioned GMRES(m) (flexible form: the preconditioned directions
    are kept); returns (steps, true relative residual)."""
    n = b.size
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    it = 0
    while it < maxit:
        r = b - Aop(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * bn:
            break
        V = np.zeros((n, m + 1), complex)
        Z = np.zeros((n, m), complex)
        H = np.zeros((m + 1, m), complex)
        V[:, 0] = r / beta
        k = 0
        y = np.zeros(0, complex)
        for j in range(m):
            Z[:, j] = M(V[:, j])
            w = Aop(Z[:, j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[:, i], w)
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            V[:, j + 1] = w / H[j + 1, j]
            it += 1
            k = j + 1
            e1 = np.zeros(k + 1, complex)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)
            if np.linalg.norm(H[:k + 1, :k] @ y - e1) <= rtol * bn or it >= maxit:
                break
        x = x + Z[:, :k] @ y
    return it, np.linalg.norm(b - Aop(x)) / bn


def _slab_preconditioner(A, nt, per, S, overlap):
    """Restricted additive Schwarz over time slabs of S layers (+ overlap layers each side)."""
    blocks = []
    for s0 in range(0, nt, S):
        lo, hi = max(0, s0 - overlap) * per, min(nt, s0 + S + overlap) * per
        own = (s0 * per - lo, min(nt, s0 + S) * per - lo)
        blocks.append((lo, hi, own, spla.splu(A[lo:hi, lo:hi].tocsc())))

    def apply(v):
        z = np.zeros_like(v)
        for lo, hi, own, lu in blocks:
            zz = lu.solve(v[lo:hi])
            z[lo + own[0]: lo + own[1]] = zz[own[0]:own[1]]
        return z
    return apply


@pytest.fixture(scope="module")
def system():
    from oracle import operator as OP
    w = W.plane_wave_1p1(n=32)
    om = oracle_mesh(w)
    A, b = OP.split(om, OP.assemble(om, w.m, w.V), w.psi0)
    A = A.tocsr()
    return A, b, 32, b.size // 32


def test_time_slab_schwarz(system):
    A, b, nt, per = system
    it0, r0 = _gmres_right(lambda v: A @ v, b, lambda v: v)
    assert r0 <= 1e-8 and 350 < it0 < 450                      # 397 steps unpreconditioned
    # one layer per slab: no preconditioning, the iteration stalls
    it1, r1 = _gmres_right(lambda v: A @ v, b, _slab_preconditioner(A, nt, per, 1, 0), maxit=300)
    assert r1 > 1e-3
    # wide slabs converge in a handful of steps (two 16-layer slabs; 8 layers with overlap 1)
    it16, r16 = _gmres_right(lambda v: A @ v, b, _slab_preconditioner(A, nt, per, 16, 0))
    assert r16 <= 1e-8 and it16 <= 10
    it8, r8 = _gmres_right(lambda v: A @ v, b, _slab_preconditioner(A, nt, per, 8, 1))
    assert r8 <= 1e-8 and it8 <= 40
