"""Time-slab Schwarz preconditioning (the time-additive Schwarz idea the paper's
conclusion proposes), studied on the CPU with the oracle's assembly.

Right-preconditioned restarted GMRES(30) on the 32 x 32 plane-wave system, with
slab solves done exactly by sparse LU: thin slabs (one time layer) stall, wide
slabs converge in a handful of steps.  This is the measurement behind the
decision not to build a GPU version: thin slabs do not precondition, and a wide
slab is itself a hard inner solve.
"""
import pytest

import workloads as W
from _helpers import oracle_mesh
from oracle import precond as PC, solvers as SO


def _fgmres(A, b, M, maxit=600):
    """Right-preconditioned (flexible) GMRES(30) to 1e-8: (steps, true relative residual)."""
    r = SO.fgmres(lambda v: A @ v, b, M, restart=30, rtol=1e-8, maxiter=maxit)
    return r.iters, r.rel_resid_true


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
    it0, r0 = _fgmres(A, b, None)
    assert r0 <= 1e-8 and 350 < it0 < 450                      # 397 steps unpreconditioned
    # one layer per slab: no preconditioning, the iteration stalls
    it1, r1 = _fgmres(A, b, PC.time_slab_schwarz(A, nt, per, 1, 0), maxit=300)
    assert r1 > 1e-3
    # wide slabs converge in a handful of steps (two 16-layer slabs; 8 layers with overlap 1)
    it16, r16 = _fgmres(A, b, PC.time_slab_schwarz(A, nt, per, 16, 0))
    assert r16 <= 1e-8 and it16 <= 10
    it8, r8 = _fgmres(A, b, PC.time_slab_schwarz(A, nt, per, 8, 1))
    assert r8 <= 1e-8 and it8 <= 40
