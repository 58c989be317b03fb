"""Pins for oracle.solvers: GMRES against dense LU, restarts, breakdown, caps."""
import numpy as np
import pytest

from oracle import mesh as M, operator as OP, solvers as SO


def _system(d=1, nel=(6, 3, 2), nt=5, bc=M.PERIODIC, seed=1):
    rng = np.random.default_rng(seed)
    me = M.Mesh(d, [nel[0], nel[1], nel[2], nt], [0, 0, 0, 0], [1.0, 1.0, 1.0, 0.5], [bc] * 3)
    psi0 = rng.standard_normal(me.spatial_shape) + 1j * rng.standard_normal(me.spatial_shape)
    V = rng.uniform(0, 1, me.nel[0] * me.nel[1] * me.nel[2])
    A22, b = OP.split(me, OP.assemble(me, 1.0, V), psi0)
    return me, A22, b


@pytest.mark.parametrize("d", [1, 2, 3])
def test_full_gmres_equals_lu(d):
    me, A, b = _system(d=d, nel=(4, 3, 2), nt=3)
    n = b.size
    x_lu = SO.dense_solve(A, b)
    r = SO.gmres(lambda v: A @ v, b, restart=n, rtol=1e-13, maxiter=n)
    assert r.converged
    assert np.linalg.norm(r.x - x_lu) / np.linalg.norm(x_lu) < 1e-11


def test_restarted_gmres_equals_lu():
    me, A, b = _system(d=1, nel=(16, 1, 1), nt=12)
    x_lu = SO.dense_solve(A, b)
    r = SO.gmres(lambda v: A @ v, b, restart=10, rtol=1e-13, maxiter=20000)
    assert r.converged and r.restarts > 1
    assert np.linalg.norm(r.x - x_lu) / np.linalg.norm(x_lu) < 1e-10
    assert r.rel_resid_true <= 1e-13
    assert abs(r.history[-1] - r.rel_resid_true) < 1e-12


def test_gmres_lucky_breakdown():
    # b in a 3-dimensional invariant subspace: exact solution after 3 steps
    A = np.diag([1.0, 2.0, 3.0, 4.0, 5.0]).astype(complex)
    b = np.array([1.0, 1.0, 1.0, 0, 0], dtype=complex)
    r = SO.gmres(lambda v: A @ v, b, restart=5, rtol=1e-15)
    assert r.breakdown and r.iters == 3
    assert np.allclose(r.x, [1, 0.5, 1 / 3, 0, 0])


def test_gmres_maxiter_reports_not_converged():
    me, A, b = _system(d=1, nel=(16, 1, 1), nt=12)
    r = SO.gmres(lambda v: A @ v, b, restart=5, rtol=1e-14, maxiter=7)
    assert not r.converged and r.iters == 7
    # history is non-increasing within a cycle (GMRES minimises the residual)
    h = r.history[:5]
    assert all(h[i + 1] <= h[i] + 1e-15 for i in range(len(h) - 1))


def test_gmres_zero_rhs():
    r = SO.gmres(lambda v: v, np.zeros(4, dtype=complex))
    assert r.converged and r.iters == 0 and np.all(r.x == 0)


def test_givens_zeroes_second_entry():
    for a, b in [(1 + 2j, 0.5), (0, 2.0), (3 - 1j, 0.0), (1e-300 + 0j, 1.0)]:
        c, s = SO.givens(a, b)
        assert abs(-np.conj(s) * a + c * b) < 1e-15 * max(abs(a), abs(b), 1)
        assert abs(c * c + abs(s) ** 2 - 1) < 1e-15


@pytest.mark.parametrize("d", [1, 2, 3])
def test_bicgstab_equals_lu(d):
    me, A, b = _system(d=d, nel=(10, 4, 3), nt=6)
    x_lu = SO.dense_solve(A, b)
    x, it, rel, ok = SO.bicgstab(lambda v: A @ v, b, rtol=1e-13, maxiter=20000)
    assert ok and rel <= 1e-13 and it > 3
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-10


# ---- flexible GMRES ------------------------------------------------------------

def test_fgmres_identity_is_gmres():
    me, A, b = _system(d=2, nel=(6, 5, 1), nt=4)
    Aop = lambda v: A @ v
    g = SO.gmres(Aop, b, restart=7, rtol=1e-12, maxiter=5000)
    f = SO.fgmres(Aop, b, None, restart=7, rtol=1e-12, maxiter=5000)
    assert f.iters == g.iters and f.restarts == g.restarts
    assert np.array_equal(f.x, g.x) and f.history == g.history


def test_fgmres_exact_inverse_one_step():
    me, A, b = _system(d=1, nel=(12, 1, 1), nt=6)
    x_lu = SO.dense_solve(A, b)
    f = SO.fgmres(lambda v: A @ v, b, lambda v: SO.dense_solve(A, v), restart=30, rtol=1e-12)
    assert f.iters == 1 and f.converged
    assert np.linalg.norm(f.x - x_lu) / np.linalg.norm(x_lu) < 1e-12


def test_fgmres_fixed_preconditioner_is_right_preconditioned_gmres():
    """x = M u with u the GMRES solution of (A M) u = b, M a fixed matrix."""
    me, A, b = _system(d=1, nel=(14, 1, 1), nt=7, seed=3)
    n = b.size
    rng = np.random.default_rng(4)
    Mm = np.eye(n) + 0.1 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    for k in (1, 4, 20):                   # k steps of one cycle: the same Krylov space M K_k(A M, b)
        f = SO.fgmres(lambda v: A @ v, b, lambda v: Mm @ v, restart=k, rtol=1e-15, maxiter=k)
        g = SO.gmres(lambda v: A @ (Mm @ v), b, restart=k, rtol=1e-15, maxiter=k)
        assert f.iters == g.iters == k
        np.testing.assert_allclose(f.history, g.history, rtol=1e-10)
        assert np.linalg.norm(f.x - Mm @ g.x) / np.linalg.norm(f.x) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_fgmres_varying_preconditioner_residual_identity(k):
    """A preconditioner that differs at every call (alternating diagonal scalings and
    a damped nonlinear map): after k steps of one cycle the implicit residual
    |g_{k+1}| / ||b|| equals the true residual of x_0 + Z_k y_k."""
    me, A, b = _system(d=1, nel=(10, 1, 1), nt=5, seed=5)
    rng = np.random.default_rng(6)
    D1 = rng.uniform(0.5, 2.0, b.size)
    D2 = rng.uniform(0.5, 2.0, b.size)
    calls = [0]

    def M(v):
        calls[0] += 1
        if calls[0] % 3 == 0:
            return v + 0.1 * np.tanh(np.abs(v)) * v
        return (D1 if calls[0] % 3 == 1 else D2) * v

    f = SO.fgmres(lambda v: A @ v, b, M, restart=k, rtol=1e-14, maxiter=k)
    assert f.iters == k and calls[0] == k
    assert abs(f.history[-1] - f.rel_resid_true) <= 1e-12 * max(1.0, f.rel_resid_true)
    h = f.history
    assert all(h[i + 1] <= h[i] + 1e-15 for i in range(len(h) - 1))


def test_fgmres_varying_preconditioner_converges_to_lu():
    me, A, b = _system(d=1, nel=(16, 1, 1), nt=12, seed=7)
    x_lu = SO.dense_solve(A, b)
    rng = np.random.default_rng(8)
    D = [rng.uniform(0.5, 2.0, b.size) for _ in range(4)]
    calls = [0]

    def M(v):
        calls[0] += 1
        return D[calls[0] % 4] * v

    f = SO.fgmres(lambda v: A @ v, b, M, restart=10, rtol=1e-12, maxiter=20000)
    assert f.converged and f.rel_resid_true <= 1e-12
    assert np.linalg.norm(f.x - x_lu) / np.linalg.norm(x_lu) < 1e-9


def test_iteration_count_generator_agrees_with_the_assembled_solve():
    """oracle/iteration_counts.py counts GMRES(30) steps through the matrix-free
    apply and right-hand side; on the 64 x 64 plane wave that route and the
    assembled D_w22 both converge, in step counts a few percent apart (994 and
    978): over ~1000 restarted steps the summation order alone moves the count."""
    import workloads as W
    from oracle import iteration_counts as IC
    rec = IC.count("plane_wave_1p1")
    w = W.plane_wave_1p1()
    me = M.Mesh(w.d, w.n_el, w.lo, w.hi, w.bc)
    A, b = OP.split(me, OP.assemble(me, w.m, w.V), w.psi0)
    ref = SO.gmres(lambda v: A @ v, b, restart=IC.RESTART, rtol=IC.RTOL, maxiter=20000)
    assert rec["converged"] and ref.converged and rec["restart"] == 30 and rec["rtol"] == 1e-8
    assert abs(rec["iters"] - ref.iters) <= 0.03 * ref.iters and rec["rel_resid_true"] <= 1e-8
