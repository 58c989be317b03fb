"""Pins of the oracle's non-learned preconditioners.

Each is the exact inverse of a matrix that is block diagonal in its own blocks:
the node blocks for block Jacobi, the (overlap-extended) time slabs for the
Schwarz method.  Such matrices are built here by masking the assembled D_w22
by block index, so a wrong block size, a slab offset off by a layer or a
restriction that keeps the overlap fails.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import mesh as M, operator as OP, precond as PC, solvers as SO


def _system(d, nel, nt, bc, seed):
    rng = np.random.default_rng(seed)
    me = M.Mesh(d, list(nel) + [nt], [0, 0, 0, 0], [1.0, 1.0, 1.0, 0.5], bc)
    psi0 = rng.standard_normal(me.spatial_shape) + 1j * rng.standard_normal(me.spatial_shape)
    V = rng.uniform(0, 1, me.nel[0] * me.nel[1] * me.nel[2])
    A, b = OP.split(me, OP.assemble(me, 1.0, V), psi0)
    return me, A.tocsr(), b


def _mask(A, block_of):
    """Keep the entries (i, j) of A with block_of[i] == block_of[j]."""
    C = A.tocoo()
    keep = block_of[C.row] == block_of[C.col]
    return sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=A.shape)


@pytest.mark.parametrize("d,nel,bc", [(1, (9, 1, 1), [M.OPEN]), (2, (5, 4, 1), [M.PERIODIC, M.DIRICHLET]),
                                      (3, (3, 3, 2), [M.PERIODIC, M.OPEN, M.PERIODIC])])
def test_node_block_jacobi_inverts_node_block_diagonal(d, nel, bc):
    me, A, b = _system(d, nel, 3, bc, seed=d)
    n = A.shape[0]
    node = np.arange(n) // me.nc
    Abd = _mask(A, node)
    Mj = PC.node_block_jacobi(me.nc, A)
    v = np.random.default_rng(9).standard_normal(n) + 0j
    np.testing.assert_allclose(Mj(Abd @ v), v, rtol=0, atol=1e-11 * np.abs(v).max())
    # the blocks are the diagonal ones: off-block entries of A do not enter
    Mbd = PC.node_block_jacobi(me.nc, Abd)
    np.testing.assert_array_equal(Mj(b), Mbd(b))


@pytest.mark.parametrize("S,overlap", [(1, 0), (2, 0), (3, 1), (4, 2), (7, 0)])
def test_time_slab_schwarz_inverts_slab_block_diagonal(S, overlap):
    nt = 7
    me, A, b = _system(2, (4, 3, 1), nt, [M.PERIODIC, M.OPEN], seed=11)
    per = me.n_spatial_nodes * me.nc
    slab = (np.arange(A.shape[0]) // per) // S
    Abd = _mask(A, slab)
    Ms = PC.time_slab_schwarz(Abd, nt, per, S, overlap)
    v = np.random.default_rng(12).standard_normal(A.shape[0]) + 1j
    np.testing.assert_allclose(Ms(Abd @ v), v, rtol=0, atol=1e-10 * np.abs(v).max())


def test_one_slab_is_the_exact_inverse():
    nt = 6
    me, A, b = _system(1, (10, 1, 1), nt, [M.DIRICHLET], seed=13)
    per = me.n_spatial_nodes * me.nc
    x_lu = SO.dense_solve(A, b)
    Ms = PC.time_slab_schwarz(A, nt, per, nt, 0)
    np.testing.assert_allclose(Ms(b), x_lu, rtol=1e-11, atol=1e-13)
    f = SO.fgmres(lambda v: A @ v, b, Ms, restart=30, rtol=1e-12)
    assert f.iters == 1 and f.converged


def test_bad_layouts_rejected():
    me, A, b = _system(1, (6, 1, 1), 4, [M.PERIODIC], seed=1)
    with pytest.raises(ValueError):
        PC.time_slab_schwarz(A, 5, A.shape[0] // 4, 2)
    with pytest.raises(ValueError):
        PC.node_block_jacobi(5, A[:-1, :-1])


# ---- Crank-Nicolson sweep ------------------------------------------------------

def _open_end_nodes(me):
    """Boolean per unknown entry: the node lies at an end of an open axis."""
    idx = np.indices((me.nu[2], me.nu[1], me.nu[0]))          # z, y, x
    end = np.zeros(idx.shape[1:], dtype=bool)
    for k in range(me.d):
        if me.bc[k] == M.OPEN:
            i = idx[2 - k]
            end |= (i == 0) | (i == me.nu[k] - 1)
    return np.repeat(end.ravel(), me.nc)


@pytest.mark.parametrize("d,nel,bc", [(1, (12, 1, 1), [M.PERIODIC]), (2, (5, 4, 1), [M.OPEN, M.PERIODIC]),
                                      (2, (6, 4, 1), [M.DIRICHLET, M.PERIODIC]),
                                      (3, (3, 4, 3), [M.PERIODIC, M.PERIODIC, M.OPEN])])
def test_crank_nicolson_sweep_blocks(d, nel, bc):
    nt = 5
    me, A, b = _system(d, nel, nt, bc, seed=20 + d)
    per = me.n_spatial_nodes * me.nc
    Mc, S, B, Ms, htK = PC.crank_nicolson_sweep(A, nt, per)
    # the mass matrix: real symmetric positive definite, entries summing to the volume per component
    Md = Ms.toarray()
    np.testing.assert_allclose(Md, Md.T, rtol=0, atol=1e-15)
    assert np.linalg.eigvalsh(Md).min() > 0
    if M.DIRICHLET not in bc:                    # the unknown hats sum to one on the whole domain
        vol = np.prod([me.hi[k] - me.lo[k] for k in range(d)])
        assert Md.sum() == pytest.approx(vol * me.nc, rel=1e-12)
    # the spatial part is Hermitian but for the outflow term of open axes, which
    # couples end nodes only
    Kd = htK.toarray()
    end = _open_end_nodes(me)
    skew = np.abs(Kd - Kd.conj().T)
    assert skew[~end, :].max(initial=0) <= 1e-14 and skew[:, ~end].max(initial=0) <= 1e-14
    assert (skew.max() > 1e-6) == (M.OPEN in bc)
    # data linear in time: S B equals D_w22 except on the last layer, where the
    # difference is (h_t / 12) K_s times the step c
    rng = np.random.default_rng(d)
    c = rng.standard_normal(per) + 1j * rng.standard_normal(per)
    x = np.concatenate([(t + 1) * c for t in range(nt)])
    diff = A @ x - S @ (B @ x)
    assert np.abs(diff[:-per]).max() <= 1e-12 * np.abs(A @ x).max()
    np.testing.assert_allclose(diff[-per:], htK @ c / 12, rtol=1e-10, atol=1e-13)
    # the preconditioner inverts S B (backward sweep for S, then the forward march)
    y = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    np.testing.assert_allclose(S @ (B @ Mc(y)), y, rtol=0, atol=1e-10 * np.abs(y).max())


def test_crank_nicolson_sweep_needs_three_layers():
    me, A, b = _system(1, (6, 1, 1), 2, [M.PERIODIC], seed=1)
    with pytest.raises(ValueError):
        PC.crank_nicolson_sweep(A, 2, A.shape[0] // 2)


@pytest.mark.parametrize("d,nel,V", [(1, (16, 1, 1), 0.0), (2, (8, 6, 1), 0.7)])
def test_crank_nicolson_sweep_is_one_scan_per_frequency_on_periodic_meshes(d, nel, V):
    """Periodic axes and a constant potential make M_s and K_s block circulant, so
    the spatial FFT turns the sweep into an independent scan over t per frequency:
    x^_t = (i M^ + (h_t/2) K^)^-1 (s^_t - (-i M^ + (h_t/2) K^) x^_{t-1}) after the
    backward scan s_t = 2 v_t - s_{t+1} (s_N = 2 v_N).  Written here from those
    recurrences alone and compared with the oracle's sparse-LU sweep."""
    nt = 6
    rng = np.random.default_rng(30 + d)
    me = M.Mesh(d, list(nel) + [nt], [0, 0, 0, 0], [1.0, 1.3, 1.0, 0.6], [M.PERIODIC] * 3)
    psi0 = rng.standard_normal(me.spatial_shape) + 1j * rng.standard_normal(me.spatial_shape)
    A, _ = OP.split(me, OP.assemble(me, 1.0, np.full(me.nel[0] * me.nel[1] * me.nel[2], V)), psi0)
    A = A.tocsr()
    nc, grid = me.nc, (me.nu[1], me.nu[0])                  # (n_y, n_x)
    per = me.n_spatial_nodes * nc
    Mc, S, B, Ms, htK = PC.crank_nicolson_sweep(A, nt, per)

    def symbol(op):
        """NC x NC symbol per frequency of a block-circulant layer operator: the FFT of
        its first block row, with the sign of a correlation (column offset j)."""
        row = op[:nc, :].toarray().reshape(nc, grid[0], grid[1], nc)   # [c_out, y, x, c_in]
        # (op u)_0 = sum_j row_j u_j; for u_j = e^{i k j} u this is sum_j row_j e^{i k j}
        return np.fft.ifft2(row, axes=(1, 2)).transpose(1, 2, 0, 3) * grid[0] * grid[1]

    Mh, Kh = symbol(Ms.tocsr()), symbol(htK.tocsr())
    Bd = 1j * Mh + 0.5 * Kh
    Bl = -1j * Mh + 0.5 * Kh
    v = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    vt = v.reshape(nt, grid[0], grid[1], nc)
    s = np.zeros_like(vt)
    s[-1] = 2 * vt[-1]
    for t in range(nt - 2, -1, -1):                           # S^-1: s_t = 2 v_t - s_{t+1}
        s[t] = 2 * vt[t] - s[t + 1]
    sh = np.fft.fft2(s, axes=(1, 2))
    xh = np.zeros_like(sh)
    for t in range(nt):                                       # B^-1: the forward march per frequency
        rhs = sh[t] - (np.einsum("yxab,yxb->yxa", Bl, xh[t - 1]) if t > 0 else 0)
        xh[t] = np.linalg.solve(Bd, rhs[..., None])[..., 0]
    x = np.fft.ifft2(xh, axes=(1, 2)).ravel()
    np.testing.assert_allclose(x, Mc(v), rtol=0, atol=1e-10 * np.abs(x).max())
