"""Pins of the oracle's U-Net (the learned preconditioner's reference network).

* convolutions in 2, 3 and 4 axes against a brute-force loop over the
  definition y[o, p] = b[o] + sum_i sum_k w[o, i, k] x[i, p + k - K//2] (zero
  outside the grid), for kernels 3 and 1;
* pool and upsample are adjoint up to the block volume:
  <upsample(x), y> = 2^D <x, pool(y)>, on even and odd grid sizes;
* autograd gradients of the whole network, with respect to every weight and
  to the input, against central finite differences (torch.autograd.gradcheck);
* the grid layout (channel 2c = Re psi_c, 2c + 1 = Im psi_c, axes t, z, y, x)
  and the positive homogeneity M(a r) = a M(r), M(0) = 0.
"""
import itertools

import numpy as np
import pytest
import torch

from oracle import unet as U
from oracle.mesh import OPEN, PERIODIC, DIRICHLET, Mesh


def _brute_conv(x, w, b):
    B, Ci = x.shape[:2]
    Co, K = w.shape[0], w.shape[2:]
    grid = x.shape[2:]
    y = np.zeros((B, Co) + grid)
    for n, o in itertools.product(range(B), range(Co)):
        for p in itertools.product(*[range(g) for g in grid]):
            acc = b[o]
            for i in range(Ci):
                for k in itertools.product(*[range(kk) for kk in K]):
                    q = tuple(pp + kk - KK // 2 for pp, kk, KK in zip(p, k, K))
                    if all(0 <= qq < g for qq, g in zip(q, grid)):
                        acc += w[(o, i) + k] * x[(n, i) + q]
            y[(n, o) + p] = acc
    return y


@pytest.mark.parametrize("grid", [(3, 5), (4, 3, 5), (3, 2, 3, 4)])
@pytest.mark.parametrize("k", [3, 1])
def test_convolution_is_the_definition(grid, k):
    rng = np.random.default_rng(len(grid) * 10 + k)
    D = len(grid)
    x = rng.standard_normal((2, 2) + grid)
    w = rng.standard_normal((3, 2) + (k,) * D)
    b = rng.standard_normal(3)
    got = U.convnd(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b)).numpy()
    np.testing.assert_allclose(got, _brute_conv(x, w, b), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("grid", [(4, 6), (5, 3), (3, 4, 5), (2, 3, 3, 5)])
def test_pool_and_upsample_are_adjoint(grid):
    rng = np.random.default_rng(sum(grid))
    D = len(grid)
    y = torch.from_numpy(rng.standard_normal((2, 3) + grid))
    coarse = U.pool(y)
    assert coarse.shape[2:] == tuple((n + 1) // 2 for n in grid)
    x = torch.from_numpy(rng.standard_normal(coarse.shape))
    lhs = float((U.upsample(x, grid) * y).sum())
    rhs = float(2 ** D * (x * coarse).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # a field constant on 2-blocks survives pool followed by upsample
    even = tuple(2 * ((n + 1) // 2) for n in grid)
    c = torch.from_numpy(rng.standard_normal((1, 1) + tuple(n // 2 for n in even)))
    f = U.upsample(c, even)
    assert torch.equal(U.pool(f), c) and torch.equal(U.upsample(U.pool(f), even), f)


@pytest.mark.parametrize("d,grid", [(1, (5, 6)), (2, (4, 3, 5)), (3, (3, 2, 3, 2))])
def test_gradients_match_finite_differences(d, grid):
    nc = 2 if d < 3 else 4
    params = U.init_params(d, nc, seed=d, channels=(2, 3, 2))
    rng = np.random.default_rng(d)
    for k in params:                               # non-zero biases so they matter
        if k.endswith(".b"):
            params[k] = torch.from_numpy(0.1 * rng.standard_normal(params[k].shape))
    names = sorted(params)
    x = torch.from_numpy(rng.standard_normal((1, 2 * nc) + grid)).requires_grad_(True)
    leaves = [params[n].clone().requires_grad_(True) for n in names]

    def f(x, *ws):
        return U.apply(dict(zip(names, ws)), x)

    assert torch.autograd.gradcheck(f, (x, *leaves), eps=1e-6, atol=1e-6, rtol=1e-4)


def test_grid_layout_and_round_trip():
    me = Mesh(2, [4, 3, 1, 2], [0, 0, 0, 0], [1, 1, 1, 1], [OPEN, DIRICHLET])   # nu = (5, 2), nt = 2
    n = me.n_unknowns
    v = np.arange(n) * (1 + 0.5j)
    g = U.to_grid(me, v)
    assert tuple(g.shape) == (1, 4, 2, 2, 5)
    t, y, x, c = 1, 0, 3, 1
    idx = (((t * me.nu[2] + 0) * me.nu[1] + y) * me.nu[0] + x) * me.nc + c
    assert g[0, 2 * c, t, y, x] == v[idx].real and g[0, 2 * c + 1, t, y, x] == v[idx].imag
    np.testing.assert_array_equal(U.from_grid(me, g)[0], v)
    assert U.grid_shape(Mesh(3, [3, 4, 5, 2], [0] * 4, [1] * 4, [PERIODIC] * 3)) == (2, 5, 4, 3)


def test_homogeneity_and_zero():
    me = Mesh(1, [8, 1, 1, 4], [0, 0, 0, 0], [1, 1, 1, 1], [PERIODIC])
    M = U.preconditioner(me, U.init_params(1, 2, seed=3))
    rng = np.random.default_rng(3)
    r = rng.standard_normal(me.n_unknowns) + 1j * rng.standard_normal(me.n_unknowns)
    Mr = M(r)
    assert np.linalg.norm(Mr) > 0
    np.testing.assert_allclose(M(7.5 * r), 7.5 * Mr, rtol=1e-12, atol=1e-14)
    assert np.all(M(np.zeros_like(r)) == 0)


# ---- the learned correction of the sweep ------------------------------------------

def test_ls_scale_is_the_least_squares_solution():
    """rho = alpha* Au + (a part orthogonal to Au) gives back alpha* (complex, so a
    conjugate taken on the wrong side shows); the residual is orthogonal to Au;
    Au = 0 gives 0."""
    rng = np.random.default_rng(41)
    n = 57
    Au = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a_star = 0.7 - 1.3j
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    r_perp = r - (np.vdot(Au, r) / np.vdot(Au, Au)) * Au       # Gram-Schmidt of r against Au
    assert abs(np.vdot(Au, r_perp)) < 1e-12 * np.linalg.norm(Au) * np.linalg.norm(r)
    assert abs(U.ls_scale(Au, a_star * Au) - a_star) < 1e-14
    assert abs(U.ls_scale(Au, a_star * Au + r_perp) - a_star) < 1e-12
    alpha = U.ls_scale(Au, r)
    assert abs(np.vdot(Au, r - alpha * Au)) < 1e-12 * np.linalg.norm(Au) * np.linalg.norm(r)
    assert U.ls_scale(np.zeros(n, complex), r) == 0


def _sweep_system():
    from oracle import operator as OP, precond as PC
    rng = np.random.default_rng(12)
    me = Mesh(1, [12, 1, 1, 8], [0, 0, 0, 0], [4.0, 1.0, 1.0, 1.0], [PERIODIC])
    psi0 = rng.standard_normal(me.spatial_shape) + 1j * rng.standard_normal(me.spatial_shape)
    A, _ = OP.split(me, OP.assemble(me, 1.0, None), psi0)
    A = A.tocsr()
    return me, A, PC.crank_nicolson_sweep(A, me.nt, me.n_spatial_nodes * me.nc)[0]


def test_learned_correction_reduces_to_the_sweep_and_never_raises_the_residual():
    me, A, sweep = _sweep_system()
    rng = np.random.default_rng(13)
    v = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    z0 = sweep(v)
    params = U.init_params(me.d, me.nc, seed=4)
    zero_out = dict(params)
    zero_out["out.w"] = torch.zeros_like(params["out.w"])
    zero_out["out.b"] = torch.zeros_like(params["out.b"])
    assert np.array_equal(U.learned_correction(me, zero_out, A, sweep)(v), z0)
    z = U.learned_correction(me, params, A, sweep)(v)
    r0 = np.linalg.norm(v - A @ z0)
    r1 = np.linalg.norm(v - A @ z)
    assert not np.allclose(z, z0)
    assert r1 <= r0 * (1 + 1e-12)
    # the residual left is orthogonal to A u, u the correction's direction
    u = (z - z0)
    assert abs(np.vdot(A @ u, v - A @ z)) < 1e-10 * np.linalg.norm(A @ u) * r1
