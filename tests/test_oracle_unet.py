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
