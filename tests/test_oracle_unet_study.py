"""A learned right preconditioner (the oracle's U-Net) in flexible GMRES,
studied on the CPU: the measurement behind not building its GPU kernels yet.

On the 32 x 32 plane-wave system (397 unpreconditioned GMRES(30) steps to
1e-8) the network is trained with Adam to minimise ||A M(r) - r||^2 / ||r||^2
over the Arnoldi vectors of the unpreconditioned solve, the very inputs
FGMRES hands to M.  It learns a real approximate inverse: the loss falls from
~1 (the best multiple of the identity gets 0.9995) to below 0.3 (0.064 after
1500 steps).  Yet FGMRES(30) with it drops the residual ~10x within a few
steps and then stagnates (0.09 after 3000 steps; alternating the network
with the identity in the flexible basis: 0.04), where plain GMRES(30)
converges.  Trained on random residuals instead, the same holds (loss 0.12,
FGMRES at 0.08 after 3000 steps).
"""
import numpy as np
import pytest
import torch

import workloads as W
from _helpers import oracle_mesh
from oracle import operator as OP, solvers as SO, unet as U


def _sparse(M):
    C = M.tocoo()
    return torch.sparse_coo_tensor(np.vstack([C.row, C.col]), C.data, M.shape, dtype=torch.float64).coalesce()


def test_unet_preconditioner_stagnates():
    w = W.plane_wave_1p1(n=32)
    me = oracle_mesh(w)
    A, b = OP.split(me, OP.assemble(me, w.m, w.V), w.psi0)
    A = A.tocsr()
    nc = me.nc
    seen = []
    plain = SO.fgmres(lambda v: A @ v, b, lambda v: (seen.append(v.copy()), v)[1], restart=30, rtol=1e-8,
                      maxiter=3000)
    assert plain.converged and 350 < plain.iters < 450
    K = np.array(seen)
    AK = (A @ K.T).T
    alpha = np.vdot(AK.ravel(), K.ravel()) / np.vdot(AK.ravel(), AK.ravel())
    assert np.mean(np.linalg.norm(alpha * AK - K, axis=1) ** 2) > 0.99      # no scaled identity helps

    ReA, ImA = _sparse(A.real), _sparse(A.imag)

    def split(g):                                  # grid batch -> (Re, Im) as (n, B)
        a = g.movedim(1, -1).reshape(g.shape[0], -1, nc, 2)
        return a[..., 0].reshape(g.shape[0], -1).T, a[..., 1].reshape(g.shape[0], -1).T

    def loss_of(params, r):
        zr, zi = split(U.apply(params, r))
        rr, ri = split(r)
        Azr = torch.sparse.mm(ReA, zr) - torch.sparse.mm(ImA, zi)
        Azi = torch.sparse.mm(ImA, zr) + torch.sparse.mm(ReA, zi)
        return (((Azr - rr) ** 2 + (Azi - ri) ** 2).sum(0) / (rr ** 2 + ri ** 2).sum(0)).mean()

    KG = U.to_grid(me, K)
    params = U.init_params(1, nc, seed=1)
    for p in params.values():
        p.requires_grad_(True)
    opt = torch.optim.Adam(params.values(), lr=2e-3)
    rng = np.random.default_rng(0)
    for _ in range(400):
        loss = loss_of(params, KG[rng.integers(0, K.shape[0], 16)])
        opt.zero_grad()
        loss.backward()
        opt.step()
    trained = {k: v.detach() for k, v in params.items()}
    with torch.no_grad():
        assert float(loss_of(trained, KG)) < 0.3

    f = SO.fgmres(lambda v: A @ v, b, U.preconditioner(me, trained), restart=30, rtol=1e-8, maxiter=600)
    assert not f.converged
    assert min(f.history[:10]) < 0.5                 # a fast first drop ...
    assert f.rel_resid_true > 1e-3                   # ... then stagnation far above 1e-8
