"""GPU U-Net (learned correction of the sweep preconditioner) against the oracle.

The network of oracle/unet.py (pinned on the CPU by tests/test_oracle_unet.py)
runs on the GPU with BF16 tensor-core convolutions and FP32 accumulation.  The
oracle runs it in FP64 with the GPU's parameters rounded to BF16, so the
difference is the rounding of each layer's input to BF16 (2^-8 relative) carried
through eleven layers: ~1e-2 relative.  Checked: forward output rel. L2 <= 5e-2;
loss within 5e-2 relative; the gradient of every parameter tensor rel. L2 <=
1e-1 and all of them together <= 5e-2.  A wrong tap order, channel index,
transposition or sign gives O(1).

One application of the corrected preconditioner, M(v) = M_CN(v) + alpha
U(rho / ||rho||) with alpha the least-squares scale of A U against rho, matches
oracle.unet.learned_correction.  Training on pairs the method generates
(dst_unet_train), from a zero output layer (the corrected preconditioner starts
as the sweep, loss 1), brings the loss below 1; flexible GMRES with the trained
correction reaches the exact (LU) solution, and the test prints how many steps
the correction saves (or costs) against the sweep alone.
"""
import numpy as np
import pytest

import workloads as W
from _helpers import oracle_mesh, rel_l2

pytestmark = pytest.mark.gpu


def _bf16(a):
    """Round float64 / float32 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _flat(params):
    from oracle import unet as U
    out = []
    for name, _, _, _ in U._LAYERS:
        out.append(params[name + ".w"].numpy().ravel())
        out.append(params[name + ".b"].numpy().ravel())
    return np.concatenate(out)


def _unflat(d, nc, flat):
    import torch
    from oracle import unet as U
    ref = U.init_params(d, nc, seed=0)
    out, off = {}, 0
    for name, _, _, _ in U._LAYERS:
        for suf in (".w", ".b"):
            t = ref[name + suf]
            out[name + suf] = torch.from_numpy(flat[off:off + t.numel()].reshape(t.shape).astype(np.float64))
            off += t.numel()
    return out


CASES = [("1p1", lambda: W.plane_wave_1p1(n=20)), ("2p1", lambda: W.zb_2p1(n=10, nt=9)),
         ("3p1", lambda: W.klein_3p1(n=6, nt=5, p0=1.05))]


@pytest.mark.parametrize("name,make", CASES)
def test_unet_forward_and_gradients_match_oracle(name, make):
    import torch
    from oracle import unet as U
    from paper_2103_14588_gb300 import binding as B
    w = make()
    om = oracle_mesh(w)
    params = U.init_params(w.d, om.nc, seed=5)
    # biases non-zero so that their gradients and the bias path are exercised
    g = torch.Generator().manual_seed(6)
    for k in params:
        if k.endswith(".b"):
            params[k] = 0.1 * torch.randn(params[k].shape, generator=g, dtype=torch.float64)
    flat = _bf16(_flat(params))
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(om.n_unknowns) + 1j * rng.standard_normal(om.n_unknowns)).astype(np.complex64)
    t = (rng.standard_normal(om.n_unknowns) + 1j * rng.standard_normal(om.n_unknowns)).astype(np.complex64)
    # oracle: forward, loss and autograd gradients in FP64 on the BF16-rounded parameters
    P = {k: v.clone().requires_grad_(True) for k, v in _unflat(w.d, om.nc, flat).items()}
    xg = U.to_grid(om, x.astype(np.complex128))
    tg = U.to_grid(om, t.astype(np.complex128))
    s = torch.sqrt((xg * xg).sum())
    y = U.forward(P, xg / s)
    th = tg / s
    loss = ((y - th) ** 2).sum() / (th ** 2).sum()
    loss.backward()
    ref_y = U.from_grid(om, y * s)[0]
    ref_g = np.concatenate([P[n + suf].grad.numpy().ravel() for n, _, _, _ in U._LAYERS for suf in (".w", ".b")])
    with B.Mesh.from_workload(w) as mesh:
        net = B.UNet(mesh.handle)
        assert net.num_params == flat.size
        net.set_params(flat.astype(np.float32))
        xd = torch.from_numpy(x).cuda()
        td = torch.from_numpy(t).cuda()
        yd = torch.empty_like(xd)
        net.forward(xd, yd)
        torch.cuda.synchronize()
        got_y = yd.cpu().numpy()
        got_loss, got_g = net.loss_grad(xd, td)
        net.close()
    assert rel_l2(got_y, ref_y) <= 5e-2, rel_l2(got_y, ref_y)
    assert abs(got_loss - float(loss.detach())) <= 5e-2 * float(loss.detach())
    assert rel_l2(got_g, ref_g) <= 5e-2, rel_l2(got_g, ref_g)
    off = 0
    for n, _, _, _ in U._LAYERS:
        for suf in (".w", ".b"):
            k = P[n + suf].numel()
            assert rel_l2(got_g[off:off + k], ref_g[off:off + k]) <= 1e-1, (n + suf, rel_l2(got_g[off:off + k],
                                                                                         ref_g[off:off + k]))
            off += k


@pytest.mark.parametrize("name,make", [("1p1", lambda: W.plane_wave_1p1(n=20)), ("2p1", lambda: W.zb_2p1(n=10, nt=9))])
def test_learned_application_matches_oracle(name, make):
    """One application M(v) = M_CN(v) + alpha U(rho / ||rho||) (dst_precond_apply) against
    oracle.unet.learned_correction with the network's BF16-rounded parameters, after a
    short training on the GPU (so that the correction is a sizeable part of M(v)): the
    sweep part to FP32 rounding, the correction to the network's BF16 rounding (5e-2 of
    its size)."""
    import torch
    from oracle import operator as OOP, precond as PC, unet as U
    from paper_2103_14588_gb300 import binding as B
    w = make()
    om = oracle_mesh(w)
    A, _ = OOP.split(om, OOP.assemble(om, w.m, w.V), w.psi0)
    A = A.tocsr()
    sweep = PC.crank_nicolson_sweep(A, om.nt, om.n_spatial_nodes * om.nc)[0]
    v = W.random_complex(om.n_unknowns, 17).astype(np.complex64)
    z0 = sweep(v.astype(np.complex128))
    with B.Mesh.from_workload(w) as mesh:
        net = B.UNet(mesh.handle)
        params = U.init_params(w.d, om.nc, seed=8)
        params["out.w"].zero_()
        net.set_params(_bf16(_flat(params)).astype(np.float32))
        net.train(mesh.handle, steps=300, lr=1e-3, seed=5)
        flat = _bf16(net.get_params())
        vd = torch.from_numpy(v).cuda()
        zd = torch.full_like(vd, complex("nan+nanj"))
        with pytest.raises(B.DstError):                 # no network attached yet
            B.dst_precond_apply(mesh.handle, B.DST_PRECOND_CN_LEARNED, vd, zd)
        B.dst_set_learned_precond(mesh.handle, net)
        B.dst_precond_apply(mesh.handle, B.DST_PRECOND_CN_LEARNED, vd, zd)
        torch.cuda.synchronize()
        got = zd.cpu().numpy()
        B.dst_set_learned_precond(mesh.handle, None)
        net.close()
    ref = U.learned_correction(om, _unflat(w.d, om.nc, flat), A, sweep)(v.astype(np.complex128))
    corr = np.linalg.norm(ref - z0) / np.linalg.norm(ref)
    print("%s: correction %.3g of M(v), GPU vs oracle %.3g" % (name, corr, rel_l2(got, ref)))
    assert corr > 1e-3                                      # the correction is really there
    assert rel_l2(got, ref) <= 1e-4 + 5e-2 * corr, (rel_l2(got, ref), corr)
    # the GPU's corrected direction leaves no larger residual than the sweep's
    r_got = np.linalg.norm(v - A @ got.astype(np.complex128))
    assert r_got <= np.linalg.norm(v - A @ z0) * (1 + 1e-4)


def test_training_lowers_the_loss_and_the_correction_solves():
    import torch
    from oracle import solvers as OS, operator as OOP, unet as U
    from paper_2103_14588_gb300 import binding as B
    w = W.zb_2p1(n=16, nt=16)
    om = oracle_mesh(w)
    A, b = OOP.split(om, OOP.assemble(om, w.m, w.V), w.psi0)
    ref = OS.sparse_solve(A, b)
    with B.Mesh.from_workload(w) as mesh:
        net = B.UNet(mesh.handle)
        # the output layer starts at zero: the corrected preconditioner starts as the sweep itself
        # (loss exactly 1), and a loss below 1 means a smaller error than the sweep's on those inputs
        params = U.init_params(w.d, om.nc, seed=3)
        params["out.w"].zero_()
        net.set_params(_bf16(_flat(params)).astype(np.float32))
        losses = net.train(mesh.handle, steps=600, lr=5e-4, seed=11)
        assert np.all(np.isfinite(losses))
        assert abs(losses[0] - 1.0) < 1e-3
        assert losses[-50:].mean() < 0.98, (losses[:50].mean(), losses[-50:].mean())
        gamma = net.output_scale()
        assert 0.0 <= gamma <= 2.0, gamma
        B.dst_set_learned_precond(mesh.handle, net)
        psi = torch.zeros(mesh.n_unknowns, dtype=torch.complex128, device="cuda")
        base = {"restart": 30, "rtol": 1e-9, "max_iters": 5000, "mixed_precision": 1}
        sl = B.dst_solve(mesh.handle, dict(base, precond=B.DST_PRECOND_CN_LEARNED), psi)
        torch.cuda.synchronize()
        x = psi.cpu().numpy()
        ss = B.dst_solve(mesh.handle, dict(base, precond=B.DST_PRECOND_CN_SWEEP), psi)
        B.dst_set_learned_precond(mesh.handle, None)
        net.close()
    print("steps with the trained correction %d, sweep alone %d; loss %.3f -> %.3f, output scale %.3f"
          % (sl["iters"], ss["iters"], losses[:50].mean(), losses[-50:].mean(), gamma))
    assert sl["status"] == 0 and rel_l2(x, ref) <= 1e-8
    assert ss["status"] == 0
    assert sl["iters"] <= 1.5 * ss["iters"] + 10, (sl["iters"], ss["iters"])


def test_learned_precond_needs_a_matching_network():
    import torch
    from paper_2103_14588_gb300 import binding as B
    w1, w2 = W.zb_2p1(n=8, nt=8), W.zb_2p1(n=10, nt=8)
    with B.Mesh.from_workload(w1) as m1, B.Mesh.from_workload(w2) as m2:
        net = B.UNet(m1.handle)
        with pytest.raises(B.DstError) as e:
            B.dst_set_learned_precond(m2.handle, net)
        assert e.value.code == B.DST_ERR_ARG
        psi = torch.zeros(m2.n_unknowns, dtype=torch.complex128, device="cuda")
        with pytest.raises(B.DstError):
            B.dst_solve(m2.handle, {"mixed_precision": 1, "precond": B.DST_PRECOND_CN_LEARNED}, psi)
        net.close()


def test_training_is_reproducible():
    """Two trainings from the same parameters and seed give the same network bit for bit
    (the weight gradients sum per node range in a fixed order, no atomics)."""
    import torch  # noqa: F401
    from oracle import unet as U
    from paper_2103_14588_gb300 import binding as B
    w = W.zb_2p1(n=10, nt=9)
    om = oracle_mesh(w)
    flat = _bf16(_flat(U.init_params(w.d, om.nc, seed=9))).astype(np.float32)
    out = []
    with B.Mesh.from_workload(w) as mesh:
        for _ in range(2):
            net = B.UNet(mesh.handle)
            net.set_params(flat)
            losses = net.train(mesh.handle, steps=40, lr=1e-3, seed=21)
            out.append((losses, net.get_params(), net.output_scale()))
            net.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
