"""Convolutional U-Net for a learned right preconditioner (test infrastructure).

The paper's conclusion (Sec. 5) asks for a preconditioner and specifies none; this is
a learned candidate for flexible GMRES: a network M that maps a residual r
(the unknown vector, layout [t][z][y][x][c]) to a correction close to
A^-1 r.  It has no counterpart in the paper; the definitions below are the
reference the GPU network is to be checked against.

Grid and channels.  The unknowns form a (D = d + 1)-dimensional grid
(t, [z], [y], x) of N_t x n_z x n_y x n_x nodes (only the axes the mesh has),
with C = 2 NC channels: channel 2c is Re psi_c, channel 2c + 1 is Im psi_c.

Network (every convolution has a bias; "conv3" has kernel 3 in each of the D
axes and zero padding that keeps the size, "conv1" has kernel 1):
  level 1:  conv3 C -> 16, ReLU, conv3 16 -> 16, ReLU                 (s1)
  level 2:  pool, conv3 16 -> 32, ReLU, conv3 32 -> 32, ReLU          (s2)
  level 3:  pool, conv3 32 -> 64, ReLU, conv3 64 -> 64, ReLU
  up 2:     upsample to s2's grid, conv1 64 -> 32, add s2, conv3 32 -> 32, ReLU
  up 1:     upsample to s1's grid, conv1 32 -> 16, add s1, conv3 16 -> 16, ReLU
  out:      conv1 16 -> C
pool = mean over blocks of 2 along every axis (a block cut by the end of an
axis counts the missing cells as zero, so the pooled grid has ceil(n/2)
cells); upsample = nearest neighbour (cell p takes coarse cell p // 2).  The
input is divided by its 2-norm and the output multiplied by it, so that
M(a r) = a M(r) for every a > 0 and M(0) = 0.

Arithmetic in float64 with torch CPU ops: conv2d / conv3d for D = 2, 3; for
D = 4 the convolution is, by its definition, the sum over the three time
offsets of 3D convolutions of the shifted time slices.  Gradients come from
torch autograd.

Correction of the Crank-Nicolson sweep (``learned_correction``): with
rho = v - A M_CN(v) and u = U(rho / ||rho||) (the network without the final
rescaling), M(v) = M_CN(v) + alpha u, alpha the complex least-squares scale
minimising ||rho - alpha A u|| (``ls_scale``), so that ||v - A M(v)|| never
exceeds ||v - A M_CN(v)||.

Only ``tests/`` imports this module.  Pinned by tests/test_oracle_unet.py:
convolutions against a brute-force loop over the definition, pool and
upsample as adjoint pairs, autograd gradients against finite differences,
the homogeneity and the grid layout; the least-squares scale against exact
solutions and its normal equation, and the correction reducing to the sweep
for a zero output layer and never raising the residual.
"""

import math

import numpy as np
import torch
import torch.nn.functional as F

CHANNELS = (16, 32, 64)

# (name, input channels, output channels, kernel) for each convolution, in
# forward order; "C" stands for the 2 NC field channels
_LAYERS = [("e1a", "C", 0, 3), ("e1b", 0, 0, 3),
           ("e2a", 0, 1, 3), ("e2b", 1, 1, 3),
           ("e3a", 1, 2, 3), ("e3b", 2, 2, 3),
           ("u2p", 2, 1, 1), ("u2c", 1, 1, 3),
           ("u1p", 1, 0, 1), ("u1c", 0, 0, 3),
           ("out", 0, "C", 1)]


def grid_shape(mesh):
    """(N_t, [n_z], [n_y], n_x) of the unknown grid."""
    return (mesh.nt,) + tuple(mesh.nu[k] for k in reversed(range(mesh.d)))


def to_grid(mesh, v):
    """Complex unknown vector(s) (..., n) -> real tensor (B, 2 NC, *grid)."""
    v = np.asarray(v, dtype=np.complex128).reshape(-1, mesh.nt, mesh.nu[2], mesh.nu[1], mesh.nu[0], mesh.nc)
    v = v.reshape((v.shape[0],) + grid_shape(mesh) + (mesh.nc,))
    re_im = np.stack([v.real, v.imag], axis=-1)                      # (..., NC, 2)
    g = re_im.reshape(re_im.shape[:-2] + (2 * mesh.nc,))
    return torch.from_numpy(np.ascontiguousarray(np.moveaxis(g, -1, 1)))


def from_grid(mesh, g):
    """Real tensor (B, 2 NC, *grid) -> complex unknown vectors (B, n)."""
    a = np.moveaxis(g.detach().numpy(), 1, -1)
    a = a.reshape(a.shape[:-1] + (mesh.nc, 2))
    return (a[..., 0] + 1j * a[..., 1]).reshape(a.shape[0], -1)


def init_params(d, nc, seed=0, channels=CHANNELS):
    """He-normal weights and zero biases, float64, from a seeded generator."""
    D = d + 1
    gen = torch.Generator().manual_seed(seed)
    params = {}
    for name, cin, cout, k in _LAYERS:
        ci = 2 * nc if cin == "C" else channels[cin]
        co = 2 * nc if cout == "C" else channels[cout]
        fan_in = ci * k ** D
        std = math.sqrt(2.0 / fan_in) if name != "out" else math.sqrt(1.0 / fan_in)
        params[name + ".w"] = torch.randn((co, ci) + (k,) * D, generator=gen, dtype=torch.float64) * std
        params[name + ".b"] = torch.zeros(co, dtype=torch.float64)
    return params


def convnd(x, w, b):
    """Zero-padded 'same' convolution (cross-correlation) of x (B, Ci, *grid) with
    w (Co, Ci, *kernel), odd kernel sizes, D = 2, 3 or 4 axes."""
    D = w.dim() - 2
    pad = [k // 2 for k in w.shape[2:]]
    if D == 2:
        return F.conv2d(x, w, b, padding=pad)
    if D == 3:
        return F.conv3d(x, w, b, padding=pad)
    if D != 4:
        raise ValueError("2, 3 or 4 convolution axes")
    kt, T = w.shape[2], x.shape[2]
    slices = []
    for t in range(T):
        acc = b.view((1, -1) + (1,) * 3).expand((x.shape[0], w.shape[0]) + x.shape[3:])
        for dt in range(kt):
            ts = t + dt - kt // 2
            if 0 <= ts < T:
                acc = acc + F.conv3d(x[:, :, ts], w[:, :, dt], None, padding=pad[1:])
        slices.append(acc)
    return torch.stack(slices, dim=2)


def pool(x):
    """Mean over blocks of 2 along every grid axis; cut blocks count missing cells as 0."""
    D = x.dim() - 2
    pad = []
    for n in reversed(x.shape[2:]):
        pad += [0, n % 2]
    x = F.pad(x, pad)
    for axis in range(2, 2 + D):
        n = x.shape[axis]
        x = x.reshape(x.shape[:axis] + (n // 2, 2) + x.shape[axis + 1:]).mean(dim=axis + 1)
    return x


def upsample(x, shape):
    """Nearest neighbour: fine cell p takes coarse cell p // 2, for the fine grid `shape`."""
    for i, n in enumerate(shape):
        axis = 2 + i
        x = x.repeat_interleave(2, dim=axis).narrow(axis, 0, n)
    return x


def forward(params, x):
    """The network on a batch of field grids x (B, 2 NC, *grid), unnormalised."""
    def c(name, h):
        return convnd(h, params[name + ".w"], params[name + ".b"])
    s1 = F.relu(c("e1b", F.relu(c("e1a", x))))
    s2 = F.relu(c("e2b", F.relu(c("e2a", pool(s1)))))
    h = F.relu(c("e3b", F.relu(c("e3a", pool(s2)))))
    h = F.relu(c("u2c", c("u2p", upsample(h, s2.shape[2:])) + s2))
    h = F.relu(c("u1c", c("u1p", upsample(h, s1.shape[2:])) + s1))
    return c("out", h)


def apply(params, x):
    """M on a batch (B, 2 NC, *grid): each sample scaled to unit 2-norm and back."""
    nrm = torch.sqrt((x * x).flatten(1).sum(dim=1)).view((-1,) + (1,) * (x.dim() - 1))
    safe = torch.where(nrm > 0, nrm, torch.ones_like(nrm))
    return forward(params, x / safe) * nrm


def preconditioner(mesh, params):
    """Callable v -> M v on complex unknown vectors, for solvers.fgmres."""
    def M(v):
        with torch.no_grad():
            return from_grid(mesh, apply(params, to_grid(mesh, v)))[0]
    return M


def ls_scale(Au, rho):
    """Complex alpha minimising ||rho - alpha Au|| over alpha: <Au, rho> / <Au, Au>
    (conjugate-linear in the first argument); 0 when Au = 0."""
    aa = np.vdot(Au, Au).real
    return complex(np.vdot(Au, rho) / aa) if aa > 0 else 0j


def learned_correction(mesh, params, A, sweep):
    """Callable v -> M_CN(v) + alpha U(rho / ||rho||) on complex unknown vectors,
    rho = v - A M_CN(v), alpha = ls_scale(A U, rho); A a sparse matrix, sweep the
    callable of precond.crank_nicolson_sweep."""
    def M(v):
        v = np.asarray(v, dtype=np.complex128)
        z0 = sweep(v)
        rho = v - A @ z0
        nrm = np.linalg.norm(rho)
        if nrm == 0:
            return z0
        with torch.no_grad():
            u = from_grid(mesh, forward(params, to_grid(mesh, rho / nrm)))[0]
        return z0 + ls_scale(A @ u, rho) * u
    return M
