"""ctypes binding of the diracst C ABI (include/diracst.h): argument marshalling only.

Every function here has the name of the C call it wraps and does nothing but
convert arguments (numpy arrays for host inputs, torch CUDA tensors or raw
integer addresses for device buffers, the current torch stream by default)
and turn negative status codes into ``DstError``.  All computation runs in the
CUDA kernels of ``lib/libdiracst.so``; if that library is missing the import
fails loudly - there is no CPU fallback.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libdiracst.so")

DST_OK, DST_NOT_CONVERGED = 0, 1
DST_ERR_ARG, DST_ERR_OOM, DST_ERR_CUDA, DST_ERR_NAN, DST_ERR_STATE = -1, -2, -3, -5, -6
DST_BC_PERIODIC, DST_BC_OPEN, DST_BC_DIRICHLET = 0, 1, 2
DST_FP64, DST_FP32 = 0, 1
DST_TEST_WAIT_LIMIT, DST_TEST_FAIL_ALLOC = 1, 2
DST_PRECOND_NONE, DST_PRECOND_CN_SWEEP, DST_PRECOND_CN_SWEEP2, DST_PRECOND_CN_LEARNED, DST_PRECOND_BLOCK_JACOBI = 0, 1, 2, 3, 4

EXPORTED = (
    "dst_create_mesh", "dst_destroy_mesh", "dst_mesh_sizes", "dst_set_mass", "dst_set_potential",
    "dst_set_initial_data", "dst_build_rhs", "dst_apply_operator", "dst_arnoldi_project",
    "dst_arnoldi_update", "dst_default_solve_opts", "dst_solve", "dst_status_string",
    "dst_last_error_detail", "dst_arnoldi_project_noalloc", "dst_observables", "dst_solve_batch",
    "dst_tune_apply", "dst_set_apply_variant", "dst_get_apply_variant", "dst_testing_set",
    "dst_set_boundary_data", "dst_precond_apply", "dst_energy",
    "dst_unet_create", "dst_unet_destroy", "dst_unet_num_params", "dst_unet_set_params", "dst_unet_get_params",
    "dst_unet_forward", "dst_unet_loss_grad", "dst_unet_train", "dst_set_learned_precond",
    "dst_testing_fp32_arnoldi", "dst_unet_output_scale",
)


class DstError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        detail = ""
        if code in (DST_ERR_CUDA, DST_ERR_ARG) and _lib is not None:
            detail = ": " + _lib.dst_last_error_detail().decode(errors="replace")
        super().__init__("%s failed with %d (%s)%s" % (where, code, dst_status_string(code), detail))


class dst_solve_opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("rtol", ctypes.c_double),
                ("mixed_precision", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("use_initial_guess", ctypes.c_int),
                ("profile", ctypes.c_int), ("inner_cycles", ctypes.c_int), ("ortho", ctypes.c_int),
                ("mixed_ortho", ctypes.c_int), ("method", ctypes.c_int), ("batch_cta_max", ctypes.c_int),
                ("precond", ctypes.c_int)]


class dst_solve_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("refinements", ctypes.c_int),
                ("status", ctypes.c_int), ("rel_resid_true", ctypes.c_double),
                ("rel_resid_est", ctypes.c_double), ("seconds", ctypes.c_double),
                ("bytes_moved", ctypes.c_double), ("launches", ctypes.c_double), ("reorths", ctypes.c_int),
                ("kernel_ms", ctypes.c_double * 9), ("kernel_launches", ctypes.c_double * 9),
                ("kernel_bytes", ctypes.c_double * 9), ("kernel_flops", ctypes.c_double * 9)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name.startswith("kernel_") else v
        return out


KERNEL_CLASSES = ("apply64", "apply32", "cast", "project", "update", "scale", "misc", "rhs", "precond")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdiracst.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_2103_14588_gb300.build" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, c_int, c_double = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "dst_create_mesh": (c_int, [c_int, P(i64), P(c_double), P(c_double), P(c_int), P(vp)]),
        "dst_destroy_mesh": (c_int, [vp]),
        "dst_mesh_sizes": (c_int, [vp, P(i64), P(i64), P(c_int)]),
        "dst_set_mass": (c_int, [vp, c_double]),
        "dst_set_potential": (c_int, [vp, vp]),
        "dst_set_initial_data": (c_int, [vp, vp]),
        "dst_set_boundary_data": (c_int, [vp, vp]),
        "dst_build_rhs": (c_int, [vp, vp, vp]),
        "dst_apply_operator": (c_int, [vp, c_int, vp, vp, vp]),
        "dst_arnoldi_project": (c_int, [i64, c_int, vp, vp, vp, vp]),
        "dst_arnoldi_update": (c_int, [i64, c_int, vp, vp, vp, vp, vp]),
        "dst_arnoldi_project_noalloc": (c_int, [i64, c_int, vp, vp, vp, vp]),
        "dst_observables": (c_int, [vp, vp, c_double, vp, vp]),
        "dst_default_solve_opts": (c_int, [P(dst_solve_opts)]),
        "dst_solve": (c_int, [vp, P(dst_solve_opts), vp, P(dst_solve_stats), vp]),
        "dst_solve_batch": (c_int, [c_int, P(vp), P(dst_solve_opts), P(vp), P(dst_solve_stats), vp]),
        "dst_tune_apply": (c_int, [vp, vp]),
        "dst_set_apply_variant": (c_int, [vp, c_int, c_int]),
        "dst_get_apply_variant": (c_int, [vp, c_int, P(c_int), P(c_int)]),
        "dst_status_string": (ctypes.c_char_p, [c_int]),
        "dst_last_error_detail": (ctypes.c_char_p, []),
        "dst_testing_set": (c_int, [c_int, i64]),
        "dst_precond_apply": (c_int, [vp, c_int, vp, vp, vp]),
        "dst_energy": (c_int, [vp, vp, vp, vp]),
        "dst_unet_create": (c_int, [vp, P(vp)]),
        "dst_unet_destroy": (c_int, [vp]),
        "dst_unet_num_params": (c_int, [vp, P(i64)]),
        "dst_unet_set_params": (c_int, [vp, vp]),
        "dst_unet_get_params": (c_int, [vp, vp]),
        "dst_unet_forward": (c_int, [vp, vp, vp, vp]),
        "dst_unet_loss_grad": (c_int, [vp, vp, vp, P(c_double), vp, vp]),
        "dst_unet_train": (c_int, [vp, vp, c_int, ctypes.c_float, ctypes.c_uint64, vp, vp]),
        "dst_set_learned_precond": (c_int, [vp, vp]),
        "dst_unet_output_scale": (c_int, [vp, P(c_double)]),
        "dst_testing_fp32_arnoldi": (c_int, [c_int, i64, c_int, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None
_lib = _load()


def library():
    return _lib


# ---- marshalling helpers -------------------------------------------------

def _dev_ptr(t, dtype=None, numel=None, what="buffer"):
    """Device address of a torch CUDA tensor (checked) or a raw integer address."""
    if isinstance(t, int):
        return t
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor or an integer device address" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (what, dtype, t.dtype))
    if numel is not None and t.numel() < numel:
        raise ValueError("%s holds %d elements, needs %d" % (what, t.numel(), numel))
    return t.data_ptr()


def _stream(stream, *tensors):
    if stream is None:
        for t in tensors:
            if not isinstance(t, int):
                import torch
                return torch.cuda.current_stream(t.device).cuda_stream
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc, where):
    if rc < 0:
        raise DstError(rc, where)
    return rc


# ---- the C ABI, one wrapper per call --------------------------------------

def dst_status_string(code):
    return _lib.dst_status_string(int(code)).decode()


def dst_create_mesh(d, n_el, lo, hi, bc):
    """Returns an opaque mesh handle (int).  n_el, lo, hi: 4 entries (x, y, z, t); bc: 3."""
    n = (ctypes.c_int64 * 4)(*[int(v) for v in n_el])
    a = (ctypes.c_double * 4)(*[float(v) for v in lo])
    b = (ctypes.c_double * 4)(*[float(v) for v in hi])
    c = (ctypes.c_int * 3)(*[int(v) for v in (list(bc) + [0, 0, 0])[:3]])
    out = ctypes.c_void_p()
    _check(_lib.dst_create_mesh(int(d), n, a, b, c, ctypes.byref(out)), "dst_create_mesh")
    return out.value


def dst_destroy_mesh(mesh):
    return _check(_lib.dst_destroy_mesh(mesh), "dst_destroy_mesh")


def dst_mesh_sizes(mesh):
    ns, nu, nc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(_lib.dst_mesh_sizes(mesh, ctypes.byref(ns), ctypes.byref(nu), ctypes.byref(nc)), "dst_mesh_sizes")
    return ns.value, nu.value, nc.value


def dst_set_mass(mesh, m):
    return _check(_lib.dst_set_mass(mesh, float(m)), "dst_set_mass")


def dst_set_potential(mesh, V):
    """V: one value per spatial element, x fastest (nel_x * nel_y * nel_z values;
    the C library reads exactly that many), or None for no potential."""
    if V is None:
        return _check(_lib.dst_set_potential(mesh, None), "dst_set_potential")
    arr = np.ascontiguousarray(V, dtype=np.float64)
    return _check(_lib.dst_set_potential(mesh, arr.ctypes.data), "dst_set_potential")


def dst_set_initial_data(mesh, psi0):
    """psi0: host data - a numpy array or a CPU torch tensor (e.g. pinned), complex128."""
    ns, _, nc = dst_mesh_sizes(mesh)
    if type(psi0).__module__.startswith("torch"):
        import torch
        if psi0.is_cuda or psi0.dtype != torch.complex128 or not psi0.is_contiguous():
            raise TypeError("psi0 must be a contiguous complex128 host tensor")
        if psi0.numel() != ns * nc:
            raise ValueError("psi0 needs %d complex values, got %d" % (ns * nc, psi0.numel()))
        return _check(_lib.dst_set_initial_data(mesh, psi0.data_ptr()), "dst_set_initial_data")
    arr = np.ascontiguousarray(psi0, dtype=np.complex128).ravel()
    if arr.size != ns * nc:
        raise ValueError("psi0 needs %d complex values, got %d" % (ns * nc, arr.size))
    return _check(_lib.dst_set_initial_data(mesh, arr.ctypes.data), "dst_set_initial_data")


def dst_set_boundary_data(mesh, psi_bd, n_values=None):
    """psi_bd: host complex128 array of the wall spinors on every layer's full node grid
    ((N_t + 1) x gz x gy x gx x NC, Dirichlet axes with both end nodes), or None."""
    if psi_bd is None:
        return _check(_lib.dst_set_boundary_data(mesh, None), "dst_set_boundary_data")
    arr = np.ascontiguousarray(psi_bd, dtype=np.complex128).ravel()
    if n_values is not None and arr.size != n_values:
        raise ValueError("psi_bd needs %d complex values, got %d" % (n_values, arr.size))
    return _check(_lib.dst_set_boundary_data(mesh, arr.ctypes.data), "dst_set_boundary_data")


def dst_build_rhs(mesh, b, stream=None):
    import torch
    _, nu, _ = dst_mesh_sizes(mesh)
    p = _dev_ptr(b, torch.complex128, nu, "b")
    return _check(_lib.dst_build_rhs(mesh, p, _stream(stream, b)), "dst_build_rhs")


def dst_apply_operator(mesh, precision, x, y, stream=None):
    import torch
    _, nu, _ = dst_mesh_sizes(mesh)
    dt = torch.complex128 if precision == DST_FP64 else torch.complex64
    px = _dev_ptr(x, dt, nu, "x")
    py = _dev_ptr(y, dt, nu, "y")
    return _check(_lib.dst_apply_operator(mesh, int(precision), px, py, _stream(stream, x, y)),
                  "dst_apply_operator")


def dst_arnoldi_project(n, nvec, V, w, h, stream=None):
    import torch
    pV = _dev_ptr(V, torch.complex128, n * nvec, "V")
    pw = _dev_ptr(w, torch.complex128, n, "w")
    ph = _dev_ptr(h, torch.complex128, nvec, "h")
    return _check(_lib.dst_arnoldi_project(int(n), int(nvec), pV, pw, ph, _stream(stream, V, w, h)),
                  "dst_arnoldi_project")


def dst_arnoldi_project_noalloc(n, nvec, V, w, h, stream=None):
    """h = V^H w using the library's static scratch instead of allocating (see diracst.h)."""
    import torch
    pV = _dev_ptr(V, torch.complex128, n * nvec, "V")
    pw = _dev_ptr(w, torch.complex128, n, "w")
    ph = _dev_ptr(h, torch.complex128, nvec, "h")
    return _check(_lib.dst_arnoldi_project_noalloc(int(n), int(nvec), pV, pw, ph, _stream(stream, V, w, h)),
                  "dst_arnoldi_project_noalloc")


def dst_arnoldi_update(n, nvec, V, h, w, nrm2, stream=None):
    import torch
    pV = _dev_ptr(V, torch.complex128, n * nvec, "V")
    ph = _dev_ptr(h, torch.complex128, nvec, "h")
    pw = _dev_ptr(w, torch.complex128, n, "w")
    pn = _dev_ptr(nrm2, torch.float64, 1, "nrm2")
    return _check(_lib.dst_arnoldi_update(int(n), int(nvec), pV, ph, pw, pn, _stream(stream, V, w)),
                  "dst_arnoldi_update")


def dst_precond_apply(mesh, kind, v, z, stream=None):
    """z = M v for the preconditioner `kind` (complex64 CUDA tensors of n_unknowns entries)."""
    import torch
    _, nu, _ = dst_mesh_sizes(mesh)
    pv = _dev_ptr(v, torch.complex64, nu, "v")
    pz = _dev_ptr(z, torch.complex64, nu, "z")
    return _check(_lib.dst_precond_apply(mesh, int(kind), pv, pz, _stream(stream, v, z)), "dst_precond_apply")


def dst_observables(mesh, psi, x0, out, stream=None):
    """Per-layer [Q, Q_right, M_x, M_y, M_z] of a solution (out: N_t x 5 float64 CUDA tensor)."""
    import torch
    ns, nu, nc = dst_mesh_sizes(mesh)
    nt = nu // (ns * nc)
    pp = _dev_ptr(psi, torch.complex128, nu, "psi")
    po = _dev_ptr(out, torch.float64, 5 * nt, "out")
    return _check(_lib.dst_observables(mesh, pp, float(x0), po, _stream(stream, psi, out)), "dst_observables")


def dst_testing_set(hook, value):
    """Testing hook (DST_TEST_WAIT_LIMIT / DST_TEST_FAIL_ALLOC, see diracst.h)."""
    return _check(_lib.dst_testing_set(int(hook), int(value)), "dst_testing_set")


def dst_energy(mesh, psi, out, stream=None):
    """Energy per time layer of a solution (out: N_t float64 CUDA tensor); periodic meshes."""
    import torch
    ns, nu, nc = dst_mesh_sizes(mesh)
    nt = nu // (ns * nc)
    pp = _dev_ptr(psi, torch.complex128, nu, "psi")
    po = _dev_ptr(out, torch.float64, nt, "out")
    return _check(_lib.dst_energy(mesh, pp, po, _stream(stream, psi, out)), "dst_energy")


def dst_default_solve_opts():
    o = dst_solve_opts()
    _check(_lib.dst_default_solve_opts(ctypes.byref(o)), "dst_default_solve_opts")
    return o


def dst_solve(mesh, opts, psi, stream=None):
    """Solve into psi (complex128 CUDA tensor).  opts: dst_solve_opts or dict of overrides.

    Returns the stats as a dict; raises DstError on an error status (not on
    DST_NOT_CONVERGED, which is reported in stats["status"]).
    """
    import torch
    o = opts if isinstance(opts, dst_solve_opts) else dst_default_solve_opts()
    if isinstance(opts, dict):
        for k, v in opts.items():
            setattr(o, k, v)
    _, nu, _ = dst_mesh_sizes(mesh)
    p = _dev_ptr(psi, torch.complex128, nu, "psi")
    st = dst_solve_stats()
    rc = _lib.dst_solve(mesh, ctypes.byref(o), p, ctypes.byref(st), _stream(stream, psi))
    _check(rc, "dst_solve")
    return st.as_dict()


def dst_tune_apply(mesh, stream=0):
    """Run the apply tile-shape autotuner on the mesh (both precisions)."""
    _check(_lib.dst_tune_apply(mesh, stream if isinstance(stream, int) else stream.cuda_stream), "dst_tune_apply")


def dst_set_apply_variant(mesh, precision, variant):
    _check(_lib.dst_set_apply_variant(mesh, precision, variant), "dst_set_apply_variant")


def dst_get_apply_variant(mesh, precision):
    """(current tile shape, number of shapes) for the precision."""
    v, c = ctypes.c_int(), ctypes.c_int()
    _check(_lib.dst_get_apply_variant(mesh, precision, ctypes.byref(v), ctypes.byref(c)), "dst_get_apply_variant")
    return v.value, c.value


def dst_solve_batch(meshes, opts, psis, stream=None):
    """Solve every mesh into its psi (complex128 CUDA tensors) in one batched call.

    meshes: mesh handles; psis: one tensor per mesh.  Returns (status, list of
    stats dicts); raises DstError on an error of the call itself.
    """
    import torch
    n = len(meshes)
    if n != len(psis) or n == 0:
        raise ValueError("one psi per mesh, at least one mesh")
    o = opts if isinstance(opts, dst_solve_opts) else dst_default_solve_opts()
    if isinstance(opts, dict):
        for k, v in opts.items():
            setattr(o, k, v)
    mh = (ctypes.c_void_p * n)(*[ctypes.c_void_p(h) for h in meshes])
    pp = []
    for h, t in zip(meshes, psis):
        _, nu, _ = dst_mesh_sizes(h)
        pp.append(_dev_ptr(t, torch.complex128, nu, "psi"))
    pa = (ctypes.c_void_p * n)(*pp)
    sts = (dst_solve_stats * n)()
    rc = _lib.dst_solve_batch(n, mh, ctypes.byref(o), pa, sts, _stream(stream, *psis))
    if rc < 0 and rc not in (DST_ERR_NAN,):
        _check(rc, "dst_solve_batch")
    return rc, [s_.as_dict() for s_ in sts]


class UNet:
    """Owning wrapper of a dst_unet handle (the learned correction of the sweep preconditioner)."""

    def __init__(self, mesh_handle):
        self.handle = None
        out = ctypes.c_void_p()
        _check(_lib.dst_unet_create(mesh_handle, ctypes.byref(out)), "dst_unet_create")
        self.handle = out.value
        n = ctypes.c_int64()
        _check(_lib.dst_unet_num_params(self.handle, ctypes.byref(n)), "dst_unet_num_params")
        self.num_params = n.value

    def set_params(self, params):
        arr = np.ascontiguousarray(params, dtype=np.float32).ravel()
        if arr.size != self.num_params:
            raise ValueError("need %d parameters, got %d" % (self.num_params, arr.size))
        _check(_lib.dst_unet_set_params(self.handle, arr.ctypes.data), "dst_unet_set_params")

    def get_params(self):
        arr = np.empty(self.num_params, dtype=np.float32)
        _check(_lib.dst_unet_get_params(self.handle, arr.ctypes.data), "dst_unet_get_params")
        return arr

    def forward(self, x, y, stream=None):
        import torch
        px = _dev_ptr(x, torch.complex64, None, "x")
        py = _dev_ptr(y, torch.complex64, None, "y")
        _check(_lib.dst_unet_forward(self.handle, px, py, _stream(stream, x, y)), "dst_unet_forward")

    def loss_grad(self, x, target, stream=None):
        """(loss, gradient as a float32 numpy array); synchronises."""
        import torch
        px = _dev_ptr(x, torch.complex64, None, "x")
        pt = _dev_ptr(target, torch.complex64, None, "target")
        loss = ctypes.c_double()
        g = np.empty(self.num_params, dtype=np.float32)
        _check(_lib.dst_unet_loss_grad(self.handle, px, pt, ctypes.byref(loss), g.ctypes.data,
                                       _stream(stream, x, target)), "dst_unet_loss_grad")
        return loss.value, g

    def train(self, mesh_handle, steps, lr, seed, stream=0):
        losses = np.empty(max(steps, 1), dtype=np.float32)
        _check(_lib.dst_unet_train(self.handle, mesh_handle, int(steps), float(lr), int(seed) & ((1 << 64) - 1),
                                   losses.ctypes.data, stream if isinstance(stream, int) else stream.cuda_stream),
               "dst_unet_train")
        return losses[:steps]

    def output_scale(self):
        g = ctypes.c_double()
        _check(_lib.dst_unet_output_scale(self.handle, ctypes.byref(g)), "dst_unet_output_scale")
        return g.value

    def close(self):
        if self.handle:
            _lib.dst_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def dst_set_learned_precond(mesh, net):
    return _check(_lib.dst_set_learned_precond(mesh, net.handle if net is not None else None),
                  "dst_set_learned_precond")


class Mesh:
    """Owning wrapper of a mesh handle built from a workload-like description."""

    def __init__(self, d, n_el, lo, hi, bc, m=None, V=None, psi0=None):
        if V is not None:
            ne = 1
            for k in range(int(d)):
                ne *= int(n_el[k])
            if np.size(V) != ne:
                raise ValueError("V needs one value per spatial element (%d), got %d" % (ne, np.size(V)))
        self.handle = None
        self.d, self.n_el, self.bc = int(d), [int(v) for v in n_el], [int(v) for v in (list(bc) + [0, 0, 0])[:3]]
        self.handle = dst_create_mesh(d, n_el, lo, hi, bc)
        self.n_spatial, self.n_unknowns, self.ncomp = dst_mesh_sizes(self.handle)
        if m is not None:
            dst_set_mass(self.handle, m)
        if V is not None:
            dst_set_potential(self.handle, V)
        if psi0 is not None:
            dst_set_initial_data(self.handle, psi0)

    @classmethod
    def from_workload(cls, w):
        return cls(w.d, w.n_el, w.lo, w.hi, w.bc, m=w.m, V=w.V, psi0=w.psi0)

    def wall_grid_shape(self):
        """Shape (N_t + 1, gz, gy, gx, NC) of the array dst_set_boundary_data reads."""
        g = []
        for k in range(3):
            if k >= self.d:
                g.append(1)
            elif self.bc[k] == DST_BC_PERIODIC:
                g.append(self.n_el[k])
            else:
                g.append(self.n_el[k] + 1)
        return (self.n_el[3] + 1, g[2], g[1], g[0], self.ncomp)

    def set_boundary_data(self, psi_bd):
        n = None if psi_bd is None else int(np.prod(self.wall_grid_shape()))
        return dst_set_boundary_data(self.handle, psi_bd, n)

    def close(self):
        if self.handle:
            dst_destroy_mesh(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
