"""Shared helpers of the GPU parity tests (no arithmetic of the method)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_rel(a, b):
    """max |a - b| / max |b| (elementwise error against the largest entry)."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def oracle_mesh(w):
    from oracle import mesh as OM
    return OM.Mesh(w.d, w.n_el, w.lo, w.hi, w.bc)
