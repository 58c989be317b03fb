"""Pins for oracle.element: closed-form integrals, golden 1+1 matrices, invariants."""
import os

import numpy as np
import pytest

from oracle import element


def _read_golden(path):
    mats, cur = {}, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            mats[cur] = []
        else:
            mats[cur].append([float(v) for v in line.split()])
    return {k: np.array(v) for k, v in mats.items()}


def test_1d_closed_forms():
    # textbook Q1 integrals on [0, h]
    h = 0.37
    D0, Dk, Dt = element.element_matrices(1, [h], 1.0)
    M = h / 6 * np.array([[2, 1], [1, 2]])
    C = np.array([[-0.5, 0.5], [-0.5, 0.5]])
    Mt = 1.0 / 6 * np.array([[2, 1], [1, 2]])
    Ct = C
    assert np.allclose(D0, np.kron(Mt, M), atol=1e-15)
    assert np.allclose(Dk[0], np.kron(Mt, C), atol=1e-15)
    assert np.allclose(Dt, np.kron(Ct, M), atol=1e-15)


@pytest.mark.parametrize("h", [1.0, 0.25])
def test_golden_1p1(golden_dir, h):
    g = _read_golden(os.path.join(golden_dir, "q1_element_1p1.txt"))
    D0, Dk, Dt = element.element_matrices(1, [h], h)
    assert np.allclose(D0 * 36 / h ** 2, g["D0*36"], atol=1e-12)
    assert np.allclose(Dk[0] * 12 / h, g["Dx*12"], atol=1e-12)
    assert np.allclose(Dt * 12 / h, g["Dt*12"], atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_invariants(d):
    hs = [0.3, 0.5, 0.7][:d]
    ht = 0.2
    D0, Dk, Dt = element.element_matrices(d, hs, ht)
    vol = np.prod(hs) * ht
    nloc = 2 ** (d + 1)
    # partition of unity: sum_j n_j = 1, so column sums of D0 are int n_i = vol / nloc
    assert np.allclose(D0.sum(axis=0), vol / nloc)
    assert np.isclose(D0.sum(), vol)
    # derivative of a constant: D^q 1 = 0 (row sums vanish)
    for D in Dk + [Dt]:
        assert np.allclose(D.sum(axis=1), 0, atol=1e-15)
    # int d_q (n_i) over the element with sum_j n_j = 1: column sums of D^q
    # equal the face integrals, +-vol/(h_q * nloc/2) / 2 ... check antisymmetry instead:
    # D^q + D^q^T = boundary term, whose total sum over i,j is zero
    for D in Dk + [Dt]:
        assert np.isclose((D + D.T).sum(), 0, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_kronecker_structure(d):
    hs = [0.3, 0.5, 0.7][:d]
    ht = 0.2
    D0, Dk, Dt = element.element_matrices(d, hs, ht)
    M = [h / 6 * np.array([[2, 1], [1, 2]]) for h in hs]
    C = np.array([[-0.5, 0.5], [-0.5, 0.5]])
    Mt = ht / 6 * np.array([[2, 1], [1, 2]])

    def kron_all(mats):
        out = np.array([[1.0]])
        for a in mats:
            out = np.kron(out, a)
        return out
    # local index = a_t 2^d + ... + a_y 2 + a_x: t slowest, x fastest
    sp = M[::-1]
    assert np.allclose(D0, kron_all([Mt] + sp))
    assert np.allclose(Dt, kron_all([C] + sp))
    for k in range(d):
        mats = [C if j == k else M[j] for j in range(d)][::-1]
        assert np.allclose(Dk[k], kron_all([Mt] + mats))


def test_forms_differ_by_gamma0():
    from oracle import dirac
    for d in (1, 2, 3):
        A0h, AVh = element.element_operator(d, [0.3, 0.4, 0.5], 0.2, 1.1, "hamiltonian")
        A0a, AVa = element.element_operator(d, [0.3, 0.4, 0.5], 0.2, 1.1, "appendix")
        G = np.kron(np.eye(2 ** (d + 1)), dirac.gammas(d)[0])
        assert np.allclose(G @ A0a, A0h)
        assert np.allclose(G @ AVa, AVh)
