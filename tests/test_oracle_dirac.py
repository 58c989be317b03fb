"""Pins for oracle.dirac: Clifford algebra and the printed 1+1 matrices (Appendix A)."""
import numpy as np
import pytest

from oracle import dirac


@pytest.mark.parametrize("d", [1, 2, 3])
def test_clifford_relation(d):
    g = dirac.gammas(d)
    eta = np.diag([1.0] + [-1.0] * d)
    n = dirac.ncomp(d)
    for mu in range(d + 1):
        for nu in range(d + 1):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2 * eta[mu, nu] * np.eye(n))


def test_printed_1p1_matrices():
    # Appendix A prints gamma^0 = [[1,0],[0,-1]] and gamma^1 = [[0,1],[-1,0]]
    g = dirac.gammas(1)
    assert np.array_equal(g[0], np.array([[1, 0], [0, -1]]))
    assert np.array_equal(g[1], np.array([[0, 1], [-1, 0]]))
    # Sec. 4.3's operator with V = 0 is gamma^0 i d_t + i gamma^1 d_x - m:
    # [[i d_t - m, i d_x], [-i d_x, -i d_t - m]]  (entry (1,2) = +i d_x, (2,1) = -i d_x)
    assert g[1][0, 1] == 1 and g[1][1, 0] == -1


@pytest.mark.parametrize("d", [1, 2, 3])
def test_alpha_beta_hermitian_anticommuting(d):
    al, be = dirac.alphas_beta(d)
    n = dirac.ncomp(d)
    mats = al + [be]
    for a in mats:
        assert np.allclose(a, a.conj().T)
        assert np.allclose(a @ a, np.eye(n))
    for i in range(len(mats)):
        for j in range(i + 1, len(mats)):
            assert np.allclose(mats[i] @ mats[j] + mats[j] @ mats[i], 0)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_hamiltonian_squares_to_energy(d):
    rng = np.random.default_rng(d)
    p = rng.standard_normal(d)
    m = 1.3
    H = dirac.hamiltonian_symbol(d, p, m)
    assert np.allclose(H @ H, (p @ p + m * m) * np.eye(dirac.ncomp(d)))


def test_3p1_dirac_representation():
    al, be = dirac.alphas_beta(3)
    assert np.allclose(be, np.diag([1, 1, -1, -1]))
    # alpha_x couples (1,4) and (2,3) - the pairs of the 3+1 -> 1+1 reduction
    ax = al[0]
    assert ax[0, 3] == 1 and ax[3, 0] == 1 and ax[1, 2] == 1 and ax[2, 1] == 1
