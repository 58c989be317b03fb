"""Gamma matrices and the Hamiltonian-form spin matrices (alpha_k, beta).

Follows the free Dirac equation (i gamma^mu d_mu - m) Psi = 0 of Sec. 2.1
(Eq. 1) and the 1+1 gamma matrices written out in Appendix A:
gamma^0 = diag(1, -1), gamma^1 = [[0, 1], [-1, 0]].

Readings (the paper leaves these unstated):
* 2+1 keeps a 2-component spinor with gamma^0 = sigma_z, gamma^1 = i sigma_y,
  gamma^2 = -i sigma_x (the 1+1 pair extended by the third anticommuting
  2x2 matrix).
* 3+1 uses the Dirac representation gamma^0 = diag(I, -I),
  gamma^k = [[0, sigma_k], [-sigma_k, 0]].
* alpha_k = gamma^0 gamma^k and beta = gamma^0 (premultiplying the equation
  by gamma^0, which is unitary, gives i d_t Psi = (alpha.p + beta m) Psi).

Pinned by tests/test_oracle_dirac.py: the Clifford relation
{gamma^mu, gamma^nu} = 2 eta^{mu nu} with eta = diag(1, -1, -1, -1), the
appendix's printed 1+1 matrices, and Hermiticity / anticommutation of alpha, beta.
"""

import numpy as np

SIGMA_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SIGMA_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SIGMA_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)
Z2 = np.zeros((2, 2), dtype=np.complex128)


def ncomp(d):
    """Spinor components: 2 in 1+1 and 2+1, 4 in 3+1 (Sec. 2.1 below Eq. 2)."""
    return 2 if d < 3 else 4


def gammas(d):
    """Return [gamma^0, gamma^1, ..., gamma^d] for spatial dimension d."""
    if d == 1:
        return [SIGMA_Z.copy(), 1j * SIGMA_Y]
    if d == 2:
        return [SIGMA_Z.copy(), 1j * SIGMA_Y, -1j * SIGMA_X]
    if d == 3:
        g0 = np.block([[I2, Z2], [Z2, -I2]])
        gk = [np.block([[Z2, s], [-s, Z2]]) for s in (SIGMA_X, SIGMA_Y, SIGMA_Z)]
        return [g0] + gk
    raise ValueError("d must be 1, 2 or 3")


def alphas_beta(d):
    """alpha_k = gamma^0 gamma^k (k = 1..d) and beta = gamma^0."""
    g = gammas(d)
    return [g[0] @ g[k] for k in range(1, d + 1)], g[0].copy()


def hamiltonian_symbol(d, p, m):
    """Free Dirac Hamiltonian in momentum space, H(p) = sum_k alpha_k p_k + beta m."""
    al, be = alphas_beta(d)
    h = be * m
    for k in range(d):
        h = h + al[k] * p[k]
    return h
