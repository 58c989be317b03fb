"""Q1 Lagrange spacetime element and its matrices, by Gauss-Legendre quadrature.

Basis (Sec. 2.2, Eqs. 13-16): on the 1+1 element [0, h] x [0, h]
    n1 = (h-x)(h-t)/h^2, n2 = x(h-t)/h^2, n3 = (h-x)t/h^2, n4 = xt/h^2.
The printed n2 and n3 divide by h only; read as h^2 so that the four
functions are the bilinear interpolants (they then sum to one).  Higher
dimensions take the tensor product of the 1D factors (h - s)/h and s/h per
coordinate, with a separate element size per axis because the meshes use
h_x != h_t.

Local node numbering follows the 1+1 listing: x is the fastest bit and t the
slowest, l = a_x + 2 a_y + 4 a_z + 2^d a_t with a_q in {0, 1}.

Element matrices (Appendix A): with row j = test function, column i = trial,
    D^0_ji = int n_j n_i,   D^t_ji = int n_j d_t n_i,   D^k_ji = int n_j d_k n_i.
Two Gauss-Legendre points per axis integrate these exactly (the integrands are
at most quadratic in each coordinate).

Element operator, Hamiltonian form (the weak form of Sec. 2.1, Eqs. 6-7, with
its rows premultiplied by gamma^0, and the scalar potential of Sec. 4.3,
Eq. 21, read as potential energy V):
    A_e = i D^t (x) I + i sum_k D^k (x) alpha_k - D^0 (x) (m beta + V_e I).
Appendix form (Appendix A as printed, potential added the same way):
    A_e = i D^t (x) gamma^0 + i sum_k D^k (x) gamma^k - D^0 (x) (m I + V_e gamma^0).
The two differ by the unitary, block-diagonal factor gamma^0 on the test side,
so the discrete solutions coincide; Krylov convergence does not.

Pinned by tests/test_oracle_element.py: closed-form 1D integrals, the 1+1
element matrices in tests/golden/q1_element_1p1.txt (derived by hand from
Eqs. 13-16), partition of unity, derivative of a constant, and Kronecker
structure in 2+1 / 3+1.
"""

import itertools

import numpy as np

from .dirac import alphas_beta, gammas, ncomp


def basis_1d(a, s, h):
    """1D Q1 factor: (h - s)/h for a = 0, s/h for a = 1."""
    return (h - s) / h if a == 0 else s / h


def dbasis_1d(a, s, h):
    """Derivative of basis_1d with respect to s."""
    return -1.0 / h if a == 0 else 1.0 / h


def local_bits(l, d):
    """Bits (a_x, a_y, a_z, a_t)[:d+1] of local node l (x fastest, t slowest)."""
    return [(l >> q) & 1 for q in range(d + 1)]


def element_matrices(d, hs, ht):
    """Return (D0, [D^x, D^y, D^z][:d], Dt), each (2^(d+1), 2^(d+1)).

    hs: element sizes of the d spatial axes; ht: time element size.
    Computed by tensor Gauss-Legendre quadrature of the basis products over
    the element [0, h_x] x ... x [0, h_t].
    """
    hq = list(hs[:d]) + [ht]            # axis q = 0..d-1 spatial, q = d time
    nloc = 2 ** (d + 1)
    gx, gw = np.polynomial.legendre.leggauss(2)
    D0 = np.zeros((nloc, nloc))
    Dq = [np.zeros((nloc, nloc)) for _ in range(d + 1)]
    bits = [local_bits(l, d) for l in range(nloc)]
    for pt in itertools.product(range(2), repeat=d + 1):
        s = [hq[q] * (gx[pt[q]] + 1.0) / 2.0 for q in range(d + 1)]
        w = np.prod([gw[pt[q]] * hq[q] / 2.0 for q in range(d + 1)])
        val = np.array([np.prod([basis_1d(bits[l][q], s[q], hq[q]) for q in range(d + 1)])
                        for l in range(nloc)])
        der = np.zeros((d + 1, nloc))
        for q in range(d + 1):
            for l in range(nloc):
                f = dbasis_1d(bits[l][q], s[q], hq[q])
                for q2 in range(d + 1):
                    if q2 != q:
                        f *= basis_1d(bits[l][q2], s[q2], hq[q2])
                der[q, l] = f
        D0 += w * np.outer(val, val)                 # [j, i] = n_j n_i
        for q in range(d + 1):
            Dq[q] += w * np.outer(val, der[q])       # [j, i] = n_j d_q n_i
    return D0, Dq[:d], Dq[d]


def element_operator(d, hs, ht, m, form="hamiltonian"):
    """Return (A0, AV): the element operator is A0 + V_e * AV.

    Shapes (2^(d+1) * NC, 2^(d+1) * NC); row/column index = l * NC + c.
    """
    D0, Dk, Dt = element_matrices(d, hs, ht)
    nc = ncomp(d)
    eye = np.eye(nc, dtype=np.complex128)
    if form == "hamiltonian":
        al, be = alphas_beta(d)
        A0 = 1j * np.kron(Dt, eye)
        for k in range(d):
            A0 = A0 + 1j * np.kron(Dk[k], al[k])
        A0 = A0 - m * np.kron(D0, be)
        AV = -np.kron(D0, eye)
    elif form == "appendix":
        g = gammas(d)
        A0 = 1j * np.kron(Dt, g[0])
        for k in range(d):
            A0 = A0 + 1j * np.kron(Dk[k], g[k + 1])
        A0 = A0 - m * np.kron(D0, eye)
        AV = -np.kron(D0, g[0])
    else:
        raise ValueError(form)
    return A0, AV
