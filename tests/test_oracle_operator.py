"""Pins for oracle.operator.

* Exact discrete Fourier reduction on periodic meshes: data exp(i k x) u
  stays a single mode, whose coefficients solve a small block system built
  here from the hand-written 1D symbols M^ = h (2 + cos th)/3, C^ = i sin th.
* Exact reduction of 2+1 (and 3+1) with data uniform in y (and z) to 1+1.
* Algorithm 1's assembled D_w22 / D_w21 = matrix-free apply / RHS = row apply.
* Hamiltonian and appendix forms give the same discrete solution.
"""
import numpy as np
import pytest

from oracle import mesh as M, operator as OP, solvers as SO


def _global_time_mats(nt, ht):
    """1D global time matrices on nodes 0..nt (textbook Q1 assembly)."""
    Mt = np.zeros((nt + 1, nt + 1))
    Ct = np.zeros((nt + 1, nt + 1))
    for e in range(nt):
        Mt[e:e + 2, e:e + 2] += ht / 6 * np.array([[2, 1], [1, 2]])
        Ct[e:e + 2, e:e + 2] += np.array([[-0.5, 0.5], [-0.5, 0.5]])
    return Mt, Ct


def _random_case(d, bc, seed, nel=(3, 4, 2), nt=3):
    rng = np.random.default_rng(seed)
    n_el = [nel[0], nel[1], nel[2], nt]
    me = M.Mesh(d, n_el, [-1.0, -0.5, 0.0, 0.0], [1.0, 1.5, 1.0, 0.6], [bc] * 3)
    nsp = me.nel[0] * me.nel[1] * me.nel[2]
    V = rng.uniform(-1, 2, nsp)
    x = rng.standard_normal(me.n_unknowns) + 1j * rng.standard_normal(me.n_unknowns)
    psi0 = rng.standard_normal(me.spatial_shape) + 1j * rng.standard_normal(me.spatial_shape)
    return me, V, x, psi0


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("bc", [M.PERIODIC, M.OPEN, M.DIRICHLET])
def test_three_routes_agree(d, bc):
    me, V, x, psi0 = _random_case(d, bc, seed=10 * d + bc)
    m = 0.8
    Dw = OP.assemble(me, m, V)
    A22, b = OP.split(me, Dw, psi0)
    y_mf = OP.apply(me, m, V, x)
    y_sp = A22 @ x
    assert np.allclose(y_mf, y_sp, rtol=0, atol=1e-13)
    assert np.allclose(OP.rhs(me, m, V, psi0), b, rtol=0, atol=1e-13)
    nodes = np.arange(me.n_unknowns // me.nc)
    y_rows = OP.apply_rows(me, m, V, x, nodes).ravel()
    assert np.allclose(y_rows, y_mf, rtol=0, atol=1e-13)


@pytest.mark.parametrize("nx,nt,kmode", [(8, 5, 1), (12, 9, 3), (7, 4, -2)])
def test_fourier_reduction_1p1(nx, nt, kmode):
    m = 1.0
    L, T = 2 * np.pi, 0.8
    me = M.Mesh(1, [nx, 1, 1, nt], [0, 0, 0, 0], [L, 1, 1, T], [M.PERIODIC] * 3)
    k = 2 * np.pi * kmode / L
    u0 = np.array([0.3 + 0.1j, -0.7 + 0.2j])
    x = me.node_coords(0)
    psi0 = np.exp(1j * k * x)[:, None] * u0[None, :]
    A22, b = OP.split(me, OP.assemble(me, m, None), psi0)
    sol = SO.dense_solve(A22, b).reshape(me.unknown_shape)
    # reduced 2 nt x 2 nt system from the symbols
    h = me.h[0]
    th = k * h
    Mh = h * (2 + np.cos(th)) / 3
    Ch = 1j * np.sin(th)
    sx = np.array([[0, 1], [1, 0]])
    sz = np.array([[1, 0], [0, -1]])
    Mt, Ct = _global_time_mats(nt, me.ht)

    def blk(n, n2):
        return 1j * Ct[n, n2] * Mh * np.eye(2) + 1j * Mt[n, n2] * Ch * sx - Mt[n, n2] * Mh * m * sz
    R = np.zeros((2 * nt, 2 * nt), dtype=complex)
    rb = np.zeros(2 * nt, dtype=complex)
    for n in range(1, nt + 1):
        for n2 in range(1, nt + 1):
            R[2 * (n - 1):2 * n, 2 * (n2 - 1):2 * n2] = blk(n, n2)
        rb[2 * (n - 1):2 * n] = -blk(n, 0) @ u0
    c = np.linalg.solve(R, rb).reshape(nt, 2)
    expect = np.exp(1j * k * x)[None, :, None] * c[:, None, :]
    assert np.allclose(sol[:, 0, 0], expect, rtol=0, atol=1e-12)


def test_fourier_reduction_2p1():
    m = 0.7
    nx, ny, nt = 6, 5, 4
    me = M.Mesh(2, [nx, ny, 1, nt], [0, 0, 0, 0], [1.0, 2.0, 1, 0.5], [M.PERIODIC] * 3)
    kx, ky = 2 * np.pi * 1 / 1.0, 2 * np.pi * 2 / 2.0
    u0 = np.array([1.0, 0.5j])
    X, Y = me.node_coords(0), me.node_coords(1)
    ph = np.exp(1j * (kx * X[None, :] + ky * Y[:, None]))
    psi0 = ph[None, :, :, None] * u0
    A22, b = OP.split(me, OP.assemble(me, m, None), psi0)
    sol = SO.dense_solve(A22, b).reshape(me.unknown_shape)
    hx, hy = me.h[0], me.h[1]
    Mx, My = hx * (2 + np.cos(kx * hx)) / 3, hy * (2 + np.cos(ky * hy)) / 3
    Cx, Cy = 1j * np.sin(kx * hx), 1j * np.sin(ky * hy)
    sx = np.array([[0, 1], [1, 0]]); sy = np.array([[0, -1j], [1j, 0]]); sz = np.diag([1, -1])
    Mt, Ct = _global_time_mats(nt, me.ht)

    def blk(n, n2):
        return (1j * Ct[n, n2] * Mx * My * np.eye(2) + 1j * Mt[n, n2] * (Cx * My * sx + Mx * Cy * sy)
                - Mt[n, n2] * Mx * My * m * sz)
    R = np.zeros((2 * nt, 2 * nt), dtype=complex)
    rb = np.zeros(2 * nt, dtype=complex)
    for n in range(1, nt + 1):
        for n2 in range(1, nt + 1):
            R[2 * (n - 1):2 * n, 2 * (n2 - 1):2 * n2] = blk(n, n2)
        rb[2 * (n - 1):2 * n] = -blk(n, 0) @ u0
    c = np.linalg.solve(R, rb).reshape(nt, 2)
    expect = ph[None, :, :, None] * c[:, None, None, :]
    assert np.allclose(sol[:, 0], expect, rtol=0, atol=1e-12)


def _solve(me, m, V, psi0):
    A22, b = OP.split(me, OP.assemble(me, m, V), psi0)
    return SO.dense_solve(A22, b).reshape(me.unknown_shape)


@pytest.mark.parametrize("bcx", [M.PERIODIC, M.OPEN, M.DIRICHLET])
def test_cross_dimension_reduction(bcx):
    rng = np.random.default_rng(5)
    m, nx, nt = 1.1, 7, 4
    a = rng.standard_normal((nx + 1, 4)) + 1j * rng.standard_normal((nx + 1, 4))
    Vx = rng.uniform(0, 2, nx)
    m1 = M.Mesh(1, [nx, 1, 1, nt], [-1, 0, 0, 0], [1, 1, 1, 0.7], [bcx, 0, 0])
    nu = m1.nu[0]
    a = a[:nu]
    s1a = _solve(m1, m, Vx, a[:, [0, 3]])
    s1b = _solve(m1, m, Vx, a[:, [1, 2]])
    # 2+1, uniform in periodic y
    ny = 3
    m2 = M.Mesh(2, [nx, ny, 1, nt], [-1, 0, 0, 0], [1, 0.9, 1, 0.7], [bcx, M.PERIODIC, 0])
    V2 = np.tile(Vx, ny)
    s2 = _solve(m2, m, V2, np.broadcast_to(a[None, :, [0, 3]], (ny, nu, 2)).copy())
    for iy in range(ny):
        assert np.allclose(s2[:, 0, iy], s1a[:, 0, 0], rtol=0, atol=1e-12)
    # 3+1, uniform in periodic y and z: pairs (1,4) and (2,3) obey 1+1
    nz = 2
    m3 = M.Mesh(3, [nx, ny, nz, nt], [-1, 0, 0, 0], [1, 0.9, 0.8, 0.7], [bcx, M.PERIODIC, M.PERIODIC])
    V3 = np.tile(Vx, ny * nz)
    s3 = _solve(m3, m, V3, np.broadcast_to(a[None, None], (nz, ny, nu, 4)).copy())
    for iz in range(nz):
        for iy in range(ny):
            assert np.allclose(s3[:, iz, iy][..., [0, 3]], s1a[:, 0, 0], rtol=0, atol=1e-12)
            assert np.allclose(s3[:, iz, iy][..., [1, 2]], s1b[:, 0, 0], rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_hamiltonian_and_appendix_forms_same_solution(d):
    me, V, x, psi0 = _random_case(d, M.OPEN, seed=3 + d, nel=(3, 2, 2), nt=3)
    m = 0.9
    sh = _solve(me, m, V, psi0)
    A22, b = OP.split(me, OP.assemble(me, m, V, form="appendix"), psi0)
    sa = SO.dense_solve(A22, b).reshape(me.unknown_shape)
    assert np.allclose(sh, sa, rtol=0, atol=1e-11 * np.abs(sh).max())


def test_potential_is_minus_V_mass():
    # A(m, V) - A(m, 0) = -V (x) mass: with V uniform it equals -V D^0-assembled x
    me, V, x, psi0 = _random_case(2, M.PERIODIC, seed=9)
    m = 0.5
    Vc = np.full_like(V, 1.7)
    dy = OP.apply(me, m, Vc, x) - OP.apply(me, m, None, x)
    # the assembled mass matrix D^0 (x) I, taken as the V-derivative of D_w
    Dw0 = OP.assemble(me, 0.0, np.full_like(V, 1.0))
    Dz = OP.assemble(me, 0.0, None)
    mass = -(Dw0 - Dz)            # = assembled D^0 (x) I
    unk = np.repeat(me.unknown_mask_geo().ravel(), me.nc)
    assert np.allclose(dy, -1.7 * (mass[unk][:, unk] @ x), atol=1e-13)
    # mass matrix is symmetric positive definite
    Mm = mass[unk][:, unk].toarray()
    assert np.allclose(Mm, Mm.T)
    assert np.all(np.linalg.eigvalsh(Mm.real) > 0)


@pytest.mark.parametrize("d,nel,bc_other", [(1, (14, 1, 1), None), (2, (10, 4, 1), M.PERIODIC)])
def test_dirichlet_data_from_an_open_solution(d, nel, bc_other):
    """The interior rows of a Dirichlet problem are the interior rows of the open
    problem on the same mesh, with the end-node values moved to the right-hand
    side.  So Dirichlet data equal to an open-axis solution's end values (and its
    initial layer) gives back that solution at every interior node, exactly."""
    from oracle import solvers as SO
    nt = 5
    rng = np.random.default_rng(40 + d)
    lo, hi = [-1.0, 0.0, 0.0, 0.0], [1.5, 1.0, 1.0, 0.8]
    rest = [bc_other] if d == 2 else []
    mo = M.Mesh(d, list(nel) + [nt], lo, hi, [M.OPEN] + rest)
    md = M.Mesh(d, list(nel) + [nt], lo, hi, [M.DIRICHLET] + rest)
    V = rng.uniform(-0.5, 1.0, nel[0] * nel[1] * nel[2])
    psi0_open = rng.standard_normal(mo.spatial_shape) + 1j * rng.standard_normal(mo.spatial_shape)
    Ao, bo = OP.split(mo, OP.assemble(mo, 0.8, V), psi0_open)
    xo = SO.dense_solve(Ao, bo)
    go = mo.to_geo(xo)                                 # open solution on every geometric node,
    go[0] = mo.layer_to_geo(psi0_open)                 # its initial layer included
    # same geometry: the open mesh's nodes are the Dirichlet mesh's geometric nodes
    assert mo.geo_shape == md.geo_shape
    inner = tuple(slice(md.u0[k], md.u0[k] + md.nu[k]) for k in (2, 1, 0))
    psi0_d = go[0][inner]                              # the initial layer on the Dirichlet unknowns
    Ad, bd = OP.split(md, OP.assemble(md, 0.8, V), psi0_d, boundary=go)
    xd = SO.dense_solve(Ad, bd)
    np.testing.assert_allclose(xd, md.from_geo(go).ravel(), rtol=0, atol=1e-11 * np.abs(xo).max())
    # without the boundary data the homogeneous problem is solved instead
    A0, b0 = OP.split(md, OP.assemble(md, 0.8, V), psi0_d)
    assert np.array_equal(A0.toarray(), Ad.toarray())
    assert np.linalg.norm(SO.dense_solve(A0, b0) - xd) > 1e-3 * np.linalg.norm(xd)
