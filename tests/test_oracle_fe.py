"""Pins of the oracle's finite-element layer against closed forms (no GPU)."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import fe

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_gll():
    rows = np.loadtxt(os.path.join(GOLDEN, "gll_rules.txt"))
    out = {}
    for p in (2, 4):
        r = rows[rows[:, 0] == p]
        out[p] = (r[:, 1], r[:, 2])
    return out


@pytest.mark.parametrize("p", [2, 4])
def test_gll_closed_form(p):
    x, w = fe.gll_rule(p)
    gx, gw = _golden_gll()[p]
    np.testing.assert_allclose(x, gx, atol=1e-15)
    np.testing.assert_allclose(w, gw, atol=1e-15)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_gll_exactness(p):
    """GLL with p+1 points integrates x^k exactly for k <= 2p-1, not 2p."""
    x, w = fe.gll_rule(p)
    for k in range(2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    assert abs(np.dot(w, x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-6


def test_reference_matrices_p2_textbook():
    rows = np.loadtxt(os.path.join(GOLDEN, "reference_1d_p2.txt"))
    A, B, _ = fe.reference_matrices(2)
    np.testing.assert_allclose(A * 6.0, rows[:3], atol=1e-13)
    np.testing.assert_allclose(B * 15.0, rows[3:], atol=1e-13)


@pytest.mark.parametrize("p", [2, 4, 6])
def test_reference_matrices_properties(p):
    A, B, w = fe.reference_matrices(p)
    assert np.allclose(A, A.T) and np.allclose(B, B.T)
    np.testing.assert_allclose(A @ np.ones(p + 1), 0.0, atol=1e-12)     # constants have no energy
    assert abs(B.sum() - 2.0) < 1e-13                                   # int 1 = 2
    xn, _ = fe.gll_rule(p)
    # u = x^2 interpolated exactly: int (u')^2 = 8/3, int u^2 = 2/5
    u = xn ** 2
    assert abs(u @ A @ u - 8.0 / 3.0) < 1e-12
    assert abs(u @ B @ u - 2.0 / 5.0) < 1e-12
    # B against Legendre-weighted integrals: int l_i dx = GLL weight w_i (exact)
    np.testing.assert_allclose(B.sum(axis=1), w, atol=1e-13)


def test_lagrange_basis_is_interpolatory():
    xn, _ = fe.gll_rule(4)
    V = fe.lagrange_values(xn, xn)
    np.testing.assert_allclose(V, np.eye(5), atol=1e-14)
    # derivative of a degree-4 polynomial is reproduced
    xq = np.linspace(-1, 1, 7)
    c = np.array([0.3, -1.0, 0.5, 2.0, -0.7])
    dP = fe.lagrange_derivs(xn, xq) @ npleg.legval(xn, c)
    np.testing.assert_allclose(dP, npleg.legval(xq, npleg.legder(c)), atol=1e-12)


@pytest.mark.parametrize("p", [2, 4])
def test_cell_matrix_properties(p):
    mesh = fe.Mesh(-1.5, 1.5, 2, p)
    Ke = mesh.Ke
    assert np.allclose(Ke, Ke.T, atol=1e-14)
    ev = np.linalg.eigvalsh(Ke)
    assert abs(ev[0]) < 1e-12 and ev[1] > 1e-3                          # exactly one zero mode
    np.testing.assert_allclose(Ke @ np.ones(Ke.shape[0]), 0.0, atol=1e-12)
    # energy identity on one cell: u = x*y*z (degree 1 per axis) on [0,h]^3
    h = mesh.h
    xn, _ = fe.gll_rule(p)
    loc = 0.5 * h * (xn + 1.0)
    Z, Y, X = np.meshgrid(loc, loc, loc, indexing="ij")
    u = (X * Y * Z).ravel()
    # 1/2 int |grad u|^2 = 1/2 * 3 * h^2 h^2 h / 9 ... computed in closed form:
    # int (yz)^2 over the cube = h * (h^3/3)^2, three equal terms.
    exact = 0.5 * 3.0 * h * (h ** 3 / 3.0) ** 2
    assert abs(u @ Ke @ u - exact) < 1e-12 * max(1.0, exact)


def _bubble(mesh):
    lo, hi = mesh.lo, mesh.hi
    xyz = mesh.coords()
    g = (xyz - lo) * (hi - xyz)
    return g.prod(axis=1)


@pytest.mark.parametrize("n,p", [(3, 2), (2, 4), (4, 2)])
def test_assembled_energy_and_mass(n, p):
    """u = prod_d (x_d - lo)(hi - x_d) vanishes on the boundary and is a degree-2
    polynomial per axis, so its interpolant is exact and
      u^T K u = 1/2 int |grad u|^2 = 1/2 * 3 * (W^3/3) (W^5/30)^2,
      sum_a m_a u_a = (W^3/6)^3 (GLL is exact to degree 2p-1 >= 2)."""
    mesh = fe.Mesh(-2.0, 3.0, n, p)
    Wd = mesh.hi - mesh.lo
    u = _bubble(mesh)
    exact_energy = 0.5 * 3.0 * (Wd ** 3 / 3.0) * (Wd ** 5 / 30.0) ** 2
    assert abs(u @ mesh.apply_K(u) - exact_energy) < 1e-11 * exact_energy
    assert abs(mesh.mass() @ u - (Wd ** 3 / 6.0) ** 3) < 1e-11 * (Wd ** 3 / 6.0) ** 3


def _assembled_1d(mesh, M1):
    N = mesh.N
    G = np.zeros((N, N))
    for e in range(mesh.n):
        s = slice(e * mesh.p, (e + 1) * mesh.p + 1)
        G[s, s] += M1
    return G[1:-1, 1:-1]


@pytest.mark.parametrize("n,p", [(3, 2), (3, 4)])
def test_separable_identity(n, p):
    """For x = a (x) b (x) c the assembled K acts as
    1/2[(K1 a)(B1 b)(B1 c) + (B1 a)(K1 b)(B1 c) + (B1 a)(B1 b)(K1 c)]
    with 1D assembled K1 = (2/h) A, B1 = (h/2) B built by a 1D loop here."""
    mesh = fe.Mesh(-1.0, 2.0, n, p)
    A, B, _ = fe.reference_matrices(p)
    s = 0.5 * mesh.h
    K1 = _assembled_1d(mesh, A / s)
    B1 = _assembled_1d(mesh, B * s)
    rng = np.random.default_rng(11)
    total_x = np.zeros(mesh.L)
    total_y = np.zeros(mesh.L)
    for _ in range(3):                      # linear combination of separable vectors
        a, b, c = (rng.standard_normal(mesh.Ni) for _ in range(3))
        x = np.einsum("k,j,i->kji", c, b, a).ravel()     # x index fastest
        y = 0.5 * (np.einsum("k,j,i->kji", B1 @ c, B1 @ b, K1 @ a)
                   + np.einsum("k,j,i->kji", B1 @ c, K1 @ b, B1 @ a)
                   + np.einsum("k,j,i->kji", K1 @ c, B1 @ b, B1 @ a)).ravel()
        total_x += x
        total_y += y
    got = mesh.apply_K(total_x)
    assert np.abs(got - total_y).max() < 1e-13 * np.abs(total_y).max()
    got2 = mesh.assemble_K() @ total_x
    assert np.abs(got2 - total_y).max() < 1e-13 * np.abs(total_y).max()


def test_htilde_standard_form():
    """H~ = M^-1/2 (K + diag(m v)) M^-1/2 (Eq. 19) equals D K D + diag(v)."""
    mesh = fe.Mesh(-2.0, 2.0, 3, 2)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(mesh.L)
    X = rng.standard_normal((mesh.L, 4))
    m = mesh.mass()
    H = mesh.assemble_K().toarray() + np.diag(m * v)
    Ht = np.diag(m ** -0.5) @ H @ np.diag(m ** -0.5)
    np.testing.assert_allclose(mesh.apply_Htilde(v, X), Ht @ X, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n,p", [(2, 4), (3, 2), (3, 4)])
def test_htilde_rows_every_row(n, p):
    """The row-wise definition of (H~X)_a (Eq. 17, 19), used to check sampled
    rows of large meshes, against the separable closed form on every row:
    with D = d1 (x) d1 (x) d1, D x is separable when x is, so
    H~ x = D K (D x) + v o x follows from the 1D assembled K1, B1 above.
    Every row is taken, so nodes inside cells, on faces, edges and vertices,
    and next to the Dirichlet boundary are all covered."""
    mesh = fe.Mesh(-1.0, 2.0, n, p)
    A, B, _ = fe.reference_matrices(p)
    s = 0.5 * mesh.h
    K1 = _assembled_1d(mesh, A / s)
    B1 = _assembled_1d(mesh, B * s)
    d1 = mesh.m1[1:-1] ** -0.5
    rng = np.random.default_rng(17)
    v = rng.standard_normal(mesh.L)
    X = np.zeros((mesh.L, 2))
    Y = np.zeros((mesh.L, 2))
    for col in range(2):
        for _ in range(3):
            a, b, c = (rng.standard_normal(mesh.Ni) for _ in range(3))
            x = np.einsum("k,j,i->kji", c, b, a).ravel()
            da, db, dc = d1 * a, d1 * b, d1 * c
            kx = 0.5 * (np.einsum("k,j,i->kji", B1 @ dc, B1 @ db, K1 @ da)
                        + np.einsum("k,j,i->kji", B1 @ dc, K1 @ db, B1 @ da)
                        + np.einsum("k,j,i->kji", K1 @ dc, B1 @ db, B1 @ da)).ravel()
            d = np.einsum("k,j,i->kji", d1, d1, d1).ravel()
            X[:, col] += x
            Y[:, col] += d * kx
        Y[:, col] += v * X[:, col]
    rows = np.arange(mesh.L)
    got = fe.htilde_rows(mesh, v, rows, lambda idx: X[idx])
    scale = np.abs(Y).max()
    assert np.abs(got - Y).max() < 1e-13 * scale
    # and the same rows of the assembled sparse operator
    np.testing.assert_allclose(got, mesh.assemble_Htilde(v) @ X, rtol=0, atol=1e-13 * scale)
