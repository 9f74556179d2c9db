"""Pins of the dense per-cell potential matrices (the Gauss-quadrature reading
of the potential term of Eq. 17): the consistent mass for a constant potential,
the collocation operator when the rule is the GLL rule, exact integrals of
polynomials, symmetry and definiteness."""
from __future__ import annotations

import os
import sys

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from oracle import fe  # noqa: E402
from oracle import potential_matrix as pm  # noqa: E402


@pytest.mark.parametrize("p", [2, 4])
def test_constant_potential_gives_the_consistent_mass(p):
    mesh = fe.Mesh(-2.0, 2.0, 3, p)          # h = 4/3 (h/2 != 1 catches a wrong Jacobian)
    Ve = pm.cell_potential_matrices(mesh, np.full(mesh.N ** 3, 1.7))
    _, B, _ = fe.reference_matrices(p)
    s = 0.5 * mesh.h
    Mc = (s ** 3) * np.kron(B, np.kron(B, B))
    for V in Ve:
        np.testing.assert_allclose(V, 1.7 * Mc, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("p", [2, 4])
def test_gll_rule_reproduces_collocation(p):
    mesh = fe.Mesh(-3.0, 3.0, 4, p)
    xyz = mesh.coords_full()
    v_full = np.cos(xyz[:, 0]) + 0.2 * xyz[:, 1] ** 2 - 0.1 * xyz[:, 2]
    Ve = pm.cell_potential_matrices(mesh, v_full, rule="gll")
    X = np.random.default_rng(3).standard_normal((mesh.L, 2))
    v_int = mesh.to_interior(v_full[:, None])[:, 0]
    np.testing.assert_allclose(pm.apply_Htilde_dense(mesh, Ve, X), mesh.apply_Htilde(v_int, X),
                               rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("p", [2, 4])
def test_polynomial_integral_is_exact(p):
    lo, hi = -2.0, 2.0
    mesh = fe.Mesh(lo, hi, 3, p)
    xyz = mesh.coords_full()
    a = (0.3, -0.2, 0.1)
    v_full = np.prod([1.0 + a[d] * xyz[:, d] for d in range(3)], axis=0)
    b = lambda t: (t - lo) * (hi - t)
    u = np.prod([b(xyz[:, d]) for d in range(3)], axis=0)
    Ve = pm.cell_potential_matrices(mesh, v_full)
    got = u @ pm.apply_V_full(mesh, Ve, u[:, None])[:, 0]
    bb = P.polymul(P.polymul([-lo, 1.0], [hi, -1.0]), P.polymul([-lo, 1.0], [hi, -1.0]))
    def one_axis(ad):
        F = P.polyint(P.polymul([1.0, ad], bb))
        return float(P.polyval(hi, F) - P.polyval(lo, F))
    exact = np.prod([one_axis(ad) for ad in a])
    assert abs(got - exact) < 1e-11 * abs(exact)


def test_cell_matrices_are_symmetric_and_definite_for_positive_v():
    mesh = fe.Mesh(-2.0, 2.0, 2, 4)
    xyz = mesh.coords_full()
    v_full = 1.0 + np.exp(-np.sum(xyz ** 2, axis=1))
    for V in pm.cell_potential_matrices(mesh, v_full):
        np.testing.assert_allclose(V, V.T, rtol=0, atol=1e-15)
        assert np.linalg.eigvalsh(V).min() > 0.0
