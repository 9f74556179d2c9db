"""Pins of the graded tensor-product mesh oracle (Sec. 4.2.2 reading): agreement
with the uniform-mesh oracle on equal breaks, exact energies of polynomials,
exact GLL integrals, and the particle-in-a-box spectrum on graded meshes."""
from __future__ import annotations

import math
import os
import sys

import numpy as np
import pytest
import scipy.sparse.linalg as spla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from oracle import fe  # noqa: E402
from oracle.graded import GradedMesh, graded_breaks  # noqa: E402


def _graded(p, n=4, lo=-2.0, hi=2.0, seed=0):
    rng = np.random.default_rng(seed)
    return [np.sort(np.concatenate([[lo, hi], rng.uniform(lo + 0.2, hi - 0.2, n - 1)]))
            for _ in range(3)]


@pytest.mark.parametrize("p", [2, 4])
def test_equal_breaks_reproduce_the_uniform_mesh(p):
    ref = fe.Mesh(-3.0, 3.0, 3, p)
    b = np.linspace(-3.0, 3.0, 4)
    g = GradedMesh(b, b, b, p)
    assert g.L == ref.L
    np.testing.assert_allclose(g.coords(), ref.coords(), atol=1e-14)
    np.testing.assert_allclose(g.mass(), ref.mass(), rtol=1e-14)
    X = np.random.default_rng(1).standard_normal((ref.L, 3))
    np.testing.assert_allclose(g.apply_K(X), ref.apply_K(X), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("p", [2, 4, 6])
def test_polynomial_energy_is_exact_on_a_graded_mesh(p):
    bx, by, bz = _graded(p, n=3, seed=p)
    g = GradedMesh(bx, by, bz, p)
    lo, hi = -2.0, 2.0
    xyz = g.coords()
    b = lambda t: (t - lo) * (hi - t)
    u = b(xyz[:, 0]) * b(xyz[:, 1]) * b(xyz[:, 2])
    ell = hi - lo
    i_b2, i_db2 = ell ** 5 / 30.0, ell ** 3 / 3.0          # int b^2, int (b')^2
    exact = 0.5 * 3.0 * i_db2 * i_b2 * i_b2               # 1/2 int |grad u|^2
    assert abs(u @ g.apply_K(u) - exact) < 1e-10 * exact
    # the assembled matrix is the same operator
    K = g.assemble_K()
    X = np.random.default_rng(2).standard_normal(g.L)
    np.testing.assert_allclose(K @ X, g.apply_K(X), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("p", [2, 4])
def test_gll_mass_integrates_degree_2p_minus_1_exactly(p):
    bx, by, bz = _graded(p, n=4, seed=10 + p)
    g = GradedMesh(bx, by, bz, p)
    xyz = g.coords_full()
    k = 2 * p - 1
    f = (xyz[:, 0] + 0.3) ** k * (xyz[:, 1] - 0.1) ** (k - 1) * (1.0 + xyz[:, 2])
    ix = lambda a, e: ((2.0 + a) ** (e + 1) - (-2.0 + a) ** (e + 1)) / (e + 1)
    exact = ix(0.3, k) * ix(-0.1, k - 1) * ix(1.0, 1)
    assert abs(g.mass_full() @ f - exact) < 1e-11 * abs(exact)
    assert abs(g.mass_full().sum() - 64.0) < 1e-12


@pytest.mark.parametrize("p,n", [(4, 3), (6, 2)])
def test_particle_in_a_box_on_a_graded_mesh(p, n):
    # [-2, 2]^3 box with breaks graded towards a point off the centre
    bx = graded_breaks(-2.0, 2.0, n, [0.7], 0.3, 1.5)
    by = graded_breaks(-2.0, 2.0, n, [-0.4], 0.3, 1.5)
    bz = graded_breaks(-2.0, 2.0, n, [0.0, 1.1], 0.3, 1.5)
    g = GradedMesh(bx, by, bz, p)
    H = g.assemble_Htilde(np.zeros(g.L))
    ev = np.sort(spla.eigsh(H, k=4, sigma=0.0, which="LM")[0])
    e111 = 0.5 * math.pi ** 2 * 3.0 / 16.0
    e211 = 0.5 * math.pi ** 2 * 6.0 / 16.0
    assert abs(ev[0] - e111) < 1e-4 * e111
    np.testing.assert_allclose(ev[1:4], e211, rtol=1e-3)


def test_box_spectrum_converges_at_order_2p():
    errs = []
    for n in (2, 4):
        b = graded_breaks(-2.0, 2.0, n, [0.5], 0.5, 2.0)
        g = GradedMesh(b, b, b, 2)
        H = g.assemble_Htilde(np.zeros(g.L))
        e = spla.eigsh(H, k=1, sigma=0.0, which="LM")[0][0]
        errs.append(abs(e - 0.5 * math.pi ** 2 * 3.0 / 16.0))
    assert errs[1] < errs[0] / 8.0          # 2p = 4: 16x per halving asymptotically


def test_graded_breaks():
    b = graded_breaks(-5.0, 5.0, 12, [1.0], 0.2, 2.0)
    assert len(b) == 13 and b[0] == -5.0 and b[-1] == 5.0
    assert np.all(np.diff(b) > 0.0)
    h = np.diff(b)
    mid = 0.5 * (b[1:] + b[:-1])
    assert h[np.argmin(np.abs(mid - 1.0))] == pytest.approx(h.min())
    assert h.max() / h.min() > 3.0
    u = graded_breaks(-5.0, 5.0, 10, [], 0.2, 2.0)
    np.testing.assert_allclose(np.diff(u), 1.0, rtol=1e-6)


def test_graded_breaks_follow_the_target_size():
    # equidistribution of 1/h: every cell holds the same integral of 1/h(x),
    # so cell size / h(midpoint) is the same constant S/n across cells
    lo, hi, n, hin, hout, g = -6.0, 6.0, 60, 0.1, 1.0, 0.4
    b = graded_breaks(lo, hi, n, [0.5], hin, hout, growth=g)
    mid = 0.5 * (b[1:] + b[:-1])
    target = np.minimum(hout, hin + g * np.abs(mid - 0.5))
    ratio = np.diff(b) / target
    assert np.max(ratio) / np.min(ratio) < 1.1
    # closed form of S = int dt / h(t) for this piecewise-linear h
    d1 = (hout - hin) / g                       # distance where h reaches h_outer
    S_lin = 2.0 * np.log(hout / hin) / g        # both sides of the centre, inside d1
    S = S_lin + ((0.5 - d1 - lo) + (hi - 0.5 - d1)) / hout
    np.testing.assert_allclose(np.median(ratio), S / n, rtol=0.02)


@pytest.mark.parametrize("p", [2, 4])
def test_assembled_operator_is_a_sum_of_kronecker_products(p):
    # the cell-by-cell K (Eq. 17 assembly) equals seven sweeps of the assembled
    # 1D axis matrices, on equal and on graded breaks
    for bx, by, bz in ([np.linspace(-3.0, 3.0, 4)] * 3, _graded(p, n=4, lo=-3.0, hi=3.0, seed=3)):
        g = GradedMesh(bx, by, bz, p)
        X = np.random.default_rng(4).standard_normal((g.L, 2))
        np.testing.assert_allclose(g.apply_K_sweeps(X), g.apply_K(X), rtol=1e-12, atol=1e-12)
    ref = fe.Mesh(-3.0, 3.0, 3, p)
    g = GradedMesh(*([np.linspace(-3.0, 3.0, 4)] * 3), p)
    X = np.random.default_rng(5).standard_normal((ref.L, 3))
    np.testing.assert_allclose(g.apply_K_sweeps(X), ref.apply_K(X), rtol=1e-12, atol=1e-12)
