"""Pins of the oracle's loss, adjoint, gradient, L-BFGS and Chebyshev layers (no GPU).

The adjoint equations (Eq. 7-11) are pinned by central finite differences of
the discrete loss: a dropped term, a wrong factor (the 4 of Eq. 7, the 2 of
Eq. 8-9) or a sign error in eta changes the directional derivative at first
order and fails these tests.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

import workloads as W
from oracle import adjoint as adj
from oracle import chebyshev as cheb
from oracle import fe, ks, lbfgs, potentials

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _setup(kT, Ne, nst, seed=5, centre=(0.3, -0.2, 0.1), noise=0.05):
    mesh = fe.Mesh(-4.0, 4.0, 3, 2)
    xyz = mesh.coords()
    rng = np.random.default_rng(seed)
    v = W.smeared_coulomb(xyz, np.array([centre]), np.array([2.0]), 0.5)
    v = v + noise * rng.standard_normal(mesh.L)
    rho_d = ks.forward(mesh, v + 0.1 * np.exp(-np.sum(xyz ** 2, 1)), Ne, nst, kT)["rho"]
    w = 1.0 + 0.5 * rng.uniform(size=mesh.L)          # a non-trivial positive weight
    return mesh, v, rho_d, w, rng


def _loss(mesh, vv, rho_d, w, Ne, nst, kT):
    fw = ks.forward(mesh, vv, Ne, nst, kT)
    return adj.loss_and_error(mesh, fw["rho"], rho_d, w)[0]


def _fd(mesh, v, dv, rho_d, w, Ne, nst, kT, h=1e-3):
    """Richardson-extrapolated central difference (error O(h^4))."""
    def cd(hh):
        return (_loss(mesh, v + hh * dv, rho_d, w, Ne, nst, kT)
                - _loss(mesh, v - hh * dv, rho_d, w, Ne, nst, kT)) / (2 * hh)
    return (4.0 * cd(h / 2) - cd(h)) / 3.0


@pytest.mark.parametrize("kT,Ne,nst,solver", [(0.0, 2.0, 4, "minres"), (0.0, 2.0, 4, "dense"),
                                              (0.02, 3.0, 8, "minres"), (0.02, 3.0, 8, "dense")])
def test_gradient_matches_finite_differences(kT, Ne, nst, solver):
    mesh, v, rho_d, w, rng = _setup(kT, Ne, nst)
    fw = ks.forward(mesh, v, Ne, nst, kT)
    G = adj.loss_upstream(mesh, fw["rho"], rho_d, w)
    P, info = adj.adjoint(mesh, v, fw["eps"], fw["psi"], fw["f"], fw["dfde"], G, solver=solver)
    g = adj.gradient(fw["psi"], P, rho_d, -1.0)
    if kT > 0:
        assert abs(info["eta"]) > 1e-6                     # the eta term is exercised
    for _ in range(4):
        dv = rng.standard_normal(mesh.L)
        fd = _fd(mesh, v, dv, rho_d, w, Ne, nst, kT)
        assert abs(fd - g @ dv) <= 1e-6 * abs(fd) + 1e-12


def _degenerate_case():
    """Nucleus at the box centre (a cell vertex): the 2p shell is an exact
    triplet by cubic symmetry; 4 electrons leave it partly filled."""
    mesh = fe.Mesh(-4.0, 4.0, 4, 2)
    xyz = mesh.coords()
    v = W.smeared_coulomb(xyz, np.zeros((1, 3)), np.array([3.0]), 0.5)
    kT, Ne, nst = 0.02, 4.0, 8
    rho_d = ks.forward(mesh, v + 0.05 * np.exp(-np.sum((xyz - 0.4) ** 2, 1)), Ne, nst, kT)["rho"]
    return mesh, v, rho_d, np.ones(mesh.L), kT, Ne, nst


def test_degenerate_shell_gradient_and_rotation_invariance():
    mesh, v, rho_d, w, kT, Ne, nst = _degenerate_case()
    fw = ks.forward(mesh, v, Ne, nst, kT)
    eps = fw["eps"]
    groups = adj.degenerate_groups(eps, 1e-8)
    trip = [g for g in groups if len(g) == 3]
    assert trip, f"expected a triplet, got {eps}"
    G = adj.loss_upstream(mesh, fw["rho"], rho_d, w)
    P, _ = adj.adjoint(mesh, v, eps, fw["psi"], fw["f"], fw["dfde"], G, solver="dense")
    g = adj.gradient(fw["psi"], P, rho_d, -1.0)
    # rotate the degenerate set by a random orthogonal Q (Sec. 2: P~ = P Q)
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    psi2 = fw["psi"].copy()
    psi2[:, trip[0]] = fw["psi"][:, trip[0]] @ Q
    P2, _ = adj.adjoint(mesh, v, eps, psi2, fw["f"], fw["dfde"], G, solver="minres")
    g2 = adj.gradient(psi2, P2, rho_d, -1.0)
    assert np.abs(g - g2).max() < 1e-9 * np.abs(g).max()
    np.testing.assert_allclose(P2[:, trip[0]], P[:, trip[0]] @ Q, atol=1e-8 * np.abs(P).max())
    for _ in range(3):
        dv = rng.standard_normal(mesh.L)
        fd = _fd(mesh, v, dv, rho_d, w, Ne, nst, kT)
        assert abs(fd - g @ dv) <= 1e-6 * abs(fd) + 1e-12


def test_minres_matches_least_squares():
    """Symmetric indefinite system: MINRES = numpy's least-squares solution."""
    rng = np.random.default_rng(2)
    n = 60
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(-3.0, 5.0, n)
    lam[np.abs(lam) < 0.1] = 0.5
    A = Q @ np.diag(lam) @ Q.T
    b = rng.standard_normal(n)
    x, it, rr = adj.minres(lambda z: A @ z, b, 1e-14, 500)
    x_ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.abs(x - x_ref).max() < 1e-10 * np.abs(x_ref).max()
    assert it <= 2 * n                                   # finite-precision Lanczos


def test_loss_definition_and_tau_mask():
    mesh = fe.Mesh(-3.0, 3.0, 2, 2)
    rng = np.random.default_rng(4)
    rho = rng.uniform(size=mesh.L)
    rho_d = rng.uniform(size=mesh.L)
    w = np.ones(mesh.L)
    Lval, e = adj.loss_and_error(mesh, rho, rho_d, w)
    # with w = 1 the loss is e_L2^2 (Eq. 1 vs Sec. 4.2.4)
    assert abs(Lval - e * e) < 1e-14 * Lval
    psi = rng.standard_normal((mesh.L, 2))
    p = rng.standard_normal((mesh.L, 2))
    rho_d[:10] = 1e-9
    g = adj.gradient(psi, p, rho_d, 1e-6)
    assert np.all(g[:10] == 0.0) and np.all(g[10:] != 0.0)


def test_paper_default_tolerances():
    d = json.load(open(os.path.join(GOLDEN, "paper_defaults.json")))
    assert (d["c_eig"], d["c_ad"], d["tau_bc"]) == (1e2, 1e5, 1e-6)


def _bfgs_matrix(S, Y, gamma):
    """Explicit inverse-Hessian recursion H <- (I - r s y^T) H (I - r y s^T) + r s s^T."""
    n = len(S[0])
    H = gamma * np.eye(n)
    for s, y in zip(S, Y):
        r = 1.0 / (y @ s)
        V = np.eye(n) - r * np.outer(y, s)
        H = V.T @ H @ V + r * np.outer(s, s)
    return H


def test_lbfgs_two_loop_equals_bfgs_matrix_and_solves_quadratic():
    rng = np.random.default_rng(8)
    n = 6
    Mq = rng.standard_normal((n, n))
    A = Mq @ Mq.T + n * np.eye(n)
    b = rng.standard_normal(n)
    f = lambda x: 0.5 * x @ A @ x - b @ x
    grad = lambda x: A @ x - b
    x = np.zeros(n)
    hist = lbfgs.History()
    for k in range(n + 1):
        g = grad(x)
        d = lbfgs.direction(g, hist)
        if hist.S:
            gamma = (hist.S[-1] @ hist.Y[-1]) / (hist.Y[-1] @ hist.Y[-1])
            H = _bfgs_matrix(hist.S, hist.Y, gamma)
            np.testing.assert_allclose(d, -H @ g, rtol=1e-10, atol=1e-12)
        # exact line search on the quadratic
        alpha = -(g @ d) / (d @ A @ d)
        x_new = x + alpha * d
        hist.push(x_new - x, grad(x_new) - g)
        x = x_new
        if np.linalg.norm(grad(x)) < 1e-10:
            break
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-8)


def test_chebyshev_closed_form_and_filter():
    x = np.linspace(-3, 3, 41)
    for m in (1, 2, 7, 30):
        c = np.zeros(m + 1)
        c[m] = 1.0
        np.testing.assert_allclose(cheb.cheb_T(m, x), npcheb.chebval(x, c), rtol=1e-9, atol=1e-9)
    # the vector recurrence equals U p_m(Lambda) U^T X on a dense symmetric matrix
    rng = np.random.default_rng(9)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(-1.0, 10.0, n))
    H = Q @ np.diag(lam) @ Q.T
    X = rng.standard_normal((n, 5))
    a, b, a0 = lam[8], lam[-1] + 0.1, lam[0]
    Y = cheb.filter_apply(lambda Z: H @ Z, X, 30, a, b, a0)
    Y_ref = Q @ (cheb.filter_scalar(30, a, b, a0, lam)[:, None] * (Q.T @ X))
    assert np.abs(Y - Y_ref).max() < 1e-9 * np.abs(Y_ref).max()


def test_hartree_matches_gaussian_closed_form():
    """Poisson solve of a Gaussian density vs its exact erf potential."""
    errs = []
    for n in (6, 8):
        mesh = fe.Mesh(-8.0, 8.0, n, 4)
        xyz = mesh.coords()
        rho = W.gaussian_density(xyz, np.zeros((1, 3)), np.array([2.0]), 1.0)
        vh = potentials.hartree(mesh, rho)
        exact = W.gaussian_density_hartree(xyz, np.zeros((1, 3)), np.array([2.0]), 1.0)
        errs.append(np.abs(vh - exact).max())
    assert errs[1] < 5e-3 and errs[1] < errs[0] / 4.0
