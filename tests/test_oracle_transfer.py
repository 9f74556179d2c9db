"""Pins of the Q1 v_xc mesh and the field transfer: exact trilinear transfer,
partition of unity, second-order convergence, and the gradient through the
transfer against finite differences of the loss in the Q1 coefficients."""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import workloads as W  # noqa: E402
from oracle import adjoint as adj  # noqa: E402
from oracle import fe, ks  # noqa: E402
from oracle.transfer import Q1Mesh, gradient_to_q1, to_orbital_mesh  # noqa: E402


def test_trilinear_fields_transfer_exactly():
    q1 = Q1Mesh(-4.0, 4.0, 5)
    mesh = fe.Mesh(-4.0, 4.0, 3, 4)
    T = q1.transfer_matrix(mesh.coords())
    f = lambda p: (0.4 + 0.3 * p[:, 0]) * (1.0 - 0.2 * p[:, 1]) * (0.7 + 0.1 * p[:, 2])
    np.testing.assert_allclose(to_orbital_mesh(T, f(q1.coords())), f(mesh.coords()),
                               rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(np.asarray(T.sum(axis=1)).ravel(), 1.0, atol=1e-14)
    assert T.nnz <= 8 * mesh.L
    # a point is interpolated within its own cell: a convex combination
    assert T.data.min() >= -1e-15
    pts = np.random.default_rng(5).uniform(-4.0, 4.0, size=(500, 3))
    assert q1.transfer_matrix(pts).data.min() >= -1e-15


def test_transfer_converges_at_second_order():
    # scattered points (orbital nodes can coincide with Q1 nodes, which hides the rate)
    pts = np.random.default_rng(11).uniform(-4.0, 4.0, size=(4000, 3))
    g = lambda p: np.exp(-0.3 * np.sum((p - 0.25) ** 2, axis=1))
    errs = []
    for nv in (8, 16, 32):
        q1 = Q1Mesh(-4.0, 4.0, nv)
        T = q1.transfer_matrix(pts)
        errs.append(np.sqrt(np.mean((to_orbital_mesh(T, g(q1.coords())) - g(pts)) ** 2)))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_gradient_through_the_transfer_matches_finite_differences():
    mesh = fe.Mesh(-4.0, 4.0, 3, 2)
    xyz = mesh.coords()
    rng = np.random.default_rng(7)
    Ne, nst, kT = 2.0, 4, 0.0
    v_fixed = W.smeared_coulomb(xyz, np.array([[0.3, -0.2, 0.1]]), np.array([2.0]), 0.5)
    q1 = Q1Mesh(-4.0, 4.0, 4)
    T = q1.transfer_matrix(xyz)
    v_q1 = 0.05 * rng.standard_normal(q1.n_nodes)
    rho_d = ks.forward(mesh, v_fixed + 0.1 * np.exp(-np.sum(xyz ** 2, 1)), Ne, nst, kT)["rho"]
    w = np.ones(mesh.L)

    def loss(vq):
        fw = ks.forward(mesh, v_fixed + to_orbital_mesh(T, vq), Ne, nst, kT)
        return adj.loss_and_error(mesh, fw["rho"], rho_d, w)[0]

    v = v_fixed + to_orbital_mesh(T, v_q1)
    fw = ks.forward(mesh, v, Ne, nst, kT)
    G = adj.loss_upstream(mesh, fw["rho"], rho_d, w)
    P, _ = adj.adjoint(mesh, v, fw["eps"], fw["psi"], fw["f"], fw["dfde"], G)
    g_q1 = gradient_to_q1(T, adj.gradient(fw["psi"], P, rho_d, -1.0))
    for _ in range(3):
        d = rng.standard_normal(q1.n_nodes)
        cd = lambda h: (loss(v_q1 + h * d) - loss(v_q1 - h * d)) / (2.0 * h)
        fd = (4.0 * cd(5e-4) - cd(1e-3)) / 3.0
        assert abs(fd - g_q1 @ d) <= 1e-6 * abs(fd) + 1e-12
