"""Pins of the initial-guess oracle (Eq. 25, Eq. 26) against facts other than
itself: the exact high-density coefficient of the correlation energy, the
independent Perdew-Zunger 1981 fit of the same quantum Monte Carlo data,
thermodynamic consistency of the potential, the -1/r tail of LB94, exactness of
the nodal gradient on polynomials, and the limits of the partition f."""
from __future__ import annotations

import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from oracle import fe, initial_guess as ig  # noqa: E402


def _pz81_eps_c(rs):
    """Perdew-Zunger 1981 fit of the Ceperley-Alder correlation energy
    (unpolarised, Hartree): a different functional form and constants."""
    rs = np.asarray(rs, dtype=np.float64)
    high = 0.0311 * np.log(rs) - 0.048 + 0.0020 * rs * np.log(rs) - 0.0116 * rs
    low = -0.1423 / (1.0 + 1.0529 * np.sqrt(rs) + 0.3334 * rs)
    return np.where(rs >= 1.0, low, high)


def test_pw92_high_density_coefficient_is_exact():
    # eps_c -> A ln r_s + const as r_s -> 0, with A = (1 - ln 2)/pi^2 exactly
    # (random-phase high-density limit); the published A carries 5 digits
    assert abs(ig.PW92_A - (1.0 - math.log(2.0)) / math.pi ** 2) < 5e-7
    rs = np.array([1e-6, 1e-7])
    slope = np.diff(ig.pw92_eps_c(rs)) / np.diff(np.log(rs))
    assert abs(slope[0] - (1.0 - math.log(2.0)) / math.pi ** 2) < 2e-5


def test_pw92_agrees_with_the_perdew_zunger_fit():
    rs = np.array([0.1, 0.3, 0.5, 1.0, 2.0, 3.0, 5.0, 10.0, 20.0, 50.0])
    e = ig.pw92_eps_c(rs)
    ref = _pz81_eps_c(rs)
    assert np.all(e < 0.0)
    assert np.all(np.diff(e) > 0.0)          # less negative as the gas thins out
    assert np.max(np.abs(e - ref) / np.abs(ref)) < 0.01


def test_pw92_potential_is_the_derivative_of_the_energy_density():
    rho = np.geomspace(1e-6, 1e2, 25)
    h = 1e-6 * rho
    e = lambda r: r * ig.pw92_eps_c(ig.wigner_seitz_radius(r))
    fd = (e(rho + h) - e(rho - h)) / (2.0 * h)
    v = ig.pw92_v_c(rho)
    assert np.max(np.abs(fd - v) / np.abs(v)) < 1e-7
    assert np.all(ig.pw92_v_c(np.array([0.0, -1.0])) == 0.0)


def test_slater_exchange_is_the_lda_derivative():
    # v_x = d(rho eps_x)/d rho with eps_x = -(3/4)(3 rho/pi)^(1/3)
    rho = np.geomspace(1e-6, 1e2, 20)
    h = 1e-6 * rho
    e = lambda r: -0.75 * r * np.cbrt(3.0 * r / math.pi)
    fd = (e(rho + h) - e(rho - h)) / (2.0 * h)
    assert np.max(np.abs(fd - ig.slater_exchange(rho)) / np.abs(fd)) < 1e-8


def test_lb94_tail_is_minus_one_over_r():
    # closed-shell rho = 2 exp(-2 r): per spin rho_s = exp(-2 r), |grad rho_s| = 2 rho_s.
    # The gradient correction tends to -1/r; the LDA part vanishes exponentially.
    r = np.array([10.0, 20.0, 40.0, 80.0])
    rho = 2.0 * np.exp(-2.0 * r)
    v = ig.lb94_exchange(rho, 2.0 * rho)
    dev = np.abs(r * v + 1.0)
    assert np.all(np.diff(dev) < 0.0)
    # leading deviation ~ 3 ln(2 a) / (a r) for rho_s = exp(-a r), a = 2
    assert np.all(dev < 1.5 * 3.0 * math.log(4.0) / (2.0 * r))
    # small reduced gradient: the correction is -beta rho_s^(1/3) x^2
    rho1 = np.array([1.0])
    g = np.array([1e-4])
    x = 0.5 * g[0] / 0.5 ** (4.0 / 3.0)
    corr = ig.lb94_exchange(rho1, g) - ig.slater_exchange(rho1)
    assert abs(corr[0] / (-0.05 * 0.5 ** (1.0 / 3.0) * x * x) - 1.0) < 1e-6


@pytest.mark.parametrize("p", [2, 4])
def test_nodal_gradient_is_exact_on_polynomials(p):
    mesh = fe.Mesh(-1.0, 1.0, 3, p)
    xyz = mesh.coords()
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    # vanishes on the boundary and has degree <= p per coordinate
    b = lambda t: 1.0 - t * t
    f = b(x) * b(y) * b(z) * (0.3 + 0.5 * x - 0.2 * y + (0.4 * z if p >= 3 else 0.0))
    g = ig.nodal_gradient(mesh, f)
    if p >= 3:
        gx = -2 * x * b(y) * b(z) * (0.3 + 0.5 * x - 0.2 * y + 0.4 * z) + 0.5 * b(x) * b(y) * b(z)
        gy = -2 * y * b(x) * b(z) * (0.3 + 0.5 * x - 0.2 * y + 0.4 * z) - 0.2 * b(x) * b(y) * b(z)
        gz = -2 * z * b(x) * b(y) * (0.3 + 0.5 * x - 0.2 * y + 0.4 * z) + 0.4 * b(x) * b(y) * b(z)
    else:
        f = b(x) * b(y) * b(z)
        g = ig.nodal_gradient(mesh, f)
        gx, gy, gz = -2 * x * b(y) * b(z), -2 * y * b(x) * b(z), -2 * z * b(x) * b(y)
    assert np.max(np.abs(g - np.stack([gx, gy, gz], axis=1))) < 1e-11


def test_nodal_gradient_converges_on_a_gaussian():
    # order-4 interpolant: the nodal gradient error falls like h^4 (16x per
    # halving asymptotically; 10.5x between h = 1.5 and 0.75 here)
    errs = []
    for n in (8, 16):
        mesh = fe.Mesh(-6.0, 6.0, n, 4)
        xyz = mesh.coords()
        r2 = np.sum(xyz ** 2, axis=1)
        f = np.exp(-r2)
        g = ig.nodal_gradient(mesh, f)
        errs.append(np.max(np.abs(g + 2.0 * xyz * f[:, None])))
    assert errs[1] < errs[0] / 8.0


def test_initial_guess_limits():
    mesh = fe.Mesh(-6.0, 6.0, 4, 2)
    xyz = mesh.coords()
    r = np.linalg.norm(xyz, axis=1)
    rho = 2.0 * (8.0 / math.pi) ** 1.5 / 8.0 * np.exp(-2.0 * r * r)   # ~2 electrons
    rho[r > 4.0] = 0.0
    tau = 1e-2
    v, parts = ig.initial_guess(mesh, rho, 2.0, tau=tau, alpha=0.8, exchange="lb94")
    f = parts["f"]
    assert np.all((f >= 0.0) & (f < 1.0))
    zero = rho == 0.0
    assert zero.any()
    np.testing.assert_allclose(v[zero], 0.8 * parts["v_fa"][zero], rtol=0, atol=1e-15)
    # where rho >> tau the guess is v0 up to a weight tau / (rho + tau) on v_FA
    dense = rho > 50.0 * tau
    assert dense.any()
    dev = np.abs(v[dense] - parts["v0"][dense]) / np.abs(parts["v0"][dense] - 0.8 * parts["v_fa"][dense])
    assert np.all(dev <= tau / (rho[dense] + tau) * (1.0 + 1e-12))
    assert np.all(dev < 0.02)
    # Fermi-Amaldi: -v_H / N_e
    np.testing.assert_allclose(parts["v_fa"] * 2.0, -ig.hartree(mesh, rho), rtol=1e-12, atol=1e-14)
