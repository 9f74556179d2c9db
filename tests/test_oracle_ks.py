"""Pins of the oracle's Kohn-Sham layer: closed-form spectra, invariants (no GPU)."""
import math

import numpy as np
import pytest
from scipy.linalg import eigh_tridiagonal

import workloads as W
from oracle import fe, ks


def test_particle_in_a_box():
    """v = 0 on [-8,8]^3: E = pi^2 (n1^2+n2^2+n3^2) / (2 W^2), W = 16."""
    mesh = fe.Mesh(-8.0, 8.0, 6, 4)
    eps, psi = ks.lowest_eigenpairs(mesh, np.zeros(mesh.L), 5)
    base = math.pi ** 2 / (2.0 * 16.0 ** 2)
    exact = base * np.array([3, 6, 6, 6, 9])
    np.testing.assert_allclose(eps, exact, rtol=2e-7)
    np.testing.assert_allclose(psi.T @ psi, np.eye(5), atol=1e-10)


def test_harmonic_oscillator_and_convergence():
    """v = r^2/2: E = 3/2, 5/2 (x3); the error falls fast under h-refinement."""
    errs = []
    for n in (6, 8):
        mesh = fe.Mesh(-8.0, 8.0, n, 4)
        v = 0.5 * np.sum(mesh.coords() ** 2, axis=1)
        eps, _ = ks.lowest_eigenpairs(mesh, v, 4)
        errs.append(np.abs(eps - np.array([1.5, 2.5, 2.5, 2.5])).max())
        assert np.ptp(eps[1:]) < 1e-9                       # cubic symmetry: exact triplet
    assert errs[1] < 1e-3
    assert errs[1] < errs[0] / 8.0                          # at least 2^3-fold per (6->8)


def _radial_ground_state(Z, s, R=10.0, n=40000):
    """s-wave -u''/2 + V u = E u, u(0) = u(R) = 0, by second-order finite
    differences on a uniform grid (an independent 1D solver)."""
    h = R / (n + 1)
    r = h * np.arange(1, n + 1)
    V = -Z * np.array([math.erf(x / s) for x in r]) / r
    d = 1.0 / h ** 2 + V
    e = np.full(n - 1, -0.5 / h ** 2)
    w = eigh_tridiagonal(d, e, select="i", select_range=(0, 0), eigvals_only=True)
    return w[0]


def test_hydrogen_like_smeared():
    """-Z erf(r/s)/r with Z = 2, s = 0.5: the FE ground state converges to a fine
    radial solve (the smearing lifts it above the point-charge -Z^2/2 = -2)."""
    Z, s = 2.0, 0.5
    e_rad = _radial_ground_state(Z, s, R=6.0)
    assert -2.0 < e_rad < -1.0
    errs = []
    for n in (6, 8):
        mesh = fe.Mesh(-6.0, 6.0, n, 4)
        v = W.smeared_coulomb(mesh.coords(), np.zeros((1, 3)), np.array([Z]), s)
        eps, _ = ks.lowest_eigenpairs(mesh, v, 1, guard=2)
        errs.append(abs(eps[0] - e_rad))
    assert errs[1] < 5e-3 and errs[1] < errs[0] / 3.0


@pytest.mark.parametrize("kT", [0.0, 1.5834e-3, 0.05])
def test_occupations_and_electron_count(kT):
    mesh = fe.Mesh(-5.0, 5.0, 4, 2)
    v = W.smeared_coulomb(mesh.coords(), np.array([[0.2, 0.0, -0.1]]), np.array([4.0]), 0.5)
    fw = ks.forward(mesh, v, 4.0, 8, kT)
    f = fw["f"]
    assert abs(f.sum() - 4.0) < 1e-12
    assert np.all(f <= 2.0 + 1e-15) and np.all(f >= 0.0)
    assert abs(ks.electron_count(mesh, fw["rho"]) - 4.0) < 1e-12     # Eq. 5
    if kT > 0:
        # f' from the closed form of the derivative equals a centred difference
        h = 1e-7
        eps = fw["eps"]
        for i in range(3):
            e2 = eps.copy(); e2[i] += h
            e1 = eps.copy(); e1[i] -= h
            mu = fw["mu"]
            fp = 2.0 / (1.0 + np.exp((e2[i] - mu) / kT))
            fm = 2.0 / (1.0 + np.exp((e1[i] - mu) / kT))
            assert abs((fp - fm) / (2 * h) - fw["dfde"][i]) < 1e-5 * max(1.0, abs(fw["dfde"][i]))


def test_zero_temperature_mu_is_the_limit_of_the_finite_temperature_one():
    # a gapped spectrum: as kT -> 0 the bisection's mu tends to mid-gap (equal
    # hole and electron tails at the band edges), which is the kT = 0
    # convention of the closed-shell branch.  Temperatures stay above ~gap/40:
    # below that every mu in the gap gives sum f = N_e to machine precision.
    eps = np.array([-2.0, -1.3, -1.25, -0.4, 0.1, 0.7])
    _, _, mu0 = ks.occupations(eps, 6.0, 0.0)
    dev = []
    for kT in (0.05, 0.03, 0.02):
        f, _, mu = ks.occupations(eps, 6.0, kT)
        assert abs(f.sum() - 6.0) < 1e-12
        dev.append(abs(mu - mu0))
        assert dev[-1] < 0.5 * kT
    assert dev[0] > dev[1] > dev[2]
    assert abs(mu0 - 0.5 * (-1.25 - 0.4)) < 1e-15
