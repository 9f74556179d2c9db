"""Initial guess of the exchange-correlation potential (oracle; test infrastructure only).

Sec. 4.2.3, Eq. 25 and Eq. 26:

    v_xc^init = f v0[rho_d] + (1 - f) alpha v_FA[rho_d],   f = rho_d / (rho_d + tau),
    v_FA[rho] = -v_H[rho] / N_e                (Fermi-Amaldi),
    v0[rho]   = v_x[rho] + v_c^PW92[rho],

with v_x the Slater (LDA) exchange potential or the LB94 exchange potential.
The paper suggests tau = 1e-2 and LB94.  f moves the guess from v0 in the
high-density region to the scaled Fermi-Amaldi potential, which decays as
-alpha / r, where rho_d < tau.

The two functionals are restated from their published definitions:
  * PW92 (Perdew and Wang, 1992): the correlation energy per electron of the
    spin-unpolarised uniform gas,
        eps_c(r_s) = -2 A (1 + a1 r_s) ln(1 + 1 / (2 A (b1 r_s^1/2 + b2 r_s
                                                       + b3 r_s^3/2 + b4 r_s^2))),
    r_s = (3 / (4 pi rho))^1/3, with the published (A, a1, b1..b4); the
    potential is v_c = d(rho eps_c)/d rho = eps_c - (r_s / 3) d eps_c / d r_s.
  * LB94 (van Leeuwen and Baerends, 1994): per spin density rho_s = rho / 2
    (closed shell), v_x = v_x^LDA(rho) - beta rho_s^1/3 x^2 / (1 + 3 beta x
    asinh x), x = |grad rho_s| / rho_s^4/3, beta = 0.05.  For an
    exponentially decaying density the correction tends to -1/r.

The nodal density gradient that LB94 needs is the gradient of the finite-
element interpolant of rho at the GLL nodes (1D derivative matrices per cell),
averaged over the cells that share a node; rho is zero on the Dirichlet
boundary.  A reading: the paper does not say how the gradient is evaluated.

Parity status: pinned (tests/test_oracle_initial_guess.py) by the exact
high-density coefficient of PW92, agreement with the independent Perdew-Zunger
1981 fit of the same QMC data, v_c against a finite difference of rho eps_c,
the -1/r tail of LB94 on an exponential density, exactness of the nodal
gradient on polynomials of degree <= p, and the limits of Eq. 25.
"""
from __future__ import annotations

import math

import numpy as np

from .fe import Mesh, gll_rule, lagrange_derivs
from .potentials import hartree

# PW92, spin-unpolarised correlation (Perdew and Wang 1992, p = 1)
PW92_A = 0.031091
PW92_A1 = 0.21370
PW92_B1, PW92_B2, PW92_B3, PW92_B4 = 7.5957, 3.5876, 1.6382, 0.49294
LB94_BETA = 0.05


def wigner_seitz_radius(rho: np.ndarray) -> np.ndarray:
    """r_s = (3 / (4 pi rho))^(1/3); inf where rho <= 0."""
    rho = np.asarray(rho, dtype=np.float64)
    out = np.full(rho.shape, np.inf)
    pos = rho > 0.0
    out[pos] = np.cbrt(3.0 / (4.0 * math.pi * rho[pos]))
    return out


def pw92_eps_c(rs: np.ndarray) -> np.ndarray:
    """Correlation energy per electron eps_c(r_s) (Hartree); 0 at r_s = inf."""
    rs = np.asarray(rs, dtype=np.float64)
    out = np.zeros(rs.shape)
    ok = np.isfinite(rs)
    r = rs[ok]
    q1 = 2.0 * PW92_A * (PW92_B1 * np.sqrt(r) + PW92_B2 * r + PW92_B3 * r ** 1.5 + PW92_B4 * r ** 2)
    out[ok] = -2.0 * PW92_A * (1.0 + PW92_A1 * r) * np.log1p(1.0 / q1)
    return out


def pw92_deps_drs(rs: np.ndarray) -> np.ndarray:
    """d eps_c / d r_s, differentiated term by term."""
    rs = np.asarray(rs, dtype=np.float64)
    out = np.zeros(rs.shape)
    ok = np.isfinite(rs)
    r = rs[ok]
    q0 = -2.0 * PW92_A * (1.0 + PW92_A1 * r)
    q1 = 2.0 * PW92_A * (PW92_B1 * np.sqrt(r) + PW92_B2 * r + PW92_B3 * r ** 1.5 + PW92_B4 * r ** 2)
    dq1 = PW92_A * (PW92_B1 / np.sqrt(r) + 2.0 * PW92_B2 + 3.0 * PW92_B3 * np.sqrt(r)
                    + 4.0 * PW92_B4 * r)
    # d/dr [q0 ln(1 + 1/q1)] = q0' ln(1 + 1/q1) - q0 q1' / (q1^2 + q1)
    out[ok] = -2.0 * PW92_A * PW92_A1 * np.log1p(1.0 / q1) - q0 * dq1 / (q1 * q1 + q1)
    return out


def pw92_v_c(rho: np.ndarray) -> np.ndarray:
    """PW92 correlation potential v_c = eps_c - (r_s / 3) d eps_c / d r_s (0 where rho <= 0)."""
    rs = wigner_seitz_radius(rho)
    out = np.zeros(rs.shape)
    ok = np.isfinite(rs)
    out[ok] = pw92_eps_c(rs[ok]) - rs[ok] / 3.0 * pw92_deps_drs(rs[ok])
    return out


def slater_exchange(rho: np.ndarray) -> np.ndarray:
    """LDA (Slater) exchange potential -(3 rho / pi)^(1/3), rho clamped at 0."""
    return -np.cbrt(3.0 * np.maximum(np.asarray(rho, dtype=np.float64), 0.0) / math.pi)


def lb94_exchange(rho: np.ndarray, grad_norm: np.ndarray) -> np.ndarray:
    """LB94 exchange potential of a closed-shell density from rho and |grad rho|.

    Per spin: rho_s = rho / 2, |grad rho_s| = |grad rho| / 2.  Where rho <= 0 the
    gradient correction is taken as 0 (the guess uses v_FA there, f = 0).
    """
    rho = np.asarray(rho, dtype=np.float64)
    g = np.asarray(grad_norm, dtype=np.float64)
    v = slater_exchange(rho)
    pos = rho > 0.0
    rs_ = 0.5 * rho[pos]
    x = 0.5 * g[pos] / rs_ ** (4.0 / 3.0)
    v[pos] -= LB94_BETA * np.cbrt(rs_) * x * x / (1.0 + 3.0 * LB94_BETA * x * np.arcsinh(x))
    return v


def nodal_gradient(mesh: Mesh, f: np.ndarray) -> np.ndarray:
    """[L, 3] gradient of the FE interpolant of f (interior nodes; zero on the
    boundary) at the interior nodes, averaged over the cells sharing a node."""
    p, n, N = mesh.p, mesh.n, mesh.N
    xi, _ = gll_rule(p)
    D = lagrange_derivs(xi, xi) * (2.0 / mesh.h)        # D[i, j] = l_j'(x_i) in physical units
    F = mesh.to_full(np.asarray(f, dtype=np.float64).reshape(-1, 1))[:, 0].reshape(N, N, N)
    grad = np.zeros((3, N, N, N))
    count = np.zeros((N, N, N))
    for cz in range(n):
        for cy in range(n):
            for cx in range(n):
                sl = (slice(cz * p, cz * p + p + 1), slice(cy * p, cy * p + p + 1),
                      slice(cx * p, cx * p + p + 1))
                Fe = F[sl]                                    # [z, y, x]
                grad[0][sl] += np.einsum("ij,zyj->zyi", D, Fe)
                grad[1][sl] += np.einsum("ij,zjx->zix", D, Fe)
                grad[2][sl] += np.einsum("ij,jyx->iyx", D, Fe)
                count[sl] += 1.0
    grad /= count[None]
    inner = (slice(1, -1),) * 3
    return np.stack([grad[d][inner].ravel() for d in range(3)], axis=1)


def fermi_amaldi(mesh: Mesh, rho: np.ndarray, n_electrons: float, v_H: np.ndarray | None = None):
    """v_FA = -v_H[rho] / N_e (v_H from the FE Poisson solve unless given)."""
    if v_H is None:
        v_H = hartree(mesh, rho)
    return -np.asarray(v_H) / float(n_electrons)


def initial_guess(mesh: Mesh, rho_d: np.ndarray, n_electrons: float, tau: float = 1e-2,
                  alpha: float = 1.0, exchange: str = "lb94", v_H: np.ndarray | None = None):
    """v_xc^init of Eq. 25 at the interior nodes; returns (v_init, parts)."""
    rho = np.maximum(np.asarray(rho_d, dtype=np.float64), 0.0)
    if exchange == "lb94":
        g = nodal_gradient(mesh, rho)
        v_x = lb94_exchange(rho, np.linalg.norm(g, axis=1))
    elif exchange == "slater":
        v_x = slater_exchange(rho)
    else:
        raise ValueError("exchange must be 'lb94' or 'slater'")
    v0 = v_x + pw92_v_c(rho)
    v_fa = fermi_amaldi(mesh, rho, n_electrons, v_H)
    f = rho / (rho + tau)
    v = f * v0 + (1.0 - f) * alpha * v_fa
    return v, dict(v0=v0, v_x=v_x, v_fa=v_fa, f=f)
