"""Kohn-Sham eigenpairs, occupations and density (oracle; test infrastructure only).

* Eigenpairs of the standard-form problem H~ psi~ = eps psi~ (Eq. 19), the
  lowest nstates of them.  The paper finds them with Chebyshev-filtered subspace
  iteration (Sec. 3.2.2); the oracle deliberately uses a different route with
  the same plain definition: a dense symmetric eigensolver (LAPACK via numpy)
  when L is small, otherwise implicitly restarted Lanczos (ARPACK via scipy).
* Occupations f_i = 2 / (1 + exp((eps_i - mu)/kT)) (Eq. 4 with the factor 2 of
  the spin-restricted formalism, so that sum f = N_e holds as in Eq. 5), with mu
  found by bisection on sum_i f_i = N_e.  kT = 0 fills the lowest N_e/2 states
  with 2 electrons each.
* Density at node a: rho_a = sum_i f_i psi~_ai^2 / m_a (Eq. 4 evaluated at the
  GLL nodes; psi = M^-1/2 psi~).  Then int rho = sum_a m_a rho_a = sum_i f_i.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla
from scipy.special import expit

from .fe import Mesh


def lowest_eigenpairs(mesh: Mesh, v: np.ndarray, nstates: int, dense_limit: int = 1500,
                      tol: float = 1e-13, guard: int = 8):
    """Lowest nstates eigenpairs of H~ = D K D + diag(v), ascending.

    Returns (eps [nstates], psi [L, nstates]) with orthonormal columns.
    """
    H = mesh.assemble_Htilde(v) if mesh.L <= 400_000 else None
    if mesh.L <= dense_limit:
        w, U = np.linalg.eigh(H.toarray())
        return w[:nstates].copy(), U[:, :nstates].copy()
    op = H if H is not None else spla.LinearOperator(
        (mesh.L, mesh.L), matvec=lambda x: mesh.apply_Htilde(v, x), dtype=np.float64)
    # extra Ritz pairs guard against Lanczos missing members of degenerate sets
    k = min(nstates + guard, mesh.L - 1)
    w, U = spla.eigsh(op, k=k, which="SA", tol=tol, ncv=min(max(2 * k + 1, 48), mesh.L))
    order = np.argsort(w)[:nstates]
    return w[order], U[:, order]


def occupations(eps: np.ndarray, n_electrons: float, kT: float, max_iter: int = 400):
    """Fermi-Dirac occupations with spin factor 2 and chemical potential.

    Returns (f, dfde, mu): f_i, df_i/deps_i (mu held fixed) and mu.
    """
    eps = np.asarray(eps, dtype=np.float64)
    if kT == 0.0:
        nocc = int(round(n_electrons / 2.0))
        if abs(2 * nocc - n_electrons) > 1e-12 or nocc > len(eps):
            raise ValueError("kT = 0 needs an even electron count and enough states")
        f = np.zeros_like(eps)
        f[:nocc] = 2.0
        mu = 0.5 * (eps[nocc - 1] + eps[nocc]) if nocc < len(eps) else eps[-1]
        return f, np.zeros_like(eps), mu

    def total(mu):
        return np.sum(2.0 * expit(-(eps - mu) / kT))

    lo, hi = eps.min() - 50.0 * kT - 1.0, eps.max() + 50.0 * kT + 1.0
    if total(hi) < n_electrons:
        raise ValueError("not enough states for the electron count")
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        if total(mid) < n_electrons:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 4e-16 * max(1.0, abs(mid)):
            break
    mu = 0.5 * (lo + hi)
    s = expit(-(eps - mu) / kT)
    f = 2.0 * s
    dfde = -(2.0 / kT) * s * (1.0 - s)
    return f, dfde, mu


def density(mesh: Mesh, psi: np.ndarray, f: np.ndarray) -> np.ndarray:
    """rho_a = sum_i f_i psi~_ai^2 / m_a over interior nodes (Eq. 4)."""
    return (psi ** 2 @ f) / mesh.mass()


def electron_count(mesh: Mesh, rho: np.ndarray) -> float:
    """int rho by GLL quadrature: sum_a m_a rho_a (Eq. 5)."""
    return float(np.dot(mesh.mass(), rho))


def forward(mesh: Mesh, v: np.ndarray, n_electrons: float, nstates: int, kT: float):
    """One Kohn-Sham solve at total potential v: eps, psi~, f, f', mu, rho."""
    eps, psi = lowest_eigenpairs(mesh, v, nstates)
    f, dfde, mu = occupations(eps, n_electrons, kT)
    rho = density(mesh, psi, f)
    return dict(eps=eps, psi=psi, f=f, dfde=dfde, mu=mu, rho=rho)
