"""Loss, adjoint solve and gradient (oracle; test infrastructure only).

Notation follows Sec. 2 and Sec. 3.2 of the paper, in the standard form of
Eq. 19-20 (tilde quantities; psi~ = M^1/2 psi, p~ = M^1/2 p, M = diag(m)).

* Loss (Eq. 1) by GLL quadrature over the unknown nodes:
      L = sum_a m_a w_a (rho_data,a - rho_a)^2,
  and e_L2 = sqrt(sum_a m_a (rho_data,a - rho_a)^2) (Sec. 4.2.4).
* Generic upstream: for any loss with dL/drho_a = G_a define
      omega_a = -G_a / (2 m_a)
  so that omega = w (rho_data - rho) for the paper's loss.  Every formula below
  is the paper's with w (rho_data - rho) replaced by omega.
* Right-hand side (Eq. 7, 18, 20): b_i = 4 f_i omega o psi~_i; the multiplier
  term Psi_k (D_k + D_k^T) with D_k + D_k^T from Eq. 10 removes exactly the
  component of b_i along the degenerate set Psi_k, so g~_i = (I - Psi_k Psi_k^T) b_i.
* (H~ - eps_i) p~_perp = g~_i on the complement of Psi_k (Sec. 3.2.2), solved by
  MINRES (Paige & Saunders 1975) with the operator projected at every step.
  The oracle runs MINRES without a preconditioner; the result is the unique
  solution in the complement, whatever the solver.
* Component along Psi_k (Eq. 8, 9):
      eta = 2 sum_i f'_i (psi~_i^T omega psi~_i) / sum_i f'_i,   (0 if sum f' = 0)
      Psi_k^T p~_i = f'_i ( -2 [Psi_k^T diag(omega) Psi_k]_{:, i} + eta e_i ),
  with f'_i = d f_i / d eps_i of the spin-factor-2 occupation.
* Gradient (Eq. 11, 22, GLL collocation): grad_b = sum_i p~_bi psi~_bi, set to
  zero where rho_data,b < tau_BC (Sec. 3.1.2).

Pinned by central finite differences of the discrete loss (tests), at kT = 0
and kT > 0, and by rotating a degenerate set (gradient invariance, Sec. 2).
"""
from __future__ import annotations

import numpy as np

from .fe import Mesh


def loss_and_error(mesh: Mesh, rho: np.ndarray, rho_data: np.ndarray, w: np.ndarray):
    """(L, e_L2) of Eq. 1 and Sec. 4.2.4 by GLL quadrature."""
    m = mesh.mass()
    d = rho_data - rho
    return float(np.sum(m * w * d * d)), float(np.sqrt(np.sum(m * d * d)))


def loss_upstream(mesh: Mesh, rho: np.ndarray, rho_data: np.ndarray, w: np.ndarray):
    """dL/drho_a = -2 m_a w_a (rho_data,a - rho_a)."""
    return -2.0 * mesh.mass() * w * (rho_data - rho)


def degenerate_groups(eps: np.ndarray, tol: float):
    """Consecutive runs of ascending eigenvalues closer than tol."""
    groups, cur = [], [0]
    for i in range(1, len(eps)):
        if eps[i] - eps[i - 1] < tol:
            cur.append(i)
        else:
            groups.append(cur)
            cur = [i]
    groups.append(cur)
    return groups


def minres(apply_A, b: np.ndarray, tol: float, maxit: int):
    """MINRES for a symmetric (possibly indefinite) operator, x0 = 0.

    Lanczos tridiagonalisation with the QR factorisation of the (k+1) x k
    tridiagonal matrix updated by Givens rotations; x_k minimises ||b - A x||
    over the Krylov space.  Stops when the recurrence residual
    |phibar| <= tol ||b||.  Returns (x, iterations, relative residual).
    """
    x = np.zeros_like(b)
    beta1 = float(np.linalg.norm(b))
    if beta1 == 0.0:
        return x, 0, 0.0
    v_prev = np.zeros_like(b)
    v = b / beta1
    beta = 0.0                       # T(k-1, k)
    c_pp, s_pp, c_p, s_p = 1.0, 0.0, 1.0, 0.0
    w_pp = np.zeros_like(b)
    w_p = np.zeros_like(b)
    phibar = beta1
    k = 0
    for k in range(1, maxit + 1):
        Av = apply_A(v)
        alpha = float(v @ Av)
        pv = Av - alpha * v - beta * v_prev
        beta_next = float(np.linalg.norm(pv))
        eps_k = s_pp * beta
        tmp = c_pp * beta
        delta = c_p * tmp + s_p * alpha
        gbar = -s_p * tmp + c_p * alpha
        gamma = float(np.hypot(gbar, beta_next))
        c, s = gbar / gamma, beta_next / gamma
        t = c * phibar
        phibar = -s * phibar
        wv = (v - eps_k * w_pp - delta * w_p) / gamma
        x = x + t * wv
        w_pp, w_p = w_p, wv
        c_pp, s_pp, c_p, s_p = c_p, s_p, c, s
        v_prev = v
        if beta_next == 0.0:
            break
        v = pv / beta_next
        beta = beta_next
        if abs(phibar) <= tol * beta1:
            break
    return x, k, abs(phibar) / beta1


def adjoint(mesh: Mesh, v: np.ndarray, eps: np.ndarray, psi: np.ndarray, f: np.ndarray,
            dfde: np.ndarray, dL_drho: np.ndarray, deg_tol: float = 1e-8,
            tol: float = 1e-13, maxit: int = 5000, occ_cut: float = 1e-14,
            solver: str = "minres"):
    """Adjoint functions p~ [L, nstates] for the upstream dL/drho (Eq. 7-10, 20).

    States with f_i <= occ_cut and f'_i == 0 carry p~_i = 0.
    solver = "dense" uses a dense eigen-decomposition of H~ (small meshes) in
    place of MINRES for a brute-force cross-check.
    Returns (p, info) with info = dict(eta, iters).
    """
    m = mesh.mass()
    omega = -dL_drho / (2.0 * m)
    nst = psi.shape[1]
    diag_I = np.einsum("ai,a,ai->i", psi, omega, psi)         # psi_i^T omega psi_i
    sdf = float(np.sum(dfde))
    eta = 2.0 * float(np.dot(dfde, diag_I)) / sdf if sdf != 0.0 else 0.0
    P = np.zeros_like(psi)
    iters = np.zeros(nst, dtype=np.int64)
    dense = None
    if solver == "dense":
        Hd = mesh.assemble_Htilde(v).toarray()
        lam, U = np.linalg.eigh(Hd)
    for grp in degenerate_groups(eps, deg_tol):
        Pk = psi[:, grp]
        J = Pk.T @ (omega[:, None] * Pk)                       # Psi_k^T omega Psi_k
        for li, i in enumerate(grp):
            if f[i] <= occ_cut and dfde[i] == 0.0:
                continue
            b = 4.0 * f[i] * omega * psi[:, i]
            g = b - Pk @ (Pk.T @ b)
            if solver == "dense":
                # pseudo-inverse of (H~ - eps_i) on the complement of Psi_k
                coef = U.T @ g
                denom = lam - eps[i]
                null = np.abs(denom) < max(deg_tol, 1e-9)       # the eigenspace of eps_i
                coef = np.where(null, 0.0, coef / np.where(null, 1.0, denom))
                p_perp = U @ coef
                p_perp -= Pk @ (Pk.T @ p_perp)
                it = 0
            else:
                def op(x, ei=eps[i], Pk=Pk):
                    x = x - Pk @ (Pk.T @ x)
                    y = mesh.apply_Htilde(v, x) - ei * x
                    return y - Pk @ (Pk.T @ y)
                p_perp, it, _ = minres(op, g, tol, maxit)
                p_perp -= Pk @ (Pk.T @ p_perp)
            e_i = np.zeros(len(grp))
            e_i[li] = 1.0
            d = dfde[i] * (-2.0 * J[:, li] + eta * e_i)
            P[:, i] = p_perp + Pk @ d
            iters[i] = it
    return P, dict(eta=eta, iters=iters)


def gradient(psi: np.ndarray, p: np.ndarray, rho_data: np.ndarray, tau_bc: float):
    """grad_b = sum_i p~_bi psi~_bi (Eq. 11, 22), zero where rho_data < tau_BC."""
    g = np.sum(p * psi, axis=1)
    g[rho_data < tau_bc] = 0.0
    return g
