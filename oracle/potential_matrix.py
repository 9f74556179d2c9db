"""Dense per-cell potential matrices (oracle; test infrastructure only).

Eq. 17 gives the potential part of H as V_ab = int N_a v N_b.  The default
reading of this build integrates it with the GLL rule that makes M diagonal
(Sec. 3.2.1), which collocates the potential: V = diag(m o v).  The alternative
reading integrates it with a Gauss-Legendre rule of n_g points per axis on each
cell, for the finite-element interpolant of v, which gives one dense
n_e x n_e matrix per cell (n_e = (p+1)^3):

    V_e[a, b] = sum_g W_g v(x_g) N_a(x_g) N_b(x_g),
    W_g = (h/2)^3 w_gx w_gy w_gz,   v(x_g) = sum_c v_c N_c(x_g)  (the cell's nodes).

The standard form keeps the lumped GLL mass: H~ = D (K + V) D, D = M^-1/2.
The potential enters through all nodes of a cell, the Dirichlet boundary
nodes included, so v is given on the full node grid.

Parity status: pinned (tests/test_oracle_potential_matrix.py) by the
consistent mass matrix for a constant potential, by reducing to the
collocation operator of oracle.fe.Mesh when the rule is the GLL rule itself,
by exact integrals of polynomial potentials and fields, and by symmetry and
definiteness.
"""
from __future__ import annotations

import numpy as np

from .fe import Mesh, gauss_rule, gll_rule, lagrange_values


def cell_potential_matrices(mesh: Mesh, v_full: np.ndarray, ng: int | None = None,
                            rule: str = "gauss") -> np.ndarray:
    """[ncell^3, n_e, n_e] matrices V_e in the (z, y, x) local order of K_e.

    rule = "gauss": n_g-point Gauss-Legendre, exact for integrands of degree
    <= 2 n_g - 1 per axis; the default n_g = 2p covers N_a v N_b (degree 3p)
    for the interpolated v.  rule = "gll": the (p+1)-point GLL rule of the
    nodes themselves.
    """
    p, q, n, N = mesh.p, mesh.q, mesh.n, mesh.N
    xi, _ = gll_rule(p)
    if rule == "gauss":
        xg, wg = gauss_rule(ng if ng is not None else 2 * p)
    elif rule == "gll":
        xg, wg = gll_rule(p)
    else:
        raise ValueError("rule must be 'gauss' or 'gll'")
    phi = lagrange_values(xi, xg)                   # [g, a]: l_a(x_g)
    s = 0.5 * mesh.h
    V = np.asarray(v_full, dtype=np.float64).reshape(N, N, N)
    ne = q ** 3
    out = np.empty((n * n * n, ne, ne))
    # tensor-product basis at the quadrature points: Phi[g, a] over (z, y, x)
    Phi = np.einsum("zk,yj,xi->zyxkji", phi, phi, phi).reshape(len(xg) ** 3, ne)
    W = (s ** 3) * np.einsum("z,y,x->zyx", wg, wg, wg).ravel()
    c = 0
    for cz in range(n):
        for cy in range(n):
            for cx in range(n):
                ve = V[cz * p:cz * p + q, cy * p:cy * p + q, cx * p:cx * p + q].ravel()
                vg = Phi @ ve                                    # v at the points
                out[c] = (Phi * (W * vg)[:, None]).T @ Phi
                c += 1
    return out


def apply_V_full(mesh: Mesh, Ve: np.ndarray, Xf: np.ndarray) -> np.ndarray:
    """sum over cells of G_e^T V_e G_e X over all nodes (X: [N^3, ncol])."""
    p, q, n, N = mesh.p, mesh.q, mesh.n, mesh.N
    ncol = Xf.shape[1]
    X = Xf.reshape(N, N, N, ncol)
    Y = np.zeros_like(X)
    c = 0
    for cz in range(n):
        for cy in range(n):
            for cx in range(n):
                sl = (slice(cz * p, cz * p + q), slice(cy * p, cy * p + q),
                      slice(cx * p, cx * p + q))
                Y[sl] += (Ve[c] @ X[sl].reshape(q ** 3, ncol)).reshape(q, q, q, ncol)
                c += 1
    return Y.reshape(N ** 3, ncol)


def apply_Htilde_dense(mesh: Mesh, Ve: np.ndarray, X: np.ndarray) -> np.ndarray:
    """H~X = D (K + V) D X over the interior nodes, V from the cell matrices."""
    squeeze = X.ndim == 1
    X2 = X.reshape(mesh.L, -1)
    d = 1.0 / np.sqrt(mesh.mass())
    DX = mesh.to_full(d[:, None] * X2)
    Y = mesh.to_interior(mesh.apply_K_full(DX) + apply_V_full(mesh, Ve, DX))
    Y = d[:, None] * Y
    return Y.ravel() if squeeze else Y
