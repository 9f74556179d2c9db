"""Hartree potential by a finite-element Poisson solve (oracle; test infrastructure only).

v_H solves -lap v_H = 4 pi rho (the Hartree potential of Eq. 2 in differential
form).  Weak form on the same spectral elements: (2K) u = 4 pi M rho on the
unknown nodes, with the stiffness 2K (K is the kinetic matrix, 1/2 of the
Laplacian's) and the lumped mass M.  Boundary values are the monopole Q/|r|
with Q = int rho (reading: the paper gives no boundary condition; v_H is fixed
during the inverse loop, so any consistent choice yields the same inverse
solution).  Solved by conjugate gradients to 1e-13 relative residual.
"""
from __future__ import annotations

import numpy as np

from .fe import Mesh


def conjugate_gradient(apply_A, b, tol=1e-13, maxit=20000):
    """Textbook CG for an SPD operator, x0 = 0."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = float(np.sqrt(b @ b))
    if bnorm == 0.0:
        return x
    for _ in range(maxit):
        Ap = apply_A(p)
        a = rr / float(p @ Ap)
        x += a * p
        r -= a * Ap
        rr_new = float(r @ r)
        if np.sqrt(rr_new) <= tol * bnorm:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def hartree(mesh: Mesh, rho: np.ndarray) -> np.ndarray:
    """v_H at the unknown nodes for a nodal density rho (unknown nodes only)."""
    m = mesh.mass()
    Q = float(m @ rho)
    xyz = mesh.coords_full()
    r = np.linalg.norm(xyz, axis=1)
    interior = mesh.interior_map() >= 0
    uB = np.where(interior, 0.0, Q / np.maximum(r, 1e-300))
    # 2 K_II u_I = 4 pi m rho - 2 K_IB u_B
    rhs = 4.0 * np.pi * m * rho - 2.0 * mesh.to_interior(mesh.apply_K_full(uB[:, None]))[:, 0]
    return conjugate_gradient(lambda x: 2.0 * mesh.apply_K(x), rhs)
