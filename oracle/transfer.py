"""Linear (Q1) v_xc mesh and field transfer to the orbital mesh (oracle; test
infrastructure only).

The paper represents v_xc with linear finite elements on a mesh of its own,
while the orbitals and adjoint functions use higher-order spectral elements
(Sec. 3.1.1), and transfers fields between the two meshes (Sec. 3.2.2):
  * v_xc to the orbital mesh: the Q1 interpolant evaluated at the orbital
    nodes, v(x_a) = sum_b v_b N_b^Q1(x_a), i.e. v_psi = T v_Q1 with T the
    sparse matrix of trilinear weights (8 per node);
  * the gradient back to the Q1 coefficients: dL/dv_b = int G N_b^Q1 with
    G = sum_i p_i psi_i (Eq. 11), by the orbital mesh's GLL quadrature,
    g_Q1 = T^T g_psi, where g_psi = m o G is the nodal gradient of the
    orbital mesh (Eq. 22).
Reading: the Q1 mesh is a uniform box mesh of n_v cells per axis over the same
box (the paper grades it outside an inner cuboid, Sec. 4.2.2), and v_xc lives
on all of its nodes, the boundary included.

Parity status: pinned (tests/test_oracle_transfer.py) by exact transfer of
trilinear fields and partition of unity, second-order convergence on a smooth
field, and the gradient through the transfer against central finite
differences of the loss as a function of the Q1 coefficients.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Q1Mesh:
    """Uniform trilinear mesh of nv cells per axis on [lo, hi]^3."""

    def __init__(self, lo: float, hi: float, nv: int):
        self.lo, self.hi, self.nv = float(lo), float(hi), int(nv)
        self.hv = (self.hi - self.lo) / self.nv
        self.Nv = self.nv + 1
        self.n_nodes = self.Nv ** 3

    def coords(self) -> np.ndarray:
        """[Nv^3, 3] node coordinates, x fastest."""
        a = self.lo + self.hv * np.arange(self.Nv)
        Z, Y, X = np.meshgrid(a, a, a, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def transfer_matrix(self, points: np.ndarray) -> sp.csr_matrix:
        """[P, Nv^3] trilinear interpolation weights at the given points."""
        pts = np.asarray(points, dtype=np.float64)
        t = (pts - self.lo) / self.hv
        c = np.clip(np.floor(t).astype(np.int64), 0, self.nv - 1)      # owning cell
        f = t - c                                                      # local coordinate in [0, 1]
        rows, cols, vals = [], [], []
        P = len(pts)
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    wx = f[:, 0] if dx else 1.0 - f[:, 0]
                    wy = f[:, 1] if dy else 1.0 - f[:, 1]
                    wz = f[:, 2] if dz else 1.0 - f[:, 2]
                    node = (c[:, 0] + dx) + self.Nv * ((c[:, 1] + dy) + self.Nv * (c[:, 2] + dz))
                    rows.append(np.arange(P))
                    cols.append(node)
                    vals.append(wx * wy * wz)
        T = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(P, self.n_nodes))
        return T.tocsr()


def to_orbital_mesh(T: sp.csr_matrix, v_q1: np.ndarray) -> np.ndarray:
    """v at the orbital nodes from the Q1 coefficients."""
    return T @ v_q1


def gradient_to_q1(T: sp.csr_matrix, grad_psi: np.ndarray) -> np.ndarray:
    """dL/dv_Q1 from the nodal gradient of the orbital mesh (Eq. 22)."""
    return T.T @ grad_psi
