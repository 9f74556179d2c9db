"""Spectral finite elements on a uniform box (oracle; test infrastructure only).

Follows Sec. 3.1.1 and Sec. 3.2.1 of the paper:
  * 1D Lagrange polynomials through the element nodes (Eq. 12), tensor
    products in 3D;
  * spectral elements: nodes at the Gauss-Lobatto-Legendre (GLL) points, with
    GLL quadrature for the mass matrix so that M is diagonal (Sec. 3.2.1, the
    paragraph after Eq. 20);
  * H_ab = int N_a H N_b (Eq. 17) with the kinetic part integrated exactly
    (Gauss-Legendre, p+1 points) and the potential part by GLL collocation
    (reading: "reduced-order GLL quadrature" applies to M and to the local
    potential), so H = K + diag(m v) and M = diag(m);
  * standard form H~ = M^-1/2 H M^-1/2 = D K D + diag(v), D = diag(m^-1/2)
    (Eq. 19).

Nodes are numbered lexicographically, x fastest.  Boundary nodes carry the
homogeneous Dirichlet condition and are not unknowns; vectors "over interior
nodes" have length L = (n_x p - 1)(n_y p - 1)(n_z p - 1).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg
import scipy.sparse as sp


# ------------------------------------------------------------------ 1D rules

def gll_rule(p: int):
    """GLL nodes (-1, 1 and the roots of P_p') and weights 2/(p(p+1) P_p(x)^2)."""
    cP = np.zeros(p + 1)
    cP[p] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(cP)))) if p > 1 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (p * (p + 1) * npleg.legval(x, cP) ** 2)
    return x, w


def gauss_rule(n: int):
    """n-point Gauss-Legendre rule (library routine)."""
    return npleg.leggauss(n)


def lagrange_values(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """ell_i(x_q) = prod_{j != i} (x_q - x_j)/(x_i - x_j) (Eq. 12); [len(x), n]."""
    n = len(nodes)
    out = np.ones((len(x), n))
    for i in range(n):
        for j in range(n):
            if j != i:
                out[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return out


def lagrange_derivs(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """d/dx of Eq. 12 by the product rule; [len(x), n]."""
    n = len(nodes)
    out = np.zeros((len(x), n))
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[k]))
            for j in range(n):
                if j != i and j != k:
                    term *= (x - nodes[j]) / (nodes[i] - nodes[j])
            out[:, i] += term
    return out


def reference_matrices(p: int):
    """1D matrices on [-1,1] for GLL Lagrange polynomials of order p.

    A_ij = int l_i' l_j' (stiffness), B_ij = int l_i l_j (consistent mass),
    both exact with p+1 Gauss points; w = GLL weights (lumped mass).
    """
    xn, w = gll_rule(p)
    xq, wq = gauss_rule(p + 1)
    V = lagrange_values(xn, xq)
    G = lagrange_derivs(xn, xq)
    A = G.T @ (wq[:, None] * G)
    B = V.T @ (wq[:, None] * V)
    return A, B, w


# ------------------------------------------------------------------ 3D mesh

class Mesh:
    """Uniform box [lo, hi]^3 cut into ncell^3 equal cells of order p."""

    def __init__(self, lo: float, hi: float, ncell: int, p: int):
        self.lo, self.hi, self.n, self.p = float(lo), float(hi), int(ncell), int(p)
        self.h = (self.hi - self.lo) / self.n
        self.q = p + 1                       # nodes per cell edge
        self.N = self.n * p + 1              # nodes per axis incl. boundary
        self.Ni = self.N - 2                 # interior nodes per axis
        self.L = self.Ni ** 3
        xn, wgll = gll_rule(p)
        # node coordinates along one axis
        c = np.empty(self.N)
        for e in range(self.n):
            c[e * p:(e + 1) * p + 1] = self.lo + e * self.h + 0.5 * self.h * (xn + 1.0)
        c[0], c[-1] = self.lo, self.hi
        self.axis = c
        # 1D lumped (GLL) mass: assembly of (h/2) w over cells
        m1 = np.zeros(self.N)
        for e in range(self.n):
            m1[e * p:(e + 1) * p + 1] += 0.5 * self.h * wgll
        self.m1 = m1
        A, B, _ = reference_matrices(p)
        self.A1, self.B1 = A, B
        # cell kinetic matrix K_e = 1/2 int grad N_a . grad N_b over a cube of side h:
        # d/dx terms scale as (2/h) A, mass-like factors as (h/2) B.
        s = 0.5 * self.h
        Ax = (1.0 / s) * A
        Bx = s * B
        # local index a = ix + q*iy + q*q*iz  ->  kron(M_z, kron(M_y, M_x))
        self.Ke = 0.5 * (np.kron(Bx, np.kron(Bx, Ax))
                         + np.kron(Bx, np.kron(Ax, Bx))
                         + np.kron(Ax, np.kron(Bx, Bx)))

    # ---- nodal fields over interior nodes
    def coords(self) -> np.ndarray:
        """[L, 3] coordinates of the interior nodes (x fastest)."""
        a = self.axis[1:-1]
        Z, Y, X = np.meshgrid(a, a, a, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def coords_full(self) -> np.ndarray:
        a = self.axis
        Z, Y, X = np.meshgrid(a, a, a, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def mass(self) -> np.ndarray:
        """Diagonal of the lumped mass M over interior nodes: m_a = m1_x m1_y m1_z."""
        m = self.m1[1:-1]
        return np.einsum("k,j,i->kji", m, m, m).ravel()

    def mass_full(self) -> np.ndarray:
        m = self.m1
        return np.einsum("k,j,i->kji", m, m, m).ravel()

    # ---- operators
    def apply_K_full(self, Xf: np.ndarray) -> np.ndarray:
        """Y = sum_e G_e^T K_e G_e X over ALL nodes (boundary included).

        Xf: [N^3, ncol].  For each local node offset (iz,iy,ix) of a cell the
        strided slice X[iz::p, iy::p, ix::p] holds that node of every cell, so
        the gather G_e, the dense product K_e X_e and the scatter-add G_e^T are
        done for all cells at once.
        """
        N, p, n, q = self.N, self.p, self.n, self.q
        ncol = Xf.shape[1]
        X = Xf.reshape(N, N, N, ncol)
        Xe = np.empty((n, n, n, q ** 3, ncol))
        for iz in range(q):
            for iy in range(q):
                for ix in range(q):
                    a = ix + q * iy + q * q * iz
                    Xe[:, :, :, a, :] = X[iz:iz + p * n:p, iy:iy + p * n:p, ix:ix + p * n:p, :]
        Ye = np.matmul(self.Ke, Xe)
        Y = np.zeros_like(X)
        for iz in range(q):
            for iy in range(q):
                for ix in range(q):
                    a = ix + q * iy + q * q * iz
                    Y[iz:iz + p * n:p, iy:iy + p * n:p, ix:ix + p * n:p, :] += Ye[:, :, :, a, :]
        return Y.reshape(N ** 3, ncol)

    def to_full(self, X: np.ndarray) -> np.ndarray:
        ncol = X.shape[1]
        Xf = np.zeros((self.N, self.N, self.N, ncol))
        Xf[1:-1, 1:-1, 1:-1, :] = X.reshape(self.Ni, self.Ni, self.Ni, ncol)
        return Xf.reshape(self.N ** 3, ncol)

    def to_interior(self, Xf: np.ndarray) -> np.ndarray:
        ncol = Xf.shape[1]
        return Xf.reshape(self.N, self.N, self.N, ncol)[1:-1, 1:-1, 1:-1, :].reshape(self.L, ncol)

    def apply_K(self, X: np.ndarray) -> np.ndarray:
        """K X for X over interior nodes (Dirichlet zeros on the boundary)."""
        squeeze = X.ndim == 1
        X2 = X.reshape(self.L, -1)
        Y = self.to_interior(self.apply_K_full(self.to_full(X2)))
        return Y.ravel() if squeeze else Y

    def apply_Htilde(self, v: np.ndarray, X: np.ndarray) -> np.ndarray:
        """Standard-form Hamiltonian (Eq. 19): H~X = D K D X + v o X, D = m^-1/2."""
        squeeze = X.ndim == 1
        X2 = X.reshape(self.L, -1)
        d = 1.0 / np.sqrt(self.mass())
        Y = d[:, None] * self.apply_K(d[:, None] * X2) + v[:, None] * X2
        return Y.ravel() if squeeze else Y

    # ---- assembled sparse matrices (small and moderate meshes only)
    def cell_node_index(self) -> np.ndarray:
        """[ncell^3, (p+1)^3] global (full-grid) node index of each local node."""
        n, p, q, N = self.n, self.p, self.q, self.N
        cz, cy, cx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        iz, iy, ix = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
        gx = (cx.ravel()[:, None] * p + ix.ravel()[None, :])
        gy = (cy.ravel()[:, None] * p + iy.ravel()[None, :])
        gz = (cz.ravel()[:, None] * p + iz.ravel()[None, :])
        return gx + N * (gy + N * gz)

    def interior_map(self) -> np.ndarray:
        """full-grid index -> interior index (or -1 on the boundary)."""
        N = self.N
        idx = -np.ones((N, N, N), dtype=np.int64)
        idx[1:-1, 1:-1, 1:-1] = np.arange(self.L).reshape(self.Ni, self.Ni, self.Ni)
        return idx.ravel()

    def assemble_K(self) -> sp.csr_matrix:
        """Sparse K over interior nodes by element-by-element assembly (Eq. 17)."""
        gi = self.interior_map()[self.cell_node_index()]      # [cells, ne]
        ne = self.q ** 3
        rows = np.repeat(gi[:, :, None], ne, axis=2)
        cols = np.repeat(gi[:, None, :], ne, axis=1)
        vals = np.broadcast_to(self.Ke[None, :, :], rows.shape)
        keep = (rows >= 0) & (cols >= 0)
        K = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(self.L, self.L))
        return K.tocsr()

    def assemble_Htilde(self, v: np.ndarray) -> sp.csr_matrix:
        d = sp.diags(1.0 / np.sqrt(self.mass()))
        return (d @ self.assemble_K() @ d + sp.diags(v)).tocsr()


def htilde_rows(mesh: Mesh, v_rows: np.ndarray, rows: np.ndarray, fetch_X) -> np.ndarray:
    """(H~ X)[rows] one row at a time from the definition (Eq. 17, Eq. 19).

    For interior node a = rows[k]: (D K D X)_a = d_a sum over the cells e that
    contain a of sum_b K_e[a_loc, b_loc] d_b X_b, plus v_a X_a.
    fetch_X(idx) must return X at the interior indices idx ([len(idx), ncol]),
    so that only the neighbourhoods of the sampled rows are needed.
    """
    p, q, Ni = mesh.p, mesh.q, mesh.Ni
    m1 = mesh.m1
    out = []
    for k, a in enumerate(rows):
        ix, iy, iz = a % Ni + 1, (a // Ni) % Ni + 1, a // (Ni * Ni) + 1   # full-grid
        acc = None
        for cz in {(iz - 1) // p, iz // p} & set(range(mesh.n)):
            for cy in {(iy - 1) // p, iy // p} & set(range(mesh.n)):
                for cx in {(ix - 1) // p, ix // p} & set(range(mesh.n)):
                    lx, ly, lz = ix - cx * p, iy - cy * p, iz - cz * p
                    if not (0 <= lx <= p and 0 <= ly <= p and 0 <= lz <= p):
                        continue
                    aloc = lx + q * ly + q * q * lz
                    idx, dvals, bloc = [], [], []
                    for bz in range(q):
                        for by in range(q):
                            for bx in range(q):
                                gx, gy, gz = cx * p + bx, cy * p + by, cz * p + bz
                                if 1 <= gx <= Ni and 1 <= gy <= Ni and 1 <= gz <= Ni:
                                    idx.append((gx - 1) + Ni * ((gy - 1) + Ni * (gz - 1)))
                                    dvals.append((m1[gx] * m1[gy] * m1[gz]) ** -0.5)
                                    bloc.append(bx + q * by + q * q * bz)
                    Xb = fetch_X(np.array(idx))
                    contrib = (mesh.Ke[aloc, bloc] * np.array(dvals)) @ Xb
                    acc = contrib if acc is None else acc + contrib
        da = (m1[ix] * m1[iy] * m1[iz]) ** -0.5
        out.append(da * acc + v_rows[k] * fetch_X(np.array([a]))[0])
    return np.array(out)
