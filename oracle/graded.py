"""Graded tensor-product spectral-element meshes (oracle; test infrastructure only).

The paper discretises the orbitals on adaptive meshes that are refined towards
the atoms, from h_outer at the surface of a sphere of radius r_b to h_inner at
the centre, and coarsen towards h_base in the far field (Sec. 4.2.2), with
element orders up to 6 in the GPU runs (Sec. 5.3).  Reading: here the
refinement is a tensor product.  Each axis carries its own sequence of cell
breaks, graded towards the nuclear coordinates, so every cell is a rectangular
box [x_i, x_i+1] x [y_j, y_j+1] x [z_k, z_k+1].  The GLL nodes then still form
a tensor-product grid, and the cell stiffness keeps the Kronecker form of the
uniform mesh with one scalar per term (Eq. 17):

    K_e = 1/2 [ c_x B (x) B (x) A + c_y B (x) A (x) B + c_z A (x) B (x) B ]   (z, y, x order),
    c_x = h_y h_z / (2 h_x),  c_y = h_x h_z / (2 h_y),  c_z = h_x h_y / (2 h_z),

with A, B the 1D reference stiffness and mass on [-1, 1].  The lumped (GLL)
mass is the tensor product of the 1D assemblies of (h_e / 2) w.  For equal
breaks this is the uniform mesh of oracle.fe.Mesh (c = h / 2 on every term).

Breaks are placed by equidistribution: with a target cell size h(x) = min(
h_outer, h_inner + g d(x)) (d = distance to the nearest nuclear coordinate on
that axis, g the growth rate), the map s(x) = int_lo^x dt / h(t), normalised
to [0, 1], is inverted at s = e / n, so that n cells follow the target sizes.

Parity status: pinned (tests/test_oracle_graded.py) by agreement with
oracle.fe.Mesh on equal breaks, exact energies of polynomials of degree <= p,
exact GLL integrals of the mass, the particle-in-a-box spectrum on graded
meshes (order-2p convergence), and the monotone, box-spanning breaks of the
generator.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fe import gll_rule, reference_matrices


def graded_breaks(lo: float, hi: float, n: int, centres, h_inner: float, h_outer: float,
                  growth: float = 0.5, samples: int = 20001) -> np.ndarray:
    """n + 1 cell breaks on [lo, hi] that equidistribute 1 / h(x)."""
    x = np.linspace(lo, hi, samples)
    c = np.asarray(centres, dtype=np.float64).reshape(-1)
    d = np.min(np.abs(x[:, None] - c[None, :]), axis=1) if c.size else np.full_like(x, np.inf)
    h = np.minimum(h_outer, h_inner + growth * d)
    dens = 1.0 / h
    # cumulative trapezoid of 1/h
    s = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(x))])
    s /= s[-1]
    b = np.interp(np.linspace(0.0, 1.0, n + 1), s, x)
    b[0], b[-1] = lo, hi
    return b


class GradedMesh:
    """Tensor-product mesh with per-axis cell breaks (bx, by, bz) and order p."""

    def __init__(self, bx, by, bz, p: int):
        self.breaks = [np.asarray(b, dtype=np.float64) for b in (bx, by, bz)]
        self.p, self.q = int(p), int(p) + 1
        self.ncell = [len(b) - 1 for b in self.breaks]             # x, y, z
        self.N = [n * self.p + 1 for n in self.ncell]               # nodes per axis incl. boundary
        self.Ni = [n - 2 for n in self.N]
        self.L = self.Ni[0] * self.Ni[1] * self.Ni[2]
        xi, w = gll_rule(self.p)
        A, B, _ = reference_matrices(self.p)
        self.A1, self.B1 = A, B
        self.h = [np.diff(b) for b in self.breaks]
        self.axis, self.m1 = [], []
        for b, h, N in zip(self.breaks, self.h, self.N):
            c = np.empty(N)
            m1 = np.zeros(N)
            for e in range(len(h)):
                c[e * p:(e + 1) * p + 1] = b[e] + 0.5 * h[e] * (xi + 1.0)
                m1[e * p:(e + 1) * p + 1] += 0.5 * h[e] * w
            c[0], c[-1] = b[0], b[-1]
            self.axis.append(c)
            self.m1.append(m1)
        # cell scalars indexed [cz, cy, cx]
        hx = self.h[0][None, None, :]
        hy = self.h[1][None, :, None]
        hz = self.h[2][:, None, None]
        self.cx = hy * hz / (2.0 * hx)
        self.cy = hx * hz / (2.0 * hy)
        self.cz = hx * hy / (2.0 * hz)

    # ---- nodal fields
    def _grid(self, inner: bool):
        ax = [a[1:-1] if inner else a for a in self.axis]
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def coords(self) -> np.ndarray:
        """[L, 3] interior node coordinates, x fastest."""
        return self._grid(True)

    def coords_full(self) -> np.ndarray:
        return self._grid(False)

    def mass(self) -> np.ndarray:
        mx, my, mz = (m[1:-1] for m in self.m1)
        return np.einsum("k,j,i->kji", mz, my, mx).ravel()

    def mass_full(self) -> np.ndarray:
        mx, my, mz = self.m1
        return np.einsum("k,j,i->kji", mz, my, mx).ravel()

    # ---- operators
    def to_full(self, X: np.ndarray) -> np.ndarray:
        Nx, Ny, Nz = self.N
        ncol = X.shape[1]
        F = np.zeros((Nz, Ny, Nx, ncol))
        F[1:-1, 1:-1, 1:-1, :] = X.reshape(Nz - 2, Ny - 2, Nx - 2, ncol)
        return F.reshape(-1, ncol)

    def to_interior(self, F: np.ndarray) -> np.ndarray:
        Nx, Ny, Nz = self.N
        ncol = F.shape[1]
        return F.reshape(Nz, Ny, Nx, ncol)[1:-1, 1:-1, 1:-1, :].reshape(self.L, ncol)

    def apply_K_full(self, Xf: np.ndarray) -> np.ndarray:
        """sum over cells of G_e^T K_e G_e X over all nodes, K_e in its three
        Kronecker terms with the cell's scalars (c_x, c_y, c_z)."""
        p, q = self.p, self.q
        nx, ny, nz = self.ncell
        Nx, Ny, Nz = self.N
        ncol = Xf.shape[1]
        X = Xf.reshape(Nz, Ny, Nx, ncol)
        Xe = np.empty((nz, ny, nx, q, q, q, ncol))
        for kz in range(q):
            for ky in range(q):
                for kx in range(q):
                    Xe[:, :, :, kz, ky, kx, :] = X[kz:kz + p * nz:p, ky:ky + p * ny:p,
                                                   kx:kx + p * nx:p, :]
        A, B = self.A1, self.B1
        tx = np.einsum("ak,bj,ci,ZYXkjin->ZYXabcn", B, B, A, Xe, optimize=True)
        ty = np.einsum("ak,bj,ci,ZYXkjin->ZYXabcn", B, A, B, Xe, optimize=True)
        tz = np.einsum("ak,bj,ci,ZYXkjin->ZYXabcn", A, B, B, Xe, optimize=True)
        s = lambda c: c[:, :, :, None, None, None, None]
        Ye = 0.5 * (s(self.cx) * tx + s(self.cy) * ty + s(self.cz) * tz)
        Y = np.zeros_like(X)
        for kz in range(q):
            for ky in range(q):
                for kx in range(q):
                    Y[kz:kz + p * nz:p, ky:ky + p * ny:p, kx:kx + p * nx:p, :] += \
                        Ye[:, :, :, kz, ky, kx, :]
        return Y.reshape(-1, ncol)

    def apply_K(self, X: np.ndarray) -> np.ndarray:
        squeeze = X.ndim == 1
        X2 = X.reshape(self.L, -1)
        Y = self.to_interior(self.apply_K_full(self.to_full(X2)))
        return Y.ravel() if squeeze else Y

    def apply_Htilde(self, v: np.ndarray, X: np.ndarray) -> np.ndarray:
        """H~X = D K D X + v o X, D = m^-1/2 (Eq. 19)."""
        squeeze = X.ndim == 1
        X2 = X.reshape(self.L, -1)
        d = 1.0 / np.sqrt(self.mass())
        Y = d[:, None] * self.apply_K(d[:, None] * X2) + v[:, None] * X2
        return Y.ravel() if squeeze else Y

    def axis_matrices(self):
        """Assembled 1D matrices of each axis over its interior nodes:
        Ad = sum_e (2 / h_e) A and Bd = sum_e (h_e / 2) B (dense, small)."""
        out = []
        for h, N in zip(self.h, self.N):
            Ad, Bd = np.zeros((N, N)), np.zeros((N, N))
            for e in range(len(h)):
                sl = slice(e * self.p, e * self.p + self.q)
                Ad[sl, sl] += (2.0 / h[e]) * self.A1
                Bd[sl, sl] += (0.5 * h[e]) * self.B1
            out.append((Ad[1:-1, 1:-1], Bd[1:-1, 1:-1]))
        return out

    def apply_K_sweeps(self, X: np.ndarray) -> np.ndarray:
        """K X by 1D sweeps of the assembled axis matrices.  The cell scalars
        separate by axis (c_x = (2/h_x)(h_y/2)(h_z/2) and cyclic), and the cells
        form a product set, so the assembled K is itself a sum of Kronecker
        products:  K = 1/2 [B_z (x) B_y (x) A_x + B_z (x) A_y (x) B_x
        + A_z (x) B_y (x) B_x]  over the interior nodes.  Seven sweeps:
        P = A_x X, Q = B_x X;  R = B_y P + A_y Q, S = B_y Q;  K X = (B_z R + A_z S) / 2."""
        (Ax, Bx), (Ay, By), (Az, Bz) = self.axis_matrices()
        nx, ny, nz = self.Ni
        squeeze = X.ndim == 1
        X4 = X.reshape(nz, ny, nx, -1)
        P = np.einsum("ia,zyan->zyin", Ax, X4)
        Q = np.einsum("ia,zyan->zyin", Bx, X4)
        R = np.einsum("ja,zaxn->zjxn", By, P) + np.einsum("ja,zaxn->zjxn", Ay, Q)
        S = np.einsum("ja,zaxn->zjxn", By, Q)
        Y = 0.5 * (np.einsum("ka,ayxn->kyxn", Bz, R) + np.einsum("ka,ayxn->kyxn", Az, S))
        Y = Y.reshape(self.L, -1)
        return Y.ravel() if squeeze else Y

    def assemble_K(self) -> sp.csr_matrix:
        """Sparse K over the interior nodes, cell by cell (small meshes)."""
        p, q = self.p, self.q
        nx, ny, nz = self.ncell
        Nx, Ny, Nz = self.N
        imap = -np.ones((Nz, Ny, Nx), dtype=np.int64)
        imap[1:-1, 1:-1, 1:-1] = np.arange(self.L).reshape(Nz - 2, Ny - 2, Nx - 2)
        A, B = self.A1, self.B1
        Tx, Ty, Tz = np.kron(B, np.kron(B, A)), np.kron(B, np.kron(A, B)), np.kron(A, np.kron(B, B))
        kz, ky, kx = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
        rows, cols, vals = [], [], []
        for cz in range(nz):
            for cy in range(ny):
                for cx in range(nx):
                    g = imap[cz * p + kz.ravel(), cy * p + ky.ravel(), cx * p + kx.ravel()]
                    Ke = 0.5 * (self.cx[cz, cy, cx] * Tx + self.cy[cz, cy, cx] * Ty
                                + self.cz[cz, cy, cx] * Tz)
                    keep = g >= 0
                    gi = g[keep]
                    sub = Ke[np.ix_(keep, keep)]
                    rows.append(np.repeat(gi, len(gi)))
                    cols.append(np.tile(gi, len(gi)))
                    vals.append(sub.ravel())
        K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.L, self.L))
        return K.tocsr()

    def assemble_Htilde(self, v: np.ndarray) -> sp.csr_matrix:
        d = sp.diags(1.0 / np.sqrt(self.mass()))
        return (d @ self.assemble_K() @ d + sp.diags(v)).tocsr()
