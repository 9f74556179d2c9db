"""Dense per-cell potential matrices on the device (the Gauss-quadrature
reading of the potential term of Eq. 17) against the oracle (needs a B300;
marked gpu).

Cell matrices: FP64 build vs oracle.potential_matrix.cell_potential_matrices,
max error <= 1e-12 of the largest entry; the FP32 tile is the same matrix
rounded to FP32 (<= 1e-6 relative).  Operator: H~X = D (K + V) D X vs
oracle.potential_matrix.apply_Htilde_dense, FP64 <= 1e-10 and FP32 <= 2e-6
(max over columns of the relative 2-norm error), on Q2 and Q4 meshes with
ragged column counts.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import fe  # noqa: E402
from oracle import potential_matrix as pm  # noqa: E402


def _cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _umma_index(a, b):
    return ((a >> 3) * 4096 + (b >> 2) * 128 + (a & 7) * 16 + (b & 3) * 4) // 4


@pytest.mark.parametrize("geom", [(-4.0, 5.0, 3, 2), (-5.0, 5.0, 3, 4), (-3.0, 3.0, 2, 4)])
def test_cell_potentials_and_dense_operator_match_oracle(geom):
    import paper_2510_10529_b300 as P
    lo, hi, n, p = geom
    mesh = fe.Mesh(lo, hi, n, p)
    xyz = mesh.coords_full()
    v_full = W.smeared_coulomb(xyz, np.array([[0.4, -0.3, 0.2]]), np.array([3.0]), 0.5)
    v_full = v_full + 0.2 * np.cos(xyz[:, 0]) * np.sin(0.7 * xyz[:, 1])
    Ve_ora = pm.cell_potential_matrices(mesh, v_full)
    pb = P.Problem(lo, hi, n, p, nstates=4)
    V64 = pb.cell_potentials(_cuda(v_full), "fp64")
    ne = (p + 1) ** 3
    Vg = V64.view(torch.float64).cpu().numpy().reshape(-1, ne, ne)
    scale = np.abs(Ve_ora).max()
    assert np.abs(Vg - Ve_ora).max() <= 1e-12 * scale
    V32 = pb.cell_potentials(_cuda(v_full), "mixed")
    tiles = V32.view(torch.float32).cpu().numpy().reshape(-1, 128 * 128)
    a, b = np.meshgrid(np.arange(ne), np.arange(ne), indexing="ij")
    Vf = tiles[:, _umma_index(a, b)]
    assert np.abs(Vf - Ve_ora).max() <= 1e-6 * scale
    rng = np.random.default_rng(n * 10 + p)
    for ncol in (1, 5, 12, 40):
        X = rng.standard_normal((mesh.L, ncol))
        Y_ora = pm.apply_Htilde_dense(mesh, Ve_ora, X)
        Y64 = pb.apply_h_dense(V64, _cuda(X)).cpu().numpy()
        e64 = np.max(np.linalg.norm(Y64 - Y_ora, axis=0) / np.linalg.norm(Y_ora, axis=0))
        Y32 = pb.apply_h_dense(V32, _cuda(X, torch.float32)).double().cpu().numpy()
        e32 = np.max(np.linalg.norm(Y32 - Y_ora, axis=0) / np.linalg.norm(Y_ora, axis=0))
        print(f"dense V p={p} n={n} ncol={ncol}: FP64 {e64:.2e}, FP32 {e32:.2e}")
        assert e64 <= 1e-10
        assert e32 <= 2e-6
