"""The Q1 v_xc mesh transfer on the device (Sec. 3.1.1, Sec. 3.2.2) against the
oracle's sparse trilinear matrix (needs a B300; marked gpu).

Both maps are FP64 sums of at most 8 (gather) or a few hundred (transpose)
products of exact-to-rounding weights: max error <= 1e-13 of the largest
entry.  The chain through the gradient: with v_xc = T v_q1 the Q1 gradient
T^T g of the device path matches the oracle's T^T g_oracle at the gradient
tolerance (1e-5 relative).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import fe, inverse  # noqa: E402
from oracle.transfer import Q1Mesh, gradient_to_q1, to_orbital_mesh  # noqa: E402


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("geom,nv", [((-4.0, 4.0, 3, 4), 5), ((-4.0, 4.0, 3, 4), 12),
                                     ((-5.0, 5.0, 5, 2), 7), ((-5.0, 5.0, 5, 2), 10)])
def test_transfer_and_transpose_match_oracle(geom, nv):
    import paper_2510_10529_b300 as P
    lo, hi, n, p = geom
    mesh = fe.Mesh(lo, hi, n, p)
    q1 = Q1Mesh(lo, hi, nv)
    T = q1.transfer_matrix(mesh.coords())
    rng = np.random.default_rng(nv)
    vq = rng.standard_normal(q1.n_nodes)
    g = rng.standard_normal(mesh.L)
    pb = P.Problem(lo, hi, n, p, nstates=4)
    v = pb.q1_to_nodes(nv, _cuda(vq)).cpu().numpy()
    gq = pb.grad_to_q1(nv, _cuda(g)).cpu().numpy()
    ref_v, ref_g = to_orbital_mesh(T, vq), gradient_to_q1(T, g)
    assert np.abs(v - ref_v).max() <= 1e-13 * np.abs(ref_v).max()
    assert np.abs(gq - ref_g).max() <= 1e-13 * np.abs(ref_g).max()


def test_gradient_through_the_q1_mesh_matches_oracle():
    import paper_2510_10529_b300 as P
    from oracle import scf
    wl = W.cube8_q2_he()
    mesh = fe.Mesh(wl.lo, wl.hi, wl.ncell, wl.order)
    d = scf.target_density(mesh, wl)
    nv = 6
    q1 = Q1Mesh(wl.lo, wl.hi, nv)
    T = q1.transfer_matrix(mesh.coords())
    vq = 0.3 * W.lda_exchange(np.maximum(
        W.gaussian_density(q1.coords(), np.zeros((1, 3)), np.array([2.0]), 1.0), 0.0))
    op = inverse.Problem(mesh=mesh, v_fixed=d["v_fixed"], rho_data=d["rho_data"],
                         w=np.ones(mesh.L), n_electrons=wl.n_electrons, nstates=wl.nstates,
                         kT=wl.kT)
    _, _, g_ora, _ = inverse.evaluate(op, to_orbital_mesh(T, vq))
    pb = P.Problem(wl.lo, wl.hi, wl.ncell, wl.order, wl.nstates, n_electrons=wl.n_electrons,
                   kT=wl.kT, prec="mixed", eig_tol=1e-10, adj_tol=1e-11,
                   cheb_degree=wl.cheb_degree)
    v_nodes = pb.q1_to_nodes(nv, _cuda(vq))
    pb.set_potential(_cuda(d["v_fixed"]), v_nodes)
    _, g, _ = pb.loss_grad(_cuda(d["rho_data"]), _cuda(np.ones(mesh.L)))
    gq = pb.grad_to_q1(nv, g).cpu().numpy()
    ref = gradient_to_q1(T, g_ora)
    err = np.linalg.norm(gq - ref) / np.linalg.norm(ref)
    print(f"Q1 gradient rel err {err:.2e}")
    assert err <= 1e-5
