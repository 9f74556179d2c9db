"""Graded and rectangular tensor-product meshes and order p = 6 on the device
(Sec. 4.2.2 graded refinement towards the nuclei, Sec. 5.3 p = 6) against the
graded-mesh oracle (needs a B300; marked gpu).

Each axis carries its own cell breaks, so cells are boxes and K_e keeps its
Kronecker form with per-cell scalars (Eq. 17).  H~X runs in the sweep form
(graded path: D and the cell scalars applied in the kernel; equal cells per
axis: folded into the coefficients) for aligned widths, and in the cell
kernel for the others.  Tolerances as for the uniform meshes: H~X FP64 1e-10,
FP32 2e-6 (max over columns of the relative 2-norm error); eigenvalues 1e-6
Ha, density L2 1e-6, gradient 1e-5 relative.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import graded, inverse, ks  # noqa: E402


def _cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _colrel(Yg, Yo):
    return float(np.max(np.linalg.norm(Yg - Yo, axis=0) / np.linalg.norm(Yo, axis=0)))


def _graded_box(order, nx=5, ny=3, nz=4):
    bx = graded.graded_breaks(-6.0, 5.0, nx, [-1.0, 2.0], 0.6, 3.0)
    by = np.linspace(-4.0, 4.0, ny + 1)
    bz = graded.graded_breaks(-5.0, 5.0, nz, [0.5], 0.8, 3.5)
    return (bx, by, bz), [bx, None, bz]


def _problem(breaks_list, order, nstates, **kw):
    import paper_2510_10529_b300 as P
    lo = [b[0] for b in breaks_list]
    hi = [b[-1] for b in breaks_list]
    nc = [len(b) - 1 for b in breaks_list]
    return P.Problem(lo, hi, nc, order, nstates, breaks=breaks_list, **kw)


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("kind", ["graded", "rectangular"])
def test_apply_h_on_box_meshes_matches_oracle(order, kind):
    if kind == "graded":
        (bx, by, bz), _ = _graded_box(order)
    else:                       # equal cells per axis, different sizes per axis
        bx, by, bz = np.linspace(-6, 5, 4), np.linspace(-4, 4, 6), np.linspace(-3, 5, 3)
    om = graded.GradedMesh(bx, by, bz, order)
    rng = np.random.default_rng(order)
    xyz = om.coords()
    v = W.smeared_coulomb(xyz, np.array([[0.3, -0.2, 0.4]]), np.array([3.0]), 0.5)
    v = v + 0.1 * rng.standard_normal(om.L)
    pb = _problem([bx, by, bz], order, nstates=4)
    pb.set_potential(_cuda(v))
    n32, n64 = pb.tune_hx(-1, 0)
    for seglen in (1, 0):
        for dtype, ncols, tol, nvar in ((torch.float64, (1, 3, 6, 18), 1e-10, n64),
                                        (torch.float32, (4, 12, 36), 2e-6, n32)):
            for var in range(nvar):
                pb.tune_hx(var, seglen)
                for ncol in ncols:
                    X = rng.standard_normal((om.L, ncol))
                    Y_ora = om.apply_Htilde(v, X)
                    Yg = pb.apply_h(_cuda(X, dtype), tensor_cores=False).double().cpu().numpy()
                    err = _colrel(Yg, Y_ora)
                    print(f"{kind} p={order} seglen={seglen} var={var} {dtype} ncol={ncol}: "
                          f"{err:.2e}")
                    assert err <= tol


@pytest.mark.parametrize("order,prec", [(4, "mixed"), (4, "fp64"), (6, "mixed")])
def test_forward_and_gradient_on_graded_mesh_match_oracle(order, prec):
    """Kohn-Sham solve, loss and masked gradient on a mesh graded towards two
    nuclei (kT > 0, four electrons in six states)."""
    R = np.array([[-1.0, 0.2, 0.5], [1.6, -0.3, 0.5]])
    bx = graded.graded_breaks(-6.0, 6.0, 5, R[:, 0], 0.8, 3.5)
    by = graded.graded_breaks(-5.0, 5.0, 4, R[:, 1], 0.9, 3.5)
    bz = graded.graded_breaks(-5.0, 6.0, 4, R[:, 2], 0.9, 3.5)
    om = graded.GradedMesh(bx, by, bz, order)
    xyz = om.coords()
    v = W.smeared_coulomb(xyz, R, np.array([2.0, 2.0]), 0.5)
    bump = 0.1 * np.exp(-np.sum((xyz - 0.3) ** 2, 1))
    Ne, nst, kT = 4.0, 6, W.KT_DEFAULT
    rho_d = ks.forward(om, v + bump, Ne, nst, kT)["rho"]
    op = inverse.Problem(mesh=om, v_fixed=v, rho_data=rho_d, w=np.ones(om.L), n_electrons=Ne,
                         nstates=nst, kT=kT)
    v_xc = 0.5 * bump
    L_ora, _, g_ora, fw = inverse.evaluate(op, v_xc)
    pb = _problem([bx, by, bz], order, nstates=nst, n_electrons=Ne, kT=kT, prec=prec,
                  eig_tol=1e-10, adj_tol=1e-11, cheb_degree=20)
    pb.set_potential(_cuda(v), _cuda(v_xc))
    out = pb.forward_solve()
    act = fw["f"] > 1e-8
    deps = np.abs(out["eps"].cpu().numpy()[act] - fw["eps"][act]).max()
    m = om.mass()
    drho = math.sqrt(np.sum(m * (out["rho"].cpu().numpy() - fw["rho"]) ** 2))
    loss, g, _ = pb.loss_grad(_cuda(rho_d), _cuda(np.ones(om.L)))
    gerr = np.linalg.norm(g.cpu().numpy() - g_ora) / np.linalg.norm(g_ora)
    print(f"graded p={order} {prec}: |d eps| {deps:.2e}, density L2 {drho:.2e}, "
          f"loss rel {abs(loss - L_ora) / L_ora:.2e}, grad rel {gerr:.2e}")
    assert deps <= 1e-6
    assert drho <= 1e-6
    assert abs(loss - L_ora) <= 1e-8 * L_ora
    assert gerr <= 1e-5
