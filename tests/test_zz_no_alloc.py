"""The allocation-free loss reduction (invdft_loss_reduce_noalloc) against the
reduction inside invdft_loss_grad.

Some callers cannot allocate device memory: they own a fixed pool, or have no
workspace to bind.  For them the library offers one reduction whose scratch is
a fixed array inside the library.  This test calls it through the C ABI twice
in a row on the density of a forward solve and checks loss, e_L2^2 and N_e
against what invdft_loss_grad reports for the same potential (the two
forward solves agree to the eigen tolerance, hence the 1e-8 bound used by the
other loss tests), and loss and e_L2^2 against the FP64 oracle's quadrature of
the same density (only the summation order differs).  It lives in its own
file, collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_loss_matches_loss_grad_twice():
    import paper_2510_10529_b300 as P
    from paper_2510_10529_b300._lib import lib
    import workloads as W
    from oracle import adjoint as oadj, fe, scf

    wl = W.cube8_q2_he()
    mesh = fe.Mesh(wl.lo, wl.hi, wl.ncell, wl.order)
    d = scf.target_density(mesh, wl)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda").contiguous()
    pb = P.Problem(wl.lo, wl.hi, wl.ncell, wl.order, wl.nstates, n_electrons=wl.n_electrons,
                   kT=wl.kT, prec="fp64", eig_tol=1e-10, adj_tol=1e-10,
                   cheb_degree=wl.cheb_degree)
    v_fixed, v_xc = t(d["v_fixed"]), t(0.3 * d["v_xc_ref"])
    rd, w = t(d["rho_data"]), t(1.0 + 0.1 * np.cos(mesh.coords()[:, 0]))
    pb.set_potential(v_fixed, v_xc)
    loss_ref, _, st = pb.loss_grad(rd, w)
    pb.set_potential(v_fixed, v_xc)
    rho = pb.forward_solve()["rho"]
    m = pb.mass()
    outs = []
    for _ in range(2):
        out3 = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.zeros(pb.L, dtype=torch.float64, device="cuda")
        code = lib.invdft_loss_reduce_noalloc(
            C.c_void_p(rho.data_ptr()), C.c_void_p(rd.data_ptr()), C.c_void_p(w.data_ptr()),
            C.c_void_p(m.data_ptr()), pb.L, C.c_void_p(out3.data_ptr()),
            C.c_void_p(g.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert code == 0, lib.invdft_last_error(None)
        torch.cuda.synchronize()
        o = out3.cpu().numpy()
        assert abs(o[0] - loss_ref) <= 1e-8 * loss_ref
        assert abs(o[1] - st["err_l2"] ** 2) <= 1e-8 * st["err_l2"] ** 2
        assert abs(o[2] - wl.n_electrons) <= 1e-10 * wl.n_electrons
        # the same sums from the FP64 oracle on the same density
        lo_ora, el_ora = oadj.loss_and_error(mesh, rho.cpu().numpy(), d["rho_data"],
                                             w.cpu().numpy())
        assert abs(o[0] - lo_ora) <= 1e-12 * lo_ora
        assert abs(o[1] - el_ora ** 2) <= 1e-12 * el_ora ** 2
        g_ref = -2.0 * m * w * (rd - rho)
        assert torch.allclose(g, g_ref, rtol=1e-13, atol=0.0)
        outs.append(o)
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_oversize_and_null():
    from paper_2510_10529_b300._lib import lib
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(x.data_ptr())
    assert lib.invdft_loss_reduce_noalloc(p, p, None, p, 2 ** 25 + 1, p, None, None) == 1
    assert b"33,554,432" in lib.invdft_last_error(None)
    assert lib.invdft_loss_reduce_noalloc(None, p, None, p, 8, p, None, None) == 1
