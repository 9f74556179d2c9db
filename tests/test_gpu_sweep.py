"""Parity of the sweep-form H~X (the owner-computes z-streamed kernel) with the
FP64 oracle, through the C ABI, for every z-segment length the autotuner may
choose (needs a B300; marked gpu).

The sweep kernel runs every FP32 and FP64 block whose rows are a multiple of
16 bytes on Q2 and Q4 meshes.  The cases below cover: tiles that overhang the
mesh edge (unknowns per axis not a multiple of the tile), several column
chunks with a ragged last chunk (36 FP32 columns = 16 + 16 + 4), z segments of
one cell (every cell has a segment top vertex and extra planes), two cells, the
whole range and the balanced persistent schedule (CTAs that take several
segments of different units; launches with the filter's W epilogue fall back
to the whole range under it), and the Chebyshev filter's W epilogue.  Tolerances as in
test_gpu_parity: FP64 1e-10, FP32 2e-6 (max over columns of the relative
2-norm error).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import chebyshev as ocheb  # noqa: E402
from oracle import fe  # noqa: E402


def _cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _colrel(Yg, Yo):
    return float(np.max(np.linalg.norm(Yg - Yo, axis=0) / np.linalg.norm(Yo, axis=0)))


MESHES = [(-5.0, 5.0, 5, 2), (-4.0, 5.0, 3, 4), (-6.0, 6.0, 5, 4)]


BALANCED = 0x7fffffff   # INVDFT_HX_SEG_BALANCED: the persistent balanced schedule


@pytest.mark.parametrize("geom", MESHES)
@pytest.mark.parametrize("seglen", [1, 2, 0, BALANCED])
@pytest.mark.parametrize("dtype,ncols,tol", [(torch.float64, (2, 6, 18), 1e-10),
                                             (torch.float32, (4, 12, 36, 64), 2e-6)])
def test_sweep_apply_h_matches_oracle(geom, seglen, dtype, ncols, tol):
    """Every tile variant of the precision, each with the segment length."""
    import paper_2510_10529_b300 as P
    lo, hi, n, p = geom
    mesh = fe.Mesh(lo, hi, n, p)
    rng = np.random.default_rng(7 * n + p)
    v = W.smeared_coulomb(mesh.coords(), np.array([[0.4, -0.2, 0.1]]), np.array([4.0]), 0.5)
    v = v + 0.1 * rng.standard_normal(mesh.L)
    pb = P.Problem(lo, hi, n, p, nstates=8)
    pb.set_potential(_cuda(v))
    n32, n64 = pb.tune_hx(-1, seglen)
    for variant in range(n64 if dtype == torch.float64 else n32):
        pb.tune_hx(variant, seglen)
        for ncol in ncols:
            X = rng.standard_normal((mesh.L, ncol))
            Y_ora = mesh.apply_Htilde(v, X)
            Yg = pb.apply_h(_cuda(X, dtype), tensor_cores=False).double().cpu().numpy()
            err = _colrel(Yg, Y_ora)
            print(f"sweep H~X p={p} n={n} variant={variant} seglen={seglen} {dtype} "
                  f"ncol={ncol}: {err:.2e}")
            assert err <= tol


@pytest.mark.parametrize("seglen", [1, 3, BALANCED])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-9), (torch.float32, 2e-5)])
def test_sweep_filter_epilogue_matches_oracle(seglen, dtype, tol):
    """The filter's three-term recurrence, Z = alpha (H~ - c) X + beta W, on
    the sweep kernel (degree 12 on a 4^3-cell Q4 mesh, 8 columns)."""
    import paper_2510_10529_b300 as P
    mesh = fe.Mesh(-5.0, 5.0, 4, 4)
    rng = np.random.default_rng(5)
    v = W.smeared_coulomb(mesh.coords(), np.array([[0.0, 0.3, -0.2]]), np.array([2.0]), 0.5)
    X = rng.standard_normal((mesh.L, 8))
    a, b, a0 = 0.5, 60.0, -1.5
    Y_ora = ocheb.filter_apply(lambda Z: mesh.apply_Htilde(v, Z), X, 12, a, b, a0)
    pb = P.Problem(-5.0, 5.0, 4, 4, nstates=8, prec="fp64" if dtype == torch.float64 else "mixed")
    pb.set_potential(_cuda(v))
    pb.tune_hx(-1, seglen)
    Yg = pb.chebyshev_filter(_cuda(X, dtype), 12, a, b, a0).double().cpu().numpy()
    err = _colrel(Yg, Y_ora)
    print(f"sweep filter seglen={seglen} {dtype}: {err:.2e}")
    assert err <= tol


@pytest.mark.parametrize("ncell,order", [(4, 4), (3, 6)])
def test_every_variant_in_the_defect_corrected_filter(ncell, order):
    """Each FP32 tile variant carries the defect-corrected Chebyshev filter
    (beta W and E terms) of a mixed forward solve: eigenvalues of the occupied
    states within 1e-6 Ha and the density within 1e-6 (L2) of the oracle's."""
    import math

    import paper_2510_10529_b300 as P
    from oracle import ks
    lo, hi = -6.0, 6.0
    mesh = fe.Mesh(lo, hi, ncell, order)
    xyz = mesh.coords()
    v = W.smeared_coulomb(xyz, np.array([[0.2, -0.3, 0.1]]), np.array([4.0]), 0.5)
    Ne, nst = 4.0, 8
    ref = ks.forward(mesh, v, Ne, nst, 0.0)
    m = mesh.mass()
    pb = P.Problem(lo, hi, ncell, order, nstates=nst, n_electrons=Ne, kT=0.0, prec="mixed",
                   eig_tol=1e-10, adj_tol=1e-11, cheb_degree=20)
    pb.set_potential(_cuda(v))
    n32, _ = pb.tune_hx(-1, 0)
    for variant in range(n32):
        pb.tune_hx(variant, 0)
        pb.reset()                      # cold start: every variant runs the full filter
        out = pb.forward_solve()
        assert out["stats"]["cheb_passes"] >= 2
        deps = float(np.max(np.abs(out["eps"].cpu().numpy()[:2] - ref["eps"][:2])))
        drho = math.sqrt(np.sum(m * (out["rho"].cpu().numpy() - ref["rho"]) ** 2))
        print(f"defect filter p={order} variant={variant}: deps={deps:.2e} drho={drho:.2e}")
        assert deps <= 1e-6
        assert drho <= 1e-6


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 2e-6), (torch.float64, 1e-10)])
def test_balanced_schedule_full_size(dtype, tol):
    """The balanced schedule on the 32^3-cell Q4 operator benchmark (2,048,383
    unknowns, 64 columns), every tile variant: each CTA takes one whole unit
    and then about 23 z-cells of the units left over, so most CTAs run two or
    three segments of different units.  48 sampled rows against the oracle's
    row-wise definition, and the whole block against the one-segment-per-CTA
    schedule of the same variant (the same operations per node in the same
    order, so the two agree to rounding)."""
    import paper_2510_10529_b300 as P
    wl = W.cube32_q4_hx()
    mesh = fe.Mesh(wl.lo, wl.hi, wl.ncell, wl.order)
    pb = P.Problem(wl.lo, wl.hi, wl.ncell, wl.order, nstates=8)
    v = W.smeared_coulomb(pb.coords(), wl.nuclei_R, wl.nuclei_Z, wl.smear)
    pb.set_potential(_cuda(v))
    X = _cuda(W.random_block(mesh.L, 64, wl.seed), dtype)
    rng = np.random.default_rng(11)
    rows = np.concatenate([rng.integers(0, mesh.L, 44), [0, mesh.L - 1, mesh.Ni - 1, mesh.L // 2]])
    Xd = X.double()

    def fetch(idx):
        return Xd[torch.as_tensor(idx, device="cuda")].cpu().numpy()

    Yo = fe.htilde_rows(mesh, v[rows], rows, fetch)
    n32, n64 = pb.tune_hx(-1, 0)
    for variant in range(n64 if dtype == torch.float64 else n32):
        pb.tune_hx(variant, wl.ncell)
        Yw = pb.apply_h(X, tensor_cores=False)
        pb.tune_hx(variant, BALANCED)
        Yb = pb.apply_h(X, tensor_cores=False)
        Yg = Yb[torch.as_tensor(rows, device="cuda")].double().cpu().numpy()
        err = float((np.linalg.norm(Yg - Yo, axis=1) / np.linalg.norm(Yo, axis=1)).max())
        diff = float((Yb.double() - Yw.double()).abs().max() / Yw.double().abs().max())
        print(f"balanced schedule {dtype} variant {variant}: sampled rows {err:.2e}, "
              f"vs whole-z schedule {diff:.1e}")
        assert err <= tol
        assert diff <= tol
