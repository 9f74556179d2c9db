"""The differentiable inverse solve on the 24^3-cell Q4 workload (857,375
unknowns, 20 electrons, 16 states, FP32 Chebyshev filter of degree 30, FP64
Rayleigh-Ritz): the Kohn-Sham density as a torch.autograd.Function whose
backward is the adjoint solve plus the gradient reduction (Eq. 7-11) must
agree with central finite differences of the loss (Eq. 1) along 16 random
nodal perturbations."""
from __future__ import annotations

import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import workloads as W  # noqa: E402


def test_config3_autograd_matches_finite_differences():
    import paper_2510_10529_b300 as P
    wl = W.cube24_q4_e20()
    pb = P.Problem(wl.lo, wl.hi, wl.ncell, wl.order, wl.nstates, n_electrons=wl.n_electrons,
                   kT=wl.kT, prec="mixed", cheb_degree=wl.cheb_degree, eig_tol=1e-10,
                   adj_tol=1e-10, seed=wl.seed + 1)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda").contiguous()
    f = W.model_fields(wl, pb.coords())
    v_fixed, v_ref = t(f["v_fixed"]), t(f["v_xc_ref"])
    pb.set_potential(v_fixed, v_ref)
    rd = pb.forward_solve()["rho"].clone()
    m = pb.mass()
    v0 = 0.5 * v_ref

    def loss_of(vx):
        with torch.no_grad():
            rho = P.KohnShamDensity.apply(vx, pb, v_fixed)
            return torch.sum(m * (rd - rho) ** 2).item()

    v = v0.clone().requires_grad_(True)
    rho = P.KohnShamDensity.apply(v, pb, v_fixed)
    torch.sum(m * (rd - rho) ** 2).backward()
    g = v.grad.clone()
    dirs = W.random_directions(pb.L, 16, seed=3100)
    h = 1e-4
    fd, ad = [], []
    for d in dirs:
        dv = t(d / np.abs(d).max())
        fd.append((loss_of(v0 + h * dv) - loss_of(v0 - h * dv)) / (2 * h))
        ad.append(torch.dot(g, dv).item())
    fd, ad = np.array(fd), np.array(ad)
    err = np.linalg.norm(fd - ad) / np.linalg.norm(ad)
    print(f"16 directions: |FD - adjoint| / |adjoint| = {err:.3e}")
    assert err <= 1e-4
