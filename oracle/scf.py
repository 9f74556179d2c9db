"""Self-consistent generation of a target density (oracle; input recipe, test only).

The paper's target densities come from correlated calculations that are not
available; the synthetic stand-in is a density generated by a Kohn-Sham model
with a known exchange-correlation potential v_xc* = v_x^LDA[rho] + bumps, so
that the inverse problem has a known answer (the validation protocol of
Sec. 5.1, recovering a potential from the density it generated).

Iterate rho -> KS density at v_ext + v_H[rho] + v_xc*[rho] with Anderson
(Pulay) mixing until the L2 change is below tol.  Afterwards rho_data is the
last output density and v_H is frozen at v_H[rho_data] (Eq. 2: the Hartree
potential of the target density).
"""
from __future__ import annotations

import numpy as np

import workloads as W
from .fe import Mesh
from .ks import forward
from .potentials import hartree


def target_density(mesh: Mesh, wl: W.Workload, tol: float = 1e-11, maxit: int = 300,
                   mix: float = 0.4, depth: int = 6):
    xyz = mesh.coords()
    m = mesh.mass()
    v_ext = W.smeared_coulomb(xyz, wl.nuclei_R, wl.nuclei_Z, wl.smear)
    bump = W.gaussian_bumps(xyz, wl.bump_c, wl.bump_a, wl.bump_b)
    rho = forward(mesh, v_ext, wl.n_electrons, wl.nstates, wl.kT)["rho"]
    R_hist, F_hist = [], []
    err = np.inf
    for it in range(maxit):
        v = v_ext + hartree(mesh, rho) + W.lda_exchange(rho) + bump
        out = forward(mesh, v, wl.n_electrons, wl.nstates, wl.kT)
        res = out["rho"] - rho
        err = float(np.sqrt(np.sum(m * res * res)))
        if err < tol:
            rho = out["rho"]
            break
        R_hist.append(res.copy())
        F_hist.append(rho.copy())
        if len(R_hist) > depth:
            R_hist.pop(0)
            F_hist.pop(0)
        if len(R_hist) >= 2:
            dR = np.array([R_hist[j + 1] - R_hist[j] for j in range(len(R_hist) - 1)]).T
            dF = np.array([F_hist[j + 1] - F_hist[j] for j in range(len(F_hist) - 1)]).T
            Wm = np.sqrt(m)[:, None]
            gam, *_ = np.linalg.lstsq(Wm * dR, np.sqrt(m) * res, rcond=None)
            rho = rho + mix * res - (dF + mix * dR) @ gam
        else:
            rho = rho + mix * res
        rho = np.maximum(rho, 0.0)
    v_H = hartree(mesh, rho)
    v_xc_ref = W.lda_exchange(rho) + bump
    return dict(rho_data=rho, v_ext=v_ext, v_H=v_H, v_fixed=v_ext + v_H,
                v_xc_ref=v_xc_ref, scf_error=err, scf_iters=it + 1)
