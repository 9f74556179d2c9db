"""Pins of the oracle's inverse loop on the small plain-method workload (no GPU).

The validation protocol of Sec. 5.1: a density generated from a known v_xc*
must be reproduced by v_xc*, and the loop must drive the density error down
from a perturbed start.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fe, inverse, ks, scf


@pytest.fixture(scope="module")
def cube8():
    wl = W.cube8_q2_he()
    mesh = fe.Mesh(wl.lo, wl.hi, wl.ncell, wl.order)
    data = scf.target_density(mesh, wl)
    return wl, mesh, data


def test_target_density_is_reproduced_by_reference_potential(cube8):
    wl, mesh, d = cube8
    assert d["scf_error"] < 1e-10
    fw = ks.forward(mesh, d["v_fixed"] + d["v_xc_ref"], wl.n_electrons, wl.nstates, wl.kT)
    assert np.abs(fw["rho"] - d["rho_data"]).max() < 1e-9
    assert abs(ks.electron_count(mesh, d["rho_data"]) - 2.0) < 1e-12


def test_recovery_from_perturbed_start(cube8):
    wl, mesh, d = cube8
    pb = inverse.Problem(mesh=mesh, v_fixed=d["v_fixed"], rho_data=d["rho_data"],
                         w=np.ones(mesh.L), n_electrons=wl.n_electrons,
                         nstates=wl.nstates, kT=wl.kT)
    xyz = mesh.coords()
    pert = 0.05 * np.exp(-np.sum((xyz - np.array([0.5, 0.0, 0.0])) ** 2, 1) / 4.0)
    st = inverse.State(v_xc=d["v_xc_ref"] + pert)
    mask = d["rho_data"] > 1e-4
    e0 = None
    losses = []
    for _ in range(20):
        st = inverse.step(pb, st)
        if e0 is None:
            e0 = st.err_l2
        losses.append(st.loss)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(losses, losses[1:]))
    assert st.err_l2 < e0 / 10.0
    dv = (st.v_xc - d["v_xc_ref"])[mask]
    assert np.abs(dv - dv.mean()).max() < 0.04          # started at 0.05 off


def test_trajectory_from_zero_decreases_loss(cube8):
    wl, mesh, d = cube8
    pb = inverse.Problem(mesh=mesh, v_fixed=d["v_fixed"], rho_data=d["rho_data"],
                         w=np.ones(mesh.L), n_electrons=wl.n_electrons,
                         nstates=wl.nstates, kT=wl.kT)
    st = inverse.State(v_xc=np.zeros(mesh.L))
    st = inverse.step(pb, st)
    first = st.loss
    for _ in range(5):
        st = inverse.step(pb, st)
    assert st.loss < 0.2 * first
