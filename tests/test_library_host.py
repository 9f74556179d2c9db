"""Host-side checks of libinvdft (no GPU): every symbol that include/invdft.h
declares is exported, and the host-only calls (mesh creation, workspace size,
node coordinates) agree with the oracle's discretisation."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(invdft_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for must in ("invdft_create_mesh", "invdft_set_potential", "invdft_forward_solve",
                 "invdft_adjoint_solve", "invdft_loss_grad", "invdft_step", "invdft_apply_h"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2510_10529_b300 import library_path
    lib = C.CDLL(library_path())
    missing = [n for n in sorted(_declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("ncell,order", [(8, 2), (3, 4)])
def test_node_coordinates_match_oracle(ncell, order):
    import paper_2510_10529_b300 as P
    from oracle import fe
    mesh = P.MeshDesc.make(-8.0, 8.0, ncell, order)
    opts = P.Opts(nstates=4, n_electrons=2.0)
    h, L = P.invdft_create_mesh(mesh, opts)
    try:
        om = fe.Mesh(-8.0, 8.0, ncell, order)
        assert L == om.L
        xyz = P.invdft_node_coords(h, L)
        np.testing.assert_allclose(xyz, om.coords(), atol=1e-13)
        assert P.invdft_workspace_size(h) > 0
    finally:
        P.invdft_destroy(h)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_graded_box_node_coordinates_match_oracle(order):
    """A box with different extents and cell counts per axis, cells graded
    towards two points on x and equal on y and z (invdft_mesh_desc with
    per-axis breaks), against the graded-mesh oracle's nodes."""
    import paper_2510_10529_b300 as P
    from oracle import graded
    bx = graded.graded_breaks(-6.0, 5.0, 5, [-1.0, 2.0], 0.6, 3.0)
    by = np.linspace(-4.0, 4.0, 4)
    bz = np.linspace(-3.0, 5.0, 3)
    mesh = P.MeshDesc.make([-6.0, -4.0, -3.0], [5.0, 4.0, 5.0], [5, 3, 2], order,
                           breaks=[bx, None, bz])
    h, L = P.invdft_create_mesh(mesh, P.Opts(nstates=2, n_electrons=2.0))
    try:
        om = graded.GradedMesh(bx, by, bz, order)
        assert L == om.L
        np.testing.assert_allclose(P.invdft_node_coords(h, L), om.coords(), atol=1e-13)
    finally:
        P.invdft_destroy(h)


def test_create_rejects_bad_breaks():
    import paper_2510_10529_b300 as P
    bad = [np.array([0.0, 0.6, 0.5, 1.0]), None, None]      # not increasing
    with pytest.raises(P.InvdftError):
        P.invdft_create_mesh(P.MeshDesc.make(0.0, 1.0, [3, 2, 2], 2, breaks=bad),
                             P.Opts(nstates=2))
    off = [np.array([0.1, 0.5, 1.0]), None, None]            # does not start at lo
    with pytest.raises(P.InvdftError):
        P.invdft_create_mesh(P.MeshDesc.make(0.0, 1.0, [2, 2, 2], 2, breaks=off),
                             P.Opts(nstates=2))


def test_create_rejects_bad_arguments():
    import paper_2510_10529_b300 as P
    with pytest.raises(P.InvdftError):
        P.invdft_create_mesh(P.MeshDesc.make(0.0, 1.0, 2, 3), P.Opts(nstates=2))
    with pytest.raises(P.InvdftError):
        P.invdft_create_mesh(P.MeshDesc.make(0.0, 1.0, 2, 2), P.Opts(nstates=0))
    with pytest.raises(P.InvdftError):
        P.invdft_create_mesh(P.MeshDesc.make(1.0, 0.0, 2, 2), P.Opts(nstates=2))


def test_device_calls_validate_on_the_host_first():
    """Every device-facing call checks its handle and arguments on the host
    before any CUDA call: on a handle without a bound workspace (or with null
    arguments) it returns an error code and leaves a message, so this runs
    without a GPU.  The non-null pointers below are never dereferenced."""
    import paper_2510_10529_b300 as P
    from paper_2510_10529_b300._lib import INVDFT_EINVAL, INVDFT_ENOMEM, lib
    h, L = P.invdft_create_mesh(P.MeshDesc.make(-4.0, 4.0, 2, 2),
                                P.Opts(nstates=2, n_electrons=2.0))
    fake = C.c_void_p(0x1000)
    st = P.Stats()
    loss = C.c_double()
    try:
        calls = {
            "bind_workspace": lambda: lib.invdft_bind_workspace(h, None, 0, None),
            "mass_diag": lambda: lib.invdft_mass_diag(h, fake, None),
            "set_potential": lambda: lib.invdft_set_potential(h, fake, None, None),
            "apply_h": lambda: lib.invdft_apply_h(h, fake, C.c_void_p(0x2000), 4,
                                                  P.INVDFT_FP64, None),
            "apply_h aliasing": lambda: lib.invdft_apply_h(h, fake, fake, 4, P.INVDFT_FP64, None),
            "chebyshev_filter": lambda: lib.invdft_chebyshev_filter(
                h, fake, C.c_void_p(0x2000), 2, 8, 0.0, 1.0, -1.0, P.INVDFT_FP64, None),
            "forward_solve": lambda: lib.invdft_forward_solve(h, None, None, None, None,
                                                              C.byref(st), None),
            "adjoint_solve": lambda: lib.invdft_adjoint_solve(h, fake, None, C.byref(st), None),
            "density_vjp": lambda: lib.invdft_density_vjp(h, fake, fake, C.byref(st), None),
            "loss_grad": lambda: lib.invdft_loss_grad(h, fake, fake, C.byref(loss), fake,
                                                      C.byref(st), None),
            "step": lambda: lib.invdft_step(h, fake, fake, fake, C.byref(st), None),
            "initial_guess": lambda: lib.invdft_initial_guess(h, fake, fake, 1e-2, 1.0, 1, fake,
                                                              None),
            "q1_to_nodes": lambda: lib.invdft_q1_to_nodes(h, 4, fake, fake, None),
            "grad_to_q1": lambda: lib.invdft_grad_to_q1(h, 4, fake, fake, None),
        }
        for name, call in calls.items():
            code = call()
            assert code in (INVDFT_EINVAL, INVDFT_ENOMEM), (name, code)
            assert lib.invdft_last_error(h), name
        # null arguments are rejected before the handle's state is looked at
        assert lib.invdft_adjoint_solve(h, None, None, None, None) == INVDFT_EINVAL
        assert lib.invdft_step(h, fake, None, fake, None, None) == INVDFT_EINVAL
        assert lib.invdft_apply_h(None, fake, fake, 4, P.INVDFT_FP64, None) == INVDFT_EINVAL
        # a batch needs bound mixed-precision problems
        arr = (C.c_void_p * 1)(h.value)
        out = C.c_void_p()
        assert lib.invdft_batch_create(arr, 1, C.byref(out)) == INVDFT_EINVAL
        assert lib.invdft_batch_create(None, 1, C.byref(out)) == INVDFT_EINVAL
    finally:
        P.invdft_destroy(h)


def test_tuning_and_timing_calls_on_the_host():
    """The tuning and timing entry points work on a handle without a GPU: the
    balanced H~X schedule is accepted as a fixed segment length, negative
    lengths and variants out of range are rejected, nothing is tuned before
    the first launch, and the deflation timing totals start at zero."""
    import numpy as np

    import paper_2510_10529_b300 as P
    from paper_2510_10529_b300._lib import INVDFT_EINVAL, INVDFT_OK, lib
    h, _ = P.invdft_create_mesh(P.MeshDesc.make(-4.0, 4.0, 2, 4),
                                P.Opts(nstates=2, n_electrons=2.0))
    try:
        n32, n64 = P.invdft_tune_hx(h, 0, P.INVDFT_HX_SEG_BALANCED)
        assert n32 >= 1 and n64 >= 1
        assert lib.invdft_tune_hx(h, 0, -5, None) == INVDFT_EINVAL
        assert lib.invdft_tune_hx(h, max(n32, n64), 0, None) == INVDFT_EINVAL
        assert lib.invdft_tune_hx(h, -1, 0, None) == INVDFT_OK
        cfg = P.invdft_hx_config(h, 60, False)
        assert all(v == (-1, -1) for v in cfg.values())
        d = P.invdft_profile_deflation(h)
        assert all(d[k][f] == 0.0 for k in ("gram", "update") for f in ("ms", "bytes", "launches"))
        assert lib.invdft_profile_deflation(h, None) == INVDFT_EINVAL
        assert lib.invdft_profile_deflation(None, np.zeros(8).ctypes.data_as(C.c_void_p)) \
            == INVDFT_EINVAL
    finally:
        P.invdft_destroy(h)
