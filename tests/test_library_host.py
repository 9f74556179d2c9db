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
    mesh = P.MeshDesc(lo=-8.0, hi=8.0, ncell=ncell, order=order)
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


def test_create_rejects_bad_arguments():
    import paper_2510_10529_b300 as P
    with pytest.raises(P.InvdftError):
        P.invdft_create_mesh(P.MeshDesc(lo=0.0, hi=1.0, ncell=2, order=3), P.Opts(nstates=2))
    with pytest.raises(P.InvdftError):
        P.invdft_create_mesh(P.MeshDesc(lo=0.0, hi=1.0, ncell=2, order=2), P.Opts(nstates=0))
    with pytest.raises(P.InvdftError):
        P.invdft_create_mesh(P.MeshDesc(lo=1.0, hi=0.0, ncell=2, order=2), P.Opts(nstates=2))
