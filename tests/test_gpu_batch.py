"""Batched multi-problem execution (invdft_batch_*) against the oracle.

Four independent problems of uneven mesh size, element order and subspace
width are stepped together; every problem must follow the oracle's L-BFGS
trajectory (Eq. 21) as it does when stepped alone."""
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
from oracle import fe, inverse, ks  # noqa: E402


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


# (lo, hi, ncell, order, nuclear charge, electrons, nstates): Q2 and Q4, widths
# 4 to 8 (a width that is not a multiple of four takes the scalar paths)
CASES = [(-8.0, 8.0, 8, 2, 2.0, 2.0, 8),
         (-6.0, 6.0, 4, 4, 2.0, 2.0, 6),
         (-6.0, 6.0, 6, 2, 4.0, 4.0, 7),
         (-5.0, 5.0, 3, 4, 2.0, 2.0, 4)]
DEGREE = 16


def _case(lo, hi, n, p, Z, Ne, nst):
    mesh = fe.Mesh(lo, hi, n, p)
    xyz = mesh.coords()
    v = W.smeared_coulomb(xyz, np.array([[0.2, -0.3, 0.1]]), np.array([Z]), 0.5)
    bump = 0.1 * np.exp(-np.sum((xyz - 0.5) ** 2, 1))
    rho_d = ks.forward(mesh, v + bump, Ne, nst, 0.0)["rho"]
    op = inverse.Problem(mesh=mesh, v_fixed=v, rho_data=rho_d, w=np.ones(mesh.L),
                         n_electrons=Ne, nstates=nst, kT=0.0)
    return mesh, v, rho_d, op


def _gpu_problem(case, v):
    import paper_2510_10529_b300 as P
    lo, hi, n, p, Z, Ne, nst = case
    pb = P.Problem(lo, hi, n, p, nst, n_electrons=Ne, kT=0.0, prec="mixed",
                   cheb_degree=DEGREE, eig_tol=1e-10, adj_tol=1e-11)
    pb.set_potential(_cuda(v))
    return pb


@pytest.fixture(scope="module")
def cases():
    return [_case(*c) for c in CASES]


def test_batch_steps_follow_the_oracle(cases):
    import paper_2510_10529_b300 as P
    problems = [_gpu_problem(c, d[1]) for c, d in zip(CASES, cases)]
    batch = P.Batch(problems)
    v_xc = [_cuda(np.zeros(d[0].L)) for d in cases]
    rd = [_cuda(d[2]) for d in cases]
    w = [_cuda(np.ones(d[0].L)) for d in cases]
    states = [inverse.State(v_xc=np.zeros(d[0].L)) for d in cases]
    for _ in range(2):
        stats, status = batch.step(rd, w, v_xc)
        assert all(s == 0 for s in status), status
        for b, d in enumerate(cases):
            states[b] = inverse.step(d[3], states[b])
            vg = v_xc[b].cpu().numpy()
            ref = states[b].v_xc
            err = np.linalg.norm(vg - ref) / np.linalg.norm(ref)
            print(f"problem {b}: v_xc rel err {err:.2e}, loss {stats[b]['loss']:.6e} "
                  f"vs {states[b].loss:.6e}")
            assert err <= 1e-6
            assert abs(stats[b]["loss"] - states[b].loss) <= 1e-6 * states[b].loss
    info = batch.info()
    print(info)
    assert info["tuned"] and info["launches"] > 0
    assert all(c in (8, 16, 32) for c in info["chunk_cols"])
    batch.close()


def test_batch_matches_problems_stepped_alone(cases):
    import paper_2510_10529_b300 as P
    alone = [_gpu_problem(c, d[1]) for c, d in zip(CASES, cases)]
    together = [_gpu_problem(c, d[1]) for c, d in zip(CASES, cases)]
    batch = P.Batch(together)
    va = [_cuda(np.zeros(d[0].L)) for d in cases]
    vb = [_cuda(np.zeros(d[0].L)) for d in cases]
    rd = [_cuda(d[2]) for d in cases]
    w = [_cuda(np.ones(d[0].L)) for d in cases]
    stats_b, _ = batch.step(rd, w, vb)
    for b in range(len(cases)):
        st = alone[b].step(rd[b], w[b], va[b])
        diff = (va[b] - vb[b]).norm().item() / va[b].norm().item()
        assert diff <= 1e-7, (b, diff)
        assert abs(st["loss"] - stats_b[b]["loss"]) <= 1e-7 * st["loss"]
    batch.close()


def test_batch_phase_wait_timeout_is_reported(cases):
    """The timeout path of the persistent filter kernel's bounded phase waits,
    without any device fault: with the wait limit at zero, the first wait of a
    CTA for the previous phase of a problem gives up at once, the kernel sets
    its error word and every CTA leaves; the step must return INVDFT_ETIMEOUT.
    With the default limit restored, the same batch steps normally again (the
    context and the handles stay usable)."""
    import paper_2510_10529_b300 as P
    from paper_2510_10529_b300._lib import INVDFT_ETIMEOUT
    problems = [_gpu_problem(c, d[1]) for c, d in zip(CASES, cases)]
    batch = P.Batch(problems)
    v_xc = [_cuda(np.zeros(d[0].L)) for d in cases]
    rd = [_cuda(d[2]) for d in cases]
    w = [_cuda(np.ones(d[0].L)) for d in cases]
    batch.step(rd, w, v_xc)                      # first step: autotuning, normal waits
    batch.set_wait_limit(0)
    with pytest.raises(P.InvdftError) as ei:
        batch.step(rd, w, v_xc)
    assert ei.value.status == INVDFT_ETIMEOUT, str(ei.value)
    assert "timed out" in str(ei.value)
    batch.set_wait_limit(-1)
    v_xc = [_cuda(np.zeros(d[0].L)) for d in cases]
    for p in problems:
        p.reset()
    stats, status = batch.step(rd, w, v_xc)
    assert all(s == 0 for s in status), status
    assert all(np.isfinite(st["loss"]) for st in stats)
    batch.close()


def _batch16_shaped():
    """The sixteen problems of the batched workload (workloads.batch16: its
    seeded orders, electron counts, nuclei, bumps, widths, degree and kT) on
    meshes of 3 to 5 cells per axis, which the oracle steps in seconds."""
    out = []
    for wl in W.batch16():
        n = 3 + wl.ncell % 3
        mesh = fe.Mesh(wl.lo, wl.hi, n, wl.order)
        xyz = mesh.coords()
        v = W.smeared_coulomb(xyz, wl.nuclei_R, wl.nuclei_Z, wl.smear)
        bump = W.gaussian_bumps(xyz, wl.bump_c, wl.bump_a, wl.bump_b)
        rho_d = ks.forward(mesh, v + bump, wl.n_electrons, wl.nstates, wl.kT)["rho"]
        op = inverse.Problem(mesh=mesh, v_fixed=v, rho_data=rho_d, w=np.ones(mesh.L),
                             n_electrons=wl.n_electrons, nstates=wl.nstates, kT=wl.kT)
        loss0 = inverse.evaluate(op, np.zeros(mesh.L), with_grad=False)[0]
        out.append((wl, n, mesh, v, rho_d, op, loss0))
    return out


def test_sixteen_problem_batch_follows_the_oracle():
    """All sixteen problems of the batched workload's recipe stepped twice as
    one batch (persistent filter kernel); every problem's v_xc and loss follow
    the oracle's L-BFGS trajectory (1e-6 relative)."""
    import paper_2510_10529_b300 as P
    cases16 = _batch16_shaped()
    problems = []
    for wl, n, mesh, v, _, _, _ in cases16:
        pb = P.Problem(wl.lo, wl.hi, n, wl.order, wl.nstates, n_electrons=wl.n_electrons,
                       kT=wl.kT, prec="mixed", cheb_degree=wl.cheb_degree, eig_tol=1e-10,
                       adj_tol=1e-11)
        pb.set_potential(_cuda(v))
        problems.append(pb)
    batch = P.Batch(problems)
    v_xc = [_cuda(np.zeros(c[2].L)) for c in cases16]
    rd = [_cuda(c[4]) for c in cases16]
    w = [_cuda(np.ones(c[2].L)) for c in cases16]
    states = [inverse.State(v_xc=np.zeros(c[2].L)) for c in cases16]
    worst = 0.0
    compared = set()
    for _ in range(2):
        stats, status = batch.step(rd, w, v_xc)
        assert all(s == 0 for s in status), status
        for b, c in enumerate(cases16):
            states[b] = inverse.step(c[5], states[b])
            if c[6] < 1e-6:
                # the start already reproduces rho_data to ~1e-3 in L2 (the bump
                # barely moves the density on this coarse mesh): the first
                # step's direction and the line search's decisions then rest
                # on losses that differ at rounding level, on both sides, so
                # the trajectory is not reproducible; these problems are only
                # required to step without error
                assert np.isfinite(stats[b]["loss"]), b
                continue
            compared.add(b)
            ref = states[b].v_xc
            err = np.linalg.norm(v_xc[b].cpu().numpy() - ref) / np.linalg.norm(ref)
            worst = max(worst, err)
            assert err <= 1e-6, (b, err)
            assert abs(stats[b]["loss"] - states[b].loss) <= 1e-6 * states[b].loss, b
    assert len(compared) >= 10, compared
    print(f"16-problem batch: {len(compared)} trajectories compared, worst v_xc rel err "
          f"{worst:.2e}, info {batch.info()}")
    batch.close()
