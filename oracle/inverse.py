"""One iteration of the inverse-DFT loop (oracle; test infrastructure only).

Follows the loop of Sec. 3.2.1 (Fig. "algorithm flowchart", Eq. 21): at the
current v_xc solve the KS problem (Eq. 19), evaluate the loss (Eq. 1), solve the
adjoint problems (Eq. 20 with Eq. 8-10) and form the gradient (Eq. 11, 22),
masked where rho_data < tau_BC (Sec. 3.1.2); then take an L-BFGS step with a
backtracking line search (readings in lbfgs.py).  Each trial point of the line
search costs one KS solve; the adjoint is solved only at the accepted point.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import adjoint as adj
from . import lbfgs
from .fe import Mesh
from .ks import forward


@dataclass
class Problem:
    mesh: Mesh
    v_fixed: np.ndarray          # v_ext + v_H[rho_data] at the unknown nodes
    rho_data: np.ndarray
    w: np.ndarray
    n_electrons: float
    nstates: int
    kT: float
    tau_bc: float = 1e-6


@dataclass
class State:
    v_xc: np.ndarray
    hist: lbfgs.History = field(default_factory=lbfgs.History)
    loss: float | None = None
    err_l2: float | None = None
    grad: np.ndarray | None = None
    fw: dict | None = None


def evaluate(pb: Problem, v_xc: np.ndarray, with_grad: bool = True):
    """KS solve, loss and (optionally) the masked gradient at v_xc."""
    fw = forward(pb.mesh, pb.v_fixed + v_xc, pb.n_electrons, pb.nstates, pb.kT)
    loss, e = adj.loss_and_error(pb.mesh, fw["rho"], pb.rho_data, pb.w)
    if not with_grad:
        return loss, e, None, fw
    G = adj.loss_upstream(pb.mesh, fw["rho"], pb.rho_data, pb.w)
    P, _ = adj.adjoint(pb.mesh, pb.v_fixed + v_xc, fw["eps"], fw["psi"], fw["f"],
                       fw["dfde"], G)
    grad = adj.gradient(fw["psi"], P, pb.rho_data, pb.tau_bc)
    return loss, e, grad, fw


def step(pb: Problem, st: State) -> State:
    """One L-BFGS iteration (Eq. 21) from st; returns the new state."""
    if st.grad is None:
        st.loss, st.err_l2, st.grad, st.fw = evaluate(pb, st.v_xc)
    d = lbfgs.direction(st.grad, st.hist)
    slope = float(st.grad @ d)
    alpha = 1.0
    for trial in range(lbfgs.MAX_TRIALS):
        v_try = st.v_xc + alpha * d
        L_try, _, _, _ = evaluate(pb, v_try, with_grad=False)
        if L_try <= st.loss + lbfgs.ARMIJO_C * alpha * slope or trial == lbfgs.MAX_TRIALS - 1:
            break
        alpha *= 0.5
    loss, e, grad, fw = evaluate(pb, v_try)
    st.hist.push(v_try - st.v_xc, grad - st.grad)
    return State(v_xc=v_try, hist=st.hist, loss=loss, err_l2=e, grad=grad, fw=fw)
