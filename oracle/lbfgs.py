"""Limited-memory BFGS update of v_xc (oracle; test infrastructure only).

Eq. 21: v^(t+1) = v^(t) - alpha_t B_t^-1 f_t, with B_t^-1 built from the last
m_h pairs (s, y) by the two-loop recursion of Nocedal (1980).  The paper does
not fix the history length, the initial matrix or the step rule; the readings
used here (shared with the CUDA path) are:
  * history m_h = 10, initial matrix gamma I with gamma = s^T y / y^T y of the
    newest pair;
  * with no pair yet, the first trial step moves v by 0.1 Ha at the node of
    largest |grad| (direction -0.1 grad / max|grad|);
  * trial step alpha = 1, then halving while the Armijo condition
    L(v + alpha d) <= L(v) + 1e-4 alpha grad^T d fails, at most 10 trials
    (the last trial is taken regardless);
  * a pair with s^T y <= 1e-12 |s| |y| is not stored.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HISTORY = 10
FIRST_STEP = 0.1
ARMIJO_C = 1e-4
MAX_TRIALS = 10


@dataclass
class History:
    S: list = field(default_factory=list)
    Y: list = field(default_factory=list)
    m: int = HISTORY

    def push(self, s: np.ndarray, y: np.ndarray) -> bool:
        sy = float(s @ y)
        if sy <= 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            return False
        self.S.append(s.copy())
        self.Y.append(y.copy())
        if len(self.S) > self.m:
            self.S.pop(0)
            self.Y.pop(0)
        return True


def direction(grad: np.ndarray, hist: History) -> np.ndarray:
    """d = -B^-1 grad by the two-loop recursion."""
    if not hist.S:
        gmax = float(np.max(np.abs(grad)))
        return -FIRST_STEP * grad / gmax if gmax > 0 else np.zeros_like(grad)
    q = grad.copy()
    k = len(hist.S)
    alpha = np.zeros(k)
    rho = np.array([1.0 / float(hist.Y[j] @ hist.S[j]) for j in range(k)])
    for j in range(k - 1, -1, -1):
        alpha[j] = rho[j] * float(hist.S[j] @ q)
        q -= alpha[j] * hist.Y[j]
    gamma = float(hist.S[-1] @ hist.Y[-1]) / float(hist.Y[-1] @ hist.Y[-1])
    r = gamma * q
    for j in range(k):
        beta = rho[j] * float(hist.Y[j] @ r)
        r += (alpha[j] - beta) * hist.S[j]
    return -r
