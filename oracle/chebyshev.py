"""Chebyshev filter of ChFSI (oracle; test infrastructure only).

Sec. 3.2.2: Y = T_m(c1 H~ + c2) X maps the unwanted spectrum [a, b] of H~ to
[-1, 1], where T_m stays bounded, and amplifies the wanted part below a.
With e = (b - a)/2 and c = (b + a)/2 the oracle uses the normalised filter of
Zhou et al. (2006),
    p_m(t) = T_m((t - c)/e) / T_m((a0 - c)/e),
a0 being an estimate of the lowest eigenvalue, which keeps the wanted
components O(1).  Two independent evaluations are provided: the scaled
three-term recurrence on vectors (what the CUDA path computes), and the
closed form T_m(x) = cos(m arccos x) on [-1,1], cosh(m arccosh |x|) sign^m
outside, for scalars.
"""
from __future__ import annotations

import numpy as np


def cheb_T(m: int, x):
    """T_m(x) by its closed form."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(m * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** m * np.cosh(m * np.arccosh(np.abs(xo)))
    return out


def filter_scalar(m: int, a: float, b: float, a0: float, t):
    """p_m(t) = T_m((t-c)/e) / T_m((a0-c)/e) by the closed form."""
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    return cheb_T(m, (np.asarray(t) - c) / e) / cheb_T(m, np.array([(a0 - c) / e]))[0]


def filter_apply(apply_H, X: np.ndarray, m: int, a: float, b: float, a0: float):
    """Scaled three-term recurrence Y = p_m(H~) X (Zhou et al. 2006).

    sigma_1 = e/(a0 - c); Y_1 = (sigma_1/e)(H - c)X;
    sigma_{k+1} = 1/(2/sigma_1 - sigma_k);
    Y_{k+1} = (2 sigma_{k+1}/e)(H - c)Y_k - sigma_k sigma_{k+1} Y_{k-1}.
    """
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    sigma1 = e / (a0 - c)
    sigma = sigma1
    Yprev = X
    Y = (sigma1 / e) * (apply_H(X) - c * X)
    for _ in range(2, m + 1):
        sigma_new = 1.0 / (2.0 / sigma1 - sigma)
        Ynew = (2.0 * sigma_new / e) * (apply_H(Y) - c * Y) - (sigma * sigma_new) * Yprev
        Yprev, Y, sigma = Y, Ynew, sigma_new
    return Y
