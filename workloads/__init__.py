"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the inverse-DFT method itself: it only draws
seeded random numbers (nuclear positions and charges, bump centres, random
vector blocks) and evaluates closed-form *input* fields (a Gaussian-smeared
Coulomb potential, Gaussian bumps, a Gaussian model density and its exact
Hartree potential) at coordinates the caller supplies.  Both the CUDA path and
the CPU oracle consume what it returns; neither is imported here.

Seeds follow one rule: seed = 1000 * (workload index) + (problem index).

Workloads (the paper's molecular densities are not available, so these stand
in for them with the same shape: a few to a hundred electrons, smeared nuclei,
millions of finite-element nodes):

  cube8_q2_he   : [-8,8]^3, 8^3 cells Q2, 2 electrons, one Z=2 nucleus at the
                  origin, reference v_xc = LDA exchange + one 0.1 Ha bump.
  cube32_q4_hx  : [-12,12]^3, 32^3 cells Q4, 64 random unit-norm vectors,
                  8 nuclei with Z in 1..8 in the inner half of the box.
  cube24_q4_e20 : [-10,10]^3, 24^3 cells Q4, 20 electrons, 16 states,
                  6 nuclei (charges rescaled to neutrality), 3 bumps.
  cube32_q4_e100: [-14,14]^3, 32^3 cells Q4, 100 electrons, 60 states,
                  12 nuclei (charges rescaled to neutrality).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import erf

KT_DEFAULT = 1.5834e-3          # k_B T at 500 K in hartree


@dataclass
class Workload:
    name: str
    lo: float
    hi: float
    ncell: int
    order: int
    n_electrons: float
    nstates: int
    kT: float
    nuclei_R: np.ndarray            # [n_nuc, 3]
    nuclei_Z: np.ndarray            # [n_nuc]
    smear: float = 0.5              # nuclear smearing width (bohr)
    bump_c: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    bump_a: np.ndarray = field(default_factory=lambda: np.zeros(0))
    bump_b: np.ndarray = field(default_factory=lambda: np.zeros(0))
    cheb_degree: int = 30
    seed: int = 0

    @property
    def n_nodes_axis(self) -> int:
        return self.ncell * self.order + 1

    @property
    def n_interior(self) -> int:
        return (self.ncell * self.order - 1) ** 3


def _rng(workload_index: int, problem_index: int = 0) -> np.random.Generator:
    return np.random.default_rng(1000 * workload_index + problem_index)


def cube8_q2_he() -> Workload:
    """Small plain-method case: one Z=2 nucleus, 2 electrons, kT = 0."""
    rng = _rng(1)
    centre = rng.uniform(-1.0, 1.0, size=(1, 3))
    return Workload(name="cube8_q2_he", lo=-8.0, hi=8.0, ncell=8, order=2,
                    n_electrons=2.0, nstates=8, kT=0.0,
                    nuclei_R=np.zeros((1, 3)), nuclei_Z=np.array([2.0]),
                    bump_c=centre, bump_a=np.array([0.1]), bump_b=np.array([1.0]),
                    cheb_degree=20, seed=1000)


def cube32_q4_hx() -> Workload:
    """Operator benchmark: 8 smeared nuclei, no electrons (only H~X is run)."""
    rng = _rng(2)
    Z = rng.integers(1, 9, size=8).astype(np.float64)
    R = rng.uniform(-6.0, 6.0, size=(8, 3))
    return Workload(name="cube32_q4_hx", lo=-12.0, hi=12.0, ncell=32, order=4,
                    n_electrons=0.0, nstates=64, kT=0.0,
                    nuclei_R=R, nuclei_Z=Z, seed=2000)


def _neutral_charges(rng, n, n_electrons):
    z = rng.integers(1, 9, size=n).astype(np.float64)
    return z * (n_electrons / z.sum())


def cube24_q4_e20() -> Workload:
    rng = _rng(3)
    Z = _neutral_charges(rng, 6, 20.0)
    R = rng.uniform(-5.0, 5.0, size=(6, 3))
    pick = rng.integers(0, 6, size=3)
    dirs = rng.normal(size=(3, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    radii = 1.5 * rng.uniform(0.0, 1.0, size=(3, 1)) ** (1.0 / 3.0)
    C = R[pick] + dirs * radii
    A = rng.uniform(-0.1, 0.1, size=3)
    return Workload(name="cube24_q4_e20", lo=-10.0, hi=10.0, ncell=24, order=4,
                    n_electrons=20.0, nstates=16, kT=KT_DEFAULT,
                    nuclei_R=R, nuclei_Z=Z, bump_c=C, bump_a=A,
                    bump_b=np.ones(3), cheb_degree=30, seed=3000)


def cube32_q4_e100() -> Workload:
    rng = _rng(4)
    Z = _neutral_charges(rng, 12, 100.0)
    R = rng.uniform(-7.0, 7.0, size=(12, 3))
    return Workload(name="cube32_q4_e100", lo=-14.0, hi=14.0, ncell=32, order=4,
                    n_electrons=100.0, nstates=60, kT=KT_DEFAULT,
                    nuclei_R=R, nuclei_Z=Z, cheb_degree=30, seed=4000)


def batch16() -> list:
    """Sixteen independent small problems for batched execution: cells per axis
    uniform in 8..16, order 2 or 4, electrons from {2, 4, 6, 10, 14, 20}, one
    to three nuclei (charges rescaled to the electron count) in the inner half
    of a [-8, 8]^3 box, one Gaussian bump each, nstates = N_e/2 + ceil(N_e/10)
    + 2, a common Chebyshev degree 20, kT = 500 K."""
    out = []
    for i in range(16):
        rng = _rng(5, i)
        ncell = int(rng.integers(8, 17))
        order = int(rng.choice([2, 4]))
        ne = float(rng.choice([2, 4, 6, 10, 14, 20]))
        nn = int(rng.integers(1, 4))
        Z = _neutral_charges(rng, nn, ne)
        R = rng.uniform(-4.0, 4.0, size=(nn, 3))
        centre = R[int(rng.integers(0, nn))] + rng.uniform(-1.0, 1.0, size=3)
        out.append(Workload(name=f"batch16_{i}", lo=-8.0, hi=8.0, ncell=ncell, order=order,
                            n_electrons=ne, nstates=int(ne // 2 + math.ceil(ne / 10) + 2),
                            kT=KT_DEFAULT, nuclei_R=R, nuclei_Z=Z,
                            bump_c=centre[None, :], bump_a=np.array([0.1]),
                            bump_b=np.array([1.0]), cheb_degree=20, seed=5000 + i))
    return out


def tiny(ncell=3, order=2, half=4.0, n_electrons=2.0, nstates=4, kT=0.0,
         Z=(2.0,), R=((0.0, 0.0, 0.0),), seed=9000) -> Workload:
    """Tiny meshes for brute-force checks (dense eigensolves, finite differences)."""
    return Workload(name=f"tiny{ncell}_q{order}", lo=-half, hi=half, ncell=ncell,
                    order=order, n_electrons=n_electrons, nstates=nstates, kT=kT,
                    nuclei_R=np.asarray(R, dtype=np.float64).reshape(-1, 3),
                    nuclei_Z=np.asarray(Z, dtype=np.float64), seed=seed)


# ---------------------------------------------------------------- random draws

def random_block(n_rows: int, ncol: int, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) columns normalised to unit 2-norm, node-major [n_rows][ncol]."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n_rows, ncol))
    X /= np.linalg.norm(X, axis=0, keepdims=True)
    return X


def random_directions(n_rows: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal((count, n_rows))


# ------------------------------------------------------ closed-form input fields

def smeared_coulomb(xyz: np.ndarray, R: np.ndarray, Z: np.ndarray, s: float) -> np.ndarray:
    """-sum_I Z_I erf(|r-R_I|/s)/|r-R_I|: potential of Gaussian-smeared nuclei.

    xyz: [n, 3] coordinates.  At r = 0 the limit -2 Z /(s sqrt(pi)) is used.
    """
    out = np.zeros(xyz.shape[0])
    for RI, ZI in zip(R, Z):
        r = np.linalg.norm(xyz - RI[None, :], axis=1)
        small = r < 1e-12
        val = np.empty_like(r)
        val[~small] = erf(r[~small] / s) / r[~small]
        val[small] = 2.0 / (s * math.sqrt(math.pi))
        out -= ZI * val
    return out


def gaussian_bumps(xyz, centres, amps, widths) -> np.ndarray:
    """sum_j a_j exp(-|r - c_j|^2 / b_j^2)."""
    out = np.zeros(xyz.shape[0])
    for c, a, b in zip(centres, amps, widths):
        d2 = np.sum((xyz - c[None, :]) ** 2, axis=1)
        out += a * np.exp(-d2 / (b * b))
    return out


def gaussian_density(xyz, R, Q, s) -> np.ndarray:
    """sum_I Q_I exp(-|r-R_I|^2/s^2) / (pi^{3/2} s^3): integrates to sum Q_I."""
    out = np.zeros(xyz.shape[0])
    norm = 1.0 / (math.pi ** 1.5 * s ** 3)
    for RI, QI in zip(R, Q):
        d2 = np.sum((xyz - RI[None, :]) ** 2, axis=1)
        out += QI * norm * np.exp(-d2 / (s * s))
    return out


def gaussian_density_hartree(xyz, R, Q, s) -> np.ndarray:
    """Exact Hartree potential of gaussian_density: sum_I Q_I erf(r/s)/r."""
    return -smeared_coulomb(xyz, R, Q, s)


def lda_exchange(rho: np.ndarray) -> np.ndarray:
    """Slater/LDA exchange potential -(3/pi)^{1/3} rho^{1/3}, rho clamped at 0.

    This is the reference exchange-correlation model of the synthetic workloads
    (an input recipe, not a step of the inverse method)."""
    return -((3.0 / math.pi) ** (1.0 / 3.0)) * np.cbrt(np.maximum(rho, 0.0))


MODEL_WIDTH = 1.0      # bohr: width of the Gaussian model density per nucleus


def model_fields(wl: Workload, xyz: np.ndarray):
    """Closed-form input fields of a workload at coordinates xyz [n, 3].

    rho_model: Gaussian charge Z_I of width MODEL_WIDTH on every nucleus;
    v_H: its exact Hartree potential; v_ext: the smeared nuclei;
    v_xc_ref: LDA exchange of rho_model, plus the workload's bumps, plus (for
    the 100-electron case) a -v_H/N_e tail switched on where rho_model is small,
    f = rho/(rho + 1e-2) -- the form of the paper's initial guess (Sec. 4.2.3)
    used here only to give the reference potential a -1/r far field.
    """
    rho = gaussian_density(xyz, wl.nuclei_R, wl.nuclei_Z, MODEL_WIDTH)
    v_h = gaussian_density_hartree(xyz, wl.nuclei_R, wl.nuclei_Z, MODEL_WIDTH)
    v_ext = smeared_coulomb(xyz, wl.nuclei_R, wl.nuclei_Z, wl.smear)
    v_xc = lda_exchange(rho) + gaussian_bumps(xyz, wl.bump_c, wl.bump_a, wl.bump_b)
    if wl.name == "cube32_q4_e100":
        f = rho / (rho + 1e-2)
        v_xc = v_xc + (1.0 - f) * (-v_h / wl.n_electrons)
    return dict(rho_model=rho, v_H=v_h, v_ext=v_ext, v_fixed=v_ext + v_h, v_xc_ref=v_xc)


WORKLOADS = {
    "cube8_q2_he": cube8_q2_he,
    "cube32_q4_hx": cube32_q4_hx,
    "cube24_q4_e20": cube24_q4_e20,
    "cube32_q4_e100": cube32_q4_e100,
}
