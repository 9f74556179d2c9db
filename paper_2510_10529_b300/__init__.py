"""B300 inverse-DFT hot path (arXiv 2510.10529) -- Python binding of libinvdft.

Thin layer over the C ABI of include/invdft.h.  Functions named `invdft_*`
forward to the entry point of the same name; torch CUDA tensors supply device
memory and the current CUDA stream.  `Problem` owns one handle and its
workspace tensor; `KohnShamDensity` is a torch.autograd.Function whose forward
is the Kohn-Sham solve and whose backward is the adjoint solve plus the
gradient reduction (Eq. 7-11), both run by the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import (INVDFT_ENOCONV, INVDFT_FP64, INVDFT_HX_SEG_BALANCED, INVDFT_MIXED,
                   INVDFT_MIXED_TF32, INVDFT_OK, InvdftError, MeshDesc, Opts, Stats, check, lib)

__all__ = ["Problem", "Batch", "KohnShamDensity", "MeshDesc", "Opts", "Stats", "InvdftError",
           "INVDFT_FP64", "INVDFT_HX_SEG_BALANCED", "INVDFT_MIXED", "INVDFT_MIXED_TF32", "library_path"]


def library_path() -> str:
    from ._lib import LIB_PATH
    return LIB_PATH


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arrays must be contiguous CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ok(name, st, h, allow_noconv=True):
    if st == INVDFT_OK or (allow_noconv and st == INVDFT_ENOCONV):
        return st
    return check(name, st, h)


# ----------------------------------------------------------- same-name wrappers

def invdft_create_mesh(mesh: MeshDesc, opts: Opts):
    h = C.c_void_p()
    n = C.c_longlong()
    _ok("invdft_create_mesh", lib.invdft_create_mesh(C.byref(mesh), C.byref(opts), C.byref(h),
                                                     C.byref(n)), None, False)
    return h, n.value


def invdft_destroy(h):
    return lib.invdft_destroy(h)


def invdft_workspace_size(h) -> int:
    n = C.c_size_t()
    _ok("invdft_workspace_size", lib.invdft_workspace_size(h, C.byref(n)), h, False)
    return n.value


def invdft_bind_workspace(h, ws: torch.Tensor):
    return _ok("invdft_bind_workspace",
               lib.invdft_bind_workspace(h, _ptr(ws), ws.numel() * ws.element_size(), _stream()),
               h, False)


def invdft_node_coords(h, L: int) -> np.ndarray:
    xyz = np.empty((L, 3), dtype=np.float64)
    _ok("invdft_node_coords", lib.invdft_node_coords(h, xyz.ctypes.data_as(C.c_void_p)), h, False)
    return xyz


def invdft_mass_diag(h, m: torch.Tensor):
    return _ok("invdft_mass_diag", lib.invdft_mass_diag(h, _ptr(m), _stream()), h, False)


def invdft_set_potential(h, v_fixed: torch.Tensor, v_xc: torch.Tensor | None):
    return _ok("invdft_set_potential",
               lib.invdft_set_potential(h, _ptr(v_fixed), _ptr(v_xc), _stream()), h, False)


def invdft_apply_h(h, X: torch.Tensor, Y: torch.Tensor, tensor_cores: bool = True):
    """Y = H~ X.  float64 blocks run in FP64; float32 blocks on the TF32 tensor
    cores (Q4 meshes) or, with tensor_cores=False, in FP32 on the CUDA cores."""
    prec = (INVDFT_FP64 if X.dtype == torch.float64
            else (INVDFT_MIXED_TF32 if tensor_cores else INVDFT_MIXED))
    if X.dtype != Y.dtype or X.dtype not in (torch.float64, torch.float32):
        raise ValueError("apply_h: X and Y must both be float64 or both float32")
    ncol = X.shape[1] if X.dim() == 2 else 1
    return _ok("invdft_apply_h", lib.invdft_apply_h(h, _ptr(X), _ptr(Y), ncol, prec, _stream()),
               h, False)


def invdft_chebyshev_filter(h, X, Y, degree, a, b, a0):
    prec = INVDFT_FP64 if X.dtype == torch.float64 else INVDFT_MIXED
    return _ok("invdft_chebyshev_filter",
               lib.invdft_chebyshev_filter(h, _ptr(X), _ptr(Y), X.shape[1], degree, a, b, a0,
                                           prec, _stream()), h, False)


def invdft_forward_solve(h, psi=None, eps=None, occ=None, rho=None):
    st = Stats()
    code = _ok("invdft_forward_solve", lib.invdft_forward_solve(
        h, _ptr(psi), _ptr(eps), _ptr(occ), _ptr(rho), C.byref(st), _stream()), h)
    return code, st


def invdft_adjoint_solve(h, dL_drho, p):
    st = Stats()
    code = _ok("invdft_adjoint_solve",
               lib.invdft_adjoint_solve(h, _ptr(dL_drho), _ptr(p), C.byref(st), _stream()), h)
    return code, st


def invdft_density_vjp(h, dL_drho, grad_v):
    st = Stats()
    code = _ok("invdft_density_vjp",
               lib.invdft_density_vjp(h, _ptr(dL_drho), _ptr(grad_v), C.byref(st), _stream()), h)
    return code, st


def invdft_loss_grad(h, rho_data, w, grad):
    st = Stats()
    loss = C.c_double()
    code = _ok("invdft_loss_grad", lib.invdft_loss_grad(
        h, _ptr(rho_data), _ptr(w), C.byref(loss), _ptr(grad), C.byref(st), _stream()), h)
    return code, loss.value, st


def invdft_step(h, rho_data, w, v_xc):
    st = Stats()
    code = _ok("invdft_step", lib.invdft_step(h, _ptr(rho_data), _ptr(w), _ptr(v_xc),
                                              C.byref(st), _stream()), h)
    return code, st


def invdft_reset(h):
    return lib.invdft_reset(h)


def invdft_profile_hx(h, enable: bool):
    """H~X launch totals by kind: fp64, fp32_filter (FP32 with the filter's
    W / E terms), fp32 (other FP32 launches: the MINRES operator), tf32."""
    out = np.zeros(16)
    _ok("invdft_profile_hx", lib.invdft_profile_hx(h, int(enable), out.ctypes.data_as(C.c_void_p)),
        h, False)
    keys = ("ms", "bytes", "flops", "launches")
    return {"fp64": dict(zip(keys, out[:4])), "fp32_filter": dict(zip(keys, out[4:8])),
            "fp32": dict(zip(keys, out[8:12])), "tf32": dict(zip(keys, out[12:]))}


def invdft_profile_deflation(h):
    """Totals of the tensor-core deflation launches (Gram, update) timed while
    invdft_profile_hx is enabled."""
    out = np.zeros(8)
    _ok("invdft_profile_deflation",
        lib.invdft_profile_deflation(h, out.ctypes.data_as(C.c_void_p)), h, False)
    keys = ("ms", "bytes", "flops", "launches")
    return {"gram": dict(zip(keys, out[:4])), "update": dict(zip(keys, out[4:]))}


def invdft_tune_hx(h, variant: int = -1, seglen: int = 0):
    """Fix the tile variant (-1: autotuned) and z-segment length (0: autotuned)
    of the sweep H~X; returns the number of FP32 and FP64 variants."""
    n = (C.c_int * 2)()
    _ok("invdft_tune_hx", lib.invdft_tune_hx(h, int(variant), int(seglen), n), h, False)
    return int(n[0]), int(n[1])


def invdft_hx_config(h, ncol: int, fp64: bool):
    """Autotuned (variant, seglen) per epilogue {plain, E, W, W+E} (-1: not tuned)."""
    out = (C.c_int * 8)()
    _ok("invdft_hx_config", lib.invdft_hx_config(h, int(ncol), int(bool(fp64)), out), h, False)
    names = ("plain", "E", "W", "WE")
    return {names[k]: (int(out[2 * k]), int(out[2 * k + 1])) for k in range(4)}


def invdft_graph_stats() -> dict:
    out = (C.c_longlong * 3)()
    lib.invdft_graph_stats(out)
    return {"captured": int(out[0]), "replays": int(out[1]), "refused": int(out[2])}


def invdft_peak_probe(kind: str) -> float:
    """Measured arithmetic rate (TFLOP/s): "fp64", "fp32", "fp32x2" or "tf32"."""
    k = {"fp64": 0, "fp32": 1, "fp32x2": 2, "tf32": 3}[kind]
    t, ms = C.c_double(), C.c_double()
    _ok("invdft_peak_probe", lib.invdft_peak_probe(k, C.byref(t), C.byref(ms), _stream()), None,
        False)
    return t.value


def invdft_kernel_launches() -> int:
    n = C.c_ulonglong()
    lib.invdft_kernel_launches(C.byref(n))
    return n.value


# ----------------------------------------------------------- owning wrapper

class Problem:
    """One inverse-DFT problem: a handle plus its torch-allocated workspace.

    prec: "fp64" (every step in FP64), "mixed" (FP32 storage and FP32 cell
    products on the CUDA cores in the Chebyshev filter and the inner MINRES,
    FP64 elsewhere) or "tf32" (as "mixed", with the filter's Q4 cell products
    on the TF32 tensor cores)."""

    def __init__(self, lo, hi, ncell, order, nstates, n_electrons=0.0, kT=0.0,
                 prec="fp64", cheb_degree=0, eig_tol=0.0, adj_tol=0.0, tau_bc=0.0,
                 max_cheb_passes=0, max_minres_iters=0, lbfgs_history=0, seed=1,
                 deg_tol=0.0, device=None, breaks=None):
        """lo, hi, ncell: scalars for a cube of equal cells, or three values
        (x, y, z); breaks: optional three sequences of cell breaks (None per
        axis for equal cells), for graded meshes."""
        self.device = torch.device(device or "cuda")
        mesh = MeshDesc.make(lo, hi, ncell, order, breaks)
        opts = Opts(nstates=int(nstates), n_electrons=float(n_electrons), kT=float(kT),
                    cheb_degree=int(cheb_degree), c_eig=0.0, c_ad=0.0, tau_bc=float(tau_bc),
                    eig_tol=float(eig_tol), adj_tol=float(adj_tol),
                    max_cheb_passes=int(max_cheb_passes), max_minres_iters=int(max_minres_iters),
                    lbfgs_history=int(lbfgs_history),
                    prec={"mixed": INVDFT_MIXED, "tf32": INVDFT_MIXED_TF32}.get(prec, INVDFT_FP64),
                    seed=int(seed),
                    deg_tol=float(deg_tol))
        self.h, self.L = invdft_create_mesh(mesh, opts)
        self.nstates = int(nstates)
        nbytes = invdft_workspace_size(self.h)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            invdft_bind_workspace(self.h, self.workspace)
        self.potential_version = 0
        self.solved_version = -1

    def close(self):
        if self.h:
            invdft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zeros(self, *shape, dtype=torch.float64):
        return torch.zeros(*shape, dtype=dtype, device=self.device)

    def coords(self) -> np.ndarray:
        return invdft_node_coords(self.h, self.L)

    def mass(self) -> torch.Tensor:
        m = self.zeros(self.L)
        invdft_mass_diag(self.h, m)
        return m

    def set_potential(self, v_fixed, v_xc=None):
        invdft_set_potential(self.h, v_fixed, v_xc)
        self.v_fixed = v_fixed
        self.potential_version += 1

    def apply_h(self, X, tensor_cores: bool = True):
        Y = torch.empty_like(X)
        invdft_apply_h(self.h, X, Y, tensor_cores)
        return Y

    def chebyshev_filter(self, X, degree, a, b, a0):
        Y = torch.empty_like(X)
        invdft_chebyshev_filter(self.h, X, Y, degree, a, b, a0)
        return Y

    def forward_solve(self):
        psi = self.zeros(self.L, self.nstates)
        eps = self.zeros(self.nstates)
        occ = self.zeros(self.nstates)
        rho = self.zeros(self.L)
        code, st = invdft_forward_solve(self.h, psi, eps, occ, rho)
        self.solved_version = self.potential_version
        return dict(psi=psi, eps=eps, occ=occ, rho=rho, stats=st.as_dict(), code=code)

    def adjoint_solve(self, dL_drho):
        p = self.zeros(self.L, self.nstates)
        code, st = invdft_adjoint_solve(self.h, dL_drho, p)
        return p, st.as_dict()

    def density_vjp(self, dL_drho):
        g = self.zeros(self.L)
        code, st = invdft_density_vjp(self.h, dL_drho, g)
        return g, st.as_dict()

    def loss_grad(self, rho_data, w):
        g = self.zeros(self.L)
        code, loss, st = invdft_loss_grad(self.h, rho_data, w, g)
        self.solved_version = self.potential_version
        return loss, g, st.as_dict()

    def step(self, rho_data, w, v_xc):
        code, st = invdft_step(self.h, rho_data, w, v_xc)
        self.potential_version += 1
        self.solved_version = self.potential_version
        return st.as_dict()

    def initial_guess(self, rho_data, v_H, tau: float = 1e-2, alpha: float = 1.0,
                      exchange: str = "lb94"):
        """v_xc of Eq. 25 (Sec. 4.2.3) from the target density and its Hartree
        potential (device [L] tensors); exchange "lb94" or "slater"."""
        v = self.zeros(self.L)
        _ok("invdft_initial_guess",
            lib.invdft_initial_guess(self.h, _ptr(rho_data), _ptr(v_H), float(tau), float(alpha),
                                     {"slater": 0, "lb94": 1}[exchange], _ptr(v), _stream()),
            self.h, False)
        return v

    def cell_potentials(self, v_full, prec: str = "fp64"):
        """Dense per-cell potential matrices (Gauss quadrature of Eq. 17) from v
        on the full node grid (boundary included); returns the device buffer."""
        pr = INVDFT_FP64 if prec == "fp64" else INVDFT_MIXED
        n = C.c_size_t()
        _ok("invdft_cell_potential_bytes",
            lib.invdft_cell_potential_bytes(self.h, pr, C.byref(n)), self.h, False)
        Ve = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        _ok("invdft_cell_potentials",
            lib.invdft_cell_potentials(self.h, _ptr(v_full), _ptr(Ve), pr, _stream()),
            self.h, False)
        return Ve

    def apply_h_dense(self, Ve, X):
        """Y = D (K + V) D X with the dense cell potentials (X double or float)."""
        Y = torch.empty_like(X)
        pr = INVDFT_FP64 if X.dtype == torch.float64 else INVDFT_MIXED
        _ok("invdft_apply_h_dense",
            lib.invdft_apply_h_dense(self.h, _ptr(Ve), _ptr(X), _ptr(Y), X.shape[1], pr,
                                     _stream()), self.h, False)
        return Y

    def q1_to_nodes(self, nv: int, v_q1):
        """v_xc at the unknown nodes from a Q1 field of nv^3 cells (trilinear)."""
        v = self.zeros(self.L)
        _ok("invdft_q1_to_nodes", lib.invdft_q1_to_nodes(self.h, int(nv), _ptr(v_q1), _ptr(v),
                                                         _stream()), self.h, False)
        return v

    def grad_to_q1(self, nv: int, g_nodes):
        """A nodal gradient pulled back to the (nv+1)^3 Q1 coefficients (T^T g)."""
        g = self.zeros((nv + 1) ** 3)
        _ok("invdft_grad_to_q1", lib.invdft_grad_to_q1(self.h, int(nv), _ptr(g_nodes), _ptr(g),
                                                       _stream()), self.h, False)
        return g

    def reset(self):
        invdft_reset(self.h)

    def profile_hx(self, enable: bool):
        return invdft_profile_hx(self.h, enable)

    def profile_deflation(self):
        return invdft_profile_deflation(self.h)

    def tune_hx(self, variant: int = -1, seglen: int = 0):
        return invdft_tune_hx(self.h, variant, seglen)

    def hx_config(self, ncol: int, fp64: bool = False):
        return invdft_hx_config(self.h, ncol, fp64)


def invdft_batch_create(handles) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    out = C.c_void_p()
    _ok("invdft_batch_create", lib.invdft_batch_create(arr, len(handles), C.byref(out)), None,
        False)
    return out.value


def invdft_batch_step(batch, handles, rho_data, w, v_xc):
    n = len(handles)
    ptrs = [(C.c_void_p * n)(*[_ptr(t) for t in ts]) for ts in (rho_data, w, v_xc)]
    stats = (Stats * n)()
    status = (C.c_int * n)()
    code = lib.invdft_batch_step(batch, ptrs[0], ptrs[1], ptrs[2], stats, status, _stream())
    if code not in (INVDFT_OK, INVDFT_ENOCONV):
        text = "; ".join(f"problem {b}: status {status[b]}: "
                         + lib.invdft_last_error(handles[b]).decode(errors="replace")
                         for b in range(n) if status[b] not in (INVDFT_OK, INVDFT_ENOCONV))
        raise InvdftError("invdft_batch_step", code, text)
    return [stats[b].as_dict() for b in range(n)], [int(status[b]) for b in range(n)]


class Batch:
    """Independent problems stepped together (invdft_batch_*): each problem's
    step runs on its own stream and the Chebyshev filter passes of all of
    them run as single cooperative persistent launches."""

    def __init__(self, problems):
        self.problems = list(problems)
        self.h = invdft_batch_create([p.h for p in self.problems])

    def set_wait_limit(self, polls: int):
        """Polls before a phase wait of the persistent kernel gives up (0: at the
        first wait; < 0: the default)."""
        _ok("invdft_batch_set_wait_limit", lib.invdft_batch_set_wait_limit(self.h, int(polls)),
            None, False)

    def step(self, rho_data, w, v_xc):
        stats, status = invdft_batch_step(self.h, [p.h for p in self.problems], rho_data, w,
                                          v_xc)
        for p in self.problems:
            p.potential_version += 1
            p.solved_version = p.potential_version
        return stats, status

    def info(self):
        n = len(self.problems)
        cols = (C.c_int * n)()
        info = (C.c_double * 4)()
        _ok("invdft_batch_info", lib.invdft_batch_info(self.h, cols, info), None, False)
        return {"chunk_cols": list(cols), "launches": int(info[0]),
                "graph_launches": int(info[1]), "ctas": int(info[2]), "tuned": bool(info[3])}

    def close(self):
        if self.h:
            lib.invdft_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KohnShamDensity(torch.autograd.Function):
    """rho(v_xc): forward = Kohn-Sham solve (Sec. 3.2.2), backward = adjoint
    solve + gradient reduction for the incoming dL/drho (Eq. 7-11).

    Orbitals are not stored by autograd: the handle keeps those of its last
    solve, and backward re-solves at the saved v_xc when another solve has
    happened in between.
    """

    @staticmethod
    def forward(ctx, v_xc, problem: Problem, v_fixed):
        problem.set_potential(v_fixed, v_xc.detach().contiguous())
        out = problem.forward_solve()
        ctx.problem = problem
        ctx.version = problem.potential_version
        ctx.save_for_backward(v_xc.detach(), v_fixed)
        return out["rho"]

    @staticmethod
    def backward(ctx, grad_rho):
        problem = ctx.problem
        v_xc, v_fixed = ctx.saved_tensors
        if problem.solved_version != ctx.version:
            problem.set_potential(v_fixed, v_xc.contiguous())
            problem.forward_solve()
            ctx.version = problem.potential_version
        g, _ = problem.density_vjp(grad_rho.contiguous().to(torch.float64))
        return g, None, None
