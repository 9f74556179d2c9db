"""ctypes binding of libinvdft.so (include/invdft.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards
its arguments; device arrays are torch CUDA tensors (their data_ptr() is
passed), host arrays are numpy arrays or ctypes structures.  No step of the
method runs in Python.  Importing this module fails loudly when the library is
missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libinvdft.so")

INVDFT_OK, INVDFT_EINVAL, INVDFT_ENOMEM, INVDFT_ECUDA, INVDFT_ENOCONV, INVDFT_ETIMEOUT, \
    INVDFT_ENOTSPD = range(7)
INVDFT_FP64, INVDFT_MIXED, INVDFT_MIXED_TF32 = 0, 1, 2
INVDFT_HX_SEG_BALANCED = 0x7fffffff   # seglen of the balanced H~X schedule
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ETIMEOUT",
                6: "ENOTSPD"}


class MeshDesc(C.Structure):
    """invdft_mesh_desc: per-axis box, cells and optional cell breaks."""
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("ncell", C.c_int * 3),
                ("order", C.c_int), ("breaks", C.POINTER(C.c_double) * 3)]

    @classmethod
    def make(cls, lo, hi, ncell, order, breaks=None):
        """lo, hi, ncell: scalars (a cube) or three values (x, y, z); breaks:
        None or three sequences (None per axis for equal cells)."""
        three = lambda x, t: [t(v) for v in (x if hasattr(x, "__len__") else (x, x, x))]
        d = cls()
        for a, (l, h, n) in enumerate(zip(three(lo, float), three(hi, float), three(ncell, int))):
            d.lo[a], d.hi[a], d.ncell[a] = l, h, n
        d.order = int(order)
        d._keep = []
        for a in range(3):
            b = None if breaks is None else breaks[a]
            if b is None:
                d.breaks[a] = C.POINTER(C.c_double)()
            else:
                arr = (C.c_double * len(b))(*[float(x) for x in b])
                d._keep.append(arr)
                d.breaks[a] = C.cast(arr, C.POINTER(C.c_double))
        return d


class Opts(C.Structure):
    _fields_ = [("nstates", C.c_int), ("n_electrons", C.c_double), ("kT", C.c_double),
                ("cheb_degree", C.c_int), ("c_eig", C.c_double), ("c_ad", C.c_double),
                ("tau_bc", C.c_double), ("eig_tol", C.c_double), ("adj_tol", C.c_double),
                ("max_cheb_passes", C.c_int), ("max_minres_iters", C.c_int),
                ("lbfgs_history", C.c_int), ("prec", C.c_int), ("seed", C.c_ulonglong),
                ("deg_tol", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("loss", C.c_double), ("err_l2", C.c_double), ("n_elec", C.c_double),
                ("mu", C.c_double), ("eig_resid_max", C.c_double),
                ("adj_resid_max", C.c_double), ("eta", C.c_double),
                ("cheb_passes", C.c_int), ("hx_calls", C.c_int), ("minres_iters_max", C.c_int),
                ("ls_trials", C.c_int), ("refinements", C.c_int),
                ("t_forward_ms", C.c_double), ("t_adjoint_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class InvdftError(RuntimeError):
    def __init__(self, name, status, text):
        super().__init__(f"{name}: {STATUS_NAMES.get(status, status)}: {text}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2510_10529_b300.build` "
            "(nvcc, sm_103a); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    H = C.c_void_p
    P = C.c_void_p
    sig = {
        "invdft_create_mesh": [C.POINTER(MeshDesc), C.POINTER(Opts), C.POINTER(H),
                               C.POINTER(C.c_longlong)],
        "invdft_destroy": [H],
        "invdft_workspace_size": [H, C.POINTER(C.c_size_t)],
        "invdft_bind_workspace": [H, P, C.c_size_t, P],
        "invdft_node_coords": [H, P],
        "invdft_mass_diag": [H, P, P],
        "invdft_set_potential": [H, P, P, P],
        "invdft_apply_h": [H, P, P, C.c_int, C.c_int, P],
        "invdft_chebyshev_filter": [H, P, P, C.c_int, C.c_int, C.c_double, C.c_double,
                                    C.c_double, C.c_int, P],
        "invdft_forward_solve": [H, P, P, P, P, C.POINTER(Stats), P],
        "invdft_adjoint_solve": [H, P, P, C.POINTER(Stats), P],
        "invdft_density_vjp": [H, P, P, C.POINTER(Stats), P],
        "invdft_loss_grad": [H, P, P, C.POINTER(C.c_double), P, C.POINTER(Stats), P],
        "invdft_step": [H, P, P, P, C.POINTER(Stats), P],
        "invdft_reset": [H],
        "invdft_initial_guess": [H, P, P, C.c_double, C.c_double, C.c_int, P, P],
        "invdft_q1_to_nodes": [H, C.c_int, P, P, P],
        "invdft_cell_potential_bytes": [H, C.c_int, C.POINTER(C.c_size_t)],
        "invdft_cell_potentials": [H, P, P, C.c_int, P],
        "invdft_apply_h_dense": [H, P, P, P, C.c_int, C.c_int, P],
        "invdft_grad_to_q1": [H, C.c_int, P, P, P],
        "invdft_profile_hx": [H, C.c_int, P],
        "invdft_profile_deflation": [H, P],
        "invdft_tune_hx": [H, C.c_int, C.c_int, P],
        "invdft_hx_config": [H, C.c_int, C.c_int, P],
        "invdft_kernel_launches": [C.POINTER(C.c_ulonglong)],
        "invdft_peak_probe": [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), P],
        "invdft_graph_stats": [P],
        "invdft_loss_reduce_noalloc": [P, P, P, P, C.c_longlong, P, P, P],
        "invdft_batch_create": [P, C.c_int, C.POINTER(H)],
        "invdft_batch_destroy": [H],
        "invdft_batch_step": [H, P, P, P, C.POINTER(Stats), P, P],
        "invdft_batch_info": [H, P, P],
        "invdft_batch_set_wait_limit": [H, C.c_int],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.invdft_last_error.argtypes = [H]
    lib.invdft_last_error.restype = C.c_char_p
    return lib


lib = _load()


def check(name, status, handle=None):
    if status not in (INVDFT_OK,):
        text = lib.invdft_last_error(handle).decode(errors="replace")
        raise InvdftError(name, status, text)
    return status
