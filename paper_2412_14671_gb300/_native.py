"""ctypes declarations of the C ABI in include/muster.h and include/muster_ops.h.

Argument marshalling only: every computation runs in the CUDA library
``libmuster.so`` of this package. Loading fails loudly when the library is
missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmuster.so")

OK, EINVAL, ESTATE, EOOM, ECUDA, ETIMEOUT, ENUMERIC = 0, -1, -2, -3, -4, -5, -6
SILNCC, LNCC = 0, 1
ADAM, SGD = 0, 1
VELOCITY, PAIR_FLOW, PAIR_DISP, WARPED, IMAGE, GRADIENT, JACOBIAN, PARAMETERS = range(8)

_ERRNAMES = {EINVAL: "EINVAL", ESTATE: "ESTATE", EOOM: "EOOM", ECUDA: "ECUDA", ETIMEOUT: "ETIMEOUT", ENUMERIC: "ENUMERIC"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class MusterParams(ctypes.Structure):
    """Mirror of muster_params (include/muster.h)."""

    _fields_ = [
        ("n_levels", ctypes.c_int),
        ("steps_per_level", ctypes.c_int * 8),
        ("flow_factor", ctypes.c_int),
        ("n_squarings", ctypes.c_int),
        ("window", ctypes.c_int),
        ("similarity", ctypes.c_int),
        ("alpha_ss", ctypes.c_float),
        ("alpha_l2", ctypes.c_float),
        ("alpha_ts", ctypes.c_float),
        ("sim_eps", ctypes.c_float),
        ("optimizer", ctypes.c_int),
        ("lr", ctypes.c_float),
        ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float),
        ("adam_eps", ctypes.c_float),
        ("warmup_frac", ctypes.c_float),
        ("deterministic", ctypes.c_int),
        ("recompute_squaring", ctypes.c_int),
        ("pair_batch", ctypes.c_int),
        ("smooth_omega", ctypes.c_float),
        ("rigid", ctypes.c_int),
        ("rigid_lr", ctypes.c_float),
        ("flow_nf", ctypes.c_int),
        ("chunk_pct", ctypes.c_int),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
    ]


class MusterError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "?"), code, msg))
        self.code = code


_lib = None

P = ctypes.c_void_p
I64P = ctypes.POINTER(ctypes.c_int64)
DP = ctypes.POINTER(ctypes.c_double)
FP = ctypes.c_void_p  # float pointers are passed as raw addresses (host or device)
SZP = ctypes.POINTER(ctypes.c_size_t)

SIGNATURES = {
    # include/muster.h
    "muster_default_params": (None, [ctypes.POINTER(MusterParams)]),
    "muster_create": (ctypes.c_int, [I64P, ctypes.c_int, DP, ctypes.POINTER(MusterParams), ctypes.POINTER(P)]),
    "muster_set_stream": (ctypes.c_int, [P, P]),
    "muster_set_images": (ctypes.c_int, [P, FP, ctypes.c_int, DP]),
    "muster_set_level": (ctypes.c_int, [P, ctypes.c_int]),
    "muster_set_velocity": (ctypes.c_int, [P, FP, ctypes.c_int]),
    "muster_step": (ctypes.c_int, [P, DP]),
    "muster_run": (ctypes.c_int, [P, DP]),
    "muster_advance": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "muster_footprint": (ctypes.c_int, [I64P, ctypes.c_int, ctypes.POINTER(MusterParams), ctypes.POINTER(ctypes.c_size_t)]),
    "muster_eval": (ctypes.c_int, [P, FP, ctypes.c_int, DP, FP]),
    "muster_get_fields": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, FP, ctypes.c_int]),
    "muster_get_loss_split": (ctypes.c_int, [P, DP]),
    "muster_get_loss_history": (ctypes.c_int, [P, DP, SZP]),
    "muster_level_dims": (ctypes.c_int, [P, ctypes.c_int, I64P, I64P]),
    "muster_get_level": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "muster_get_state": (ctypes.c_int, [P, P, SZP]),
    "muster_set_state": (ctypes.c_int, [P, P, ctypes.c_size_t]),
    "muster_profile_begin": (ctypes.c_int, [P]),
    "muster_profile_end": (ctypes.c_int, [P]),
    "muster_kernel_stat": (
        ctypes.c_int,
        [P, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), I64P, DP, DP],
    ),
    "muster_kernel_launches": (ctypes.c_int, [P, ctypes.c_int, I64P]),
    "muster_last_error": (ctypes.c_char_p, [P]),
    "muster_destroy": (None, [P]),
    "muster_get_rigid": (ctypes.c_int, [P, DP, DP]),
    "muster_set_rigid": (ctypes.c_int, [P, DP]),
    # include/muster_ops.h
    "muster_op_downsample": (ctypes.c_int, [FP, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, FP, P]),
    "muster_op_exp": (
        ctypes.c_int,
        [FP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_float, FP, P],
    ),
    "muster_op_similarity": (
        ctypes.c_int,
        [FP, FP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_float, DP, FP, P],
    ),
    "muster_op_similarity_noalloc": (
        ctypes.c_int,
        [FP, FP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_float, DP, FP, P],
    ),
    "muster_op_jacobian_det": (ctypes.c_int, [FP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, FP, P]),
    "muster_op_deformation_metrics": (
        ctypes.c_int,
        [FP, FP, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, DP, P],
    ),
    "muster_ops_last_error": (ctypes.c_char_p, []),
}


def lib() -> ctypes.CDLL:
    """Load libmuster.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libmuster.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'` "
                "(the CUDA library is required; there is no CPU fallback)"
            )
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int, ctx=None) -> None:
    if rc != OK:
        L = lib()
        if ctx is None:
            msg = L.muster_last_error(None)
        else:
            msg = L.muster_last_error(ctx)
        raise MusterError(rc, (msg or b"").decode(errors="replace"))


def check_op(rc: int) -> None:
    if rc != OK:
        raise MusterError(rc, (lib().muster_ops_last_error() or b"").decode(errors="replace"))
