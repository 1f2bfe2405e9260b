"""ctypes loader of libshg.so and the raw C signatures of include/shg.h.

The library is built in-tree by ``paper_2304_04612_gb300.build``; loading
fails loudly when it is missing.  There is no other implementation to fall
back to.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libshg.so")

c_i64 = ctypes.c_int64
c_int = ctypes.c_int
c_u64 = ctypes.c_uint64
c_vp = ctypes.c_void_p
c_sz = ctypes.c_size_t

# name -> (restype, argtypes), mirroring include/shg.h
SIGNATURES = {
    "shg_status_string": (ctypes.c_char_p, [c_int]),
    "shg_version": (c_int, []),
    "shg_flags_status": (c_int, [ctypes.c_int32]),
    "shg_gaussian_f16": (c_int, [c_u64, c_u64, c_i64, c_i64, c_vp, c_i64, c_vp]),
    "shg_sparse_sign_f16": (c_int, [c_u64, c_u64, c_i64, c_i64, ctypes.c_double, c_vp, c_i64, c_vp]),
    "shgemm_project": (c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_int, c_vp, c_i64, c_vp, c_i64,
                               c_int, c_vp, c_vp]),
    "shg_gemm_split3": (c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_int, c_vp, c_i64, c_vp, c_i64,
                                c_int, c_vp, c_vp]),
    "shg_sgemm": (c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_int, c_vp, c_i64, c_int, c_vp, c_i64,
                          c_int, c_vp]),
    "shg_cholqr2_workspace_size": (c_int, [c_i64, c_i64, ctypes.POINTER(c_sz)]),
    "shg_gram": (c_int, [c_i64, c_i64, c_vp, c_i64, c_vp, c_vp]),
    "shg_cholqr2": (c_int, [c_i64, c_i64, c_vp, c_i64, c_vp, c_sz, c_vp, c_vp]),
    "shg_cholqr2_static": (c_int, [c_i64, c_i64, c_vp, c_i64, c_vp, c_vp]),
    "shg_alpha_y_f16": (ctypes.c_double, []),
    "shg_diag_wait_timeout": (c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_u64, c_vp, c_vp]),
    "shg_rsvd_batched_workspace_size": (c_int, [c_int, c_vp, c_vp, c_vp, c_i64, c_int, ctypes.POINTER(c_sz)]),
    "shg_autotune_project": (c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_int, c_vp, c_i64, c_vp, c_i64, c_int,
                                     c_int, c_vp, c_vp, c_vp]),
    "shg_autotune_lookup": (c_int, [c_i64, c_i64, c_i64, c_int, c_int, c_vp]),
    "shg_autotune_clear": (c_int, []),
    "shg_autotune_export": (c_int, [c_vp, ctypes.c_int32, c_vp]),
    "shg_autotune_import": (c_int, [c_vp, ctypes.c_int32, c_vp]),
    "shg_rsvd_batched_autotune": (c_int, [c_int, c_vp, c_vp, c_vp, c_i64, c_vp, c_vp, c_u64, c_vp, c_sz, c_int,
                                          c_vp, c_vp, c_vp]),
    "shg_rsvd_batched": (c_int, [c_int, c_vp, c_vp, c_vp, c_i64, c_int, c_vp, c_vp, c_vp, c_vp, c_u64, c_vp, c_vp,
                                 c_vp, c_vp, c_sz, c_int, c_int, c_vp, c_vp]),
    "shg_round_f16": (c_int, [c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp]),
    "shg_residual_estimate_workspace_size": (c_int, [c_i64, c_i64, c_i64, c_i64, ctypes.POINTER(c_sz)]),
    "shg_residual_estimate": (c_int, [c_i64, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_u64, c_u64,
                                      ctypes.c_double, c_vp, c_vp, c_sz, c_vp, c_vp]),
    "shg_sketch_loss_grad_workspace_size": (c_int, [c_i64, c_i64, c_i64, ctypes.POINTER(c_sz)]),
    "shg_sketch_loss_grad": (c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_int, c_vp, c_i64, c_vp,
                                     c_vp, c_sz, c_vp, c_vp]),
    "shg_rsvd_workspace_size": (c_int, [c_i64, c_i64, c_i64, c_i64, c_int, ctypes.POINTER(c_sz)]),
    "shg_rsvd": (c_int, [c_i64, c_i64, c_i64, c_i64, c_int, c_vp, c_i64, c_vp, c_i64, c_u64, c_vp, c_vp, c_vp,
                         c_vp, c_vp, c_sz, c_int, c_vp, c_vp, c_vp]),
    "shg_mode_project": (c_int, [c_int, ctypes.POINTER(c_i64), c_int, c_i64, c_vp, c_vp, c_i64, c_vp, c_i64, c_int,
                                 c_vp, c_vp]),
    "shg_rp_hosvd_workspace_size": (c_int, [c_int, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), c_i64,
                                            ctypes.POINTER(c_sz)]),
    "shg_rp_hosvd": (c_int, [c_int, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), c_i64, c_vp,
                             c_vp, c_vp, c_u64, c_vp, ctypes.POINTER(c_vp), c_vp, c_sz,
                             c_int, c_vp, c_vp]),
}

PHASES = ("omega", "project", "orth", "power", "B", "svd", "lift", "estimate")


class Report(ctypes.Structure):
    """struct shg_report of include/shg.h."""
    _fields_ = [("flags", ctypes.c_int32), ("status", ctypes.c_int32), ("min_pivot", ctypes.c_double),
                ("est_residual", ctypes.c_double), ("phase_ms", ctypes.c_float * len(PHASES))]

    def as_dict(self) -> dict:
        return {"flags": self.flags, "status": self.status, "min_pivot": self.min_pivot,
                "est_residual": self.est_residual,
                "phase_ms": {name: float(self.phase_ms[i]) for i, name in enumerate(PHASES)}}

_lib = None


def load() -> ctypes.CDLL:
    """Load libshg.so (once) and attach the argument types."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2304_04612_gb300.build` "
                "(or __graft_entry__.build()); there is no fallback implementation")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib
