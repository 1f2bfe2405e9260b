"""GB300-native mixed-precision random projection (SHGEMM) and the randomized
factorizations built on it (Ootomo & Yokota, arXiv 2304.04612).

This module is a thin binding over the C ABI of ``libshg.so``
(include/shg.h): it checks tensors, passes device pointers, leading
dimensions and the current CUDA stream, and turns status codes into
exceptions.  Every computation runs in the library's CUDA kernels; PyTorch
only provides device memory and streams.

Functions (same names as the C entry points)
--------------------------------------------
shg_gaussian_f16   FP16 Gaussian test matrix (Philox4x32-10 + Box-Muller, RN)
shg_sparse_sign_f16  sparse {-1, 0, +1} test matrix (Sec. 3.4), same Philox stream
shgemm_project     Y = op(A) Omega by SHGEMM (or the BF16 / FP32 SIMT variants)
shg_gemm_split3    FP32-accurate op(A) B of two FP32 matrices (TCEC split)
shg_sgemm          plain FP32 SIMT GEMM (the single-precision baseline)
shg_gram           G = X^T X in FP64 (compensated FP32 sums), the CholeskyQR Gram step
shg_cholqr2        CholeskyQR2 orthonormalisation (in place)
shg_cholqr2_static the same on the library's static scratch (allocates nothing)
shg_rsvd           randomized SVD (Algorithm 1, power scheme of Sec. 2.1)
shg_mode_project   mode-i projection W = X_(i) Omega of a 3-way tensor (Algorithm 2)
shg_rp_hosvd       random-projection HOSVD of a 3-way tensor (Algorithm 2)
shg_rsvd_batched   many uneven randomized SVDs at once (concurrent branches, CUDA graph)
shg_autotune_project, shg_autotune_lookup, shg_autotune_clear, shg_rsvd_batched_autotune
                   launch configuration of the tensor-core projection per shape class
shg_autotune_export, shg_autotune_import, save_autotune, load_autotune
                   the tuner's cache as records / as JSON keyed by GPU name and SM count
rsvd_workspace_size, rp_hosvd_workspace_size, rsvd_batched_workspace_size
                   workspace bytes of the factorizations (caller-allocated)
shg_alpha_y_f16    variance of an FP16-rounded N(0,1) value (alpha_Y, Sec. 3.2)
shg_round_f16      RN_fp16 of an FP32 matrix
shg_residual_estimate   a-posteriori range-finder residual with FP16 probes (Thms. 1, 3)
shg_sketch_loss_grad    loss and gradient of a learned sketch
sketch.SketchFn    torch.autograd.Function over the two above; sketch.choose_sketch
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _lib

SHG_DETERMINISTIC = 0x100  # OR'ed into a projection's variant: bitwise reproducible Y

VARIANTS = {"f16": 0, "bf16x3": 1, "bf16x2": 2, "fp32": 3, "tf32": 4, "auto": 5}
FLAG_RANGE, FLAG_NOT_SPD, FLAG_TIMEOUT = 1, 2, 4


class ShgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.load().shg_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def _check(rc: int, where: str):
    if rc != 0:
        raise ShgError(rc, where)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _mat(t: torch.Tensor, name: str, dtypes):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise TypeError(f"{name} must have dtype in {dtypes}, got {t.dtype}")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be a 2-D row-major tensor (unit column stride)")
    return t.stride(0) if t.shape[0] > 1 else max(t.shape[1], t.stride(0))


def _variant(v):
    if isinstance(v, str):
        return VARIANTS[v]
    return int(v)


def new_flags(device=None) -> torch.Tensor:
    """A zeroed device word for the SHG_FLAG_* bits."""
    return torch.zeros(1, dtype=torch.int32, device=device or "cuda")


def check_flags(flags: torch.Tensor, where: str = "shg"):
    """Synchronise on the flags word and raise ShgError when a bit is set."""
    f = int(flags.item())
    _check(_lib.load().shg_flags_status(f), where)


def shg_gaussian_f16(seed: int, offset: int, rows: int, cols: int, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(rows, cols, dtype=torch.float16, device="cuda")
    ld = _mat(out, "out", (torch.float16,))
    _check(_lib.load().shg_gaussian_f16(seed, offset, rows, cols, _ptr(out), ld, _stream(stream)),
           "shg_gaussian_f16")
    return out


def shg_sparse_sign_f16(seed: int, offset: int, rows: int, cols: int, s: float = 3.0,
                        out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Sparse sign test matrix of {-1, 0, +1} in FP16 (Sec. 3.4), P(nonzero) ~ 1/s."""
    if out is None:
        out = torch.empty(rows, cols, dtype=torch.float16, device="cuda")
    ld = _mat(out, "out", (torch.float16,))
    _check(_lib.load().shg_sparse_sign_f16(seed, offset, rows, cols, float(s), _ptr(out), ld, _stream(stream)),
           "shg_sparse_sign_f16")
    return out


def shgemm_project(A: torch.Tensor, omega: torch.Tensor, variant="f16", trans_a: bool = False,
                   out: torch.Tensor | None = None, flags: torch.Tensor | None = None,
                   check: bool = True, stream=None, deterministic: bool = False) -> torch.Tensor:
    """Y = A @ omega (trans_a: A.T @ omega).  omega: float16 (bfloat16 for the
    BF16 variants).  With check=True the call synchronises and raises on a
    device flag (e.g. SHG_ERR_RANGE).  deterministic: every output tile summed
    by one CTA in K order (SHG_DETERMINISTIC), Y reproducible bit for bit."""
    v = _variant(variant)
    lda = _mat(A, "A", (torch.float32,))
    ldo = _mat(omega, "omega", (torch.bfloat16,) if v in (1, 2) else (torch.float16,))
    m = A.shape[1] if trans_a else A.shape[0]
    n = A.shape[0] if trans_a else A.shape[1]
    k = omega.shape[1]
    if omega.shape[0] != n:
        raise ValueError(f"omega has {omega.shape[0]} rows, expected {n}")
    if out is None:
        out = torch.empty(m, k, dtype=torch.float32, device=A.device)
    ldy = _mat(out, "out", (torch.float32,))
    fl = flags if flags is not None else new_flags(A.device)
    _check(_lib.load().shgemm_project(m, n, k, _ptr(A), lda, int(trans_a), _ptr(omega), ldo, _ptr(out), ldy,
                                      v | (SHG_DETERMINISTIC if deterministic else 0), _ptr(fl), _stream(stream)),
           "shgemm_project")
    if check:
        check_flags(fl, "shgemm_project")
    return out


def _config(arr) -> dict:
    return {"a_stages": arr[0], "b_stages": arr[1], "drain_kblocks": arr[2], "n_groups": bool(arr[3]),
            "cached": bool(arr[4]), "wide": bool(arr[5]), "pair": arr[5] == 2}


def shg_autotune_project(A: torch.Tensor, omega: torch.Tensor, variant="f16", trans_a: bool = False, reps: int = 3,
                         out: torch.Tensor | None = None, flags: torch.Tensor | None = None, stream=None) -> dict:
    """Time the launch configurations of the projection A @ omega and cache
    the fastest for its shape class (synchronises; ``out`` is overwritten)."""
    v = _variant(variant)
    lda = _mat(A, "A", (torch.float32,))
    ldo = _mat(omega, "omega", (torch.bfloat16,) if v in (1, 2) else (torch.float16,))
    m = A.shape[1] if trans_a else A.shape[0]
    n = A.shape[0] if trans_a else A.shape[1]
    k = omega.shape[1]
    if omega.shape[0] != n:
        raise ValueError(f"omega has {omega.shape[0]} rows, expected {n}")
    if out is None:
        out = torch.empty(m, k, dtype=torch.float32, device=A.device)
    ldy = _mat(out, "out", (torch.float32,))
    fl = flags if flags is not None else new_flags(A.device)
    cfg = (ctypes.c_int32 * 6)()
    _check(_lib.load().shg_autotune_project(m, n, k, _ptr(A), lda, int(trans_a), _ptr(omega), ldo, _ptr(out), ldy,
                                            v, reps, _ptr(fl), _stream(stream), cfg), "shg_autotune_project")
    return _config(cfg)


def shg_autotune_lookup(m: int, n: int, k: int, trans_a: bool = False, variant="f16") -> dict:
    cfg = (ctypes.c_int32 * 6)()
    _check(_lib.load().shg_autotune_lookup(m, n, k, int(trans_a), _variant(variant), cfg), "shg_autotune_lookup")
    return _config(cfg)


def shg_autotune_clear() -> None:
    _check(_lib.load().shg_autotune_clear(), "shg_autotune_clear")


TUNE_RECORD = 15
_TUNE_FIELDS = ("a_layout", "b_mode", "pieces", "n_tile", "n_tiles", "m_log2", "k_log2", "k_pieces",
                "a_stages", "b_stages", "drain_kblocks", "n_groups", "wide", "pair", "whole_tiles")


def shg_autotune_export() -> list[dict]:
    """The autotuner's cache, one dict per shape class."""
    lib = _lib.load()
    n = ctypes.c_int32(0)
    _check(lib.shg_autotune_export(None, 0, ctypes.byref(n)), "shg_autotune_export")
    buf = (ctypes.c_int32 * max(1, n.value * TUNE_RECORD))()
    _check(lib.shg_autotune_export(buf, n.value, ctypes.byref(n)), "shg_autotune_export")
    return [dict(zip(_TUNE_FIELDS, buf[i * TUNE_RECORD:(i + 1) * TUNE_RECORD])) for i in range(n.value)]


def shg_autotune_import(entries: list[dict]) -> int:
    """Add cache entries (as shg_autotune_export gives them) for the classes
    not cached yet; returns how many were added."""
    vals = [int(e[f]) for e in entries for f in _TUNE_FIELDS]
    buf = (ctypes.c_int32 * max(1, len(vals)))(*vals)
    added = ctypes.c_int32(0)
    _check(_lib.load().shg_autotune_import(buf, len(entries), ctypes.byref(added)), "shg_autotune_import")
    return added.value


def save_autotune(path: str, gpu_name: str | None = None, sm_count: int | None = None) -> int:
    """Write the autotuner's cache to a JSON file keyed by the GPU's name and
    SM count (those of the current CUDA device unless given); returns the
    number of entries written."""
    import json
    if gpu_name is None or sm_count is None:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        gpu_name = props.name if gpu_name is None else gpu_name
        sm_count = props.multi_processor_count if sm_count is None else sm_count
    entries = shg_autotune_export()
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump({"format": "shg-autotune-1", "gpu": gpu_name, "sm_count": int(sm_count), "entries": entries}, f,
                  indent=1)
    os.replace(tmp, path)
    return len(entries)


def load_autotune(path: str, gpu_name: str | None = None, sm_count: int | None = None) -> int:
    """Load a cache written by save_autotune when it was made on the same kind
    of GPU (name and SM count); returns the number of entries added (0 for a
    missing file or another GPU)."""
    import json
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        d = json.load(f)
    if d.get("format") != "shg-autotune-1":
        raise ValueError(f"{path}: not an autotune cache")
    if gpu_name is None or sm_count is None:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        gpu_name = props.name if gpu_name is None else gpu_name
        sm_count = props.multi_processor_count if sm_count is None else sm_count
    if d.get("gpu") != gpu_name or int(d.get("sm_count", -1)) != int(sm_count):
        return 0
    return shg_autotune_import(d["entries"])


def shg_rsvd_batched_autotune(As, ranks, oversampling: int, seed: int = 0, reps: int = 3,
                              workspace: torch.Tensor | None = None, flags: torch.Tensor | None = None,
                              stream=None) -> int:
    """Tune the projection of every shape class of a batch; returns the
    number of classes timed."""
    b = len(As)
    ms, ns = [int(A.shape[0]) for A in As], [int(A.shape[1]) for A in As]
    ldas = [_mat(A, f"A[{i}]", (torch.float32,)) for i, A in enumerate(As)]
    dev_ = As[0].device
    need = rsvd_batched_workspace_size(ms, ns, ranks, oversampling, 0)
    ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=dev_)
    fl = flags if flags is not None else new_flags(dev_)
    tuned = ctypes.c_int32()
    _check(_lib.load().shg_rsvd_batched_autotune(
        b, _host_array(ctypes.c_int64, ms), _host_array(ctypes.c_int64, ns), _host_array(ctypes.c_int64, ranks),
        oversampling, _host_array(ctypes.c_void_p, [A.data_ptr() for A in As]), _host_array(ctypes.c_int64, ldas),
        seed, _ptr(ws), ws.numel(), reps, _ptr(fl), _stream(stream), ctypes.byref(tuned)), "shg_rsvd_batched_autotune")
    return tuned.value


def shg_gemm_split3(A: torch.Tensor, B: torch.Tensor, trans_a: bool = False, out: torch.Tensor | None = None,
                    accumulate: bool = False, flags: torch.Tensor | None = None, check: bool = True,
                    stream=None) -> torch.Tensor:
    lda = _mat(A, "A", (torch.float32,))
    ldb = _mat(B, "B", (torch.float32,))
    m = A.shape[1] if trans_a else A.shape[0]
    kk = A.shape[0] if trans_a else A.shape[1]
    n = B.shape[1]
    if B.shape[0] != kk:
        raise ValueError("inner dimensions differ")
    if out is None:
        out = torch.empty(m, n, dtype=torch.float32, device=A.device)
    ldc = _mat(out, "out", (torch.float32,))
    fl = flags if flags is not None else new_flags(A.device)
    _check(_lib.load().shg_gemm_split3(m, n, kk, _ptr(A), lda, int(trans_a), _ptr(B), ldb, _ptr(out), ldc,
                                       int(accumulate), _ptr(fl), _stream(stream)), "shg_gemm_split3")
    if check:
        check_flags(fl, "shg_gemm_split3")
    return out


def shg_sgemm(A: torch.Tensor, B: torch.Tensor, trans_a: bool = False, out: torch.Tensor | None = None,
              accumulate: bool = False, stream=None) -> torch.Tensor:
    lda = _mat(A, "A", (torch.float32,))
    ldb = _mat(B, "B", (torch.float32, torch.float16))
    m = A.shape[1] if trans_a else A.shape[0]
    kk = A.shape[0] if trans_a else A.shape[1]
    n = B.shape[1]
    if B.shape[0] != kk:
        raise ValueError("inner dimensions differ")
    if out is None:
        out = torch.empty(m, n, dtype=torch.float32, device=A.device)
    ldc = _mat(out, "out", (torch.float32,))
    _check(_lib.load().shg_sgemm(m, n, kk, _ptr(A), lda, int(trans_a), _ptr(B), ldb,
                                 int(B.dtype == torch.float16), _ptr(out), ldc, int(accumulate), _stream(stream)),
           "shg_sgemm")
    return out


def shg_gram(X: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """G = X^T X (k x k FP64; upper triangle, zeros below)."""
    ldx = _mat(X, "X", (torch.float32,))
    m, k = X.shape
    if out is None:
        out = torch.empty(k, k, dtype=torch.float64, device=X.device)
    if out.dtype != torch.float64 or tuple(out.shape) != (k, k) or not out.is_contiguous():
        raise ValueError("out must be a contiguous k x k float64 tensor")
    _check(_lib.load().shg_gram(m, k, _ptr(X), ldx, _ptr(out), _stream(stream)), "shg_gram")
    return out


def shg_cholqr2(X: torch.Tensor, workspace: torch.Tensor | None = None, flags: torch.Tensor | None = None,
                check: bool = True, stream=None) -> torch.Tensor:
    ldx = _mat(X, "X", (torch.float32,))
    m, k = X.shape
    lib = _lib.load()
    need = ctypes.c_size_t()
    _check(lib.shg_cholqr2_workspace_size(m, k, ctypes.byref(need)), "shg_cholqr2_workspace_size")
    ws = workspace if workspace is not None else torch.empty(need.value, dtype=torch.uint8, device=X.device)
    fl = flags if flags is not None else new_flags(X.device)
    _check(lib.shg_cholqr2(m, k, _ptr(X), ldx, _ptr(ws), ws.numel(), _ptr(fl), _stream(stream)), "shg_cholqr2")
    if check:
        check_flags(fl, "shg_cholqr2")
    return X


def shg_cholqr2_static(X: torch.Tensor, flags: torch.Tensor | None = None, check: bool = True,
                       stream=None) -> torch.Tensor:
    """shg_cholqr2 on the library's static scratch (no workspace argument)."""
    ldx = _mat(X, "X", (torch.float32,))
    m, k = X.shape
    lib = _lib.load()
    _check(lib.shg_cholqr2_static(m, k, _ptr(X), ldx, _ptr(flags) if flags is not None else None,
                                  _stream(stream)), "shg_cholqr2_static")
    if check and flags is not None:
        check_flags(flags, "shg_cholqr2_static")
    return X


def _host_array(ctype, values):
    return (ctype * len(values))(*values)


def rsvd_batched_workspace_size(ms, ns, ranks, oversampling: int, power_iters: int = 0) -> int:
    b = len(ms)
    need = ctypes.c_size_t()
    _check(_lib.load().shg_rsvd_batched_workspace_size(
        b, _host_array(ctypes.c_int64, ms), _host_array(ctypes.c_int64, ns), _host_array(ctypes.c_int64, ranks),
        oversampling, power_iters, ctypes.byref(need)), "shg_rsvd_batched_workspace_size")
    return need.value


def shg_rsvd_batched(As, ranks, oversampling: int, power_iters: int = 0, omegas=None, seed: int = 0,
                     variant="f16", use_graph: bool = True, out=None, workspace: torch.Tensor | None = None,
                     flags: torch.Tensor | None = None, check: bool = True, stream=None):
    """Randomized SVD of every A in As (Algorithm 1 per problem, run concurrently).

    omegas: None (all generated from ``seed``) or a list whose entries are FP16
    tensors or None.  Returns (Us, Ss, Vs) lists; ``out`` may pass them in
    (needed for graph replay, which is keyed on the output pointers).
    """
    b = len(As)
    ms, ns = [int(A.shape[0]) for A in As], [int(A.shape[1]) for A in As]
    ldas = [_mat(A, f"A[{i}]", (torch.float32,)) for i, A in enumerate(As)]
    dev_ = As[0].device
    if out is None:
        Us = [torch.empty(m, r, device=dev_) for m, r in zip(ms, ranks)]
        Ss = [torch.empty(r, device=dev_) for r in ranks]
        Vs = [torch.empty(n, r, device=dev_) for n, r in zip(ns, ranks)]
    else:
        Us, Ss, Vs = out
    lib = _lib.load()
    if workspace is None:   # (a caller's workspace is checked against the need by the library)
        need = rsvd_batched_workspace_size(ms, ns, ranks, oversampling, power_iters)
        workspace = torch.empty(need, dtype=torch.uint8, device=dev_)
    ws = workspace
    fl = flags if flags is not None else new_flags(dev_)
    if omegas is None:
        om_arr, ldo_arr = None, None
    else:
        om_arr = _host_array(ctypes.c_void_p, [o.data_ptr() if o is not None else 0 for o in omegas])
        ldo_arr = _host_array(ctypes.c_int64, [o.stride(0) if o is not None else 0 for o in omegas])
    _check(lib.shg_rsvd_batched(
        b, _host_array(ctypes.c_int64, ms), _host_array(ctypes.c_int64, ns), _host_array(ctypes.c_int64, ranks),
        oversampling, power_iters, _host_array(ctypes.c_void_p, [A.data_ptr() for A in As]),
        _host_array(ctypes.c_int64, ldas), om_arr, ldo_arr, seed,
        _host_array(ctypes.c_void_p, [U.data_ptr() for U in Us]), _host_array(ctypes.c_void_p, [S.data_ptr() for S in Ss]),
        _host_array(ctypes.c_void_p, [V.data_ptr() for V in Vs]), _ptr(ws), ws.numel(), _variant(variant),
        int(use_graph), _ptr(fl), _stream(stream)), "shg_rsvd_batched")
    if check:
        check_flags(fl, "shg_rsvd_batched")
    return Us, Ss, Vs


def shg_alpha_y_f16() -> float:
    """Variance of an FP16-rounded N(0,1) value (alpha_Y of Sec. 3.2)."""
    return float(_lib.load().shg_alpha_y_f16())


def shg_round_f16(x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """RN_fp16 of an FP32 matrix, in the library's kernel."""
    ldx = _mat(x, "x", (torch.float32,))
    rows, cols = x.shape
    y = out if out is not None else torch.empty(rows, cols, dtype=torch.float16, device=x.device)
    ldy = _mat(y, "out", (torch.float16,))
    _check(_lib.load().shg_round_f16(rows, cols, _ptr(x), ldx, _ptr(y), ldy, _stream(stream)), "shg_round_f16")
    return y


def shg_residual_estimate(A: torch.Tensor, Q: torch.Tensor, t: int = 16, seed: int = 0, offset: int = 0,
                          alpha: float = 0.0, flags: torch.Tensor | None = None, check: bool = True,
                          stream=None) -> torch.Tensor:
    """Device doubles [est, ||(I - QQ^T) A G||_F^2, ||A||_F^2] with t FP16 Gaussian probes."""
    lda = _mat(A, "A", (torch.float32,))
    ldq = _mat(Q, "Q", (torch.float32,))
    m, n = A.shape
    k = Q.shape[1]
    if Q.shape[0] != m:
        raise ValueError("Q must have as many rows as A")
    lib = _lib.load()
    need = ctypes.c_size_t()
    _check(lib.shg_residual_estimate_workspace_size(m, n, k, t, ctypes.byref(need)),
           "shg_residual_estimate_workspace_size")
    ws = torch.empty(need.value, dtype=torch.uint8, device=A.device)
    out = torch.empty(3, dtype=torch.float64, device=A.device)
    fl = flags if flags is not None else new_flags(A.device)
    _check(lib.shg_residual_estimate(m, n, k, t, _ptr(A), lda, _ptr(Q), ldq, seed, offset, float(alpha), _ptr(out),
                                     _ptr(ws), ws.numel(), _ptr(fl), _stream(stream)), "shg_residual_estimate")
    if check:
        check_flags(fl, "shg_residual_estimate")
    return out


def shg_sketch_loss_grad(A: torch.Tensor, Y: torch.Tensor, want_grad: bool = True,
                         flags: torch.Tensor | None = None, check: bool = True, stream=None):
    """(loss as a device double, dloss/dOmega n x k FP32 or None) for Y = A fp16(Omega)."""
    lda = _mat(A, "A", (torch.float32,))
    ldy = _mat(Y, "Y", (torch.float32,))
    m, n = A.shape
    k = Y.shape[1]
    if Y.shape[0] != m:
        raise ValueError("Y must have as many rows as A")
    lib = _lib.load()
    need = ctypes.c_size_t()
    _check(lib.shg_sketch_loss_grad_workspace_size(m, n, k, ctypes.byref(need)),
           "shg_sketch_loss_grad_workspace_size")
    ws = torch.empty(need.value, dtype=torch.uint8, device=A.device)
    loss = torch.empty((), dtype=torch.float64, device=A.device)
    grad = torch.empty(n, k, dtype=torch.float32, device=A.device) if want_grad else None
    fl = flags if flags is not None else new_flags(A.device)
    _check(lib.shg_sketch_loss_grad(m, n, k, _ptr(A), lda, _ptr(Y), ldy, int(want_grad), _ptr(grad),
                                    k if want_grad else 0, _ptr(loss), _ptr(ws), ws.numel(), _ptr(fl),
                                    _stream(stream)), "shg_sketch_loss_grad")
    if check:
        check_flags(fl, "shg_sketch_loss_grad")
    return loss, grad


def rsvd_workspace_size(m: int, n: int, rank: int, oversampling: int, power_iters: int = 0) -> int:
    need = ctypes.c_size_t()
    _check(_lib.load().shg_rsvd_workspace_size(m, n, rank, oversampling, power_iters, ctypes.byref(need)),
           "shg_rsvd_workspace_size")
    return need.value


def shg_rsvd(A: torch.Tensor, omega: torch.Tensor | None, rank: int, oversampling: int, power_iters: int = 0,
             variant="f16", want_q: bool = False, workspace: torch.Tensor | None = None,
             out=None, flags: torch.Tensor | None = None, check: bool = True, stream=None, seed: int = 0,
             report: bool = False):
    """Randomized SVD (Algorithm 1).  Returns (U, S, V[, Q][, report]) with
    A ~= U diag(S) V^T.  omega=None generates the test matrix from ``seed``
    (shg_gaussian_f16(seed, 0, n, k)).  report=True synchronises and adds
    the shg_report as a dict (phase times of Algorithm 1, smallest Cholesky
    pivot ratio, a-posteriori residual estimate)."""
    v = _variant(variant)
    lda = _mat(A, "A", (torch.float32,))
    m, n = A.shape
    k = rank + oversampling
    if omega is not None:
        ldo = _mat(omega, "omega", (torch.bfloat16,) if v in (1, 2) else (torch.float16,))
        if omega.shape != (n, k):
            raise ValueError(f"omega must be {n} x {k}")
    else:
        ldo = 0
    dev = A.device
    if out is None:
        U = torch.empty(m, rank, dtype=torch.float32, device=dev)
        S = torch.empty(rank, dtype=torch.float32, device=dev)
        V = torch.empty(n, rank, dtype=torch.float32, device=dev)
        Q = torch.empty(m, k, dtype=torch.float32, device=dev) if want_q else None
    else:
        U, S, V, Q = out
    need = rsvd_workspace_size(m, n, rank, oversampling, power_iters)
    ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=dev)
    fl = flags if flags is not None else new_flags(dev)
    rep = _lib.Report() if report else None
    _check(_lib.load().shg_rsvd(m, n, rank, oversampling, power_iters, _ptr(A), lda, _ptr(omega), ldo, seed,
                                _ptr(U), _ptr(S), _ptr(V), _ptr(Q), _ptr(ws), ws.numel(), v, _ptr(fl),
                                _stream(stream), ctypes.byref(rep) if rep is not None else None), "shg_rsvd")
    if check:
        check_flags(fl, "shg_rsvd")
    res = (U, S, V, Q) if want_q else (U, S, V)
    return res + (rep.as_dict(),) if report else res


def rp_hosvd_workspace_size(dims, ranks, oversampling: int = 0) -> int:
    d = (ctypes.c_int64 * 3)(*dims)
    r = (ctypes.c_int64 * 3)(*ranks)
    need = ctypes.c_size_t()
    _check(_lib.load().shg_rp_hosvd_workspace_size(3, d, r, oversampling, ctypes.byref(need)),
           "shg_rp_hosvd_workspace_size")
    return need.value


def _omega_rows(dims, i):
    rows = 1
    for j, d in enumerate(dims):
        if j != i:
            rows *= d
    return rows


def shg_mode_project(X: torch.Tensor, omega: torch.Tensor, mode: int, variant="f16", out: torch.Tensor | None = None,
                     flags: torch.Tensor | None = None, check: bool = True, stream=None) -> torch.Tensor:
    """W = X_(mode) @ omega for a contiguous 3-way float32 tensor (the mode
    projection of Algorithm 2); omega is (prod of the other dims) x J FP16."""
    if X.dim() != 3 or not X.is_contiguous() or X.dtype != torch.float32 or not X.is_cuda:
        raise ValueError("X must be a contiguous 3-way float32 CUDA tensor")
    dims = list(X.shape)
    ldo = _mat(omega, "omega", (torch.float16,))
    J = omega.shape[1]
    if omega.shape[0] != _omega_rows(dims, mode):
        raise ValueError(f"omega must have {_omega_rows(dims, mode)} rows")
    if out is None:
        out = torch.empty(dims[mode], J, dtype=torch.float32, device=X.device)
    ldw = _mat(out, "out", (torch.float32,))
    fl = flags if flags is not None else new_flags(X.device)
    d = (ctypes.c_int64 * 3)(*dims)
    _check(_lib.load().shg_mode_project(3, d, int(mode), J, _ptr(X), _ptr(omega), ldo, _ptr(out), ldw,
                                        _variant(variant), _ptr(fl), _stream(stream)), "shg_mode_project")
    if check:
        check_flags(fl, "shg_mode_project")
    return out


def shg_rp_hosvd(X: torch.Tensor, omegas, ranks, variant="f16", workspace: torch.Tensor | None = None,
                 out=None, flags: torch.Tensor | None = None, check: bool = True, stream=None,
                 oversampling: int = 0, seed: int = 0):
    """RP-HOSVD (Algorithm 2) of a contiguous 3-way float32 tensor with target
    ranks r_i and oversampling s (J_i = r_i + s columns per mode).  omegas:
    None (all generated from ``seed``) or a list of FP16 tensors / None.
    Returns (core J0 x J1 x J2, [Q_0, Q_1, Q_2])."""
    if X.dim() != 3 or not X.is_contiguous() or X.dtype != torch.float32 or not X.is_cuda:
        raise ValueError("X must be a contiguous 3-way float32 CUDA tensor")
    dims = list(X.shape)
    ranks = [int(r) for r in ranks]
    J = [r + oversampling for r in ranks]
    oms = list(omegas) if omegas is not None else [None, None, None]
    for i, om in enumerate(oms):
        if om is None:
            continue
        rows = _omega_rows(dims, i)
        if om.dtype != torch.float16 or tuple(om.shape) != (rows, J[i]) or om.stride(1) != 1:
            raise ValueError(f"omega {i} must be a row-major float16 {rows} x {J[i]} tensor")
    dev = X.device
    if out is None:
        core = torch.empty(*J, dtype=torch.float32, device=dev)
        facs = [torch.empty(dims[i], J[i], dtype=torch.float32, device=dev) for i in range(3)]
    else:
        core, facs = out
    need = rp_hosvd_workspace_size(dims, ranks, oversampling)
    ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=dev)
    fl = flags if flags is not None else new_flags(dev)
    d = (ctypes.c_int64 * 3)(*dims)
    r = (ctypes.c_int64 * 3)(*ranks)
    om_ptrs = (ctypes.c_void_p * 3)(*[o.data_ptr() if o is not None else 0 for o in oms])
    om_lds = (ctypes.c_int64 * 3)(*[o.stride(0) if o is not None else 0 for o in oms])
    f_ptrs = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in facs])
    _check(_lib.load().shg_rp_hosvd(3, d, r, oversampling, _ptr(X), om_ptrs, om_lds, seed, _ptr(core), f_ptrs,
                                    _ptr(ws), ws.numel(), _variant(variant), _ptr(fl), _stream(stream)),
           "shg_rp_hosvd")
    if check:
        check_flags(fl, "shg_rp_hosvd")
    return core, facs
