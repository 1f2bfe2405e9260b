"""CPU-only checks of the C ABI: libshg.so loads, exports every symbol that
include/shg.h declares, and rejects bad arguments on the host (no GPU work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "shg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(shg\w+|shgemm\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2304_04612_gb300 import build as b
    b.build()
    from paper_2304_04612_gb300 import _lib
    return _lib.load()


def test_header_declares_the_paper_entry_points():
    names = declared_functions()
    for want in ("shgemm_project", "shg_rsvd", "shg_rp_hosvd", "shg_mode_project", "shg_gaussian_f16",
                 "shg_gemm_split3", "shg_sgemm", "shg_cholqr2"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2304_04612_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks a signature for {name}"


def test_status_strings(lib):
    for s in range(8):
        assert lib.shg_status_string(s)
    assert lib.shg_status_string(99) == b"unknown shg_status"
    assert lib.shg_flags_status(0) == 0
    assert lib.shg_flags_status(1) == 2      # RANGE
    assert lib.shg_flags_status(3) == 3      # NOT_SPD outranks RANGE
    assert lib.shg_flags_status(7) == 6      # TIMEOUT outranks all


def test_host_argument_validation(lib):
    null = ctypes.c_void_p(0)
    # m = 0 is rejected before any CUDA call
    assert lib.shgemm_project(0, 8, 8, null, 8, 0, null, 8, null, 8, 0, null, null) == 1
    # ld smaller than the row length
    one = ctypes.c_void_p(16)
    assert lib.shgemm_project(8, 8, 8, one, 4, 0, one, 8, one, 8, 0, one, null) == 1
    assert lib.shg_gaussian_f16(0, 0, -1, 4, null, 4, null) == 1
    assert lib.shg_gaussian_f16(0, 0, 0, 4, null, 4, null) == 0       # empty is a no-op
    sz = ctypes.c_size_t()
    assert lib.shg_rsvd_workspace_size(100, 100, 90, 20, 0, ctypes.byref(sz)) == 1   # k > min(m, n)
    assert lib.shg_rsvd_workspace_size(1024, 1024, 32, 32, 0, ctypes.byref(sz)) == 0
    assert sz.value > 1024 * 64 * 4
    assert lib.shg_rsvd_workspace_size(1 << 31, 1024, 32, 32, 0, ctypes.byref(sz)) == 1   # m >= 2^31
    d = (ctypes.c_int64 * 3)(8, 8, 8)
    r = (ctypes.c_int64 * 3)(4, 9, 4)                                 # J > I
    assert lib.shg_rp_hosvd_workspace_size(3, d, r, 0, ctypes.byref(sz)) == 1
    assert lib.shg_rp_hosvd_workspace_size(4, d, r, 0, ctypes.byref(sz)) == 7
    r = (ctypes.c_int64 * 3)(4, 4, 4)
    assert lib.shg_rp_hosvd_workspace_size(3, d, r, 5, ctypes.byref(sz)) == 1     # rank + s > I
    assert lib.shg_rp_hosvd_workspace_size(3, d, r, -1, ctypes.byref(sz)) == 1
    assert lib.shg_rp_hosvd_workspace_size(3, d, r, 4, ctypes.byref(sz)) == 0
    # room for the three generated test matrices (64 x 8 FP16 each)
    assert sz.value >= 3 * 64 * 8 * 2
    # mode projection: bad mode, J > ld, NULL tensor, unsupported variant
    assert lib.shg_mode_project(3, d, 3, 4, one, one, 8, one, 8, 0, one, null) == 1
    assert lib.shg_mode_project(3, d, 0, 9, one, one, 8, one, 8, 0, one, null) == 1
    assert lib.shg_mode_project(3, d, 0, 4, null, one, 8, one, 8, 0, one, null) == 1
    assert lib.shg_mode_project(3, d, 0, 4, one, one, 8, one, 8, 1, one, null) == 7
    # CholeskyQR2: m >= 2^31 rejected by the workspace query and the static entry
    assert lib.shg_cholqr2_workspace_size(1 << 31, 16, ctypes.byref(sz)) == 1
    assert lib.shg_cholqr2_static(1 << 31, 16, one, 16, null, null) == 1
    # m k beyond the static scratch, with m k * 4 wrapping 64 bits: no wrap-around
    assert lib.shg_cholqr2_static((1 << 31) - 1, 1024, one, 1024, null, null) == 4
    # randomized SVD: NULL A, bad variant, short workspace (host checks only)
    assert lib.shg_rsvd(64, 64, 8, 8, 0, null, 64, null, 0, 0, one, one, one, null, one, 1 << 30, 0, one, null,
                        null) == 1
    assert lib.shg_rsvd(64, 64, 8, 8, 0, one, 64, null, 0, 0, one, one, one, null, one, 1 << 30, 9, one, null,
                        null) == 1
    assert lib.shg_rsvd(64, 64, 8, 8, 0, one, 64, null, 0, 0, one, one, one, null, one, 16, 0, one, null,
                        null) == 4
    # a passed Omega needs ldo >= k; a NULL Omega ignores ldo
    assert lib.shg_rsvd(64, 64, 8, 8, 0, one, 64, one, 8, 0, one, one, one, null, one, 1 << 30, 0, one, null,
                        null) == 1
    # autotuner: bad shapes, reps out of range and the SIMT variant (nothing
    # to tune) are rejected before any launch; lookup of an untuned class
    cfg = (ctypes.c_int32 * 6)()
    assert lib.shg_autotune_project(0, 8, 8, one, 8, 0, one, 8, one, 8, 0, 3, one, null, cfg) == 1
    assert lib.shg_autotune_project(8, 8, 8, one, 8, 0, one, 8, one, 8, 0, 0, one, null, cfg) == 1
    assert lib.shg_autotune_project(8, 8, 8, one, 8, 0, one, 8, one, 8, 3, 3, one, null, cfg) == 7
    assert lib.shg_autotune_clear() == 0
    assert lib.shg_autotune_lookup(4096, 4096, 64, 0, 0, cfg) == 0 and cfg[4] == 0
    assert lib.shg_autotune_lookup(4096, 4096, 64, 0, 3, cfg) == 7
    # Gram matrix: k = 0, k > 1024 and ldx < k are rejected before any launch
    assert lib.shg_gram(8, 0, one, 8, one, null) == 1
    assert lib.shg_gram(8, 1025, one, 1025, one, null) == 1
    assert lib.shg_gram(8, 8, one, 4, one, null) == 1


def test_alpha_y_f16_matches_the_oracle(lib):
    # the library computes alpha_Y (Sec. 3.2) on the host from its definition;
    # the oracle computes it independently in numpy / scipy
    from oracle.gaussian import FP16, alpha_Y
    a = lib.shg_alpha_y_f16()
    assert abs(a - alpha_Y(FP16)) <= 1e-13
    assert 0.99999990 < a < 1.0


def test_sketch_and_estimator_host_validation(lib):
    null = ctypes.c_void_p(0)
    sz = ctypes.c_size_t()
    assert lib.shg_residual_estimate_workspace_size(100, 80, 120, 16, ctypes.byref(sz)) == 1   # k > m
    assert lib.shg_residual_estimate_workspace_size(100, 80, 20, 0, ctypes.byref(sz)) == 1     # t < 1
    assert lib.shg_residual_estimate_workspace_size(100, 80, 20, 16, ctypes.byref(sz)) == 0
    assert sz.value >= 100 * 16 * 4 + 80 * 16 * 2
    assert lib.shg_sketch_loss_grad_workspace_size(100, 80, 2000, ctypes.byref(sz)) == 1       # k > m
    assert lib.shg_sketch_loss_grad_workspace_size(2048, 2048, 96, ctypes.byref(sz)) == 0
    # NULL operands are rejected before any CUDA call
    assert lib.shg_residual_estimate(100, 80, 20, 16, null, 80, null, 20, 0, 0, 0.0, null, null, 0, null,
                                     null) == 1
    assert lib.shg_sketch_loss_grad(100, 80, 20, null, 80, null, 20, 1, null, 20, null, null, 0, null, null) == 1
    assert lib.shg_round_f16(-1, 4, null, 4, null, 4, null) == 1
    assert lib.shg_round_f16(0, 4, null, 4, null, 4, null) == 0


def test_batched_workspace_host_validation(lib):
    sz = ctypes.c_size_t()
    m = (ctypes.c_int64 * 3)(512, 300, 2048)
    n = (ctypes.c_int64 * 3)(256, 300, 1024)
    r = (ctypes.c_int64 * 3)(32, 16, 64)
    assert lib.shg_rsvd_batched_workspace_size(3, m, n, r, 16, 1, ctypes.byref(sz)) == 0
    one = ctypes.c_size_t()
    assert lib.shg_rsvd_workspace_size(2048, 1024, 64, 16, 1, ctypes.byref(one)) == 0
    # one slice per branch (3 branches here), each at least the largest problem's need
    assert sz.value >= 3 * one.value
    bad = (ctypes.c_int64 * 3)(32, 300, 64)                          # rank + s > min(m, n)
    assert lib.shg_rsvd_batched_workspace_size(3, m, n, bad, 16, 1, ctypes.byref(sz)) == 1
    assert lib.shg_rsvd_batched_workspace_size(0, m, n, r, 16, 1, ctypes.byref(sz)) == 1
    null = ctypes.c_void_p(0)
    # NULL pointer arrays are rejected before any CUDA call
    assert lib.shg_rsvd_batched(3, m, n, r, 16, 1, null, null, null, null, 0, null, null, null, null, 0, 0, 0,
                                null, null) == 1
    # diagnostic entry: out-of-range wait limit rejected on the host
    assert lib.shg_diag_wait_timeout(8, 8, 8, ctypes.c_void_p(16), 8, ctypes.c_void_p(16), 8, ctypes.c_void_p(16), 8,
                                     10, ctypes.c_void_p(16), null) == 1


def test_report_struct_layout():
    # the ctypes mirror of struct shg_report: two int32, two doubles, the
    # phase times (no padding surprises between the int32 pair and the doubles)
    from paper_2304_04612_gb300 import _lib
    R = _lib.Report
    assert R.flags.offset == 0 and R.status.offset == 4
    assert R.min_pivot.offset == 8 and R.est_residual.offset == 16
    assert R.phase_ms.offset == 24 and ctypes.sizeof(R) == 24 + 4 * len(_lib.PHASES)
    src = open(HEADER).read()
    assert f"#define SHG_NUM_PHASES     {len(_lib.PHASES)}" in src


def test_deterministic_flag_matches_header():
    import paper_2304_04612_gb300 as shg
    src = open(HEADER).read()
    assert f"#define SHG_DETERMINISTIC 0x{shg.SHG_DETERMINISTIC:x}" in src
    # it lies above every variant number, so OR-ing it in never changes the variant
    assert all(v < shg.SHG_DETERMINISTIC for v in shg.VARIANTS.values())


def test_rsvd_workspace_covers_the_eigensolver_scratch(lib):
    # host-side sizing only: the workspace of a randomized SVD holds the
    # eigensolver's scratch on both sides of the one-CTA limit (k <= 158: the
    # rotation log of 40 sweeps x (k - 1) rounds x k / 2 (c, s) pairs; beyond:
    # three kpb x kpb buffers of A, V and two sets of 16 x 16 tile factors per
    # block pair, kpb = k rounded up to 16), odd k included
    sz = ctypes.c_size_t()
    for k in (33, 158, 159, 160, 266, 577, 1024):
        assert lib.shg_rsvd_workspace_size(2048, 2048, k - 16, 16, 0, ctypes.byref(sz)) == 0
        kp = k + (k & 1)
        kpb = (k + 15) // 16 * 16
        if kp <= 158:
            need = 40 * (kp - 1) * (kp // 2) * 8
        else:
            need = (4 * kpb * kpb + 2 * (kpb // 16) * 256) * 4
        assert sz.value >= need + 2048 * k * 4, k
