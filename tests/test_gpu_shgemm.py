"""GPU parity of the projection kernels against the FP64 oracle.

Tolerances (from the method, Sec. 4.3 / 4.4.1):
* SHGEMM-FP16: relative Frobenius error <= 1e-5 and <= 2x the FP32 SIMT
  error on the same inputs; every element within the paper's bound
  (1/8) n u |A||Omega| plus the split's representation bound u16^2 |A||Omega|.
* BF16x3: same FP32-level bound; BF16x2: 2^-16-level (two 8-bit pieces).
* TCEC split product: FP32-level relative error <= 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import shgemm as OS
from oracle import gaussian as OG
from oracle.lowp import FP16, BF16, round_rn, encode_bf16
from synth import uniform, omega_f16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shg():
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as m
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def padded_f32(A):
    """FP32 matrix stored with a leading dimension rounded up to a multiple of 4
    (the 16-byte TMA stride rule); returns the (rows x cols) view."""
    r, c = A.shape
    buf = torch.zeros(r, (c + 3) // 4 * 4, dtype=torch.float32, device="cuda")
    buf[:, :c] = dev(A)
    return buf[:, :c]


def padded_omega(Om, ld):
    """n x k FP16 Omega stored with leading dimension ld (TMA wants ld % 8 == 0)."""
    n, k = Om.shape
    buf = torch.zeros(n, ld, dtype=torch.float16, device="cuda")
    buf[:, :k] = dev(Om)
    return buf[:, :k]


SHAPES = [(300, 1000, 64), (129, 67, 1), (256, 512, 200), (1000, 300, 256), (200, 640, 512),
          (64, 4096, 48), (1, 130, 8), (513, 2048, 96), (128, 64, 128), (77, 1536, 144)]


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("trans", [False, True])
def test_shgemm_f16_parity(shg, m, n, k, trans):
    A = uniform(n, m, seed=2) if trans else uniform(m, n, seed=2)
    Om = omega_f16(n, k, seed=1)
    om_t = padded_omega(Om, (k + 7) // 8 * 8)
    At = padded_f32(A)
    Y = shg.shgemm_project(At, om_t, "f16", trans_a=trans).cpu().numpy()
    A_op = A.T.copy() if trans else A
    ref = OS.project_exact(A_op, Om)
    err = OS.rel_fro_error(Y, ref)
    Ys = shg.shgemm_project(At, om_t, "fp32", trans_a=trans).cpu().numpy()
    err_simt = OS.rel_fro_error(Ys, ref)
    # no worse than 2x the FP32 SIMT path; the split's own representation
    # error (hi + 2^-11 lo with exact products, no accumulation error) is a
    # floor no accumulation order can go below
    err_repr = OS.rel_fro_error(OS.shgemm_emulated(A_op, Om), ref)
    assert err <= 1e-5, (err, err_simt)
    assert err <= max(2.0 * err_simt, 2.0 * err_repr), (err, err_simt, err_repr)
    bound = OS.elementwise_bound(A_op, Om) * (1 if n >= 8 else 8.0 / n) + \
        OS.U_FP16 ** 2 * (np.abs(A_op.astype(np.float64)) @ np.abs(Om.astype(np.float64)))
    viol = np.abs(Y - ref) > bound * (1 + 1e-6) + 1e-30
    assert not viol.any(), f"{viol.sum()} elements exceed the Sec. 4.3 bound"


@pytest.mark.parametrize("m,n,k", [(256, 512, 200), (1000, 300, 256), (200, 640, 512), (77, 1536, 144),
                                   (513, 2048, 160), (300, 1000, 320)])
@pytest.mark.parametrize("tiles", ["pair", "wide", "narrow"])
def test_shgemm_f16_tile_widths(shg, monkeypatch, m, n, k, tiles):
    """k > 128 runs on 256 x 256 output tiles computed by pairs of CTAs
    (SHG_PAIR=1), on 128 x 256 tiles per CTA whose A operand is split in
    shared memory (SHG_PAIR=0), or on 128-column tiles split into tensor
    memory (SHG_WIDE=0); each against the exact product with the same
    tolerances as above."""
    monkeypatch.setenv("SHG_WIDE", "0" if tiles == "narrow" else "1")
    monkeypatch.setenv("SHG_PAIR", "1" if tiles == "pair" else "0")
    A = uniform(m, n, seed=12)
    Om = omega_f16(n, k, seed=13)
    Y = shg.shgemm_project(padded_f32(A), padded_omega(Om, (k + 7) // 8 * 8), "f16").cpu().numpy()
    ref = OS.project_exact(A, Om)
    err = OS.rel_fro_error(Y, ref)
    Ys = shg.shgemm_project(padded_f32(A), padded_omega(Om, (k + 7) // 8 * 8), "fp32").cpu().numpy()
    err_simt = OS.rel_fro_error(Ys, ref)
    err_repr = OS.rel_fro_error(OS.shgemm_emulated(A, Om), ref)
    assert err <= 1e-5, (err, err_simt)
    assert err <= max(2.0 * err_simt, 2.0 * err_repr), (err, err_simt, err_repr)
    bound = OS.elementwise_bound(A, Om) + \
        OS.U_FP16 ** 2 * (np.abs(A.astype(np.float64)) @ np.abs(Om.astype(np.float64)))
    assert not (np.abs(Y - ref) > bound * (1 + 1e-6) + 1e-30).any()


def test_shgemm_ld_and_offsets(shg):
    """Leading dimensions larger than the row length on A, Omega and Y."""
    m, n, k = 200, 700, 40
    A = uniform(m, n + 12, seed=5)
    Om = omega_f16(n, k, seed=6)
    At = dev(A)[:, :n]
    Yb = torch.full((m, k + 9), 7.0, device="cuda")
    shg.shgemm_project(At, padded_omega(Om, 56), out=Yb[:, :k])
    Y = Yb.cpu().numpy()
    assert OS.rel_fro_error(Y[:, :k], OS.project_exact(A[:, :n], Om)) < 1e-5
    assert np.all(Y[:, k:] == 7.0)              # nothing written past the row


def padded_bf16(W):
    """n x k BF16 tensor of the float64 values W (exact in BF16), stored with a
    leading dimension rounded up to a multiple of 8 (TMA stride rule)."""
    n, k = W.shape
    buf = torch.zeros(n, (k + 7) // 8 * 8, dtype=torch.bfloat16, device="cuda")
    buf[:, :k] = torch.from_numpy(encode_bf16(W).view(np.int16)).cuda().view(torch.bfloat16)
    return buf[:, :k]


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("pieces,tol", [(3, 1e-5), (2, 2e-4)])
def test_shgemm_bf16_parity(shg, m, n, k, trans, pieces, tol):
    """BF16 split (three or two pieces at 2^0, 2^-8, 2^-16) against the exact
    product with Omega rounded RN to BF16, on the ragged, k = 1 and
    transposed shapes of the FP16 test.  Three pieces carry the 24 bits of
    an FP32 value (FP32-level tolerance); two pieces carry 16 (2^-16 level)."""
    A = uniform(n, m, seed=2) if trans else uniform(m, n, seed=2)
    Om = omega_f16(n, k, seed=1)
    Wb = OS.bf16_omega(Om)                      # RN_bf16 of the FP16 values
    A_op = A.T.copy() if trans else A
    Y = shg.shgemm_project(padded_f32(A), padded_bf16(Wb), "bf16x3" if pieces == 3 else "bf16x2",
                           trans_a=trans).cpu().numpy()
    ref = A_op.astype(np.float64) @ Wb
    err = OS.rel_fro_error(Y, ref)
    assert err <= tol, err
    emu = OS.shgemm_bf16_emulated(A_op, Om, pieces)
    assert OS.rel_fro_error(emu, ref) <= tol


@pytest.mark.parametrize("m,n,kk,trans", [(300, 64, 1000, False), (1000, 48, 300, True), (130, 200, 257, False),
                                          (1024, 64, 1024, True), (96, 136, 640, True)])
def test_split3_parity(shg, m, n, kk, trans):
    A = uniform(kk, m, seed=3) if trans else uniform(m, kk, seed=3)
    B = uniform(kk, n, seed=4)
    C = shg.shg_gemm_split3(padded_f32(A), padded_f32(B), trans_a=trans).cpu().numpy()
    A_op = A.T if trans else A
    ref = A_op.astype(np.float64) @ B.astype(np.float64)
    assert OS.rel_fro_error(C, ref) <= 1e-5


def test_split3_accumulate(shg):
    A = uniform(200, 300, seed=7)
    B = uniform(300, 64, seed=8)
    C0 = uniform(200, 64, seed=9)
    C = dev(C0)
    shg.shg_gemm_split3(dev(A), dev(B), out=C, accumulate=True)
    ref = C0.astype(np.float64) + A.astype(np.float64) @ B.astype(np.float64)
    assert OS.rel_fro_error(C.cpu().numpy(), ref) < 1e-6


@pytest.mark.parametrize("trans,bf16", [(False, False), (True, False), (False, True), (True, True)])
def test_sgemm_parity(shg, trans, bf16):
    m, n, kk = 257, 70, 900
    A = uniform(kk, m, seed=3) if trans else uniform(m, kk, seed=3)
    if bf16:
        Bn = omega_f16(kk, n, seed=4)
        Bt = dev(Bn)
        Bref = Bn.astype(np.float64)
    else:
        Bn = uniform(kk, n, seed=4)
        Bt = dev(Bn)
        Bref = Bn.astype(np.float64)
    C = shg.shg_sgemm(dev(A), Bt, trans_a=trans).cpu().numpy()
    ref = (A.T if trans else A).astype(np.float64) @ Bref
    assert OS.rel_fro_error(C, ref) < 1e-5


def test_range_flag_raises(shg):
    A = uniform(256, 512, seed=1)
    A[17, 33] = 70000.0
    Om = omega_f16(512, 64, seed=1)
    with pytest.raises(shg.ShgError) as ei:
        shg.shgemm_project(dev(A), dev(Om), "f16")
    assert ei.value.status == 2
    # the FP32 path and the BF16 split have the full exponent range
    shg.shgemm_project(dev(A), dev(Om), "fp32")
    A[17, 33] = 65519.0                    # still rounds to a finite FP16 value
    shg.shgemm_project(dev(A), dev(Om), "f16")


def test_gaussian_generator_matches_philox_oracle(shg):
    rows, cols = 333, 77
    g = shg.shg_gaussian_f16(seed=1234, offset=5, rows=rows, cols=cols).cpu().numpy().astype(np.float64)
    ref = OG.gaussian_f16(1234, 5, rows, cols)
    same = g == ref
    assert same.mean() > 0.999
    # the rest differs only by FP16 rounding of FP32 vs FP64 Box-Muller values
    d = np.abs(g - ref)[~same]
    assert np.all(d <= 2.0 ** -10 * np.maximum(np.abs(ref[~same]), 2.0 ** -14))


def test_gaussian_generator_layout_independent(shg):
    a = shg.shg_gaussian_f16(7, 0, 40, 30).cpu()
    buf = torch.zeros(40, 64, dtype=torch.float16, device="cuda")
    shg.shg_gaussian_f16(7, 0, 40, 30, out=buf[:, :30])
    assert torch.equal(a, buf[:, :30].cpu())
    assert torch.count_nonzero(buf[:, 30:]) == 0


@pytest.mark.parametrize("variant,k", [("f16", 64), ("f16", 512), ("tf32", 96), ("fp32", 64)])
def test_deterministic_projection_is_bitwise_reproducible(shg, variant, k):
    """SHG_DETERMINISTIC: each output tile summed by one CTA in K order, so two
    runs give the same bits; the result still meets the projection bound.  The
    shape (40 tiles of 128 rows, fewer than the SMs, and a long K range) is one
    where the default stream-K schedule splits every tile across CTAs."""
    m, n = 5000, 6144
    A_h = uniform(m, n, seed=41)
    Om_h = omega_f16(n, k, seed=42)
    A, Om = dev(A_h), dev(Om_h)
    ys = [shg.shgemm_project(A, Om, variant, deterministic=True) for _ in range(3)]
    for y in ys[1:]:
        assert torch.equal(y, ys[0])
    ref = OS.project_exact(A_h, Om_h)
    err = np.linalg.norm(ys[0].cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err


@pytest.mark.parametrize("tiles", ["pair", "wide"])
def test_deterministic_wide_tiles(shg, monkeypatch, tiles):
    """SHG_DETERMINISTIC on the two kernels of k > 128 (256 x 256 tiles on CTA
    pairs, 128 x 256 tiles per CTA): whole output tiles per CTA range, the
    same bits on every run, within the projection tolerance."""
    monkeypatch.setenv("SHG_PAIR", "1" if tiles == "pair" else "0")
    m, n, k = 3000, 4096, 384
    A_h = uniform(m, n, seed=43)
    Om_h = omega_f16(n, k, seed=44)
    A, Om = dev(A_h), dev(Om_h)
    ys = [shg.shgemm_project(A, Om, "f16", deterministic=True) for _ in range(3)]
    for y in ys[1:]:
        assert torch.equal(y, ys[0])
    ref = OS.project_exact(A_h, Om_h)
    err = OS.rel_fro_error(ys[0].cpu().numpy(), ref)
    assert err <= 1e-5, err
    Yd = shg.shgemm_project(A, Om, "f16").cpu().numpy()   # the stream-K schedule, same tolerance
    assert OS.rel_fro_error(Yd, ref) <= 1e-5
