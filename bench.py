"""Benchmark of the SHGEMM random projection on GB300 (one JSON line on stdout).

Workload (one step): the SHGEMM sweep Y_k = A * Omega_k at m = n = 16384,
k in {64, 128, 256, 512}; A i.i.d. U[-1, 1] FP32 (seed 2, 1 GiB, larger than
L2), Omega N(0,1) FP16 16384 x 512 (seed 1), Omega_k its first k columns.
value = sum of 2 m n k over the step / step time (TFLOP/s, the paper's
2mnk/t convention).

Also reported (outside the timed steps): the FP32 SIMT path and the BF16x3
split on the same sweep, sampled-row errors against the FP64 oracle, the
4096^2 / 8192^2 points (L2 flushed between repetitions), the randomized SVD
of the 1024^2 planted matrix and RP-HOSVD of the 512^3 Tucker tensor with
the SHGEMM path vs the FP32 path, the roofline of the dominant kernel, the
end-to-end number through host buffers and the oracle's CPU time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--quick]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RSVD/RP-HOSVD time & SHGEMM TFLOP/s vs FP32 path, same GB300, matched error"
KS = (64, 128, 256, 512)
M = N = 16384

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one SHGEMM-FP16
# launch at m = n = 16384, from one-pass ncu captures of
# `bench.py --case 16384 K` (128-column tiles for k = 64, 128; 256-column tiles
# for k = 256, 512), with the SHA-256 of the kernel sources they apply to;
# reported only while the sources are unchanged.
TRAFFIC = {
    "sources": ["paper_2304_04612_gb300/csrc/shgemm_tc.cu", "paper_2304_04612_gb300/csrc/ptx.cuh",
                "paper_2304_04612_gb300/csrc/tc_common.cuh", "paper_2304_04612_gb300/csrc/shgemm_pair.cuh"],
    "sha256": "a5e71337b5ca2ddfe8df7df7a70095e8e4f538e739edc6c9a96a38a36409ef7b",
    "bytes_per_launch": {"64": 1092125440, "128": 1109030912, "256": 1151876096, "512": 1171567616},
}


def kernel_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "_fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return summarize_clocks(self.lines)


def summarize_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen active
    in nvidia-smi CSV lines of ClockSampler.Q (lines that do not parse are
    skipped)."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest of the ranks' values (a MAX all-reduce over the process
    group); a single rank's own value."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flop_per_step: float, steps: int, ws: int, ms_total: float) -> float:
    """Rate of ws replicas that each ran `steps` steps of `flop_per_step`,
    over the slowest replica's time."""
    return flop_per_step * steps * ws / (ms_total * 1e-3) / 1e12


def oracle_rate(A_host, Om_host, budget_s=10.0, ks=KS):
    """Oracle (FP64 CPU) throughput on a bounded row sample of the sweep."""
    from oracle import shgemm as OS
    rows, flops, t0 = 0, 0.0, time.perf_counter()
    step = 512
    while time.perf_counter() - t0 < budget_s and rows < A_host.shape[0]:
        blk = A_host[rows:rows + step]
        for k in ks:
            OS.project_exact(blk, Om_host[:, :k])
            flops += 2.0 * blk.shape[0] * A_host.shape[1] * k
        rows += blk.shape[0]
    dt = time.perf_counter() - t0
    return flops / dt / 1e12, rows, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from synth import omega_f16
    rng = np.random.default_rng(2)
    rows = 1024
    A = rng.uniform(-1.0, 1.0, size=(rows, N)).astype(np.float32)   # rows of the same U[-1,1] matrix
    Om = omega_f16(N, max(KS), seed=1)
    for _ in range(args.warmup):
        oracle_rate(A[:256], Om, budget_s=0.0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rate, r, dt = oracle_rate(A, Om, budget_s=1e9)
        times.append(time.perf_counter() - t0)
    flops = 2.0 * rows * N * sum(KS)
    value = flops * len(times) / sum(times) / 1e12
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "shgemm_sweep m=n=16384 k=64,128,256,512 (oracle: 1024-row sample)",
                       "sample_rows": rows},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"rows 0..{rows} of A (U[-1,1], 16384 cols) times Omega_k, all four k"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the side measurements")
    ap.add_argument("--case", type=int, nargs=2, metavar=("MN", "K"),
                    help="profiling case: only W + K launches of one m=n=MN, k=K SHGEMM (no JSON contract line)")
    ap.add_argument("--variant", default="f16", help="variant for --case")
    ap.add_argument("--factor", choices=["rsvd", "hosvd", "rsvd4096", "batched"],
                    help="profiling case: W + K calls of the randomized SVD of the 1024^2 planted matrix, "
                         "of the 4096^2 p = 256 matrix, of RP-HOSVD of the 512^3 Tucker tensor or of the "
                         "256-problem batched randomized SVD on the stream pool (no JSON contract line)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.case:
        run_case(args)
        return
    if args.factor:
        run_factor(args)
        return

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as shg
    from synth import omega_f16
    from oracle import shgemm as OS

    pk = peaks()
    dev = torch.device("cuda", local)
    # ---------------------------------------------------------------- inputs
    rng = np.random.default_rng(2)
    A_host = rng.uniform(-1.0, 1.0, size=(M, N)).astype(np.float32)
    Om_host = omega_f16(N, max(KS), seed=1)
    A = torch.from_numpy(A_host).to(dev)
    Om = torch.from_numpy(Om_host).to(dev)
    Ys = {k: torch.empty(M, k, dtype=torch.float32, device=dev) for k in KS}
    flags = shg.new_flags(dev)
    stream = torch.cuda.current_stream(dev)

    def step(variant="f16", events=None):
        for k in KS:
            if events is not None:
                events[k][0].record(stream)
            shg.shgemm_project(A, Om[:, :k], variant, out=Ys[k], flags=flags, check=False, stream=stream)
            if events is not None:
                events[k][1].record(stream)

    # launch configuration per shape class, timed once before the warm-up
    tuned = {str(k): shg.shg_autotune_project(A, Om[:, :k], "f16", reps=3, out=Ys[k], flags=flags, stream=stream)
             for k in KS}
    # whether each class kept stream-K ranges or whole output tiles per CTA
    # (a class's N tiling: n_tile x n_tiles = k for these k)
    for e in shg.shg_autotune_export():
        if e["a_layout"] == 0 and e["b_mode"] == 0 and str(e["n_tile"] * e["n_tiles"]) in tuned:
            tuned[str(e["n_tile"] * e["n_tiles"])]["whole_tiles"] = bool(e["whole_tiles"])
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    shg.check_flags(flags, "warmup")

    ev = {k: [] for k in KS}
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        e = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in KS}
        step(events=e)
        for k in KS:
            ev[k].append(e[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms_total = max_over_ranks(t0.elapsed_time(t1), ws, dev)
    clk = clocks.stop()
    ms_step = ms_total / args.steps
    flop_step = sum(2.0 * M * N * k for k in KS)
    value = whole_job_tflops(flop_step, args.steps, ws, ms_total)
    per_k_ms = {k: float(np.mean([a.elapsed_time(b) for a, b in ev[k]])) for k in KS}
    shg.check_flags(flags, "timed steps")

    # -------------------------------------------------------------- roofline
    bw = pk["hbm_gbs"] * 1e9
    tc = pk["bf16_tflops"] * 1e12
    roof = {}
    for k in KS:
        byts = 4.0 * M * N + 2.0 * N * k + 4.0 * M * k
        fl = 4.0 * M * N * k
        t = per_k_ms[k] * 1e-3
        floor = max(byts / bw, fl / tc)
        roof[k] = {"ms": per_k_ms[k], "tflops_2mnk": 2.0 * M * N * k / t / 1e12,
                   "achieved_gbs": byts / t / 1e9, "tensor_tflops_4mnk": fl / t / 1e12,
                   "bound": "hbm" if byts / bw >= fl / tc else "tensor", "frac_of_floor": floor / t}
    # the dominant launch: the largest share of the step
    k0 = max(KS, key=lambda k: per_k_ms[k])
    b0 = 4.0 * M * N + 2.0 * N * k0 + 4.0 * M * k0
    f0 = 4.0 * M * N * k0
    t0s = per_k_ms[k0] * 1e-3
    traffic = None
    if TRAFFIC["sha256"] is not None and kernel_sha() == TRAFFIC["sha256"]:
        traffic = TRAFFIC["bytes_per_launch"].get(str(k0))
    src = "MEASURED_PEAKS.json" if "_fallback" not in pk else "fallback"
    if roof[k0]["bound"] == "hbm":
        roofline = {"bound": "hbm", "achieved": b0 / t0s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": b0 / t0s / 1e9 / pk["hbm_gbs"], "traffic": traffic,
                    "peak_source": f"{src} hbm_gbs (burst copy)"}
    else:
        roofline = {"bound": "tensor", "achieved": f0 / t0s / 1e12, "peak": pk["bf16_tflops"],
                    "unit": "TFLOP/s", "frac": f0 / t0s / 1e12 / pk["bf16_tflops"], "traffic": traffic,
                    "peak_source": f"{src} bf16_tflops (burst; FP16 and BF16 dense rates are equal)"}
        if pk.get("bf16_tflops_sustained"):
            roofline["frac_of_sustained"] = f0 / t0s / 1e12 / pk["bf16_tflops_sustained"]
    roofline.update({
        "kernel": (f"tc_wide_kernel (SHGEMM-FP16, 256-column tiles), m=n={M}, k={k0}" if tuned[str(k0)].get("wide")
                   else f"tc_gemm_kernel<K-major A, FP16 Omega> (SHGEMM-FP16, 128-column tiles), m=n={M}, k={k0}"),
        "share_of_step": per_k_ms[k0] / sum(per_k_ms.values()),
        "algorithmic": {"bytes": b0, "tensor_flops_4mnk": f0},
        "per_k": {str(k): roof[k] for k in KS}})

    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16x2-split/f32-acc", "data": "synthetic",
            "config": {"workload": "shgemm_sweep m=n=16384 k=64,128,256,512 (SHGEMM-FP16, tcgen05)",
                       "A": "16384x16384 FP32 U[-1,1] seed 2", "omega": "16384x512 FP16 N(0,1) seed 1",
                       "l2": "inputs larger than L2 (A = 1 GiB per projection)",
                       "autotuned": tuned,
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "gpu_launches": len(KS) * args.steps, "clocks": clk, "roofline": roofline}

    if rank == 0 and not args.quick:
        side = side_measurements(shg, OS, torch, dev, A, A_host, Om, Om_host, Ys, flags, stream, pk,
                                 clk_mhz=clk.get("sm_mhz"))
        line.update(side)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def paper_rsvd_inputs(torch, dev):
    """The randomized-SVD shape of the paper's throughput study (Sec. 5.1):
    N = 4096, p = 256, s = 10, A_exp-like spectrum sigma_i = 2^(-i a) with
    sigma_p = 1e-3.  Built as Q1 diag(sigma) Q2^T with Q1, Q2 orthonormal bases
    of seeded Gaussians (512 leading singular values; input generation only)."""
    from synth import omega_f16
    N, p, s = 4096, 256, 10
    k = p + s
    rng = np.random.default_rng(7)
    r = 512
    sig = 2.0 ** (-np.arange(1, r + 1) * (np.log2(1e3) / p))
    q1 = np.linalg.qr(rng.standard_normal((N, r)))[0]
    q2 = np.linalg.qr(rng.standard_normal((N, r)))[0]
    A = torch.from_numpy(((q1 * sig) @ q2.T).astype(np.float32)).to(dev)
    ldo = (k + 7) // 8 * 8
    Om = torch.zeros(N, ldo, dtype=torch.float16, device=dev)
    Om[:, :k] = torch.from_numpy(omega_f16(N, k, seed=1)).to(dev)
    return A, Om[:, :k], p, s


def run_factor(args):
    """One factorization workload, for ncu launch lists: W warm-up calls then K timed ones."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as shg
    from synth import rsvd_planted, tucker, hosvd_omegas
    dev = torch.device("cuda", 0)
    fl = shg.new_flags(dev)
    if args.factor == "rsvd4096":
        A, Om, p, s_ = paper_rsvd_inputs(torch, dev)
        ws = torch.empty(shg.rsvd_workspace_size(4096, 4096, p, s_, 0), dtype=torch.uint8, device=dev)
        fn = lambda: shg.shg_rsvd(A, Om, p, s_, 0, args.variant, workspace=ws, flags=fl, check=False)
    elif args.factor == "rsvd":
        A_h, Om_h = rsvd_planted(1024, 1024, rate=8.0, seed_a=0, seed_omega=1, k=64)
        A, Om = torch.from_numpy(A_h).to(dev), torch.from_numpy(Om_h).to(dev)
        ws = torch.empty(shg.rsvd_workspace_size(1024, 1024, 32, 32, 0), dtype=torch.uint8, device=dev)
        fn = lambda: shg.shg_rsvd(A, Om, 32, 32, 0, args.variant, workspace=ws, flags=fl, check=False)
    elif args.factor == "batched":
        As, ranks, s_, q_, ws, out = batched_problems(shg, torch, dev, dct_bases=True)
        # the grouped launches in lanes, enqueued directly (no graph)
        fn = lambda: shg.shg_rsvd_batched(As, ranks, s_, q_, omegas=None, seed=4, use_graph=False, out=out,
                                          workspace=ws, flags=fl, check=False)
    else:
        dims, J = (512, 512, 512), (48, 48, 48)
        X_h, _, _ = tucker(dims, (32, 32, 32), seed=3, noise_std=1e-4)
        X = torch.from_numpy(X_h).to(dev)
        oms = [torch.from_numpy(o).to(dev) for o in hosvd_omegas(dims, J, seed=3)]
        fn = lambda: shg.shg_rp_hosvd(X, oms, J, args.variant, flags=fl, check=False)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    shg.check_flags(fl, args.factor)
    print(json.dumps({"factor": args.factor, "variant": args.variant, "ms": a.elapsed_time(b) / args.steps}))


def run_case(args):
    """A single SHGEMM shape, for ncu captures: W warm-up launches then K timed ones."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2304_04612_gb300 as shg
    mn, k = args.case
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev).manual_seed(2)
    A = torch.rand(mn, mn, device=dev, generator=gen) * 2 - 1
    Om = torch.randn(mn, k, device=dev, generator=gen).half()
    if args.variant.startswith("bf16"):
        Om = Om.bfloat16()
    Y = torch.empty(mn, k, device=dev)
    fl = shg.new_flags(dev)
    for _ in range(args.warmup):
        shg.shgemm_project(A, Om, args.variant, out=Y, flags=fl, check=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        shg.shgemm_project(A, Om, args.variant, out=Y, flags=fl, check=False)
    b.record()
    torch.cuda.synchronize()
    shg.check_flags(fl, "case")
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"case": [mn, k], "variant": args.variant, "ms": ms,
                      "tflops_2mnk": 2.0 * mn * mn * k / (ms * 1e-3) / 1e12,
                      "gbs": (4.0 * mn * mn + 2.0 * mn * k + 4.0 * mn * k) / (ms * 1e-3) / 1e9}))


def time_ms(torch, stream, fn, reps=5, flush=None):
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def side_measurements(shg, OS, torch, dev, A, A_host, Om, Om_host, Ys, flags, stream, pk, clk_mhz=None):
    out = {}
    flush_buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def flush():
        flush_buf.zero_()

    # FP32 SIMT path and BF16x3 on the same sweep
    from oracle.lowp import encode_bf16
    cmp = {}
    Omb = torch.from_numpy(encode_bf16(OS.bf16_omega(Om_host)).view(np.int16)).to(dev).view(torch.bfloat16)
    for variant, om in (("fp32", Om), ("bf16x3", Omb), ("tf32", Om), ("f16", Om)):
        per = {}
        for k in KS:
            reps = 2 if variant == "fp32" else 5
            ms = time_ms(torch, stream, lambda: shg.shgemm_project(A, om[:, :k], variant, out=Ys[k], flags=flags,
                                                                    check=False, stream=stream), reps=reps)
            per[str(k)] = {"ms": ms, "tflops_2mnk": 2.0 * M * N * k / (ms * 1e-3) / 1e12}
        cmp[variant] = per
    out["sweep_16384"] = cmp
    out["speedup_vs_fp32_simt"] = {str(k): cmp["fp32"][str(k)]["ms"] / cmp["f16"][str(k)]["ms"] for k in KS}
    # SHGEMM-TF32 (full exponent range) against its own floor: A's bytes at the
    # measured HBM rate or 4mnk at half the FP16 tensor rate (TF32 runs at half)
    tf = {}
    for k in KS:
        t = cmp["tf32"][str(k)]["ms"] * 1e-3
        byts = 4.0 * M * N + 2.0 * N * k + 4.0 * M * k
        floor = max(byts / (pk["hbm_gbs"] * 1e9), 4.0 * M * N * k / (0.5 * pk["bf16_tflops"] * 1e12))
        tf[str(k)] = {"frac_of_floor": floor / t,
                      "bound": "hbm" if byts / (pk["hbm_gbs"] * 1e9) >= 4.0 * M * N * k / (0.5 * pk["bf16_tflops"] * 1e12)
                      else "tensor (TF32 = half the FP16 rate)"}
    out["tf32_roofline"] = tf
    # the FP32 SIMT path against the FFMA peak: 128 FP32 FMA per clock per SM
    # (4 sub-partitions x 32 lanes) x 2 flop x SMs x the SM clock under load
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk_mhz if clk_mhz else pk.get("sm_max_mhz", 2070.0)
    ffma_peak = 128 * 2 * sms * mhz * 1e6 / 1e12
    out["fp32_simt_roofline"] = {"bound": "alu", "peak": ffma_peak, "unit": "TFLOP/s",
                                 "peak_derivation": f"128 FFMA/clk/SM x 2 x {sms} SMs x {mhz:.0f} MHz",
                                 "per_k": {str(k): {"achieved": cmp["fp32"][str(k)]["tflops_2mnk"],
                                                    "frac": cmp["fp32"][str(k)]["tflops_2mnk"] / ffma_peak}
                                           for k in KS}}

    # context only (a library GEMM, not on the path): cuBLAS SGEMM of the same
    # product with FP32 inputs (Omega widened exactly), TF32 off, beside the
    # project's FP32 SIMT path
    tf32_was = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    ctx = {}
    try:
        Omf = Om.float()
        for k in KS:
            Bk = Omf[:, :k].contiguous()
            torch.matmul(A, Bk, out=Ys[k])  # library set-up outside the timing
            ms = time_ms(torch, stream, lambda: torch.matmul(A, Bk, out=Ys[k]), reps=3)
            ctx[str(k)] = {"ms": ms, "tflops_2mnk": 2.0 * M * N * k / (ms * 1e-3) / 1e12,
                           "shgemm_speedup": ms / cmp["f16"][str(k)]["ms"]}
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32_was
    out["context_cublas_sgemm"] = ctx

    # sampled-row error vs the FP64 oracle (same inputs), per variant
    rows = np.random.default_rng(0).choice(M, 128, replace=False)
    errs = {}
    for variant, om in (("f16", Om), ("fp32", Om), ("bf16x3", Omb), ("tf32", Om)):
        e = {}
        for k in KS:
            Y = shg.shgemm_project(A, om[:, :k], variant, out=Ys[k], flags=flags, check=True, stream=stream)
            ref = OS.project_exact(A_host[rows], Om_host[:, :k]) if variant != "bf16x3" else \
                A_host[rows].astype(np.float64) @ OS.bf16_omega(Om_host[:, :k])
            e[str(k)] = OS.rel_fro_error(Y[rows].cpu().numpy(), ref)
        errs[variant] = e
    out["rel_err_sampled_rows"] = errs

    # smaller square sizes, L2 flushed before each repetition
    small = {}
    for mm in (4096, 8192):
        As = A[:mm, :mm]
        per = {}
        for variant in ("f16", "fp32"):
            for k in KS:
                ms = time_ms(torch, stream, lambda: shg.shgemm_project(As, Om[:mm, :k], variant, out=Ys[k][:mm],
                                                                        flags=flags, check=False, stream=stream),
                             reps=3 if variant == "fp32" else 5, flush=flush)
                per[f"{variant}_k{k}"] = {"ms": ms, "tflops_2mnk": 2.0 * mm * mm * k / (ms * 1e-3) / 1e12}
        small[str(mm)] = per
    out["sweep_small"] = small

    # end to end through host buffers: H2D of A and Omega, the sweep, D2H of Y.
    # A crosses in row blocks on four copy streams; the four projections of a
    # block start as soon as its copy has landed and its rows of every Y go
    # back on a fifth stream, so the copies of later blocks overlap the
    # projections of earlier ones.
    A_pin = torch.from_numpy(A_host).pin_memory()
    Om_pin = torch.from_numpy(Om_host).pin_memory()
    Yh = {k: torch.empty(M, k, dtype=torch.float32).pin_memory() for k in KS}
    nblk, ncs = 8, 4
    rows_per = M // nblk
    cstreams = [torch.cuda.Stream(dev) for _ in range(ncs)]
    dstream = torch.cuda.Stream(dev)

    def e2e_step():
        with torch.cuda.stream(cstreams[0]):
            Om.copy_(Om_pin, non_blocking=True)
        om_ready = torch.cuda.Event()
        om_ready.record(cstreams[0])
        stream.wait_event(om_ready)
        for b in range(nblk):
            r0, r1 = b * rows_per, (b + 1) * rows_per
            cs = cstreams[b % ncs]
            with torch.cuda.stream(cs):
                A[r0:r1].copy_(A_pin[r0:r1], non_blocking=True)
            landed = torch.cuda.Event()
            landed.record(cs)
            stream.wait_event(landed)
            for k in KS:
                shg.shgemm_project(A[r0:r1], Om[:, :k], "f16", out=Ys[k][r0:r1], flags=flags, check=False,
                                   stream=stream)
            done = torch.cuda.Event()
            done.record(stream)
            dstream.wait_event(done)
            with torch.cuda.stream(dstream):
                for k in KS:
                    Yh[k][r0:r1].copy_(Ys[k][r0:r1], non_blocking=True)
        back = torch.cuda.Event()
        back.record(dstream)
        stream.wait_event(back)
    # the host link's own rate: one whole-A copy from the same pinned buffer
    link_ms = time_ms(torch, stream, lambda: A.copy_(A_pin, non_blocking=True), reps=5)
    e2e_step()
    torch.cuda.synchronize()
    ms = time_ms(torch, stream, e2e_step, reps=10)
    shg.check_flags(flags, "e2e")
    ok_rows = np.random.default_rng(1).choice(M, 16, replace=False)
    e2e_err = OS.rel_fro_error(Yh[512][ok_rows].numpy(), OS.project_exact(A_host[ok_rows], Om_host))
    h2d = A_host.nbytes + Om_host.nbytes
    d2h = sum(M * k * 4 for k in KS)
    out["e2e"] = {"value": sum(2.0 * M * N * k for k in KS) / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                  "ms_per_step": ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                  "h2d_gbs_if_copy_bound": h2d / (ms * 1e-3) / 1e9, "reps": 10,
                  "h2d_link_gbs": A_host.nbytes / (link_ms * 1e-3) / 1e9,
                  "fraction_of_copy_floor": (h2d / (A_host.nbytes / (link_ms * 1e-3))) / (ms * 1e-3),
                  "pipeline": f"A in {nblk} row blocks on {ncs} copy streams, projections per block, Y rows "
                              "back on a fifth stream",
                  "check_rel_err_sampled_rows_k512": e2e_err}

    # randomized SVD of the planted 1024^2 matrix and RP-HOSVD of the 512^3 tensor
    out["rsvd_1024"] = rsvd_times(shg, torch, dev, stream)
    out["rp_hosvd_512"] = hosvd_times(shg, torch, dev, stream)
    out["rsvd_batched_256"] = batched_times(shg, torch, dev, stream)
    out["rsvd_4096_p256"] = rsvd4096_times(shg, torch, dev, stream)
    out["rsvd_16384_k64"] = rsvd16384_times(shg, torch, dev, stream)
    out["learned_sketch_2048"] = sketch_times(shg, torch, dev, stream)

    # CPU baseline: the oracle on a bounded row sample of the same sweep
    rate, rows_done, dt = oracle_rate(A_host, Om_host, budget_s=10.0)
    out["cpu_baseline"] = {"value": rate, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                           "sample": f"first {rows_done} rows of A times Omega_k for all four k ({dt:.1f} s, "
                                     "numpy float64)"}
    return out


def rsvd_times(shg, torch, dev, stream):
    from synth import rsvd_planted
    from oracle import rsvd as OR
    A_h, Om_h = rsvd_planted(1024, 1024, rate=8.0, seed_a=0, seed_omega=1, k=64)
    A = torch.from_numpy(A_h).to(dev)
    Om = torch.from_numpy(Om_h).to(dev)
    ws = torch.empty(shg.rsvd_workspace_size(1024, 1024, 32, 32, 0), dtype=torch.uint8, device=dev)
    fl = shg.new_flags(dev)
    res = {}
    ref = OR.rsvd(A_h, Om_h, p=32)
    for v in ("f16", "fp32"):
        outs = (torch.empty(1024, 32, device=dev), torch.empty(32, device=dev), torch.empty(1024, 32, device=dev),
                None)
        fn = lambda: shg.shg_rsvd(A, Om, 32, 32, 0, v, workspace=ws, out=outs, flags=fl, check=False, stream=stream)
        fn()
        ms = time_ms(torch, stream, fn, reps=10)
        U, S, V = (t.cpu().numpy().astype(np.float64) for t in outs[:3])
        A64 = A_h.astype(np.float64)
        r_p = np.linalg.norm(A64 - (U * S) @ V.T) / np.linalg.norm(A64)
        res[v] = {"ms": ms, "sigma_max_rel_err": float(np.max(np.abs(S - ref["S"]) / ref["S"])),
                  "residual": float(r_p), "oracle_residual": ref["r_p"]}
    res["speedup_f16_vs_fp32"] = res["fp32"]["ms"] / res["f16"]["ms"]
    return res


def rsvd4096_times(shg, torch, dev, stream):
    """Randomized SVD in the paper's throughput configuration (Sec. 5.1): N = 4096,
    p = 256, s = 10, SHGEMM path vs FP32 path; residual ||A - U S V^T||_F / ||A||_F
    (torch on the GPU, outside the timed calls) against the planted tail."""
    A, Om, p, s = paper_rsvd_inputs(torch, dev)
    N = A.shape[0]
    ws = torch.empty(shg.rsvd_workspace_size(N, N, p, s, 0), dtype=torch.uint8, device=dev)
    fl = shg.new_flags(dev)
    res = {"config": "A 4096x4096 FP32, sigma_i = 2^(-i log2(1e3) / 256) (512 planted), p = 256, s = 10, q = 0"}
    for v in ("f16", "fp32"):
        outs = (torch.empty(N, p, device=dev), torch.empty(p, device=dev), torch.empty(N, p, device=dev), None)
        fn = lambda: shg.shg_rsvd(A, Om, p, s, 0, v, workspace=ws, out=outs, flags=fl, check=False, stream=stream)
        fn()
        ms = time_ms(torch, stream, fn, reps=5)
        U, S, V = outs[:3]
        r = torch.linalg.norm(A - (U * S) @ V.T) / torch.linalg.norm(A)
        res[v] = {"ms": ms, "residual": float(r)}
    shg.check_flags(fl, "rsvd_4096")
    res["speedup_f16_vs_fp32"] = res["fp32"]["ms"] / res["f16"]["ms"]
    sig = 2.0 ** (-np.arange(1, 513) * (np.log2(1e3) / p))
    res["optimal_residual"] = float(np.sqrt(np.sum(sig[p:] ** 2) / np.sum(sig ** 2)))
    res["l2"] = "A (64 MiB) stays in L2 between calls; the k x k steps dominate"
    return res


def rsvd16384_times(shg, torch, dev, stream):
    """Randomized SVD where the passes over A dominate: A 16384 x 16384 FP32
    (1 GiB, larger than L2) = U diag(sigma) V^T with sigma_i = 2^(-i/8) on 512
    planted directions (U, V orthonormal Q factors of seeded Gaussians, built on
    the GPU outside the timed calls), rank 32, oversampling 32 (k = 64), q = 0
    and q = 1; SHGEMM path vs FP32 path, residual ||A - U S V^T||_F / ||A||_F
    against the optimal rank-32 residual of the planted spectrum."""
    N, r, p, s = 16384, 512, 32, 32
    g = torch.Generator(device=dev).manual_seed(6)
    U0 = torch.linalg.qr(torch.randn(N, r, device=dev, generator=g))[0]
    V0 = torch.linalg.qr(torch.randn(N, r, device=dev, generator=g))[0]
    sig = torch.pow(2.0, -torch.arange(1, r + 1, device=dev, dtype=torch.float32) / 8.0)
    A = ((U0 * sig) @ V0.T).contiguous()
    del U0, V0
    Om = torch.randn(N, p + s, device=dev, generator=g).half()
    nA = torch.linalg.norm(A)
    fl = shg.new_flags(dev)
    sig_h = 2.0 ** (-np.arange(1, r + 1) / 8.0)
    res = {"config": "A 16384x16384 FP32, sigma_i = 2^(-i/8) (512 planted), rank 32, s = 32",
           "optimal_residual": float(np.sqrt(np.sum(sig_h[p:] ** 2) / np.sum(sig_h ** 2)))}
    for q in (0, 1):
        ws = torch.empty(shg.rsvd_workspace_size(N, N, p, s, q), dtype=torch.uint8, device=dev)
        row = {}
        for v in ("f16", "fp32"):
            outs = (torch.empty(N, p, device=dev), torch.empty(p, device=dev), torch.empty(N, p, device=dev), None)
            fn = lambda: shg.shg_rsvd(A, Om, p, s, q, v, workspace=ws, out=outs, flags=fl, check=False,
                                      stream=stream)
            fn()
            ms = time_ms(torch, stream, fn, reps=5)
            U, S, V = outs[:3]
            row[v] = {"ms": ms, "residual": float(torch.linalg.norm(A - (U * S) @ V.T) / nA)}
        row["speedup_f16_vs_fp32"] = row["fp32"]["ms"] / row["f16"]["ms"]
        res[f"q{q}"] = row
        del ws
    shg.check_flags(fl, "rsvd_16384")
    return res


def sketch_times(shg, torch, dev, stream, n_train=4096, n_test=512, k=96):
    """Learned FP16 sketch for the 2048 x 2048 family A = U diag(sigma) (V0 cos T +
    W sin T)^T + E (r = 64, sigma_j = 2^(-j/8), theta_j ~ U[0, 0.2], ||E|| = 1e-3
    ||signal||): Omega (FP32 master, 2048 x 96) trained with Adam through SketchFn
    (the library's SHGEMM projection and loss / gradient kernels) on n_train
    generated matrices, one pass, batch 1; then the mean test loss
    ||A - QQ^T A||_F^2 / ||A||_F^2 on n_test fresh matrices against a Gaussian
    Omega of the same k, and the estimator's choice (choose_sketch, 16 probes)
    on the first 64 test matrices.  The matrices are generated on the GPU from
    seeded Gaussians in batches of 16 (input generation, not timed)."""
    from paper_2304_04612_gb300.sketch import SketchFn, choose_sketch
    n, r = 2048, 64
    g = torch.Generator(device=dev).manual_seed(5)
    V0 = torch.linalg.qr(torch.randn(n, r, device=dev, generator=g))[0]
    sig = torch.pow(2.0, -torch.arange(1, r + 1, device=dev, dtype=torch.float32) / 8.0)

    def family(count):
        U = torch.linalg.qr(torch.randn(count, n, r, device=dev, generator=g))[0]
        W = torch.randn(count, n, r, device=dev, generator=g)
        W = torch.linalg.qr(W - V0 @ (V0.T @ W))[0]
        th = torch.rand(count, 1, r, device=dev, generator=g) * 0.2
        S = (U * sig) @ (V0 * torch.cos(th) + W * torch.sin(th)).transpose(1, 2)
        E = torch.randn(count, n, n, device=dev, generator=g)
        E *= (1e-3 * torch.linalg.norm(S, dim=(1, 2)) / torch.linalg.norm(E, dim=(1, 2)))[:, None, None]
        return (S + E).contiguous()

    omega = torch.randn(n, k, device=dev, generator=g).requires_grad_(True)
    gauss = omega.detach().clone()
    opt = torch.optim.Adam([omega], lr=0.01)
    step_ms = []
    for b in range(n_train // 16):
        As = family(16)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for A in As:
            opt.zero_grad()
            SketchFn.apply(A, omega).backward()
            opt.step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1) / 16)
    learned, base, better, used = [], [], 0, 0
    with torch.no_grad():
        for b in range(n_test // 16):
            As = family(16)
            for j, A in enumerate(As):
                ll = SketchFn.apply(A, omega.detach()).item()
                lg = SketchFn.apply(A, gauss).item()
                learned.append(ll)
                base.append(lg)
                better += ll < lg
                if b * 16 + j < 64:
                    used += bool(choose_sketch(A, omega.detach(), seed=1000 + b * 16 + j, probes=16)[3])
    return {"n": n, "k": k, "train_matrices": n_train, "test_matrices": n_test,
            "train_step_ms": float(np.median(step_ms)),
            "test_loss_learned": float(np.mean(learned)), "test_loss_gaussian": float(np.mean(base)),
            "loss_ratio_learned_over_gaussian": float(np.mean(learned) / np.mean(base)),
            "learned_better_fraction": better / len(learned),
            "estimator_keeps_learned_of_64": used}


def batched_problems(shg, torch, dev, dct_bases=False):
    """256 uneven randomized SVDs (m in [256, 4096], n in [256, 2048], rank in
    {16, 32, 64, 128}, s = 16, q = 1, sigma_i = 2^(-i/rate), rate in [8, 64]).
    The matrices are Q1 diag(sigma) Q2^T with Q1, Q2 orthonormal bases of 256
    columns (the spectrum beyond 256 is below 2^-4 at the slowest decay and is
    dropped): by default the Q factors of seeded Gaussians, built on the GPU;
    with dct_bases, randomly chosen and signed columns of the orthonormal
    DCT-II matrix, built on the host (no torch.linalg, whose lazily loaded
    library does not load under the profiler).  Input generation only,
    outside every timed region.  Returns the matrices, ranks, s, q, a
    workspace and the output tensors."""
    from synth import batch_specs
    specs = batch_specs(256, seed=4)
    g = torch.Generator(device=dev).manual_seed(4)
    rng = np.random.default_rng(4)

    def dct_basis(m, r):
        from scipy.fft import dct
        E = np.zeros((m, r), dtype=np.float32)
        E[rng.choice(m, r, replace=False), np.arange(r)] = 1.0
        Q = dct(E, axis=0, norm="ortho").astype(np.float32)
        return Q * rng.choice(np.array([-1.0, 1.0], dtype=np.float32), size=(m, 1))

    As, ranks = [], []
    for sp in specs:
        m, n = sp["m"], sp["n"]
        r = min(m, n, 256)
        ld = (n + 3) // 4 * 4
        buf = torch.zeros(m, ld, device=dev)
        if dct_bases:
            sig = (2.0 ** (-np.arange(1, r + 1) / sp["rate"])).astype(np.float32)
            buf[:, :n] = torch.from_numpy((dct_basis(m, r) * sig) @ dct_basis(n, r).T).to(dev)
        else:
            sig = torch.pow(2.0, -torch.arange(1, r + 1, device=dev, dtype=torch.float32) / sp["rate"])
            q1 = torch.linalg.qr(torch.randn(m, r, device=dev, generator=g))[0]
            q2 = torch.linalg.qr(torch.randn(n, r, device=dev, generator=g))[0]
            buf[:, :n] = (q1 * sig) @ q2.T
        As.append(buf[:, :n])
        ranks.append(sp["rank"])
    s, q = 16, 1
    ms_, ns_ = [A.shape[0] for A in As], [A.shape[1] for A in As]
    ws = torch.empty(shg.rsvd_batched_workspace_size(ms_, ns_, ranks, s, q), dtype=torch.uint8, device=dev)
    out = ([torch.empty(m, r, device=dev) for m, r in zip(ms_, ranks)], [torch.empty(r, device=dev) for r in ranks],
           [torch.empty(n, r, device=dev) for n, r in zip(ns_, ranks)])
    return As, ranks, s, q, ws, out


def batched_times(shg, torch, dev, stream):
    """The 256-problem batch of `batched_problems` as one CUDA graph, on the
    stream pool without the graph, and one problem after another."""
    As, ranks, s, q, ws, out = batched_problems(shg, torch, dev)
    ms_, ns_ = [A.shape[0] for A in As], [A.shape[1] for A in As]
    fl = shg.new_flags(dev)
    res = {"problems": 256, "bytes_of_A": int(sum(4 * m * n for m, n in zip(ms_, ns_)))}
    # grouped launches (one per step of Algorithm 1 for each lane of
    # problems of one k class, the lanes on their own streams), as a graph,
    # as a graph with all problems in one lane, and enqueued directly; then
    # the per-problem launches on the library's stream pool
    # (SHG_BATCHED_GROUPED=0), as a graph and directly
    for mode, use_graph, grouped, lanes in (("graph", True, "1", "4"), ("graph_one_lane", True, "1", "1"),
                                            ("grouped_direct", False, "1", "4"),
                                            ("stream_pool_graph", True, "0", "4"), ("streams", False, "0", "4")):
        os.environ["SHG_BATCHED_GROUPED"] = grouped
        os.environ["SHG_BATCHED_LANES"] = lanes
        fn = lambda: shg.shg_rsvd_batched(As, ranks, s, q, omegas=None, seed=4, use_graph=use_graph, out=out,
                                          workspace=ws, flags=fl, check=False, stream=stream)
        fn()
        ms = time_ms(torch, stream, fn, reps=5)
        res[mode] = {"ms": ms, "problems_per_s": 256 / (ms * 1e-3)}
    os.environ.pop("SHG_BATCHED_GROUPED", None)
    os.environ.pop("SHG_BATCHED_LANES", None)
    # the same problems one after another through shg_rsvd on one stream
    oms = [shg.shg_gaussian_f16(4, i << 32, n, r + s,
                                out=torch.empty(n, (r + s + 7) // 8 * 8, dtype=torch.float16, device=dev)[:, :r + s])
           for i, (n, r) in enumerate(zip(ns_, ranks))]
    ws1 = torch.empty(max(shg.rsvd_workspace_size(m, n, r, s, q) for m, n, r in zip(ms_, ns_, ranks)),
                      dtype=torch.uint8, device=dev)

    def seq():
        for i in range(256):
            shg.shg_rsvd(As[i], oms[i], ranks[i], s, q, "f16", workspace=ws1,
                         out=(out[0][i], out[1][i], out[2][i], None), flags=fl, check=False, stream=stream)
    seq()
    ms = time_ms(torch, stream, seq, reps=2)
    res["sequential"] = {"ms": ms, "problems_per_s": 256 / (ms * 1e-3)}
    res["device_flags"] = int(fl.item())
    return res


def hosvd_times(shg, torch, dev, stream):
    from synth import tucker, hosvd_omegas
    dims, J = (512, 512, 512), (48, 48, 48)
    A_h, _, _ = tucker(dims, (32, 32, 32), seed=3, noise_std=1e-4)
    oms_h = hosvd_omegas(dims, J, seed=3)
    X = torch.from_numpy(A_h).to(dev)
    oms = [torch.from_numpy(o).to(dev) for o in oms_h]
    ws = torch.empty(shg.rp_hosvd_workspace_size(dims, J), dtype=torch.uint8, device=dev)
    fl = shg.new_flags(dev)
    res = {}
    for v in ("f16", "fp32"):
        core = torch.empty(*J, device=dev)
        facs = [torch.empty(512, 48, device=dev) for _ in range(3)]
        fn = lambda: shg.shg_rp_hosvd(X, oms, J, v, workspace=ws, out=(core, facs), flags=fl, check=False,
                                      stream=stream)
        fn()
        shg.check_flags(fl, "rp_hosvd")
        ms = time_ms(torch, stream, fn, reps=5)
        c = core.double()
        Fs = [f.double() for f in facs]
        rec = torch.einsum("abc,ia,jb,kc->ijk", c, Fs[0], Fs[1], Fs[2])
        err = float(torch.linalg.norm(X.double() - rec) / torch.linalg.norm(X.double()))
        res[v] = {"ms": ms, "rel_err": err}
    res["speedup_f16_vs_fp32"] = res["fp32"]["ms"] / res["f16"]["ms"]
    return res


if __name__ == "__main__":
    main()
