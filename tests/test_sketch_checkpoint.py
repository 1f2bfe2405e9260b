"""Checkpoint of the learned sketch (save_sketch / load_sketch / restore_adam)
and persistence of the autotuner's cache, on the host (no GPU)."""
import json

import numpy as np
import pytest
import torch

from paper_2304_04612_gb300 import sketch as SK


def _train(omega, opt, steps, target):
    for _ in range(steps):
        opt.zero_grad()
        ((omega - target) ** 2 * torch.linspace(0.5, 2.0, omega.numel()).view_as(omega)).sum().backward()
        opt.step()


def test_resume_equals_uninterrupted_training(tmp_path):
    """Six Adam steps in one go and three + save + load + three give the
    same bits: weights, moments and step count all survive the file."""
    g = torch.Generator().manual_seed(3)
    w0 = torch.randn(96, 16, generator=g)
    target = torch.randn(96, 16, generator=g)
    a = w0.clone().requires_grad_(True)
    opt_a = torch.optim.Adam([a], lr=0.05)
    _train(a, opt_a, 6, target)

    b = w0.clone().requires_grad_(True)
    opt_b = torch.optim.Adam([b], lr=0.05)
    _train(b, opt_b, 3, target)
    path = str(tmp_path / "sketch.npz")
    SK.save_sketch(path, b, opt_b, step=3)
    c, step, adam = SK.load_sketch(path)
    assert step == 3 and adam is not None
    opt_c = torch.optim.Adam([c], lr=0.5)          # hyperparameters come from the file
    SK.restore_adam(opt_c, c, adam)
    _train(c, opt_c, 3, target)
    assert torch.equal(c.detach(), a.detach())


def test_checkpoint_holds_fp16_rounding_and_no_pickles(tmp_path):
    w = torch.randn(40, 8) * 1000
    path = str(tmp_path / "s.npz")
    SK.save_sketch(path, w, step=7)
    with np.load(path, allow_pickle=False) as z:
        assert z["omega_fp32"].dtype == np.float32
        h = z["omega_fp16"].view(np.float16)
        assert np.array_equal(h, z["omega_fp32"].astype(np.float16))   # RN to nearest even
    om, step, adam = SK.load_sketch(path)
    assert step == 7 and adam is None and om.requires_grad
    # a corrupted FP16 copy is refused
    with np.load(path, allow_pickle=False) as z:
        arrs = {k: z[k] for k in z.files}
    arrs["omega_fp16"] = arrs["omega_fp16"].copy()
    arrs["omega_fp16"][0, 0] ^= 1
    bad = str(tmp_path / "bad.npz")
    np.savez(bad, **arrs)
    with pytest.raises(ValueError):
        SK.load_sketch(bad)


def test_autotune_cache_round_trip(tmp_path):
    """Records written to JSON with the GPU's name and SM count come back on
    the same kind of GPU, are ignored on another, and malformed records are
    refused without touching the cache."""
    import paper_2304_04612_gb300 as shg
    shg.shg_autotune_clear()
    e = {"a_layout": 0, "b_mode": 0, "pieces": 2, "n_tile": 128, "n_tiles": 2, "m_log2": 14, "k_log2": 14,
         "k_pieces": 0, "a_stages": 4, "b_stages": 3, "drain_kblocks": 8, "n_groups": 1, "wide": 1, "pair": 1, "whole_tiles": 0}
    assert shg.shg_autotune_import([e]) == 1
    assert shg.shg_autotune_import([e]) == 0                # the class is cached already
    assert shg.shg_autotune_export() == [e]
    cfg = shg.shg_autotune_lookup(16384, 16384, 256)
    assert cfg["cached"] and cfg["pair"] and (cfg["a_stages"], cfg["b_stages"], cfg["drain_kblocks"]) == (4, 3, 8)
    path = str(tmp_path / "tune.json")
    assert shg.save_autotune(path, gpu_name="GPU X", sm_count=152) == 1
    assert json.load(open(path))["gpu"] == "GPU X"
    shg.shg_autotune_clear()
    assert shg.load_autotune(path, gpu_name="GPU Y", sm_count=152) == 0
    assert shg.load_autotune(path, gpu_name="GPU X", sm_count=148) == 0
    assert shg.load_autotune(path, gpu_name="GPU X", sm_count=152) == 1
    assert shg.shg_autotune_export() == [e]
    shg.shg_autotune_clear()
    with pytest.raises(RuntimeError):
        shg.shg_autotune_import([dict(e, a_stages=9)])
    assert shg.shg_autotune_export() == []


def test_tune_record_size_matches_header():
    import os
    import re
    import paper_2304_04612_gb300 as shg
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "shg.h")).read()
    n = int(re.search(r"#define SHG_TUNE_RECORD (\d+)", hdr).group(1))
    assert n == shg.TUNE_RECORD == len(shg._TUNE_FIELDS)
