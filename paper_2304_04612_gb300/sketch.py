"""Learned sketch: a trainable test matrix for the range finder of Algorithm 1.

The sketch Omega is kept as FP32 master weights; the projection uses its FP16
rounding, Y = A fp16(Omega) by SHGEMM, and the loss is the relative
range-finder residual ||A - Q Q^T A||_F^2 / ||A||_F^2 with Q = orth(Y).  Its
gradient with respect to the FP16 values is passed straight through to the
master weights (the rounding is treated as the identity).

``SketchFn`` is the autograd function; ``choose_sketch`` keeps a trained
sketch only when the a-posteriori residual estimate (Theorems 1 and 3) does
not exceed that of a fresh Gaussian sketch, otherwise it falls back to the
Gaussian one.  Every step runs in ``libshg.so``.
"""
from __future__ import annotations

import torch

from . import (new_flags, check_flags, shg_round_f16, shgemm_project, shg_sketch_loss_grad,
               shg_residual_estimate, shg_gaussian_f16, shg_cholqr2)


def _f16_buffer(n: int, k: int, device) -> torch.Tensor:
    """n x k FP16 view with a leading dimension rounded up to 8 (the TMA row
    stride of the projection must be a multiple of 16 bytes)."""
    ld = (k + 7) // 8 * 8
    return torch.empty(n, ld, dtype=torch.float16, device=device)[:, :k]


class SketchFn(torch.autograd.Function):
    """loss = SketchFn.apply(A, omega): A (m x n FP32, no gradient), omega
    (n x k FP32 master weights); returns the FP64 loss as a 0-d tensor."""

    @staticmethod
    def forward(ctx, A: torch.Tensor, omega: torch.Tensor) -> torch.Tensor:
        fl = new_flags(A.device)
        om16 = shg_round_f16(omega.detach(), out=_f16_buffer(*omega.shape, omega.device))
        Y = shgemm_project(A, om16, "f16", flags=fl, check=False)
        loss, grad = shg_sketch_loss_grad(A, Y, want_grad=ctx.needs_input_grad[1], flags=fl, check=False)
        check_flags(fl, "SketchFn.forward")
        ctx.save_for_backward(grad if grad is not None else torch.empty(0, device=A.device))
        return loss

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (grad,) = ctx.saved_tensors
        if grad.numel() == 0:
            return None, None
        return None, grad * g.to(grad.dtype)


def range_basis(A: torch.Tensor, omega16: torch.Tensor) -> torch.Tensor:
    """Q = CholeskyQR2(A omega16) (m x k FP32)."""
    fl = new_flags(A.device)
    Y = shgemm_project(A, omega16, "f16", flags=fl, check=False)
    shg_cholqr2(Y, flags=fl, check=False)
    check_flags(fl, "range_basis")
    return Y


def choose_sketch(A: torch.Tensor, omega_learned: torch.Tensor, seed: int, probes: int = 16,
                  probe_seed: int = 0x5EED):
    """Return (omega16, est_learned, est_gaussian, used_learned).

    The learned FP32 sketch is rounded to FP16; a Gaussian FP16 sketch of the
    same shape is drawn from ``seed``.  Both bases are scored by the same
    ``probes`` fresh FP16 Gaussian probes (stream ``probe_seed``); the learned
    sketch is kept when its estimate is not larger.
    """
    n, k = omega_learned.shape
    om_l = shg_round_f16(omega_learned.detach(), out=_f16_buffer(n, k, A.device))
    om_g = shg_gaussian_f16(seed, 0, n, k, out=_f16_buffer(n, k, A.device))
    est_l = shg_residual_estimate(A, range_basis(A, om_l), t=probes, seed=probe_seed)
    est_g = shg_residual_estimate(A, range_basis(A, om_g), t=probes, seed=probe_seed)
    el, eg = float(est_l[0].item()), float(est_g[0].item())
    use_learned = el <= eg
    return (om_l if use_learned else om_g), el, eg, use_learned


# ---------------------------------------------------------------- checkpoint
def save_sketch(path: str, omega: torch.Tensor, optimizer: torch.optim.Optimizer | None = None, step: int = 0) -> None:
    """Checkpoint of a learned sketch as an .npz file (plain arrays, no pickled
    objects): the FP32 master weights, their FP16 rounding (the sketch the
    projection uses), the training step, and, when ``optimizer`` is an Adam
    optimizer holding ``omega``, its moment estimates and step count so that
    training resumes where it stopped.  Written to a temporary file and
    renamed, so an interrupted save leaves the previous checkpoint intact."""
    import numpy as np
    import os
    w = omega.detach().to("cpu", torch.float32).contiguous()
    arrays = {"format": np.array("shg-sketch-1"), "omega_fp32": w.numpy(),
              "omega_fp16": w.half().view(torch.int16).numpy(), "step": np.array(int(step), dtype=np.int64)}
    if optimizer is not None:
        st = optimizer.state.get(omega, {})
        if st:
            group = next(g for g in optimizer.param_groups if any(p is omega for p in g["params"]))
            arrays["adam_exp_avg"] = st["exp_avg"].detach().cpu().numpy()
            arrays["adam_exp_avg_sq"] = st["exp_avg_sq"].detach().cpu().numpy()
            arrays["adam_step"] = np.array(float(st["step"]), dtype=np.float64)
            arrays["adam_hyper"] = np.array([group["lr"], group["betas"][0], group["betas"][1], group["eps"],
                                             group["weight_decay"]], dtype=np.float64)
    tmp = path + ".tmp.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path)


def load_sketch(path: str, device="cpu"):
    """Read a checkpoint written by save_sketch.  Returns (omega, step, adam):
    omega the FP32 master weights on ``device`` as a leaf tensor that requires
    a gradient, step the saved training step, adam the saved optimizer state
    (a dict) or None.  The stored FP16 copy is checked against the rounding of
    the master weights."""
    import numpy as np
    with np.load(path, allow_pickle=False) as z:
        if str(z["format"]) != "shg-sketch-1":
            raise ValueError(f"{path}: not a sketch checkpoint")
        w = torch.from_numpy(z["omega_fp32"].copy())
        if not torch.equal(w.half().view(torch.int16), torch.from_numpy(z["omega_fp16"].copy())):
            raise ValueError(f"{path}: the FP16 copy does not match the FP32 master weights")
        step = int(z["step"])
        adam = None
        if "adam_exp_avg" in z.files:
            adam = {"exp_avg": torch.from_numpy(z["adam_exp_avg"].copy()),
                    "exp_avg_sq": torch.from_numpy(z["adam_exp_avg_sq"].copy()),
                    "step": float(z["adam_step"]), "hyper": [float(x) for x in z["adam_hyper"]]}
    omega = w.to(device).requires_grad_(True)
    return omega, step, adam


def restore_adam(optimizer: torch.optim.Adam, omega: torch.Tensor, adam: dict | None) -> None:
    """Put the moment estimates and step count of a checkpoint back into an
    Adam optimizer built over ``omega`` (the tensor load_sketch returned)."""
    if adam is None:
        return
    group = next(g for g in optimizer.param_groups if any(p is omega for p in g["params"]))
    lr, b1, b2, eps, wd = adam["hyper"]
    group.update(lr=lr, betas=(b1, b2), eps=eps, weight_decay=wd)
    optimizer.state[omega] = {"step": torch.tensor(adam["step"], dtype=torch.float32),
                              "exp_avg": adam["exp_avg"].to(omega.device),
                              "exp_avg_sq": adam["exp_avg_sq"].to(omega.device)}
