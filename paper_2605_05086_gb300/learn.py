"""Training of the learned proposal network on pairs logged by the exact path.

Host orchestration only: every feature, forward, gradient and optimiser step
runs in the library's kernels (chap_bs_features, chap_mlp_loss_grad,
chap_mlp_adam); this module slices minibatches and keeps the loss curve.
"""
from __future__ import annotations

import numpy as np

from . import chap

F, H = 12, 64


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases; flat FP32 in the
    library's order W1, b1, W2, b2, w3, b3."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))):
        if name in ("W1", "W2", "w3"):
            lim = np.sqrt(6.0 / shape[0])
            parts.append(rng.uniform(-lim, lim, size=shape).ravel())
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(parts).astype(np.float32)


def to_bf16_bits(a):
    """BF16 bits (round to nearest even) of a float32 torch tensor, as int16."""
    import torch
    return a.to(torch.bfloat16).view(torch.int16)


def log_pairs(bs: "chap.BestShift", passes: int, iters_between: int):
    """Training pairs (features, scaled exact score) of every variable, logged at
    `passes` exact passes of the plain exact driver, `iters_between` iterations apart."""
    import torch
    n = bs.n
    xs, ts = [], []
    for _ in range(passes):
        chap.chap_bs_refresh_features(bs.h)
        f = torch.empty((n, F), dtype=torch.int16, device="cuda")
        t = torch.empty(n, dtype=torch.float32, device="cuda")
        chap.chap_bs_features(bs.h, f, t)
        xs.append(f)
        ts.append(t)
        bs.run(max_iters=iters_between, stop_at_feasible=0)
    return torch.cat(xs), torch.cat(ts)


def train(x, t, epochs=2, batch=4096, lr=1e-3, seed=0):
    """Adam on the MSE; returns (BF16 weights as int16 tensor, FP32 masters, loss per epoch)."""
    import torch
    w32 = torch.tensor(init_params(seed), device="cuda")
    wbf = to_bf16_bits(w32).contiguous()
    m = torch.zeros_like(w32)
    v = torch.zeros_like(w32)
    g = torch.zeros_like(w32)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    n = x.shape[0]
    rng = np.random.default_rng(seed)
    curve = []
    step = 0
    for _ in range(epochs):
        perm = torch.tensor(rng.permutation(n), device="cuda")
        xs, ts = x[perm].contiguous(), t[perm].contiguous()
        loss.zero_()
        for b0 in range(0, n, batch):
            xb, tb = xs[b0:b0 + batch], ts[b0:b0 + batch]
            chap.chap_mlp_loss_grad(wbf, xb, tb, g, loss)
            step += 1
            chap.chap_mlp_adam(w32, wbf, m, v, g, step, lr)
        torch.cuda.synchronize()
        curve.append(float(loss.item()) / n)
    return wbf, w32, curve
