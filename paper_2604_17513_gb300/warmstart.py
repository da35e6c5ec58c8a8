"""Learned warm start: data collection from the simulator's own converged
steps and training of the per-contact network with the library's kernels.

The host only orders the work: features and targets are written by the step
kernels (flash_record_contacts), losses, gradients and Adam updates by the
network kernels.  Parameter initialisation is seeded (He-uniform).
"""
from __future__ import annotations

import numpy as np
import torch

from . import flash

NI, NH, NO = 10, 128, 6


def init_params(seed=0, device="cuda"):
    """Flat float32 parameters W1 b1 W2 b2 W3 b3 (He-uniform weights, zero biases)."""
    g = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((NI, NH), (NH, NH), (NH, NO)):
        lim = np.sqrt(6.0 / fan_in)
        parts.append(g.uniform(-lim, lim, (fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == flash.mlp_num_params()
    return torch.from_numpy(p).to(device)


def collect(sim, sc, first_step, n_steps, device):
    """Run n_steps of ``sim`` (scene ``sc``) with recording on; returns the
    stacked (features, targets) of every contact of every step."""
    sim.record(True)
    xs, ts = [], []
    for s in range(first_step, first_step + n_steps):
        sim.set_poses(flash.poses_tensor(sc, s + 1, device))
        sim.step(1)
        X, T = sim.recorded()
        xs.append(X.clone())
        ts.append(T.clone())
    sim.record(False)
    return torch.cat(xs), torch.cat(ts)


def usable(X, T, clip=100.0):
    """Rows with a target (converged environments) and no entry beyond ``clip``."""
    ok = torch.isfinite(T).all(1) & (T.abs() <= clip).all(1) & (X.abs() <= clip).all(1)
    return X[ok].contiguous(), T[ok].contiguous()


def input_range(X, T, clip=100.0):
    """Per-feature (lo, hi) of the usable training rows: the range the network
    was fitted on (host float32 arrays for ``Sim.warmstart(bounds=...)``)."""
    Xu, _ = usable(X, T, clip)
    return Xu.min(0).values.cpu().numpy(), Xu.max(0).values.cpu().numpy()


def in_range(X, lo, hi):
    """Rows of X inside [lo, hi] feature by feature (the library's gate)."""
    lo = torch.as_tensor(lo, device=X.device)
    hi = torch.as_tensor(hi, device=X.device)
    return ((X >= lo) & (X <= hi)).all(1)


def train(X, T, epochs=5, batch=4096, lr=1e-3, seed=0, params=None, holdout=0.1):
    """Adam on the mean squared error; returns (params, train losses per
    epoch, held-out loss).  Rows are shuffled once on the host (seeded)."""
    dev = X.device
    X, T = usable(X, T)
    n = X.shape[0]
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(n)).to(dev)
    X, T = X[perm].contiguous(), T[perm].contiguous()
    n_hold = int(n * holdout)
    Xh, Th = X[:n_hold], T[:n_hold]
    Xt, Tt = X[n_hold:], T[n_hold:]
    p = init_params(seed, dev) if params is None else params.clone()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    work = None
    step = 0
    hist = []
    for _ in range(epochs):
        tot = torch.zeros((), dtype=torch.float64, device=dev)
        for b0 in range(0, Xt.shape[0] - batch + 1, batch):
            sse, g = flash.mlp_loss_grad(p, Xt[b0:b0 + batch], Tt[b0:b0 + batch], work)
            step += 1
            flash.mlp_adam(p, g, m, v, step, lr)
            tot += sse[0].double()
        hist.append(0.5 * tot.item() / max(1, (Xt.shape[0] // batch) * batch))
    held = None
    if n_hold >= 1:
        y = flash.mlp_forward(p, Xh)
        held = 0.5 * ((y - Th) ** 2).sum(1).mean().item()
    return p, hist, held
