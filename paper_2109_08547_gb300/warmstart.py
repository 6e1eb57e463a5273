"""Learned warm start of the coupled BTE iteration: training data from converged solves,
full-batch training of the network, and its use as the starting point of later solves.

Device memory comes from PyTorch; every computation (features, targets, forward and backward
passes, Adam) runs in the library's kernels.  The host selects the active rows and scales the
targets (a few tens of thousands of numbers).  The library calls synchronise their own stream
before returning, and buffers written by PyTorch are synchronised before they are handed over.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def _sync():
    torch.cuda.synchronize()


def thermo_points(wl, n_train: int, n_held: int, seed: int):
    """Seeded (T, mu, window) points uniform over T in [100, 500] K and mu in mu0 +- 0.2 eV, all on
    the workload's window: (training points, held-out points)."""
    rng = np.random.default_rng(seed)
    pts = [(float(rng.uniform(100.0, 500.0)), float(wl.mu_eV + rng.uniform(-0.2, 0.2)), float(wl.window[0]),
            float(wl.window[1])) for _ in range(n_train + n_held)]
    return pts[:n_train], pts[n_train:]


def instance_data(ctx: B.Context, insts, device, targets: bool = True):
    """Features (and targets) of the active states of the given solved instances, stacked on
    the device.  The kernels fill per-instance buffers; the active rows (inactive states have
    all-zero features) are selected on the host."""
    n = B.num_states(ctx)
    f = torch.empty((n, B.NFEAT), dtype=torch.float32, device=device)
    t = torch.empty((n, 2), dtype=torch.float32, device=device)
    xs, ts = [], []
    for i in insts:
        _sync()
        B.state_features(ctx, i, f.data_ptr())
        fh = f.cpu().numpy()
        active = fh[:, 3] > 0            # T/300 is set for active states only
        xs.append(fh[active])
        if targets:
            B.state_targets(ctx, i, t.data_ptr())
            ts.append(t.cpu().numpy()[active])
    X = torch.from_numpy(np.ascontiguousarray(np.concatenate(xs))).to(device)
    T = torch.from_numpy(np.ascontiguousarray(np.concatenate(ts))).to(device) if targets else None
    _sync()
    return X, T


def train(net: B.MLP, X: torch.Tensor, T: torch.Tensor, steps: int = 400, lr: float = 2e-3, clip: float = 20.0):
    """Full-batch Adam on targets clipped to +-clip and divided by their per-output RMS; the
    RMS is folded back into the output layer afterwards, so the network predicts the targets
    themselves.  Returns the loss (of the scaled targets) before each step."""
    th = np.clip(T.cpu().numpy().astype(np.float64), -clip, clip)
    scale = np.maximum(np.sqrt(np.mean(th * th, axis=0)), 1e-12)
    Ts = torch.from_numpy(np.ascontiguousarray((th / scale).astype(np.float32))).to(X.device)
    _sync()
    losses = [net.train_step(X.data_ptr(), Ts.data_ptr(), X.shape[0], lr) for _ in range(steps)]
    p = net.get_params()
    nb = net.n_out
    fan_in = net.width if net.depth > 0 else net.n_in
    last = p.size - nb * fan_in - nb           # output layer: W [n_out][fan_in] then b [n_out]
    p[last:last + nb * fan_in] *= np.repeat(scale, fan_in).astype(p.dtype)
    p[last + nb * fan_in:] *= scale.astype(p.dtype)
    net.set_params(p)
    return losses


def apply(ctx: B.Context, net: B.MLP, inst: int, device) -> None:
    """Predict the scale factors of every state of instance inst and set them as its start."""
    n = B.num_states(ctx)
    f = torch.empty((n, B.NFEAT), dtype=torch.float32, device=device)
    a = torch.empty((n, 2), dtype=torch.float32, device=device)
    _sync()
    B.state_features(ctx, inst, f.data_ptr())
    net.forward(f.data_ptr(), n, a.data_ptr())
    B.set_warm_start(ctx, inst, a.data_ptr())
