"""Learned warm start of the coupled BTE iteration: training data from converged solves,
full-batch training of the network, and its use as the starting point of later solves.

Device memory comes from PyTorch; every computation (features, targets, forward and backward
passes, Adam) runs in the library's kernels.  The library calls synchronise their own stream
before returning, and buffers written by PyTorch are synchronised before they are handed over.
"""
from __future__ import annotations

import torch

from . import binding as B


def _sync():
    torch.cuda.synchronize()


def instance_data(ctx: B.Context, insts, device, targets: bool = True):
    """Features (and targets) of the active states of the given solved instances, stacked."""
    n = B.num_states(ctx)
    xs, ts = [], []
    for i in insts:
        f = torch.empty((n, B.NFEAT), dtype=torch.float32, device=device)
        _sync()
        B.state_features(ctx, i, f.data_ptr())
        active = f[:, 3] > 0            # T/300 is set for active states only
        xs.append(f[active])
        if targets:
            t = torch.empty((n, 2), dtype=torch.float32, device=device)
            _sync()
            B.state_targets(ctx, i, t.data_ptr())
            ts.append(t[active])
    X = torch.cat(xs).contiguous()
    T = torch.cat(ts).contiguous() if targets else None
    _sync()
    return X, T


def train(net: B.MLP, X: torch.Tensor, T: torch.Tensor, steps: int = 400, lr: float = 2e-3):
    """Full-batch Adam; returns the loss before each step."""
    _sync()
    return [net.train_step(X.data_ptr(), T.data_ptr(), X.shape[0], lr) for _ in range(steps)]


def apply(ctx: B.Context, net: B.MLP, inst: int, device) -> None:
    """Predict the scale factors of every state of instance inst and set them as its start."""
    n = B.num_states(ctx)
    f = torch.empty((n, B.NFEAT), dtype=torch.float32, device=device)
    a = torch.empty((n, 2), dtype=torch.float32, device=device)
    _sync()
    B.state_features(ctx, inst, f.data_ptr())
    net.forward(f.data_ptr(), n, a.data_ptr())
    B.set_warm_start(ctx, inst, a.data_ptr())
