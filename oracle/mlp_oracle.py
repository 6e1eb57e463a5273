"""FP64 reference of the learned warm start (test infrastructure only; see the package docstring).

The warm start is an extension of the method, not a part of arXiv 2109.08547: a small fully
connected network proposes, per electron state, the starting deviation functions of the
coupled iteration of section "Coupled and decoupled BTEs", which otherwise starts from the
RTA solution (Eqs. I0/J0).  The iteration itself is unchanged, so the converged answer is too;
only the number of sweeps can change.  This module restates, in plain double precision:

  * the per-state inputs (features) and training targets,
  * the network: tanh hidden layers, linear output, loss 1/(2N) sum_i |y_i - t_i|^2,
  * the gradient of that loss by reverse-mode differentiation, layer by layer.

Pins (tests): central finite differences of the loss; invariants of a network whose hidden
weights are zero; gradient descent on a network without hidden layers reaching the
numpy.linalg.lstsq solution; targets and features on cases with known values.
"""
from __future__ import annotations

import numpy as np

from .ephb_oracle import KB_EVK

NFEAT = 6          # inputs per electron state
NOUT = 2           # outputs: scale factors of I (temperature gradient) and J (electric field)


# ----------------------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------------------

def init_params(n_in: int, width: int, depth: int, n_out: int, seed: int):
    """[(W, b)] with W of shape (fan_out, fan_in): uniform(+-sqrt(6/(fan_in+fan_out))) weights
    (Glorot), zero biases.  depth hidden layers of the given width."""
    rng = np.random.default_rng(seed)
    dims = [n_in] + [width] * depth + [n_out]
    out = []
    for a, b in zip(dims[:-1], dims[1:]):
        lim = np.sqrt(6.0 / (a + b))
        out.append((rng.uniform(-lim, lim, size=(b, a)), np.zeros(b)))
    return out


def forward(params, x):
    """y = W_L h_{L-1} + b_L with h_l = tanh(W_l h_{l-1} + b_l), h_0 = x.  Returns y and the
    list [h_0, h_1, ..., h_{L-1}]."""
    h = [np.asarray(x, dtype=np.float64)]
    for W, b in params[:-1]:
        h.append(np.tanh(h[-1] @ W.T + b))
    W, b = params[-1]
    return h[-1] @ W.T + b, h


def loss(params, x, t):
    y, _ = forward(params, x)
    return 0.5 * np.sum((y - t) ** 2) / len(x)


def gradients(params, x, t):
    """d loss / d (W_l, b_l) for every layer (backpropagation):
    delta_L = (y - t) / N;  dW_l = delta_l^T h_{l-1};  db_l = sum_i delta_l;
    delta_{l-1} = (delta_l W_l) * (1 - h_{l-1}^2)."""
    y, h = forward(params, x)
    delta = (y - t) / len(x)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        grads[l] = (delta.T @ h[l], delta.sum(axis=0))
        if l > 0:
            delta = (delta @ W) * (1.0 - h[l] ** 2)
    return grads


def flatten(params):
    """Parameters in one vector: layer by layer, W (row-major) then b."""
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unflatten(vec, like):
    out, o = [], 0
    for W, b in like:
        nW, nb = W.size, b.size
        out.append((vec[o:o + nW].reshape(W.shape), vec[o + nW:o + nW + nb]))
        o += nW + nb
    return out


# ----------------------------------------------------------------------------------------
# inputs and targets per electron state
# ----------------------------------------------------------------------------------------

def state_features(eps, vel, W_e, T, mu):
    """Per state: (eps-mu)/kT clipped to +-40 and divided by 10, log10(W_e) - 13, |v| / max|v|,
    T/300 K, mu/0.1 eV, eps/0.3 eV.  States without a rate (W_e = 0) get log10 term 0."""
    eps = np.asarray(eps, dtype=np.float64)
    kT = KB_EVK * T
    speed = np.linalg.norm(vel, axis=1)
    vmax = speed.max() if speed.size and speed.max() > 0 else 1.0
    lw = np.where(W_e > 0, np.log10(np.where(W_e > 0, W_e, 1.0)) - 13.0, 0.0)
    return np.stack([np.clip((eps - mu) / kT, -40.0, 40.0) / 10.0, lw, speed / vmax, np.full_like(eps, T / 300.0),
                     np.full_like(eps, mu / 0.1), eps / 0.3], axis=1)


def scale_targets(I, J, J0, x, speed, speed_cut=1e-6):
    """Per state, along the RTA direction J0 = v/W:
         a_I = (I.J0)/(J0.J0)/k_B - x,   a_J = (J.J0)/(J0.J0) - 1,
    with x = (eps-mu)/(k_B T), so the RTA solution (I0 = (eps-mu)/T J0) has a = 0.  Zero where
    J0 = 0 or the speed is below speed_cut of the largest (velocities that vanish by symmetry
    carry no direction)."""
    d = np.sum(J0 * J0, axis=1)
    ok = (d > 0) & (speed > speed_cut * (speed.max() if speed.size else 0.0))
    dd = np.where(ok, d, 1.0)
    aI = np.where(ok, np.sum(I * J0, axis=1) / dd / KB_EVK - x, 0.0)
    aJ = np.where(ok, np.sum(J * J0, axis=1) / dd - 1.0, 0.0)
    return np.stack([aI, aJ], axis=1)


def warm_start(I0, J0, a):
    """Starting responses I = I0 + a_I k_B J0, J = J0 (1 + a_J)."""
    return I0 + (a[:, 0:1] * KB_EVK) * J0, J0 * (1.0 + a[:, 1:2])


__all__ = ["NFEAT", "NOUT", "init_params", "forward", "loss", "gradients", "flatten", "unflatten",
           "state_features", "scale_targets", "warm_start"]
