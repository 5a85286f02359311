"""CPU float64 oracle for the learned preconditioner's network.

TEST INFRASTRUCTURE ONLY (used by tests/ and bench.py's baseline leg, never by
the product path).  The network is a plain stack of 3x3x3 convolutions with
zero padding ("same"), stride 1, a bias per output channel and a ReLU after
every layer but the last:

    a_0 = input (C_0 x D x H x W)
    z_l = W_l * a_{l-1} + b_l          (cross-correlation, W_l: C_l x C_{l-1} x 3 x 3 x 3)
    a_l = relu(z_l) for l < L, a_L = z_L

It is written as 27 shifted array products per layer (no im2col, no blocking)
so a reader can check it against the definition of a convolution.  The loss
is the relative squared error on the mask voxels,
    loss = sum_b sum_v m_v (a_L - t)^2 / sum_b sum_v m_v t^2,
and the backward pass is the chain rule of exactly these steps.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """y[..., z, y, x] = x[..., z + dz, y + dy, x + dx], zero outside the box."""
    out = np.zeros_like(x)
    D, H, W = x.shape[-3:]
    zs, ze = max(0, -dz), min(D, D - dz)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    out[..., zs:ze, ys:ye, xs:xe] = x[..., zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv(a: np.ndarray, Wt: np.ndarray, b: np.ndarray) -> np.ndarray:
    """z[co] = b[co] + sum_ci sum_taps W[co, ci, tap] * a[ci] shifted by tap.  a: (B, Ci, D, H, W)."""
    Bn, Ci = a.shape[:2]
    Co = Wt.shape[0]
    z = np.zeros((Bn, Co) + a.shape[2:])
    z += b.reshape(1, Co, 1, 1, 1)
    for t, (dz, dy, dx) in enumerate(TAPS):
        s = shift(a, dz, dy, dx)  # (B, Ci, D, H, W)
        z += np.einsum("oc,bczyx->bozyx", Wt[:, :, t], s)
    return z


def forward(x: np.ndarray, weights, biases):
    """Returns the list of activations a_0 .. a_L (a_L has the output)."""
    acts = [x]
    L = len(weights)
    for l in range(L):
        z = conv(acts[-1], weights[l], biases[l])
        acts.append(np.maximum(z, 0.0) if l < L - 1 else z)
    return acts


def loss_and_grad_out(out: np.ndarray, target: np.ndarray, mask: np.ndarray):
    """Relative masked squared error and its gradient w.r.t. out (out, target: (B, 1, D, H, W))."""
    m = mask.reshape(1, 1, *mask.shape)
    den = float(np.sum(m * target ** 2))
    diff = m * (out - target)
    return float(np.sum(diff * (out - target))) / den, 2.0 * diff / den


def backward(acts, weights, grad_out):
    """Gradients (dW_l, db_l) for all layers given dloss/da_L."""
    L = len(weights)
    dWs, dbs = [None] * L, [None] * L
    g = grad_out  # dloss/dz_L (last layer is linear)
    for l in range(L - 1, -1, -1):
        a_in = acts[l]
        dbs[l] = g.sum(axis=(0, 2, 3, 4))
        dW = np.zeros_like(weights[l])
        for t, (dz, dy, dx) in enumerate(TAPS):
            s = shift(a_in, dz, dy, dx)
            dW[:, :, t] = np.einsum("bozyx,bczyx->oc", g, s)
        dWs[l] = dW
        if l > 0:
            # dloss/da_{l-1} = sum_taps W^T g shifted back
            ga = np.zeros_like(a_in)
            for t, (dz, dy, dx) in enumerate(TAPS):
                ga += shift(np.einsum("oc,bozyx->bczyx", weights[l][:, :, t], g), -dz, -dy, -dx)
            g = ga * (acts[l] > 0.0)  # relu'(z_{l-1}) with a_{l-1} = relu(z_{l-1})
    return dWs, dbs
