"""FP64 reference of the learned preconditioner network.  TEST INFRASTRUCTURE ONLY.

The network (not from the paper; it is the project's learned right
preconditioner for the Lippmann-Schwinger solve) is a 3-level 3D U-Net on one
sample of S^3 voxels, channel-major [C][S][S][S]:

  E1a conv 3->C, E1b conv C->C                      -> skip1      (S)
  pool 2, E2a conv C->C, E2b conv C->C              -> skip2      (S/2)
  pool 2, B1 conv C->C, B2 conv C->C                              (S/4)
  up 2, concat [up, skip2], D2a conv 2C->C, D2b conv C->C         (S/2)
  up 2, concat [up, skip1], D1a conv 2C->C, D1b conv C->2 (linear) (S)

conv: 3x3x3 cross-correlation with zero padding 1 and a bias,
  y[co](p) = b[co] + sum_ci sum_k w[co, ci, k] x[ci](p + k - 1),
  k = (kz, ky, kx) in {0,1,2}^3 flattened as (kz*3 + ky)*3 + kx;
activation: leaky ReLU, slope 0.1 by default (1: a linear network), after every
conv but the last;
pool: mean of 2x2x2 blocks; up: nearest-neighbour x2.
Loss: mean squared error over all output elements.

Backward is the chain rule written out layer by layer; ``grad_fd`` checks it
by central differences.
"""
from __future__ import annotations

import itertools

import numpy as np

SLOPE = 0.1
OFFSETS = list(itertools.product(range(3), repeat=3))  # (kz, ky, kx), index (kz*3+ky)*3+kx


def layer_shapes(C: int = 16, cin: int = 3, cout: int = 2):
    """(C_out, C_in) of the ten convolutions in network order."""
    return [(C, cin), (C, C), (C, C), (C, C), (C, C), (C, C), (C, 2 * C), (C, C), (C, 2 * C), (cout, C)]


def conv3d(x, w, b):
    S = x.shape[1]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    y = np.broadcast_to(b[:, None, None, None], (w.shape[0], S, S, S)).copy()
    for o, (kz, ky, kx) in enumerate(OFFSETS):
        y += np.tensordot(w[:, :, o], xp[:, kz:kz + S, ky:ky + S, kx:kx + S], axes=([1], [0]))
    return y


def conv3d_backward(x, w, dy):
    S = x.shape[1]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for o, (kz, ky, kx) in enumerate(OFFSETS):
        xs = xp[:, kz:kz + S, ky:ky + S, kx:kx + S]
        dw[:, :, o] = np.tensordot(dy, xs, axes=([1, 2, 3], [1, 2, 3]))
        dxp[:, kz:kz + S, ky:ky + S, kx:kx + S] += np.tensordot(w[:, :, o], dy, axes=([0], [0]))
    db = dy.sum(axis=(1, 2, 3))
    return dxp[:, 1:-1, 1:-1, 1:-1], dw, db


def lrelu(x, slope=SLOPE):
    return np.where(x > 0, x, slope * x)


def lrelu_back(x, dy, slope=SLOPE):
    return np.where(x > 0, dy, slope * dy)


def pool(x):
    C, S = x.shape[0], x.shape[1]
    return x.reshape(C, S // 2, 2, S // 2, 2, S // 2, 2).mean(axis=(2, 4, 6))


def pool_back(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, 1), 2, 2), 2, 3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 1), 2, 2), 2, 3)


def up_back(dy):
    C, S = dy.shape[0], dy.shape[1]
    return dy.reshape(C, S // 2, 2, S // 2, 2, S // 2, 2).sum(axis=(2, 4, 6))


def forward(params, x, slope=SLOPE):
    """params: list of (w, b); returns (output, cache)."""
    c = {"slope": slope}
    h = x
    acts = []

    def cv(i, inp, act=True):
        z = conv3d(inp, *params[i])
        acts.append((i, inp, z))
        return lrelu(z, slope) if act else z

    h = cv(0, h)
    s1 = cv(1, h)
    h = cv(2, pool(s1))
    s2 = cv(3, h)
    h = cv(4, pool(s2))
    h = cv(5, h)
    h = cv(6, np.concatenate([up(h), s2]))
    h = cv(7, h)
    h = cv(8, np.concatenate([up(h), s1]))
    out = cv(9, h, act=False)
    c["acts"] = acts
    return out, c


def backward(params, cache, dout):
    """Gradients (list of (dw, db)) and d/dx of the network for output cotangent dout."""
    acts = {i: (inp, z) for i, inp, z in cache["acts"]}
    grads = [None] * len(params)
    C = params[0][0].shape[0]

    def cvb(i, dh, act=True):
        inp, z = acts[i]
        dz = lrelu_back(z, dh, cache["slope"]) if act else dh
        dx, dw, db = conv3d_backward(inp, params[i][0], dz)
        grads[i] = (dw, db)
        return dx

    d = cvb(9, dout, act=False)           # D1b, input = D1a output
    d = cvb(8, d)                          # D1a, input = concat[up(D2b), s1]
    d_up1, d_s1 = d[:C], d[C:]
    d = cvb(7, up_back(d_up1))             # D2b
    d = cvb(6, d)                          # D2a, input = concat[up(B2), s2]
    d_up2, d_s2 = d[:C], d[C:]
    d = cvb(5, up_back(d_up2))             # B2
    d = cvb(4, d)                          # B1, input = pool(s2)
    d_s2 = d_s2 + pool_back(d)
    d = cvb(3, d_s2)                       # E2b
    d = cvb(2, d)                          # E2a, input = pool(s1)
    d_s1 = d_s1 + pool_back(d)
    d = cvb(1, d_s1)                       # E1b
    dx = cvb(0, d)                         # E1a
    return grads, dx


def mse(out, target):
    return float(np.mean((out - target) ** 2)), 2.0 * (out - target) / out.size


def loss_and_grads(params, x, target, slope=SLOPE):
    out, cache = forward(params, x, slope)
    L, dout = mse(out, target)
    grads, _ = backward(params, cache, dout)
    return L, grads


def grad_fd(params, x, target, layer, idx, h=1e-6):
    """Central difference of the loss in one weight (layer, flat index)."""
    w, b = params[layer]
    w2 = w.copy().ravel()
    w2[idx] += h
    p_plus = [(p[0], p[1]) for p in params]
    p_plus[layer] = (w2.reshape(w.shape), b)
    w3 = w.copy().ravel()
    w3[idx] -= h
    p_minus = [(p[0], p[1]) for p in params]
    p_minus[layer] = (w3.reshape(w.shape), b)
    return (mse(forward(p_plus, x)[0], target)[0] - mse(forward(p_minus, x)[0], target)[0]) / (2 * h)


def init_params(seed: int, C: int = 16, cin: int = 3, cout: int = 2):
    """The shared seeded initial weights (float64 copies)."""
    from paper_1604_03155_gb300 import inputs as I
    return [(w.astype(np.float64), b.astype(np.float64)) for w, b in I.unet_init_weights(seed, C, cin, cout)]
