"""FP64 CPU oracle of the learned initial-iterate network (TEST
INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU leg; the CUDA path shares no code with it).

The network proposes a load step's change of state from the previous one.
The paper has no learned component: architecture, features and scaling
are this library's readings (listed in the design notes):

  encoder  level k = 0..3, channels C = (16, 32, 64, 128):
           two 3x3 convolutions (zero padding 1) each followed by ReLU;
           2x2 average pooling between levels
  decoder  level k = 2, 1, 0: nearest-neighbour 2x upsampling of the level
           below, concatenation [upsampled, encoder skip], two 3x3
           convolutions + ReLU
  head     1x1 convolution to 3 outputs (no activation)

Tensors are (channels, H, W) float64 arrays, H and W multiples of 8.
Convolutions are written as im2col followed by one matrix product.
Parity status: pinned by central finite differences of a scalar loss
through every parameter tensor and the input; Adam by its closed-form first
step from zero moments and a second step worked by hand
(tests/test_unet_oracle.py).
"""
from __future__ import annotations

import numpy as np

CHANNELS = (16, 32, 64, 128)
N_IN = 5
N_OUT = 3


def layer_shapes(n_in=N_IN, n_out=N_OUT, ch=CHANNELS):
    """(name, c_out, c_in, k) of every convolution, in parameter order."""
    shapes = []
    c_prev = n_in
    for k, c in enumerate(ch):
        shapes.append((f"enc{k}a", c, c_prev, 3))
        shapes.append((f"enc{k}b", c, c, 3))
        c_prev = c
    for k in range(len(ch) - 2, -1, -1):
        shapes.append((f"dec{k}a", ch[k], ch[k + 1] + ch[k], 3))
        shapes.append((f"dec{k}b", ch[k], ch[k], 3))
    shapes.append(("head", n_out, ch[0], 1))
    return shapes


def init_params(seed: int, n_in=N_IN, n_out=N_OUT, ch=CHANNELS):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = {}
    for name, co, ci, k in layer_shapes(n_in, n_out, ch):
        std = np.sqrt(2.0 / (ci * k * k))
        params[name + ".w"] = rng.standard_normal((co, ci, k, k)) * std
        params[name + ".b"] = np.zeros(co)
    return params


def n_params(params) -> int:
    return int(sum(v.size for v in params.values()))


# ---------------------------------------------------------------- primitives
def _im2col3(x):
    """(C, H, W) -> (C*9, H*W) patches of a 3x3 window, zero padding 1;
    row index c*9 + dy*3 + dx with offsets dy, dx - 1."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    cols = np.empty((C, 9, H, W))
    for dy in range(3):
        for dx in range(3):
            cols[:, dy * 3 + dx] = xp[:, dy:dy + H, dx:dx + W]
    return cols.reshape(C * 9, H * W)


def _col2im3(cols, C, H, W):
    """Adjoint of _im2col3."""
    cols = cols.reshape(C, 9, H, W)
    xp = np.zeros((C, H + 2, W + 2))
    for dy in range(3):
        for dx in range(3):
            xp[:, dy:dy + H, dx:dx + W] += cols[:, dy * 3 + dx]
    return xp[:, 1:-1, 1:-1]


def conv(x, w, b):
    co, ci, k, _ = w.shape
    C, H, W = x.shape
    if k == 1:
        return (w.reshape(co, ci) @ x.reshape(ci, H * W)).reshape(co, H, W) + b[:, None, None]
    cols = _im2col3(x)
    return (w.reshape(co, ci * 9) @ cols).reshape(co, H, W) + b[:, None, None]


def conv_backward(x, w, dy):
    """Gradients of conv(x, w, b) with respect to x, w and b given dL/dy."""
    co, ci, k, _ = w.shape
    C, H, W = x.shape
    dyf = dy.reshape(co, H * W)
    db = dyf.sum(axis=1)
    if k == 1:
        xf = x.reshape(ci, H * W)
        dw = (dyf @ xf.T).reshape(co, ci, 1, 1)
        dx = (w.reshape(co, ci).T @ dyf).reshape(ci, H, W)
        return dx, dw, db
    cols = _im2col3(x)
    dw = (dyf @ cols.T).reshape(co, ci, 3, 3)
    dcols = w.reshape(co, ci * 9).T @ dyf
    dx = _col2im3(dcols, ci, H, W)
    return dx, dw, db


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    C, H, W = x.shape
    return x.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def avgpool2_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) * 0.25


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(dy):
    C, H, W = dy.shape
    return dy.reshape(C, H // 2, 2, W // 2, 2).sum(axis=(2, 4))


# ---------------------------------------------------------------- network
def forward(params, x, ch=CHANNELS, keep=False):
    """y = net(x); with keep, also the activations the backward pass needs."""
    acts = {}
    skips = []
    h = x
    L = len(ch)
    for k in range(L):
        if k > 0:
            h = avgpool2(h)
        acts[f"enc{k}a.in"] = h
        h = relu(conv(h, params[f"enc{k}a.w"], params[f"enc{k}a.b"]))
        acts[f"enc{k}a.out"] = h
        acts[f"enc{k}b.in"] = h
        h = relu(conv(h, params[f"enc{k}b.w"], params[f"enc{k}b.b"]))
        acts[f"enc{k}b.out"] = h
        skips.append(h)
    for k in range(L - 2, -1, -1):
        h = np.concatenate([up2(h), skips[k]], axis=0)
        acts[f"dec{k}a.in"] = h
        h = relu(conv(h, params[f"dec{k}a.w"], params[f"dec{k}a.b"]))
        acts[f"dec{k}a.out"] = h
        acts[f"dec{k}b.in"] = h
        h = relu(conv(h, params[f"dec{k}b.w"], params[f"dec{k}b.b"]))
        acts[f"dec{k}b.out"] = h
    acts["head.in"] = h
    y = conv(h, params["head.w"], params["head.b"])
    return (y, acts) if keep else y


def backward(params, acts, dy, ch=CHANNELS):
    """dL/dparams and dL/dx for dL/dy at the activations of forward(keep=True)."""
    grads = {}
    dh, grads["head.w"], grads["head.b"] = conv_backward(acts["head.in"], params["head.w"], dy)
    L = len(ch)
    dskip = [None] * L

    def through(name, dh):
        dpre = dh * (acts[name + ".out"] > 0)
        dx, grads[name + ".w"], grads[name + ".b"] = conv_backward(
            acts[name + ".in"], params[name + ".w"], dpre)
        return dx

    # decoder, in reverse of the forward order (level 0 first)
    for k in range(0, L - 1):
        dh = through(f"dec{k}b", dh)
        dh = through(f"dec{k}a", dh)
        c_up = ch[k + 1]
        dskip[k] = dh[c_up:]
        dh = up2_backward(dh[:c_up])  # into the output of the level below
    # encoder, from the bottleneck up; skips add to their level's output
    for k in range(L - 1, -1, -1):
        if k < L - 1:
            dh = dh + dskip[k]
        dh = through(f"enc{k}b", dh)
        dh = through(f"enc{k}a", dh)
        if k > 0:
            dh = avgpool2_backward(dh)
    return grads, dh


def mse_loss(y, target, mask=None):
    """L = mean over valid pixels and channels of (y - target)^2 / 2."""
    d = y - target
    if mask is not None:
        d = d * mask
        n = mask.sum() * y.shape[0]
    else:
        n = d.size
    return 0.5 * float(np.sum(d * d)) / n, d / n


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of every parameter, in place."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m." + k, np.zeros_like(params[k]))
        v = state.setdefault("v." + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        params[k] -= lr * mh / (np.sqrt(vh) + eps)
