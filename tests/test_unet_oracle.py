"""Pins of the U-Net oracle: every parameter tensor's and the input's
gradient against central finite differences of the loss (the network is
piecewise smooth; the step is far below the distance to a ReLU kink at the
seeded point), plus the primitive identities (adjoint pairs)."""
import numpy as np
import pytest

from oracle import unet_oracle as U


def _small(seed=3):
    ch = (4, 6, 8, 10)
    p = U.init_params(seed, ch=ch)
    r = np.random.Generator(np.random.PCG64(seed + 1))
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * r.standard_normal(p[k].shape)
    x = r.standard_normal((U.N_IN, 16, 16))
    t = r.standard_normal((U.N_OUT, 16, 16))
    return ch, p, x, t


def test_architecture_and_parameter_count():
    p = U.init_params(0)
    assert U.n_params(p) == 487619
    y = U.forward(p, np.zeros((5, 16, 24)))
    assert y.shape == (3, 16, 24)


def test_adjoint_pairs():
    r = np.random.Generator(np.random.PCG64(7))
    x = r.standard_normal((3, 8, 10))
    y = r.standard_normal((3, 4, 5))
    assert abs(np.sum(U.avgpool2(x) * y) - np.sum(x * U.avgpool2_backward(y))) < 1e-12
    z = r.standard_normal((3, 8, 10))
    assert abs(np.sum(U.up2(y) * z) - np.sum(y * U.up2_backward(z))) < 1e-12
    c = r.standard_normal((27, 80))
    assert abs(np.sum(U._im2col3(x) * c) - np.sum(x * U._col2im3(c, 3, 8, 10))) < 1e-12


def test_conv_matches_direct_sum():
    r = np.random.Generator(np.random.PCG64(9))
    x = r.standard_normal((2, 5, 6))
    w = r.standard_normal((3, 2, 3, 3))
    b = r.standard_normal(3)
    y = U.conv(x, w, b)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    for co in range(3):
        for i in range(5):
            for j in range(6):
                ref = b[co] + np.sum(w[co] * xp[:, i:i + 3, j:j + 3])
                assert abs(y[co, i, j] - ref) < 1e-12


def test_gradients_match_central_differences():
    ch, p, x, t = _small()
    y, acts = U.forward(p, x, ch=ch, keep=True)
    loss, dy = U.mse_loss(y, t)
    grads, dx = U.backward(p, acts, dy, ch=ch)
    r = np.random.Generator(np.random.PCG64(11))
    eps = 1e-6

    def L(pp, xx):
        return U.mse_loss(U.forward(pp, xx, ch=ch), t)[0]

    for name in p:
        for _ in range(3):
            idx = tuple(r.integers(0, s) for s in p[name].shape)
            old = p[name][idx]
            p[name][idx] = old + eps
            lp = L(p, x)
            p[name][idx] = old - eps
            lm = L(p, x)
            p[name][idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - grads[name][idx]) <= 1e-6 * max(1e-3, abs(fd)), (name, idx, fd, grads[name][idx])
    for _ in range(5):
        idx = tuple(r.integers(0, s) for s in x.shape)
        xp = x.copy(); xp[idx] += eps
        xm = x.copy(); xm[idx] -= eps
        fd = (L(p, xp) - L(p, xm)) / (2 * eps)
        assert abs(fd - dx[idx]) <= 1e-6 * max(1e-3, abs(fd))


def test_adam_step_decreases_loss():
    ch, p, x, t = _small(5)
    st = {}
    l0 = None
    for _ in range(30):
        y, acts = U.forward(p, x, ch=ch, keep=True)
        loss, dy = U.mse_loss(y, t)
        l0 = loss if l0 is None else l0
        grads, _ = U.backward(p, acts, dy, ch=ch)
        U.adam_step(p, grads, st, lr=1e-2)
    assert loss < 0.8 * l0


def _adam_pin(adam):
    """Adam (Kingma & Ba, Algorithm 1) from zero moments: the first step is
    -lr g / (|g| + eps) for every entry (bias-corrected moments are g and
    g^2); the second step, for g1 = 0.5 then g2 = -0.25 with lr = 0.1,
    beta1 = 0.9, beta2 = 0.999, eps = 1e-8, worked by hand:
    m2 = 0.9*0.05 - 0.1*0.25 = 0.02, m2/(1-0.81) = 0.10526315789473684;
    v2 = 0.999*0.00025 + 0.001*0.0625 = 0.00031225, v2/(1-0.998001)
    = 0.1562031015507775, sqrt = 0.3952253807016...;
    step = -0.1 * 0.10526315789473684 / (0.3952253807016 + 1e-8)... = -0.0266337033..."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = {"w": np.array([1.0, 1.0, 1.0, 1.0])}
    st = {}
    adam(p, {"w": g.copy()}, st, lr=0.1)
    first = np.array([1.0 - 0.1 * 0.5 / (0.5 + 1e-8), 1.0 + 0.1 * 2.0 / (2.0 + 1e-8),
                      1.0 - 0.1 * 1e-3 / (1e-3 + 1e-8), 1.0])
    assert np.max(np.abs(p["w"] - first)) <= 1e-15
    p2 = {"w": np.array([0.0])}
    st2 = {}
    adam(p2, {"w": np.array([0.5])}, st2, lr=0.1)
    w1 = float(p2["w"][0])
    adam(p2, {"w": np.array([-0.25])}, st2, lr=0.1)
    assert abs(w1 - (-0.1 * 0.5 / (0.5 + 1e-8))) <= 1e-15
    assert abs((float(p2["w"][0]) - w1) - (-0.0266337033)) <= 1e-9


def test_adam_first_and_second_step_closed_form():
    _adam_pin(U.adam_step)


def test_pins_catch_a_dropped_bias_correction():
    """Adam without the bias correction of its moments fails the pin."""
    def no_bias(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        for k in params:
            m = state.setdefault("m." + k, np.zeros_like(params[k]))
            v = state.setdefault("v." + k, np.zeros_like(params[k]))
            m[...] = beta1 * m + (1 - beta1) * grads[k]
            v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
            params[k] -= lr * m / (np.sqrt(v) + eps)

    with pytest.raises(AssertionError):
        _adam_pin(no_bias)
