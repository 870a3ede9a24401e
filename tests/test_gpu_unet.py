"""The CUDA U-Net (BF16 weights/activations, tensor-core convolutions with
FP32 accumulation) against the FP64 oracle on a 64 x 64 input, and the
learned-iterate glue.

Tolerances: BF16 keeps 8 significant bits (relative rounding 2^-9 ~ 2e-3
per stored value); through 15 layers the output and the weight gradients
agree with the FP64 oracle to a few 1e-2 in relative L2 norm and to a
cosine above 0.999 (the bar for BF16 training kernels)."""
import numpy as np
import pytest

import pfinputs as PI
from oracle import pf_oracle as O
from oracle import unet_oracle as U
from tests.gpu_common import dev, host, pair, require_cuda

pytestmark = pytest.mark.gpu


def _flat(params):
    out = []
    for name, co, ci, k in U.layer_shapes():
        out.append(params[name + ".w"].ravel())
        out.append(params[name + ".b"].ravel())
    return np.concatenate(out)


def _unflat(vec):
    params, off = {}, 0
    for name, co, ci, k in U.layer_shapes():
        n = co * ci * k * k
        params[name + ".w"] = vec[off:off + n].reshape(co, ci, k, k).astype(np.float64)
        off += n
        params[name + ".b"] = vec[off:off + co].astype(np.float64)
        off += co
    return params


def _bf16(a):
    """Round float64 values to the nearest BF16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> 16) & 1
    r = ((f + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cos(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.fixture(scope="module")
def setup():
    torch = require_cuda()
    from paper_2007_12908_gb300 import _binding as B
    p = U.init_params(21)
    r = np.random.Generator(np.random.PCG64(22))
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.05 * r.standard_normal(p[k].shape)
    # 64 x 64: the deepest level then sums 8 x 8 pixels; on smaller inputs a
    # few ReLU decisions that BF16 activation storage flips dominate its sums
    x = r.standard_normal((5, 64, 64))
    t = r.standard_normal((3, 64, 64))
    net = B.Unet(64, 64)
    assert net.n_params == U.n_params(p) == 487619
    net.set_params(_flat(p).astype(np.float32))
    return torch, B, p, x, t, net


def test_forward_matches_oracle(setup):
    torch, B, p, x, t, net = setup
    y = host(net.forward(dev(x, torch.float32)))
    pb = {k: _bf16(v) if k.endswith(".w") else v for k, v in p.items()}
    yo = U.forward(pb, _bf16(x))
    assert _rel(y, yo) < 3e-2 and _cos(y, yo) > 0.999


def test_gradients_match_oracle(setup):
    torch, B, p, x, t, net = setup
    net.set_params(_flat(p).astype(np.float32))
    xd, td = dev(x, torch.float32), dev(t, torch.float32)
    y = net.forward(xd)
    loss, dy = net.mse(y, td)
    net.backward(dy)
    g = _unflat(net.get_grads())
    pb = {k: _bf16(v) if k.endswith(".w") else v for k, v in p.items()}
    yo, acts = U.forward(pb, _bf16(x), keep=True)
    lo, dyo = U.mse_loss(yo, t)
    go, _ = U.backward(pb, acts, dyo)
    assert abs(loss - lo) / lo < 3e-2
    for name, co, ci, k in U.layer_shapes():
        for suf in (".w", ".b"):
            a, b = g[name + suf], go[name + suf]
            assert _cos(a, b) > 0.999, (name + suf, _cos(a, b))
            assert _rel(a, b) < 5e-2, (name + suf, _rel(a, b))


def test_adam_step_matches_oracle(setup):
    torch, B, p, x, t, net = setup
    net.set_params(_flat(p).astype(np.float32))
    y = net.forward(dev(x, torch.float32))
    loss, dy = net.mse(y, dev(t, torch.float32))
    net.backward(dy)
    g = net.get_grads().astype(np.float64)
    net.adam(1e-3)
    got = net.get_params().astype(np.float64)
    po = {"w": _flat(p).astype(np.float32).astype(np.float64)}
    U.adam_step(po, {"w": g}, {}, lr=1e-3)
    assert np.max(np.abs(got - po["w"])) < 1e-6
    assert np.all(net.get_grads() == 0.0)


def test_learned_glue_round_trip_and_gate():
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from paper_2007_12908_gb300 import _binding as B
    H, Ho = pair(2, (17, 17), 2, 1 / 16, p=1e-3)
    g = Ho.fine
    x0 = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_LINE2D, PI.centred_crack_2d(0.2), g.h, x0)
    x1 = x0.clone()
    pf.rmtr_load_step(H, x1, pf.default_params(rtol=1e-12))
    pf.pressure_set(H, 2e-3)
    x2 = x1.clone()
    pf.rmtr_load_step(H, x2, pf.default_params(rtol=1e-12))
    Hp, Wp = 40, 40
    f = B.learned_features(H, x1, x0[2 * g.N:], 1e-3, 2e-3, Hp, Wp)
    fo = host(f)
    assert np.all(fo[:, g.n[1]:, :] == 0) and np.all(fo[3, :g.n[1], :g.n[0]] == np.float32(2.0))
    tg = B.learned_target(H, x1, x2, 1e-3, 2e-3, Hp, Wp)
    xh = host(B.learned_apply(H, x1, tg, 1e-3, 2e-3))
    # zero network output = the linear extrapolation of u, c unchanged
    xe = host(B.learned_apply(H, x1, torch.zeros_like(tg), 1e-3, 2e-3))
    x1h = host(x1)
    assert np.allclose(xe[: 2 * g.N], 2.0 * x1h[: 2 * g.N], rtol=0, atol=1e-18)
    assert np.array_equal(xe[2 * g.N:], x1h[2 * g.N:])
    ref = host(x2)
    assert np.max(np.abs(xh - ref)) <= 1e-6 * np.max(np.abs(ref))
    # the converged next state passes the gate with rho close to 1 ...
    xs = x1.clone()
    rho, acc = B.learned_propose(H, xs, x2)
    assert acc and 0.5 < rho < 1.5
    # ... and a proposal that raises the energy is refused, x unchanged
    bad = x2.clone()
    bad[: 2 * g.N] *= -3.0
    xs2 = x1.clone()
    rho2, acc2 = B.learned_propose(H, xs2, bad)
    assert not acc2 and torch.equal(xs2, x1)


def test_learned_gate_rho_matches_oracle():
    """pf_learned_propose's ratio, decision and accepted state against the
    oracle's trust-region gate (eq. rho_tr, Algorithm 3's acceptance) on the
    same states: the converged next state, the linear extrapolation, and a
    proposal that raises the energy."""
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from paper_2007_12908_gb300 import _binding as B
    H, Ho = pair(2, (17, 17), 2, 1 / 16, p=1e-3)
    g = Ho.fine
    x0 = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_LINE2D, PI.centred_crack_2d(0.2), g.h, x0)
    x1 = x0.clone()
    pf.rmtr_load_step(H, x1, pf.default_params(rtol=1e-12))
    pf.pressure_set(H, 2e-3)
    x2 = x1.clone()
    pf.rmtr_load_step(H, x2, pf.default_params(rtol=1e-12))
    Ho.prm.p = 2e-3
    ext = x1.clone()
    ext[: 2 * g.N] *= 2.0
    bad = x2.clone()
    bad[: 2 * g.N] *= -3.0
    for prop, want in ((x2, True), (ext, True), (bad, False)):
        xs = x1.clone()
        rho, acc = B.learned_propose(H, xs, prop, 0.1)
        rho_o, acc_o, x_o = O.trust_region_gate(Ho, host(x1), host(prop), 0.1)
        assert acc == acc_o == want
        if np.isinf(rho_o):
            assert rho == rho_o
        else:
            assert abs(rho - rho_o) <= 1e-9 * abs(rho_o), (rho, rho_o)
        assert np.max(np.abs(host(xs) - x_o)) <= 1e-15 * max(np.max(np.abs(x_o)), 1e-300)
    H.close()
