"""Learned initial iterate for the pressure ramp (2D): trajectories from the
solver, U-Net training, and load steps started from a trust-region-gated
network proposal.  Orchestration only: features, targets, the network,
its gradients, Adam, the proposal and its acceptance test all run in
libpf's kernels.

Modes of starting load step t from the converged x_{t-1}:
  plain         x_{t-1} (the method without a learned part)
  extrapolated  x_{t-1} with u scaled by p_t / p_{t-1} (a non-learned
                predictor: the displacement is nearly linear in p)
  learned       the extrapolated start, then the network's correction
                network(x_{t-1}, c_{t-2}, p_{t-1}, p_t) on top of it; each is
                kept only if its trust-region ratio (against the point before
                it) exceeds eta and the FP64 energy decreases
"""
from __future__ import annotations

import time

import numpy as np

from . import _binding as B

CHANNELS = (16, 32, 64, 128)


def layer_shapes(n_in=5, n_out=3, ch=CHANNELS):
    """(c_out, c_in, k) of every convolution in the C-ABI parameter order."""
    out = []
    c = n_in
    for k in range(4):
        out += [(ch[k], c, 3), (ch[k], ch[k], 3)]
        c = ch[k]
    for k in (2, 1, 0):
        out += [(ch[k], ch[k + 1] + ch[k], 3), (ch[k], ch[k], 3)]
    out.append((n_out, ch[0], 1))
    return out


def he_init(seed: int, n_in=5, n_out=3, ch=CHANNELS) -> np.ndarray:
    """He-normal weights, zero biases, flat FP32 in the C-ABI layout; the
    head starts at zero so an untrained network proposes no change."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    shapes = layer_shapes(n_in, n_out, ch)
    for i, (co, ci, k) in enumerate(shapes):
        std = np.sqrt(2.0 / (ci * k * k)) if i < len(shapes) - 1 else 0.0
        parts.append(rng.standard_normal(co * ci * k * k) * std)
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def padded(n: int) -> int:
    return (n + 7) // 8 * 8


class LearnedIterate:
    """The network for one 2D hierarchy's finest grid."""

    def __init__(self, H, seed=0, channels=CHANNELS):
        import torch
        (nx, ny), _, _ = H.levels[-1]
        self.H = H
        self.nx, self.ny = nx, ny
        self.Hp, self.Wp = padded(ny), padded(nx)
        self.net = B.Unet(self.Hp, self.Wp, 5, 3, channels)
        self.net.set_params(he_init(seed, ch=channels))
        mask = np.zeros((self.Hp, self.Wp), dtype=np.float32)
        mask[:ny, :nx] = 1.0
        self.mask = torch.from_numpy(mask).cuda()
        self.n_valid = float(nx * ny)

    def features(self, x_prev, c_before, p_prev, p_new):
        return B.learned_features(self.H, x_prev, c_before, p_prev, p_new, self.Hp, self.Wp)

    def target(self, x_prev, x_new, p_prev, p_new):
        return B.learned_target(self.H, x_prev, x_new, p_prev, p_new, self.Hp, self.Wp)

    def proposal(self, x_prev, c_before, p_prev, p_new):
        y = self.net.forward(self.features(x_prev, c_before, p_prev, p_new))
        return B.learned_apply(self.H, x_prev, y, p_prev, p_new)

    def extrapolation(self, x_prev, p_prev, p_new):
        """The proposal of a zero network output: u scaled by p_new/p_prev."""
        import torch
        if not hasattr(self, "_zero"):
            self._zero = torch.zeros((3, self.Hp, self.Wp), dtype=torch.float32, device="cuda")
        return B.learned_apply(self.H, x_prev, self._zero, p_prev, p_new)


def trajectory(H, x0, pressures, params):
    """Converged states x_t for p_t in pressures, starting from x0 (which
    holds the fracture network)."""
    states = [x0.clone()]
    x = x0.clone()
    for p in pressures:
        B.pressure_set(H, p)
        B.rmtr_load_step(H, x, params)
        states.append(x.clone())
    return states


def trajectories(Hs, x0s, pressures, params, n_threads=0):
    """trajectory() of several networks at once: at every pressure one
    batched load step over the hierarchies Hs (same grid, one stream each),
    run concurrently by the library's host workers."""
    import torch
    xs = [x0.clone() for x0 in x0s]
    states = [[x.clone()] for x in xs]
    for p in pressures:
        for H in Hs:
            B.pressure_set(H, p)
        torch.cuda.synchronize()
        B.rmtr_load_step_batch(Hs, xs, params, n_threads=n_threads)
        torch.cuda.synchronize()
        for k, x in enumerate(xs):
            states[k].append(x.clone())
    return states


def samples(learner, states, pressures):
    """(features, target) pairs of every transition t-1 -> t with p_{t-1} > 0."""
    out = []
    N = learner.H.nodes()
    for t in range(2, len(states)):
        p_prev, p_new = pressures[t - 2], pressures[t - 1]
        c_before = states[t - 2][2 * N:]
        f = learner.features(states[t - 1], c_before, p_prev, p_new)
        tg = learner.target(states[t - 1], states[t], p_prev, p_new)
        out.append((f.clone(), tg.clone()))
    return out


def train(learner, data, steps, lr=1e-3, batch=4, seed=0):
    """Adam on the masked mean-squared error of the scaled state change."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    net = learner.net
    losses = []
    for it in range(steps):
        idx = rng.integers(0, len(data), size=batch)
        tot = 0.0
        for i in idx:
            f, tg = data[i]
            y = net.forward(f)
            loss, dy = net.mse(y, tg, learner.mask, learner.n_valid)
            net.backward(dy)
            tot += loss
        net.adam(lr, grad_scale=1.0 / batch)
        losses.append(tot / batch)
    torch.cuda.synchronize()
    return losses


def run_ramp(H, x0, pressures, params, mode="plain", learner=None, eta=0.1):
    """Load steps over the ramp from x0; returns per-step records (cycles,
    seconds, energy, and for the learned mode the gate's rho/acceptance).
    The time of a learned step includes the network and the gate."""
    import torch
    x = x0.clone()
    N = H.nodes()
    c_before = x0[2 * N:].clone()  # c of the state before x (c_{t-2})
    recs = []
    p_prev = 0.0
    for t, p in enumerate(pressures):
        B.pressure_set(H, p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rec = {"t": t + 1, "p": p}
        c_now = x[2 * N:].clone()  # c_{t-1}
        # every mode stops at the accuracy relative to the plain start x_{t-1}
        ref = B.projected_gradient(H, x)
        prm = B.default_params(**{k: getattr(params, k) for k, _ in params._fields_})
        prm.pg_ref = ref
        if mode == "extrapolated" and p_prev > 0:
            prm.start = B.PF_START_EXTRAPOLATE  # u scaled by p / p_{t-1} inside the load step
        elif mode == "learned" and p_prev > 0:
            xh = learner.proposal(x, c_before, p_prev, p)
            xe = learner.extrapolation(x, p_prev, p)
            rho_e, acc_e = B.learned_propose(H, x, xe, eta)  # c_prev := c_{t-1}
            rho, acc = B.learned_propose(H, x, xh, eta)      # c of x is still c_{t-1}
            rec.update(rho=rho, accepted=acc, rho_extrapolated=rho_e, accepted_extrapolated=acc_e)
            prm.keep_c_prev = 1
        st = B.rmtr_load_step(H, x, prm, check=False)
        torch.cuda.synchronize()
        rec.update(cycles=st["cycles"], converged=st["converged"], status=st["status"],
                   energy=st["energy"], pg0=st["pg0"], pg=st["pg"],
                   seconds=time.perf_counter() - t0, cg=st["cg"], fe_hessvec=st["fe_hessvec"])
        recs.append(rec)
        c_before = c_now
        p_prev = p
    return recs, x
