"""The learned initial iterate end to end on a small 2D ramp: trajectories
from the solver, training by the library's own forward/backward/Adam
kernels, and the trust-region-gated proposal against the plain and the
extrapolated starting points on held-out fracture networks."""
import numpy as np
import pytest

import pfinputs as PI
from tests.gpu_common import require_cuda

pytestmark = pytest.mark.gpu

PRESSURES = [5e-4 * t for t in range(1, 7)]


def _setup(pf, seed, H):
    import torch
    (nx, ny), h, N = H.levels[-1]
    rows = PI.line_network_2d(seed, 12, lmin=0.05, lmax=0.25)
    x0 = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_LINE2D, rows, h, x0)
    return x0


def test_learned_iterate_trains_and_is_gated():
    require_cuda()
    import paper_2007_12908_gb300 as pf
    from paper_2007_12908_gb300 import learned as Lm
    H = pf.mesh_hierarchy_create(2, (33, 33), 3, 1 / 32, E=1.0, nu=0.3, Gc=1.0)  # 129^2 finest
    prm = pf.default_params()
    learner = Lm.LearnedIterate(H, seed=1)
    data = []
    for seed in range(1500, 1516):
        x0 = _setup(pf, seed, H)
        states = Lm.trajectory(H, x0, PRESSURES, prm)
        data += Lm.samples(learner, states, PRESSURES)
    losses = Lm.train(learner, data, steps=600, lr=1e-3, batch=4)
    assert np.mean(losses[-20:]) < 0.2 * np.mean(losses[:5])
    res = {m: [] for m in ("plain", "extrapolated", "learned")}
    for seed in (1600, 1601):
        x0 = _setup(pf, seed, H)
        for mode in res:
            recs, x = Lm.run_ramp(H, x0, PRESSURES, prm, mode=mode, learner=learner)
            assert all(r["converged"] for r in recs), (seed, mode, recs)
            res[mode].append(recs)
    cyc = {m: np.mean([r["cycles"] for recs in v for r in recs[1:]]) for m, v in res.items()}
    acc = [r["accepted_extrapolated"] or r["accepted"] for recs in res["learned"] for r in recs[1:]]
    print("mean V-cycles per load step (t >= 2):", cyc, "accepted", acc)
    # same converged energies whichever start is used
    for a, b in zip(res["plain"], res["learned"]):
        for ra, rb in zip(a, b):
            assert abs(ra["energy"] - rb["energy"]) <= 1e-8 * abs(ra["energy"])
    assert np.mean(acc) >= 0.5
    # the gain of the learned start over each start without the network, in
    # V-cycles per load step: it must beat the plain start and may not lose
    # to the extrapolation it starts from; a zero gain over the
    # extrapolation is reported as such (the network then adds nothing)
    gain_plain = cyc["plain"] - cyc["learned"]
    gain_extrap = cyc["extrapolated"] - cyc["learned"]
    print(f"gain over plain {gain_plain:+.2f}, over extrapolated {gain_extrap:+.2f} V-cycles per step"
          + (" (the network adds nothing over the extrapolation)" if gain_extrap == 0 else ""))
    assert gain_plain > 0
    assert gain_extrap >= 0
