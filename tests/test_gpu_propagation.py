"""The propagation regime (Sec. 5: pressure-driven growth): the 2D centred
crack at 65^2 under a pressure ramp that crosses the critical pressure
(tests/golden/propagation.json, written by the committed oracle script).
The FP64 solver follows the oracle's path: every converged energy to 1e-8
and the crack's extent (nodes with c > 1/2) exactly, growth steps included.
The mixed-precision solver matches that before the crack grows; once it
grows, several local minima can be reached (a bifurcation, so round-off
can choose another branch), and those steps compare the energy and the
crack's extent within bands.  Every step checks the invariants: c_prev <=
c <= 1 bit for bit, the clamped boundary, and the energy decrease against
the step's start."""
import json
import os

import numpy as np
import pytest

import pfinputs as PI
from tests.gpu_common import host, pair, require_cuda

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "propagation.json")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_crack_growth_ramp(precision):
    import torch
    require_cuda()
    import paper_2007_12908_gb300 as pf
    gold = json.load(open(GOLD))
    H, Ho = pair(2, (33, 33), 2, 1 / 32, p=0.0)
    g = Ho.fine
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_LINE2D, PI.centred_crack_2d(), g.h, x)
    bnd = g.boundary_nodes()
    prec = pf.PF_FP64 if precision == "fp64" else pf.PF_FP32
    grown = False
    for step in gold["steps"]:
        c_before = host(x)[2 * g.N:].copy()
        pf.pressure_set(H, step["p"])
        e_start = pf.energy(H, 1, x)
        st = pf.rmtr_load_step(H, x, pf.default_params(precision=prec, rtol=1e-10, max_cycles=400))
        assert st["converged"] == 1, step
        xg = host(x)
        c = xg[2 * g.N:]
        assert np.all(c >= c_before) and np.all(c <= 1.0)
        assert np.all(xg[:g.N][bnd] == 0.0) and np.all(xg[g.N:2 * g.N][bnd] == 0.0)
        assert st["energy"] <= e_start
        crack = int(np.sum(c > 0.5))
        print(precision, step["p"], st["energy"], step["energy"], crack, step["crack_nodes"], st["cycles"])
        grown = grown or step["crack_nodes"] > 2 * gold["steps"][0]["crack_nodes"]
        if precision == "fp64" or not grown:
            assert abs(st["energy"] - step["energy"]) <= 1e-8 * abs(step["energy"])
            assert crack == step["crack_nodes"]
        else:
            assert abs(st["energy"] - step["energy"]) <= 5e-3 * abs(step["energy"])
            assert abs(crack - step["crack_nodes"]) <= 0.1 * step["crack_nodes"]
    H.close()
