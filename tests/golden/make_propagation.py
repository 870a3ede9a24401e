"""Writes propagation.json: the FP64 oracle on the 2D centred crack (65^2,
two levels, E = 1, nu = 0.3, G_c = 1, l_s = 2h) under a pressure ramp that
crosses the critical pressure, so the crack grows (the propagation regime of
Sec. 5: pressure-driven growth).  Per step: pressure, converged energy,
V-cycles and the number of nodes with c > 1/2 (the crack's extent).
Calls only the oracle and the seeded inputs.  Run from the repository root:
    python tests/golden/make_propagation.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import pfinputs as PI  # noqa: E402
from oracle import pf_oracle as O  # noqa: E402

PRESSURES = [0.5, 1.0, 1.5, 2.0, 2.5, 3.0]


def main():
    Ho = O.Hierarchy(2, (33, 33), 1 / 32, 2, O.Params(E=1.0, nu=0.3, Gc=1.0, p=0.0))
    g = Ho.fine
    x = np.zeros(3 * g.N)
    x[2 * g.N:] = O.rasterize(g, O.LINE2D, PI.centred_crack_2d(), g.h)
    steps = []
    for p in PRESSURES:
        r = O.rmtr_load_step(Ho, x, O.TRParams(rtol=1e-10), p=p)
        assert r.converged
        x = r.x
        steps.append({"p": p, "energy": r.energy, "cycles": r.cycles,
                      "crack_nodes": int(np.sum(x[2 * g.N:] > 0.5))})
    out = {"cite": "Sec. 5 (pressure-driven propagation); FP64 oracle, rtol 1e-10",
           "grid": [65, 65], "levels": 2, "E": 1.0, "nu": 0.3, "Gc": 1.0, "crack": "centred, half-length 0.1",
           "steps": steps}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "propagation.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
