"""Writes field_samples_65.json: one FP64 oracle load step of the 3D
workload's disc network on a 65^3 three-level hierarchy (17^3 -> 33^3 ->
65^3; 20 discs of radius U[0.03, 0.1], E = 1, nu = 0.25, G_c = 1, l_s = 2h,
p = 5e-4 from the fractured state, rtol 1e-12), and the converged fields at
1,500 seeded nodes whose displacements the minimiser determines (a node with
an element that is not fully broken), plus the energy and each field's
max-norm.  A 65^3 field is too large to store whole; the GPU tests compare
these samples.  Calls only the oracle and the seeded inputs.  Run from the
repository root (a few minutes):
    python tests/golden/make_field_samples_65.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import pfinputs as PI  # noqa: E402
from oracle import pf_oracle as O  # noqa: E402


def main():
    Ho = O.Hierarchy(3, (17, 17, 17), 1 / 16, 3, O.Params(E=1.0, nu=0.25, Gc=1.0, p=5e-4))
    g = Ho.fine
    x = np.zeros(4 * g.N)
    x[3 * g.N:] = O.rasterize(g, O.DISC3D, PI.disc_network_3d(PI.SEED_3D_PLAIN, 20), g.h)
    r = O.rmtr_load_step(Ho, x, O.TRParams(rtol=1e-12), p=5e-4)
    assert r.converged
    c = r.x[3 * g.N:]
    conn = g.element_connectivity()
    broken = np.all(c[conn] == 1.0, axis=1)
    determined = np.zeros(g.N, dtype=bool)
    for k in range(conn.shape[1]):
        determined[conn[~broken, k]] = True
    cand = np.where(determined)[0]
    nodes = np.sort(PI.rng(1651).choice(cand, size=1500, replace=False))
    out = {"cite": "Sec. 5.2 3D scenario (disc network), Algorithm 1 load step; FP64 oracle, rtol 1e-12",
           "n_coarse": 17, "levels": 3, "grid": [65, 65, 65], "p": 5e-4, "fractures": 20,
           "seed": PI.SEED_3D_PLAIN, "energy": r.energy, "cycles": r.cycles,
           "nodes": nodes.tolist(),
           "fields": [r.x[f * g.N + nodes].tolist() for f in range(4)],
           "field_max": [float(np.max(np.abs(r.x[f * g.N:(f + 1) * g.N]))) for f in range(4)],
           "undetermined_nodes": int(np.sum(~determined))}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "field_samples_65.json"), "w") as f:
        json.dump(out, f)
    print("energy", r.energy, "cycles", r.cycles, "undetermined", out["undetermined_nodes"])


if __name__ == "__main__":
    main()
