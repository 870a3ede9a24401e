"""Batched load steps: instances of uneven size, each on its own stream,
run concurrently by the library's host workers, reproduce their one-by-one
solves bit for bit (the kernels and reductions are deterministic)."""
import numpy as np
import pytest

import pfinputs as PI
from tests.gpu_common import host, require_cuda

pytestmark = pytest.mark.gpu


def _instance(pf, torch, levels, seed, nfrac):
    st = torch.cuda.Stream()
    H = pf.mesh_hierarchy_create(2, (9, 9), levels, 1 / 8, E=1.0, nu=0.3, Gc=1.0, stream=st)
    (nx, ny), h, N = H.levels[-1]
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    pf.fractures_set(H, pf.PF_LINE2D, PI.line_network_2d(seed, nfrac), h, x)
    pf.pressure_set(H, 1e-3)
    return H, x


def test_batch_equals_sequential():
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    spec = [(3, 1, 5), (4, 2, 40), (2, 3, 12), (5, 4, 80), (3, 5, 20)]  # 33^2 .. 129^2
    seq, bat = [], []
    for levels, seed, nf in spec:
        H, x = _instance(pf, torch, levels, seed, nf)
        seq.append((H, x.clone()))
        bat.append((H, x.clone()))
    prm = pf.default_params()
    ref = []
    for H, x in seq:
        ref.append(pf.rmtr_load_step(H, x, prm))
        torch.cuda.synchronize()
    out = pf.rmtr_load_step_batch([H for H, _ in bat], [x for _, x in bat], prm, n_threads=4)
    torch.cuda.synchronize()
    for (Hs, xs), (Hb, xb), r, o in zip(seq, bat, ref, out):
        assert o["status"] == 0 and o["converged"] == 1
        assert o["cycles"] == r["cycles"] and o["energy"] == r["energy"]
        assert np.array_equal(host(xs), host(xb))
