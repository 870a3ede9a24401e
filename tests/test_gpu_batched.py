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


@pytest.mark.parametrize("dim,nc,L,hc", [(2, (35, 23), 2, 1 / 34), (3, (10, 7, 6), 3, 0.125)])
def test_every_tile_variant_matches_oracle(dim, nc, L, hc):
    """Each tile variant of the FP32 Hessian product (the autotuner's
    candidates) against the oracle on ragged grids, and each deterministic."""
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from oracle import pf_oracle as O
    from tests.gpu_common import dev, pair, relinf
    H, Ho = pair(dim, nc, L, hc, nu=0.25 if dim == 3 else 0.3, p=5e-3)
    g = Ho.fine
    x = PI.random_state(91, dim, g.N, u_scale=1e-3, c_hi=1.0)
    v = PI.random_direction(92, x.size)
    ho = O.hessvec(g, Ho.prm, x, v)
    xd, vd = dev(x, torch.float32), dev(v, torch.float32)
    for var in ((1, 2, 3) if dim == 3 else (0, 1, 2, 3)):
        pf.tile_variant_set(H, L - 1, var)
        assert pf.tile_variant_get(H, L - 1) == var
        a = pf.hessvec(H, L - 1, xd, vd)
        b = pf.hessvec(H, L - 1, xd, vd)
        assert torch.equal(a, b), var
        assert relinf(host(a), ho) <= 2e-5, (var, relinf(host(a), ho))
    H.close()


def test_autotune_keeps_the_solution():
    """pf_autotune picks a variant per level from measured times, and a load
    step after it converges to the energy of the untuned hierarchy."""
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    H, x = _instance(pf, torch, 5, 7, 60)  # 129^2 finest
    x0 = x.clone()
    prm = pf.default_params(precision=pf.PF_FP32)
    ref = pf.rmtr_load_step(H, x0, prm)
    var, us = pf.autotune(H)
    assert len(var) == H.n_levels
    for l, (v, t) in enumerate(zip(var, us)):
        assert t[v] > 0 and t[v] == min(u for u in t if u > 0)
    got = pf.rmtr_load_step(H, x, prm)
    assert got["converged"] == 1
    assert abs(got["energy"] - ref["energy"]) <= 1e-8 * abs(ref["energy"])


@pytest.mark.parametrize("size", [129, 1025])
def test_batch_draw_instance_matches_oracle(size):
    """An instance of the uneven 2D batch (the config's seeded draw, its
    line-fracture network) against the oracle: rasterisation bit for bit,
    the energy in full, gradient and Hessian products at sampled nodes."""
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from oracle import pf_oracle as O
    from tests.gpu_common import dev, pair, relinf
    sizes, counts = PI.batched_grid_draw(PI.SEED_2D_BATCHED, 64)
    i = sizes.index(size)
    levels = int(round(np.log2((size - 1) / 16))) + 1
    H, Ho = pair(2, (17, 17), levels, 1 / 16, p=1e-3)
    g = Ho.fine
    rows = PI.line_network_2d(PI.SEED_2D_BATCHED + 1 + i, counts[i])
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_LINE2D, rows, g.h, x)
    c = O.rasterize(g, O.LINE2D, rows, g.h)
    assert np.array_equal(host(x)[2 * g.N:], c)
    xs = PI.random_state(93, 2, g.N, u_scale=1e-3, c_hi=1.0)
    xs[2 * g.N:] = np.maximum(xs[2 * g.N:], c)
    v = PI.random_direction(94, xs.size)
    xd, vd = dev(xs), dev(v)
    e = pf.energy(H, levels - 1, xd)
    assert abs(e - O.energy(g, Ho.prm, xs)) <= 1e-10 * abs(e)
    nodes = np.unique(np.concatenate([PI.rng(95).choice(g.N, size=300, replace=False), [0, g.N - 1]]))
    elems = g.elements_touching(nodes)
    idx = np.concatenate([f * g.N + nodes for f in range(3)])
    assert relinf(host(pf.gradient(H, levels - 1, xd))[idx], O.gradient(g, Ho.prm, xs, elems)[idx]) <= 1e-10
    ho = O.hessvec(g, Ho.prm, xs, v, elems)[idx]
    assert relinf(host(pf.hessvec(H, levels - 1, xd, vd))[idx], ho) <= 1e-10
    assert relinf(host(pf.hessvec(H, levels - 1, xd.float(), vd.float()))[idx], ho) <= 2e-5
    H.close()
