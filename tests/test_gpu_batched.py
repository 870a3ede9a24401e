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
    for var in ((1, 2, 3) if dim == 3 else (0, 1, 2, 3, 4)):
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


# ---------------------------------------------------------------- batched operators
_RAGGED = [  # (n_coarse, levels, h_coarse, E, nu, k_res, p): finest grids 3^2 .. 129x9, 3 strips
    ((3, 3), 1, 0.5, 1.0, 0.3, 0.0, 1e-3),
    ((35, 23), 1, 1 / 34, 2.5, 0.25, 1e-3, 4e-3),
    ((17, 17), 3, 1 / 16, 1.0, 0.3, 0.0, 2e-3),
    ((65, 5), 2, 1 / 64, 1.0, 0.3, 0.0, 5e-3),
    ((2, 40), 2, 1 / 39, 1.7, 0.2, 0.0, 0.0),
]


def _ragged_batch(torch, pf):
    from oracle import pf_oracle as O
    from tests.gpu_common import dev, pair
    inst = []
    for k, (nc, L, hc, E, nu, kr, p) in enumerate(_RAGGED):
        H, Ho = pair(2, nc, L, hc, E=E, nu=nu, k_res=kr, p=p)
        g = Ho.fine
        x = PI.random_state(300 + k, 2, g.N, u_scale=1e-3, c_hi=1.0)
        v = PI.random_direction(400 + k, x.size)
        inst.append((H, Ho, x, v, dev(x, torch.float32), dev(v, torch.float32)))
    return inst, pf.Batch([t[0] for t in inst])


def test_batched_hessvec_matches_oracle():
    """One persistent launch over five ragged instances (3^2 to 129x9 nodes,
    their own materials and pressures): every instance's product against
    the oracle's, and the segmented v.Hv against the oracle's dot."""
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from oracle import pf_oracle as O
    from tests.gpu_common import relinf
    inst, B = _ragged_batch(torch, pf)
    vhv = torch.empty(len(inst), dtype=torch.float64, device="cuda")
    ys = B.hessvec([t[4] for t in inst], [t[5] for t in inst], vhv=vhv)
    torch.cuda.synchronize()
    d = host(vhv)
    for k, ((H, Ho, x, v, _, _), y) in enumerate(zip(inst, ys)):
        ho = O.hessvec(Ho.fine, Ho.prm, x, v)
        assert relinf(host(y), ho) <= 2e-5, (k, relinf(host(y), ho))
        scale = float(np.sum(np.abs(v) * np.abs(ho)))
        assert abs(d[k] - float(v @ ho)) <= 2e-5 * scale, k
        # the segmented sum against the FP64 dot of the kernel's own product
        yk = host(y)
        v32 = v.astype(np.float32).astype(np.float64)
        assert abs(d[k] - float(v32 @ yk)) <= 1e-6 * float(np.sum(np.abs(v32 * yk))), k
    B.close()
    for t in inst:
        t[0].close()


def test_batched_hessvec_variants_bitwise_and_pressure():
    """Every launch configuration gives the same bits (node sums in a fixed
    order whatever the warp ranges); a pressure change on a hierarchy is
    picked up by the next call."""
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from oracle import pf_oracle as O
    from tests.gpu_common import relinf
    inst, B = _ragged_batch(torch, pf)
    xs, vs = [t[4] for t in inst], [t[5] for t in inst]
    vhv0 = torch.empty(len(inst), dtype=torch.float64, device="cuda")
    ref = [y.clone() for y in B.hessvec(xs, vs, vhv=vhv0)]
    occ = B.info()["blocks_per_sm"]
    for bps in range(1, occ + 1):
        B.variant_set(bps)
        vhv = torch.empty_like(vhv0)
        ys = B.hessvec(xs, vs, vhv=vhv)
        assert all(torch.equal(a, b) for a, b in zip(ys, ref)), bps
        assert torch.equal(vhv, vhv0), bps
    best, us = B.autotune(xs, vs, [torch.empty_like(v) for v in vs])
    assert 1 <= best <= occ and us[best - 1] == min(u for u in us if u > 0)
    H, Ho, x, v = inst[3][:4]
    pf.pressure_set(H, 2e-2)
    Ho.prm.p = 2e-2
    y = B.hessvec(xs, vs)[3]
    ho = O.hessvec(Ho.fine, Ho.prm, x, v)
    assert relinf(host(y), ho) <= 2e-5
    with pytest.raises(pf.PfError):
        B.hessvec(xs, vs, ys=[xs[0]] + ref[1:])  # Hv aliasing x
    B.close()
    for t in inst:
        t[0].close()


def test_batched_hessvec_strip_edges():
    """Grid widths around the 63-column strips and the 32-lane halves
    (62 .. 65, 94 .. 96, 126 .. 128 nodes, two to four rows) in one launch,
    each against the oracle."""
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from oracle import pf_oracle as O
    from tests.gpu_common import dev, pair, relinf
    widths = [62, 63, 64, 65, 94, 95, 96, 126, 127, 128]
    inst = []
    for k, w in enumerate(widths):
        H, Ho = pair(2, (w, 2 + k % 3), 1, 1 / (w - 1), p=3e-3)
        g = Ho.fine
        x = PI.random_state(800 + k, 2, g.N, u_scale=1e-3, c_hi=1.0)
        v = PI.random_direction(900 + k, x.size)
        inst.append((H, Ho, x, v))
    B = pf.Batch([t[0] for t in inst])
    vhv = torch.empty(len(inst), dtype=torch.float64, device="cuda")
    ys = B.hessvec([dev(t[2], torch.float32) for t in inst], [dev(t[3], torch.float32) for t in inst],
                   vhv=vhv)
    d = host(vhv)
    for k, ((H, Ho, x, v), y) in enumerate(zip(inst, ys)):
        ho = O.hessvec(Ho.fine, Ho.prm, x, v)
        assert relinf(host(y), ho) <= 2e-5, (widths[k], relinf(host(y), ho))
        assert abs(d[k] - float(v @ ho)) <= 2e-5 * float(np.sum(np.abs(v) * np.abs(ho))), widths[k]
    B.close()
    for t in inst:
        t[0].close()


def test_batched_energy_matches_oracle():
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from oracle import pf_oracle as O
    from tests.gpu_common import dev
    inst, B = _ragged_batch(torch, pf)
    E = B.energy([dev(t[2]) for t in inst])
    for k, (H, Ho, x, *_rest) in enumerate(inst):
        eo = O.energy(Ho.fine, Ho.prm, x)
        assert abs(E[k] - eo) <= 1e-10 * abs(eo), k
        e1 = pf.energy(H, H.n_levels - 1, dev(x))
        assert abs(E[k] - e1) <= 1e-12 * abs(e1), k
    B.close()
    for t in inst:
        t[0].close()


def test_batched_energy_non_finite():
    """A NaN in one instance's state makes pf_batch_energy return
    PF_ENONFINITE; the other instances' energies are still written."""
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from oracle import pf_oracle as O
    from tests.gpu_common import dev
    inst, B = _ragged_batch(torch, pf)
    xs = [dev(t[2]) for t in inst]
    xs[2][5] = float("nan")
    with pytest.raises(pf.PfError) as e:
        B.energy(xs)
    assert e.value.status == pf.PF_ENONFINITE
    xs[2][5] = 0.0
    E = B.energy(xs)
    assert all(np.isfinite(E))
    B.close()
    for t in inst:
        t[0].close()


def test_batched_rejects_3d():
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    H3 = pf.mesh_hierarchy_create(3, (3, 3, 3), 1, 0.5)
    with pytest.raises(pf.PfError):
        pf.Batch([H3])
    H3.close()


def test_batched_draw_sampled_against_oracle():
    """Eight instances of the uneven batch draw (two of each size, their
    line networks) in one launch: sampled nodes of a 1025^2 and a 129^2
    instance and their energies against the oracle, and v.Hv of every
    instance against the FP64 dot of its product."""
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from oracle import pf_oracle as O
    from tests.gpu_common import relinf
    sizes, counts = PI.batched_grid_draw(PI.SEED_2D_BATCHED, 64)
    pick = []
    for n in (129, 257, 513, 1025):
        pick += [i for i, s in enumerate(sizes) if s == n][:2]
    Hs, xs, vs, xs64 = [], [], [], []
    for i in pick:
        levels = int(round(np.log2((sizes[i] - 1) / 16))) + 1
        H = pf.mesh_hierarchy_create(2, (17, 17), levels, 1 / 16, E=1.0, nu=0.3, Gc=1.0)
        pf.pressure_set(H, 1e-3)
        (nx, ny), h, N = H.levels[-1]
        x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
        pf.fractures_set(H, pf.PF_LINE2D, PI.line_network_2d(PI.SEED_2D_BATCHED + 1 + i, counts[i]), h, x)
        xr = PI.random_state(500 + i, 2, N, u_scale=1e-3, c_hi=0.5)
        xh = host(x)
        xr[2 * N:] = np.maximum(xr[2 * N:], xh[2 * N:])
        Hs.append(H)
        xs64.append(xr)
        xs.append(torch.from_numpy(xr).cuda().float())
        vs.append(torch.from_numpy(PI.random_direction(600 + i, 3 * N)).cuda().float())
    B = pf.Batch(Hs)
    vhv = torch.empty(len(Hs), dtype=torch.float64, device="cuda")
    ys = B.hessvec(xs, vs, vhv=vhv)
    torch.cuda.synchronize()
    d = host(vhv)
    for k in range(len(Hs)):
        yk, vk = host(ys[k]), host(vs[k])
        assert abs(d[k] - float(vk @ yk)) <= 1e-6 * float(np.sum(np.abs(vk * yk))), k
    E = B.energy([torch.from_numpy(x).cuda() for x in xs64])
    for k in (0, len(Hs) - 1):  # a 129^2 and a 1025^2 instance
        n = sizes[pick[k]]
        levels = int(round(np.log2((n - 1) / 16))) + 1
        Ho = O.Hierarchy(2, (17, 17), 1 / 16, levels, O.Params(E=1.0, nu=0.3, Gc=1.0, p=1e-3))
        g = Ho.fine
        eo = O.energy(g, Ho.prm, xs64[k])
        assert abs(E[k] - eo) <= 1e-10 * abs(eo), (n, E[k], eo)
        nodes = np.unique(np.concatenate([PI.rng(700 + k).choice(g.N, size=300, replace=False),
                                          [0, g.N - 1, g.n[0] - 1, g.N - g.n[0]]]))
        elems = g.elements_touching(nodes)
        idx = np.concatenate([f * g.N + nodes for f in range(3)])
        x32 = host(xs[k]); v32 = host(vs[k])
        ho = O.hessvec(g, Ho.prm, x32, v32, elems)[idx]
        assert relinf(host(ys[k])[idx], ho) <= 2e-5, (n, relinf(host(ys[k])[idx], ho))
    B.close()
    for H in Hs:
        H.close()
