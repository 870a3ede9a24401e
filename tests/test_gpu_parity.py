"""Element kernels, transfers and rasterisation on the GPU against the FP64
oracle, element by element (small grids spanning several CUDA tiles with
ragged tails) and on sampled outputs at the full workload sizes.

Tolerances: FP64 results within 1e-10 (relative, max-norm); FP32 hessvec
within 2e-5 relative (FP32 unit round-off 6e-8 times the O(100) operations
on a dependency chain and the cancellation of the assembled sums)."""
import numpy as np
import pytest

import pfinputs as PI
from oracle import pf_oracle as O
from tests.gpu_common import dev, host, pair, relinf, require_cuda

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5

SMALL = [
    (2, (35, 23), 2, 1 / 34),   # fine 69 x 45: 3 x 6 tiles of 32 x 8, ragged
    (3, (10, 7, 6), 2, 1 / 9),  # fine 19 x 13 x 11: 3 x 2 x 2 tiles of 8^3, ragged
    (2, (2, 2), 1, 1.0),        # a single element
    (3, (2, 2, 2), 1, 1.0),
]


@pytest.fixture(scope="module")
def pf():
    require_cuda()
    import paper_2007_12908_gb300 as m
    return m


@pytest.mark.parametrize("dim,nc,L,hc", SMALL)
@pytest.mark.parametrize("k_res", [0.0, 0.01])
def test_energy_gradient_hessvec_fp64(pf, dim, nc, L, hc, k_res):
    H, Ho = pair(dim, nc, L, hc, E=1.3, nu=0.27, Gc=0.9, k_res=k_res, p=0.05)
    for level in range(L):
        g = Ho.grids[level]
        x = PI.random_state(100 + level, dim, g.N, u_scale=0.05)
        v = PI.random_direction(200 + level, x.size)
        xd, vd = dev(x), dev(v)
        e = pf.energy(H, level, xd)
        eo = O.energy(g, Ho.prm, x)
        assert abs(e - eo) <= TOL64 * abs(eo)
        assert relinf(host(pf.gradient(H, level, xd)), O.gradient(g, Ho.prm, x)) <= TOL64
        ho = O.hessvec(g, Ho.prm, x, v)
        assert relinf(host(pf.hessvec(H, level, xd, vd)), ho) <= TOL64
        # Hessian lagging: stored Gauss-point coefficients, applied twice
        pf.hessvec_lag_set(H, level, xd)
        for _ in range(2):
            assert relinf(host(pf.hessvec_lagged(H, level, vd)), ho) <= TOL64
        a = pf.energy_diff(H, level, xd, dev(0.1 * v))
        ao = O.energy_diff_coeffs(g, Ho.prm, x, 0.1 * v)
        assert np.max(np.abs(a - ao)) <= TOL64 * np.max(np.abs(ao))


@pytest.mark.parametrize("dim,nc,L,hc", SMALL[:2])
def test_hessvec_fp32(pf, dim, nc, L, hc):
    import torch
    H, Ho = pair(dim, nc, L, hc, p=1e-3)
    g = Ho.grids[-1]
    x = PI.random_state(7, dim, g.N, u_scale=1e-2)
    v = PI.random_direction(8, x.size)
    hv = pf.hessvec(H, L - 1, dev(x, torch.float32), dev(v, torch.float32))
    assert hv.dtype == torch.float32
    ho = O.hessvec(g, Ho.prm, x, v)
    assert relinf(host(hv), ho) <= TOL32
    pf.hessvec_lag_set(H, L - 1, dev(x, torch.float32))
    assert relinf(host(pf.hessvec_lagged(H, L - 1, dev(v, torch.float32))), ho) <= TOL32
    gr = pf.gradient(H, L - 1, dev(x, torch.float32))
    assert relinf(host(gr), O.gradient(g, Ho.prm, x)) <= TOL32


def test_hessvec_fp32_element_owned_ragged(pf):
    """The element-owned 3D FP32 product on ragged tiles: a 69 x 73 x 77
    grid (68 x 72 x 76 elements, so the last tile along x and along z is
    part-filled) has 9 x 9 x 10 element tiles of 8^3, enough for the
    element-owned path.  In full against the oracle, plain and lagged, and
    the same bits on a second call."""
    import torch
    H, Ho = pair(3, (18, 19, 20), 3, 1 / 17, nu=0.25, p=2e-3)
    g = Ho.grids[-1]
    assert g.n == (69, 73, 77)
    x = PI.random_state(51, 3, g.N, u_scale=1e-2)
    v = PI.random_direction(52, x.size)
    x32, v32 = dev(x, torch.float32), dev(v, torch.float32)
    ho = O.hessvec(g, Ho.prm, x, v)
    h1 = host(pf.hessvec(H, 2, x32, v32))
    assert relinf(h1, ho) <= TOL32
    assert np.array_equal(h1, host(pf.hessvec(H, 2, x32, v32)))
    pf.hessvec_lag_set(H, 2, x32)
    assert relinf(host(pf.hessvec_lagged(H, 2, v32)), ho) <= TOL32


@pytest.mark.parametrize("dim,nc,L,hc", SMALL[:2])
@pytest.mark.parametrize("k_res", [0.0, 0.01])
@pytest.mark.parametrize("scale", [0.1, 1e-6])
def test_mixed_difference_kernels(pf, dim, nc, L, hc, k_res, scale):
    """FP32 higher-order energy-difference coefficients and the FP32 gradient
    step: their error is relative to the size of the change along s, at any
    step size (no difference of two large totals is formed)."""
    H, Ho = pair(dim, nc, L, hc, E=1.3, nu=0.27, Gc=0.9, k_res=k_res, p=0.05)
    level = L - 1
    g = Ho.grids[level]
    x = PI.random_state(300, dim, g.N, u_scale=0.05)
    s = scale * PI.random_direction(301, x.size)
    go = O.gradient(g, Ho.prm, x)
    a = pf.energy_diff_mixed(H, level, dev(x), dev(s), dev(go))
    ao = O.energy_diff_coeffs(g, Ho.prm, x, s)
    assert abs(a[0] - ao[0]) <= 1e-9 * abs(ao[0])
    assert np.max(np.abs(a[1:] - ao[1:])) <= TOL32 * np.max(np.abs(ao[1:]))
    g_before = O.gradient(g, Ho.prm, x - s)
    y = pf.gradient_step(H, level, dev(x), dev(s), dev(g_before))
    change = go - g_before
    assert np.max(np.abs(host(y) - go)) <= TOL32 * np.max(np.abs(change))


@pytest.mark.parametrize("dim,nc,L,hc", SMALL)
@pytest.mark.parametrize("k_res", [0.0, 0.01])
def test_double_float_gradient_energy(pf, dim, nc, L, hc, k_res):
    """Gradient and energy in double-float arithmetic (two FP32 words,
    about 48 significant bits) against the FP64 oracle."""
    H, Ho = pair(dim, nc, L, hc, E=1.3, nu=0.27, Gc=0.9, k_res=k_res, p=0.05)
    for level in range(L):
        g = Ho.grids[level]
        x = PI.random_state(400 + level, dim, g.N, u_scale=0.05)
        xd = dev(x)
        if g.NE == 1 and dim == 2:  # too few elements for the scratch layout
            with pytest.raises(pf.PfError):
                pf.gradient_df(H, level, xd)
            continue
        assert relinf(host(pf.gradient_df(H, level, xd)), O.gradient(g, Ho.prm, x)) <= 1e-11
        eo = O.energy(g, Ho.prm, x)
        assert abs(pf.energy_df(H, level, xd) - eo) <= 1e-12 * abs(eo)


def test_deterministic(pf):
    H, Ho = pair(3, (10, 7, 6), 2, 1 / 9, p=1e-3)
    g = Ho.grids[-1]
    x = dev(PI.random_state(9, 3, g.N))
    v = dev(PI.random_direction(10, x.numel()))
    a = host(pf.hessvec(H, 1, x, v))
    b = host(pf.hessvec(H, 1, x, v))
    assert np.array_equal(a, b)
    assert pf.energy(H, 1, x) == pf.energy(H, 1, x)


@pytest.mark.parametrize("dim,nc,L,hc", [(2, (6, 5), 3, 0.2), (3, (4, 3, 5), 2, 0.25)])
def test_transfers(pf, dim, nc, L, hc):
    H, Ho = pair(dim, nc, L, hc)
    for c in range(L - 1):
        T = Ho.transfers[c]
        vc = PI.random_direction(11 + c, (dim + 1) * T.coarse.N)
        vf = PI.random_direction(21 + c, (dim + 1) * T.fine.N)
        assert relinf(host(pf.prolong(H, c, dev(vc))), T.prolong(vc)) <= 1e-14
        assert relinf(host(pf.restrict(H, c, dev(vf))), T.restrict(vf)) <= 1e-14
        assert relinf(host(pf.project(H, c, dev(vf))), T.project(vf)) <= 1e-14
        lo = -np.abs(vf)
        hi = np.abs(PI.random_direction(31 + c, vf.size))
        lc, hcb = pf.coarse_bounds(H, c, dev(lo), dev(hi))
        assert np.array_equal(host(lc), T.support_max(lo))
        assert np.array_equal(host(hcb), T.support_min(hi))


def _raster_pair(pf, dim, nc, L, hc, kind, rows):
    import torch
    H, Ho = pair(dim, nc, L, hc)
    g = Ho.fine
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, kind, rows, g.h, x)
    c = host(x)[dim * g.N:]
    co = O.rasterize(g, kind, rows, g.h)
    assert np.array_equal(c, co)
    assert np.array_equal(host(pf.get_c_prev(H)), co)
    assert np.all(host(x)[: dim * g.N] == 0.0)
    return c


def test_raster_centred_crack(pf):
    c = _raster_pair(pf, 2, (33, 33), 2, 1 / 32, pf.PF_LINE2D, PI.centred_crack_2d())
    assert c.sum() == 39


def test_raster_line_network(pf):
    rows = PI.line_network_2d(PI.SEED_2D_BATCHED, 500)
    c = _raster_pair(pf, 2, (65, 65), 3, 1 / 64, pf.PF_LINE2D, rows)
    assert c.sum() > 500


def test_raster_discs_full_size(pf):
    rows = PI.disc_network_3d(PI.SEED_3D_PLAIN, 20)
    c = _raster_pair(pf, 3, (17, 17, 17), 4, 1 / 16, pf.PF_DISC3D, rows)
    assert c.sum() > 1000


def test_raster_boxes_full_size(pf):
    """100 plates of the paper-scale network on the 129^3 grid, bit-exact."""
    rows = PI.box_network_3d(PI.SEED_3D_PAPER, 100)
    c = _raster_pair(pf, 3, (17, 17, 17), 4, 1 / 16, pf.PF_BOX3D, rows)
    assert c.sum() > 10000


def _sampled_nodes(g, n, seed):
    r = PI.rng(seed)
    nodes = r.choice(g.N, size=n, replace=False)
    # always include corners and a boundary face node
    return np.unique(np.concatenate([nodes, [0, g.N - 1, g.n[0] // 2]]))


@pytest.mark.parametrize("dim,nc,L,hc", [(3, (17, 17, 17), 4, 1 / 16), (2, (65, 65), 5, 1 / 64)])
def test_full_size_sampled(pf, dim, nc, L, hc):
    """Workload sizes (129^3 four levels; 1025^2): the energy in full, the
    gradient and hessvec at sampled nodes from the oracle's elements around
    them, FP64 and FP32."""
    import torch
    H, Ho = pair(dim, nc, L, hc, nu=0.25 if dim == 3 else 0.3, p=5e-3)
    g = Ho.fine
    x = PI.random_state(41, dim, g.N, u_scale=1e-3, c_hi=1.0)
    v = PI.random_direction(42, x.size)
    xd, vd = dev(x), dev(v)
    e = pf.energy(H, L - 1, xd)
    eo = O.energy(g, Ho.prm, x)
    assert abs(e - eo) <= TOL64 * abs(eo)
    nodes = _sampled_nodes(g, 400, 43)
    elems = g.elements_touching(nodes)
    idx = np.concatenate([f * g.N + nodes for f in range(dim + 1)])
    go = O.gradient(g, Ho.prm, x, elems)[idx]
    ho = O.hessvec(g, Ho.prm, x, v, elems)[idx]
    assert relinf(host(pf.gradient(H, L - 1, xd))[idx], go) <= TOL64
    assert relinf(host(pf.hessvec(H, L - 1, xd, vd))[idx], ho) <= TOL64
    pf.hessvec_lag_set(H, L - 1, xd)
    assert relinf(host(pf.hessvec_lagged(H, L - 1, vd))[idx], ho) <= TOL64
    h32 = pf.hessvec(H, L - 1, xd.float(), vd.float())
    assert relinf(host(h32)[idx], ho) <= TOL32
