"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: each checks a closed form, an
exactness property, an independent assembly, or a number the paper prints.
"""
import json
import math
import os

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg  # noqa: F401
import pytest

import pfinputs as PI
from oracle import pf_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _fd5(f, tau):
    """5-point central difference; exact for polynomials of degree <= 4."""
    return (f(-2 * tau) - 8 * f(-tau) + 8 * f(tau) - f(2 * tau)) / (12 * tau)


CASES = [
    (2, (4, 5), 0.25),
    (2, (6, 3), 0.2),
    (3, (3, 4, 3), 0.25),
]


def _prm(k=0.0):
    return O.Params(E=1.3, nu=0.27, Gc=0.9, ls=0.4, p=0.07, k_res=k)


# ---------------------------------------------------------------- sizes
def test_dof_counts_printed_in_paper():
    gold = json.load(open(os.path.join(GOLD, "dof_counts.json")))
    for case in gold["cases"]:
        sizes = O.level_sizes(case["n_coarse"], case["levels"])
        fine = sizes[-1]
        dofs = (case["dim"] + 1) * int(np.prod(fine))
        assert dofs == case["dofs"], case["cite"]
        assert all(v == 8 * c - 7 for v, c in zip(fine, case["n_coarse"]))


def test_workload_sizes():
    # 3D 129^3 four-level hierarchy 17^3 -> 129^3, 2D 65^2 two-level 33^2 -> 65^2
    assert O.level_sizes((17, 17, 17), 4) == [(17,) * 3, (33,) * 3, (65,) * 3, (129,) * 3]
    assert 4 * 129 ** 3 == 8586756
    assert O.level_sizes((33, 33), 2)[-1] == (65, 65)


# ---------------------------------------------------------------- P1 patch test
@pytest.mark.parametrize("dim", [2, 3])
def test_patch_affine_u_constant_c(dim):
    n = (5, 4, 3)[:dim]
    h = 0.2
    g = O.Grid(dim, n, h)
    prm = O.Params(E=2.0, nu=0.2, Gc=1.5, ls=0.3, p=0.05)
    A = np.array([[0.011, -0.004, 0.006], [0.003, 0.008, -0.002], [0.001, 0.005, -0.007]])[:dim, :dim]
    c0 = 0.37
    X = g.node_coords() * h
    x = np.empty((dim + 1) * g.N)
    for i in range(dim):
        x[i * g.N:(i + 1) * g.N] = A[i] @ X
    x[dim * g.N:] = c0
    eps = 0.5 * (A + A.T)
    tr = np.trace(A)
    psi = 0.5 * prm.lam * tr ** 2 + prm.mu * np.sum(eps * eps)
    vol = np.prod([(v - 1) * h for v in n])
    E_exact = vol * ((1 - c0) ** 2 * (psi + prm.p * tr) + prm.Gc * c0 ** 2 / (2 * prm.ls))
    assert abs(O.energy(g, prm, x) - E_exact) <= 1e-13 * abs(E_exact)
    gr = O.gradient(g, prm, x)
    interior = ~g.boundary_nodes()
    for i in range(dim):
        assert np.max(np.abs(gr[i * g.N:(i + 1) * g.N][interior])) < 1e-15
    gc_exact = h ** dim * (-2 * (1 - c0) * (psi + prm.p * tr) + prm.Gc * c0 / prm.ls)
    np.testing.assert_allclose(gr[dim * g.N:][interior], gc_exact, rtol=1e-12)


# ---------------------------------------------------------------- P2 exact FD
@pytest.mark.parametrize("dim,n,h", CASES)
@pytest.mark.parametrize("k", [0.0, 0.02])
def test_gradient_is_exact_fd_of_energy(dim, n, h, k):
    g = O.Grid(dim, n, h)
    prm = _prm(k)
    x = PI.random_state(11, dim, g.N, u_scale=0.3)
    for seed in (1, 2, 3):
        v = PI.random_direction(seed, x.size)
        fd = _fd5(lambda t: O.energy(g, prm, x + t * v), 1e-3)
        an = O.gradient(g, prm, x) @ v
        assert abs(fd - an) <= 1e-11 * max(1.0, abs(an))


@pytest.mark.parametrize("dim,n,h", CASES)
def test_hessvec_is_exact_fd_of_gradient(dim, n, h):
    g = O.Grid(dim, n, h)
    prm = _prm(0.01)
    x = PI.random_state(12, dim, g.N, u_scale=0.3)
    v = PI.random_direction(4, x.size)
    fd = _fd5(lambda t: O.gradient(g, prm, x + t * v), 1e-3)
    hv = O.hessvec(g, prm, x, v)
    assert np.max(np.abs(fd - hv)) <= 1e-11 * np.max(np.abs(hv))


# ---------------------------------------------------------------- P3 symmetry
@pytest.mark.parametrize("dim,n,h", CASES)
def test_hessian_symmetry(dim, n, h):
    g = O.Grid(dim, n, h)
    prm = _prm()
    x = PI.random_state(13, dim, g.N, u_scale=0.3)
    v = PI.random_direction(5, x.size)
    w = PI.random_direction(6, x.size)
    a = w @ O.hessvec(g, prm, x, v)
    b = v @ O.hessvec(g, prm, x, w)
    assert abs(a - b) <= 1e-13 * max(abs(a), 1.0)


# ---------------------------------------------------------------- P4 dense Hessian
@pytest.mark.parametrize("dim,n", [(2, (3, 3)), (2, (4, 4)), (3, (3, 3, 3))])
def test_brute_force_dense_hessian(dim, n):
    g = O.Grid(dim, n, 0.5)
    prm = _prm(0.0)
    x = PI.random_state(14, dim, g.N, u_scale=0.3)
    D = O.dense_hessian(g, prm, x)
    nd = x.size
    cols = np.empty((nd, nd))
    for j in range(nd):
        e = np.zeros(nd)
        e[j] = 1.0
        cols[:, j] = O.hessvec(g, prm, x, e)
    scale = np.max(np.abs(D))
    assert np.max(np.abs(cols - D)) <= 1e-13 * scale
    assert np.max(np.abs(D - D.T)) <= 1e-14 * scale
    for j in range(0, nd, max(1, nd // 7)):
        e = np.zeros(nd)
        e[j] = 1.0
        fd = _fd5(lambda t: O.gradient(g, prm, x + t * e), 1e-3)
        assert np.max(np.abs(fd - D[:, j])) <= 1e-10 * scale


# ---------------------------------------------------------------- quartic reduction
@pytest.mark.parametrize("dim,n,h", CASES)
def test_energy_difference_polynomial(dim, n, h):
    g = O.Grid(dim, n, h)
    prm = _prm(0.03)
    x = PI.random_state(15, dim, g.N, u_scale=0.3)
    s = PI.random_direction(7, x.size, 0.4)
    a = O.energy_diff_coeffs(g, prm, x, s)
    # a1 = grad.s, 2 a2 = s.Hs ; the full sum equals the plain difference
    assert abs(a[0] - O.gradient(g, prm, x) @ s) <= 1e-13 * max(1, abs(a[0]))
    assert abs(2 * a[1] - s @ O.hessvec(g, prm, x, s)) <= 1e-13 * max(1, abs(a[1]))
    for t in (0.3, 1.0, -0.7):
        direct = O.energy(g, prm, x + t * s) - O.energy(g, prm, x)
        poly = a[0] * t + a[1] * t ** 2 + a[2] * t ** 3 + a[3] * t ** 4
        assert abs(direct - poly) <= 1e-12 * max(1, abs(direct))


def test_energy_difference_resolves_tiny_steps():
    g = O.Grid(2, (9, 9), 1 / 8)
    prm = _prm()
    x = PI.random_state(16, 2, g.N, u_scale=0.1)
    s = 1e-9 * PI.random_direction(8, x.size)
    lin = O.gradient(g, prm, x) @ s + 0.5 * s @ O.hessvec(g, prm, x, s)
    d = O.energy_diff(g, prm, x, s)
    assert abs(d - lin) <= 1e-9 * abs(lin)


# ---------------------------------------------------------------- transfers
@pytest.mark.parametrize("dim,nc", [(2, (3, 4)), (3, (3, 3, 4))])
def test_prolongation_reproduces_linear_fields(dim, nc):
    hc = 0.5
    gc = O.Grid(dim, nc, hc)
    gf = O.Grid(dim, tuple(2 * v - 1 for v in nc), hc / 2)
    T = O.Transfer(gc, gf)
    coef = np.array([0.3, -1.2, 0.7, 2.0])
    def lin(grid):
        X = grid.node_coords() * grid.h
        f = coef[dim] + sum(coef[k] * X[k] for k in range(dim))
        return np.concatenate([f] * (dim + 1))
    np.testing.assert_allclose(T.prolong(lin(gc)), lin(gf), atol=1e-14)
    # P preserves constants and maps [0,1] into [0,1]
    one_f = np.ones((dim + 1) * gf.N)
    np.testing.assert_allclose(T.project(one_f), 1.0, atol=1e-15)
    r = PI.rng(3).uniform(0, 1, size=(dim + 1) * gf.N)
    pr = T.project(r)
    assert pr.min() >= 0.0 and pr.max() <= 1.0


def test_restriction_is_adjoint_and_weights():
    gc = O.Grid(2, (4, 3), 0.5)
    gf = O.Grid(2, (7, 5), 0.25)
    T = O.Transfer(gc, gf)
    a = PI.random_direction(1, 3 * gf.N)
    b = PI.random_direction(2, 3 * gc.N)
    assert abs(T.restrict(a) @ b - a @ T.prolong(b)) < 1e-13
    # 1D weights 1/2, 1, 1/2: interior coarse node of R 1 sums to 2 per axis
    rs = T.restrict(np.ones(3 * gf.N))[: gc.N].reshape(3, 4)
    assert rs[1, 1] == 4.0 and rs[0, 0] == 1.5 * 1.5 and rs[0, 1] == 1.5 * 2


def test_coarse_feasible_set_keeps_prolongated_corrections_feasible():
    gc = O.Grid(3, (3, 4, 3), 0.5)
    gf = O.Grid(3, (5, 7, 5), 0.25)
    T = O.Transfer(gc, gf)
    r = PI.rng(9)
    lo_f = -r.uniform(0, 1, size=4 * gf.N)
    hi_f = r.uniform(0, 1, size=4 * gf.N)
    lo_f[r.uniform(size=lo_f.size) < 0.2] = 0.0
    lo_c = T.support_max(lo_f)
    hi_c = T.support_min(hi_f)
    assert np.all(lo_c <= 0) and np.all(hi_c >= 0)
    for _ in range(20):
        sc = lo_c + (hi_c - lo_c) * r.uniform(size=lo_c.size)
        sf = T.prolong(sc)
        assert np.all(sf >= lo_f - 1e-15) and np.all(sf <= hi_f + 1e-15)


# ---------------------------------------------------------------- rasterisation
def test_centred_crack_band_covers_three_rows():
    g = O.Grid(2, (65, 65), 1 / 64)
    c = O.rasterize(g, O.LINE2D, PI.centred_crack_2d(), g.h).reshape(65, 65)
    rows = np.where(c.any(axis=1))[0]
    cols = np.where(c.any(axis=0))[0]
    assert list(rows) == [31, 32, 33]
    assert list(cols) == list(range(26, 39))
    assert c.sum() == 39


def test_disc_rasterisation_counts_lattice_points():
    g = O.Grid(3, (11, 11, 11), 0.1)
    disc = np.array([[0.5, 0.5, 0.52, 0.0, 0.0, 1.0, 0.21]])
    c = O.rasterize(g, O.DISC3D, disc, g.h).reshape(11, 11, 11)
    # planes z = 0.5, 0.6 lie within h of 0.52; 13 lattice points of the
    # 0.1-spaced grid lie within radius 0.21 of the axis
    assert list(np.where(c.any(axis=(1, 2)))[0]) == [5, 6]
    assert c.sum() == 26


def test_box_rasterisation_counts_lattice_points():
    """An axis-aligned plate (normal z, sides along x and y) centred on a
    node of the 1/64 grid: the band |dz| <= h holds 3 planes, |dx| <= 0.1
    holds 2 floor(6.4) + 1 = 13 columns and |dy| <= 0.05 holds
    2 floor(3.2) + 1 = 7 rows: 273 nodes.  Rotating the in-plane axes by 90
    degrees exchanges the two extents (same count, transposed footprint);
    tilting the plate onto the x-z plane moves the band to 3 y-rows."""
    g = O.Grid(3, (65, 65, 65), 1 / 64)
    box = np.array([[0.5, 0.5, 0.5, 0, 0, 1, 1, 0, 0, 0, 1, 0, 0.1, 0.05]], dtype=float)
    c = O.rasterize(g, O.BOX3D, box, g.h).reshape(65, 65, 65)  # [z, y, x]
    assert c.sum() == 273
    assert list(np.where(c.any(axis=(1, 2)))[0]) == [31, 32, 33]
    assert list(np.where(c.any(axis=(0, 1)))[0]) == list(range(26, 39))
    assert list(np.where(c.any(axis=(0, 2)))[0]) == list(range(29, 36))
    rot = box.copy()
    rot[0, 6:12] = [0, 1, 0, -1, 0, 0]
    cr = O.rasterize(g, O.BOX3D, rot, g.h).reshape(65, 65, 65)
    assert cr.sum() == 273 and np.array_equal(cr, np.transpose(c, (0, 2, 1)))
    tilt = box.copy()
    tilt[0, 3:12] = [0, 1, 0, 1, 0, 0, 0, 0, 1]
    ct = O.rasterize(g, O.BOX3D, tilt, g.h).reshape(65, 65, 65)
    assert ct.sum() == 273 and list(np.where(ct.any(axis=(0, 2)))[0]) == [31, 32, 33]


# ---------------------------------------------------------------- solver pins
def _closed_form_profile(m, h, ls):
    """Exact minimiser of the 1D Q1 AT2 energy right of a c = 1 band:
    interior rows give c_k = A r^k + B r^-k with r + 1/r set by the Q1 mass
    (h/6)[2 1;1 2] and stiffness (1/h)[1 -1;-1 1]; the domain edge carries
    the natural (half-stencil) row."""
    al = h / (6 * ls) - ls / h
    be = 4 * h / (6 * ls) + 2 * ls / h
    s = -be / al
    r = (s - math.sqrt(s * s - 4)) / 2
    # m + 1 nodes from the band edge (c = 1) to the domain edge
    # edge row: (h/(6ls))(c_{m-1} + 2 c_m) + (ls/h)(c_m - c_{m-1}) = 0
    k = np.arange(m + 1)
    ea = r ** k
    eb = r ** (-k.astype(float))
    def edge(v):
        return h / (6 * ls) * (v[m - 1] + 2 * v[m]) + ls / h * (v[m] - v[m - 1])
    M = np.array([[1.0, 1.0], [edge(ea), edge(eb)]])
    A, B = np.linalg.solve(M, np.array([1.0, 0.0]))
    return A * ea + B * eb, r


def test_closed_form_r_for_ls_2h():
    _, r = _closed_form_profile(14, 0.1, 0.2)
    assert abs(r + 1 / r - 52 / 23) < 1e-14


@pytest.mark.parametrize("model", [O.FIRST_ORDER, O.GALERKIN])
def test_pure_phase_field_matches_1d_closed_form(model):
    prm = O.Params(E=1.0, nu=0.3, Gc=1.0)
    H = O.Hierarchy(2, (17, 3), 1 / 16, 2, prm)
    g = H.fine
    # a vertical crack through the whole domain, offset by h/4 so that no
    # node sits exactly on the band edge
    c0 = O.rasterize(g, O.LINE2D, np.array([[0.5 + 0.25 * g.h, 0.5, math.pi / 2, 10.0]]), g.h)
    x = np.zeros(3 * g.N)
    x[2 * g.N:] = c0
    band = np.where(c0.reshape(g.n[1], g.n[0])[0] > 0)[0]
    assert list(band) == [16, 17]
    res = O.rmtr_load_step(H, x, O.TRParams(coarse_model=model), p=0.0)
    assert res.converged
    c = res.x[2 * g.N:].reshape(g.n[1], g.n[0])
    right, _ = _closed_form_profile(g.n[0] - 1 - band[-1], g.h, prm.ls)
    left, _ = _closed_form_profile(band[0], g.h, prm.ls)
    for row in c:
        np.testing.assert_allclose(row[band[-1]:], right, rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(row[: band[0] + 1][::-1], left, rtol=1e-8, atol=1e-12)
    assert np.all(res.x[: 2 * g.N] == 0.0)


def _sneddon_run(model):
    prm = O.Params(E=1.0, nu=0.3, Gc=1.0)
    H = O.Hierarchy(2, (33, 33), 1 / 32, 2, prm)
    g = H.fine
    c0 = O.rasterize(g, O.LINE2D, PI.centred_crack_2d(), g.h)
    x = np.zeros(3 * g.N)
    x[2 * g.N:] = c0
    e0 = O.energy(g, H.prm, x)
    res = O.rmtr_load_step(H, x, O.TRParams(coarse_model=model), p=1e-3)
    return H, c0, e0, res


@pytest.mark.slow
def test_sneddon_opening_and_invariants():
    gold = json.load(open(os.path.join(GOLD, "sneddon.json")))
    H, c0, e0, res = _sneddon_run(O.FIRST_ORDER)
    g = H.fine
    assert res.converged
    uy = res.x[g.N:2 * g.N].reshape(65, 65)
    cod = uy[34, 32] - uy[30, 32]
    assert cod > 0  # the pressure opens the crack (sign reading of eq. pressurized)
    assert abs(cod / gold["w_centre"] - 1) < gold["rel_band"]
    # opening profile follows sqrt(a^2 - x^2) in shape along the crack
    xs = np.arange(27, 38)
    w = uy[34, xs] - uy[30, xs]
    ref = np.sqrt(np.maximum(0.1 ** 2 - (xs / 64 - 0.5) ** 2, 0))
    assert np.corrcoef(w, ref)[0, 1] > 0.98
    # P7 invariants: bounds bit for bit, clamped boundary exactly zero, decrease
    c = res.x[2 * g.N:]
    assert np.all(c >= c0) and np.all(c <= 1.0)
    bnd = g.boundary_nodes()
    assert np.all(res.x[: g.N][bnd] == 0.0) and np.all(res.x[g.N:2 * g.N][bnd] == 0.0)
    assert res.energy < e0


# ---------------------------------------------------------------- coherence (c13)
def test_level_model_coherence():
    prm = O.Params(E=1.0, nu=0.3, Gc=1.0, p=1e-3)
    H = O.Hierarchy(2, (5, 5), 1 / 4, 3, prm)
    g = H.fine
    x = PI.random_state(21, 2, g.N, u_scale=1e-2, c_hi=0.5)
    fine = O.LevelModel(H, 2, x)
    T = H.transfers[1]
    x0c = T.project(x)
    Rg = T.restrict(fine.grad(x))
    dg = Rg - H.df(1, x0c)
    mid = O.LevelModel(H, 1, x0c, finer=fine, dg=dg, kind=O.GALERKIN)
    np.testing.assert_allclose(mid.grad(x0c), Rg, rtol=1e-12, atol=1e-16)
    assert mid.value(x0c) == H.f(1, x0c)
    v = PI.random_direction(3, x0c.size)
    np.testing.assert_allclose(mid.Hlag(v), T.restrict(fine.Hlag(T.prolong(v))), rtol=1e-12, atol=1e-16)
    # recursion to the next level: model Hessian = R R H I I
    T0 = H.transfers[0]
    y0 = T0.project(x0c)
    coarse = O.LevelModel(H, 0, y0, finer=mid, dg=T0.restrict(mid.grad(x0c)) - H.df(0, y0), kind=O.GALERKIN)
    w = PI.random_direction(4, y0.size)
    ref = T0.restrict(T.restrict(H.d2f(2, x, T.prolong(T0.prolong(w)))))
    np.testing.assert_allclose(coarse.Hlag(w), ref, rtol=1e-11, atol=1e-16)
    # diff() agrees with value differences for an O(1) step
    s = PI.random_direction(5, x0c.size, 1e-2)
    assert abs(mid.diff(x0c + s, s) - (mid.value(x0c + 2 * s) - mid.value(x0c + s))) < 1e-12


# ---------------------------------------------------------------- subproblem
# Closed forms of the box-constrained quadratic subproblem
# min g.s + 1/2 s.Hs over lo <= s <= hi (the TR subproblem of Sec. 3):
# with H = diag(h), h > 0, the problem separates and its minimiser is
# clamp(-g/h, lo, hi) coordinate by coordinate.
def _diag_qp(seed, n):
    r = PI.rng(seed)
    h = r.uniform(0.5, 4.0, n)
    g = r.normal(0.0, 1.0, n)
    lo = -r.uniform(0.05, 1.0, n)
    hi = r.uniform(0.05, 1.0, n)
    return g, h, lo, hi


@pytest.mark.parametrize("g,h,lo,hi", [
    (1.0, 2.0, -1.0, 1.0),    # interior minimiser -0.5
    (-3.0, 1.0, -1.0, 2.0),   # interior minimiser 3 cut at hi = 2
    (4.0, 0.5, -1.5, 0.3),    # minimiser -8 cut at lo = -1.5
    (0.2, 10.0, -1.0, 1.0),   # small step -0.02
])
def test_subproblem_1d_closed_form(g, h, lo, hi):
    tr = O.TRParams()
    s = O.solve_subproblem(np.array([g]), lambda v: h * v, np.array([lo]), np.array([hi]),
                           delta=10.0, cg_max=10, tr=tr)
    assert abs(s[0] - min(max(-g / h, lo), hi)) <= 1e-14


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_subproblem_separable_box_minimiser(seed):
    """Diagonal H, bounds wider than the radius delta, some unconstrained
    minimisers outside the box.  The Cauchy point -delta g / max|g| is then
    interior; one Jacobi-preconditioned CG iteration (M^-1 H = I) reaches
    -g/h and leaves the box; the projected search clamps it, which is the
    exact separable minimiser; the restart finds a zero residual on the free
    set.  (A coordinate that reaches a bound stays fixed for the rest of the
    subproblem, so the bounds are kept clear of the Cauchy point.)"""
    n = 24
    r = PI.rng(seed)
    h = r.uniform(0.5, 4.0, n)
    g = r.normal(0.0, 1.0, n)
    delta = 0.01
    lo = -r.uniform(0.05, 1.0, n)
    hi = r.uniform(0.05, 1.0, n)
    exact = np.clip(-g / h, lo, hi)
    assert 3 <= np.sum(exact != -g / h) <= n - 3
    s = O.solve_subproblem(g, lambda v: h * v, lo, hi, delta=delta, cg_max=500, tr=O.TRParams(),
                           minv=1.0 / h)
    assert np.all(s >= lo) and np.all(s <= hi)
    assert np.max(np.abs(s - exact)) <= 1e-12


def test_subproblem_backtracks_a_bent_cauchy_path():
    """SPD H = [[1, -0.9], [-0.9, 1]], g = (1, 1), lo = (-10, -0.1): the
    curvature along -g gives t = 10, and projecting -t g onto the box bends
    the path so that the model rises (m = 39 at t = 10, 7.0 at 5, 0.3 at
    2.5); backtracking accepts t = 1.25, and CG on the one free coordinate
    then reaches the KKT point (-1.09, -0.1): d m / d s_0 = 0 there, and
    s_1 sits on its lower bound with d m / d s_1 = 1.881 > 0."""
    H = np.array([[1.0, -0.9], [-0.9, 1.0]])
    g = np.array([1.0, 1.0])
    lo, hi = np.array([-10.0, -0.1]), np.array([10.0, 10.0])
    s = O.solve_subproblem(g, lambda v: H @ v, lo, hi, delta=100.0, cg_max=50, tr=O.TRParams(),
                           minv=np.ones(2))
    assert np.max(np.abs(s - np.array([-1.09, -0.1]))) <= 1e-12
    assert g @ s + 0.5 * s @ H @ s < 0.0


def test_subproblem_radius_caps_the_cauchy_step():
    """A box tighter than the unconstrained step (the TR radius delta enters
    as the box |s_i| <= delta): every coordinate ends on the bound that -g
    points to, as the separable minimiser says."""
    g, h, _, _ = _diag_qp(5, 16)
    delta = 1e-3
    lo, hi = -delta * np.ones(16), delta * np.ones(16)
    s = O.solve_subproblem(g, lambda v: h * v, lo, hi, delta=delta, cg_max=50, tr=O.TRParams(),
                           minv=1.0 / h)
    exact = np.clip(-g / h, lo, hi)
    assert np.all(np.abs(-g / h) > delta)  # every step is cut
    assert np.max(np.abs(s - exact)) <= 1e-15


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_a_planted_sign_error(monkeypatch):
    g = O.Grid(2, (4, 4), 0.25)
    prm = _prm()
    x = PI.random_state(31, 2, g.N, u_scale=0.3)
    v = PI.random_direction(1, x.size)
    orig = O._degradation

    def wrong(prm_, c):
        gg, dg, ddg = orig(prm_, c)
        return gg, -dg, ddg

    monkeypatch.setattr(O, "_degradation", wrong)
    fd = _fd5(lambda t: O.energy(g, prm, x + t * v), 1e-3)
    assert abs(fd - O.gradient(g, prm, x) @ v) > 1e-6


def test_pins_catch_a_dropped_pressure_term(monkeypatch):
    g = O.Grid(2, (3, 3), 0.5)
    prm = _prm()
    x = PI.random_state(32, 2, g.N, u_scale=0.3)
    D = O.dense_hessian(g, prm, x)
    # plant: hessvec forgets the pressure (p = 0 inside hessvec only)
    real_hessvec = O.hessvec

    def bad_hessvec(grid, prm_, xx, vv, elems=None):
        q = O.Params(prm_.E, prm_.nu, prm_.Gc, prm_.ls, 0.0, prm_.k_res)
        return real_hessvec(grid, q, xx, vv, elems)

    monkeypatch.setattr(O, "hessvec", bad_hessvec)
    e = np.zeros(x.size)
    e[2 * g.N + 4] = 1.0
    assert np.max(np.abs(O.hessvec(g, prm, x, e) - D[:, 2 * g.N + 4])) > 1e-4


def test_pins_catch_a_planted_model_sign_error(monkeypatch):
    """The subproblem's acceptance tests with the quadratic term of the model
    negated accept the first, rising trial of the bent Cauchy path."""
    monkeypatch.setattr(O, "_model", lambda g, s, Hs: float(g @ s) - 0.5 * float(s @ Hs))
    with pytest.raises(AssertionError):
        test_subproblem_backtracks_a_bent_cauchy_path()


def test_pins_catch_a_planted_projection_error(monkeypatch):
    """A projection that forgets the upper bounds fails the separable pin."""
    monkeypatch.setattr(O, "proj_box", lambda s, lo, hi: np.maximum(s, lo))
    with pytest.raises(AssertionError):
        test_subproblem_separable_box_minimiser(1)


# ---------------------------------------------------------------- Jacobi diagonal
@pytest.mark.parametrize("dim,n,k", [(2, (3, 3), 0.0), (2, (4, 4), 0.05), (3, (3, 3, 3), 0.0)])
def test_hess_diag_is_the_dense_hessian_diagonal(dim, n, k):
    """The subproblem's Jacobi preconditioner must be the diagonal of the
    Hessian (eq. model_qp's H): compared with the independently assembled
    dense Hessian of P4, entry by entry, with the pressure term active."""
    g = O.Grid(dim, n, 0.5)
    prm = _prm(k)
    x = PI.random_state(41, dim, g.N, u_scale=0.3)
    D = np.diag(O.dense_hessian(g, prm, x))
    d = O.hess_diag(g, prm, x)
    assert np.max(np.abs(d - D)) <= 1e-13 * np.max(np.abs(D))


def test_pins_catch_a_planted_diagonal_error(monkeypatch):
    """A Jacobi diagonal that forgets g'' (psi + p div u) in its c entries
    fails the dense-diagonal pin (the dense Hessian builds its own g'')."""
    g = O.Grid(2, (3, 3), 0.5)
    prm = _prm()
    x = PI.random_state(41, 2, g.N, u_scale=0.3)
    D = np.diag(O.dense_hessian(g, prm, x))
    orig = O._degradation

    def no_ddg(prm_, c):
        gg, dg, ddg = orig(prm_, c)
        return gg, dg, 0.0 * ddg

    monkeypatch.setattr(O, "_degradation", no_ddg)
    d = O.hess_diag(g, prm, x)
    assert np.max(np.abs(d - D)) > 1e-6 * np.max(np.abs(D))


# ---------------------------------------------------------------- Algorithm 3
# Convergence_control with eta1 = 0.1, eta2 = 0.75, gamma1 = 0.5, gamma2 = 2,
# delta_max = 1: each row is (rho, delta in, accepted?, delta out), the
# expected radius written out by hand from Algorithm 3's three cases
# (rho < eta1 shrink, eta1 <= rho <= eta2 keep, rho > eta2 expand, capped).
RADIUS_TABLE = [
    (-3.0, 0.4, False, 0.2),     # energy rose: reject, shrink
    (0.05, 0.4, False, 0.2),     # below eta1: reject, shrink
    (0.1, 0.4, False, 0.4),      # rho = eta1: not accepted (strict), radius kept
    (0.3, 0.4, True, 0.4),       # between: accept, keep
    (0.75, 0.4, True, 0.4),      # rho = eta2: keep
    (0.9, 0.4, True, 0.8),       # above eta2: accept, expand
    (1.7, 0.7, True, 1.0),       # expansion capped at delta_max
    (0.9, 1.0, True, 1.0),       # already at the cap
]


def test_convergence_control_radius_table():
    tr = O.TRParams()
    lb = np.array([0.0, -np.inf, 0.2])
    ub = np.array([1.0, np.inf, 1.0])
    x = np.array([0.5, 3.0, 0.3])
    s = np.array([0.7, -1.0, -0.25])  # the first and last leave the box
    for rho, delta, acc, delta_out in RADIUS_TABLE:
        xn, dn = O.convergence_control(rho, x, s, delta, lb, ub, tr)
        assert dn == delta_out, (rho, delta)
        if acc:
            assert np.array_equal(xn, np.array([1.0, 2.0, 0.2])), rho
        else:
            assert np.array_equal(xn, x), rho


def test_pins_catch_swapped_radius_factors(monkeypatch):
    """Convergence_control with gamma1 and gamma2 exchanged fails the table."""
    real = O.convergence_control

    def swapped(rho, x, s, delta, lb, ub, tr):
        t = O.TRParams(**{**tr.__dict__, "gamma1": tr.gamma2, "gamma2": tr.gamma1})
        return real(rho, x, s, delta, lb, ub, t)

    monkeypatch.setattr(O, "convergence_control", swapped)
    with pytest.raises(AssertionError):
        test_convergence_control_radius_table()


def test_pins_catch_swapped_thresholds(monkeypatch):
    """Convergence_control with eta1 and eta2 exchanged fails the table."""
    real = O.convergence_control

    def swapped(rho, x, s, delta, lb, ub, tr):
        t = O.TRParams(**{**tr.__dict__, "eta1": tr.eta2, "eta2": tr.eta1})
        return real(rho, x, s, delta, lb, ub, t)

    monkeypatch.setattr(O, "convergence_control", swapped)
    with pytest.raises(AssertionError):
        test_convergence_control_radius_table()


# ---------------------------------------------------------------- trust-region gate
def _gate_case():
    H = O.Hierarchy(2, (5, 5), 0.25, 2, O.Params(E=1.0, nu=0.3, Gc=1.0, p=1e-3))
    g = H.fine
    x = np.zeros(3 * g.N)
    x[2 * g.N:] = O.rasterize(g, O.LINE2D, PI.centred_crack_2d(0.2), g.h)
    r = O.rmtr_load_step(H, x, O.TRParams(rtol=1e-12), p=1e-3)
    return H, g, r.x


def test_trust_region_gate_ratio_from_the_quartic():
    """The gate's ratio is eq. (rho_tr) along s: the plain difference of
    the two energies over the model's decrease, agreeing to the plain
    difference's cancellation bound (1e-15 |E| / |actual|); its predicted
    decrease is -(a1 + a2) of the quartic coefficients (a1 = grad E.s,
    a2 = s.Hs/2, pinned above).  A proposal that triples the displacement
    is refused (the energy rises); the converged state at a higher
    pressure, proposed from the lower one, is accepted with rho near 1 (the
    quadratic model is nearly exact there)."""
    H, g, x1 = _gate_case()
    H.prm.p = 2e-3
    r2 = O.rmtr_load_step(H, x1, O.TRParams(rtol=1e-12), p=2e-3)
    rho, acc, xn = O.trust_region_gate(H, x1, r2.x, 0.1)
    s = r2.x - x1
    e0, e1 = O.energy(g, H.prm, x1), O.energy(g, H.prm, x1 + s)
    a = O.energy_diff_coeffs(g, H.prm, x1, s)
    pred = -(a[0] + a[1])
    plain = (e0 - e1) / pred
    assert abs(rho - plain) <= 4e-15 * abs(e0) / abs(e0 - e1) * abs(rho)
    assert abs(rho - (-(a.sum())) / pred) <= 1e-12 * abs(rho)
    assert acc and 0.9 < rho < 1.1
    assert np.array_equal(xn, x1 + (r2.x - x1))
    bad = x1.copy()
    bad[:2 * g.N] *= 3.0
    rho_b, acc_b, xb = O.trust_region_gate(H, x1, bad, 0.1)
    assert not acc_b and np.array_equal(xb, x1)


def test_pins_catch_a_planted_gate_sign_error(monkeypatch):
    """A gate whose predicted decrease forgets the minus sign never sees a
    positive prediction for a descent step, so it refuses the good proposal."""
    real = O.trust_region_gate

    def wrong(H, x, xhat, eta):
        real_hv = O.hessvec
        try:
            O.hessvec = lambda g, prm, xx, v, elems=None: -real_hv(g, prm, xx, v, elems)
            return real(H, x, xhat, eta)
        finally:
            O.hessvec = real_hv

    monkeypatch.setattr(O, "trust_region_gate", wrong)
    with pytest.raises(AssertionError):
        test_trust_region_gate_ratio_from_the_quartic()


# ---------------------------------------------------------------- the paper's QP solvers
def _qp_case(dim=2, n=(6, 5), seed=51):
    """A box QP from the functional's Hessian at a mild state (SPD there):
    bounds as a TR subproblem at a fracture state would give them."""
    g = O.Grid(dim, n, 0.25)
    prm = O.Params(E=1.0, nu=0.3, Gc=1.0, ls=0.5, p=0.0)
    x = PI.random_state(seed, dim, g.N, u_scale=1e-3, c_hi=0.3)
    A = O.probe_sparse(g, lambda v: O.hessvec(g, prm, x, v))
    r = PI.rng(seed + 1)
    gv = r.standard_normal(x.size)
    lo = -r.uniform(0.01, 0.2, x.size)
    hi = r.uniform(0.01, 0.2, x.size)
    # clamped displacement dofs on the boundary, as in every TR subproblem
    fixed = np.zeros(x.size, dtype=bool)
    bnd = g.boundary_nodes()
    for f in range(dim):
        fixed[f * g.N:(f + 1) * g.N] = bnd
    lo[fixed] = 0.0
    hi[fixed] = 0.0
    return g, A, gv, lo, hi


def _kkt_residual(A, g, lo, hi, s):
    """|| s - P(s - (g + A s)) ||: zero exactly at the box QP's KKT point."""
    gr = g + A @ s
    return float(np.linalg.norm(s - np.minimum(np.maximum(s - gr, lo), hi)))


def test_probe_sparse_is_the_dense_hessian():
    g = O.Grid(3, (3, 4, 3), 0.3)
    prm = _prm()
    x = PI.random_state(52, 3, g.N, u_scale=0.3)
    A = O.probe_sparse(g, lambda v: O.hessvec(g, prm, x, v)).toarray()
    D = O.dense_hessian(g, prm, x)
    assert np.max(np.abs(A - D)) <= 1e-14 * np.max(np.abs(D))


def test_pgs_diagonal_qp_is_exact_in_one_sweep():
    """For a diagonal H every dof is independent: one sweep gives the
    closed-form minimiser clamp(-g_i / h_i, lo_i, hi_i)."""
    g = O.Grid(2, (4, 3), 0.5)
    r = PI.rng(53)
    h = r.uniform(0.5, 2.0, 3 * g.N)
    A = sp.diags(h).tocsr()
    gv = r.standard_normal(3 * g.N)
    lo, hi = -0.3 * np.ones(3 * g.N), 0.2 * np.ones(3 * g.N)
    s = O.pgs_sweeps(A, g, gv, lo, hi, 1)
    assert np.max(np.abs(s - np.clip(-gv / h, lo, hi))) <= 1e-15


def test_pgs_decreases_the_model_and_reaches_kkt():
    g, A, gv, lo, hi = _qp_case()
    m = lambda s: float(gv @ s) + 0.5 * float(s @ (A @ s))
    s, prev = np.zeros_like(gv), 0.0
    for _ in range(200):
        s = O.pgs_sweeps(A, g, gv, lo, hi, 1, s)
        assert m(s) <= prev + 1e-15
        prev = m(s)
    assert np.all(s >= lo) and np.all(s <= hi)
    assert _kkt_residual(A, gv, lo, hi, s) <= 1e-10 * np.linalg.norm(gv)


def test_mprgp_reaches_the_kkt_point_of_pgs():
    g, A, gv, lo, hi = _qp_case(3, (4, 4, 3), 54)
    Hv = lambda v: A @ v
    dd = A.diagonal()
    lam = float(sp.linalg.eigsh(sp.diags(1 / np.sqrt(dd)) @ A @ sp.diags(1 / np.sqrt(dd)), k=1,
                                return_eigenvectors=False)[0])
    s = O.mprgp(Hv, gv, lo, hi, dd, 1e-12 * np.linalg.norm(gv), 5000, lam_max=1.01 * lam)
    assert np.all(s >= lo - 1e-15) and np.all(s <= hi + 1e-15)
    assert _kkt_residual(A, gv, lo, hi, s) <= 1e-10 * np.linalg.norm(gv)
    sp_ = O.pgs_sweeps(A, g, gv, lo, hi, 3000)
    assert np.max(np.abs(s - sp_)) <= 1e-8 * np.max(np.abs(s))


def test_mprgp_1d_closed_form():
    """A 1x1 box QP: the minimiser clamp(-g/h, lo, hi) in one proportioning
    or CG step."""
    for gv, h, lo, hi in ((2.0, 4.0, -1.0, 1.0), (-3.0, 0.5, -1.0, 2.0), (5.0, 1.0, -1.0, 1.0)):
        s = O.mprgp(lambda v: h * v, np.array([gv]), np.array([lo]), np.array([hi]), np.array([h]),
                    1e-14, 50, lam_max=1.0)
        assert abs(s[0] - min(max(-gv / h, lo), hi)) <= 1e-14


def test_pins_catch_an_unprojected_gauss_seidel(monkeypatch):
    """Gauss-Seidel without the projection leaves the box: the KKT pin fails."""
    real = O.pgs_sweeps

    def unprojected(A, grid, g, lo, hi, sweeps, s=None):
        return real(A, grid, g, np.full_like(lo, -np.inf), np.full_like(hi, np.inf), sweeps, s)

    monkeypatch.setattr(O, "pgs_sweeps", unprojected)
    with pytest.raises(AssertionError):
        test_pgs_decreases_the_model_and_reaches_kkt()


def test_pins_catch_a_gradient_sign_error_in_mprgp(monkeypatch):
    """MPRGP handed the model's gradient with the wrong sign solves another
    QP: the KKT pin fails."""
    real = O.mprgp

    def wrong(Hv, g, lo, hi, dscale, tol, maxit, gamma=1.0, lam_max=None):
        return real(Hv, -g, lo, hi, dscale, tol, maxit, gamma=gamma, lam_max=lam_max)

    monkeypatch.setattr(O, "mprgp", wrong)
    with pytest.raises(AssertionError):
        test_mprgp_reaches_the_kkt_point_of_pgs()


def test_propagation_starts_at_the_griffith_pressure():
    """The oracle's ramp (tests/golden/propagation.json, written by
    tests/golden/make_propagation.py) grows the centred crack between
    p = 2.0 and 2.5.  Griffith's critical pressure of a line crack of
    half-length a in plane strain, p_c = sqrt(E' G / (pi a)), E' = E/(1 -
    nu^2), with AT2's discrete effective toughness G = G_c (1 + h/(2 l_s))
    = 1.25 G_c at l_s = 2h, is 2.09 for a = 0.1: inside that bracket.
    Below it the crack's extent barely moves; above it, it at least
    quadruples and the energy falls."""
    gold = json.load(open(os.path.join(GOLD, "propagation.json")))
    E, nu, Gc, a = gold["E"], gold["nu"], gold["Gc"], 0.1
    pc = math.sqrt(E / (1 - nu * nu) * 1.25 * Gc / (math.pi * a))
    assert 2.0 < pc < 2.5
    steps = gold["steps"]
    n0 = steps[0]["crack_nodes"]
    below = [s for s in steps if s["p"] < pc]
    above = [s for s in steps if s["p"] > pc]
    assert all(s["crack_nodes"] < 1.5 * n0 for s in below)
    assert all(s["crack_nodes"] > 4 * n0 for s in above)
    es = [s["energy"] for s in steps]
    assert all(b < a_ for a_, b in zip(es, es[1:]))
