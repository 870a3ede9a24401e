"""The device RMTR load step against the oracle (converged fields on the 2D
65^2 workload, small 3D hierarchies, the 1D closed form) and its invariants
at the 3D 129^3 workload size."""
import json
import math
import os

import numpy as np
import pytest

import pfinputs as PI
from oracle import pf_oracle as O
from tests.gpu_common import dev, host, pair, relinf, require_cuda

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")

# converged-field parity (relative, per field, max norm) and energy parity
FIELD_TOL = 1e-8
ENERGY_TOL = 1e-10


@pytest.fixture(scope="module")
def pf():
    require_cuda()
    import paper_2007_12908_gb300 as m
    return m


def _fields(x, dim, N):
    return [x[f * N:(f + 1) * N] for f in range(dim + 1)]


def _undetermined_nodes(grid, c):
    """Nodes all of whose elements have c = 1 at every corner: g(c) = 0 at
    every Gauss point there, so their displacement dofs carry no energy (zero
    gradient row, zero Hessian row) and any value is a minimiser."""
    conn = grid.element_connectivity()
    broken = np.all(c[conn] == 1.0, axis=1)
    ok = np.zeros(grid.N, dtype=bool)
    for k in range(conn.shape[1]):
        ok[conn[~broken, k]] = True
    return ~ok


def _compare_fields(xg, xo, dim, N, grid=None, prm=None):
    """Converged fields agree on every dof the minimiser determines; the
    displacement of nodes inside fully broken regions is free (see
    _undetermined_nodes) and is checked for validity instead: the GPU
    state's gradient vanishes there too."""
    und = np.zeros(N, dtype=bool)
    if grid is not None:
        und = _undetermined_nodes(grid, xo[dim * N:]) | _undetermined_nodes(grid, xg[dim * N:])
        if prm is not None and und.any():
            gr = O.gradient(grid, prm, xg)
            scale = np.max(np.abs(gr[:dim * N]))
            for f in range(dim):
                assert np.all(np.abs(gr[f * N:(f + 1) * N][und]) <= 1e-20 * scale)
    for f, (a, b) in enumerate(zip(_fields(xg, dim, N), _fields(xo, dim, N))):
        keep = ~und if f < dim else np.ones(N, dtype=bool)
        scale = max(np.max(np.abs(b)), 1e-300)
        err = np.abs(a - b)[keep]
        assert err.max() <= FIELD_TOL * scale, (f, err.max() / scale, int(np.argmax(np.where(keep, np.abs(a - b), 0))))


def _sneddon_setup(pf, model):
    H, Ho = pair(2, (33, 33), 2, 1 / 32, p=1e-3)
    import torch
    g = Ho.fine
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_LINE2D, PI.centred_crack_2d(), g.h, x)
    xo = np.zeros(3 * g.N)
    xo[2 * g.N:] = O.rasterize(g, O.LINE2D, PI.centred_crack_2d(), g.h)
    return H, Ho, x, xo


@pytest.fixture(scope="module")
def sneddon_runs(pf):
    out = {}
    for model in (O.FIRST_ORDER, O.GALERKIN):
        H, Ho, x, xo = _sneddon_setup(pf, model)
        tr = O.TRParams(coarse_model=model, rtol=1e-13)
        ro = O.rmtr_load_step(Ho, xo, tr, p=1e-3)
        st = pf.rmtr_load_step(H, x, pf.default_params(coarse_model=model, rtol=1e-13))
        out[model] = (H, Ho, host(x), ro, st)
    return out


@pytest.mark.parametrize("model", [O.FIRST_ORDER, O.GALERKIN])
def test_2d_load_step_matches_oracle(sneddon_runs, model):
    H, Ho, xg, ro, st = sneddon_runs[model]
    assert st["converged"] == 1 and ro.converged
    _compare_fields(xg, ro.x, 2, Ho.fine.N, Ho.fine, Ho.prm)
    assert abs(st["energy"] - ro.energy) <= ENERGY_TOL * abs(ro.energy)


def test_2d_sneddon_and_invariants(sneddon_runs):
    gold = json.load(open(os.path.join(GOLD, "sneddon.json")))
    H, Ho, xg, ro, st = sneddon_runs[O.FIRST_ORDER]
    g = Ho.fine
    uy = xg[g.N:2 * g.N].reshape(65, 65)
    cod = uy[34, 32] - uy[30, 32]
    assert cod > 0 and abs(cod / gold["w_centre"] - 1) < gold["rel_band"]
    c = xg[2 * g.N:]
    c0 = O.rasterize(g, O.LINE2D, PI.centred_crack_2d(), g.h)
    assert np.all(c >= c0) and np.all(c <= 1.0)
    bnd = g.boundary_nodes()
    assert np.all(xg[:g.N][bnd] == 0) and np.all(xg[g.N:2 * g.N][bnd] == 0)


def test_deterministic_and_host_entry(pf):
    import torch
    H, Ho, x1, _ = _sneddon_setup(pf, O.FIRST_ORDER)
    x2 = x1.clone()
    xh = host(x1).copy()
    prm = pf.default_params(rtol=1e-8)
    pf.rmtr_load_step(H, x1, prm)
    pf.rmtr_load_step(H, x2, prm)
    pf.rmtr_load_step_host(H, xh, prm)
    assert torch.equal(x1, x2)
    assert np.array_equal(host(x1), xh)


def test_pure_phase_field_closed_form(pf):
    import torch
    H, Ho = pair(2, (17, 3), 2, 1 / 16, p=0.0)
    g = Ho.fine
    rows = np.array([[0.5 + 0.25 * g.h, 0.5, math.pi / 2, 10.0]])
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_LINE2D, rows, g.h, x)
    st = pf.rmtr_load_step(H, x, pf.default_params(rtol=1e-12))
    assert st["converged"]
    from tests.test_oracle_pins import _closed_form_profile
    c = host(x)[2 * g.N:].reshape(g.n[1], g.n[0])
    right, _ = _closed_form_profile(g.n[0] - 1 - 17, g.h, Ho.prm.ls)
    left, _ = _closed_form_profile(16, g.h, Ho.prm.ls)
    for row in c:
        np.testing.assert_allclose(row[17:], right, rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(row[:17][::-1], left, rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("model", [O.FIRST_ORDER, O.GALERKIN])
def test_3d_small_load_steps_match_oracle(pf, model):
    """Two load steps on a 3-level 3D hierarchy with discs (irreversibility
    carries over between steps)."""
    import torch
    H, Ho = pair(3, (3, 3, 3), 3, 0.5, nu=0.25, p=0.0)
    g = Ho.fine
    rows = np.array([[0.5, 0.45, 0.52, 0.0, 0.6, 0.8, 0.3], [0.3, 0.6, 0.4, 1.0, 0.0, 0.0, 0.2]])
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_DISC3D, rows, g.h, x)
    xo = np.zeros(4 * g.N)
    xo[3 * g.N:] = O.rasterize(g, O.DISC3D, rows, g.h)
    assert np.array_equal(host(x), xo)
    tr = O.TRParams(coarse_model=model, rtol=1e-13)
    for p in (0.5, 1.0):
        pf.pressure_set(H, p)
        st = pf.rmtr_load_step(H, x, pf.default_params(coarse_model=model, rtol=1e-13))
        ro = O.rmtr_load_step(Ho, xo, tr, p=p)
        xo = ro.x
        assert st["converged"] and ro.converged
        _compare_fields(host(x), xo, 3, g.N, g, Ho.prm)


@pytest.mark.slow
def test_3d_workload_load_step_properties(pf):
    """One load step of the 129^3 four-level workload with 20 discs
    (p = 5e-4): convergence, bounds, clamped boundary, energy decrease, and the
    projected gradient re-evaluated by the oracle."""
    import torch
    H, Ho = pair(3, (17, 17, 17), 4, 1 / 16, nu=0.25, p=5e-4)
    g = Ho.fine
    rows = PI.disc_network_3d(PI.SEED_3D_PLAIN, 20)
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_DISC3D, rows, g.h, x)
    c0 = host(x)[3 * g.N:].copy()
    e0 = pf.energy(H, 3, x)
    st = pf.rmtr_load_step(H, x, pf.default_params())
    assert st["converged"] == 1
    xg = host(x)
    assert st["energy"] < e0
    c = xg[3 * g.N:]
    assert np.all(c >= c0) and np.all(c <= 1.0)
    bnd = g.boundary_nodes()
    for f in range(3):
        assert np.all(xg[f * g.N:(f + 1) * g.N][bnd] == 0.0)
    # oracle re-check of first-order criticality at the returned point
    Ho.c_prev = c0
    lb, ub = Ho.fine_bounds()
    gr = O.gradient(g, Ho.prm, xg)
    pg = O.projected_gradient_norm(xg, gr, lb, ub)
    assert pg <= 1e-9 * st["pg0"]
    assert abs(O.energy(g, Ho.prm, xg) - st["energy"]) <= ENERGY_TOL * abs(st["energy"])


def test_mixed_load_step_element_owned_cg(pf):
    """A mixed-precision load step on a 65^3 three-level hierarchy with 20
    discs (p = 5e-4).  Its finest level has 9^3 element tiles of 8^3, so the
    FP32 CG there runs three launches per iteration: the element-owned
    Hessian with the direction update formed in its operand, the gather with
    p.Hp and alpha, and the update.  The step converges inside the box, to the
    FP64 solver's energy, and the oracle's projected gradient at the result is
    below the stopping tolerance."""
    import torch
    H, Ho = pair(3, (17, 17, 17), 3, 1 / 16, nu=0.25, p=5e-4)
    g = Ho.fine
    assert g.n == (65, 65, 65)
    rows = PI.disc_network_3d(PI.SEED_3D_PLAIN, 20)
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_DISC3D, rows, g.h, x)
    x64 = x.clone()
    c0 = host(x)[3 * g.N:].copy()
    s64 = pf.rmtr_load_step(H, x64, pf.default_params())
    s32 = pf.rmtr_load_step(H, x, pf.default_params(precision=pf.PF_FP32))
    assert s64["converged"] == 1 and s32["converged"] == 1
    assert abs(s32["energy"] - s64["energy"]) <= 1e-8 * abs(s64["energy"])
    xg = host(x)
    c = xg[3 * g.N:]
    assert np.all(c >= c0) and np.all(c <= 1.0)
    Ho.c_prev = c0
    lb, ub = Ho.fine_bounds()
    pg = O.projected_gradient_norm(xg, O.gradient(g, Ho.prm, xg), lb, ub)
    assert pg <= 1e-9 * s32["pg0"]
    assert abs(O.energy(g, Ho.prm, xg) - s32["energy"]) <= ENERGY_TOL * abs(s32["energy"])


def test_mixed_precision_reaches_fp64_energy(pf):
    H, Ho, x, _ = _sneddon_setup(pf, O.FIRST_ORDER)
    x2 = x.clone()
    s64 = pf.rmtr_load_step(H, x, pf.default_params(rtol=1e-12))
    s32 = pf.rmtr_load_step(H, x2, pf.default_params(rtol=1e-12, precision=pf.PF_FP32))
    assert s32["converged"]
    assert abs(s32["energy"] - s64["energy"]) <= 1e-8 * abs(s64["energy"])


def test_stopping_reference(pf):
    """An extrapolated load step stops relative to the projected gradient at
    the plain start under the new pressure (the state as given), which the
    stats report: equal to pf_projected_gradient at that state."""
    import torch
    H, Ho = pair(3, (5, 5, 5), 3, 0.25, nu=0.25, p=0.0)
    g = Ho.fine
    rows = np.array([[0.5, 0.45, 0.52, 0.0, 0.6, 0.8, 0.3], [0.3, 0.6, 0.4, 1.0, 0.0, 0.0, 0.2]])
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_DISC3D, rows, g.h, x)
    for prec in (pf.PF_FP32, pf.PF_FP64):
        prm = pf.default_params(precision=prec, start=pf.PF_START_EXTRAPOLATE)
        for p in (1e-3, 1.5e-3, 2e-3):
            pf.pressure_set(H, p)
            direct = pf.projected_gradient(H, x)
            st = pf.rmtr_load_step(H, x, prm)
            assert st["converged"]
            if st["pg_ref"] != st["pg0"]:  # extrapolated steps
                assert abs(st["pg_ref"] - direct) <= 1e-10 * direct


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_3d_65_load_step_fields_match_oracle(pf, precision):
    """One load step of the disc network on a 65^3 three-level hierarchy:
    its finest level takes the element-owned FP32 products (mixed) and the
    full-grid FP64 stencil product (k_stencil_apply, FP64).  The converged
    fields at 1,500 sampled determined nodes match the oracle's
    (tests/golden/field_samples_65.json, written by the committed oracle
    script) to 1e-8 of each field's max-norm, and the energy to 1e-10 (FP64)
    or 1e-8 (mixed)."""
    import torch
    gold = json.load(open(os.path.join(GOLD, "field_samples_65.json")))
    H, Ho = pair(3, (17, 17, 17), 3, 1 / 16, nu=0.25, p=gold["p"])
    g = Ho.fine
    assert list(g.n) == gold["grid"]
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_DISC3D, PI.disc_network_3d(gold["seed"], gold["fractures"]), g.h, x)
    prec = pf.PF_FP64 if precision == "fp64" else pf.PF_FP32
    st = pf.rmtr_load_step(H, x, pf.default_params(precision=prec, rtol=1e-12))
    assert st["converged"] == 1
    tol_e = ENERGY_TOL if precision == "fp64" else 1e-8
    assert abs(st["energy"] - gold["energy"]) <= tol_e * abs(gold["energy"])
    xg = host(x)
    nodes = np.asarray(gold["nodes"])
    for f in range(4):
        got = xg[f * g.N + nodes]
        want = np.asarray(gold["fields"][f])
        assert np.max(np.abs(got - want)) <= FIELD_TOL * gold["field_max"][f], (f, np.max(np.abs(got - want)))
    H.close()


def test_get_fields(pf):
    """pf_get_fields: c_prev against the oracle's rasterisation, the fixed-dof
    mask against the boundary, the finest feasible set of eq. (space_pf)
    after a load step, and the coarse feasible set's shape (lower <= upper,
    boundary displacement corrections fixed)."""
    import torch
    H, Ho = pair(2, (9, 9), 2, 1 / 8, p=1e-3)
    g = Ho.fine
    N = g.N
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    rows = PI.centred_crack_2d(0.2)
    pf.fractures_set(H, pf.PF_LINE2D, rows, g.h, x)
    c_or = O.rasterize(g, O.LINE2D, rows, g.h)
    assert np.array_equal(host(pf.get_fields(H, 1, pf.PF_FIELD_C_PREV)), c_or)
    with pytest.raises(pf.PfError) as e:
        pf.get_fields(H, 1, pf.PF_FIELD_LOWER)
    assert e.value.status == pf.PF_ESTATE
    with pytest.raises(pf.PfError):
        pf.get_fields(H, 0, pf.PF_FIELD_C_PREV)
    ix, iy = np.meshgrid(np.arange(g.n[0]), np.arange(g.n[1]), indexing="xy")
    bnd = ((ix == 0) | (iy == 0) | (ix == g.n[0] - 1) | (iy == g.n[1] - 1)).ravel()
    fixed = host(pf.get_fields(H, 1, pf.PF_FIELD_FIXED))
    assert np.array_equal(fixed, np.concatenate([bnd, bnd, np.zeros(N, bool)]).astype(float))
    st = pf.rmtr_load_step(H, x, pf.default_params())
    assert st["converged"]
    cp = host(pf.get_fields(H, 1, pf.PF_FIELD_C_PREV))
    lo, up = host(pf.get_fields(H, 1, pf.PF_FIELD_LOWER)), host(pf.get_fields(H, 1, pf.PF_FIELD_UPPER))
    assert np.array_equal(lo[2 * N:], cp) and np.all(up[2 * N:] == 1.0)
    for f in range(2):
        lf, uf = lo[f * N:(f + 1) * N], up[f * N:(f + 1) * N]
        assert np.all(lf[bnd] == 0.0) and np.all(uf[bnd] == 0.0)
        assert np.all(np.isneginf(lf[~bnd])) and np.all(np.isposinf(uf[~bnd]))
    gc = Ho.grids[0]
    lc, uc = host(pf.get_fields(H, 0, pf.PF_FIELD_LOWER)), host(pf.get_fields(H, 0, pf.PF_FIELD_UPPER))
    assert np.all(lc <= uc)
    jx, jy = np.meshgrid(np.arange(gc.n[0]), np.arange(gc.n[1]), indexing="xy")
    bc_ = ((jx == 0) | (jy == 0) | (jx == gc.n[0] - 1) | (jy == gc.n[1] - 1)).ravel()
    for f in range(2):
        assert np.array_equal(lc[f * gc.N:(f + 1) * gc.N][bc_], uc[f * gc.N:(f + 1) * gc.N][bc_])
    pf.fractures_set(H, pf.PF_LINE2D, rows, g.h, x)
    with pytest.raises(pf.PfError):
        pf.get_fields(H, 1, pf.PF_FIELD_UPPER)
    H.close()
