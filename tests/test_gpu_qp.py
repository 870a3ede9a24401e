"""The paper's QP solvers on the GPU (Sec. 4.2.2) against the oracle:
symmetric multicolour projected Gauss-Seidel sweeps and MPRGP on a level's
lagged FP64 Hessian, and whole load steps with them (PGS smoothing, MPRGP on
the coarsest level) reaching the oracle's converged fields."""
import numpy as np
import pytest
import scipy.sparse as sp

import pfinputs as PI
from oracle import pf_oracle as O
from tests.gpu_common import dev, host, pair, relinf, require_cuda
from tests.test_gpu_solver import _compare_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    require_cuda()
    import paper_2007_12908_gb300 as m
    return m


def _qp(pf, dim, nc, L, hc, seed):
    H, Ho = pair(dim, nc, L, hc, nu=0.25 if dim == 3 else 0.3, p=1e-2)
    lvl = L - 1
    g = Ho.grids[lvl]
    x = PI.random_state(seed, dim, g.N, u_scale=1e-3, c_hi=0.3)
    pf.hessvec_lag_set(H, lvl, dev(x))
    A = O.probe_sparse(g, lambda v: O.hessvec(g, Ho.prm, x, v))
    r = PI.rng(seed + 1)
    gv = r.standard_normal(x.size)
    lo = -r.uniform(0.01, 0.2, x.size)
    hi = r.uniform(0.01, 0.2, x.size)
    fixed = np.zeros(x.size, dtype=bool)
    for f in range(dim):
        fixed[f * g.N:(f + 1) * g.N] = g.boundary_nodes()
    lo[fixed] = 0.0
    hi[fixed] = 0.0
    return H, Ho, g, lvl, A, gv, lo, hi


@pytest.mark.parametrize("dim,nc,L,hc", [(2, (9, 7), 2, 0.125), (3, (5, 4, 5), 2, 0.25)])
def test_pgs_sweeps_match_oracle(pf, dim, nc, L, hc):
    H, Ho, g, lvl, A, gv, lo, hi = _qp(pf, dim, nc, L, hc, 81)
    s = dev(np.zeros(gv.size))
    so = np.zeros(gv.size)
    for sweeps in (1, 2, 5):
        pf.qp_pgs(H, lvl, dev(gv), dev(lo), dev(hi), s, sweeps)
        so = O.pgs_sweeps(A, g, gv, lo, hi, sweeps, so)
        assert relinf(host(s), so) <= 1e-12, sweeps
    H.close()


@pytest.mark.parametrize("dim,nc,L,hc", [(2, (9, 7), 2, 0.125), (3, (5, 4, 5), 2, 0.25)])
def test_mprgp_matches_oracle(pf, dim, nc, L, hc):
    H, Ho, g, lvl, A, gv, lo, hi = _qp(pf, dim, nc, L, hc, 82)
    tol = 1e-11 * np.linalg.norm(gv)
    s, used = pf.qp_mprgp(H, lvl, dev(gv), dev(lo), dev(hi), tol, 20000)
    dd = A.diagonal()
    dd = np.where(dd > 0, dd, 1.0)
    sq = np.sqrt(dd)
    lam = float(np.max(np.asarray(abs(sp.diags(1 / sq) @ A @ sp.diags(1 / sq)).sum(axis=1)).ravel()))
    so = O.mprgp(lambda v: A @ v, gv, lo, hi, dd, tol, 20000, lam_max=lam)
    assert used < 20000
    assert relinf(host(s), so) <= 1e-8
    gr = gv + A @ host(s)
    sh = host(s)
    assert np.linalg.norm(sh - np.minimum(np.maximum(sh - gr, lo), hi)) <= 1e-9 * np.linalg.norm(gv)
    H.close()


@pytest.mark.parametrize("L,nc", [(2, 33), (3, 17)])
def test_load_step_with_the_papers_qp_solvers(pf, L, nc):
    """2D centred crack at 65^2 (p = 1e-3): FP64 load steps with PGS
    smoothing and MPRGP on the coarsest level converge to the oracle's
    fields with the same solvers, and to the same energy as the projected-CG
    configuration."""
    import torch
    H, Ho = pair(2, (nc, nc), L, 1 / (nc - 1), p=1e-3)
    g = Ho.fine
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_LINE2D, PI.centred_crack_2d(), g.h, x)
    xo = np.zeros(3 * g.N)
    xo[2 * g.N:] = O.rasterize(g, O.LINE2D, PI.centred_crack_2d(), g.h)
    xc = x.clone()
    st = pf.rmtr_load_step(H, x, pf.default_params(rtol=1e-12, qp_solver=pf.PF_QP_PAPER, pgs_sweeps=2))
    sc = pf.rmtr_load_step(H, xc, pf.default_params(rtol=1e-12))
    ro = O.rmtr_load_step(Ho, xo, O.TRParams(rtol=1e-12, qp_solver=O.QP_PAPER, pgs_sweeps=2), p=1e-3)
    assert st["converged"] == 1 and ro.converged and sc["converged"] == 1
    _compare_fields(host(x), ro.x, 2, g.N, g, Ho.prm)
    assert abs(st["energy"] - ro.energy) <= 1e-10 * abs(ro.energy)
    assert abs(st["energy"] - sc["energy"]) <= 1e-10 * abs(sc["energy"])
    assert abs(st["cycles"] - ro.cycles) <= 2
    H.close()


def test_papers_qp_solvers_need_fp64_first_order(pf):
    import torch
    H, Ho = pair(2, (9, 9), 2, 1 / 8, p=1e-3)
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    for kw in ({"precision": pf.PF_FP32}, {"coarse_model": pf.PF_GALERKIN}):
        st = pf.rmtr_load_step(H, x, pf.default_params(qp_solver=pf.PF_QP_PAPER, **kw), check=False)
        assert st["status"] == pf.PF_EINVAL
    H.close()
