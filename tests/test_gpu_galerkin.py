"""Stored Galerkin coarse operators (the second-order coherent level model,
eq. (second_order_consistency) and eq. (delta_terms) under Hessian lagging):
the FP32 stencils of pf_galerkin_set against the oracle's recursive
R H^{l+1} I, on every coarse level of 2D and 3D hierarchies; symmetry; and
mixed-precision GALERKIN load steps that reach the FP64 energy."""
import numpy as np
import pytest

import pfinputs as PI
from oracle import pf_oracle as O
from tests.gpu_common import dev, host, pair, relinf, require_cuda

pytestmark = pytest.mark.gpu

# FP32 entries: each sums up to 2^d x 2^d fine Gauss-point terms per child
# (and 8 children per coarser level) in FP32; the product adds 3^d (d+1)
# of them per row
TOL = 2e-5


@pytest.fixture(scope="module")
def pf():
    require_cuda()
    import paper_2007_12908_gb300 as m
    return m


@pytest.mark.parametrize("dim,nc,L,hc", [(3, (3, 3, 3), 3, 0.5), (3, (3, 4, 3), 3, 0.5),
                                          (2, (5, 5), 4, 0.25), (2, (4, 6), 3, 0.3)])
def test_galerkin_stencils_match_oracle(pf, dim, nc, L, hc):
    import torch
    H, Ho = pair(dim, nc, L, hc, nu=0.25 if dim == 3 else 0.3, p=3e-2, k_res=0.0)
    g = Ho.fine
    x = PI.random_state(71, dim, g.N, u_scale=0.05, c_hi=0.9)
    x32 = x.astype(np.float32)
    pf.galerkin_set(H, dev(x32))
    # the oracle's level models on the same (FP32-rounded) lag point
    models = [O.LevelModel(Ho, L - 1, x32.astype(np.float64))]
    for l in range(L - 2, -1, -1):
        z = np.zeros(Ho.ndof(l))
        models.append(O.LevelModel(Ho, l, z, finer=models[-1], dg=z, kind=O.GALERKIN))
    for m in models[1:]:
        l = m.level
        v = PI.random_direction(72 + l, Ho.ndof(l))
        ho = m.Hlag(v)
        h64 = host(pf.galerkin_apply(H, l, dev(v)))
        h32 = host(pf.galerkin_apply(H, l, dev(v, torch.float32)))
        assert relinf(h64, ho) <= TOL, (l, relinf(h64, ho))
        assert relinf(h32, ho) <= TOL, (l, relinf(h32, ho))
        w = PI.random_direction(90 + l, Ho.ndof(l))
        a = w @ h64
        b = v @ host(pf.galerkin_apply(H, l, dev(w)))
        assert abs(a - b) <= 1e-5 * np.linalg.norm(w) * np.linalg.norm(h64)


@pytest.mark.parametrize("dim", [2, 3])
def test_mixed_galerkin_load_step_reaches_fp64_energy(pf, dim):
    """A mixed-precision GALERKIN load step (stored FP32 coarse operators)
    converges to the FP64 solver's energy within 1e-8, and the oracle's
    projected gradient at its result is below the stopping tolerance."""
    import torch
    if dim == 2:
        H, Ho = pair(2, (17, 17), 3, 1 / 16, p=1e-3)
        g = Ho.fine
        rows, kind = PI.centred_crack_2d(), pf.PF_LINE2D
    else:
        H, Ho = pair(3, (5, 5, 5), 3, 0.25, nu=0.25, p=5e-3)
        g = Ho.fine
        rows, kind = PI.disc_network_3d(PI.SEED_3D_PLAIN, 20, rmin=0.1, rmax=0.25), pf.PF_DISC3D
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, kind, rows, g.h, x)
    x64 = x.clone()
    c0 = host(x)[dim * g.N:].copy()
    s64 = pf.rmtr_load_step(H, x64, pf.default_params(coarse_model=pf.PF_GALERKIN, rtol=1e-12))
    s32 = pf.rmtr_load_step(H, x, pf.default_params(coarse_model=pf.PF_GALERKIN, rtol=1e-12,
                                                    precision=pf.PF_FP32))
    assert s64["converged"] == 1 and s32["converged"] == 1
    assert abs(s32["energy"] - s64["energy"]) <= 1e-8 * abs(s64["energy"])
    xg = host(x)
    Ho.c_prev = c0
    lb, ub = Ho.fine_bounds()
    pg = O.projected_gradient_norm(xg, O.gradient(g, Ho.prm, xg), lb, ub)
    assert pg <= 1e-9 * s32["pg0"]
