"""The paper's own 3D scenario at its own size on one GPU (Sec. 5.2,
three-dimensional scenarios): 393^3 nodes on four levels (242,793,828 dofs),
100 rectangular-plate fractures, lambda = mu = 1e5, G_c = 1, clamped
boundary, p = p0 = 0.01.  The element kernels are compared with the oracle
at sampled nodes (its elements around them) on a random state; one
mixed-precision load step is checked by its properties: convergence, energy
decrease, c_prev <= c <= 1 and the clamped boundary, evaluated on the
device."""
import numpy as np
import pytest

import pfinputs as PI
from oracle import pf_oracle as O
from tests.gpu_common import dev, host, relinf, require_cuda

pytestmark = pytest.mark.gpu

E, NU, GC = 2.5e5, 0.25, 1.0


@pytest.fixture(scope="module")
def paper():
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    H = pf.mesh_hierarchy_create(3, (50, 50, 50), 4, 1 / 49, E=E, nu=NU, Gc=GC, ls_over_h=2.0)
    assert H.ndof() == 242793828  # the dof count the paper prints for this scenario
    yield torch, pf, H
    H.close()


def test_paper_scale_kernels_at_sampled_nodes(paper):
    torch, pf, H = paper
    n, h, N = H.levels[-1]
    g = O.Grid(3, n, h)
    prm = O.Params(E=E, nu=NU, Gc=GC, ls=2.0 * h, p=0.01)
    pf.pressure_set(H, 0.01)
    x = PI.random_state(61, 3, N, u_scale=1e-7, c_hi=1.0)
    v = PI.random_direction(62, x.size)
    xd, vd = dev(x), dev(v)
    nodes = np.unique(np.concatenate([PI.rng(63).choice(N, size=200, replace=False), [0, N - 1]]))
    elems = g.elements_touching(nodes)
    idx = np.concatenate([f * N + nodes for f in range(4)])
    go = O.gradient(g, prm, x, elems)[idx]
    ho = O.hessvec(g, prm, x, v, elems)[idx]
    assert relinf(host(pf.gradient(H, 3, xd))[idx], go) <= 1e-10
    assert relinf(host(pf.hessvec(H, 3, xd, vd))[idx], ho) <= 1e-10
    assert relinf(host(pf.hessvec(H, 3, xd.float(), vd.float()))[idx], ho) <= 2e-5
    del xd, vd


def test_paper_scale_load_step(paper):
    torch, pf, H = paper
    n, h, N = H.levels[-1]
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_BOX3D, PI.box_network_3d(PI.SEED_3D_PAPER, 100), h, x)
    c0 = x[3 * N:].clone()
    assert int(c0.sum()) > 100000
    pf.pressure_set(H, 0.01)
    e0 = pf.energy(H, 3, x)
    st = pf.rmtr_load_step(H, x, pf.default_params(precision=pf.PF_FP32))
    assert st["converged"] == 1 and st["energy"] < e0
    c = x[3 * N:]
    assert bool((c >= c0).all()) and bool((c <= 1.0).all())
    u = x[: 3 * N].view(3, n[2], n[1], n[0])
    for face in (u[:, 0], u[:, -1], u[:, :, 0], u[:, :, -1], u[:, :, :, 0], u[:, :, :, -1]):
        assert bool((face == 0.0).all())
