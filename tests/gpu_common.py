"""Shared set-up for the GPU parity tests (imported by tests marked gpu)."""
import numpy as np

import pfinputs as PI
from oracle import pf_oracle as O


def require_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2007_12908_gb300 import build
    build.build()
    return torch


def pair(dim, n_coarse, L, h_coarse, E=1.0, nu=0.3, Gc=1.0, k_res=0.0, p=0.0):
    """The same hierarchy on the CUDA path and in the oracle."""
    import paper_2007_12908_gb300 as pf
    H = pf.mesh_hierarchy_create(dim, n_coarse, L, h_coarse, E=E, nu=nu, Gc=Gc, ls_over_h=2.0, k_res=k_res)
    pf.pressure_set(H, p)
    Ho = O.Hierarchy(dim, n_coarse, h_coarse, L, O.Params(E=E, nu=nu, Gc=Gc, k_res=k_res, p=p))
    return H, Ho


def relinf(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t if dtype is None else t.to(dtype)


def host(t):
    return t.detach().double().cpu().numpy()
