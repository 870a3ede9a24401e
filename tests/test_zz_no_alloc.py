"""pf_energy_noalloc: the energy for callers that cannot allocate device
memory (for example a plug-in inside a host program that owns the whole
device memory budget, or a real-time loop where cudaMalloc may block and
synchronise the device).  Its reduction scratch is a fixed array inside the
library, so the call must give what pf_energy gives, call after call, and
refuse grids larger than that array can serve.

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes as C

import numpy as np
import pytest

import pfinputs as PI
from tests.gpu_common import dev, require_cuda

pytestmark = pytest.mark.gpu


def test_energy_noalloc_matches_energy_twice():
    torch = require_cuda()
    import paper_2007_12908_gb300 as pf
    from paper_2007_12908_gb300 import _binding as B
    cases = [
        # dim, coarse nodes, levels, coarse spacing, nu, pressure
        (3, (17, 17, 17), 4, 1 / 16, 0.25, 5e-3),
        (2, (35, 23), 2, 1 / 34, 0.3, 1e-3),
    ]
    for dim, nc, L, hc, nu, p in cases:
        H = pf.mesh_hierarchy_create(dim, nc, L, hc, E=1.0, nu=nu, Gc=1.0, ls_over_h=2.0)
        pf.pressure_set(H, p)
        n, h, N = H.levels[-1]
        ls = 2.0 * h
        for prec_dtype in (torch.float64, torch.float32):
            x = dev(PI.random_state(5 + dim, dim, N, u_scale=1e-3, c_hi=1.0), prec_dtype)
            ref = pf.energy(H, L - 1, x)
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            for _ in range(2):  # the shared scratch keeps the last call's contents
                out.fill_(float("nan"))
                B.energy_noalloc(dim, n, h, 1.0, nu, 1.0, ls, 0.0, p, x, out)
                torch.cuda.synchronize()
                got = float(out.item())
                assert abs(got - ref) <= 1e-10 * abs(ref), (dim, prec_dtype, got, ref)
        H.close()


def test_energy_noalloc_rejects_oversized_grids():
    torch = require_cuda()
    from paper_2007_12908_gb300 import _binding as B
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = (C.c_int * 3)(4098, 4098, 2)  # 4097 * 4097 > 16,777,216 elements
    rc = B.lib().pf_energy_noalloc(2, n, 1e-3, 1.0, 0.3, 1.0, 2e-3, 0.0, 0.0, C.c_void_p(x.data_ptr()),
                                   B.PF_FP64, C.c_void_p(out.data_ptr()), None)
    assert rc == B.PF_EINVAL
    assert b"16,777,216" in B.lib().pf_last_error()


def test_energy_noalloc_leaves_device_memory_unchanged():
    """After the first call on the device (which looks up the scratch
    array's address), further calls change the device's free memory by
    nothing: the call allocates no device memory of its own."""
    torch = require_cuda()
    from paper_2007_12908_gb300 import _binding as B
    n = (65, 65, 65)
    N = n[0] * n[1] * n[2]
    x = dev(PI.random_state(9, 3, N, u_scale=1e-3, c_hi=1.0), torch.float64)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.energy_noalloc(3, n, 1 / 64, 1.0, 0.25, 1.0, 2 / 64, 0.0, 1e-3, x, out)
    torch.cuda.synchronize()
    first = float(out.item())
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        B.energy_noalloc(3, n, 1 / 64, 1.0, 0.25, 1.0, 2 / 64, 0.0, 1e-3, x, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert float(out.item()) == first  # fixed-order reduction: the same value every call


def test_energy_noalloc_captures_in_global_mode():
    """After the first call, the call records into a CUDA graph under
    global capture mode, where any device allocation (in any thread) would
    invalidate the capture; the replayed graph gives the same energy."""
    torch = require_cuda()
    from paper_2007_12908_gb300 import _binding as B
    n = (33, 33, 33)
    N = n[0] * n[1] * n[2]
    x = dev(PI.random_state(11, 3, N, u_scale=1e-3, c_hi=1.0), torch.float64)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    args = (3, n, 1 / 32, 1.0, 0.25, 1.0, 2 / 32, 0.0, 1e-3, x, out)
    B.energy_noalloc(*args)
    torch.cuda.synchronize()
    ref = float(out.item())
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="global"):
        B.energy_noalloc(*args, stream=s)
    out.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert float(out.item()) == ref
