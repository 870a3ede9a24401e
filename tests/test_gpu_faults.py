"""Failure handling and checkpoint/resume, with every failure made on the
host (no GPU fault is ever provoked): a NaN or Inf planted in the state or a
fracture row, a hierarchy too large for the device, a corrupted or
mismatched state file.  Each failure must return its status and leave the
caller's state exactly as it was; a resumed ramp must reproduce the
uninterrupted one bit for bit."""
import os

import numpy as np
import pytest

import pfinputs as PI
from tests.gpu_common import require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    require_cuda()
    import paper_2007_12908_gb300 as m
    return m


def _setup(pf, precision=None):
    import torch
    H = pf.mesh_hierarchy_create(3, (5, 5, 5), 3, 1 / 4, E=1.0, nu=0.25, Gc=1.0)
    x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
    pf.fractures_set(H, pf.PF_DISC3D, PI.disc_network_3d(PI.SEED_3D_PLAIN, 20), H.levels[-1][1], x)
    return H, x


def _ramp(pf, H, x, ts, precision):
    out = []
    for t in ts:
        pf.pressure_set(H, 5e-4 * t)
        st = pf.rmtr_load_step(H, x, pf.default_params(precision=precision, start=pf.PF_START_EXTRAPOLATE,
                                                       p_prev=5e-4 * (t - 1)))
        out.append(st)
    return out


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
@pytest.mark.parametrize("field", [0, 3])
def test_nonfinite_state_is_refused_and_left_unchanged(pf, bad, field):
    import torch
    H, x = _setup(pf)
    _ramp(pf, H, x, [1], pf.PF_FP32)
    N = H.nodes()
    x[field * N + N // 3] = bad
    before = x.clone()
    cprev = pf.get_c_prev(H).clone()
    pf.pressure_set(H, 1e-3)
    st = pf.rmtr_load_step(H, x, pf.default_params(precision=pf.PF_FP32), check=False)
    torch.cuda.synchronize()
    assert st["status"] == pf.PF_ENONFINITE
    assert torch.equal(x.isnan(), before.isnan())
    same = (x == before) | (x.isnan() & before.isnan())
    assert bool(same.all())
    assert torch.equal(pf.get_c_prev(H), cprev)
    H.close()


def test_failed_step_does_not_change_the_next_one(pf):
    """A refused step in between leaves no trace: the ramp continues exactly
    as if it had not been attempted (c_prev and the last converged pressure
    unchanged)."""
    import torch
    Ha, xa = _setup(pf)
    Hb, xb = _setup(pf)
    _ramp(pf, Ha, xa, [1, 2], pf.PF_FP32)
    _ramp(pf, Hb, xb, [1], pf.PF_FP32)
    bad = xb.clone()
    bad[5] = float("nan")
    pf.pressure_set(Hb, 1e-3)
    st = pf.rmtr_load_step(Hb, bad, pf.default_params(precision=pf.PF_FP32,
                                                      start=pf.PF_START_EXTRAPOLATE), check=False)
    assert st["status"] == pf.PF_ENONFINITE
    _ramp(pf, Hb, xb, [2], pf.PF_FP32)
    torch.cuda.synchronize()
    assert torch.equal(xa, xb)
    Ha.close()
    Hb.close()


def test_nonfinite_fracture_row_is_refused(pf):
    import torch
    H, x = _setup(pf)
    before = x.clone()
    rows = PI.disc_network_3d(PI.SEED_3D_PLAIN, 20)
    rows[7, 6] = float("inf")
    with pytest.raises(pf.PfError) as e:
        pf.fractures_set(H, pf.PF_DISC3D, rows, H.levels[-1][1], x)
    assert e.value.status == pf.PF_ENONFINITE
    torch.cuda.synchronize()
    assert torch.equal(x, before)
    H.close()


def test_oversized_hierarchy_is_refused_with_nothing_allocated(pf):
    """A 3D hierarchy with 2049^3 finest nodes needs far more than the
    device holds: refused with PF_ENOMEM before any allocation, so the free
    device memory is unchanged."""
    import torch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    with pytest.raises(pf.PfError) as e:
        pf.mesh_hierarchy_create(3, (257, 257, 257), 4, 1 / 256)
    assert e.value.status == pf.PF_ENOMEM
    assert b"nothing was allocated" in str(e.value).encode()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_resume_reproduces_the_ramp(pf, precision, tmp_path):
    """Steps 1-2, checkpoint, step 3 in one hierarchy; a fresh hierarchy
    resumed from the checkpoint runs step 3 to the same state bit for bit."""
    import torch
    prec = pf.PF_FP64 if precision == "fp64" else pf.PF_FP32
    H, x = _setup(pf)
    _ramp(pf, H, x, [1, 2], prec)
    path = str(tmp_path / "state.pfs")
    pf.state_save(H, x, path)
    ref = _ramp(pf, H, x, [3], prec)[0]
    H2 = pf.mesh_hierarchy_create(3, (5, 5, 5), 3, 1 / 4, E=1.0, nu=0.25, Gc=1.0)
    x2 = torch.zeros(H2.ndof(), dtype=torch.float64, device="cuda")
    pf.state_load(H2, x2, path)
    got = _ramp(pf, H2, x2, [3], prec)[0]
    torch.cuda.synchronize()
    assert torch.equal(x, x2)
    assert got["energy"] == ref["energy"] and got["cycles"] == ref["cycles"]
    assert torch.equal(pf.get_c_prev(H), pf.get_c_prev(H2))
    H.close()
    H2.close()


def test_checkpoint_rejects_corrupt_and_mismatched_files(pf, tmp_path):
    import torch
    H, x = _setup(pf)
    _ramp(pf, H, x, [1], pf.PF_FP32)
    path = str(tmp_path / "state.pfs")
    pf.state_save(H, x, path)
    raw = bytearray(open(path, "rb").read())
    target = torch.full_like(x, 7.0)
    before = target.clone()
    # a flipped payload byte: checksum mismatch
    bad = bytearray(raw)
    bad[-100] ^= 0x10
    p_bad = str(tmp_path / "bad.pfs")
    open(p_bad, "wb").write(bad)
    with pytest.raises(pf.PfError) as e:
        pf.state_load(H, target, p_bad)
    assert e.value.status == pf.PF_EINVAL and "checksum" in str(e.value)
    # a truncated file
    p_short = str(tmp_path / "short.pfs")
    open(p_short, "wb").write(raw[:-8])
    with pytest.raises(pf.PfError) as e:
        pf.state_load(H, target, p_short)
    assert e.value.status == pf.PF_EIO
    # another grid
    H3 = pf.mesh_hierarchy_create(3, (5, 5, 5), 2, 1 / 4, E=1.0, nu=0.25, Gc=1.0)
    x3 = torch.zeros(H3.ndof(), dtype=torch.float64, device="cuda")
    with pytest.raises(pf.PfError) as e:
        pf.state_load(H3, x3, path)
    assert e.value.status == pf.PF_EINVAL and "grid" in str(e.value)
    # another material
    H4 = pf.mesh_hierarchy_create(3, (5, 5, 5), 3, 1 / 4, E=2.0, nu=0.25, Gc=1.0)
    with pytest.raises(pf.PfError) as e:
        pf.state_load(H4, target, path)
    assert e.value.status == pf.PF_EINVAL and "material" in str(e.value)
    # a missing file
    with pytest.raises(pf.PfError) as e:
        pf.state_load(H, target, str(tmp_path / "missing.pfs"))
    assert e.value.status == pf.PF_EIO
    torch.cuda.synchronize()
    assert torch.equal(target, before)
    # a state holding a NaN is not written
    x[3] = float("nan")
    with pytest.raises(pf.PfError) as e:
        pf.state_save(H, x, str(tmp_path / "nan.pfs"))
    assert e.value.status == pf.PF_ENONFINITE
    assert not os.path.exists(str(tmp_path / "nan.pfs"))
    for h in (H, H3, H4):
        h.close()
