"""C-ABI checks that need no GPU: every symbol include/pf.h declares is
exported, the ctypes structures match the C layout, and host-side argument
validation rejects bad input before any device work."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_2007_12908_gb300 import _binding as B
from paper_2007_12908_gb300 import build as BUILD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pf.h")


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_what_the_binding_lists():
    assert declared_functions() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pf_[a-z0-9_]+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def _c_layout():
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "pf.h"
#define F(T, f) printf(#T " " #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("pf_mesh_desc size %zu\n", sizeof(pf_mesh_desc));
  printf("pf_rmtr_params size %zu\n", sizeof(pf_rmtr_params));
  printf("pf_rmtr_stats size %zu\n", sizeof(pf_rmtr_stats));
  F(pf_mesh_desc, n_levels) F(pf_mesh_desc, h_coarse) F(pf_mesh_desc, k_res) F(pf_mesh_desc, stream)
  F(pf_rmtr_params, mu1) F(pf_rmtr_params, cauchy_c) F(pf_rmtr_params, max_cycles)
  F(pf_rmtr_params, rtol) F(pf_rmtr_params, precision)
  F(pf_rmtr_stats, energy) F(pf_rmtr_stats, hessvecs) F(pf_rmtr_stats, seconds)
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        return subprocess.run([exe], capture_output=True, text=True, check=True).stdout


def test_struct_layouts_match_header():
    got = {}
    for line in _c_layout().strip().splitlines():
        t, f, v = line.split()
        got[(t, f)] = int(v)
    py = {"pf_mesh_desc": B.MeshDesc, "pf_rmtr_params": B.RmtrParams, "pf_rmtr_stats": B.RmtrStats}
    for (t, f), v in got.items():
        cls = py[t]
        if f == "size":
            assert C.sizeof(cls) == v, t
        else:
            assert getattr(cls, f).offset == v, (t, f)


def test_defaults_and_validation_on_host(lib):
    p = B.default_params()
    assert (p.eta1, p.eta2, p.gamma1, p.gamma2) == (0.1, 0.75, 0.5, 2.0)
    assert p.mu1 == 1 and p.mu2 == 1 and p.coarse_its == 10
    d = B.MeshDesc()
    d.dim = 4
    h = C.c_void_p()
    assert lib.pf_mesh_hierarchy_create(C.byref(d), C.byref(h)) == B.PF_EINVAL
    assert b"dim" in lib.pf_last_error()
    d.dim = 2
    d.n_coarse[0] = 1
    d.n_coarse[1] = 5
    d.n_levels = 2
    d.h_coarse = 0.25
    d.E, d.nu, d.Gc, d.ls_over_h = 1.0, 0.3, 1.0, 2.0
    assert lib.pf_mesh_hierarchy_create(C.byref(d), C.byref(h)) == B.PF_EINVAL
    d.n_coarse[0] = 5
    d.nu = 0.5
    assert lib.pf_mesh_hierarchy_create(C.byref(d), C.byref(h)) == B.PF_EINVAL
    out = C.c_double()
    assert lib.pf_energy(None, 0, None, 0, C.byref(out)) == B.PF_EINVAL
    assert lib.pf_hessvec(None, 0, None, None, None, 0) == B.PF_EINVAL
    assert lib.pf_rmtr_load_step(None, None, None, None) == B.PF_EINVAL
    assert lib.pf_mesh_hierarchy_destroy(None) == B.PF_OK
    assert lib.pf_state_save(None, None, b"x") == B.PF_EINVAL
    assert lib.pf_state_load(None, None, None) == B.PF_EINVAL
    assert lib.pf_get_fields(None, 0, B.PF_FIELD_C_PREV, None) == B.PF_EINVAL


def test_batch_validation_on_host(lib):
    assert lib.pf_rmtr_load_step_batch(-1, None, None, None, 0, None, None) == B.PF_EINVAL
    hv = (C.c_void_p * 1)(None)
    xv = (C.c_void_p * 1)(None)
    assert lib.pf_rmtr_load_step_batch(1, hv, xv, None, 0, None, None) == B.PF_EINVAL
    assert lib.pf_rmtr_load_step_batch(0, None, None, None, 0, None, None) == B.PF_OK


def test_batched_operators_validation_on_host(lib):
    out = C.c_void_p()
    assert lib.pf_batch_create(0, None, None, C.byref(out)) == B.PF_EINVAL
    hv = (C.c_void_p * 2)(None, None)
    assert lib.pf_batch_create(2, hv, None, C.byref(out)) == B.PF_EINVAL
    assert b"null hierarchy" in lib.pf_last_error()
    assert lib.pf_batch_create(1, hv, None, None) == B.PF_EINVAL
    assert lib.pf_batch_hessvec(None, None, None, None, None) == B.PF_EINVAL
    assert lib.pf_batch_energy(None, None, None) == B.PF_EINVAL
    assert lib.pf_batch_info(None, None, None, None) == B.PF_EINVAL
    assert lib.pf_batch_autotune(None, None, None, None, None, None) == B.PF_EINVAL
    assert lib.pf_batch_variant_set(None, 1) == B.PF_EINVAL
    assert lib.pf_batch_destroy(None) == B.PF_OK
