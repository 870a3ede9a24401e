"""ctypes binding of libpf (argument marshalling only: every step of the
path runs in the library's CUDA kernels).  Device vectors are torch CUDA
tensors (float64 or float32, contiguous); PyTorch supplies device memory and
the stream, nothing else.  Importing this module fails loudly if libpf.so
has not been built."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpf.so")

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ENONFINITE, PF_ENOTCONV, PF_ETIMEOUT, PF_ESTATE, PF_EIO = \
    range(9)
PF_FP64, PF_FP32 = 0, 1
PF_GALERKIN, PF_FIRST_ORDER = 0, 1
PF_LINE2D, PF_DISC3D, PF_BOX3D = 0, 1, 2
PF_START_PLAIN, PF_START_EXTRAPOLATE = 0, 1
PF_QP_CG, PF_QP_PAPER = 0, 1

STATUS_NAMES = {0: "PF_OK", 1: "PF_EINVAL", 2: "PF_ENOMEM", 3: "PF_ECUDA", 4: "PF_ENONFINITE",
                5: "PF_ENOTCONV", 6: "PF_ETIMEOUT", 7: "PF_ESTATE", 8: "PF_EIO"}

# every symbol include/pf.h declares
EXPORTS = [
    "pf_rmtr_params_default", "pf_last_error", "pf_mesh_hierarchy_create",
    "pf_mesh_hierarchy_destroy", "pf_level_info", "pf_fractures_set", "pf_pressure_set",
    "pf_energy", "pf_energy_diff", "pf_gradient", "pf_hessvec", "pf_prolong", "pf_restrict",
    "pf_project", "pf_coarse_bounds", "pf_rmtr_load_step", "pf_rmtr_load_step_host",
    "pf_get_c_prev", "pf_probe_fma", "pf_energy_noalloc", "pf_hessvec_lag_set",
    "pf_hessvec_lagged", "pf_unet_create", "pf_unet_destroy", "pf_unet_num_params",
    "pf_unet_set_params", "pf_unet_get_params", "pf_unet_get_grads", "pf_unet_forward",
    "pf_unet_backward", "pf_unet_mse", "pf_unet_adam", "pf_learned_features", "pf_learned_target",
    "pf_learned_apply", "pf_learned_propose", "pf_projected_gradient", "pf_rmtr_load_step_batch",
    "pf_energy_diff_mixed", "pf_gradient_step", "pf_gradient_df", "pf_energy_df",
    "pf_state_save", "pf_state_load", "pf_galerkin_set", "pf_galerkin_apply", "pf_qp_pgs",
    "pf_qp_mprgp", "pf_autotune", "pf_tile_variant_set", "pf_tile_variant_get",
    "pf_batch_create", "pf_batch_destroy", "pf_batch_info", "pf_batch_hessvec", "pf_batch_energy",
    "pf_batch_autotune", "pf_batch_variant_set", "pf_get_fields",
]


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_coarse", C.c_int * 3), ("n_levels", C.c_int),
                ("h_coarse", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("Gc", C.c_double), ("ls_over_h", C.c_double), ("k_res", C.c_double),
                ("stream", C.c_void_p)]


class RmtrParams(C.Structure):
    _fields_ = [("eta1", C.c_double), ("eta2", C.c_double), ("gamma1", C.c_double),
                ("gamma2", C.c_double), ("delta0", C.c_double), ("delta_max", C.c_double),
                ("mu1", C.c_int), ("mu2", C.c_int), ("coarse_its", C.c_int),
                ("cg_fine", C.c_int), ("cg_smooth", C.c_int), ("cg_coarse", C.c_int),
                ("cauchy_backtracks", C.c_int), ("cauchy_c", C.c_double),
                ("max_cycles", C.c_int), ("rtol", C.c_double), ("atol", C.c_double),
                ("coarse_model", C.c_int), ("precision", C.c_int),
                ("precondition", C.c_int), ("level_rtol", C.c_double),
                ("max_restarts", C.c_int), ("keep_c_prev", C.c_int), ("pg_ref", C.c_double),
                ("start", C.c_int), ("p_prev", C.c_double), ("qp_solver", C.c_int),
                ("pgs_sweeps", C.c_int)]


class RmtrStats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("converged", C.c_int), ("energy", C.c_double),
                ("pg0", C.c_double), ("pg", C.c_double), ("hessvecs", C.c_longlong),
                ("cg", C.c_longlong), ("tr_its", C.c_longlong), ("tr_rejected", C.c_longlong),
                ("coarse_rejected", C.c_longlong), ("seconds", C.c_double),
                ("launches", C.c_longlong), ("fe_hessvec", C.c_double),
                ("fe_gradient", C.c_double), ("fe_energy", C.c_double),
                ("cg_level", C.c_longlong * 8), ("tr_level", C.c_longlong * 8),
                ("rej_level", C.c_longlong * 8), ("hv_cauchy", C.c_longlong),
                ("hv_search", C.c_longlong), ("cg_restarts", C.c_longlong),
                ("pg_ref", C.c_double)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if k.endswith("_level") else v
        return out


class PfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libpf.so not built at {path}; run paper_2007_12908_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "pf_rmtr_params_default": (None, [C.POINTER(RmtrParams)]),
        "pf_last_error": (C.c_char_p, []),
        "pf_mesh_hierarchy_create": (i, [C.POINTER(MeshDesc), C.POINTER(vp)]),
        "pf_mesh_hierarchy_destroy": (i, [vp]),
        "pf_level_info": (i, [vp, i, C.POINTER(C.c_int), C.POINTER(d), C.POINTER(C.c_longlong)]),
        "pf_fractures_set": (i, [vp, i, i, vp, d, vp]),
        "pf_pressure_set": (i, [vp, d]),
        "pf_energy": (i, [vp, i, vp, i, C.POINTER(d)]),
        "pf_energy_diff": (i, [vp, i, vp, vp, i, vp]),
        "pf_gradient": (i, [vp, i, vp, vp, i]),
        "pf_energy_diff_mixed": (i, [vp, i, vp, vp, vp, vp]),
        "pf_gradient_step": (i, [vp, i, vp, vp, vp]),
        "pf_gradient_df": (i, [vp, i, vp, vp]),
        "pf_energy_df": (i, [vp, i, vp, C.POINTER(d)]),
        "pf_hessvec": (i, [vp, i, vp, vp, vp, i]),
        "pf_prolong": (i, [vp, i, vp, vp, i]),
        "pf_restrict": (i, [vp, i, vp, vp, i]),
        "pf_project": (i, [vp, i, vp, vp, i]),
        "pf_coarse_bounds": (i, [vp, i, vp, vp, vp, vp]),
        "pf_rmtr_load_step": (i, [vp, vp, C.POINTER(RmtrParams), C.POINTER(RmtrStats)]),
        "pf_rmtr_load_step_host": (i, [vp, vp, C.POINTER(RmtrParams), C.POINTER(RmtrStats)]),
        "pf_get_c_prev": (i, [vp, vp]),
        "pf_state_save": (i, [vp, vp, C.c_char_p]),
        "pf_state_load": (i, [vp, vp, C.c_char_p]),
        "pf_galerkin_set": (i, [vp, vp]),
        "pf_qp_pgs": (i, [vp, i, vp, vp, vp, vp, i]),
        "pf_autotune": (i, [vp, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "pf_tile_variant_set": (i, [vp, i, i]),
        "pf_tile_variant_get": (i, [vp, i, C.POINTER(C.c_int)]),
        "pf_qp_mprgp": (i, [vp, i, vp, vp, vp, vp, d, i, C.POINTER(C.c_int)]),
        "pf_galerkin_apply": (i, [vp, i, vp, vp, i]),
        "pf_probe_fma": (i, [i, C.POINTER(d)]),
        "pf_energy_noalloc": (i, [i, C.POINTER(C.c_int), d, d, d, d, d, d, d, vp, i, vp, vp]),
        "pf_hessvec_lag_set": (i, [vp, i, vp, i]),
        "pf_hessvec_lagged": (i, [vp, i, vp, vp, i]),
        "pf_unet_create": (i, [i, i, i, i, C.POINTER(C.c_int), vp, C.POINTER(vp)]),
        "pf_unet_destroy": (i, [vp]),
        "pf_unet_num_params": (i, [vp, C.POINTER(C.c_longlong)]),
        "pf_unet_set_params": (i, [vp, vp]),
        "pf_unet_get_params": (i, [vp, vp]),
        "pf_unet_get_grads": (i, [vp, vp]),
        "pf_unet_forward": (i, [vp, vp, vp]),
        "pf_unet_backward": (i, [vp, vp]),
        "pf_unet_mse": (i, [vp, vp, vp, vp, d, vp, C.POINTER(d)]),
        "pf_unet_adam": (i, [vp, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float]),
        "pf_learned_features": (i, [vp, vp, vp, d, d, i, i, vp]),
        "pf_learned_target": (i, [vp, vp, vp, d, d, i, i, vp]),
        "pf_learned_apply": (i, [vp, vp, vp, d, d, i, i, vp]),
        "pf_learned_propose": (i, [vp, vp, vp, d, C.POINTER(d), C.POINTER(C.c_int)]),
        "pf_projected_gradient": (i, [vp, vp, C.POINTER(d)]),
        "pf_rmtr_load_step_batch": (i, [i, C.POINTER(vp), C.POINTER(vp), C.POINTER(RmtrParams), i,
                                        C.POINTER(RmtrStats), C.POINTER(C.c_int)]),
        "pf_batch_create": (i, [i, C.POINTER(vp), vp, C.POINTER(vp)]),
        "pf_batch_destroy": (i, [vp]),
        "pf_batch_info": (i, [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "pf_batch_hessvec": (i, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), vp]),
        "pf_batch_energy": (i, [vp, C.POINTER(vp), C.POINTER(d)]),
        "pf_batch_autotune": (i, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int),
                                  C.POINTER(d)]),
        "pf_batch_variant_set": (i, [vp, i]),
        "pf_get_fields": (i, [vp, i, i, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def _check(status):
    if status != PF_OK:
        raise PfError(status, lib().pf_last_error().decode())


def default_params(**overrides) -> RmtrParams:
    p = RmtrParams()
    lib().pf_rmtr_params_default(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# ------------------------------------------------------------------ tensors
def _prec(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return PF_FP64
    if t.dtype == torch.float32:
        return PF_FP32
    raise TypeError("vectors must be float64 or float32")


def _dev(t, n=None, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} values, got {t.numel()}")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


class Hierarchy:
    """Owns a pf_hierarchy*.  Level 0 is the coarsest grid."""

    def __init__(self, handle, dim, n_levels, stream):
        self.handle = handle
        self.dim = dim
        self.n_levels = n_levels
        self.stream = stream
        self.levels = []
        for l in range(n_levels):
            n = (C.c_int * 3)()
            hh = C.c_double()
            nodes = C.c_longlong()
            _check(lib().pf_level_info(handle, l, n, C.byref(hh), C.byref(nodes)))
            self.levels.append((tuple(n[k] for k in range(dim)), hh.value, nodes.value))

    def nodes(self, level=-1):
        return self.levels[level][2]

    def ndof(self, level=-1):
        return (self.dim + 1) * self.nodes(level)

    def close(self):
        if self.handle:
            lib().pf_mesh_hierarchy_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mesh_hierarchy_create(dim, n_coarse, n_levels, h_coarse, E=1.0, nu=0.3, Gc=1.0,
                          ls_over_h=2.0, k_res=0.0, stream=None) -> Hierarchy:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    d = MeshDesc()
    d.dim = dim
    for k in range(3):
        d.n_coarse[k] = int(n_coarse[k]) if k < dim else 1
    d.n_levels = n_levels
    d.h_coarse = h_coarse
    d.E, d.nu, d.Gc, d.ls_over_h, d.k_res = E, nu, Gc, ls_over_h, k_res
    d.stream = C.c_void_p(stream.cuda_stream)
    h = C.c_void_p()
    _check(lib().pf_mesh_hierarchy_create(C.byref(d), C.byref(h)))
    return Hierarchy(h, dim, n_levels, stream)


def fractures_set(H: Hierarchy, kind: int, rows, band_half_width: float, x):
    import torch
    rows = np.ascontiguousarray(np.atleast_2d(np.asarray(rows, dtype=np.float64)))
    width = {PF_LINE2D: 4, PF_DISC3D: 7, PF_BOX3D: 14}.get(kind, 0)
    if rows.size and rows.shape[1] != width:
        raise ValueError(f"fracture rows must have {width} columns")
    n = rows.shape[0] if rows.size else 0
    _check(lib().pf_fractures_set(H.handle, kind, n, rows.ctypes.data_as(C.c_void_p),
                                  band_half_width, _dev(x, H.ndof(), torch.float64)))


def pressure_set(H: Hierarchy, p: float):
    _check(lib().pf_pressure_set(H.handle, float(p)))


def energy(H: Hierarchy, level: int, x) -> float:
    out = C.c_double()
    _check(lib().pf_energy(H.handle, level, _dev(x, H.ndof(level)), _prec(x), C.byref(out)))
    return out.value


def energy_diff(H: Hierarchy, level: int, x, s) -> np.ndarray:
    if x.dtype != s.dtype:
        raise TypeError("x and s must share a dtype")
    out = np.zeros(4)
    _check(lib().pf_energy_diff(H.handle, level, _dev(x, H.ndof(level)), _dev(s, H.ndof(level)),
                                _prec(x), out.ctypes.data_as(C.c_void_p)))
    return out


def energy_diff_mixed(H: Hierarchy, level: int, x, s, g) -> np.ndarray:
    """(g.s, a2, a3, a4): FP64 dot product and the FP32 higher-order
    coefficients of E(x + t s) - E(x); x, s, g FP64."""
    import torch
    n = H.ndof(level)
    out = np.zeros(4)
    _check(lib().pf_energy_diff_mixed(H.handle, level, _dev(x, n, torch.float64),
                                      _dev(s, n, torch.float64), _dev(g, n, torch.float64),
                                      out.ctypes.data_as(C.c_void_p)))
    return out


def gradient_df(H: Hierarchy, level: int, x, out=None):
    """Gradient of FP64 x in double-float arithmetic (FP64 result)."""
    import torch
    if out is None:
        out = torch.empty_like(x)
    n = H.ndof(level)
    _check(lib().pf_gradient_df(H.handle, level, _dev(x, n, torch.float64),
                                _dev(out, n, torch.float64)))
    return out


def energy_df(H: Hierarchy, level: int, x) -> float:
    """Energy of FP64 x in double-float arithmetic."""
    import torch
    out = C.c_double()
    _check(lib().pf_energy_df(H.handle, level, _dev(x, H.ndof(level), torch.float64), C.byref(out)))
    return out.value


def gradient_step(H: Hierarchy, level: int, x, s, g):
    """g += grad E(x) - grad E(x - s) in place (FP64 vectors, FP32 difference)."""
    import torch
    n = H.ndof(level)
    _check(lib().pf_gradient_step(H.handle, level, _dev(x, n, torch.float64),
                                  _dev(s, n, torch.float64), _dev(g, n, torch.float64)))
    return g


def gradient(H: Hierarchy, level: int, x, out=None):
    import torch
    if out is None:
        out = torch.empty_like(x)
    _check(lib().pf_gradient(H.handle, level, _dev(x, H.ndof(level)), _dev(out, H.ndof(level), x.dtype),
                             _prec(x)))
    return out


def hessvec(H: Hierarchy, level: int, x_lin, v, out=None):
    import torch
    if out is None:
        out = torch.empty_like(v)
    n = H.ndof(level)
    _check(lib().pf_hessvec(H.handle, level, _dev(x_lin, n, v.dtype), _dev(v, n), _dev(out, n, v.dtype),
                            _prec(v)))
    return out


def hessvec_lag_set(H: Hierarchy, level: int, x_lag):
    _check(lib().pf_hessvec_lag_set(H.handle, level, _dev(x_lag, H.ndof(level)), _prec(x_lag)))


def hessvec_lagged(H: Hierarchy, level: int, v, out=None):
    import torch
    if out is None:
        out = torch.empty_like(v)
    n = H.ndof(level)
    _check(lib().pf_hessvec_lagged(H.handle, level, _dev(v, n), _dev(out, n, v.dtype), _prec(v)))
    return out


def _xfer(fn, H, coarse, src, n_src, n_dst, out):
    import torch
    if out is None:
        out = torch.empty(n_dst, dtype=src.dtype, device=src.device)
    _check(fn(H.handle, coarse, _dev(src, n_src), _dev(out, n_dst, src.dtype), _prec(src)))
    return out


def prolong(H: Hierarchy, coarse: int, vc, out=None):
    return _xfer(lib().pf_prolong, H, coarse, vc, H.ndof(coarse), H.ndof(coarse + 1), out)


def restrict(H: Hierarchy, coarse: int, vf, out=None):
    return _xfer(lib().pf_restrict, H, coarse, vf, H.ndof(coarse + 1), H.ndof(coarse), out)


def project(H: Hierarchy, coarse: int, xf, out=None):
    return _xfer(lib().pf_project, H, coarse, xf, H.ndof(coarse + 1), H.ndof(coarse), out)


def coarse_bounds(H: Hierarchy, coarse: int, lo_f, hi_f):
    import torch
    nf, nc = H.ndof(coarse + 1), H.ndof(coarse)
    lo_c = torch.empty(nc, dtype=torch.float64, device=lo_f.device)
    hi_c = torch.empty_like(lo_c)
    _check(lib().pf_coarse_bounds(H.handle, coarse, _dev(lo_f, nf, torch.float64),
                                  _dev(hi_f, nf, torch.float64), _dev(lo_c, nc), _dev(hi_c, nc)))
    return lo_c, hi_c


def rmtr_load_step(H: Hierarchy, x, params: RmtrParams | None = None, check=True) -> dict:
    import torch
    st = RmtrStats()
    p = params if params is not None else default_params()
    rc = lib().pf_rmtr_load_step(H.handle, _dev(x, H.ndof(), torch.float64), C.byref(p), C.byref(st))
    if check and rc not in (PF_OK,):
        _check(rc)
    d = st.as_dict()
    d["status"] = rc
    return d


def rmtr_load_step_host(H: Hierarchy, x: np.ndarray, params: RmtrParams | None = None,
                        check=True) -> dict:
    if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"] or x.size != H.ndof():
        raise ValueError("x must be a contiguous float64 array of the finest size")
    st = RmtrStats()
    p = params if params is not None else default_params()
    rc = lib().pf_rmtr_load_step_host(H.handle, x.ctypes.data_as(C.c_void_p), C.byref(p), C.byref(st))
    if check and rc not in (PF_OK,):
        _check(rc)
    d = st.as_dict()
    d["status"] = rc
    return d


def projected_gradient(H: Hierarchy, x) -> float:
    import torch
    out = C.c_double()
    _check(lib().pf_projected_gradient(H.handle, _dev(x, H.ndof(), torch.float64), C.byref(out)))
    return out.value


def rmtr_load_step_batch(Hs, xs, params: RmtrParams | None = None, n_threads=0, check=True):
    """One load step of every (hierarchy, state) pair, run concurrently by the
    library's host workers; each hierarchy should own its stream."""
    import torch
    n = len(Hs)
    hv = (C.c_void_p * n)(*[H.handle for H in Hs])
    xv = (C.c_void_p * n)(*[_dev(x, H.ndof(), torch.float64).value for H, x in zip(Hs, xs)])
    st = (RmtrStats * n)()
    status = (C.c_int * n)()
    p = params if params is not None else default_params()
    rc = lib().pf_rmtr_load_step_batch(n, hv, xv, C.byref(p), n_threads, st, status)
    if check and rc != PF_OK:
        _check(rc)
    out = []
    for i in range(n):
        d = st[i].as_dict()
        d["status"] = status[i]
        out.append(d)
    return out


def get_c_prev(H: Hierarchy):
    import torch
    out = torch.empty(H.nodes(), dtype=torch.float64, device="cuda")
    _check(lib().pf_get_c_prev(H.handle, _dev(out, H.nodes())))
    return out


PF_FIELD_C_PREV, PF_FIELD_LOWER, PF_FIELD_UPPER, PF_FIELD_FIXED = 0, 1, 2, 3


def get_fields(H: Hierarchy, level: int, which: int):
    """A field the solver keeps for a level (pf_get_fields): c_prev (finest
    level), the feasible set's lower / upper bounds, or the fixed-dof mask."""
    import torch
    n = H.nodes(level) if which == PF_FIELD_C_PREV else H.ndof(level)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    _check(lib().pf_get_fields(H.handle, level, which, _dev(out, n)))
    return out


def state_save(H: Hierarchy, x, path):
    """Checkpoint: the finest state x (float64 CUDA tensor), c_prev and the
    pressures to the file `path`."""
    import torch
    _check(lib().pf_state_save(H.handle, _dev(x, H.ndof(), torch.float64), os.fsencode(path)))


def state_load(H: Hierarchy, x, path):
    """Resume: restores a pf_state_save file into H and the float64 CUDA
    tensor x (nothing changes unless the file passes every check)."""
    import torch
    _check(lib().pf_state_load(H.handle, _dev(x, H.ndof(), torch.float64), os.fsencode(path)))
    return x


def autotune(H: Hierarchy):
    """Times every tile variant of each level's FP32 Hessian product and
    keeps the fastest; returns (variants per level, microseconds per
    (level, variant), -1 where a variant does not apply)."""
    var = (C.c_int * H.n_levels)()
    us = (C.c_double * (5 * H.n_levels))()
    _check(lib().pf_autotune(H.handle, var, us))
    return list(var), [list(us[5 * l:5 * l + 5]) for l in range(H.n_levels)]


def tile_variant_set(H: Hierarchy, level: int, variant: int):
    _check(lib().pf_tile_variant_set(H.handle, level, variant))


def tile_variant_get(H: Hierarchy, level: int) -> int:
    out = C.c_int()
    _check(lib().pf_tile_variant_get(H.handle, level, C.byref(out)))
    return out.value


class Batch:
    """Batched 2D operators over the finest levels of several hierarchies:
    one persistent launch per call over every instance (pf_batch_*).  The
    hierarchies must stay open while the batch is used."""

    def __init__(self, Hs, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.Hs = list(Hs)
        hv = (C.c_void_p * len(self.Hs))(*[H.handle for H in self.Hs])
        out = C.c_void_p()
        _check(lib().pf_batch_create(len(self.Hs), hv, C.c_void_p(stream.cuda_stream), C.byref(out)))
        self.handle = out

    def info(self):
        dofs, bps, sms = C.c_longlong(), C.c_int(), C.c_int()
        _check(lib().pf_batch_info(self.handle, C.byref(dofs), C.byref(bps), C.byref(sms)))
        return {"dofs": dofs.value, "blocks_per_sm": bps.value, "sms": sms.value}

    def _tables(self, xs, vs, ys):
        import torch
        n = len(self.Hs)
        if not (len(xs) == len(vs) == len(ys) == n):
            raise ValueError("one x, v and Hv per instance")
        xt = (C.c_void_p * n)(*[_dev(x, H.ndof(), torch.float32).value for H, x in zip(self.Hs, xs)])
        vt = (C.c_void_p * n)(*[_dev(v, H.ndof(), torch.float32).value for H, v in zip(self.Hs, vs)])
        yt = (C.c_void_p * n)(*[_dev(y, H.ndof(), torch.float32).value for H, y in zip(self.Hs, ys)])
        return xt, vt, yt

    def hessvec(self, xs, vs, ys=None, vhv=None):
        """ys[i] = H(xs[i]) vs[i] (float32 CUDA tensors); with vhv (a float64
        CUDA tensor of one value per instance) also vs[i] . ys[i]."""
        import torch
        ys = [torch.empty_like(v) for v in vs] if ys is None else ys
        xt, vt, yt = self._tables(xs, vs, ys)
        dp = _dev(vhv, len(self.Hs), torch.float64) if vhv is not None else None
        _check(lib().pf_batch_hessvec(self.handle, xt, vt, yt, dp))
        return ys

    def energy(self, xs):
        """Energies of float64 states xs[i], one float per instance."""
        import torch
        n = len(self.Hs)
        xt = (C.c_void_p * n)(*[_dev(x, H.ndof(), torch.float64).value for H, x in zip(self.Hs, xs)])
        out = (C.c_double * n)()
        _check(lib().pf_batch_energy(self.handle, xt, out))
        return list(out)

    def autotune(self, xs, vs, ys):
        xt, vt, yt = self._tables(xs, vs, ys)
        bps = C.c_int()
        us = (C.c_double * 4)()
        _check(lib().pf_batch_autotune(self.handle, xt, vt, yt, C.byref(bps), us))
        return bps.value, list(us)

    def variant_set(self, blocks_per_sm):
        _check(lib().pf_batch_variant_set(self.handle, blocks_per_sm))

    def close(self):
        if self.handle:
            lib().pf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qp_pgs(H: Hierarchy, level: int, g, lo, hi, s, sweeps):
    """Symmetric multicolour projected Gauss-Seidel sweeps on s (in place)
    with the level's lagged FP64 stencil (pf_hessvec_lag_set first)."""
    import torch
    n = H.ndof(level)
    _check(lib().pf_qp_pgs(H.handle, level, _dev(g, n, torch.float64), _dev(lo, n, torch.float64),
                           _dev(hi, n, torch.float64), _dev(s, n, torch.float64), sweeps))
    return s


def qp_mprgp(H: Hierarchy, level: int, g, lo, hi, tol, maxit, out=None):
    """MPRGP on the level's lagged FP64 stencil; returns (s, products)."""
    import torch
    n = H.ndof(level)
    out = torch.empty_like(g) if out is None else out
    used = C.c_int()
    _check(lib().pf_qp_mprgp(H.handle, level, _dev(g, n, torch.float64), _dev(lo, n, torch.float64),
                             _dev(hi, n, torch.float64), _dev(out, n, torch.float64), float(tol),
                             int(maxit), C.byref(used)))
    return out, used.value


def galerkin_set(H: Hierarchy, x_lag_fine):
    """Builds the stored FP32 Galerkin operators R G I of every coarse level
    from the finest level's lag point (a float32 CUDA tensor)."""
    import torch
    _check(lib().pf_galerkin_set(H.handle, _dev(x_lag_fine, H.ndof(), torch.float32)))


def galerkin_apply(H: Hierarchy, level: int, v, out=None):
    """The stored Galerkin operator of coarse level `level` applied to v
    (float32 or float64 CUDA tensor of that level's size)."""
    import torch
    n = H.ndof(level)
    out = torch.empty_like(v) if out is None else out
    _check(lib().pf_galerkin_apply(H.handle, level, _dev(v, n), _dev(out, n, v.dtype), _prec(v)))
    return out


def probe_fma(prec: int) -> float:
    """Measured FMA throughput (flop/s) of this GPU in the given precision."""
    out = C.c_double()
    _check(lib().pf_probe_fma(prec, C.byref(out)))
    return out.value


def energy_noalloc(dim, n, h, E, nu, Gc, ls, k_res, p, x, out, stream=None):
    """pf_energy_noalloc: the energy written to the one-element float64 CUDA
    tensor `out` on `stream`, with no device allocation inside the call."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    nn = (C.c_int * 3)(*[int(v) for v in list(n) + [1] * (3 - len(n))])
    _check(lib().pf_energy_noalloc(dim, nn, h, E, nu, Gc, ls, k_res, p, _dev(x), _prec(x),
                                   _dev(out, 1, torch.float64), C.c_void_p(stream.cuda_stream)))
    return out


# ------------------------------------------------------------------ learned iterate
class Unet:
    """Owns a pf_unet* (the learned initial-iterate network)."""

    def __init__(self, height, width, n_in=5, n_out=3, channels=(16, 32, 64, 128), stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.H, self.W, self.n_in, self.n_out = height, width, n_in, n_out
        ch = (C.c_int * 4)(*channels)
        h = C.c_void_p()
        _check(lib().pf_unet_create(height, width, n_in, n_out, ch, C.c_void_p(stream.cuda_stream),
                                    C.byref(h)))
        self.handle = h
        n = C.c_longlong()
        _check(lib().pf_unet_num_params(h, C.byref(n)))
        self.n_params = n.value

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        if flat.size != self.n_params:
            raise ValueError("parameter vector has the wrong size")
        _check(lib().pf_unet_set_params(self.handle, flat.ctypes.data_as(C.c_void_p)))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib().pf_unet_get_params(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out

    def get_grads(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib().pf_unet_get_grads(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out

    def forward(self, x, out=None):
        import torch
        if out is None:
            out = torch.empty((self.n_out, self.H, self.W), dtype=torch.float32, device="cuda")
        _check(lib().pf_unet_forward(self.handle, _dev(x, self.n_in * self.H * self.W, torch.float32),
                                     _dev(out, self.n_out * self.H * self.W, torch.float32)))
        return out

    def backward(self, dy):
        import torch
        _check(lib().pf_unet_backward(self.handle, _dev(dy, self.n_out * self.H * self.W, torch.float32)))

    def mse(self, y, t, mask=None, n_valid=None, dy=None):
        import torch
        if dy is None:
            dy = torch.empty_like(y)
        loss = C.c_double()
        m = _dev(mask, self.H * self.W, torch.float32) if mask is not None else None
        nv = float(n_valid) if mask is not None else 1.0
        _check(lib().pf_unet_mse(self.handle, _dev(y), _dev(t), m, nv, _dev(dy), C.byref(loss)))
        return loss.value, dy

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0):
        _check(lib().pf_unet_adam(self.handle, lr, beta1, beta2, eps, grad_scale))

    def close(self):
        if getattr(self, "handle", None):
            lib().pf_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def learned_features(H: Hierarchy, x_prev, c_before, p_prev, p_new, height, width, out=None):
    import torch
    if out is None:
        out = torch.empty((5, height, width), dtype=torch.float32, device="cuda")
    cb = _dev(c_before, H.nodes(), torch.float64) if c_before is not None else None
    _check(lib().pf_learned_features(H.handle, _dev(x_prev, H.ndof(), torch.float64), cb, p_prev, p_new,
                                     height, width, _dev(out, 5 * height * width, torch.float32)))
    return out


def learned_target(H: Hierarchy, x_prev, x_new, p_prev, p_new, height, width, out=None):
    import torch
    if out is None:
        out = torch.empty((3, height, width), dtype=torch.float32, device="cuda")
    _check(lib().pf_learned_target(H.handle, _dev(x_prev, H.ndof(), torch.float64),
                                   _dev(x_new, H.ndof(), torch.float64), p_prev, p_new, height, width,
                                   _dev(out, 3 * height * width, torch.float32)))
    return out


def learned_apply(H: Hierarchy, x_prev, y, p_prev, p_new, out=None):
    import torch
    if out is None:
        out = torch.empty_like(x_prev)
    _check(lib().pf_learned_apply(H.handle, _dev(x_prev, H.ndof(), torch.float64),
                                  _dev(y, None, torch.float32), p_prev, p_new, y.shape[1], y.shape[2],
                                  _dev(out, H.ndof(), torch.float64)))
    return out


def learned_propose(H: Hierarchy, x, xhat, eta=0.1):
    import torch
    rho = C.c_double()
    acc = C.c_int()
    _check(lib().pf_learned_propose(H.handle, _dev(x, H.ndof(), torch.float64),
                                    _dev(xhat, H.ndof(), torch.float64), eta, C.byref(rho), C.byref(acc)))
    return rho.value, bool(acc.value)
