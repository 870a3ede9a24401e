"""GB300 (sm_103a) hot path of the RMTR solver for pressure-induced AT2
phase-field fracture (Zulian, Kopanicakova et al., arXiv 2007.12908).

The compute path is libpf.so (hand-written CUDA kernels behind a C-ABI,
declared in include/pf.h); this package is its thin ctypes binding.  There
is no CPU fallback: calls raise if the library is not built or no CUDA
device is present."""
from ._binding import (  # noqa: F401
    PF_BOX3D, PF_DISC3D, PF_FIRST_ORDER, PF_FP32, PF_FP64, PF_GALERKIN, PF_LINE2D, PF_START_EXTRAPOLATE,
    PF_START_PLAIN, PfError,
    coarse_bounds, default_params, energy, energy_diff, fractures_set, get_c_prev, gradient,
    hessvec, hessvec_lag_set, hessvec_lagged, mesh_hierarchy_create, pressure_set, project, prolong, restrict, rmtr_load_step,
    rmtr_load_step_host, projected_gradient, rmtr_load_step_batch, energy_diff_mixed,
    gradient_step, gradient_df, energy_df, state_save, state_load, galerkin_set, galerkin_apply, qp_pgs, qp_mprgp, autotune, tile_variant_set, tile_variant_get,
    Batch, get_fields, PF_FIELD_C_PREV, PF_FIELD_LOWER, PF_FIELD_UPPER, PF_FIELD_FIXED,
    PF_QP_CG, PF_QP_PAPER,
    PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ENONFINITE, PF_ENOTCONV, PF_ETIMEOUT, PF_ESTATE, PF_EIO,
)
