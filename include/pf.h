/*
 * libpf -- GB300 (sm_103a) hot path of the recursive multilevel trust-region
 * (RMTR) solver for pressure-induced AT2 phase-field fracture.
 *
 * Method: Zulian, Kopanicakova et al., "Large scale simulation of pressure
 * induced phase-field fracture propagation using Utopia" (arXiv 2007.12908).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns a pf_status and never aborts.  pf_last_error() returns
 *   a message for the calling thread's most recent failure.
 * - State vectors hold (d+1) planes [u_x, u_y, (u_z), c] of N nodal values
 *   each, lexicographic with x fastest (node (i,j,k) -> i + n_x (j + n_y k)).
 *   A level's vector therefore has (d+1) * N entries.
 * - "dev" pointers are device memory owned by the caller (borrowed: they must
 *   stay valid until the library's stream is synchronised).  "host" pointers
 *   are ordinary host memory read or written before the call returns.
 * - All device work is enqueued on the cudaStream_t given in pf_mesh_desc
 *   (passed as void*).  Calls returning host scalars synchronise that stream.
 * - Precision codes: PF_FP64 (double) or PF_FP32 (float) for vector arguments.
 * - Level index 0 is the coarsest grid, n_levels-1 the finest (the paper's
 *   l = 1 ... L).
 * - The library owns only its internal buffers; pf_mesh_hierarchy_destroy
 *   frees them.
 */
#ifndef PF_H
#define PF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef int pf_status;
#define PF_OK 0
#define PF_EINVAL 1      /* bad argument (size, level, pointer, kind)        */
#define PF_ENOMEM 2      /* device or host allocation failed                 */
#define PF_ECUDA 3       /* a CUDA runtime call failed                       */
#define PF_ENONFINITE 4  /* a NaN/Inf appeared in an input or a result       */
#define PF_ENOTCONV 5    /* rmtr_load_step hit max_cycles                    */
#define PF_ETIMEOUT 6    /* a bounded device wait ran out                    */
#define PF_ESTATE 7      /* call order violated (e.g. no fractures set)      */
#define PF_EIO 8         /* a state file could not be read or written        */

#define PF_FP64 0
#define PF_FP32 1

#define PF_GALERKIN 0    /* coarse model Hessian R H_{l+1} I (second order)   */
#define PF_FIRST_ORDER 1 /* coarse model Hessian = Hessian of f~ at x0        */

#define PF_LINE2D 0 /* rows [cx, cy, theta, half_length]                      */
#define PF_DISC3D 1 /* rows [cx, cy, cz, nx, ny, nz, radius], |n| = 1         */
#define PF_BOX3D 2  /* rows [cx, cy, cz, nx, ny, nz, ax, ay, az, bx, by, bz,
                       half_a, half_b]: a rectangular plate (the paper's
                       "smooth parallelepiped" before its band width) with
                       unit normal n and unit in-plane axes a, b           */

typedef struct pf_hierarchy pf_hierarchy;

/* Structured grid hierarchy and material (Sec. 2 and Sec. 4.1, steps 2-4). */
typedef struct {
  int dim;            /* 2 or 3                                              */
  int n_coarse[3];    /* nodes per axis on the coarsest level (>= 2)         */
  int n_levels;       /* 1 .. 8; level l has (n_coarse-1) 2^l + 1 nodes/axis */
  double h_coarse;    /* node spacing of the coarsest level                  */
  double E, nu;       /* Young's modulus, Poisson ratio (Lame via plane strain
                         in 2D)                                              */
  double Gc;          /* fracture toughness                                  */
  double ls_over_h;   /* l_s = ls_over_h * h_finest on every level (Sec. 5: 2) */
  double k_res;       /* residual stiffness in g(c) = (1-k)(1-c)^2 + k (0)   */
  void* stream;       /* cudaStream_t for all work (NULL = legacy stream)    */
} pf_mesh_desc;

/* Trust-region and RMTR controls (Algorithms 1-3). */
typedef struct {
  double eta1, eta2;     /* acceptance / expansion thresholds (0.1, 0.75)    */
  double gamma1, gamma2; /* radius shrink / expand factors (0.5, 2.0)        */
  double delta0;         /* initial TR radius (inf-norm) per load step (1.0) */
  double delta_max;      /* cap on the radius (1.0)                          */
  int mu1, mu2;          /* pre/post smoothing TR steps (1, 1)               */
  int coarse_its;        /* TR steps on the coarsest level (10)              */
  int cg_fine;           /* CG budget per subproblem, finest level (50)      */
  int cg_smooth;         /* ... intermediate levels (10)                     */
  int cg_coarse;         /* ... coarsest level (500)                         */
  int cauchy_backtracks; /* Cauchy / projected-search halvings (30)          */
  double cauchy_c;       /* sufficient-decrease constant (0.01)              */
  int max_cycles;        /* V-cycles per load step (200)                     */
  double rtol;           /* stop when ||x - P(x - grad f)|| <= rtol * start  */
  double atol;           /* ... or <= atol                                   */
  int coarse_model;      /* PF_GALERKIN or PF_FIRST_ORDER                    */
  int precision;         /* PF_FP64, or PF_FP32 = mixed: on every level an
                            FP32 Hessian and FP32 subproblem, FP32 gradient
                            steps after accepted steps and FP32 higher-order
                            terms of rho's energy difference; double-float
                            (pf_gradient_df) stopping-test gradients and
                            energy; FP64 first-order term of rho, radius and
                            norms                                            */
  int precondition;      /* 1: Jacobi (Hessian-diagonal) preconditioned CG (1) */
  double level_rtol;     /* a non-finest level stops its TR steps once its
                            projected gradient fell by this factor (1e-3;
                            0 = always take the full count)                  */
  int max_restarts;      /* CG restarts after a projected search, per
                            subproblem (1000000 = unlimited)                 */
  int keep_c_prev;       /* 0: c_prev := c of x on entry; 1: keep the
                            hierarchy's c_prev (set by pf_learned_propose)   */
  double pg_ref;         /* > 0: the stopping test is relative to this value
                            instead of the start's own projected gradient,
                            so that every starting point stops at the same
                            accuracy (see pf_projected_gradient); 0 = start  */
  int start;             /* PF_START_PLAIN: iterate from x as given;
                            PF_START_EXTRAPOLATE: scale u by p / p_last (the
                            pressure of the last converged step), c kept,
                            with the stopping test relative to the plain
                            start (pg_ref taken at x as given)               */
  double p_prev;         /* > 0: the previous pressure for
                            PF_START_EXTRAPOLATE instead of p_last           */
  int qp_solver;         /* PF_QP_CG: projected truncated CG on every level
                            (default); PF_QP_PAPER: the paper's QP solvers
                            (Sec. 4.2.2): pgs_sweeps symmetric multicolour
                            projected Gauss-Seidel sweeps on the
                            non-coarsest levels, MPRGP (cg_coarse products)
                            on the coarsest; needs precision PF_FP64 and
                            coarse_model PF_FIRST_ORDER (assembled FP64
                            Hessians on every level)                        */
  int pgs_sweeps;        /* symmetric PGS sweeps per TR subproblem (2)      */
} pf_rmtr_params;

#define PF_START_PLAIN 0
#define PF_START_EXTRAPOLATE 1
#define PF_QP_CG 0
#define PF_QP_PAPER 1

typedef struct {
  int cycles;            /* V-cycles taken                                   */
  int converged;         /* 1 if the stopping test passed                    */
  double energy;         /* E(x) at return (FP64; double-float in mixed mode) */
  double pg0, pg;        /* projected-gradient norm at start / at return;
                            pg0 of an extrapolated mixed-precision start uses
                            the FP32 gradient step from x_{t-1} (its error is
                            relative to the change of the gradient)         */
  long long hessvecs;    /* Hessian-vector products on any level             */
  long long cg;          /* CG iterations                                    */
  long long tr_its;      /* TR iterations on all levels                      */
  long long tr_rejected; /* rejected TR steps                                */
  long long coarse_rejected; /* rejected coarse corrections (eq. rho_ml)     */
  double seconds;        /* wall time of the call                            */
  long long launches;    /* CUDA kernel launches made by the call            */
  double fe_hessvec;     /* Hessian-vector products, in finest-level units
                            (a level-l call counts N_l / N_finest)           */
  double fe_gradient;    /* gradients, finest-level units                    */
  double fe_energy;      /* energy / energy-difference passes, finest units  */
  long long cg_level[8]; /* CG iterations per level (index = level, <= 8)    */
  long long tr_level[8]; /* TR iterations per level                          */
  long long rej_level[8];/* rejected TR steps per level                      */
  long long hv_cauchy;   /* Hessian applications in Cauchy-point searches    */
  long long hv_search;   /* Hessian applications in projected searches       */
  long long cg_restarts; /* CG runs restarted after a projected search       */
  double pg_ref;         /* the stopping test's reference: params.pg_ref if
                            given, else the projected gradient at the plain
                            start (extrapolated start), else pg0           */
} pf_rmtr_stats;

/* Fills p with the defaults listed beside each field above. */
void pf_rmtr_params_default(pf_rmtr_params* p);

/* Message of this thread's last failure ("" if none). */
const char* pf_last_error(void);

/* Builds the level grids, Gauss/shape tables, transfer stencils and per-level
 * work buffers (Sec. 4.1 steps 2-4 and 6).  *out receives an owned handle.
 * The device memory all of it needs is compared with the device's free
 * memory before the first allocation: a hierarchy that does not fit (with
 * 1 GB kept in reserve) is refused with PF_ENOMEM and nothing allocated.
 * Not counted there: a level's assembled FP64 Hessian stencil (27 x 16
 * doubles per node in 3D), allocated on the level's first FP64 lag (an
 * FP64-precision load step, a GALERKIN coarse level, or
 * pf_hessvec_lag_set with PF_FP64); if it does not fit, that call returns
 * PF_ENOMEM.
 * Errors: PF_EINVAL for a bad descriptor, PF_ENOMEM, PF_ECUDA. */
pf_status pf_mesh_hierarchy_create(const pf_mesh_desc* desc, pf_hierarchy** out);
pf_status pf_mesh_hierarchy_destroy(pf_hierarchy* h);

/* Nodes per axis, spacing and node count of one level. */
pf_status pf_level_info(const pf_hierarchy* h, int level, int n_out[3],
                        double* h_out, long long* nodes_out);

/* Fracture initialisation (Sec. 5): the c plane of the finest-level FP64
 * state x_dev is set to 1 at nodes within band_half_width of a fracture's
 * mid-line (PF_LINE2D), mid-disc (PF_DISC3D) or mid-rectangle (PF_BOX3D)
 * and inside its extent, else 0 (union over rows).  u planes are not
 * touched.  c_prev := c.
 * rows_host: n rows of 4 (LINE2D), 7 (DISC3D) or 14 (BOX3D) doubles.  Node
 * coordinates are i*h in FP64; comparisons are inclusive.
 * Errors: PF_EINVAL (kind/dim mismatch, n < 0, band <= 0), PF_ENONFINITE
 * (a non-finite value in a row; nothing is changed). */
pf_status pf_fractures_set(pf_hierarchy* h, int kind, int n, const double* rows_host,
                           double band_half_width, void* x_dev);

/* Uniform pressure p of eq. (pressurized) for all following calls.  Also
 * writes an FP32 copy of p to the device on the hierarchy's stream (the 3D
 * FP32 Hessian products read it there) and synchronises that stream.
 * Errors: PF_EINVAL (null handle), PF_ENONFINITE (p not finite), PF_ECUDA. */
pf_status pf_pressure_set(pf_hierarchy* h, double p);

/* Discrete energy of eq. (pressurized) (AT2, sign reading +p g(c) div u,
 * clamped boundary terms vanish) on `level`, unconstrained, at x_dev
 * (precision prec).  FP64 result written to *E_host (stream synchronised).
 * Deterministic: fixed-order reduction. */
pf_status pf_energy(pf_hierarchy* h, int level, const void* x_dev, int prec, double* E_host);

/* E(x + s) - E(x) = a1 + a2 + a3 + a4, the exact quartic expansion along s
 * (coefficients written to a_host[4]); used for the trust-region ratios
 * eq. (rho_tr) and eq. (rho_ml) without cancellation. */
pf_status pf_energy_diff(pf_hierarchy* h, int level, const void* x_dev, const void* s_dev,
                         int prec, double* a_host);

/* Mixed-precision form of pf_energy_diff used by the FP32 levels of the
 * solver: a_host[0] = g . s over all dofs in FP64 (the first-order
 * coefficient a1 when g_dev is grad E(x)), a_host[1..3] = a2, a3, a4 in FP32
 * arithmetic from the FP64 x_dev and s_dev (each a sum of terms of order two
 * and higher in s, so their error is relative to their own size).  All
 * vectors FP64 device arrays of (dim+1)*N values. */
pf_status pf_energy_diff_mixed(pf_hierarchy* h, int level, const double* x_dev,
                               const double* s_dev, const double* g_dev, double* a_host);

/* Gradient of the energy at x_dev written to g_dev (same precision, same
 * layout), all dofs, no boundary masking. */
pf_status pf_gradient(pf_hierarchy* h, int level, const void* x_dev, void* g_dev, int prec);

/* Gradient (to g_dev) and energy (to *E_host, stream synchronised) of the
 * FP64 state x_dev in double-float arithmetic: every value an unevaluated
 * sum of two FP32 numbers (about 48 significant bits, FP32's exponent
 * range), run on the FP32 pipes, which GB300 issues at 64x its FP64 rate.
 * The mixed-precision solver takes its stopping-test gradients and the
 * returned energy this way (Sec. 2 energy and its gradient).  FP64 device
 * vectors of (dim+1)*N values.  PF_EINVAL on grids whose coefficient
 * buffer cannot hold the double-float scratch (only grids with very few
 * elements per axis). */
pf_status pf_gradient_df(pf_hierarchy* h, int level, const double* x_dev, double* g_dev);
pf_status pf_energy_df(pf_hierarchy* h, int level, const double* x_dev, double* E_host);

/* Gradient step: g_dev += grad E(x_dev) - grad E(x_dev - s_dev), so that
 * g_dev = grad E(x - s) on entry leaves grad E(x).  FP64 vectors; the
 * difference is evaluated in FP32 arithmetic as a sum of terms of order one
 * and higher in s (no two gradients are subtracted), so its error is
 * relative to the size of the change.  The mixed-precision solver updates
 * its model gradient this way after an accepted step (Algorithm 2); every
 * stopping test still evaluates the FP64 gradient. */
pf_status pf_gradient_step(pf_hierarchy* h, int level, const double* x_dev, const double* s_dev,
                           double* g_dev);

/* Hessian of the energy at x_lin_dev applied to v_dev, written to Hv_dev;
 * matrix-free (Sec. 4.2.1 Hessian; applied, not assembled).  All three
 * vectors in precision prec, computed in that precision.  3D FP32 products
 * on grids of at least 304 element tiles of 8^3 evaluate each element once
 * and sum a node's tiles in a fixed order; every product is deterministic. */
pf_status pf_hessvec(pf_hierarchy* h, int level, const void* x_lin_dev, const void* v_dev,
                     void* Hv_dev, int prec);

/* Hessian lagging (Sec. 4.2.1): pf_hessvec_lag_set fixes the lagged point
 * x_lag of `level` (precision prec; FP64 precomputes the Gauss-point
 * coefficients A = w g/h^2, B = w g'(sigma(u)+pI)/h, M = w(g''(psi+p tr)
 * + Gc/l_s) and assembles the Hessian into a 3^d-point block stencil held
 * by the hierarchy; FP32 keeps x_lag only); pf_hessvec_lagged then applies
 * H(x_lag) to v (same precision) as many times as needed.  The pressure at
 * lag_set time is used.  These share the level's lag buffers with
 * pf_rmtr_load_step, which resets them. */
pf_status pf_hessvec_lag_set(pf_hierarchy* h, int level, const void* x_lag_dev, int prec);
pf_status pf_hessvec_lagged(pf_hierarchy* h, int level, const void* v_dev, void* Hv_dev, int prec);

/* Stored Galerkin coarse operators (eq. (second_order_consistency) with
 * eq. (delta_terms) under Hessian lagging, Sec. 4.2.1): the model Hessian of
 * coarse level l is G^l = R G^{l+1} I, G^{L-1} = H(x_lag) of the finest
 * level.  pf_galerkin_set builds every coarse level's G^l from the finest
 * lag point x_lag_fine_dev (FP32, (dim+1) N_finest values) as an FP32
 * 3^d-point block stencil: element matrices of the next-to-finest level by
 * integrating the coarse Q1 basis against the fine Gauss-point Hessian
 * density of x_lag, then I^T K I element by element for coarser levels,
 * then a fixed-order assembly (deterministic).  The mixed-precision solver
 * builds them itself once per V-cycle when coarse_model = PF_GALERKIN.
 * pf_galerkin_apply applies level's G^l (level < n_levels-1) to v_dev
 * (precision prec; FP32 sums for FP32 vectors, FP64 sums of the FP32
 * entries for FP64).  Memory: per coarse level 4 (2^d (d+1))^2 bytes per
 * element and 4 (3^d (d+1)^2) bytes per node, allocated on first use.
 * Errors: PF_EINVAL, PF_ESTATE (apply before set), PF_ENOMEM, PF_ECUDA. */
pf_status pf_galerkin_set(pf_hierarchy* h, const float* x_lag_fine_dev);
pf_status pf_galerkin_apply(pf_hierarchy* h, int level, const void* v_dev, void* Hv_dev, int prec);

/* The paper's QP solvers for eq. (model_qp), min g.s + s.H s / 2 over
 * lo <= s <= hi (Sec. 4.2.2), on `level` with H the level's lagged FP64
 * Hessian as assembled by pf_hessvec_lag_set(..., PF_FP64) (else
 * PF_ESTATE).  All vectors FP64 device arrays of the level's size.
 * pf_qp_pgs: `sweeps` symmetric multicolour projected Gauss-Seidel sweeps
 * on s_inout (colours = node parity classes 0 .. 2^d-1, fields of a node
 * in order, then colours and fields reversed; s_i <- clamp(s_i -
 * (g + H s)_i / H_ii, lo_i, hi_i) where H_ii > 0).  Deterministic: nodes of
 * one colour do not couple.
 * pf_qp_mprgp: MPRGP (modified proportioning with reduced gradient
 * projections) from s = 0 on the diagonally scaled problem, the expansion
 * step length 1 / (Gershgorin bound of the scaled H); stops when the
 * projected gradient's norm <= tol or after maxit products; the result to
 * s_out, the products used to *products_host (may be NULL). */
pf_status pf_qp_pgs(pf_hierarchy* h, int level, const double* g_dev, const double* lo_dev,
                    const double* hi_dev, double* s_inout_dev, int sweeps);
pf_status pf_qp_mprgp(pf_hierarchy* h, int level, const double* g_dev, const double* lo_dev,
                      const double* hi_dev, double* s_out_dev, double tol, int maxit,
                      int* products_host);

/* Transfers between level `coarse` and coarse+1 (Sec. 3), per plane:
 * prolong: Q1 interpolation I (fine = I coarse);
 * restrict: R = I^T (coarse = R fine);
 * project: P = diag(R 1)^-1 R (coarse = P fine), for iterates. */
pf_status pf_prolong(pf_hierarchy* h, int coarse, const void* vc_dev, void* vf_dev, int prec);
pf_status pf_restrict(pf_hierarchy* h, int coarse, const void* vf_dev, void* vc_dev, int prec);
pf_status pf_project(pf_hierarchy* h, int coarse, const void* vf_dev, void* vc_dev, int prec);

/* Coarse feasible set (Sec. 3.2 F^l): lo_c = max of lo_f over the fine
 * support of each coarse basis function, hi_c = min of hi_f.  FP64. */
pf_status pf_coarse_bounds(pf_hierarchy* h, int coarse, const double* lo_f_dev,
                           const double* hi_f_dev, double* lo_c_dev, double* hi_c_dev);

/* One pseudo-time load step (Sec. 4.1 step 7): c_prev := c of x, then RMTR
 * V-cycles (Algorithm 1, mu1 = mu2 = 1, Hessian lagging of Sec. 4.2.1) until
 * the projected gradient meets rtol/atol or max_cycles.  x_dev: finest FP64
 * state, updated in place.  params NULL = defaults.  stats may be NULL.
 * Each level's CG loop runs as one CUDA graph (a conditional while node
 * around one CG iteration), built on first use, rebuilt when the pressure,
 * precision or coarse model change, and held by the hierarchy until
 * pf_mesh_hierarchy_destroy.  The call synchronises the hierarchy's stream
 * (it reads scalars back) and cannot itself be captured into a graph.
 * Errors: PF_ENOTCONV (x still updated), PF_ENONFINITE (a NaN/Inf in x on
 * entry, or a non-finite projected gradient during the step: x, c_prev and
 * the last converged pressure are left as they were on entry), PF_ECUDA. */
pf_status pf_rmtr_load_step(pf_hierarchy* h, void* x_dev, const pf_rmtr_params* params,
                            pf_rmtr_stats* stats);

/* Same as pf_rmtr_load_step with the state in host memory: copied to the
 * device, solved, copied back, all inside the call. */
pf_status pf_rmtr_load_step_host(pf_hierarchy* h, double* x_host, const pf_rmtr_params* params,
                                 pf_rmtr_stats* stats);

/* || x - P_F(x - grad E(x)) ||_2 on the finest level at the current
 * pressure, with the feasible set a load step starting from x would use
 * (c(x) <= c <= 1, clamped u): the reference for pf_rmtr_params.pg_ref.
 * Synchronises the stream. */
pf_status pf_projected_gradient(pf_hierarchy* h, const double* x_dev, double* pg_host);

/* Batched load steps: one load step of each of n independent instances
 * (hierarchies of any sizes, each with its own stream; hierarchies sharing a
 * stream serialise), run concurrently by n_threads host workers of the
 * library (<= 0: one per instance, at most 64), largest instances first.
 * xs[i] is the finest FP64 state of hs[i] (device).  params (NULL =
 * defaults) apply to every instance; stats[i] and status[i] (either may be
 * NULL) receive each instance's outcome.  Returns PF_OK if every instance
 * converged, else the first non-OK status in instance order. */
pf_status pf_rmtr_load_step_batch(int n, pf_hierarchy* const* hs, double* const* xs,
                                  const pf_rmtr_params* params, int n_threads,
                                  pf_rmtr_stats* stats, pf_status* status);

/* Copies the finest-level c_prev (FP64, N values) to c_prev_dev. */
pf_status pf_get_c_prev(pf_hierarchy* h, double* c_prev_dev);

/* Fields the solver keeps for a level, copied to out_dev (FP64, device):
 *   PF_FIELD_C_PREV  the irreversibility bound c_prev (finest level only;
 *                    N values), eq. (space_pf);
 *   PF_FIELD_LOWER,  the level's feasible set as the last load step left it
 *   PF_FIELD_UPPER   ((d+1) N values): on the finest level eq. (space_pf)
 *                    (c_prev <= c <= 1, u = 0 on the boundary, u free
 *                    elsewhere as -inf / +inf); on a coarser level the
 *                    coarse feasible set F^l of the last V-cycle around
 *                    its start x0 = P x (Alg. 1); PF_ESTATE before the
 *                    first load step and after pf_fractures_set or
 *                    pf_state_load;
 *   PF_FIELD_FIXED   1 for the dofs the clamped boundary fixes (every u
 *                    component on the boundary), 0 elsewhere ((d+1) N).
 * PF_EINVAL for another `which` or c_prev asked of a coarse level.
 * Asynchronous on the hierarchy's stream. */
#define PF_FIELD_C_PREV 0
#define PF_FIELD_LOWER 1
#define PF_FIELD_UPPER 2
#define PF_FIELD_FIXED 3
pf_status pf_get_fields(pf_hierarchy* h, int level, int which, double* out_dev);

/* Checkpoint and resume (Sec. 4.1 workflow: the state is exported after
 * every pseudo-time step).  pf_state_save writes the finest FP64 state x_dev
 * ((dim+1) N values), the hierarchy's c_prev, the current pressure and the
 * last converged pressure (the extrapolated start's base) to the file
 * `path`, with the grid and material in its header and an FNV-1a checksum
 * of the payload; it writes `path`.tmp and renames it, so a reader never
 * sees a partial file.  pf_state_load restores all of that into a hierarchy
 * of the same grid and material (x_dev receives the state; the pressure is
 * set as by pf_pressure_set), after which the next load step reproduces the
 * uninterrupted run bit for bit.  The per-level trust-region radius and the
 * lagged Hessians are not state: every load step starts them afresh.
 * Both synchronise the hierarchy's stream.  Errors: PF_EINVAL (null
 * argument; a file for another grid or material, of another version or byte
 * order, or with a wrong checksum), PF_EIO (file cannot be opened, read or
 * written, or its size disagrees with its header), PF_ENONFINITE (a
 * non-finite value in the state or file), PF_ECUDA.  pf_state_load changes
 * nothing unless every check passed. */
pf_status pf_state_save(pf_hierarchy* h, const double* x_dev, const char* path);
pf_status pf_state_load(pf_hierarchy* h, double* x_dev, const char* path);

/* Energy of pf_energy for callers that cannot allocate device memory.
 * The paper has no counterpart: this exists for callers such as plug-ins
 * that run inside a host application which owns the whole device memory
 * budget, or real-time loops where cudaMalloc/cudaFree are not allowed
 * because they can block and synchronise the device.  The call takes the
 * grid and material directly (no pf_hierarchy, whose creation allocates),
 * allocates nothing and frees nothing.
 *   dim, n[0..dim): nodes per axis; h: spacing; E, nu, Gc, ls, k_res, p: as
 *   in pf_mesh_desc / pf_pressure_set (ls is l_s itself); x_dev: (dim+1)
 *   planes of prod(n) values in precision prec; E_dev: one device double
 *   that receives the FP64 energy, written on `stream` (cudaStream_t, NULL =
 *   legacy stream); the call does not synchronise.
 * Scratch: a fixed 512 KiB + 256 B array in the library's device memory,
 * loaded on every device that uses the library and held until the process
 * exits.  It holds 65,536 block partials, so grids of more than 16,777,216
 * elements are rejected with PF_EINVAL (use pf_energy for those).
 * The first call on a device looks up that array's device address (with
 * the device current), so make the first call on each device before any
 * stream capture; the lookup is repeated only when the device's context has
 * changed (after cudaDeviceReset), so make the first call after such a
 * reset before any stream capture too.  Every call shares the one array and
 * clears its counter
 * on entry; calls whose kernels overlap on the GPU (two streams, two host
 * threads) race on it and must be serialised by the caller. */
pf_status pf_energy_noalloc(int dim, const int n[3], double h, double E, double nu, double Gc,
                            double ls, double k_res, double p, const void* x_dev, int prec,
                            double* E_dev, void* stream);

/* Tile autotuner (no counterpart in the paper): times the FP32 Hessian
 * product of every level of h on each of its tile variants (3D: 1
 * element-owned 8^3 element tiles, 2 owner-computes 8^3 node tiles, 3
 * owner-computes 4^3; 2D: 0 32x8, 1 16x8, 2 64x4, 3 32x4 node tiles, 4
 * strips of 63 node columns marched one element row at a time) with
 * CUDA events on h's stream (one warm-up and five timed launches each on the
 * level's own buffers), and keeps the fastest for the level's FP32
 * products from then on, in the solver and in pf_hessvec.  The variants
 * compute the same product with different summation orders (results agree
 * to FP32 rounding; each is deterministic).  variant_out (n_levels ints)
 * and us_out (5 n_levels doubles, microseconds per product of variants
 * 0 .. 4, -1 where a variant does not apply) may be NULL.  Rebuilds the hierarchy's CUDA
 * graphs on next use.  Call between load steps; synchronises the stream. */
pf_status pf_autotune(pf_hierarchy* h, int* variant_out, double* us_out);
/* The tile variant of one level (0 = the default rule: 3D element-owned
 * tiles on grids of at least 304 8^3 tiles, else owner-computes 8^3 or 4^3
 * node tiles; 2D marching strips on grids of at least 200,000 nodes, else
 * 32x8 node tiles), e.g. to reuse a
 * choice of pf_autotune in later runs so that they repeat bit for bit.
 * set also rebuilds the hierarchy's CUDA graphs on next use. */
pf_status pf_tile_variant_set(pf_hierarchy* h, int level, int variant);
pf_status pf_tile_variant_get(const pf_hierarchy* h, int level, int* variant);

/* ------------------------------------------------------------------------
 * Batched 2D operators (no counterpart in the paper, which solves one
 * network per run): the finest levels of n 2D hierarchies of any sizes
 * evaluated by ONE persistent launch over an (instance, strip, row) work
 * list -- strips of 63 node columns, every warp an equal share of all
 * instances' rows -- with per-instance (segmented) reductions.  The
 * operators are those of pf_hessvec and pf_energy (Sec. 2 functional,
 * Sec. 4.2.1 Hessian), on each instance's own grid, material and current
 * pressure (read from its hierarchy at every call).
 *
 * pf_batch_create keeps the hierarchies (they must outlive the batch) and
 * runs on `stream` (cudaStream_t, NULL = legacy stream).  2D only
 * (PF_EINVAL otherwise).  Device scratch: one double per node row of each
 * strip and per element row (about 8 B per 60 nodes). */
typedef struct pf_batch pf_batch;
pf_status pf_batch_create(int n, pf_hierarchy* const* hs, void* stream, pf_batch** out);
pf_status pf_batch_destroy(pf_batch* b);
/* Total dofs, blocks per SM of the product launch, SM count. */
pf_status pf_batch_info(const pf_batch* b, long long* dofs, int* blocks_per_sm, int* sms);
/* Hv_dev[i] = H(x_dev[i]) v_dev[i] for every instance, FP32 vectors of
 * 3 N_i values (planes u_x, u_y, c), computed in FP32 with paired-FP32
 * instructions.  Hv_dev[i] must not overlap x_dev[i] or v_dev[i].  With
 * vHv_dev (device, n doubles; may be NULL) also v_i . H v_i per instance
 * (FP32 node-row sums, FP64 across rows, fixed order).  Asynchronous on
 * the batch's stream; results are the same bit for bit for every launch
 * configuration.  The pointer tables are copied to the device when they
 * change (the call then synchronises the stream once). */
pf_status pf_batch_hessvec(pf_batch* b, const float* const* x_dev, const float* const* v_dev,
                           float* const* Hv_dev, double* vHv_dev);
/* E_host[i] = energy of FP64 x_dev[i] (3 N_i values), FP64 arithmetic,
 * element rows summed in a fixed order.  Synchronous; PF_ENONFINITE if
 * any energy is not finite. */
pf_status pf_batch_energy(pf_batch* b, const double* const* x_dev, double* E_host);
/* Autotuner of the product launch: times blocks per SM 1 .. 4 (those the
 * kernel's occupancy allows; us_out[k-1] = -1 otherwise) on the given
 * vectors with CUDA events (one warm-up, five timed) and keeps the
 * fastest.  bps_out, us_out (4 doubles) may be NULL. */
pf_status pf_batch_autotune(pf_batch* b, const float* const* x_dev, const float* const* v_dev,
                            float* const* Hv_dev, int* bps_out, double* us_out);
pf_status pf_batch_variant_set(pf_batch* b, int blocks_per_sm);

/* Measurement helper with no counterpart in the paper: runs a kernel of
 * independent fused multiply-adds in precision prec on the legacy stream
 * and writes the achieved rate (flop/s, an FMA counted as 2) to *flops_host.
 * Used as the ALU roofline denominator of the element kernels. */
pf_status pf_probe_fma(int prec, double* flops_host);

/* ------------------------------------------------------------------------
 * Learned initial iterate (no counterpart in the paper; the network, its
 * features and its acceptance test are this library's extension).  A 2D
 * U-Net proposes each load step's change of state; the proposal is
 * accepted only through the trust-region ratio (eq. rho_tr) of the FP64
 * energy, otherwise the plain iterate is kept.
 * ---------------------------------------------------------------------- */
typedef struct pf_unet pf_unet;

/* Network on an H x W grid (multiples of 8): 4 levels with channels[0..3],
 * two 3x3 convolutions + ReLU per level, 2x2 average pooling, nearest 2x
 * upsampling with skip concatenation [up, skip], 1x1 head; n_in input and
 * n_out output planes.  BF16 weights/activations, FP32 arithmetic, FP32
 * master weights.  Parameter vector layout: for every layer in the order
 * enc0a enc0b ... enc3a enc3b dec2a dec2b dec1a dec1b dec0a dec0b head,
 * its weights [c_out][c_in][k][k] then its biases [c_out]. */
pf_status pf_unet_create(int height, int width, int n_in, int n_out, const int channels[4],
                         void* stream, pf_unet** out);
pf_status pf_unet_destroy(pf_unet* u);
pf_status pf_unet_num_params(const pf_unet* u, long long* n);
/* host FP32 parameter vectors; set also clears the Adam moments and the
 * accumulated gradient */
pf_status pf_unet_set_params(pf_unet* u, const float* params_host);
pf_status pf_unet_get_params(pf_unet* u, float* params_host);
pf_status pf_unet_get_grads(pf_unet* u, float* grads_host);
/* y = net(x): x_dev n_in x H x W FP32 planes, y_dev n_out x H x W FP32;
 * keeps the activations for pf_unet_backward. */
pf_status pf_unet_forward(pf_unet* u, const float* x_dev, float* y_dev);
/* adds dL/dparams for dL/dy (FP32, n_out x H x W) at the last forward */
pf_status pf_unet_backward(pf_unet* u, const float* dy_dev);
/* masked mean-squared error L = sum mask (y - t)^2 / (2 n_out n_valid);
 * writes dL/dy to dy_dev and L to *loss_host (mask_dev: H x W, NULL = all
 * pixels, n_valid its number of ones). */
pf_status pf_unet_mse(pf_unet* u, const float* y_dev, const float* t_dev, const float* mask_dev,
                      double n_valid, float* dy_dev, double* loss_host);
/* one Adam step (Kingma & Ba) with the accumulated gradient times
 * grad_scale, then clears the gradient */
pf_status pf_unet_adam(pf_unet* u, float lr, float beta1, float beta2, float eps, float grad_scale);

/* Network input planes (H x W, zero outside the finest 2D grid) from the
 * previous converged state x_prev (pressure p_prev > 0), the phase field
 * c_before of the step before it (NULL = c of x_prev) and the new pressure:
 * [u_x E/p_prev, u_y E/p_prev, c, p_new/p_prev, c - c_before]. */
pf_status pf_learned_features(pf_hierarchy* h, const double* x_prev_dev, const double* c_before_dev,
                              double p_prev, double p_new, int H, int W, float* feat_dev);
/* Training target planes from two converged states: the change beyond the
 * linear extrapolation r = p_new/p_prev of the displacement,
 * [(u_new - r u_prev) E/dp (2 planes), (c_new - c_prev)/dp],
 * dp = p_new - p_prev (p_prev > 0). */
pf_status pf_learned_target(pf_hierarchy* h, const double* x_prev_dev, const double* x_new_dev,
                            double p_prev, double p_new, int H, int W, float* target_dev);
/* Proposal from the network output y (the target's scaling inverted):
 * xhat = [r u_prev + dp/E y_u, c_prev + dp y_c]; y = 0 gives the linear
 * extrapolation of the displacement. */
pf_status pf_learned_apply(pf_hierarchy* h, const double* x_prev_dev, const float* y_dev,
                           double p_prev, double p_new, int H, int W, double* xhat_dev);
/* Acceptance test at the current pressure: c_prev := c of x (kept for the
 * next load step, which must run with keep_c_prev = 1); xhat is projected
 * onto the feasible set; s = xhat - x; rho = (E(x) - E(x + s)) /
 * (-(grad E(x).s + s.H(x)s/2)) with FP64 energy difference, gradient and
 * Hessian; x := x + s when rho > eta and E decreases.  Writes rho and
 * accepted (0/1). */
pf_status pf_learned_propose(pf_hierarchy* h, double* x_dev, const double* xhat_dev, double eta,
                             double* rho_host, int* accepted_host);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
