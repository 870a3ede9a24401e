// The opaque pf_hierarchy: level grids, material, reduction scratch and the
// per-level solver buffers (all device-resident, allocated once at create).
#pragma once
#include <string>
#include <vector>

#include "../../include/pf.h"
#include "pf_internal.h"

namespace pf {

// Device buffers of one level.  Vectors hold (dim+1)*N doubles.
struct LevelBuf {
  long long n = 0;  // dofs
  double *x = nullptr, *lb = nullptr, *ub = nullptr;  // iterate and feasible set
  double *x0 = nullptr, *xlag = nullptr, *dg = nullptr;  // level model
  double* g0 = nullptr;  // gradient of the level model at x0 (R of the finer gradient)
  double *g = nullptr, *s = nullptr, *lo = nullptr, *hi = nullptr;  // TR step
  double *Hs = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;    // CG
  double *w = nullptr, *Hw = nullptr, *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;
  double *gin = nullptr, *gout = nullptr;  // Galerkin recursion through this level
  double *dh = nullptr;                    // dH scratch
  double *minv = nullptr;                  // Jacobi preconditioner of the lagged Hessian
  float* xlag32 = nullptr;  // FP32 copy of x_lag (mixed precision)
  double* coef = nullptr;   // lagged Gauss-point coefficients (FP64 Hessian)
  double* stencil = nullptr;  // assembled lagged FP64 Hessian (3^d block stencil)
  float* gk = nullptr;        // FP32 Galerkin element matrices (mixed GALERKIN coarse levels)
  float* gs = nullptr;        // FP32 Galerkin operator as a 3^d block stencil
};


void set_error(const std::string& msg);

}  // namespace pf

struct pf_hierarchy {
  int dim = 0, L = 0;
  std::vector<pf::Geom> geo;
  std::vector<pf::Mat<double>> mat;  // per level (ls = ls_over_h * h_finest)
  double E = 1, nu = 0.3, Gc = 1, ls = 0, k_res = 0, p = 0;
  double p_last = 0;  // pressure of the last converged load step (0 = none)
  cudaStream_t st = nullptr;
  pf::Scratch scratch{nullptr, nullptr};
  double* d_res = nullptr;  // device result slots
  double* h_res = nullptr;  // pinned host mirror
  double* c_prev = nullptr; // finest N values
  double* c_prev_save = nullptr;  // c_prev at the start of a load step (restored on failure)
  pf::CgCtrl* ctrl = nullptr;    // device CG control block
  pf::CgCtrl* h_ctrl = nullptr;  // pinned host mirror
  void* etile_part = nullptr;  // node sums of the element-owned FP32 Hessian tiles (3D)
  float* p_dev = nullptr;      // the pressure in FP32 on the device (kept by pf_pressure_set)
  // executable graphs of the FP32 CG loop per level (built by the solver)
  struct CgGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // what the captured launches depend on besides the level's fixed buffers
    double p = 0.0;               // pressure (argument of the FP32 Hessian)
    int pc = -1;                  // preconditioning flag
    int vsize = 0;                // 4: FP32 vectors, 8: FP64 vectors
    int precision = -1;           // PF_FP64 / PF_FP32 (selects the Hessian kernel)
    int coarse_model = -1;        // selects the level's model Hessian
    const void* vp = nullptr;     // direction vector
    int nodes = 0;                // kernel launches per iteration of the body
  };
  std::vector<CgGraph> cg_graphs;
  bool cg_graph_ok = true;  // false once the CUDA driver refused to build one
  bool have_fractures = false;
  bool bounds_set = false;  // lv[].lb / ub hold a load step's feasible sets
  std::vector<pf::LevelBuf> lv;
  std::vector<void*> allocations;
};

namespace pf {
pf_status rmtr_load_step_impl(pf_hierarchy* H, double* x_dev, const pf_rmtr_params& P,
                              pf_rmtr_stats* stats);
pf_status projected_gradient_impl(pf_hierarchy* H, const double* x_dev, double* out);
// sweeps > 0: PGS sweeps on s; else MPRGP into s (tol, maxit, *products)
pf_status qp_impl(pf_hierarchy* H, int level, const double* g, const double* lo, const double* hi,
                  double* s, int sweeps, double tol, int maxit, int* products);
void refresh_pressure(pf_hierarchy* H);
// Allocates level l's FP64 stencil on first use (held until destroy).
cudaError_t ensure_stencil(pf_hierarchy* H, int l);
// Allocates level l's Galerkin element matrices and FP32 stencil on first
// use, and builds the FP32 Galerkin operators of every coarse level from
// the finest level's FP32 lag x (R G I chain, see pf_galerkin.cu).
cudaError_t ensure_galerkin(pf_hierarchy* H, int l);
cudaError_t galerkin_build(pf_hierarchy* H, const float* x_fine, cudaStream_t st);
// out[i] = 1 for the dofs the clamped boundary fixes (u on the boundary), 0
// elsewhere; (dim + 1) g.N values.
cudaError_t fixed_mask(const Geom& g, double* out, cudaStream_t st);
}  // namespace pf
