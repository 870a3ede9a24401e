// Internal interfaces between the kernel, solver and C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include "pf_element.cuh"

namespace pf {

// One level's structured grid: n[k] nodes per axis, spacing h.
struct Geom {
  int dim;
  int n[3];
  long long N;   // nodes
  int ne[3];     // elements per axis
  long long NE;  // elements
  double h;
  // tile variant of the FP32 Hessian products on this grid (0: the default
  // rule; set per level by the autotuner, pf_autotune): 3D 1 element-owned
  // 8^3 tiles, 2 owner-computes 8^3, 3 owner-computes 4^3; 2D 1 16x8,
  // 2 64x4, 3 32x4 node tiles, 4 marching strips (0: strips on grids of
  // at least 200,000 nodes, else 32x8)
  int hv_variant;
};

// Fixed-size deterministic reduction scratch: one partial per block (up to
// kMaxBlocks per slot, kMaxSlots slots) and a completion counter.  The last
// block to finish sums the partials in block order.
constexpr int kMaxBlocks = 1216;  // 8 x 152 SMs
constexpr int kMaxSlots = 8;
struct Scratch {
  double* partials;   // kMaxSlots * kMaxBlocks
  unsigned* counter;  // 1, zero between reductions
};

// Device-resident control block of one projected CG run: the scalars each
// iteration needs and the reason it stopped, updated by the last block of
// each reduction so the host only polls it.
struct CgCtrl {
  double rr;      // r.r of the current residual
  double rz;      // r.M^-1 r (preconditioned CG)
  double tol;     // forcing tolerance on ||r||
  double alpha;   // step of the current iteration
  double beta;    // direction update of the current iteration
  double kappa;   // p.Hp of the current iteration
  int done;       // 1 once the run has stopped; later launches are no-ops
  int state;      // why it stopped (CG_*)
  int used;       // Hessian-vector products spent by the CG loop
  int cg_max;     // budget
};
enum { CG_RUNNING = 0, CG_NEGCURV = 1, CG_LEAVE = 2, CG_CONV = 3, CG_BUDGET = 4 };

// The CG direction of one dof, M^-1 r + beta p (mi = 1 without a
// preconditioner), rounded the same way wherever it is formed.
__device__ __forceinline__ float cg_direction(float mi, float r, float beta, float p) {
  return __fmaf_rn(beta, p, __fmul_rn(mi, r));
}

// Inputs of the direction update fused into the FP32 CG product: the
// product's operand becomes p = M^-1 r + beta p (beta from the control
// block), formed where the operand is read and stored back by the gather
// pass.  mi null: no preconditioner.
struct CgDirIn {
  const float* r;
  const float* mi;
};

// The curvature step of a CG iteration from kappa = p.Hp: counts the
// product, then alpha = r.M^-1 r / kappa, or a stop on non-positive
// curvature.  Run by the last block of the p.Hp reduction.
__device__ __forceinline__ void cg_take_curvature(CgCtrl* c, double kappa) {
  c->kappa = kappa;
  c->used += 1;
  if (kappa <= 0.0) {
    c->done = 1;
    c->state = CG_NEGCURV;
  } else {
    c->alpha = c->rz / kappa;
  }
}

Geom make_geom(int dim, const int n[3], double h);
Mat<double> make_mat(const Geom& g, double E, double nu, double Gc, double ls, double k,
                     double p);

// Element kernels.  x, v, y hold (dim+1) planes of g.N values in precision
// prec (0 = double, 1 = float).  Reductions write FP64 results to out_dev.
cudaError_t elem_energy(const Geom& g, const Mat<double>& m, const void* x, int prec,
                        const Scratch& s, double* out_dev, cudaStream_t st);
// The energy kernel launched with nblocks blocks of 256 threads, block
// partials at partials[0 .. nblocks) (needs nblocks <= partials' length).
cudaError_t elem_energy_blocks(const Geom& g, const Mat<double>& m, const void* x, int prec,
                               double* partials, unsigned* counter, int nblocks, double* out,
                               cudaStream_t st);
cudaError_t elem_energy_diff(const Geom& g, const Mat<double>& m, const void* x, const void* sv,
                             int prec, const Scratch& s, double* out_dev, cudaStream_t st);
// (gx . s, a2, a3, a4) to out_dev[0..4): the higher-order coefficients of
// E(x + t s) - E(x) in FP32 arithmetic from FP64 x and s, and the FP64 dot
// product of gx (skipped when null) with s.
cudaError_t elem_energy_diff_hi(const Geom& g, const Mat<double>& m, const double* x,
                                const double* sv, const double* gx, const Scratch& s,
                                double* out_dev, cudaStream_t st);
cudaError_t elem_gradient(const Geom& g, const Mat<double>& m, const void* x, void* y, int prec,
                          cudaStream_t st);
// FP64 gradient evaluating every element once: corner contributions go to
// scratch (NE * 2^d * (d+1) doubles, e.g. a level's coefficient buffer),
// then each node sums its elements' in a fixed order.
cudaError_t elem_gradient_fp64(const Geom& g, const Mat<double>& m, const double* x, double* y,
                               double* scratch, cudaStream_t st);
// y += grad E(x) - grad E(x - s) with the difference in FP32 arithmetic from
// FP64 x and s (every term of order one or higher in s): the gradient at x
// from the one at x - s.
cudaError_t elem_gradient_step(const Geom& g, const Mat<double>& m, const double* x,
                               const double* s, double* y, cudaStream_t st);
// The gradient (to y, FP64) and the energy (to out_dev[0]) of FP64 x in
// double-float arithmetic on the FP32 pipes (about 48 significant bits).
// scratch: a level's coefficient buffer (coef_count(g) doubles), which
// holds x in double-float and the gradient's corner contributions;
// cudaErrorInvalidValue where it is too small (df_scratch_fits false: only
// grids with very few elements per axis).
bool df_scratch_fits(const Geom& g);
cudaError_t elem_gradient_df(const Geom& g, const Mat<double>& m, const double* x, double* y,
                             double* scratch, cudaStream_t st);
cudaError_t elem_energy_df(const Geom& g, const Mat<double>& m, const double* x, double* scratch,
                           const Scratch& s, double* out_dev, cudaStream_t st);
// part: optional scratch of etile_part_count(g) float4; with it, 3D FP32
// products on grids of at least two 8^3 tiles per SM evaluate every element
// once (element-owned tiles, then a gather of the tiles' node sums).
// p_dev: optional device copy of the pressure (FP32), read by the 3D FP32
// products instead of m.p, so that CUDA graphs capturing them stay valid
// across pressure changes.
cudaError_t elem_hessvec(const Geom& g, const Mat<double>& m, const void* x, const void* v,
                         void* y, int prec, cudaStream_t st, const int* skip = nullptr,
                         void* part = nullptr, const float* p_dev = nullptr);
long long etile_part_count(const Geom& g);
// kernel launches of one 3D FP32 product (1, or 2 on the element-owned path)
int hessvec32_launches(const Geom& g, const void* part);
// The FP32 CG product q = H p with p.q taken in the same launches: on the
// element-owned path the gather pass reduces p.q and its last block runs
// cg_take_curvature on c.  Returns cudaErrorNotSupported, launching
// nothing, where that path does not apply (the caller then takes p.q in a
// pass of its own).  partials needs kMaxBlocks doubles.
// With dir.r set, p is first replaced by M^-1 r + beta p (beta =
// c->beta), the direction update of the previous iteration; the product and
// p.q use the new p.
cudaError_t elem_hessvec32_dot(const Geom& g, const Mat<double>& m, const float* x, float* p,
                               float* q, CgCtrl* c, double* partials, unsigned* counter,
                               void* part, const float* p_dev, CgDirIn dir, cudaStream_t st);
bool hessvec32_dot_fused(const Geom& g, const void* part);
// FP64 lagged Hessian: Gauss-point coefficients of x (coef holds
// NE * 2^d * (2 + d(d+1)/2) doubles), the input of the stencil assembly.
cudaError_t elem_hess_coef(const Geom& g, const Mat<double>& m, const double* x, double* coef,
                           cudaStream_t st);
inline long long coef_count(const Geom& g) {
  const int d = g.dim;
  return g.NE * (1LL << d) * (2 + d * (d + 1) / 2);
}
// The lagged FP64 Hessian assembled into a 3^d-point block stencil (S holds
// stencil_count(g) doubles) from the stored coefficients, and its product.
inline long long stencil_count(const Geom& g) {
  const int f = g.dim + 1;
  return (g.dim == 3 ? 27LL : 9LL) * f * f * g.N;
}
cudaError_t stencil_assemble(const Geom& g, const Mat<double>& m, const double* coef, double* S,
                             cudaStream_t st);
cudaError_t stencil_apply(const Geom& g, const double* S, const double* v, double* y,
                          cudaStream_t st, const int* skip = nullptr);
// One half of a symmetric multicolour projected Gauss-Seidel sweep with the
// FP64 stencil S (colours in order, or reversed with fields reversed), and
// the row sums of the diagonally scaled |S| (a Gershgorin bound).
cudaError_t pgs_sweep(const Geom& g, const double* S, const double* gv, const double* lo,
                      const double* hi, double* s, bool reverse, cudaStream_t st);
cudaError_t scaled_rowsum(const Geom& g, const double* S, double* out, cudaStream_t st);
// Diagonal of the Hessian at x (precision prec), written as FP64.
cudaError_t elem_hessdiag(const Geom& g, const Mat<double>& m, const void* x, int prec,
                          double* y, cudaStream_t st);
// FP32 Hessian at an FP32 copy of x applied to an FP64 v, written as FP64
// (the mixed-precision solver's operator; conversions happen in registers).
cudaError_t elem_hessvec_mixed(const Geom& g, const Mat<double>& m, const float* x32,
                               const double* v, double* y, cudaStream_t st,
                               const int* skip = nullptr, void* part = nullptr,
                               const float* p_dev = nullptr);

// Stored Galerkin coarse operators (pf_galerkin.cu): FP32 element
// matrices of the next-to-finest level gc from the finest FP32 lag, their
// element-wise coarsening, the 3^d-point FP32 stencil of a level, and its
// product with FP32 (prec PF_FP32) or FP64 vectors.
long long galerkin_elem_count(const Geom& g);
long long galerkin_stencil_count(const Geom& g);
cudaError_t galerkin_fine(const Geom& gc, const Geom& gf, const Mat<double>& mf, const float* x_fine,
                          float* K, cudaStream_t st);
cudaError_t galerkin_rap(const Geom& gc, const Geom& gf, const float* Kf, float* Kc, cudaStream_t st);
cudaError_t galerkin_assemble(const Geom& g, const float* K, float* S, cudaStream_t st);
cudaError_t galerkin_apply(const Geom& g, const float* S, const void* v, void* y, int prec,
                           cudaStream_t st, const int* skip = nullptr);

// The 2D FP32 Hessian product on 63-column strips marched one element row
// at a time (pf_batch.cu), one instance: y = H(x) v, FP32 planes.  The
// node sums are in a fixed order, so the result does not depend on the
// launch shape.  skip as for the other element kernels.
cudaError_t hess2_march(const Geom& g, const Mat<double>& m, const float* x, const float* v,
                        float* y, const int* skip, cudaStream_t st);

// Fracture band rasterisation into the c plane (FP64) of x and c_prev.
// rows: device array of precomputed shape rows of kRasterRow doubles (see
// pf_fractures_set); kind 0 line (2D), 1 disc, 2 rectangle (3D).
constexpr int kRasterRow = 14;
cudaError_t rasterize(const Geom& g, int kind, int n, const double* rows_dev, double band,
                      double* c_plane, double* c_prev, cudaStream_t st);

// Transfers between a coarse grid gc and its 2:1 refinement gf, nf planes.
cudaError_t xfer_prolong(const Geom& gc, const Geom& gf, int nf, const void* in, void* out,
                         int prec, cudaStream_t st, const int* skip = nullptr);
cudaError_t xfer_restrict(const Geom& gc, const Geom& gf, int nf, const void* in, void* out,
                          int prec, bool normalise, cudaStream_t st, const int* skip = nullptr);
cudaError_t xfer_bounds(const Geom& gc, const Geom& gf, int nf, const double* lo_f,
                        const double* hi_f, double* lo_c, double* hi_c, cudaStream_t st);

}  // namespace pf
