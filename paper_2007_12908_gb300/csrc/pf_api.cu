// C-ABI of libpf: argument checks, hierarchy set-up and dispatch to kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "pf_hier.h"

namespace pf {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace pf

using namespace pf;

#define PF_TRY_CUDA(call, what)                                                       \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_error(std::string(what) + ": " + cudaGetErrorString(e_));                   \
      return e_ == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA;                  \
    }                                                                                 \
  } while (0)

static bool valid_level(const pf_hierarchy* h, int level) {
  return h && level >= 0 && level < h->L;
}

static pf_status bad(const char* msg) {
  set_error(msg);
  return PF_EINVAL;
}

namespace pf {
cudaError_t ensure_stencil(pf_hierarchy* h, int l) {
  LevelBuf& B = h->lv[l];
  if (B.stencil) return cudaSuccess;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(double) * stencil_count(h->geo[l]));
  if (e != cudaSuccess) return e;
  h->allocations.push_back(p);
  B.stencil = static_cast<double*>(p);
  return cudaSuccess;
}
cudaError_t ensure_galerkin(pf_hierarchy* h, int l) {
  LevelBuf& B = h->lv[l];
  if (B.gs) return cudaSuccess;
  void *k = nullptr, *sg = nullptr;
  cudaError_t e = cudaMalloc(&k, sizeof(float) * galerkin_elem_count(h->geo[l]));
  if (e != cudaSuccess) return e;
  h->allocations.push_back(k);
  e = cudaMalloc(&sg, sizeof(float) * galerkin_stencil_count(h->geo[l]));
  if (e != cudaSuccess) return e;
  h->allocations.push_back(sg);
  B.gk = static_cast<float*>(k);
  B.gs = static_cast<float*>(sg);
  return cudaSuccess;
}

cudaError_t galerkin_build(pf_hierarchy* h, const float* x_fine, cudaStream_t st) {
  const int L = h->L;
  for (int l = 0; l < L - 1; ++l) {
    cudaError_t e = ensure_galerkin(h, l);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = galerkin_fine(h->geo[L - 2], h->geo[L - 1], h->mat[L - 1], x_fine, h->lv[L - 2].gk, st);
  for (int l = L - 3; l >= 0 && e == cudaSuccess; --l)
    e = galerkin_rap(h->geo[l], h->geo[l + 1], h->lv[l + 1].gk, h->lv[l].gk, st);
  for (int l = 0; l <= L - 2 && e == cudaSuccess; ++l)
    e = galerkin_assemble(h->geo[l], h->lv[l].gk, h->lv[l].gs, st);
  return e;
}
}  // namespace pf

template <class T>
__global__ void k_fma_probe(T* out, int reps, T a, T b) {
  T v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = T(threadIdx.x + k) * T(1e-3);
  for (int r = 0; r < reps; ++r) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = v[k] * a + b;
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += v[k];
  if (s == T(-12345.678)) out[0] = s;  // keeps the chains live
}

extern "C" {

void pf_rmtr_params_default(pf_rmtr_params* p) {
  if (!p) return;
  p->eta1 = 0.1;
  p->eta2 = 0.75;
  p->gamma1 = 0.5;
  p->gamma2 = 2.0;
  p->delta0 = 1.0;
  p->delta_max = 1.0;
  p->mu1 = 1;
  p->mu2 = 1;
  p->coarse_its = 10;
  p->cg_fine = 50;
  p->cg_smooth = 10;
  p->cg_coarse = 500;
  p->cauchy_backtracks = 30;
  p->cauchy_c = 0.01;
  p->max_cycles = 200;
  p->rtol = 1e-10;
  p->atol = 0.0;
  p->coarse_model = PF_FIRST_ORDER;
  p->precision = PF_FP64;
  p->precondition = 1;
  p->level_rtol = 1e-3;
  p->max_restarts = 1000000;
  p->keep_c_prev = 0;
  p->pg_ref = 0.0;
  p->start = PF_START_PLAIN;
  p->p_prev = 0.0;
  p->qp_solver = PF_QP_CG;
  p->pgs_sweeps = 2;
}

const char* pf_last_error(void) { return g_last_error.c_str(); }

static pf_status alloc(pf_hierarchy* h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return PF_ENOMEM;
  }
  h->allocations.push_back(*p);
  return PF_OK;
}

pf_status pf_mesh_hierarchy_destroy(pf_hierarchy* h) {
  if (!h) return PF_OK;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  for (auto& G : h->cg_graphs) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
  }
  for (void* p : h->allocations) cudaFree(p);
  if (h->h_res) cudaFreeHost(h->h_res);
  if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
  delete h;
  return PF_OK;
}

pf_status pf_mesh_hierarchy_create(const pf_mesh_desc* d, pf_hierarchy** out) {
  if (!d || !out) return bad("mesh_hierarchy_create: null argument");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return bad("mesh_hierarchy_create: dim must be 2 or 3");
  if (d->n_levels < 1 || d->n_levels > 8) return bad("mesh_hierarchy_create: n_levels must be 1 .. 8");
  for (int k = 0; k < d->dim; ++k)
    if (d->n_coarse[k] < 2) return bad("mesh_hierarchy_create: n_coarse must be >= 2");
  if (!(d->h_coarse > 0) || !(d->E > 0) || !(d->Gc > 0) || !(d->ls_over_h > 0) ||
      !(d->nu > -1.0 && d->nu < 0.5) || !(d->k_res >= 0 && d->k_res < 1))
    return bad("mesh_hierarchy_create: invalid material or spacing");
  pf_hierarchy* h = new pf_hierarchy();
  h->dim = d->dim;
  h->L = d->n_levels;
  h->E = d->E;
  h->nu = d->nu;
  h->Gc = d->Gc;
  h->k_res = d->k_res;
  h->st = static_cast<cudaStream_t>(d->stream);
  for (int l = 0; l < h->L; ++l) {
    int n[3] = {1, 1, 1};
    for (int k = 0; k < d->dim; ++k) {
      const long long v = (long long)(d->n_coarse[k] - 1) * (1LL << l) + 1;
      if (v > (1LL << 20)) {
        delete h;
        return bad("mesh_hierarchy_create: grid too large");
      }
      n[k] = int(v);
    }
    h->geo.push_back(make_geom(d->dim, n, d->h_coarse / double(1LL << l)));
  }
  h->ls = d->ls_over_h * h->geo.back().h;
  for (int l = 0; l < h->L; ++l)
    h->mat.push_back(make_mat(h->geo[l], h->E, h->nu, h->Gc, h->ls, h->k_res, 0.0));
  pf_status rc;
  const int F = d->dim + 1;
  long long part = 0;
  for (const Geom& g : h->geo) part = std::max(part, etile_part_count(g));
  {
    // Everything the hierarchy will hold, checked against the device's free
    // memory before the first allocation: a hierarchy that cannot fit is
    // refused with nothing allocated (and nothing to leak).  Each buffer is
    // counted with 2 MiB of allocation slack, and 1 GiB is left free.
    const double slack = 2.0 * 1024 * 1024;
    double need = 0.0;
    int count = 0;
    auto add = [&](double bytes) { need += bytes + slack; ++count; };
    add(8.0 * kMaxSlots * kMaxBlocks);
    add(4.0);
    add(8.0 * kMaxSlots);
    add(8.0 * h->geo.back().N);
    add(8.0 * h->geo.back().N);
    add(double(sizeof(CgCtrl)));
    add(16.0 * part);
    add(4.0);
    for (int l = 0; l < h->L; ++l) {
      const double n = double(F) * double(h->geo[l].N);
      for (int v = 0; v < 24; ++v) add(8.0 * (n + 4));
      add(4.0 * n);
      add(8.0 * double(coef_count(h->geo[l])));
    }
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
      delete h;
      set_error(std::string("mesh_hierarchy_create: cudaMemGetInfo: ") + cudaGetErrorString(e));
      return PF_ECUDA;
    }
    const double headroom = 1024.0 * 1024 * 1024;
    if (need + headroom > double(free_b)) {
      delete h;
      char msg[256];
      snprintf(msg, sizeof msg,
               "mesh_hierarchy_create: the hierarchy needs %.3g GB of device memory in %d "
               "buffers, %.3g GB are free (1 GB kept in reserve); nothing was allocated",
               need / 1e9, count, double(free_b) / 1e9);
      set_error(msg);
      return PF_ENOMEM;
    }
  }
  if ((rc = alloc(h, (void**)&h->scratch.partials, sizeof(double) * kMaxSlots * kMaxBlocks)) ||
      (rc = alloc(h, (void**)&h->scratch.counter, sizeof(unsigned))) ||
      (rc = alloc(h, (void**)&h->d_res, sizeof(double) * kMaxSlots)) ||
      (rc = alloc(h, (void**)&h->c_prev, sizeof(double) * h->geo.back().N)) ||
      (rc = alloc(h, (void**)&h->c_prev_save, sizeof(double) * h->geo.back().N)) ||
      (rc = alloc(h, (void**)&h->ctrl, sizeof(CgCtrl)))) {
    pf_mesh_hierarchy_destroy(h);
    return rc;
  }
  if ((part > 0 && (rc = alloc(h, &h->etile_part, sizeof(float4) * part))) ||
      (rc = alloc(h, (void**)&h->p_dev, sizeof(float)))) {
    pf_mesh_hierarchy_destroy(h);
    return rc;
  }
  if (cudaMallocHost((void**)&h->h_res, sizeof(double) * kMaxSlots) != cudaSuccess ||
      cudaMallocHost((void**)&h->h_ctrl, sizeof(CgCtrl)) != cudaSuccess) {
    pf_mesh_hierarchy_destroy(h);
    set_error("cudaMallocHost failed");
    return PF_ENOMEM;
  }
  cudaMemsetAsync(h->scratch.counter, 0, sizeof(unsigned), h->st);
  cudaMemsetAsync(h->p_dev, 0, sizeof(float), h->st);  // the material starts at p = 0
  cudaMemsetAsync(h->c_prev, 0, sizeof(double) * h->geo.back().N, h->st);
  h->lv.resize(h->L);
  for (int l = 0; l < h->L; ++l) {
    LevelBuf& B = h->lv[l];
    B.n = F * h->geo[l].N;
    // 4 spare values: the FP32 subproblem keeps two 16-byte-aligned FP32
    // vectors of padded length in one buffer
    const size_t bytes = sizeof(double) * (B.n + 4);
    double** vecs[] = {&B.x, &B.lb, &B.ub, &B.x0, &B.xlag, &B.dg, &B.g, &B.s, &B.lo, &B.hi,
                       &B.Hs, &B.r, &B.p, &B.q, &B.w, &B.Hw, &B.t1, &B.t2, &B.t3, &B.gin,
                       &B.gout, &B.dh, &B.minv, &B.g0};
    for (double** v : vecs)
      if ((rc = alloc(h, (void**)v, bytes))) {
        pf_mesh_hierarchy_destroy(h);
        return rc;
      }
    float** f32[] = {&B.xlag32};
    for (float** v : f32)
      if ((rc = alloc(h, (void**)v, sizeof(float) * B.n))) {
        pf_mesh_hierarchy_destroy(h);
        return rc;
      }
    // the FP64 stencil (27 x 16 doubles per node in 3D) is allocated on a
    // level's first FP64 lag (ensure_stencil): mixed-precision runs never
    // hold it on their FIRST_ORDER levels
    if ((rc = alloc(h, (void**)&B.coef, sizeof(double) * coef_count(h->geo[l])))) {
      pf_mesh_hierarchy_destroy(h);
      return rc;
    }
  }
  if (cudaStreamSynchronize(h->st) != cudaSuccess) {
    pf_mesh_hierarchy_destroy(h);
    set_error("mesh_hierarchy_create: stream error");
    return PF_ECUDA;
  }
  *out = h;
  return PF_OK;
}

pf_status pf_level_info(const pf_hierarchy* h, int level, int n_out[3], double* h_out,
                        long long* nodes_out) {
  if (!valid_level(h, level)) return bad("level_info: bad handle or level");
  const Geom& g = h->geo[level];
  if (n_out)
    for (int k = 0; k < 3; ++k) n_out[k] = g.n[k];
  if (h_out) *h_out = g.h;
  if (nodes_out) *nodes_out = g.N;
  return PF_OK;
}

pf_status pf_fractures_set(pf_hierarchy* h, int kind, int n, const double* rows,
                           double band_half_width, void* x_dev) {
  if (!h || !x_dev) return bad("fractures_set: null argument");
  if (n < 0 || (n > 0 && !rows)) return bad("fractures_set: bad row count");
  if (!(band_half_width > 0)) return bad("fractures_set: band_half_width must be > 0");
  if ((kind == PF_LINE2D && h->dim != 2) || ((kind == PF_DISC3D || kind == PF_BOX3D) && h->dim != 3) ||
      (kind != PF_LINE2D && kind != PF_DISC3D && kind != PF_BOX3D))
    return bad("fractures_set: kind does not match the dimension");
  const Geom& g = h->geo.back();
  // device rows of kRasterRow doubles:
  //   LINE2D [cx, cy, cos, sin, -sin, cos, half_length]
  //   DISC3D [cx, cy, cz, nx, ny, nz, radius]
  //   BOX3D  [cx, cy, cz, nx, ny, nz, ax, ay, az, bx, by, bz, half_a, half_b]
  const int width = kind == PF_LINE2D ? 4 : (kind == PF_DISC3D ? 7 : 14);
  double* pack = new double[kRasterRow * (n > 0 ? n : 1)]();
  for (int k = 0; k < n; ++k) {
    double* q = pack + kRasterRow * k;
    const double* r = rows + width * k;
    if (kind == PF_LINE2D) {
      const double c = std::cos(r[2]), s = std::sin(r[2]);
      q[0] = r[0]; q[1] = r[1]; q[2] = c; q[3] = s; q[4] = -s; q[5] = c; q[6] = r[3];
    } else {
      for (int j = 0; j < width; ++j) q[j] = r[j];
    }
    for (int j = 0; j < kRasterRow; ++j)
      if (!std::isfinite(q[j])) {
        delete[] pack;
        set_error("fractures_set: non-finite fracture row");
        return PF_ENONFINITE;
      }
  }
  double* rows_dev = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&rows_dev, sizeof(double) * kRasterRow * (n > 0 ? n : 1), h->st);
  if (e != cudaSuccess) {
    delete[] pack;
    set_error("fractures_set: allocation failed");
    return PF_ENOMEM;
  }
  e = cudaMemcpyAsync(rows_dev, pack, sizeof(double) * kRasterRow * n, cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess)
    e = rasterize(g, kind, n, rows_dev, band_half_width,
                  static_cast<double*>(x_dev) + h->dim * g.N, h->c_prev, h->st);
  cudaFreeAsync(rows_dev, h->st);
  cudaError_t e2 = cudaStreamSynchronize(h->st);
  delete[] pack;
  if (e != cudaSuccess || e2 != cudaSuccess) {
    set_error(std::string("fractures_set: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    return PF_ECUDA;
  }
  h->have_fractures = true;
  h->bounds_set = false;
  h->p_last = 0.0;
  return PF_OK;
}

pf_status pf_pressure_set(pf_hierarchy* h, double p) {
  if (!h) return bad("pressure_set: null handle");
  if (!std::isfinite(p)) {
    set_error("pressure_set: non-finite pressure");
    return PF_ENONFINITE;
  }
  h->p = p;
  for (auto& m : h->mat) m.p = p;
  const float pf = float(p);
  PF_TRY_CUDA(cudaMemcpyAsync(h->p_dev, &pf, sizeof(float), cudaMemcpyHostToDevice, h->st),
              "pressure_set");
  PF_TRY_CUDA(cudaStreamSynchronize(h->st), "pressure_set");
  return PF_OK;
}

static pf_status check_prec(int prec) {
  return (prec == PF_FP64 || prec == PF_FP32) ? PF_OK : bad("precision must be PF_FP64 or PF_FP32");
}

pf_status pf_energy(pf_hierarchy* h, int level, const void* x, int prec, double* E_host) {
  if (!valid_level(h, level) || !x || !E_host) return bad("energy: bad argument");
  if (check_prec(prec)) return PF_EINVAL;
  PF_TRY_CUDA(elem_energy(h->geo[level], h->mat[level], x, prec, h->scratch, h->d_res, h->st), "energy");
  PF_TRY_CUDA(cudaMemcpyAsync(h->h_res, h->d_res, sizeof(double), cudaMemcpyDeviceToHost, h->st), "energy");
  PF_TRY_CUDA(cudaStreamSynchronize(h->st), "energy");
  *E_host = h->h_res[0];
  if (!std::isfinite(*E_host)) {
    set_error("energy: non-finite result");
    return PF_ENONFINITE;
  }
  return PF_OK;
}

pf_status pf_energy_diff(pf_hierarchy* h, int level, const void* x, const void* s, int prec,
                         double* a_host) {
  if (!valid_level(h, level) || !x || !s || !a_host) return bad("energy_diff: bad argument");
  if (check_prec(prec)) return PF_EINVAL;
  PF_TRY_CUDA(elem_energy_diff(h->geo[level], h->mat[level], x, s, prec, h->scratch, h->d_res, h->st),
              "energy_diff");
  PF_TRY_CUDA(cudaMemcpyAsync(h->h_res, h->d_res, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st),
              "energy_diff");
  PF_TRY_CUDA(cudaStreamSynchronize(h->st), "energy_diff");
  for (int k = 0; k < 4; ++k) a_host[k] = h->h_res[k];
  return PF_OK;
}

pf_status pf_energy_diff_mixed(pf_hierarchy* h, int level, const double* x, const double* s,
                               const double* g, double* a_host) {
  if (!valid_level(h, level) || !x || !s || !g || !a_host)
    return bad("energy_diff_mixed: bad argument");
  PF_TRY_CUDA(elem_energy_diff_hi(h->geo[level], h->mat[level], x, s, g, h->scratch, h->d_res, h->st),
              "energy_diff_mixed");
  PF_TRY_CUDA(cudaMemcpyAsync(h->h_res, h->d_res, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st),
              "energy_diff_mixed");
  PF_TRY_CUDA(cudaStreamSynchronize(h->st), "energy_diff_mixed");
  for (int k = 0; k < 4; ++k) a_host[k] = h->h_res[k];
  return PF_OK;
}

pf_status pf_gradient(pf_hierarchy* h, int level, const void* x, void* g, int prec) {
  if (!valid_level(h, level) || !x || !g) return bad("gradient: bad argument");
  if (check_prec(prec)) return PF_EINVAL;
  if (prec == PF_FP64)
    PF_TRY_CUDA(elem_gradient_fp64(h->geo[level], h->mat[level], static_cast<const double*>(x),
                                   static_cast<double*>(g), h->lv[level].coef, h->st),
                "gradient");
  else
    PF_TRY_CUDA(elem_gradient(h->geo[level], h->mat[level], x, g, prec, h->st), "gradient");
  return PF_OK;
}

pf_status pf_gradient_df(pf_hierarchy* h, int level, const double* x, double* g) {
  if (!valid_level(h, level) || !x || !g) return bad("gradient_df: bad argument");
  if (!df_scratch_fits(h->geo[level])) return bad("gradient_df: grid too small for the scratch");
  PF_TRY_CUDA(elem_gradient_df(h->geo[level], h->mat[level], x, g, h->lv[level].coef, h->st),
              "gradient_df");
  return PF_OK;
}

pf_status pf_energy_df(pf_hierarchy* h, int level, const double* x, double* E_host) {
  if (!valid_level(h, level) || !x || !E_host) return bad("energy_df: bad argument");
  if (!df_scratch_fits(h->geo[level])) return bad("energy_df: grid too small for the scratch");
  PF_TRY_CUDA(elem_energy_df(h->geo[level], h->mat[level], x, h->lv[level].coef, h->scratch,
                             h->d_res, h->st),
              "energy_df");
  PF_TRY_CUDA(cudaMemcpyAsync(h->h_res, h->d_res, sizeof(double), cudaMemcpyDeviceToHost, h->st),
              "energy_df");
  PF_TRY_CUDA(cudaStreamSynchronize(h->st), "energy_df");
  *E_host = h->h_res[0];
  return PF_OK;
}

pf_status pf_gradient_step(pf_hierarchy* h, int level, const double* x, const double* s,
                           double* g) {
  if (!valid_level(h, level) || !x || !s || !g) return bad("gradient_step: bad argument");
  PF_TRY_CUDA(elem_gradient_step(h->geo[level], h->mat[level], x, s, g, h->st), "gradient_step");
  return PF_OK;
}

pf_status pf_hessvec(pf_hierarchy* h, int level, const void* x, const void* v, void* Hv, int prec) {
  if (!valid_level(h, level) || !x || !v || !Hv) return bad("hessvec: bad argument");
  if (check_prec(prec)) return PF_EINVAL;
  PF_TRY_CUDA(elem_hessvec(h->geo[level], h->mat[level], x, v, Hv, prec, h->st, nullptr,
                           h->etile_part, h->p_dev),
              "hessvec");
  return PF_OK;
}

pf_status pf_hessvec_lag_set(pf_hierarchy* h, int level, const void* x, int prec) {
  if (!valid_level(h, level) || !x) return bad("hessvec_lag_set: bad argument");
  if (check_prec(prec)) return PF_EINVAL;
  LevelBuf& B = h->lv[level];
  if (prec == PF_FP64) {
    PF_TRY_CUDA(cudaMemcpyAsync(B.xlag, x, sizeof(double) * B.n, cudaMemcpyDeviceToDevice, h->st),
                "hessvec_lag_set");
    PF_TRY_CUDA(ensure_stencil(h, level), "hessvec_lag_set: FP64 stencil");
    PF_TRY_CUDA(elem_hess_coef(h->geo[level], h->mat[level], B.xlag, B.coef, h->st), "hessvec_lag_set");
    PF_TRY_CUDA(stencil_assemble(h->geo[level], h->mat[level], B.coef, B.stencil, h->st),
                "hessvec_lag_set");
  } else {
    PF_TRY_CUDA(cudaMemcpyAsync(B.xlag32, x, sizeof(float) * B.n, cudaMemcpyDeviceToDevice, h->st),
                "hessvec_lag_set");
  }
  return PF_OK;
}

pf_status pf_tile_variant_set(pf_hierarchy* h, int level, int variant) {
  if (!valid_level(h, level) || variant < 0 || variant > (h->dim == 2 ? 4 : 3))
    return bad("tile_variant_set: bad level or variant (0 .. 3, 2D 0 .. 4)");
  h->geo[level].hv_variant = variant;
  for (auto& G : h->cg_graphs) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G = pf_hierarchy::CgGraph{};
  }
  return PF_OK;
}

pf_status pf_tile_variant_get(const pf_hierarchy* h, int level, int* variant) {
  if (!valid_level(h, level) || !variant) return bad("tile_variant_get: bad argument");
  *variant = h->geo[level].hv_variant;
  return PF_OK;
}

constexpr int kTileVariants = 5;  // slots per level in pf_autotune's us_out

pf_status pf_autotune(pf_hierarchy* h, int* variant_out, double* us_out) {
  if (!h) return bad("autotune: null handle");
  cudaEvent_t e0, e1;
  PF_TRY_CUDA(cudaEventCreate(&e0), "autotune");
  PF_TRY_CUDA(cudaEventCreate(&e1), "autotune");
  pf_status rc = PF_OK;
  for (int l = 0; l < h->L && rc == PF_OK; ++l) {
    LevelBuf& B = h->lv[l];
    Geom& g = h->geo[l];
    float* v = reinterpret_cast<float*>(B.p);
    float* y = reinterpret_cast<float*>(B.q);
    cudaError_t e = cudaMemsetAsync(v, 0, sizeof(float) * B.n, h->st);
    const int first = h->dim == 3 ? 1 : 0, last = h->dim == 3 ? 3 : 4;
    int best = 0;
    double best_us = 1e300;
    for (int var = 0; var < kTileVariants && e == cudaSuccess; ++var) {
      if (us_out) us_out[kTileVariants * l + var] = -1.0;
      if (var > last) continue;
      if (var < first) continue;
      g.hv_variant = var;
      e = elem_hessvec(g, h->mat[l], B.xlag32, v, y, 1, h->st, nullptr, h->etile_part, h->p_dev);
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->st);
      for (int r = 0; r < 5 && e == cudaSuccess; ++r)
        e = elem_hessvec(g, h->mat[l], B.xlag32, v, y, 1, h->st, nullptr, h->etile_part, h->p_dev);
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      const double us = 1e3 * double(ms) / 5.0;
      if (us_out) us_out[kTileVariants * l + var] = us;
      if (us < best_us) {
        best_us = us;
        best = var;
      }
    }
    g.hv_variant = best;
    if (variant_out) variant_out[l] = best;
    if (e != cudaSuccess) {
      set_error(std::string("autotune: ") + cudaGetErrorString(e));
      rc = PF_ECUDA;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // CG graphs captured the old tiles: rebuild on next use
  for (auto& G : h->cg_graphs) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G = pf_hierarchy::CgGraph{};
  }
  return rc;
}

pf_status pf_qp_pgs(pf_hierarchy* h, int level, const double* g, const double* lo, const double* hi,
                    double* s, int sweeps) {
  if (!valid_level(h, level) || !g || !lo || !hi || !s || sweeps < 1) return bad("qp_pgs: bad argument");
  if (!h->lv[level].stencil) {
    set_error("qp_pgs: no FP64 lag set on this level (pf_hessvec_lag_set)");
    return PF_ESTATE;
  }
  return qp_impl(h, level, g, lo, hi, s, sweeps, 0.0, 0, nullptr);
}

pf_status pf_qp_mprgp(pf_hierarchy* h, int level, const double* g, const double* lo, const double* hi,
                      double* s, double tol, int maxit, int* products) {
  if (!valid_level(h, level) || !g || !lo || !hi || !s || maxit < 1 || !(tol >= 0))
    return bad("qp_mprgp: bad argument");
  if (!h->lv[level].stencil) {
    set_error("qp_mprgp: no FP64 lag set on this level (pf_hessvec_lag_set)");
    return PF_ESTATE;
  }
  return qp_impl(h, level, g, lo, hi, s, 0, tol, maxit, products);
}

pf_status pf_galerkin_set(pf_hierarchy* h, const float* x_lag_fine) {
  if (!h || !x_lag_fine) return bad("galerkin_set: null argument");
  if (h->L < 2) return bad("galerkin_set: the hierarchy has no coarse level");
  PF_TRY_CUDA(galerkin_build(h, x_lag_fine, h->st), "galerkin_set");
  PF_TRY_CUDA(cudaStreamSynchronize(h->st), "galerkin_set");
  return PF_OK;
}

pf_status pf_galerkin_apply(pf_hierarchy* h, int level, const void* v, void* Hv, int prec) {
  if (!valid_level(h, level) || level >= h->L - 1 || !v || !Hv)
    return bad("galerkin_apply: bad argument (level must be a coarse level)");
  if (check_prec(prec)) return PF_EINVAL;
  if (!h->lv[level].gs) {
    set_error("galerkin_apply: no Galerkin operator built (pf_galerkin_set)");
    return PF_ESTATE;
  }
  PF_TRY_CUDA(galerkin_apply(h->geo[level], h->lv[level].gs, v, Hv, prec, h->st), "galerkin_apply");
  return PF_OK;
}

pf_status pf_hessvec_lagged(pf_hierarchy* h, int level, const void* v, void* Hv, int prec) {
  if (!valid_level(h, level) || !v || !Hv) return bad("hessvec_lagged: bad argument");
  if (check_prec(prec)) return PF_EINVAL;
  LevelBuf& B = h->lv[level];
  if (prec == PF_FP64 && !B.stencil) {
    set_error("hessvec_lagged: no FP64 lag set on this level");
    return PF_ESTATE;
  }
  if (prec == PF_FP64)
    PF_TRY_CUDA(stencil_apply(h->geo[level], B.stencil, static_cast<const double*>(v),
                              static_cast<double*>(Hv), h->st),
                "hessvec_lagged");
  else
    PF_TRY_CUDA(elem_hessvec(h->geo[level], h->mat[level], B.xlag32, v, Hv, 1, h->st, nullptr,
                             h->etile_part, h->p_dev),
                "hessvec_lagged");
  return PF_OK;
}

pf_status pf_prolong(pf_hierarchy* h, int coarse, const void* vc, void* vf, int prec) {
  if (!h || coarse < 0 || coarse + 1 >= h->L || !vc || !vf) return bad("prolong: bad argument");
  if (check_prec(prec)) return PF_EINVAL;
  PF_TRY_CUDA(xfer_prolong(h->geo[coarse], h->geo[coarse + 1], h->dim + 1, vc, vf, prec, h->st), "prolong");
  return PF_OK;
}

pf_status pf_restrict(pf_hierarchy* h, int coarse, const void* vf, void* vc, int prec) {
  if (!h || coarse < 0 || coarse + 1 >= h->L || !vc || !vf) return bad("restrict: bad argument");
  if (check_prec(prec)) return PF_EINVAL;
  PF_TRY_CUDA(xfer_restrict(h->geo[coarse], h->geo[coarse + 1], h->dim + 1, vf, vc, prec, false, h->st),
              "restrict");
  return PF_OK;
}

pf_status pf_project(pf_hierarchy* h, int coarse, const void* vf, void* vc, int prec) {
  if (!h || coarse < 0 || coarse + 1 >= h->L || !vc || !vf) return bad("project: bad argument");
  if (check_prec(prec)) return PF_EINVAL;
  PF_TRY_CUDA(xfer_restrict(h->geo[coarse], h->geo[coarse + 1], h->dim + 1, vf, vc, prec, true, h->st),
              "project");
  return PF_OK;
}

pf_status pf_coarse_bounds(pf_hierarchy* h, int coarse, const double* lo_f, const double* hi_f,
                           double* lo_c, double* hi_c) {
  if (!h || coarse < 0 || coarse + 1 >= h->L || !lo_f || !hi_f || !lo_c || !hi_c)
    return bad("coarse_bounds: bad argument");
  PF_TRY_CUDA(xfer_bounds(h->geo[coarse], h->geo[coarse + 1], h->dim + 1, lo_f, hi_f, lo_c, hi_c, h->st),
              "coarse_bounds");
  return PF_OK;
}

static pf_status check_params(const pf_rmtr_params& P) {
  if (!(P.eta1 > 0 && P.eta1 <= P.eta2 && P.eta2 <= 1) || !(P.gamma1 > 0 && P.gamma1 <= 1) ||
      !(P.gamma2 >= 1) || !(P.delta0 > 0) || !(P.delta_max >= P.delta0) || P.mu1 < 0 ||
      P.mu2 < 0 || P.coarse_its < 0 || P.cg_fine < 0 || P.cg_smooth < 0 || P.cg_coarse < 0 ||
      P.cauchy_backtracks < 0 || !(P.cauchy_c > 0 && P.cauchy_c < 1) || P.max_cycles < 0 ||
      !(P.rtol >= 0) || !(P.atol >= 0) ||
      (P.coarse_model != PF_GALERKIN && P.coarse_model != PF_FIRST_ORDER) ||
      (P.precision != PF_FP64 && P.precision != PF_FP32) ||
      (P.precondition != 0 && P.precondition != 1) || !(P.level_rtol >= 0 && P.level_rtol < 1) ||
      P.max_restarts < 0 || (P.keep_c_prev != 0 && P.keep_c_prev != 1) || !(P.pg_ref >= 0) ||
      (P.start != PF_START_PLAIN && P.start != PF_START_EXTRAPOLATE) || !(P.p_prev >= 0) ||
      (P.qp_solver != PF_QP_CG && P.qp_solver != PF_QP_PAPER) || P.pgs_sweeps < 1)
    return bad("rmtr_load_step: invalid parameters");
  if (P.qp_solver == PF_QP_PAPER && (P.precision != PF_FP64 || P.coarse_model != PF_FIRST_ORDER))
    return bad("rmtr_load_step: the paper's QP solvers need precision PF_FP64 and coarse_model "
               "PF_FIRST_ORDER (assembled FP64 Hessians on every level)");
  return PF_OK;
}

pf_status pf_rmtr_load_step(pf_hierarchy* h, void* x, const pf_rmtr_params* params,
                            pf_rmtr_stats* stats) {
  if (!h || !x) return bad("rmtr_load_step: null argument");
  pf_rmtr_params P;
  if (params) P = *params;
  else pf_rmtr_params_default(&P);
  if (check_params(P)) return PF_EINVAL;
  return rmtr_load_step_impl(h, static_cast<double*>(x), P, stats);
}

pf_status pf_rmtr_load_step_host(pf_hierarchy* h, double* x_host, const pf_rmtr_params* params,
                                 pf_rmtr_stats* stats) {
  if (!h || !x_host) return bad("rmtr_load_step_host: null argument");
  pf_rmtr_params P;
  if (params) P = *params;
  else pf_rmtr_params_default(&P);
  if (check_params(P)) return PF_EINVAL;
  // the finest level's dH scratch is unused by a load step: stage the state there
  LevelBuf& B = h->lv.back();
  double* stage = B.dh;
  PF_TRY_CUDA(cudaMemcpyAsync(stage, x_host, sizeof(double) * B.n, cudaMemcpyHostToDevice, h->st),
              "rmtr_load_step_host");
  pf_status rc = rmtr_load_step_impl(h, stage, P, stats);
  if (rc != PF_OK && rc != PF_ENOTCONV && rc != PF_ENONFINITE) return rc;
  PF_TRY_CUDA(cudaMemcpyAsync(x_host, stage, sizeof(double) * B.n, cudaMemcpyDeviceToHost, h->st),
              "rmtr_load_step_host");
  PF_TRY_CUDA(cudaStreamSynchronize(h->st), "rmtr_load_step_host");
  return rc;
}

pf_status pf_rmtr_load_step_batch(int n, pf_hierarchy* const* hs, double* const* xs,
                                  const pf_rmtr_params* params, int n_threads,
                                  pf_rmtr_stats* stats, pf_status* status) {
  if (n < 0 || (n > 0 && (!hs || !xs))) return bad("rmtr_load_step_batch: bad argument");
  for (int i = 0; i < n; ++i)
    if (!hs[i] || !xs[i]) return bad("rmtr_load_step_batch: null instance");
  pf_rmtr_params P;
  if (params) P = *params;
  else pf_rmtr_params_default(&P);
  if (check_params(P)) return PF_EINVAL;
  if (n == 0) return PF_OK;
  int dev = 0;
  PF_TRY_CUDA(cudaGetDevice(&dev), "rmtr_load_step_batch");
  // largest instances first (longest-processing-time order)
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return hs[a]->lv.back().n > hs[b]->lv.back().n;
  });
  std::vector<pf_status> st(n, PF_OK);
  std::vector<pf_rmtr_stats> ss(n);
  std::vector<std::string> errs(n);
  std::atomic<int> next{0};
  const int nt = std::max(1, std::min(n_threads > 0 ? n_threads : n, std::min(n, 64)));
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n) break;
      const int i = order[k];
      st[i] = rmtr_load_step_impl(hs[i], xs[i], P, &ss[i]);
      if (st[i] != PF_OK) errs[i] = pf_last_error();
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  pf_status rc = PF_OK;
  for (int i = 0; i < n; ++i) {
    if (stats) stats[i] = ss[i];
    if (status) status[i] = st[i];
    if (rc == PF_OK && st[i] != PF_OK) {
      rc = st[i];
      set_error("rmtr_load_step_batch: instance " + std::to_string(i) + ": " + errs[i]);
    }
  }
  return rc;
}

pf_status pf_projected_gradient(pf_hierarchy* h, const double* x, double* pg) {
  if (!h || !x || !pg) return bad("projected_gradient: null argument");
  return projected_gradient_impl(h, x, pg);
}

pf_status pf_get_c_prev(pf_hierarchy* h, double* out) {
  if (!h || !out) return bad("get_c_prev: null argument");
  PF_TRY_CUDA(cudaMemcpyAsync(out, h->c_prev, sizeof(double) * h->geo.back().N,
                              cudaMemcpyDeviceToDevice, h->st),
              "get_c_prev");
  return PF_OK;
}

pf_status pf_get_fields(pf_hierarchy* h, int level, int which, double* out) {
  if (!valid_level(h, level) || !out) return bad("get_fields: bad argument");
  const Geom& g = h->geo[level];
  const long long n = (long long)(h->dim + 1) * g.N;
  switch (which) {
    case PF_FIELD_C_PREV:
      if (level != h->L - 1) return bad("get_fields: c_prev lives on the finest level");
      PF_TRY_CUDA(cudaMemcpyAsync(out, h->c_prev, sizeof(double) * g.N, cudaMemcpyDeviceToDevice,
                                  h->st),
                  "get_fields");
      return PF_OK;
    case PF_FIELD_LOWER:
    case PF_FIELD_UPPER:
      if (!h->bounds_set) {
        set_error("get_fields: no load step has set the feasible sets");
        return PF_ESTATE;
      }
      PF_TRY_CUDA(cudaMemcpyAsync(out, which == PF_FIELD_LOWER ? h->lv[level].lb : h->lv[level].ub,
                                  sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st),
                  "get_fields");
      return PF_OK;
    case PF_FIELD_FIXED:
      PF_TRY_CUDA(fixed_mask(g, out, h->st), "get_fields");
      return PF_OK;
    default:
      return bad("get_fields: unknown field");
  }
}

pf_status pf_probe_fma(int prec, double* flops) {
  if (!flops) return bad("probe_fma: null argument");
  if (check_prec(prec)) return PF_EINVAL;
  int dev = 0, sms = 0;
  PF_TRY_CUDA(cudaGetDevice(&dev), "probe_fma");
  PF_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "probe_fma");
  void* out = nullptr;
  PF_TRY_CUDA(cudaMalloc(&out, 16), "probe_fma");
  const int blocks = sms * 8, threads = 256;
  const int reps = prec ? 1 << 16 : 1 << 11;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  for (int pass = 0; pass < 2; ++pass) {  // first pass warms up
    cudaEventRecord(e0, 0);
    if (prec)
      k_fma_probe<float><<<blocks, threads>>>(static_cast<float*>(out), reps, 0.999f, 1e-4f);
    else
      k_fma_probe<double><<<blocks, threads>>>(static_cast<double*>(out), reps, 0.999, 1e-4);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) {
    set_error(std::string("probe_fma: ") + cudaGetErrorString(e));
    return PF_ECUDA;
  }
  *flops = 2.0 * 8.0 * double(reps) * double(blocks) * threads / (double(ms) * 1e-3);
  return PF_OK;
}

}  // extern "C"
