// Glue between the 2D solver state and the U-Net: input features, training
// targets, proposals from the network output, and the trust-region
// acceptance test of a proposal (eq. rho_tr with FP64 energy difference,
// gradient and Hessian).
#include <cmath>
#include <string>

#include "pf_hier.h"
#include "pf_reduce.cuh"

namespace pf {

namespace {

__global__ void k_features(Geom g, const double* __restrict__ x, const double* __restrict__ cb,
                           double su, float ratio, int H, int W, float* __restrict__ f) {
  const long long HW = (long long)H * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < HW;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = int(t / W), i = int(t % W);
    float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < g.n[0] && j < g.n[1]) {
      const long long k = i + (long long)g.n[0] * j;
      const double c = x[2 * g.N + k];
      v[0] = float(x[k] * su);
      v[1] = float(x[g.N + k] * su);
      v[2] = float(c);
      v[3] = ratio;
      v[4] = cb ? float(c - cb[k]) : 0.f;
    }
#pragma unroll
    for (int ch = 0; ch < 5; ++ch) f[ch * HW + t] = v[ch];
  }
}

__global__ void k_target(Geom g, const double* __restrict__ xp, const double* __restrict__ xn,
                         double ratio, double su, double sc, int H, int W, float* __restrict__ tg) {
  const long long HW = (long long)H * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < HW;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = int(t / W), i = int(t % W);
    float v[3] = {0.f, 0.f, 0.f};
    if (i < g.n[0] && j < g.n[1]) {
      const long long k = i + (long long)g.n[0] * j;
      v[0] = float((xn[k] - ratio * xp[k]) * su);
      v[1] = float((xn[g.N + k] - ratio * xp[g.N + k]) * su);
      v[2] = float((xn[2 * g.N + k] - xp[2 * g.N + k]) * sc);
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) tg[ch * HW + t] = v[ch];
  }
}

__global__ void k_apply(Geom g, const double* __restrict__ xp, const float* __restrict__ y,
                        double ratio, double su, double sc, int H, int W, double* __restrict__ xh) {
  const long long HW = (long long)H * W;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < g.N;
       k += (long long)gridDim.x * blockDim.x) {
    const long long i = k % g.n[0], j = k / g.n[0];
    const long long t = j * W + i;
    xh[k] = ratio * xp[k] + su * double(y[t]);
    xh[g.N + k] = ratio * xp[g.N + k] + su * double(y[HW + t]);
    xh[2 * g.N + k] = xp[2 * g.N + k] + sc * double(y[2 * HW + t]);
  }
}

// s = P_F(xhat) - x on the finest bounds (c_prev <= c <= 1, clamped u)
__global__ void k_step(Geom g, int dim, const double* __restrict__ x, const double* __restrict__ xh,
                       const double* __restrict__ cprev, double* __restrict__ s) {
  const long long n = (long long)(dim + 1) * g.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = int(i / g.N);
    const long long k = i - f * g.N;
    double lo, hi;
    if (f == dim) {
      lo = cprev[k];
      hi = 1.0;
    } else {
      const long long ix = k % g.n[0], r = k / g.n[0], iy = r % g.n[1], iz = r / g.n[1];
      bool b = ix == 0 || ix == g.n[0] - 1 || iy == 0 || iy == g.n[1] - 1;
      if (dim == 3) b = b || iz == 0 || iz == g.n[2] - 1;
      lo = b ? 0.0 : -INFINITY;
      hi = b ? 0.0 : INFINITY;
    }
    s[i] = fmin(fmax(xh[i], lo), hi) - x[i];
  }
}

__global__ void __launch_bounds__(256) k_dots(long long n, const double* __restrict__ g,
                                              const double* __restrict__ s,
                                              const double* __restrict__ hs, double* partials,
                                              unsigned* counter, double* out) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    acc[0] += g[i] * s[i];
    acc[1] += s[i] * hs[i];
  }
  grid_finish<2, OpSum>(acc, partials, counter, out);
}

__global__ void k_accept(long long n, double* __restrict__ x, const double* __restrict__ s) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += s[i];
}

int grid_n(long long n) {
  long long b = (n + 255) / 256;
  if (b > 8192) b = 8192;
  return int(b < 1 ? 1 : b);
}

pf_status check_2d(pf_hierarchy* h, int H, int W, const char* what) {
  if (!h || h->dim != 2) {
    set_error(std::string(what) + ": needs a 2D hierarchy");
    return PF_EINVAL;
  }
  const Geom& g = h->geo.back();
  if (H < g.n[1] || W < g.n[0] || H % 8 || W % 8) {
    set_error(std::string(what) + ": H x W must cover the finest grid and be multiples of 8");
    return PF_EINVAL;
  }
  return PF_OK;
}

pf_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PF_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return PF_ECUDA;
}

}  // namespace
}  // namespace pf

using namespace pf;

extern "C" {

pf_status pf_learned_features(pf_hierarchy* h, const double* x_prev, const double* c_before,
                              double p_prev, double p_new, int H, int W, float* feat) {
  if (pf_status rc = check_2d(h, H, W, "learned_features")) return rc;
  if (!x_prev || !feat || !(p_prev > 0) || !std::isfinite(p_new)) {
    set_error("learned_features: bad argument (p_prev must be > 0)");
    return PF_EINVAL;
  }
  const Geom& g = h->geo.back();
  k_features<<<grid_n((long long)H * W), 256, 0, h->st>>>(g, x_prev, c_before, h->E / p_prev,
                                                           float(p_new / p_prev), H, W, feat);
  return cuda_status(cudaGetLastError(), "learned_features");
}

pf_status pf_learned_target(pf_hierarchy* h, const double* x_prev, const double* x_new, double p_prev,
                            double p_new, int H, int W, float* target) {
  if (pf_status rc = check_2d(h, H, W, "learned_target")) return rc;
  if (!x_prev || !x_new || !target || !(p_new != p_prev) || !(p_prev > 0)) {
    set_error("learned_target: bad argument (p_prev > 0 and p_new != p_prev needed)");
    return PF_EINVAL;
  }
  const double dp = p_new - p_prev;
  k_target<<<grid_n((long long)H * W), 256, 0, h->st>>>(h->geo.back(), x_prev, x_new, p_new / p_prev,
                                                         h->E / dp, 1.0 / dp, H, W, target);
  return cuda_status(cudaGetLastError(), "learned_target");
}

pf_status pf_learned_apply(pf_hierarchy* h, const double* x_prev, const float* y, double p_prev,
                           double p_new, int H, int W, double* xhat) {
  if (pf_status rc = check_2d(h, H, W, "learned_apply")) return rc;
  if (!x_prev || !y || !xhat || !(p_prev > 0)) {
    set_error("learned_apply: bad argument (p_prev must be > 0)");
    return PF_EINVAL;
  }
  const double dp = p_new - p_prev;
  const Geom& g = h->geo.back();
  k_apply<<<grid_n(g.N), 256, 0, h->st>>>(g, x_prev, y, p_new / p_prev, dp / h->E, dp, H, W, xhat);
  return cuda_status(cudaGetLastError(), "learned_apply");
}

pf_status pf_learned_propose(pf_hierarchy* h, double* x, const double* xhat, double eta,
                             double* rho_out, int* accepted_out) {
  if (!h || !x || !xhat || !rho_out || !accepted_out || !(eta > 0 && eta < 1)) {
    set_error("learned_propose: bad argument");
    return PF_EINVAL;
  }
  const int L = h->L, dim = h->dim;
  const Geom& g = h->geo[L - 1];
  LevelBuf& B = h->lv[L - 1];
  const long long n = B.n;
  double* s = B.t1;
  double* gr = B.t2;
  double* hs = B.t3;
  cudaError_t e = cudaMemcpyAsync(h->c_prev, x + dim * g.N, sizeof(double) * g.N,
                                  cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess) {
    k_step<<<grid_n(n), 256, 0, h->st>>>(g, dim, x, xhat, h->c_prev, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = elem_energy_diff(g, h->mat[L - 1], x, s, 0, h->scratch, h->d_res, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_res, h->d_res, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_status(e, "learned_propose");
  const double actual = -(h->h_res[0] + h->h_res[1] + h->h_res[2] + h->h_res[3]);
  e = elem_gradient_fp64(g, h->mat[L - 1], x, gr, B.coef, h->st);
  if (e == cudaSuccess) e = elem_hessvec(g, h->mat[L - 1], x, s, hs, 0, h->st);
  if (e == cudaSuccess) {
    k_dots<<<reduce_grid(n), 256, 0, h->st>>>(n, gr, s, hs, h->scratch.partials, h->scratch.counter, h->d_res);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_res, h->d_res, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_status(e, "learned_propose");
  const double pred = -(h->h_res[0] + 0.5 * h->h_res[1]);
  const double rho = pred > 0.0 ? actual / pred : -INFINITY;
  const int acc = (rho > eta && actual > 0.0) ? 1 : 0;
  if (acc) {
    k_accept<<<grid_n(n), 256, 0, h->st>>>(n, x, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_status(e, "learned_propose");
  }
  *rho_out = rho;
  *accepted_out = acc;
  return PF_OK;
}

}  // extern "C"
