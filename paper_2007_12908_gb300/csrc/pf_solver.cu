// RMTR load step on the device (Algorithm 1 V-cycle, Algorithm 2 trust-region
// method, Algorithm 3 Convergence_control, eq. rho_tr / rho_ml, Hessian
// lagging of Sec. 4.2.1), with a projected-search truncated CG for the
// trust-region subproblem eq. (model_qp).
//
// All vectors stay on the device.  The host keeps only the control flow: it
// reads back the few scalars each branch needs (dot products, ratios) from
// deterministic grid reductions.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "pf_hier.h"
#include "pf_reduce.cuh"

namespace pf {

struct CudaFail {
  cudaError_t e;
  const char* where;
};

static inline void ck(cudaError_t e, const char* where) {
  if (e != cudaSuccess) throw CudaFail{e, where};
}

template <class F>
__global__ void k_map(long long n, F f) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    f(i);
}

template <class F>
__global__ void k_map_skip(long long n, F f, const int* __restrict__ skip) {
  if (*skip) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    f(i);
}

// Each thread combines its elements in precision A (FP32 for FP32 vectors,
// whose dot products then cost no FP64 instructions per element); blocks
// and the grid combine in FP64.
template <int K, class Op, class A, class F>
__device__ __forceinline__ void thread_part(long long n, F& f, double (&out)[K]) {
  A acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = A(Op::id());
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    A v[K];
    f(i, v);
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = Op::op(acc[k], v[k]);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = double(acc[k]);
}

// Reduction whose last block passes the combined values to fin() on the
// device; a no-op launch when *skip is set.
template <int K, class Op, class A, class F, class Fin>
__global__ void __launch_bounds__(256) k_red_fin(long long n, F f, Fin fin, double* partials,
                                                 unsigned* counter, const int* __restrict__ skip) {
  if (*skip) return;
  double acc[K];
  thread_part<K, Op, A>(n, f, acc);
  grid_finish_fn<K, Op>(acc, partials, counter, fin);
}

__global__ void k_ctrl_start(CgCtrl* c, double rr, double rz, double tol, int used, int cg_max) {
  c->rr = rr;
  c->rz = rz;
  c->tol = tol;
  c->alpha = 0.0;
  c->beta = 0.0;
  c->kappa = 0.0;
  c->done = 0;
  c->state = CG_RUNNING;
  c->used = used;
  c->cg_max = cg_max;
}

// Start of a CG run from the restart reduction's (r.r, r.M^-1 r) on the
// device: the forcing tolerance min(0.1, sqrt||r0||) ||r0|| on the first run
// of a subproblem, and a run that starts already converged is stopped before
// its first iteration (CG_CONV), so the host needs no read-back before it.
__global__ void k_ctrl_start_dev(CgCtrl* c, const double* rrz, int first, int used, int cg_max) {
  const double rr = rrz[0];
  if (first) {
    const double r0 = sqrt(rr);
    c->tol = fmin(0.1, sqrt(r0)) * r0;
  }
  c->rr = rr;
  c->rz = rrz[1];
  c->alpha = 0.0;
  c->beta = 0.0;
  c->kappa = 0.0;
  c->used = used;
  c->cg_max = cg_max;
  const bool stop = sqrt(rr) <= c->tol || rr == 0.0;
  c->done = stop ? 1 : 0;
  c->state = stop ? CG_CONV : CG_RUNNING;
}

template <int K, class Op, class A, class F>
__global__ void __launch_bounds__(256) k_red(long long n, F f, double* partials, unsigned* counter,
                                             double* out) {
  double acc[K];
  thread_part<K, Op, A>(n, f, acc);
  grid_finish<K, Op>(acc, partials, counter, out);
}

// ---------------------------------------------------------------- FP32 CG passes
// The vector passes of one projected-CG iteration on FP32 vectors, on groups
// of four dofs (n a multiple of 4, 16-byte aligned vectors; 16-byte loads
// keep more bytes in flight per instruction).  ga/gb are the free gaps
// (a < 0 < b on the free set, both 0 elsewhere); off the free set r, p and
// w are 0 and stay 0, so a group whose four dofs are all outside reads only
// its gaps.
__device__ __forceinline__ float4 ld4(const float* v, long long j) {
  return reinterpret_cast<const float4*>(v)[j];
}
__device__ __forceinline__ void st4(float* v, long long j, float4 x) {
  reinterpret_cast<float4*>(v)[j] = x;
}
__device__ __forceinline__ bool any_free(float4 a) {
  return (a.x < 0.f) | (a.y < 0.f) | (a.z < 0.f) | (a.w < 0.f);
}

// Restart of the CG loop at s: r = -(g + Hs) and p = M^-1 r on the free set
// of s (0 elsewhere), w = 0, the gaps of s; (r.r, r.M^-1 r) to out.
struct CgInitOp {
  __device__ __forceinline__ static void lane(float lo, float hi, float s, float g, float hs,
                                              float m, float& r, float& p, float& a, float& b,
                                              float& rr, float& rz) {
    const float ai = lo - s, bi = hi - s;
    const bool fr = ai < 0.f && 0.f < bi;
    const float ri = fr ? -(g + hs) : 0.f;
    const float zi = m * ri;
    r = ri;
    p = zi;
    a = fr ? ai : 0.f;
    b = fr ? bi : 0.f;
    rr += ri * ri;
    rz += ri * zi;
  }
};

__global__ void __launch_bounds__(256) k_cg_init4(long long n4, const float* __restrict__ lo,
                                                  const float* __restrict__ hi,
                                                  const float* __restrict__ s,
                                                  const float* __restrict__ g,
                                                  const float* __restrict__ Hs,
                                                  const float* __restrict__ mi, bool pc,
                                                  float* __restrict__ r, float* __restrict__ p,
                                                  float* __restrict__ w, float* __restrict__ ga,
                                                  float* __restrict__ gb, double* partials,
                                                  unsigned* counter, double* out) {
  float rr = 0.f, rz = 0.f;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n4;
       j += (long long)gridDim.x * blockDim.x) {
    const float4 l4 = ld4(lo, j), h4 = ld4(hi, j), s4 = ld4(s, j);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 g4 = z4, hs4 = z4, m4 = make_float4(1.f, 1.f, 1.f, 1.f);
    const float4 a4 = make_float4(l4.x - s4.x, l4.y - s4.y, l4.z - s4.z, l4.w - s4.w);
    const float4 b4 = make_float4(h4.x - s4.x, h4.y - s4.y, h4.z - s4.z, h4.w - s4.w);
    const bool any = ((a4.x < 0.f) & (b4.x > 0.f)) | ((a4.y < 0.f) & (b4.y > 0.f)) |
                     ((a4.z < 0.f) & (b4.z > 0.f)) | ((a4.w < 0.f) & (b4.w > 0.f));
    if (any) {
      g4 = ld4(g, j);
      hs4 = ld4(Hs, j);
      if (pc) m4 = ld4(mi, j);
    }
    float4 r4, p4, ga4, gb4;
    CgInitOp::lane(l4.x, h4.x, s4.x, g4.x, hs4.x, m4.x, r4.x, p4.x, ga4.x, gb4.x, rr, rz);
    CgInitOp::lane(l4.y, h4.y, s4.y, g4.y, hs4.y, m4.y, r4.y, p4.y, ga4.y, gb4.y, rr, rz);
    CgInitOp::lane(l4.z, h4.z, s4.z, g4.z, hs4.z, m4.z, r4.z, p4.z, ga4.z, gb4.z, rr, rz);
    CgInitOp::lane(l4.w, h4.w, s4.w, g4.w, hs4.w, m4.w, r4.w, p4.w, ga4.w, gb4.w, rr, rz);
    st4(r, j, r4);
    st4(p, j, p4);
    st4(w, j, z4);
    st4(ga, j, ga4);
    st4(gb, j, gb4);
  }
  double acc[2] = {double(rr), double(rz)};
  grid_finish<2, OpSum>(acc, partials, counter, out);
}

// Update after the product q = H p: w += alpha p, r -= alpha q (free set);
// the last block tests the box, the forcing term and the budget, and sets
// beta (CG_* states of the control block).
__device__ __forceinline__ void cg_update_lane(float al, float a, float b, float q, float p,
                                               float& w, float& r, float m, float& rr, float& lv,
                                               float& rz) {
  const float qi = a < 0.f ? q : 0.f;
  w = w + al * p;
  r = r - al * qi;
  rr += r * r;
  lv += ((w < a) | (w > b)) ? 1.f : 0.f;
  rz += r * (m * r);
}

__global__ void __launch_bounds__(256) k_cg_update4(long long n4, const float* __restrict__ ga,
                                                    const float* __restrict__ gb,
                                                    const float* __restrict__ q,
                                                    const float* __restrict__ p,
                                                    const float* __restrict__ mi, bool pc,
                                                    float* __restrict__ w, float* __restrict__ r,
                                                    CgCtrl* c, double* partials,
                                                    unsigned* counter) {
  if (c->done) return;
  const float al = float(c->alpha);
  float rr = 0.f, lv = 0.f, rz = 0.f;
  // two groups per iteration, every load of both issued before any store
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; j0 < n4; j0 += 2 * stride) {
    const long long j1 = j0 + stride;
    const bool h1 = j1 < n4;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f), one4 = make_float4(1.f, 1.f, 1.f, 1.f);
    const float4 a0 = ld4(ga, j0), a1 = h1 ? ld4(ga, j1) : z4;
    const bool f0 = any_free(a0), f1 = any_free(a1);
    float4 b[2] = {z4, z4}, qq[2] = {z4, z4}, pp[2] = {z4, z4}, ww[2] = {z4, z4}, rv[2] = {z4, z4};
    float4 mm[2] = {one4, one4};
    if (f0) {
      b[0] = ld4(gb, j0); qq[0] = ld4(q, j0); pp[0] = ld4(p, j0); ww[0] = ld4(w, j0); rv[0] = ld4(r, j0);
      if (pc) mm[0] = ld4(mi, j0);
    }
    if (f1) {
      b[1] = ld4(gb, j1); qq[1] = ld4(q, j1); pp[1] = ld4(p, j1); ww[1] = ld4(w, j1); rv[1] = ld4(r, j1);
      if (pc) mm[1] = ld4(mi, j1);
    }
    const float4 aa[2] = {a0, a1};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      cg_update_lane(al, aa[k].x, b[k].x, qq[k].x, pp[k].x, ww[k].x, rv[k].x, mm[k].x, rr, lv, rz);
      cg_update_lane(al, aa[k].y, b[k].y, qq[k].y, pp[k].y, ww[k].y, rv[k].y, mm[k].y, rr, lv, rz);
      cg_update_lane(al, aa[k].z, b[k].z, qq[k].z, pp[k].z, ww[k].z, rv[k].z, mm[k].z, rr, lv, rz);
      cg_update_lane(al, aa[k].w, b[k].w, qq[k].w, pp[k].w, ww[k].w, rv[k].w, mm[k].w, rr, lv, rz);
    }
    if (f0) {
      st4(w, j0, ww[0]);
      st4(r, j0, rv[0]);
    }
    if (f1) {
      st4(w, j1, ww[1]);
      st4(r, j1, rv[1]);
    }
  }
  double acc[3] = {double(rr), double(lv), double(rz)};
  auto fin = [c](double(&a)[3]) {
    if (a[1] > 0.0) {
      c->done = 1;
      c->state = CG_LEAVE;
    } else if (sqrt(a[0]) <= c->tol) {
      c->done = 1;
      c->state = CG_CONV;
    } else if (c->used >= c->cg_max) {
      c->done = 1;
      c->state = CG_BUDGET;
    } else {
      c->beta = a[2] / c->rz;
      c->rr = a[0];
      c->rz = a[2];
    }
  };
  grid_finish_fn<3, OpSum>(acc, partials, counter, fin);
}

// p . q for q = H p, and the step alpha = r.M^-1 r / p.q (or a stop on
// non-positive curvature); a group with p = 0 (outside the free set) reads
// only p.
__global__ void __launch_bounds__(256) k_cg_dot4(long long n4, const float* __restrict__ p,
                                                 const float* __restrict__ q, CgCtrl* c,
                                                 double* partials, unsigned* counter) {
  if (c->done) return;
  float pq = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; j0 < n4; j0 += 2 * stride) {
    const long long j1 = j0 + stride;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 p0 = ld4(p, j0), p1 = j1 < n4 ? ld4(p, j1) : z4;
    const bool n0 = p0.x != 0.f || p0.y != 0.f || p0.z != 0.f || p0.w != 0.f;
    const bool n1 = p1.x != 0.f || p1.y != 0.f || p1.z != 0.f || p1.w != 0.f;
    const float4 q0 = n0 ? ld4(q, j0) : z4, q1 = n1 ? ld4(q, j1) : z4;
    pq += p0.x * q0.x + p0.y * q0.y + p0.z * q0.z + p0.w * q0.w;
    pq += p1.x * q1.x + p1.y * q1.y + p1.z * q1.z + p1.w * q1.w;
  }
  double acc[1] = {double(pq)};
  auto fin = [c](double(&a)[1]) { cg_take_curvature(c, a[0]); };
  grid_finish_fn<1, OpSum>(acc, partials, counter, fin);
}

// Direction update p = M^-1 r + beta p (free set; p stays 0 elsewhere).
__global__ void __launch_bounds__(256) k_cg_dir4(long long n4, const float* __restrict__ ga,
                                                 const float* __restrict__ r,
                                                 const float* __restrict__ mi, bool pc,
                                                 float* __restrict__ p, const CgCtrl* c) {
  if (c->done) return;
  const float be = float(c->beta);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; j0 < n4; j0 += 2 * stride) {
    const long long j1 = j0 + stride;
    const bool h1 = j1 < n4;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f), one4 = make_float4(1.f, 1.f, 1.f, 1.f);
    const bool f0 = any_free(ld4(ga, j0)), f1 = h1 && any_free(ld4(ga, j1));
    float4 rv[2] = {z4, z4}, pp[2] = {z4, z4}, mm[2] = {one4, one4};
    if (f0) {
      rv[0] = ld4(r, j0); pp[0] = ld4(p, j0);
      if (pc) mm[0] = ld4(mi, j0);
    }
    if (f1) {
      rv[1] = ld4(r, j1); pp[1] = ld4(p, j1);
      if (pc) mm[1] = ld4(mi, j1);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float4 m4 = mm[k], r4 = rv[k], p4 = pp[k];
      pp[k] = make_float4(cg_direction(m4.x, r4.x, be, p4.x), cg_direction(m4.y, r4.y, be, p4.y),
                          cg_direction(m4.z, r4.z, be, p4.z), cg_direction(m4.w, r4.w, be, p4.w));
    }
    if (f0) st4(p, j0, pp[0]);
    if (f1) st4(p, j1, pp[1]);
  }
}

// Condition of the CG loop's while node: repeat while the run is not done.
// The update pass stops the run at the budget; the cap here only guards
// against a control block that stopped counting.
__global__ void k_cg_cond(CgCtrl* c, cudaGraphConditionalHandle h) {
  if (!c->done && c->used > c->cg_max) {
    c->done = 1;
    c->state = CG_BUDGET;
  }
  cudaGraphSetConditional(h, c->done ? 0u : 1u);
}

// Grid for a grid-stride kernel of 256-thread blocks over `items` work
// items: every block resident at once (occupancy x SMs, computed once per
// kernel), no more than the items need and no more than the reduction
// scratch holds.  A second, partial wave of blocks would leave SMs idle.
template <class K>
static int resident_grid(K kernel, long long items) {
  static const int cap = [kernel] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
    const int r = per_sm * sms;
    return r > 0 ? std::min(r, kMaxBlocks) : kMaxBlocks;
  }();
  const long long want = (items + 255) / 256;
  return int(std::max(1LL, std::min<long long>(want, cap)));
}

static inline long long pad4(long long n) { return (n + 3) & ~3LL; }

// Zero lanes [n, np) of up to 16 FP32 vectors.
struct PadLanes {
  float* v[16];
  int count;
  long long n, np;
};
__global__ void k_zero_pad(PadLanes z) {
  const long long pad = z.np - z.n;
  for (int t = threadIdx.x; t < z.count * pad; t += blockDim.x) z.v[t / pad][z.n + t % pad] = 0.f;
}

static int map_grid(long long n) {
  long long b = (n + 255) / 256;
  return int(std::max(1LL, std::min(b, 4LL * 1216)));
}

// Is plane-local node i on the domain boundary?
__device__ __forceinline__ bool on_boundary(const Geom& g, long long i) {
  const int ix = int(i % g.n[0]);
  const long long r = i / g.n[0];
  const int iy = int(r % g.n[1]);
  const int iz = int(r / g.n[1]);
  bool b = ix == 0 || ix == g.n[0] - 1 || iy == 0 || iy == g.n[1] - 1;
  if (g.dim == 3) b = b || iz == 0 || iz == g.n[2] - 1;
  return b;
}

__global__ void k_fixed_mask(Geom g, double* __restrict__ out) {
  const long long n = (long long)(g.dim + 1) * g.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = int(i / g.N);
    out[i] = (f < g.dim && on_boundary(g, i - f * g.N)) ? 1.0 : 0.0;
  }
}

cudaError_t fixed_mask(const Geom& g, double* out, cudaStream_t st) {
  const long long n = (long long)(g.dim + 1) * g.N;
  const int blocks = int(std::min<long long>((n + 255) / 256, 4LL * 1216));
  k_fixed_mask<<<blocks, 256, 0, st>>>(g, out);
  return cudaGetLastError();
}

__device__ __forceinline__ double clampv(double x, double lo, double hi) {
  return fmin(fmax(x, lo), hi);
}
__device__ __forceinline__ float clampv(float x, float lo, float hi) {
  return fminf(fmaxf(x, lo), hi);
}

struct Solver {
  pf_hierarchy* H;
  const pf_rmtr_params& P;
  pf_rmtr_stats& S;
  cudaStream_t st;
  int L, F;
  bool mixed;
  // What each level's B.g holds: G_NONE, G_AT_X (grad h at B.x) or G_STEP
  // (grad h at B.x - B.s: an accepted step not yet applied to the gradient)
  enum { G_NONE = 0, G_AT_X = 1, G_STEP = 2 };
  std::vector<int> gstate;

  Solver(pf_hierarchy* h, const pf_rmtr_params& p, pf_rmtr_stats& s)
      : H(h), P(p), S(s), st(h->st), L(h->L), F(h->dim + 1), mixed(p.precision == PF_FP32),
        gstate(h->L, G_NONE) {}

  // ---------------------------------------------------------------- helpers
  template <class Fn>
  void map(long long n, Fn f) {
    k_map<<<resident_grid(k_map<Fn>, n), 256, 0, st>>>(n, f);
    ck(cudaGetLastError(), "map");
    S.launches += 1;
  }

  template <class Fn>
  void map_skip(long long n, Fn f, const int* skip) {
    k_map_skip<<<map_grid(n), 256, 0, st>>>(n, f, skip);
    ck(cudaGetLastError(), "map_skip");
    S.launches += 1;
  }

  template <int K, class Op, class A = double, class Fn, class Fin>
  void red_fin(long long n, Fn f, Fin fin, const int* skip) {
    k_red_fin<K, Op, A><<<reduce_grid(n), 256, 0, st>>>(n, f, fin, H->scratch.partials,
                                                         H->scratch.counter, skip);
    ck(cudaGetLastError(), "red_fin");
    S.launches += 1;
  }

  template <int K, class Op, class A = double, class Fn>
  void reduce(long long n, Fn f, double* out) {
    k_red<K, Op, A><<<resident_grid(k_red<K, Op, A, Fn>, n), 256, 0, st>>>(
        n, f, H->scratch.partials, H->scratch.counter, H->d_res);
    ck(cudaGetLastError(), "reduce");
    S.launches += 1;
    fetch(K, out);
  }

  // reduce() without the read-back: results stay at out_dev
  template <int K, class Op, class A = double, class Fn>
  void reduce_dev(long long n, Fn f, double* out_dev) {
    k_red<K, Op, A><<<resident_grid(k_red<K, Op, A, Fn>, n), 256, 0, st>>>(
        n, f, H->scratch.partials, H->scratch.counter, out_dev);
    ck(cudaGetLastError(), "reduce");
    S.launches += 1;
  }

  void fetch(int K, double* out) {
    ck(cudaMemcpyAsync(H->h_res, H->d_res, sizeof(double) * K, cudaMemcpyDeviceToHost, st), "fetch");
    ck(cudaStreamSynchronize(st), "sync");
    for (int k = 0; k < K; ++k) out[k] = H->h_res[k];
  }

  long long nd(int l) const { return H->lv[l].n; }
  double frac(int l) const { return double(H->geo[l].N) / double(H->geo[L - 1].N); }

  template <class V>
  void copy(V* dst, const V* src, long long n) {
    ck(cudaMemcpyAsync(dst, src, sizeof(V) * n, cudaMemcpyDeviceToDevice, st), "copy");
  }
  template <class V>
  void zero(V* a, long long n) { ck(cudaMemsetAsync(a, 0, sizeof(V) * n, st), "zero"); }

  double dot(const double* a, const double* b, long long n) {
    double r;
    reduce<1, OpSum>(n, [=] __device__(long long i, double(&v)[1]) { v[0] = a[i] * b[i]; }, &r);
    return r;
  }

  // ---------------------------------------------------------------- element ops
  // Gradient and energy of f~ on level l: FP64, or double-float on the FP32
  // pipes in the mixed mode; elements evaluated once; the level's
  // coefficient buffer is free scratch outside the assembly in set_lag.
  bool use_df(int l) const { return mixed && df_scratch_fits(H->geo[l]); }
  void gradient(int l, const double* x, double* out) {
    if (use_df(l)) {
      ck(elem_gradient_df(H->geo[l], H->mat[l], x, out, H->lv[l].coef, st), "gradient_df");
      S.launches += 3;
    } else {
      ck(elem_gradient_fp64(H->geo[l], H->mat[l], x, out, H->lv[l].coef, st), "gradient");
      S.launches += 2;
    }
    S.fe_gradient += frac(l);
  }
  double ediff(int l, const double* x, const double* s) {
    ck(elem_energy_diff(H->geo[l], H->mat[l], x, s, 0, H->scratch, H->d_res, st), "ediff");
    S.fe_energy += frac(l);
    S.launches += 1;
    double a[4];
    fetch(4, a);
    return a[0] + a[1] + a[2] + a[3];
  }
  double energy(int l, const double* x) {
    if (use_df(l)) {
      ck(elem_energy_df(H->geo[l], H->mat[l], x, H->lv[l].coef, H->scratch, H->d_res, st),
         "energy_df");
      S.launches += 2;
    } else {
      ck(elem_energy(H->geo[l], H->mat[l], x, 0, H->scratch, H->d_res, st), "energy");
      S.launches += 1;
    }
    S.fe_energy += frac(l);
    double e;
    fetch(1, &e);
    return e;
  }

  void set_lag(int l, const double* x) {
    LevelBuf& B = H->lv[l];
    copy(B.xlag, x, B.n);
    if (mixed32(l)) {
      float* d = B.xlag32;
      const double* src = B.xlag;
      map(B.n, [=] __device__(long long i) { d[i] = float(src[i]); });
    }
    if (!mixed32(l)) {
      // FP64 Hessian of this level: Gauss-point coefficients, once per lag
      ck(ensure_stencil(H, l), "FP64 stencil allocation");
      ck(elem_hess_coef(H->geo[l], H->mat[l], B.xlag, B.coef, st), "hess_coef");
      ck(stencil_assemble(H->geo[l], H->mat[l], B.coef, B.stencil, st), "assemble");
      S.launches += 2;
      S.fe_gradient += frac(l);
    }
    if (P.precondition) {
      // Jacobi: inverse of the positive part of the lagged Hessian's diagonal
      // (the level's own Hessian at x0 for GALERKIN levels); FP32 on levels
      // whose subproblem runs on FP32 vectors (the diagonal goes through B.Hw,
      // free outside the subproblem)
      const bool m32 = mixed32(l);
      double* d = sub32(l) ? B.Hw : B.minv;
      if (gstored(l)) {
        // the stored Galerkin operator's own diagonal (its centre blocks)
        const float* gsv = B.gs;
        const long long N = H->geo[l].N;
        const int Fd = F, c = H->dim == 3 ? 13 : 4;
        map(B.n, [=] __device__(long long i) {
          const int f = int(i / N);
          const long long k = i - f * N;
          d[i] = double(gsv[((long long)(c * Fd + f) * Fd + f) * N + k]);
        });
      } else {
        ck(elem_hessdiag(H->geo[l], H->mat[l], m32 ? (const void*)B.xlag32 : (const void*)B.xlag,
                         m32 ? 1 : 0, d, st),
           "hessdiag");
        S.launches += 1;
      }
      if (sub32(l)) {
        float* mi = reinterpret_cast<float*>(B.minv);
        map(B.n, [=] __device__(long long i) {
          const double di = d[i];
          mi[i] = di > 0.0 ? float(1.0 / di) : 0.0f;
        });
      } else {
        double* mi = B.minv;
        map(B.n, [=] __device__(long long i) {
          const double di = mi[i];
          mi[i] = di > 0.0 ? 1.0 / di : 0.0;
        });
      }
    }
  }

  // ---------------------------------------------------------------- level model h^l
  bool finest(int l) const { return l == L - 1; }
  bool galerkin(int l) const { return !finest(l) && P.coarse_model == PF_GALERKIN; }
  // mixed precision: FP32 Hessian (and FP32 subproblem) on every level
  bool mixed32(int l) const { return mixed; }

  // GALERKIN levels of the mixed mode apply their model Hessian R G^{l+1} I
  // as a stored FP32 stencil built once per finest lag (galerkin_build)
  bool gstored(int l) const { return mixed && galerkin(l); }

  // finest-level units of one application of the lagged model Hessian
  double hlag_units(int l) const {
    return galerkin(l) && !gstored(l) ? hlag_units(l + 1) : frac(l);
  }

  // Lagged model Hessian: finest / FIRST_ORDER: Hessian at x_lag of the level;
  // GALERKIN: R H_{l+1} I.  With skip, a no-op once *skip is set; count
  // false leaves the work counters to the caller.
  void Hlag(int l, const double* v, double* out, const int* skip = nullptr, bool count = true) {
    if (gstored(l)) {
      ck(galerkin_apply(H->geo[l], H->lv[l].gs, v, out, PF_FP64, st, skip), "galerkin_apply");
      S.launches += 1;
      if (count) {
        S.hessvecs += 1;
        S.fe_hessvec += frac(l);
      }
      return;
    }
    if (!galerkin(l)) {
      LevelBuf& B = H->lv[l];
      if (mixed32(l))
        ck(elem_hessvec_mixed(H->geo[l], H->mat[l], B.xlag32, v, out, st, skip, H->etile_part,
                              H->p_dev),
           "hessvec32");
      else
        ck(stencil_apply(H->geo[l], B.stencil, v, out, st, skip), "hessvec");
      S.launches += mixed32(l) ? hessvec32_launches(H->geo[l], H->etile_part) : 1;
      if (count) {
        S.hessvecs += 1;
        S.fe_hessvec += frac(l);
      }
      return;
    }
    LevelBuf& F1 = H->lv[l + 1];
    ck(xfer_prolong(H->geo[l], H->geo[l + 1], F, v, F1.gin, 0, st, skip), "prolong");
    S.launches += 1;
    Hlag(l + 1, F1.gin, F1.gout, skip, count);
    ck(xfer_restrict(H->geo[l], H->geo[l + 1], F, F1.gout, out, 0, false, st, skip), "restrict");
    S.launches += 1;
  }

  // dH v = R H_{l+1} I v - Hess f~(x0) v  (GALERKIN); 0 otherwise.
  void dH(int l, const double* v, double* out) {
    LevelBuf& B = H->lv[l];
    Hlag(l, v, out);
    // the level's own Hessian at x0 (= its lag point): the assembled FP64
    // stencil, or in the mixed mode the FP32 matrix-free product at x0
    if (mixed32(l)) {
      ck(elem_hessvec_mixed(H->geo[l], H->mat[l], B.xlag32, v, B.dh, st, nullptr, H->etile_part,
                            H->p_dev),
         "hessvec32");
      S.launches += hessvec32_launches(H->geo[l], H->etile_part);
    } else {
      ck(stencil_apply(H->geo[l], B.stencil, v, B.dh, st), "hessvec");
      S.launches += 1;
    }
    S.hessvecs += 1;
    S.fe_hessvec += frac(l);
    const double* t = B.dh;
    map(B.n, [=] __device__(long long i) { out[i] -= t[i]; });
  }

  // grad h(x) = grad f~(x) + dg + dH (x - x0)
  void grad_h(int l, const double* x, double* out) {
    gradient(l, x, out);
    if (finest(l)) return;
    LevelBuf& B = H->lv[l];
    const double* dg = B.dg;
    if (!galerkin(l)) {
      map(B.n, [=] __device__(long long i) { out[i] += dg[i]; });
      return;
    }
    const double* x0 = B.x0;
    double* d = B.t3;
    map(B.n, [=] __device__(long long i) { d[i] = x[i] - x0[i]; });
    dH(l, d, B.gout == nullptr ? B.t2 : B.t2);
    const double* e = B.t2;
    map(B.n, [=] __device__(long long i) { out[i] += dg[i] + e[i]; });
  }

  // Levels whose gradient follows accepted steps by FP32 gradient steps
  // (mixed mode, FP32-Hessian levels whose model gradient differs from that
  // of f~ by a constant).  The exact FP64 gradient is still taken for every
  // stopping test and at every new coarse start.
  bool step_update(int l) const { return mixed32(l) && !galerkin(l); }

  // B.g := grad h(B.x)
  void grad_at(int l) {
    LevelBuf& B = H->lv[l];
    if (gstate[l] == G_STEP && step_update(l)) {
      // grad h(x) = grad h(x - s) + [grad f~(x) - grad f~(x - s)]
      ck(elem_gradient_step(H->geo[l], H->mat[l], B.x, B.s, B.g, st), "gradient_step");
      S.launches += 1;
      S.fe_gradient += frac(l);
    } else if (gstate[l] != G_AT_X) {
      grad_h(l, B.x, B.g);
    }
    gstate[l] = G_AT_X;
  }

  // h(x + s) - h(x) without subtracting totals; gx = grad h(x) (FP64).
  // h(x + t s) - h(x) is a quartic in t whose first-order coefficient is
  // gx . s, so the FP32-Hessian levels of the mixed mode take that term in
  // FP64 from gx and only the higher-order terms of f~ from an FP32 pass
  // (GALERKIN adds 1/2 s.dH s; dg and dH (x - x0) are inside gx).
  double diff_h(int l, const double* x, const double* s, const double* gx) {
    if (mixed32(l)) {
      LevelBuf& B = H->lv[l];
      ck(elem_energy_diff_hi(H->geo[l], H->mat[l], x, s, gx, H->scratch, H->d_res, st),
         "ediff_hi");
      S.fe_energy += frac(l);
      S.launches += 1;
      double a[4];
      fetch(4, a);
      double d = a[0] + a[1] + a[2] + a[3];
      if (galerkin(l)) {
        dH(l, s, B.t2);
        d += 0.5 * dot(s, B.t2, B.n);
      }
      return d;
    }
    double d = ediff(l, x, s);
    if (finest(l)) return d;
    LevelBuf& B = H->lv[l];
    d += dot(B.dg, s, B.n);
    if (!galerkin(l)) return d;
    const double* x0 = B.x0;
    double* t = B.t3;
    map(B.n, [=] __device__(long long i) { t[i] = x[i] - x0[i]; });
    dH(l, t, B.t2);
    d += dot(s, B.t2, B.n);
    dH(l, s, B.t2);
    d += 0.5 * dot(s, B.t2, B.n);
    return d;
  }

  // ---------------------------------------------------------------- subproblem
  // Levels whose subproblem runs on FP32 vectors: the FP32-Hessian levels of
  // the mixed mode (GALERKIN levels apply their operator through FP64
  // transfers and keep FP64 vectors).
  bool sub32(int l) const { return mixed32(l) && (!galerkin(l) || gstored(l)); }

  // The lagged model Hessian on vectors of precision V.
  template <class V>
  void hv(int l, const V* v, V* out, const int* skip = nullptr, bool count = true) {
    if constexpr (std::is_same<V, double>::value) {
      Hlag(l, v, out, skip, count);
    } else if (gstored(l)) {
      ck(galerkin_apply(H->geo[l], H->lv[l].gs, v, out, PF_FP32, st, skip), "galerkin_apply");
      S.launches += 1;
      if (count) {
        S.hessvecs += 1;
        S.fe_hessvec += frac(l);
      }
    } else {
      ck(elem_hessvec(H->geo[l], H->mat[l], H->lv[l].xlag32, v, out, 1, st, skip, H->etile_part,
                      H->p_dev),
         "hessvec32");
      S.launches += hessvec32_launches(H->geo[l], H->etile_part);
      if (count) {
        S.hessvecs += 1;
        S.fe_hessvec += frac(l);
      }
    }
  }

  // Vectors of one subproblem solve in precision V.  a and b hold the free
  // gaps lo - s < 0 < hi - s of the current s on its free set and 0 elsewhere,
  // so a[i] < 0 is the free-set test and w outside [a, b] leaves the box.
  template <class V>
  struct SubVecs {
    const V *g, *lo, *hi, *mi;
    V *s, *Hs, *r, *p, *q, *w, *a, *b, *t1, *t2;
  };

  // One projected-CG iteration on FP32 vectors with float4 passes (n a
  // multiple of 4) on stream s: q = H p, p.q and alpha (in the product's
  // gather pass where it has one), the update with its tests and beta, the
  // direction.  No-ops once the control block is done.  Returns the
  // launches.
  int cg_iter4(int l, const float* p, float* q, const float* ga, const float* gb,
               const float* mi, float* w, float* r, bool pc, cudaStream_t s) {
    LevelBuf& B = H->lv[l];
    CgCtrl* c = H->ctrl;
    const long long n4 = pad4(B.n) / 4;
    if (!gstored(l) && hessvec32_dot_fused(H->geo[l], H->etile_part)) {
      // the direction update of the previous iteration (beta = 0 after a
      // restart, where p = M^-1 r already) is formed inside the product
      ck(elem_hessvec32_dot(H->geo[l], H->mat[l], B.xlag32, const_cast<float*>(p), q, c,
                            H->scratch.partials, H->scratch.counter, H->etile_part, H->p_dev,
                            CgDirIn{r, pc ? mi : nullptr}, s),
         "hessvec32_dot");
      k_cg_update4<<<resident_grid(k_cg_update4, n4), 256, 0, s>>>(
          n4, ga, gb, q, p, mi, pc, w, r, c, H->scratch.partials, H->scratch.counter);
      ck(cudaGetLastError(), "cg_update");
      return 3;
    }
    int launches = 2;
    {
      if (gstored(l)) {
        ck(galerkin_apply(H->geo[l], B.gs, p, q, PF_FP32, s, &c->done), "galerkin_apply");
      } else {
        ck(elem_hessvec(H->geo[l], H->mat[l], B.xlag32, p, q, 1, s, &c->done, H->etile_part,
                        H->p_dev),
           "hessvec32");
      }
      k_cg_dot4<<<resident_grid(k_cg_dot4, n4), 256, 0, s>>>(n4, p, q, c, H->scratch.partials,
                                                              H->scratch.counter);
      ck(cudaGetLastError(), "cg_dot");
      launches += 1 + (gstored(l) ? 1 : hessvec32_launches(H->geo[l], H->etile_part));
    }
    k_cg_update4<<<resident_grid(k_cg_update4, n4), 256, 0, s>>>(
        n4, ga, gb, q, p, mi, pc, w, r, c, H->scratch.partials, H->scratch.counter);
    ck(cudaGetLastError(), "cg_update");
    k_cg_dir4<<<resident_grid(k_cg_dir4, n4), 256, 0, s>>>(n4, ga, r, mi, pc, const_cast<float*>(p),
                                                            c);
    ck(cudaGetLastError(), "cg_dir");
    return launches;
  }

  // One projected-CG iteration on level l on the solver's stream: q = H p,
  // p.q and alpha, the update with its tests and beta, the direction.
  // Launches after the control block is done are no-ops.
  template <class V>
  void cg_iter(int l, V* p, V* q, const V* ga, const V* gb, const V* mi, V* w, V* r, bool pc) {
    const long long n = H->lv[l].n;
    CgCtrl* c = H->ctrl;
    const int* skip = &H->ctrl->done;
    const V Z = V(0);
    if constexpr (std::is_same<V, float>::value) {
      S.launches += cg_iter4(l, p, q, ga, gb, mi, w, r, pc, st);
      return;
    }
    hv<V>(l, p, q, skip, false);
    red_fin<1, OpSum, V>(n, [=] __device__(long long i, V(&o)[1]) { o[0] = p[i] * q[i]; },
                         [=] __device__(double(&a)[1]) { cg_take_curvature(c, a[0]); }, skip);
    red_fin<3, OpSum, V>(n, [=] __device__(long long i, V(&o)[3]) {
      const V al = V(c->alpha);
      const V a = ga[i];
      const V qi = a < Z ? q[i] : Z;
      const V wi = w[i] + al * p[i];
      w[i] = wi;
      const V ri = r[i] - al * qi;
      r[i] = ri;
      o[0] = ri * ri;
      o[1] = (wi < a || wi > gb[i]) ? V(1) : Z;
      o[2] = ri * (pc ? mi[i] * ri : ri);
    }, [=] __device__(double(&a)[3]) {
      if (a[1] > 0.0) {
        c->done = 1;
        c->state = CG_LEAVE;
      } else if (sqrt(a[0]) <= c->tol) {
        c->done = 1;
        c->state = CG_CONV;
      } else if (c->used >= c->cg_max) {
        c->done = 1;
        c->state = CG_BUDGET;
      } else {
        c->beta = a[2] / c->rz;
        c->rr = a[0];
        c->rz = a[2];
      }
    }, skip);
    map_skip(n, [=] __device__(long long i) {
      p[i] = (pc ? mi[i] * r[i] : r[i]) + V(c->beta) * p[i];
    }, skip);
  }

  // The CG loop of level l as an executable graph: a while node whose body
  // is cg_iter and k_cg_cond.  Built on first use and rebuilt when the
  // pressure (a kernel argument of the FP32 Hessian) or the preconditioning
  // flag changes; a level's subproblem vectors sit at fixed addresses.  Null where the CUDA driver cannot build it (the caller then
  // drives the loop from the host).
  template <class V>
  cudaGraphExec_t cg_graph(int l, V* p, V* q, const V* ga, const V* gb, const V* mi, V* w, V* r,
                           bool pc) {
    if (!H->cg_graph_ok) return nullptr;
    if ((int)H->cg_graphs.size() < L) H->cg_graphs.resize(L);
    pf_hierarchy::CgGraph& G = H->cg_graphs[l];
    // 3D products read the pressure from the device; 2D ones take it as an
    // argument, so a 2D graph is rebuilt when it changes
    const bool p_ok = H->dim == 3 || G.p == H->p;
    if (G.exec && p_ok && G.pc == (pc ? 1 : 0) && G.vsize == int(sizeof(V)) &&
        G.precision == P.precision && G.coarse_model == P.coarse_model && G.vp == p)
      return G.exec;
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G = pf_hierarchy::CgGraph{};
    cudaGraph_t g = nullptr;
    cudaStream_t cs = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    cudaGraphConditionalHandle h{};
    cudaGraph_t body = nullptr;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
      if (ok) body = cp.conditional.phGraph_out[0];
    }
    // occupancy queries of the captured launches happen before the capture
    resident_grid(k_cg_dot4, 1);
    resident_grid(k_cg_update4, 1);
    resident_grid(k_cg_dir4, 1);
    if (ok) ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      bool launched = true;
      const cudaStream_t saved = st;
      const long long saved_launches = S.launches;
      st = cs;  // cg_iter launches on st
      try {
        cg_iter<V>(l, p, q, ga, gb, mi, w, r, pc);
        k_cg_cond<<<1, 1, 0, cs>>>(H->ctrl, h);
        launched = cudaGetLastError() == cudaSuccess;
      } catch (const CudaFail&) {
        launched = false;
      }
      st = saved;
      G.nodes = int(S.launches - saved_launches) + 1;  // + the condition kernel
      S.launches = saved_launches;
      cudaGraph_t out = nullptr;
      ok = cudaStreamEndCapture(cs, &out) == cudaSuccess && launched;
    }
    if (cs) cudaStreamDestroy(cs);
    cudaGraphExec_t ex = nullptr;
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();  // clear a non-sticky error of the failed build
      if (g) cudaGraphDestroy(g);
      H->cg_graph_ok = false;
      return nullptr;
    }
    const int nodes = G.nodes;
    G.graph = g;
    G.exec = ex;
    G.nodes = nodes;
    G.p = H->p;
    G.pc = pc ? 1 : 0;
    G.vsize = int(sizeof(V));
    G.precision = P.precision;
    G.coarse_model = P.coarse_model;
    G.vp = p;
    return ex;
  }

  // ---------------------------------------------------------------- the paper's QP solvers
  // (Sec. 4.2.2) on the level's FP64 stencil: symmetric multicolour
  // projected Gauss-Seidel and MPRGP.  g, lo, hi and s are level vectors.
  void pgs_solve(int l, const double* g, const double* lo, const double* hi, double* s, int sweeps) {
    const double* Sx = H->lv[l].stencil;
    for (int k = 0; k < sweeps; ++k) {
      ck(pgs_sweep(H->geo[l], Sx, g, lo, hi, s, false, st), "pgs");
      ck(pgs_sweep(H->geo[l], Sx, g, lo, hi, s, true, st), "pgs");
      S.launches += 2 << H->dim;
    }
  }

  // MPRGP from s = 0 on the diagonally scaled problem y = D^(1/2) s; the
  // expansion step 1 / (Gershgorin bound of D^(-1/2) H D^(-1/2)).  tol < 0:
  // the forcing tolerance min(0.1, sqrt(|nu0|)) |nu0| of the initial
  // projected gradient nu0.  Returns the products used.  Uses B.s (y),
  // B.Hs (gradient), B.p, B.q (A p), B.r, B.t1 (scale), B.t2, B.w, B.Hw
  // (scaled bounds).
  int mprgp_solve(int l, const double* g, const double* lo, const double* hi, double* out,
                  double tol, int maxit) {
    LevelBuf& B = H->lv[l];
    const long long n = B.n;
    const Geom geo = H->geo[l];
    const int Fd = F;
    const double* Sx = B.stencil;
    double *y = B.s, *gr = B.Hs, *p = B.p, *Ap = B.q, *d = B.r, *sq = B.t1, *tmp = B.t2;
    double *lw = B.w, *up = B.Hw;
    const long long N = geo.N;
    const int center = H->dim == 3 ? 13 : 4;
    map(n, [=] __device__(long long i) {
      const int f = int(i / N);
      const long long node = i - f * N;
      const double dd = Sx[((long long)(center * Fd + f) * Fd + f) * N + node];
      const double q = dd > 0.0 ? sqrt(dd) : 1.0;
      sq[i] = q;
      lw[i] = lo[i] * q;
      up[i] = hi[i] * q;
      y[i] = 0.0;
      gr[i] = g[i] / q;  // A 0 - b, b = -D^(-1/2) g
    });
    ck(scaled_rowsum(geo, Sx, tmp, st), "rowsum");
    S.launches += 1;
    double lam;
    reduce<1, OpMax>(n, [=] __device__(long long i, double(&v)[1]) { v[0] = tmp[i]; }, &lam);
    const double abar = 1.0 / lam;
    auto A = [&](const double* v, double* out_) {
      map(n, [=] __device__(long long i) { tmp[i] = v[i] / sq[i]; });
      ck(stencil_apply(geo, Sx, tmp, out_, st), "hessvec");
      map(n, [=] __device__(long long i) { out_[i] /= sq[i]; });
      S.launches += 1;
      S.hessvecs += 1;
      S.fe_hessvec += frac(l);
    };
    // free / chopped / reduced free gradient of element i
    auto phi_of = [=] __device__(long long i) {
      const double yi = y[i];
      return (lw[i] < yi && yi < up[i]) ? gr[i] : 0.0;
    };
    auto beta_of = [=] __device__(long long i) {
      const double yi = y[i], li = lw[i], ui = up[i], gi = gr[i];
      if (li < yi && yi < ui) return 0.0;
      if (!(li < ui)) return 0.0;
      return yi <= li ? fmin(gi, 0.0) : fmax(gi, 0.0);
    };
    auto set_p_phi = [&]() { map(n, [=] __device__(long long i) { p[i] = phi_of(i); }); };
    set_p_phi();
    int used = 1;
    double nrm0 = -1.0;
    while (true) {
      double r3[3];
      reduce<3, OpSum>(n, [=] __device__(long long i, double(&v)[3]) {
        const double ph = phi_of(i), be = beta_of(i);
        const double yi = y[i];
        double pt = 0.0;
        if (lw[i] < yi && yi < up[i])
          pt = ph > 0.0 ? fmin((yi - lw[i]) / abar, ph) : fmax((yi - up[i]) / abar, ph);
        v[0] = (ph + be) * (ph + be);
        v[1] = be * be;
        v[2] = pt * ph;
      }, r3);
      const double nrm = std::sqrt(r3[0]);
      if (nrm0 < 0.0) {
        nrm0 = nrm;
        if (tol < 0.0) tol = std::min(0.1, std::sqrt(nrm0)) * nrm0;
      }
      if (!(nrm > tol) || used >= maxit) break;
      if (r3[1] <= r3[2]) {  // proportional (Gamma = 1)
        A(p, Ap);
        ++used;
        double r2[2];
        reduce<2, OpSum>(n, [=] __device__(long long i, double(&v)[2]) {
          v[0] = p[i] * Ap[i];
          v[1] = gr[i] * p[i];
        }, r2);
        if (!(r2[0] > 0.0)) break;
        const double acg = r2[1] / r2[0];
        double af;
        reduce<1, OpMin>(n, [=] __device__(long long i, double(&v)[1]) {
          const double pi = p[i];
          v[0] = pi > 0.0 ? (y[i] - lw[i]) / pi : (pi < 0.0 ? (y[i] - up[i]) / pi : INFINITY);
        }, &af);
        if (acg <= af) {
          map(n, [=] __device__(long long i) {
            y[i] -= acg * p[i];
            gr[i] -= acg * Ap[i];
          });
          double ga;
          reduce<1, OpSum>(n, [=] __device__(long long i, double(&v)[1]) { v[0] = phi_of(i) * Ap[i]; }, &ga);
          const double gam = ga / r2[0];
          map(n, [=] __device__(long long i) { p[i] = phi_of(i) - gam * p[i]; });
        } else {
          map(n, [=] __device__(long long i) {
            y[i] -= af * p[i];
            gr[i] -= af * Ap[i];
          });
          map(n, [=] __device__(long long i) { d[i] = phi_of(i); });
          map(n, [=] __device__(long long i) { y[i] = fmin(fmax(y[i] - abar * d[i], lw[i]), up[i]); });
          A(y, gr);
          ++used;
          const double* gg = g;
          map(n, [=] __device__(long long i) { gr[i] += gg[i] / sq[i]; });
          set_p_phi();
        }
      } else {  // proportioning along the chopped gradient
        map(n, [=] __device__(long long i) { d[i] = beta_of(i); });
        A(d, Ap);
        ++used;
        double r2[2];
        reduce<2, OpSum>(n, [=] __device__(long long i, double(&v)[2]) {
          v[0] = d[i] * Ap[i];
          v[1] = gr[i] * d[i];
        }, r2);
        if (!(r2[0] > 0.0)) break;
        const double a = r2[1] / r2[0];
        map(n, [=] __device__(long long i) {
          y[i] -= a * d[i];
          gr[i] -= a * Ap[i];
        });
        set_p_phi();
      }
    }
    map(n, [=] __device__(long long i) { out[i] = y[i] / sq[i]; });
    return used;
  }

  // The TR subproblem with the paper's QP solvers: MPRGP on the coarsest
  // level (cg_max products), pgs_sweeps symmetric PGS sweeps elsewhere.
  void paper_subproblem(int l, int cg_max) {
    LevelBuf& B = H->lv[l];
    if (l == 0) {
      // MPRGP leaves its result in B.s, the step
      const int used = mprgp_solve(l, B.g, B.lo, B.hi, B.s, -1.0, cg_max);
      S.cg += used;
      S.cg_level[0] += used;
      return;
    }
    zero(B.s, B.n);
    pgs_solve(l, B.g, B.lo, B.hi, B.s, P.pgs_sweeps);
    S.cg_level[std::min(l, 7)] += P.pgs_sweeps;
    S.hessvecs += 2 * P.pgs_sweeps;
    S.fe_hessvec += 2.0 * P.pgs_sweeps * frac(l);
  }

  // Projected-search truncated CG for min g.s + 1/2 s.Hs over lo <= s <= hi
  // (eq. model_qp); the step is left in B.s (FP64).  On sub32 levels the
  // solve runs on FP32 copies of g and of the box, rounded towards zero so
  // that the FP32 box lies inside the FP64 one, in FP32 halves of the FP64
  // work buffers.  Uses B.s, B.Hs, B.r, B.p, B.q, B.w, B.Hw, B.t1, B.t2, B.t3.
  void subproblem(int l, double delta, int cg_max) {
    LevelBuf& B = H->lv[l];
    const long long n = B.n;
    if (P.qp_solver == PF_QP_PAPER) {
      paper_subproblem(l, cg_max);
      return;
    }
    if (!sub32(l)) {
      subproblem_t<double>(l, delta, cg_max,
                           {B.g, B.lo, B.hi, B.minv, B.s, B.Hs, B.r, B.p, B.q, B.w, B.Hw, B.t3,
                            B.t1, B.t2});
      return;
    }
    // two FP32 vectors per FP64 buffer, each on a 16-byte boundary (stride
    // pad4(n); the buffers carry 4 spare doubles for it)
    const long long np = pad4(n);
    auto half = [np](double* d, int k) { return reinterpret_cast<float*>(d) + k * np; };
    float *g32 = half(B.t3, 0), *lo32 = half(B.t3, 1), *hi32 = half(B.Hw, 0);
    {
      const double *g = B.g, *lo = B.lo, *hi = B.hi;
      map(n, [=] __device__(long long i) {
        g32[i] = __double2float_rn(g[i]);
        lo32[i] = __double2float_ru(lo[i]);  // lo <= 0 <= hi
        hi32[i] = __double2float_rd(hi[i]);
      });
    }
    const SubVecs<float> v{g32, lo32, hi32, reinterpret_cast<const float*>(B.minv),
                           half(B.Hw, 1), half(B.Hs, 0), half(B.Hs, 1), half(B.p, 0),
                           half(B.p, 1), half(B.w, 0), half(B.w, 1), half(B.r, 0),
                           half(B.r, 1), half(B.q, 0)};
    if (np != n) {
      // lanes n .. np-1 of every view: 0, so that they act as fixed dofs
      // (zero gaps) in the float4 passes and no stale value meets a 0
      PadLanes z{{g32, lo32, hi32, reinterpret_cast<float*>(B.minv), v.s, v.Hs, v.r, v.p, v.q, v.w,
                  v.a, v.b, v.t1, v.t2},
                 14, n, np};
      k_zero_pad<<<1, 64, 0, st>>>(z);
      ck(cudaGetLastError(), "zero_pad");
      S.launches += 1;
    }
    subproblem_t<float>(l, delta, cg_max, v);
    const float* s32 = v.s;
    double* s = B.s;
    map(n, [=] __device__(long long i) { s[i] = double(s32[i]); });
  }

  template <class V>
  void subproblem_t(int l, double delta, int cg_max, const SubVecs<V>& vec) {
    const long long n = H->lv[l].n;
    const V *g = vec.g, *lo = vec.lo, *hi = vec.hi, *mi = vec.mi;
    V *s = vec.s, *Hs = vec.Hs, *r = vec.r, *p = vec.p, *q = vec.q, *w = vec.w;
    V *ga = vec.a, *gb = vec.b, *t1 = vec.t1, *t2 = vec.t2;
    const V Z = V(0);
    double gmax;
    reduce<1, OpMax, V>(n, [=] __device__(long long i, V(&o)[1]) {
      const V gi = g[i];
      const bool mv = (gi < Z && hi[i] > Z) || (gi > Z && lo[i] < Z);
      o[0] = mv ? (gi < Z ? -gi : gi) : Z;
    }, &gmax);
    zero(s, n);
    if (!(gmax > 0.0)) return;
    double t = delta / gmax;
    // exact minimiser of the model along the movable part of -g
    map(n, [=] __device__(long long i) {
      const V gi = g[i];
      const bool mv = (gi < Z && hi[i] > Z) || (gi > Z && lo[i] < Z);
      t1[i] = mv ? gi : Z;
    });
    hv<V>(l, t1, t2);
    S.hv_cauchy += 1;
    double cg2[2];
    reduce<2, OpSum, V>(n, [=] __device__(long long i, V(&o)[2]) {
      o[0] = t1[i] * t2[i];
      o[1] = t1[i] * t1[i];
    }, cg2);
    if (cg2[0] > 0.0) t = std::min(t, cg2[1] / cg2[0]);
    bool ok = false;
    for (int bt = 0; bt <= P.cauchy_backtracks; ++bt) {
      const V tt = V(t);
      // s = P(-t g).  Where no movable dof is cut by its bound, s = -t t1
      // exactly, so Hs = -t H t1, g.s = -t t1.t1 and s.Hs = t^2 t1.Ht1 come
      // from the products above; the pass counts the cut dofs.
      double cut;
      reduce<1, OpSum, V>(n, [=] __device__(long long i, V(&o)[1]) {
        const V gi = g[i], di = -tt * gi;
        const V si = clampv(di, lo[i], hi[i]);
        s[i] = si;
        Hs[i] = -tt * t2[i];
        const bool mv = (gi < Z && hi[i] > Z) || (gi > Z && lo[i] < Z);
        o[0] = (mv && si != di) ? V(1) : Z;
      }, &cut);
      double a[2];
      if (cut == 0.0) {
        a[0] = -double(tt) * cg2[1];
        a[1] = double(tt) * double(tt) * cg2[0];
      } else {
        hv<V>(l, s, Hs);
        S.hv_cauchy += 1;
        reduce<2, OpSum, V>(n, [=] __device__(long long i, V(&o)[2]) {
          o[0] = g[i] * s[i];
          o[1] = s[i] * Hs[i];
        }, a);
      }
      if (a[0] + 0.5 * a[1] <= P.cauchy_c * a[0]) {
        ok = true;
        break;
      }
      t *= 0.5;
    }
    if (!ok) {
      zero(s, n);
      return;
    }
    int used = 0;
    int restarts = 0;
    double tol = -1.0;
    CgCtrl* c = H->ctrl;
    const int* skip = &H->ctrl->done;
    const bool pc = P.precondition != 0;
    while (used < cg_max) {
      double rr2[2];
      // residual of the model on the free set of s, its gaps, p = M^-1 r
      cudaGraphExec_t graph = cg_graph<V>(l, p, q, ga, gb, mi, w, r, pc);
      bool ran = false;
      if constexpr (std::is_same<V, float>::value) {
        const long long n4 = pad4(n) / 4;
        k_cg_init4<<<resident_grid(k_cg_init4, n4), 256, 0, st>>>(
            n4, lo, hi, s, g, Hs, mi, pc, r, p, w, ga, gb, H->scratch.partials, H->scratch.counter,
            H->d_res);
        ck(cudaGetLastError(), "cg_init");
        S.launches += 1;
        if (graph) {
          // start, run and stop on the device: one read-back per CG run
          k_ctrl_start_dev<<<1, 1, 0, st>>>(c, H->d_res, tol < 0.0 ? 1 : 0, used, cg_max);
          ck(cudaGetLastError(), "ctrl");
          ck(cudaGraphLaunch(graph, st), "cg_graph");
          ck(cudaMemcpyAsync(H->h_ctrl, c, sizeof(CgCtrl), cudaMemcpyDeviceToHost, st), "ctrl");
          ck(cudaStreamSynchronize(st), "sync");
          S.launches += 1 + (long long)H->cg_graphs[l].nodes * (H->h_ctrl->used - used);
          tol = H->h_ctrl->tol;
          ran = true;
        } else {
          fetch(2, rr2);
        }
      } else {
        reduce<2, OpSum, V>(n, [=] __device__(long long i, V(&o)[2]) {
          const V a = lo[i] - s[i], b = hi[i] - s[i];
          const bool fr = a < Z && Z < b;
          const V ri = fr ? -(g[i] + Hs[i]) : Z;
          const V zi = pc ? mi[i] * ri : ri;
          r[i] = ri;
          p[i] = zi;
          w[i] = Z;
          ga[i] = fr ? a : Z;
          gb[i] = fr ? b : Z;
          o[0] = ri * ri;
          o[1] = ri * zi;
        }, rr2);
      }
      if (!ran) {
        const double rr = rr2[0];
        if (tol < 0.0) {
          const double r0 = std::sqrt(rr);
          tol = std::min(0.1, std::sqrt(r0)) * r0;
        }
        if (std::sqrt(rr) <= tol || rr == 0.0) break;
      }
      // CG on the free set, driven on the device: each iteration is the
      // model Hessian, a reduction for p.Hp (its last block sets alpha or
      // flags non-positive curvature; p vanishes off the free set, so the
      // unmasked product is the masked one), an update reduction (its last
      // block tests the box, the forcing term and the budget and sets beta)
      // and the direction update.  The host polls the control block between
      // chunks of iterations; launches after a stop are no-ops.
      // the whole loop as one CUDA graph: a while node around one
      // iteration, repeated on the device until the control block stops the
      // run (no host polls); the host-polled loop below where no graph can
      // be built
      if (!ran) {
        k_ctrl_start<<<1, 1, 0, st>>>(c, rr2[0], rr2[1], tol, used, cg_max);
        ck(cudaGetLastError(), "ctrl");
        S.launches += 1;
        if (graph) {
          ck(cudaGraphLaunch(graph, st), "cg_graph");
          ck(cudaMemcpyAsync(H->h_ctrl, c, sizeof(CgCtrl), cudaMemcpyDeviceToHost, st), "ctrl");
          ck(cudaStreamSynchronize(st), "sync");
          S.launches += (long long)H->cg_graphs[l].nodes * (H->h_ctrl->used - used);
          ran = true;
        }
      }
      int chunk = 2;
      while (!ran) {
        for (int k = 0; k < chunk; ++k) cg_iter<V>(l, p, q, ga, gb, mi, w, r, pc);
        ck(cudaMemcpyAsync(H->h_ctrl, c, sizeof(CgCtrl), cudaMemcpyDeviceToHost, st), "ctrl");
        ck(cudaStreamSynchronize(st), "sync");
        if (H->h_ctrl->done) break;
        chunk = std::min(chunk * 2, 16);
      }
      const CgCtrl cs = *H->h_ctrl;
      const int its = cs.used - used;
      used = cs.used;
      S.cg += its;
      S.cg_level[std::min(l, 7)] += its;
      S.hessvecs += its;
      S.fe_hessvec += its * hlag_units(l);
      bool leave = cs.state == CG_LEAVE;
      if (cs.state == CG_NEGCURV) {
        // to the box along p
        double amax;
        reduce<1, OpMin, V>(n, [=] __device__(long long i, V(&o)[1]) {
          const V pi = p[i];
          V a = V(INFINITY);
          if (pi > Z) a = (gb[i] - w[i]) / pi;
          if (pi < Z) a = (ga[i] - w[i]) / pi;
          o[0] = a;
        }, &amax);
        amax = std::max(amax, 0.0);
        if (std::isfinite(amax)) {
          const V am = V(amax);
          map(n, [=] __device__(long long i) { w[i] += am * p[i]; });
        }
        leave = true;
      }
      if (!leave) {
        map(n, [=] __device__(long long i) { s[i] += w[i]; });
        break;
      }
      // projected search along w
      double ms[2];
      reduce<2, OpSum, V>(n, [=] __device__(long long i, V(&o)[2]) {
        o[0] = g[i] * s[i];
        o[1] = s[i] * Hs[i];
      }, ms);
      const double m_s = ms[0] + 0.5 * ms[1];
      double beta = 1.0;
      bool accepted = false;
      for (int bt = 0; bt <= P.cauchy_backtracks; ++bt) {
        const V bb = V(beta);
        map(n, [=] __device__(long long i) { t1[i] = clampv(s[i] + bb * w[i], lo[i], hi[i]); });
        hv<V>(l, t1, t2);
        S.hv_search += 1;
        double a[3];
        reduce<3, OpSum, V>(n, [=] __device__(long long i, V(&o)[3]) {
          o[0] = g[i] * t1[i];
          o[1] = t1[i] * t2[i];
          o[2] = (g[i] + Hs[i]) * (t1[i] - s[i]);
        }, a);
        if (a[0] + 0.5 * a[1] <= m_s + P.cauchy_c * a[2]) {
          accepted = true;
          break;
        }
        beta *= 0.5;
      }
      if (!accepted) break;
      copy(s, t1, n);
      copy(Hs, t2, n);
      S.cg_restarts += 1;
      if (++restarts > P.max_restarts) break;
    }
    map(n, [=] __device__(long long i) { s[i] = clampv(s[i], lo[i], hi[i]); });
  }

  // ---------------------------------------------------------------- TR method
  void tr_box(int l, const double* x, double delta) {
    LevelBuf& B = H->lv[l];
    const double *lb = B.lb, *ub = B.ub;
    double *lo = B.lo, *hi = B.hi;
    map(B.n, [=] __device__(long long i) {
      lo[i] = fmax(lb[i] - x[i], -delta);
      hi[i] = fmin(ub[i] - x[i], delta);
    });
  }

  void control(double rho, int l, double* x, double& delta) {
    LevelBuf& B = H->lv[l];
    if (rho > P.eta1) {
      const double *s = B.s, *lb = B.lb, *ub = B.ub;
      map(B.n, [=] __device__(long long i) { x[i] = fmin(fmax(x[i] + s[i], lb[i]), ub[i]); });
      gstate[l] = gstate[l] == G_AT_X ? G_STEP : G_NONE;
    }
    if (rho < P.eta1) delta = P.gamma1 * delta;
    else if (rho > P.eta2) delta = std::min(P.gamma2 * delta, P.delta_max);
  }

  // Algorithm 2 on level l, iterate in B.x, `iters` TR steps.
  void nonlinear_solve(int l, double& delta, int iters, int cg_max) {
    LevelBuf& B = H->lv[l];
    double chi0 = -1.0;
    for (int it = 0; it < iters; ++it) {
      grad_at(l);
      if (P.level_rtol > 0.0 && !finest(l)) {
        // stop once the level's projected gradient fell by level_rtol
        const double chi = pg_norm_level(l);
        if (chi0 < 0.0) chi0 = chi;
        else if (chi <= P.level_rtol * chi0) break;
      }
      tr_box(l, B.x, delta);
      subproblem(l, delta, cg_max);
      Hlag(l, B.s, B.t2);
      const double *g = B.g, *s = B.s, *hs = B.t2;
      auto pred_terms = [=] __device__(long long i, double(&v)[2]) {
        v[0] = g[i] * s[i];
        v[1] = s[i] * hs[i];
      };
      double pred, dh = 0.0;
      const bool merged = mixed32(l) && !galerkin(l);
      if (merged) {
        // the prediction's terms and the energy difference in one read-back
        reduce_dev<2, OpSum>(B.n, pred_terms, H->d_res + 4);
        ck(elem_energy_diff_hi(H->geo[l], H->mat[l], B.x, B.s, B.g, H->scratch, H->d_res, st),
           "ediff_hi");
        S.fe_energy += frac(l);
        S.launches += 1;
        double r6[6];
        fetch(6, r6);
        pred = -(r6[4] + 0.5 * r6[5]);
        dh = r6[0] + r6[1] + r6[2] + r6[3];
      } else {
        double a[2];
        reduce<2, OpSum>(B.n, pred_terms, a);
        pred = -(a[0] + 0.5 * a[1]);
      }
      S.tr_its += 1;
      S.tr_level[std::min(l, 7)] += 1;
      if (!(pred > 0.0)) break;
      const double rho = -(merged ? dh : diff_h(l, B.x, B.s, B.g)) / pred;
      if (rho <= P.eta1) {
        S.tr_rejected += 1;
        S.rej_level[std::min(l, 7)] += 1;
      }
      control(rho, l, B.x, delta);
    }
  }

  // Algorithm 1 on level l starting from B.x (B.xlag set by the caller).
  void vcycle(int l, double& delta) {
    LevelBuf& B = H->lv[l];
    const int cg = finest(l) ? P.cg_fine : P.cg_smooth;
    nonlinear_solve(l, delta, P.mu1, cg);
    if (l == 0) return;
    LevelBuf& C = H->lv[l - 1];
    const Geom &gc = H->geo[l - 1], &gf = H->geo[l];
    // fine correction bounds at x_mu1 -> coarse feasible set
    tr_box(l, B.x, delta);
    ck(xfer_bounds(gc, gf, F, B.lo, B.hi, C.lo, C.hi, st), "bounds");
    S.launches += 1;
    ck(xfer_restrict(gc, gf, F, B.x, C.x0, 0, true, st), "project");
    S.launches += 1;
    {
      const double *x0 = C.x0, *lo = C.lo, *hi = C.hi;
      double *lb = C.lb, *ub = C.ub, *xc = C.x;
      map(C.n, [=] __device__(long long i) {
        lb[i] = x0[i] + lo[i];
        ub[i] = x0[i] + hi[i];
        xc[i] = x0[i];
      });
    }
    // dg = R grad h^l(x_mu1) - grad f~(x0); g0 = R grad h^l(x_mu1) is the
    // coarse model's gradient at x0 (first-order coherence)
    grad_at(l);
    ck(xfer_restrict(gc, gf, F, B.g, C.g0, 0, false, st), "restrict");
    S.launches += 1;
    gradient(l - 1, C.x0, C.t1);
    {
      double* dg = C.dg;
      const double *t = C.t1, *g0 = C.g0;
      map(C.n, [=] __device__(long long i) { dg[i] = g0[i] - t[i]; });
    }
    set_lag(l - 1, C.x0);
    // the coarse iterate starts at x0, where grad h^{l-1} = g0
    copy(C.g, C.g0, C.n);
    gstate[l - 1] = G_AT_X;
    double dc = delta;
    if (l - 1 == 0) nonlinear_solve(0, dc, P.coarse_its, P.cg_coarse);
    else vcycle(l - 1, dc);
    // s = I (x* - x0), pred = h^{l-1}(x0) - h^{l-1}(x*)
    {
      const double* x0 = C.x0;
      const double* xs = C.x;
      double* d = C.t3;
      map(C.n, [=] __device__(long long i) { d[i] = xs[i] - x0[i]; });
    }
    // C.t3 holds the coarse correction; diff_h uses C.t2/C.t3 as scratch, so
    // keep a copy in C.w
    copy(C.w, C.t3, C.n);
    const double pred = -diff_h(l - 1, C.x0, C.w, C.g0);
    ck(xfer_prolong(gc, gf, F, C.w, B.s, 0, st), "prolong");
    S.launches += 1;
    if (pred > 0.0) {
      const double rho = -diff_h(l, B.x, B.s, B.g) / pred;
      if (rho <= P.eta1) S.coarse_rejected += 1;
      control(rho, l, B.x, delta);
    }
    nonlinear_solve(l, delta, P.mu2, cg);
  }

  // || x - P_F(x - g) || on level l for the level's current x and g
  double pg_norm_level(int l) {
    LevelBuf& B = H->lv[l];
    const double *x = B.x, *g = B.g, *lb = B.lb, *ub = B.ub;
    double r;
    reduce<1, OpSum>(B.n, [=] __device__(long long i, double(&v)[1]) {
      const double d = x[i] - fmin(fmax(x[i] - g[i], lb[i]), ub[i]);
      v[0] = d * d;
    }, &r);
    return std::sqrt(r);
  }

  double pg_norm(const double* x) {
    LevelBuf& B = H->lv[L - 1];
    gradient(L - 1, x, B.g);
    gstate[L - 1] = (x == B.x) ? G_AT_X : G_NONE;
    const double *g = B.g, *lb = B.lb, *ub = B.ub;
    double r;
    reduce<1, OpSum>(B.n, [=] __device__(long long i, double(&v)[1]) {
      const double d = x[i] - fmin(fmax(x[i] - g[i], lb[i]), ub[i]);
      v[0] = d * d;
    }, &r);
    return std::sqrt(r);
  }

  // projected gradient at x for the feasible set c(x) <= c <= 1, clamped u
  double pg_at(const double* x_user) {
    LevelBuf& B = H->lv[L - 1];
    const Geom g = H->geo[L - 1];
    const long long N = g.N;
    const int dim = H->dim;
    copy(B.t3, x_user, B.n);
    {
      double *lb = B.lb, *ub = B.ub;
      const double* x = B.t3;
      map(B.n, [=] __device__(long long i) {
        const int f = int(i / N);
        const long long k = i - f * N;
        double l, u;
        if (f == dim) {
          l = x[dim * N + k];
          u = 1.0;
        } else if (on_boundary(g, k)) {
          l = 0.0;
          u = 0.0;
        } else {
          l = -INFINITY;
          u = INFINITY;
        }
        lb[i] = l;
        ub[i] = u;
      });
    }
    return pg_norm(B.t3);
  }

  pf_status run(double* x_user) {
    LevelBuf& B = H->lv[L - 1];
    const Geom g = H->geo[L - 1];
    const long long N = g.N;
    const int dim = H->dim;
    double pg_ref = P.pg_ref;
    // a non-finite input is refused before anything is touched: x_user,
    // c_prev and the last converged pressure stay as they were
    {
      const double* xu = x_user;
      double bad_count;
      reduce<1, OpSum>(B.n, [=] __device__(long long i, double(&v)[1]) {
        v[0] = isfinite(xu[i]) ? 0.0 : 1.0;
      }, &bad_count);
      if (bad_count != 0.0) return PF_ENONFINITE;
    }
    // c_prev of the caller's last step, restored if this step fails
    copy(H->c_prev_save, H->c_prev, N);
    bool g_at_t3 = false;  // B.g holds the FP64 gradient at B.t3 = the plain start
    const double p_before = P.p_prev > 0.0 ? P.p_prev : H->p_last;
    copy(B.x, x_user, B.n);
    if (P.start == PF_START_EXTRAPOLATE && p_before > 0.0 && H->p != p_before) {
      // the displacement is nearly linear in p: start from u p / p_last, c
      // unchanged, and stop at the accuracy of the plain start
      if (!(pg_ref > 0.0)) {
        pg_ref = pg_at(x_user);  // B.g = grad f(x_{t-1}), B.t3 = x_{t-1}
        g_at_t3 = true;
      }
      const double r = H->p / p_before;
      double* xs = B.x;
      map((long long)dim * N, [=] __device__(long long i) { xs[i] *= r; });
    }
    // c_prev := c (unless kept from an accepted proposal); finest bounds of
    // eq. (space_pf), clamped displacement
    if (!P.keep_c_prev) copy(H->c_prev, B.x + dim * N, N);
    {
      double *lb = B.lb, *ub = B.ub, *x = B.x;
      const double* cp = H->c_prev;
      map(B.n, [=] __device__(long long i) {
        const int f = int(i / N);
        const long long k = i - f * N;
        double l, u;
        if (f == dim) {
          l = cp[k];
          u = 1.0;
        } else if (on_boundary(g, k)) {
          l = 0.0;
          u = 0.0;
        } else {
          l = -INFINITY;
          u = INFINITY;
        }
        lb[i] = l;
        ub[i] = u;
        x[i] = fmin(fmax(x[i], l), u);
      });
      H->bounds_set = true;
    }
    double pg0;
    if (g_at_t3 && step_update(L - 1)) {
      // the gradient at the extrapolated start by an FP32 gradient step from
      // the FP64 one at x_{t-1} (only u moved); the stopping tests of the
      // cycles evaluate the FP64 gradient again
      const double* x0 = B.t3;
      const double* x = B.x;
      double* sv = B.s;
      map(B.n, [=] __device__(long long i) { sv[i] = x[i] - x0[i]; });
      ck(elem_gradient_step(H->geo[L - 1], H->mat[L - 1], B.x, B.s, B.g, st), "gradient_step");
      S.launches += 1;
      S.fe_gradient += 1.0;
      gstate[L - 1] = G_AT_X;
      pg0 = pg_norm_level(L - 1);
    } else {
      pg0 = pg_norm(B.x);
    }
    if (!std::isfinite(pg0)) {
      copy(H->c_prev, H->c_prev_save, N);
      ck(cudaStreamSynchronize(st), "sync");
      return PF_ENONFINITE;
    }
    double pg = pg0;
    double delta = P.delta0;
    int cycles = 0;
    const double ref = pg_ref > 0.0 ? pg_ref : pg0;
    const double target = std::max(P.rtol * ref, P.atol);
    bool conv = pg0 <= (pg_ref > 0.0 ? target : P.atol);
    while (!conv && cycles < P.max_cycles) {
      set_lag(L - 1, B.x);
      if (L > 1 && mixed && P.coarse_model == PF_GALERKIN) {
        // the coarse model Hessians R G I of every level, from this lag
        ck(galerkin_build(H, B.xlag32, st), "galerkin_build");
        S.launches += 2 * (L - 1);
      }
      vcycle(L - 1, delta);
      ++cycles;
      pg = pg_norm(B.x);
      if (!std::isfinite(pg)) break;
      conv = pg <= target;
    }
    S.cycles = cycles;
    S.converged = conv ? 1 : 0;
    S.pg0 = pg0;
    S.pg = pg;
    S.pg_ref = ref;
    if (!std::isfinite(pg)) {
      // an aborted step leaves the caller's state as it was
      copy(H->c_prev, H->c_prev_save, N);
      ck(cudaStreamSynchronize(st), "sync");
      return PF_ENONFINITE;
    }
    S.energy = energy(L - 1, B.x);
    copy(x_user, B.x, B.n);
    ck(cudaStreamSynchronize(st), "sync");
    if (conv) H->p_last = H->p;
    return conv ? PF_OK : PF_ENOTCONV;
  }
};

pf_status projected_gradient_impl(pf_hierarchy* H, const double* x_dev, double* out) {
  pf_rmtr_stats S{};
  pf_rmtr_params P;
  pf_rmtr_params_default(&P);
  try {
    Solver solver(H, P, S);
    *out = solver.pg_at(x_dev);
  } catch (const CudaFail& f) {
    set_error(std::string("CUDA error in ") + f.where + ": " + cudaGetErrorString(f.e));
    return PF_ECUDA;
  }
  return std::isfinite(*out) ? PF_OK : PF_ENONFINITE;
}

pf_status qp_impl(pf_hierarchy* H, int level, const double* g, const double* lo, const double* hi,
                  double* s, int sweeps, double tol, int maxit, int* products) {
  pf_rmtr_stats S{};
  pf_rmtr_params P;
  pf_rmtr_params_default(&P);
  try {
    Solver solver(H, P, S);
    if (sweeps > 0) {
      solver.pgs_solve(level, g, lo, hi, s, sweeps);
      ck(cudaStreamSynchronize(H->st), "sync");
    } else {
      const int used = solver.mprgp_solve(level, g, lo, hi, s, tol, maxit);
      ck(cudaStreamSynchronize(H->st), "sync");
      if (products) *products = used;
    }
  } catch (const CudaFail& f) {
    set_error(std::string("CUDA error in ") + f.where + ": " + cudaGetErrorString(f.e));
    return PF_ECUDA;
  }
  return PF_OK;
}

pf_status rmtr_load_step_impl(pf_hierarchy* H, double* x_dev, const pf_rmtr_params& P,
                              pf_rmtr_stats* stats) {
  pf_rmtr_stats S{};
  const auto t0 = std::chrono::steady_clock::now();
  pf_status rc;
  try {
    Solver solver(H, P, S);
    rc = solver.run(x_dev);
  } catch (const CudaFail& f) {
    set_error(std::string("CUDA error in ") + f.where + ": " + cudaGetErrorString(f.e));
    return f.e == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA;
  }
  S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rc == PF_ENOTCONV) set_error("rmtr_load_step: max_cycles reached before the tolerance");
  if (rc == PF_ENONFINITE)
    set_error("rmtr_load_step: non-finite value in x or in the projected gradient (x and c_prev "
              "left unchanged)");
  if (stats) *stats = S;
  return rc;
}

}  // namespace pf
