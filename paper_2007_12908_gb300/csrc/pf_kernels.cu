// Element kernels (energy, quartic energy difference, gradient, Hessian-vector
// product), fracture rasterisation and grid transfers for sm_103a.
//
// Element loops are owner-computes: a CTA owns a tile of nodes, evaluates
// every element touching them (one halo layer on the low side) and sums the
// corner contributions in shared memory in 2^d colour phases (phase a adds
// corner a of every element; distinct elements hit distinct nodes within a
// phase).  Each owned node therefore receives its element contributions in
// a fixed order: results are bitwise reproducible, with no atomics.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdio>

#include "pf_df.cuh"
#include "pf_element_f2.cuh"
#include "pf_internal.h"
#include "pf_reduce.cuh"

namespace pf {

Geom make_geom(int dim, const int n[3], double h) {
  Geom g;
  g.dim = dim;
  g.N = 1;
  g.NE = 1;
  for (int k = 0; k < 3; ++k) {
    g.n[k] = k < dim ? n[k] : 1;
    g.ne[k] = k < dim ? n[k] - 1 : 1;
    g.N *= g.n[k];
    g.NE *= g.ne[k];
  }
  g.h = h;
  g.hv_variant = 0;
  return g;
}

Mat<double> make_mat(const Geom& g, double E, double nu, double Gc, double ls, double k,
                     double p) {
  Mat<double> m;
  m.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  m.mu = E / (2.0 * (1.0 + nu));
  m.Gc = Gc;
  m.ls = ls;
  m.k = k;
  m.p = p;
  m.inv_h = 1.0 / g.h;
  m.w = std::pow(g.h, g.dim) / double(1 << g.dim);
  return m;
}

template <class T>
static Mat<T> cast_mat(const Mat<double>& m) {
  Mat<T> r;
  r.lam = T(m.lam); r.mu = T(m.mu); r.Gc = T(m.Gc); r.ls = T(m.ls); r.k = T(m.k);
  r.p = T(m.p); r.inv_h = T(m.inv_h); r.w = T(m.w);
  return r;
}

// ------------------------------------------------------------ gathers
template <int D>
__device__ __forceinline__ long long corner_node(const Geom& g, int ex, int ey, int ez, int a) {
  const long long ix = ex + (a & 1), iy = ey + ((a >> 1) & 1);
  if constexpr (D == 3) {
    const long long iz = ez + ((a >> 2) & 1);
    return ix + g.n[0] * (iy + (long long)g.n[1] * iz);
  } else {
    return ix + g.n[0] * iy;
  }
}

template <int D, class T>
__device__ __forceinline__ void gather(const Geom& g, const T* __restrict__ x, int ex, int ey,
                                       int ez, T (*xe)[1 << D]) {
#pragma unroll
  for (int a = 0; a < (1 << D); ++a) {
    const long long idx = corner_node<D>(g, ex, ey, ez, a);
#pragma unroll
    for (int f = 0; f <= D; ++f) xe[f][a] = x[f * g.N + idx];
  }
}

template <int D>
__device__ __forceinline__ void elem_coords(const Geom& g, long long e, int& ex, int& ey, int& ez) {
  ex = int(e % g.ne[0]);
  const long long r = e / g.ne[0];
  if constexpr (D == 3) {
    ey = int(r % g.ne[1]);
    ez = int(r / g.ne[1]);
  } else {
    ey = int(r);
    ez = 0;
  }
}

// ------------------------------------------------------------ energy
template <int D, class T>
__global__ void __launch_bounds__(256) k_energy(Geom g, Mat<double> m, const T* __restrict__ x,
                                                double* partials, unsigned* counter, double* out) {
  double acc[1] = {0.0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.NE;
       e += (long long)gridDim.x * blockDim.x) {
    int ex, ey, ez;
    elem_coords<D>(g, e, ex, ey, ez);
    T xt[D + 1][1 << D];
    gather<D, T>(g, x, ex, ey, ez, xt);
    double xe[D + 1][1 << D];
#pragma unroll
    for (int f = 0; f <= D; ++f)
#pragma unroll
      for (int a = 0; a < (1 << D); ++a) xe[f][a] = double(xt[f][a]);
    acc[0] += elem_energy<D, double>(xe, m);
  }
  grid_finish<1, OpSum>(acc, partials, counter, out);
}

template <int D, class T>
__global__ void __launch_bounds__(256) k_energy_diff(Geom g, Mat<double> m,
                                                     const T* __restrict__ x,
                                                     const T* __restrict__ s, double* partials,
                                                     unsigned* counter, double* out) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.NE;
       e += (long long)gridDim.x * blockDim.x) {
    int ex, ey, ez;
    elem_coords<D>(g, e, ex, ey, ez);
    T xt[D + 1][1 << D], st[D + 1][1 << D];
    gather<D, T>(g, x, ex, ey, ez, xt);
    gather<D, T>(g, s, ex, ey, ez, st);
    double xe[D + 1][1 << D], se[D + 1][1 << D];
#pragma unroll
    for (int f = 0; f <= D; ++f)
#pragma unroll
      for (int a = 0; a < (1 << D); ++a) {
        xe[f][a] = double(xt[f][a]);
        se[f][a] = double(st[f][a]);
      }
    double a4[4];
    elem_energy_diff<D, double>(xe, se, m, a4);
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] += a4[k];
  }
  grid_finish<4, OpSum>(acc, partials, counter, out);
}

// Second- to fourth-order coefficients a2..a4 of E(x + t s) - E(x) from FP64
// x and s in FP32 arithmetic (each a sum of terms of order two and higher in
// s, free of the cancellation of energy totals), plus the FP64 dot product
// gx . s over the n dofs when gx is given (the first-order coefficient when
// gx is the gradient at x).  out = (gx . s, a2, a3, a4).
template <int D>
__global__ void __launch_bounds__(256) k_energy_diff_hi(Geom g, Mat<float> m,
                                                        const double* __restrict__ x,
                                                        const double* __restrict__ s,
                                                        const double* __restrict__ gx,
                                                        long long n, double* partials,
                                                        unsigned* counter, double* out) {
  float acc[3] = {0.f, 0.f, 0.f};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.NE;
       e += (long long)gridDim.x * blockDim.x) {
    int ex, ey, ez;
    elem_coords<D>(g, e, ex, ey, ez);
    double xt[D + 1][1 << D], st[D + 1][1 << D];
    gather<D, double>(g, x, ex, ey, ez, xt);
    gather<D, double>(g, s, ex, ey, ez, st);
    float xe[D + 1][1 << D], se[D + 1][1 << D];
#pragma unroll
    for (int f = 0; f <= D; ++f)
#pragma unroll
      for (int a = 0; a < (1 << D); ++a) {
        xe[f][a] = float(xt[f][a]);
        se[f][a] = float(st[f][a]);
      }
    float a4[4];
    elem_energy_diff<D, float>(xe, se, m, a4);
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] += a4[k + 1];
  }
  double d[4] = {0.0, double(acc[0]), double(acc[1]), double(acc[2])};
  if (gx)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
      d[0] += gx[i] * s[i];
  grid_finish<4, OpSum>(d, partials, counter, out);
}

// ------------------------------------------------------------ scatter ops
template <int D>
struct Tile;
template <>
struct Tile<3> {
  static constexpr int X = 8, Y = 8, Z = 8, THREADS = 256;
};
template <>
struct Tile<2> {
  static constexpr int X = 32, Y = 8, Z = 1, THREADS = 128;
};
// the other 2D node tiles the autotuner chooses from
struct Tile2_16x8 {
  static constexpr int X = 16, Y = 8, Z = 1, THREADS = 128;
};
struct Tile2_64x4 {
  static constexpr int X = 64, Y = 4, Z = 1, THREADS = 128;
};
struct Tile2_32x4 {
  static constexpr int X = 32, Y = 4, Z = 1, THREADS = 128;
};

// OP_GDIFF: y += grad E(x) - grad E(x - v), the gradient step from x - v to
// x in the arithmetic of TC (elem_gradient_diff at x with step -v).
enum { OP_GRAD = 0, OP_HESS = 1, OP_DIAG = 2, OP_GDIFF = 3 };

// Lagged Gauss-point coefficients of the Hessian, one element per thread;
// stored coef[(q * NCOEF + k) * NE + e] so that consecutive elements are
// consecutive in memory.
template <int D, class T>
__global__ void __launch_bounds__(256) k_hess_coef(Geom g, Mat<T> m, const T* __restrict__ x,
                                                   T* __restrict__ coef) {
  constexpr int NQ = 1 << D, NCF = NCoef<D>::value;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.NE;
       e += (long long)gridDim.x * blockDim.x) {
    int ex, ey, ez;
    elem_coords<D>(g, e, ex, ey, ez);
    T xe[D + 1][NQ];
    gather<D, T>(g, x, ex, ey, ez, xe);
    T cf[NQ][NCF];
    hess_coef<D, T>(xe, m, cf);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int k = 0; k < NCF; ++k) coef[(q * NCF + k) * g.NE + e] = cf[q][k];
  }
}

// TC: compute precision; TIO: precision of v and y; TM: precision of x in
// memory (converted to TC in registers).
// skip: when non-null and *skip != 0 the launch does nothing (the solver's
// device-side CG stops this way without a host round trip).
// FP32 instances are limited to 128 registers so that two CTAs (16 warps)
// share an SM and hide the gather and barrier latency.
template <int D, class TC, class TIO, int OP, class TM = TC, class TS = Tile<D>>
__global__ void __launch_bounds__(TS::THREADS, sizeof(TC) == 4 ? 2 : 1)
    k_elem_scatter(Geom g, Mat<TC> m, const TM* __restrict__ x, const TIO* __restrict__ v,
                   TIO* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int F = D + 1, NC = 1 << D;
  constexpr int TX = TS::X, TY = TS::Y, TZ = TS::Z;
  constexpr int EX = TX + 1, EY = TY + 1, EZ = D == 3 ? TZ + 1 : 1;
  constexpr int NEL = EX * EY * EZ, NOWN = TX * TY * TZ, NT = TS::THREADS;
  __shared__ TC acc[F][NOWN];
  const int ox = blockIdx.x * TX, oy = blockIdx.y * TY, oz = D == 3 ? blockIdx.z * TZ : 0;
  for (int i = threadIdx.x; i < F * NOWN; i += NT) (&acc[0][0])[i] = TC(0);
  __syncthreads();
  for (int base = 0; base < NEL; base += NT) {
    const int e = base + threadIdx.x;
    const int lx = e % EX - 1, ly = (e / EX) % EY - 1, lz = D == 3 ? e / (EX * EY) - 1 : 0;
    const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
    bool valid = e < NEL && gx >= 0 && gx < g.ne[0] && gy >= 0 && gy < g.ne[1];
    if constexpr (D == 3) valid = valid && gz >= 0 && gz < g.ne[2];
    TC out[F][NC];
    if (valid) {
      TC xe[F][NC];
      if constexpr (std::is_same<TM, TC>::value) {
        gather<D, TC>(g, x, gx, gy, gz, xe);
      } else {
        TM xt[F][NC];
        gather<D, TM>(g, x, gx, gy, gz, xt);
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
          for (int a = 0; a < NC; ++a) xe[f][a] = TC(xt[f][a]);
      }
      if constexpr (OP == OP_GDIFF) {
        TC se[F][NC];
#pragma unroll
        for (int a = 0; a < NC; ++a) {
          const long long idx = corner_node<D>(g, gx, gy, gz, a);
#pragma unroll
          for (int f = 0; f < F; ++f) se[f][a] = -TC(v[f * g.N + idx]);
        }
        elem_gradient_diff<D, TC>(xe, se, m, out);
      } else if constexpr (OP == OP_HESS) {
        TC ve[F][NC];
#pragma unroll
        for (int a = 0; a < NC; ++a) {
          const long long idx = corner_node<D>(g, gx, gy, gz, a);
#pragma unroll
          for (int f = 0; f < F; ++f) ve[f][a] = TC(v[f * g.N + idx]);
        }
        elem_hessvec<D, TC>(xe, ve, m, out);  // 3D FP32 products use k_hess_tile3
      } else if constexpr (OP == OP_DIAG) {
        elem_hessdiag<D, TC>(xe, m, out);
      } else {
        elem_gradient<D, TC>(xe, m, out);
      }
    }
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      const int nx = lx + (a & 1), ny = ly + ((a >> 1) & 1), nz = lz + ((a >> 2) & 1);
      bool own = valid && nx >= 0 && nx < TX && ny >= 0 && ny < TY;
      if constexpr (D == 3) own = own && nz >= 0 && nz < TZ;
      if (own) {
        const int li = nx + TX * (ny + TY * (D == 3 ? nz : 0));
#pragma unroll
        for (int f = 0; f < F; ++f) acc[f][li] += out[f][a];
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < NOWN; i += NT) {
    const int nx = i % TX, ny = (i / TX) % TY, nz = D == 3 ? i / (TX * TY) : 0;
    const int gx = ox + nx, gy = oy + ny, gz = oz + nz;
    if (gx < g.n[0] && gy < g.n[1] && gz < g.n[2]) {
      const long long idx = gx + g.n[0] * (gy + (long long)g.n[1] * gz);
#pragma unroll
      for (int f = 0; f < F; ++f) {
        if constexpr (OP == OP_GDIFF) y[f * g.N + idx] -= TIO(acc[f][i]);
        else y[f * g.N + idx] = TIO(acc[f][i]);
      }
    }
  }
}

// 3D FP32 Hessian product with the tile's inputs staged in shared memory.
// A CTA owns 8^3 nodes and evaluates the 9^3 elements touching them; their
// corners span the 10^3 nodes [o-1, o+8] per axis.  Those nodes' x_lag and v
// are loaded once per tile (coalesced along x, converted from TV) and kept
// as one float4 per node, so an element reads its 8 corners of each vector
// with 8 16-byte shared loads at fixed offsets, and the colour-phase sums
// add one float4 per node.  Same element algebra and the same fixed
// summation order as k_elem_scatter<3, float, ..., OP_HESS>.
// T: tile edge in nodes, 8 (128 threads, six element rounds, four CTAs per
// SM) or 4 (128 threads, one round) for grids too small to give every SM
// two 8^3 tiles.
template <int T>
struct HessTile {
  static constexpr int THREADS = 128;  // four CTAs per SM at 128 registers (8^3 tiles)
};

// OP: OP_HESS (y = H(x) v, paired FP32 algebra) or OP_GDIFF (y += grad E(x)
// - grad E(x - v), scalar FP32 algebra); TX: type of x in memory.
// p_dev: when non-null, the pressure is read from it (a CUDA graph that
// captured the launch then follows pf_pressure_set).
template <class TV, int T = 8, int OP = OP_HESS, class TX = float>
__global__ void __launch_bounds__(HessTile<T>::THREADS, 4)
    k_hess_tile3(Geom g, Mat<float> m, const TX* __restrict__ x, const TV* __restrict__ v,
                 TV* __restrict__ y, const int* __restrict__ skip,
                 const float* __restrict__ p_dev = nullptr) {
  if (skip && *skip) return;
  if (p_dev) m.p = *p_dev;
  constexpr int E = T + 1, NN = T + 2, NH = NN * NN * NN, NT = HessTile<T>::THREADS;
  __shared__ float4 xs[NH], vs[NH];
  __shared__ float4 acc[T * T * T];
  const int ox = blockIdx.x * T, oy = blockIdx.y * T, oz = blockIdx.z * T;
  const int nx0 = g.n[0], ny0 = g.n[1], nz0 = g.n[2];
  const long long N = g.N;
  for (int j = threadIdx.x; j < NH; j += NT) {
    const int i = j % NN, jj = (j / NN) % NN, k = j / (NN * NN);
    const int gx = ox - 1 + i, gy = oy - 1 + jj, gz = oz - 1 + k;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (gx >= 0 && gx < nx0 && gy >= 0 && gy < ny0 && gz >= 0 && gz < nz0) {
      const long long idx = gx + (long long)nx0 * (gy + (long long)ny0 * gz);
      a = make_float4(float(x[idx]), float(x[N + idx]), float(x[2 * N + idx]), float(x[3 * N + idx]));
      b = make_float4(float(v[idx]), float(v[N + idx]), float(v[2 * N + idx]), float(v[3 * N + idx]));
      if constexpr (OP == OP_GDIFF) b = make_float4(-b.x, -b.y, -b.z, -b.w);
    }
    xs[j] = a;
    vs[j] = b;
  }
  for (int i = threadIdx.x; i < T * T * T; i += NT) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  constexpr int NEL = E * E * E;
  for (int base = 0; base < NEL; base += NT) {
    const int e = base + threadIdx.x;
    const int lx = e % E - 1, ly = (e / E) % E - 1, lz = e / (E * E) - 1;
    const bool valid = e < NEL && ox + lx >= 0 && ox + lx < g.ne[0] && oy + ly >= 0 &&
                       oy + ly < g.ne[1] && oz + lz >= 0 && oz + lz < g.ne[2];
    float out[4][8];
    if (valid) {
      const int c0 = (lx + 1) + NN * ((ly + 1) + NN * (lz + 1));
      float xe[4][8], ve[4][8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int c = c0 + (a & 1) + NN * ((a >> 1) & 1) + NN * NN * ((a >> 2) & 1);
        const float4 xa = xs[c], va = vs[c];
        xe[0][a] = xa.x; xe[1][a] = xa.y; xe[2][a] = xa.z; xe[3][a] = xa.w;
        ve[0][a] = va.x; ve[1][a] = va.y; ve[2][a] = va.z; ve[3][a] = va.w;
      }
      if constexpr (OP == OP_GDIFF) elem_gradient_diff<3, float>(xe, ve, m, out);
      else p2::elem_hessvec(xe, ve, m, out);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int nx = lx + (a & 1), ny = ly + ((a >> 1) & 1), nz = lz + ((a >> 2) & 1);
      if (valid && nx >= 0 && nx < T && ny >= 0 && ny < T && nz >= 0 && nz < T) {
        const int li = nx + T * (ny + T * nz);
        float4 t = acc[li];
        t.x += out[0][a];
        t.y += out[1][a];
        t.z += out[2][a];
        t.w += out[3][a];
        acc[li] = t;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < T * T * T; i += NT) {
    const int nx = i % T, ny = (i / T) % T, nz = i / (T * T);
    const int gx = ox + nx, gy = oy + ny, gz = oz + nz;
    if (gx < nx0 && gy < ny0 && gz < nz0) {
      const long long idx = gx + (long long)nx0 * (gy + (long long)ny0 * gz);
      const float4 t = acc[i];
      if constexpr (OP == OP_GDIFF) {
        y[idx] -= TV(t.x);
        y[N + idx] -= TV(t.y);
        y[2 * N + idx] -= TV(t.z);
        y[3 * N + idx] -= TV(t.w);
      } else {
        y[idx] = TV(t.x);
        y[N + idx] = TV(t.y);
        y[2 * N + idx] = TV(t.z);
        y[3 * N + idx] = TV(t.w);
      }
    }
  }
}

template <int D, class TS = Tile<D>>
static dim3 scatter_grid(const Geom& g) {
  return dim3((g.n[0] + TS::X - 1) / TS::X, (g.n[1] + TS::Y - 1) / TS::Y,
              D == 3 ? (g.n[2] + TS::Z - 1) / TS::Z : 1);
}

template <int D, class TC, class TIO, int OP, class TM = TC, class TS = Tile<D>>
static cudaError_t launch_scatter(const Geom& g, const Mat<double>& m, const void* x,
                                  const void* v, void* y, const int* skip, cudaStream_t st) {
  k_elem_scatter<D, TC, TIO, OP, TM, TS><<<scatter_grid<D, TS>(g), TS::THREADS, 0, st>>>(
      g, cast_mat<TC>(m), static_cast<const TM*>(x), static_cast<const TIO*>(v),
      static_cast<TIO*>(y), skip);
  return cudaGetLastError();
}

// The 2D FP32 Hessian product on the node tile of the grid's variant.
static cudaError_t launch_hess2_f32(const Geom& g, const Mat<double>& m, const void* x,
                                   const void* v, void* y, const int* skip, cudaStream_t st) {
  switch (g.hv_variant) {
    case 1: return launch_scatter<2, float, float, OP_HESS, float, Tile2_16x8>(g, m, x, v, y, skip, st);
    case 2: return launch_scatter<2, float, float, OP_HESS, float, Tile2_64x4>(g, m, x, v, y, skip, st);
    case 3: return launch_scatter<2, float, float, OP_HESS, float, Tile2_32x4>(g, m, x, v, y, skip, st);
    case 4:
      return hess2_march(g, m, static_cast<const float*>(x), static_cast<const float*>(v),
                         static_cast<float*>(y), skip, st);
    default:
      // the default rule: marching strips on grids of at least 200,000
      // nodes (1.4x the node tiles at 1025^2), 32 x 8 node tiles below
      // (the strips' row-by-row march is latency-bound on small grids)
      if (g.N >= 200000)
        return hess2_march(g, m, static_cast<const float*>(x), static_cast<const float*>(v),
                           static_cast<float*>(y), skip, st);
      return launch_scatter<2, float, float, OP_HESS>(g, m, x, v, y, skip, st);
  }
}

cudaError_t elem_gradient_step(const Geom& g, const Mat<double>& m, const double* x,
                               const double* s, double* y, cudaStream_t st) {
  if (g.dim == 3) {
    const dim3 b8((g.n[0] + 7) / 8, (g.n[1] + 7) / 8, (g.n[2] + 7) / 8);
    k_hess_tile3<double, 8, OP_GDIFF, double><<<b8, HessTile<8>::THREADS, 0, st>>>(
        g, cast_mat<float>(m), x, s, y, nullptr);
    return cudaGetLastError();
  }
  return launch_scatter<2, float, double, OP_GDIFF, double>(g, m, x, s, y, nullptr, st);
}

cudaError_t elem_gradient(const Geom& g, const Mat<double>& m, const void* x, void* y, int prec,
                          cudaStream_t st) {
  if (g.dim == 3)
    return prec ? launch_scatter<3, float, float, OP_GRAD>(g, m, x, nullptr, y, nullptr, st)
                : launch_scatter<3, double, double, OP_GRAD>(g, m, x, nullptr, y, nullptr, st);
  return prec ? launch_scatter<2, float, float, OP_GRAD>(g, m, x, nullptr, y, nullptr, st)
              : launch_scatter<2, double, double, OP_GRAD>(g, m, x, nullptr, y, nullptr, st);
}

// Element-owned 3D FP32 Hessian product, pass 1: a CTA owns 8^3 elements
// and evaluates each once (no halo re-evaluation).  It stages their 9^3
// corner nodes of x_lag and v, sums the corner contributions into those
// nodes in the colour phases of k_hess_tile3, and writes the 9^3 node sums
// to part (one block of 729 float4 per tile).
// With dir.r set (FP32 CG), v is the previous direction and the staged
// operand is M^-1 r + beta v, beta = *beta.
constexpr int kEtileThreads = 128;  // 4 CTAs per SM at 128 registers
template <class TV>
__global__ void __launch_bounds__(kEtileThreads, 512 / kEtileThreads)
    k_hess_etile3(Geom g, Mat<float> m, const float* __restrict__ x, const TV* __restrict__ v,
                  float4* __restrict__ part, const int* __restrict__ skip,
                  const float* __restrict__ p_dev, CgDirIn dir, const double* beta) {
  if (skip && *skip) return;
  if (p_dev) m.p = *p_dev;
  const float be = dir.r ? float(*beta) : 0.f;
  constexpr int T = 8, NN = T + 1, NH = NN * NN * NN, NT = kEtileThreads;
  __shared__ float4 xs[NH], vs[NH], acc[NH];
  const int ox = blockIdx.x * T, oy = blockIdx.y * T, oz = blockIdx.z * T;
  const int nx0 = g.n[0], ny0 = g.n[1], nz0 = g.n[2];
  const long long N = g.N;
  for (int j = threadIdx.x; j < NH; j += NT) {
    const int i = j % NN, jj = (j / NN) % NN, k = j / (NN * NN);
    const int gx = ox + i, gy = oy + jj, gz = oz + k;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (gx < nx0 && gy < ny0 && gz < nz0) {
      const long long idx = gx + (long long)nx0 * (gy + (long long)ny0 * gz);
      a = make_float4(x[idx], x[N + idx], x[2 * N + idx], x[3 * N + idx]);
      b = make_float4(float(v[idx]), float(v[N + idx]), float(v[2 * N + idx]), float(v[3 * N + idx]));
      if (dir.r) {
        const float* r = dir.r;
        const float4 m4 = dir.mi ? make_float4(dir.mi[idx], dir.mi[N + idx], dir.mi[2 * N + idx],
                                               dir.mi[3 * N + idx])
                                 : make_float4(1.f, 1.f, 1.f, 1.f);
        b = make_float4(cg_direction(m4.x, r[idx], be, b.x),
                        cg_direction(m4.y, r[N + idx], be, b.y),
                        cg_direction(m4.z, r[2 * N + idx], be, b.z),
                        cg_direction(m4.w, r[3 * N + idx], be, b.w));
      }
    }
    xs[j] = a;
    vs[j] = b;
    acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  for (int base = 0; base < T * T * T; base += NT) {
    const int e = base + threadIdx.x;
    const int lx = e % T, ly = (e / T) % T, lz = e / (T * T);
    const bool valid = ox + lx < g.ne[0] && oy + ly < g.ne[1] && oz + lz < g.ne[2];
    const int c0 = lx + NN * (ly + NN * lz);
    float out[4][8];
    if (valid) {
      float xe[4][8], ve[4][8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int c = c0 + (a & 1) + NN * ((a >> 1) & 1) + NN * NN * ((a >> 2) & 1);
        const float4 xa = xs[c], va = vs[c];
        xe[0][a] = xa.x; xe[1][a] = xa.y; xe[2][a] = xa.z; xe[3][a] = xa.w;
        ve[0][a] = va.x; ve[1][a] = va.y; ve[2][a] = va.z; ve[3][a] = va.w;
      }
      p2::elem_hessvec(xe, ve, m, out);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      if (valid) {
        const int c = c0 + (a & 1) + NN * ((a >> 1) & 1) + NN * NN * ((a >> 2) & 1);
        float4 t = acc[c];
        t.x += out[0][a];
        t.y += out[1][a];
        t.z += out[2][a];
        t.w += out[3][a];
        acc[c] = t;
      }
      __syncthreads();
    }
  }
  const long long tile = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
  float4* o = part + tile * NH;
  for (int j = threadIdx.x; j < NH; j += NT) o[j] = acc[j];
}

// Sum at node n of the blocks of the up to 8 element tiles that contain
// it, in ascending tile order (z, y, x).  Along each axis a node lies in
// one tile, or in two where it sits on a tile boundary.  Only the tiles that
// hold the node are loaded and added; the loads of each z layer of
// candidates are issued together, so a node costs one memory latency (two
// on a z boundary), not one per tile.
__device__ __forceinline__ float4 etile_node_sum(const Geom& g, const float4* __restrict__ part,
                                                 long long n, int tx, int ty, int tz) {
  constexpr int T = 8, NN = T + 1, NH = NN * NN * NN;
  int i, j, k;
  if (g.N <= 0xffffffffLL) {  // 32-bit index arithmetic where it suffices
    unsigned u = unsigned(n);
    i = int(u % unsigned(g.n[0]));
    u /= unsigned(g.n[0]);
    j = int(u % unsigned(g.n[1]));
    k = int(u / unsigned(g.n[1]));
  } else {
    i = int(n % g.n[0]);
    const long long r = n / g.n[0];
    j = int(r % g.n[1]);
    k = int(r / g.n[1]);
  }
  // tiles t with 8t <= coordinate <= 8t + 8: t0, and t0 + 1 if present
  const int x0 = i >= T ? (i - 1) / T : 0, y0 = j >= T ? (j - 1) / T : 0;
  const int z0 = k >= T ? (k - 1) / T : 0;
  const bool hx = min(i / T, tx - 1) > x0, hy = min(j / T, ty - 1) > y0;
  const bool hz = min(k / T, tz - 1) > z0;
  // the node's entry in tile (x0, y0, z0); the next tile along an axis
  // holds it at a constant offset (one tile on, T nodes back)
  const long long base = (x0 + (long long)tx * (y0 + (long long)ty * z0)) * NH +
                         ((i - T * x0) + NN * ((j - T * y0) + NN * (k - T * z0)));
  const long long dX = NH - T, dY = (long long)tx * NH - T * NN;
  const long long dZ = (long long)tx * ty * NH - T * NN * NN;
  // candidates q = dx + 2 dy + 4 dz, added in q order; the loads of a z
  // layer (q = 0..3, then 4..7 where the node is on a z boundary) are all
  // issued before its first add
  float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    if (dz && !hz) break;
    const long long b = base + dz * dZ;
    float4 c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int dx = q & 1, dy = q >> 1;
      if ((!dx || hx) && (!dy || hy)) c[q] = part[b + dx * dX + dy * dY];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int dx = q & 1, dy = q >> 1;
      if (dz == 0 && q == 0) {
        sum = c[0];
      } else if ((!dx || hx) && (!dy || hy)) {
        sum.x += c[q].x;
        sum.y += c[q].y;
        sum.z += c[q].z;
        sum.w += c[q].w;
      }
    }
  }
  return sum;
}

// Pass 2: each node sums the blocks of the tiles that contain it and
// writes y.
template <class TV>
__global__ void __launch_bounds__(256) k_etile_gather3(Geom g, const float4* __restrict__ part,
                                                       TV* __restrict__ y,
                                                       const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int T = 8;
  const int tx = (g.ne[0] + T - 1) / T, ty = (g.ne[1] + T - 1) / T, tz = (g.ne[2] + T - 1) / T;
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const float4 sum = etile_node_sum(g, part, n, tx, ty, tz);
    y[n] = TV(sum.x);
    y[N + n] = TV(sum.y);
    y[2 * N + n] = TV(sum.z);
    y[3 * N + n] = TV(sum.w);
  }
}

// Pass 2 with p.q: as k_etile_gather3 for FP32 y = q, and each thread adds
// p.q over its nodes; the blocks' partials are combined in block order and
// the last block takes the CG curvature step.  Launched on at most
// kMaxBlocks blocks (one completion ticket per block).
// With dir.r set, p is first replaced by M^-1 r + beta p (the operand the
// element pass formed) and stored back.
__global__ void __launch_bounds__(256, 4) k_etile_gather3_dot(Geom g,
                                                              const float4* __restrict__ part,
                                                              float* __restrict__ p,
                                                              float* __restrict__ y, CgCtrl* c,
                                                              double* partials,
                                                              unsigned* counter, CgDirIn dir) {
  if (c->done) return;
  constexpr int T = 8;
  const int tx = (g.ne[0] + T - 1) / T, ty = (g.ne[1] + T - 1) / T, tz = (g.ne[2] + T - 1) / T;
  const long long N = g.N;
  const float be = dir.r ? float(c->beta) : 0.f;
  float pq = 0.f;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    float p0 = p[n], p1 = p[N + n], p2 = p[2 * N + n], p3 = p[3 * N + n];
    if (dir.r) {
      const float* r = dir.r;
      const float4 m4 = dir.mi ? make_float4(dir.mi[n], dir.mi[N + n], dir.mi[2 * N + n],
                                             dir.mi[3 * N + n])
                               : make_float4(1.f, 1.f, 1.f, 1.f);
      p0 = cg_direction(m4.x, r[n], be, p0);
      p1 = cg_direction(m4.y, r[N + n], be, p1);
      p2 = cg_direction(m4.z, r[2 * N + n], be, p2);
      p3 = cg_direction(m4.w, r[3 * N + n], be, p3);
      p[n] = p0;
      p[N + n] = p1;
      p[2 * N + n] = p2;
      p[3 * N + n] = p3;
    }
    const float4 sum = etile_node_sum(g, part, n, tx, ty, tz);
    y[n] = sum.x;
    y[N + n] = sum.y;
    y[2 * N + n] = sum.z;
    y[3 * N + n] = sum.w;
    pq += p0 * sum.x + p1 * sum.y + p2 * sum.z + p3 * sum.w;
  }
  double acc[1] = {double(pq)};
  auto fin = [c](double(&a)[1]) { cg_take_curvature(c, a[0]); };
  grid_finish_fn<1, OpSum>(acc, partials, counter, fin);
}

long long etile_part_count(const Geom& g) {
  if (g.dim != 3) return 0;
  const long long t = (long long)((g.ne[0] + 7) / 8) * ((g.ne[1] + 7) / 8) * ((g.ne[2] + 7) / 8);
  return t * 729;
}

static bool etile_eligible(const Geom& g) {
  const long long b8 = (long long)((g.n[0] + 7) / 8) * ((g.n[1] + 7) / 8) * ((g.n[2] + 7) / 8);
  return g.dim == 3 && b8 >= 2 * 152;
}

// Whether the 3D FP32 product runs on element-owned tiles: by the grid's
// variant (1 yes, 2 and 3 no), else by the default rule (at least two 8^3
// tiles per SM).
static bool etile_used(const Geom& g, const void* part) {
  if (g.dim != 3 || !part) return false;
  if (g.hv_variant) return g.hv_variant == 1;
  return etile_eligible(g);
}

int hessvec32_launches(const Geom& g, const void* part) { return etile_used(g, part) ? 2 : 1; }

bool hessvec32_dot_fused(const Geom& g, const void* part) { return etile_used(g, part); }

cudaError_t elem_hessvec32_dot(const Geom& g, const Mat<double>& m, const float* x, float* p,
                               float* q, CgCtrl* c, double* partials, unsigned* counter,
                               void* part, const float* p_dev, CgDirIn dir, cudaStream_t st) {
  if (!hessvec32_dot_fused(g, part)) return cudaErrorNotSupported;
  const dim3 be((g.ne[0] + 7) / 8, (g.ne[1] + 7) / 8, (g.ne[2] + 7) / 8);
  float4* pp = static_cast<float4*>(part);
  k_hess_etile3<float><<<be, kEtileThreads, 0, st>>>(g, cast_mat<float>(m), x, p, pp, &c->done, p_dev, dir,
                                           &c->beta);
  // kMaxBlocks = two waves of 4 blocks per SM
  const int nb = int(std::min<long long>((g.N + 255) / 256, kMaxBlocks));
  k_etile_gather3_dot<<<nb, 256, 0, st>>>(g, pp, p, q, c, partials, counter, dir);
  return cudaGetLastError();
}

template <class TV>
static cudaError_t launch_hess_tile3(const Geom& g, const Mat<double>& m, const float* x,
                                     const TV* v, TV* y, const int* skip, cudaStream_t st,
                                     void* part = nullptr, const float* p_dev = nullptr) {
  auto tiles = [&g](int t) {
    return dim3((g.n[0] + t - 1) / t, (g.n[1] + t - 1) / t, (g.n[2] + t - 1) / t);
  };
  if (etile_used(g, part)) {
    const dim3 be((g.ne[0] + 7) / 8, (g.ne[1] + 7) / 8, (g.ne[2] + 7) / 8);
    float4* pp = static_cast<float4*>(part);
    k_hess_etile3<TV><<<be, kEtileThreads, 0, st>>>(g, cast_mat<float>(m), x, v, pp, skip, p_dev,
                                          CgDirIn{nullptr, nullptr}, nullptr);
    const int nb = int(std::min<long long>((g.N + 255) / 256, 8LL * 1216));
    k_etile_gather3<TV><<<nb, 256, 0, st>>>(g, pp, y, skip);
    return cudaGetLastError();
  }
  const dim3 b8 = tiles(8);
  const bool t8 = g.hv_variant ? g.hv_variant != 3 : (long long)b8.x * b8.y * b8.z >= 2 * 152;
  if (t8)
    k_hess_tile3<TV, 8><<<b8, HessTile<8>::THREADS, 0, st>>>(g, cast_mat<float>(m), x, v, y, skip,
                                                              p_dev);
  else
    k_hess_tile3<TV, 4><<<tiles(4), HessTile<4>::THREADS, 0, st>>>(g, cast_mat<float>(m), x, v, y,
                                                                  skip, p_dev);
  return cudaGetLastError();
}

cudaError_t elem_hessvec(const Geom& g, const Mat<double>& m, const void* x, const void* v,
                         void* y, int prec, cudaStream_t st, const int* skip, void* part,
                         const float* p_dev) {
  if (g.dim == 3)
    return prec ? launch_hess_tile3<float>(g, m, static_cast<const float*>(x),
                                           static_cast<const float*>(v), static_cast<float*>(y),
                                           skip, st, part, p_dev)
                : launch_scatter<3, double, double, OP_HESS>(g, m, x, v, y, skip, st);
  return prec ? launch_hess2_f32(g, m, x, v, y, skip, st)
              : launch_scatter<2, double, double, OP_HESS>(g, m, x, v, y, skip, st);
}

cudaError_t elem_hess_coef(const Geom& g, const Mat<double>& m, const double* x, double* coef,
                           cudaStream_t st) {
  const int nb = int(std::min<long long>((g.NE + 255) / 256, 8LL * 1216));
  if (g.dim == 3)
    k_hess_coef<3, double><<<nb, 256, 0, st>>>(g, cast_mat<double>(m), x, coef);
  else
    k_hess_coef<2, double><<<nb, 256, 0, st>>>(g, cast_mat<double>(m), x, coef);
  return cudaGetLastError();
}

// ------------------------------------------------------------ FP64 gradient, two passes
// Element-parallel: every element is evaluated once (no halo) and writes its
// corner contributions to scratch[(f * 2^d + a) * NE + e]; then every node
// sums the contributions of its up to 2^d elements in corner order, so the
// result is deterministic.
template <int D>
__global__ void __launch_bounds__(128) k_grad_elem(Geom g, Mat<double> m, const double* __restrict__ x,
                                                   double* __restrict__ scratch) {
  constexpr int F = D + 1, NC = 1 << D;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.NE;
       e += (long long)gridDim.x * blockDim.x) {
    int ex, ey, ez;
    elem_coords<D>(g, e, ex, ey, ez);
    double xe[F][NC], out[F][NC];
    gather<D, double>(g, x, ex, ey, ez, xe);
    elem_gradient<D, double>(xe, m, out);
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int a = 0; a < NC; ++a) scratch[(f * NC + a) * g.NE + e] = out[f][a];
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_grad_gather(Geom g, const double* __restrict__ scratch,
                                                     double* __restrict__ y) {
  constexpr int F = D + 1, NC = 1 << D;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = int(i % g.n[0]);
    const long long r = i / g.n[0];
    const int iy = int(r % g.n[1]);
    const int iz = int(r / g.n[1]);
    const int ic[3] = {ix, iy, iz};
    double acc[F];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = 0.0;
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      int ec[3] = {0, 0, 0};
      bool ok = true;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        ec[k] = ic[k] - ((a >> k) & 1);
        ok = ok && ec[k] >= 0 && ec[k] < g.ne[k];
      }
      if (!ok) continue;
      const long long e = ec[0] + (long long)g.ne[0] * (ec[1] + (long long)g.ne[1] * ec[2]);
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f] += scratch[(f * NC + a) * g.NE + e];
    }
#pragma unroll
    for (int f = 0; f < F; ++f) y[f * g.N + i] = acc[f];
  }
}

cudaError_t elem_gradient_fp64(const Geom& g, const Mat<double>& m, const double* x, double* y,
                               double* scratch, cudaStream_t st) {
  const int nb = int(std::min<long long>((g.NE + 127) / 128, 32LL * 1216));
  const int nn = int(std::min<long long>((g.N + 255) / 256, 16LL * 1216));
  if (g.dim == 3) {
    k_grad_elem<3><<<nb, 128, 0, st>>>(g, m, x, scratch);
    k_grad_gather<3><<<nn, 256, 0, st>>>(g, scratch, y);
  } else {
    k_grad_elem<2><<<nb, 128, 0, st>>>(g, m, x, scratch);
    k_grad_gather<2><<<nn, 256, 0, st>>>(g, scratch, y);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------ double-float passes
// The gradient and the energy in double-float arithmetic (pf_df.cuh) on the
// FP32 pipes: x is split once per call into (hi, lo) planes, the element
// algebra is the FP64 code instantiated with df, and nodal sums and totals
// are formed in df (gradient) or FP64 (energy totals across threads).
__global__ void k_to_df(long long n, const double* __restrict__ x, float2* __restrict__ xd) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const df v = df_from(x[i]);
    xd[i] = make_float2(v.hi, v.lo);
  }
}

template <int D>
__device__ __forceinline__ void gather_df(const Geom& g, const float2* __restrict__ xd, int ex,
                                          int ey, int ez, df (*xe)[1 << D]) {
#pragma unroll
  for (int a = 0; a < (1 << D); ++a) {
    const long long idx = corner_node<D>(g, ex, ey, ez, a);
#pragma unroll
    for (int f = 0; f <= D; ++f) {
      const float2 v = xd[f * g.N + idx];
      xe[f][a] = df(v.x, v.y);
    }
  }
}

template <int D>
__global__ void __launch_bounds__(128) k_grad_elem_df(Geom g, Mat<df> m,
                                                      const float2* __restrict__ xd,
                                                      float2* __restrict__ scratch) {
  constexpr int F = D + 1, NC = 1 << D;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.NE;
       e += (long long)gridDim.x * blockDim.x) {
    int ex, ey, ez;
    elem_coords<D>(g, e, ex, ey, ez);
    df xe[F][NC], out[F][NC];
    gather_df<D>(g, xd, ex, ey, ez, xe);
    elem_gradient<D, df>(xe, m, out);
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int a = 0; a < NC; ++a)
        scratch[(f * NC + a) * g.NE + e] = make_float2(out[f][a].hi, out[f][a].lo);
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_grad_gather_df(Geom g, const float2* __restrict__ scratch,
                                                        double* __restrict__ y) {
  constexpr int F = D + 1, NC = 1 << D;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = int(i % g.n[0]);
    const long long r = i / g.n[0];
    const int iy = int(r % g.n[1]);
    const int iz = int(r / g.n[1]);
    const int ic[3] = {ix, iy, iz};
    df acc[F];
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      int ec[3] = {0, 0, 0};
      bool ok = true;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        ec[k] = ic[k] - ((a >> k) & 1);
        ok = ok && ec[k] >= 0 && ec[k] < g.ne[k];
      }
      if (!ok) continue;
      const long long e = ec[0] + (long long)g.ne[0] * (ec[1] + (long long)g.ne[1] * ec[2]);
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const float2 v = scratch[(f * NC + a) * g.NE + e];
        acc[f] = add_accurate(acc[f], df(v.x, v.y));
      }
    }
#pragma unroll
    for (int f = 0; f < F; ++f) y[f * g.N + i] = df_to_double(acc[f]);
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_energy_df(Geom g, Mat<df> m, const float2* __restrict__ xd,
                                                   double* partials, unsigned* counter,
                                                   double* out) {
  df part;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.NE;
       e += (long long)gridDim.x * blockDim.x) {
    int ex, ey, ez;
    elem_coords<D>(g, e, ex, ey, ez);
    df xe[D + 1][1 << D];
    gather_df<D>(g, xd, ex, ey, ez, xe);
    part = add_accurate(part, elem_energy<D, df>(xe, m));
  }
  double acc[1] = {df_to_double(part)};
  grid_finish<1, OpSum>(acc, partials, counter, out);
}

// Scratch of the double-float passes inside a buffer of `cap` doubles
// (a level's coefficient buffer): x in df, then the gradient's corner
// contributions.  False when the buffer is too small.
static bool df_layout(const Geom& g, long long cap, long long& off_contrib) {
  const long long n = (long long)(g.dim + 1) * g.N;
  const long long contrib = (long long)(g.dim + 1) * (1LL << g.dim) * g.NE;
  off_contrib = n;
  return n + contrib <= cap;
}

bool df_scratch_fits(const Geom& g) {
  long long off;
  return df_layout(g, coef_count(g), off);
}

cudaError_t elem_gradient_df(const Geom& g, const Mat<double>& m, const double* x, double* y,
                             double* scratch, cudaStream_t st) {
  long long off;
  if (!df_layout(g, coef_count(g), off)) return cudaErrorInvalidValue;
  float2* xd = reinterpret_cast<float2*>(scratch);
  float2* contrib = reinterpret_cast<float2*>(scratch) + off;
  const long long n = (long long)(g.dim + 1) * g.N;
  const int nv = int(std::min<long long>((n + 255) / 256, 16LL * 1216));
  const int nb = int(std::min<long long>((g.NE + 127) / 128, 32LL * 1216));
  const int nn = int(std::min<long long>((g.N + 255) / 256, 16LL * 1216));
  k_to_df<<<nv, 256, 0, st>>>(n, x, xd);
  if (g.dim == 3) {
    k_grad_elem_df<3><<<nb, 128, 0, st>>>(g, cast_mat<df>(m), xd, contrib);
    k_grad_gather_df<3><<<nn, 256, 0, st>>>(g, contrib, y);
  } else {
    k_grad_elem_df<2><<<nb, 128, 0, st>>>(g, cast_mat<df>(m), xd, contrib);
    k_grad_gather_df<2><<<nn, 256, 0, st>>>(g, contrib, y);
  }
  return cudaGetLastError();
}

cudaError_t elem_energy_df(const Geom& g, const Mat<double>& m, const double* x, double* scratch,
                           const Scratch& s, double* out, cudaStream_t st) {
  long long off;
  if (!df_layout(g, coef_count(g), off)) return cudaErrorInvalidValue;
  float2* xd = reinterpret_cast<float2*>(scratch);
  const long long n = (long long)(g.dim + 1) * g.N;
  const int nv = int(std::min<long long>((n + 255) / 256, 16LL * 1216));
  const int nb = reduce_grid(g.NE, 256);
  k_to_df<<<nv, 256, 0, st>>>(n, x, xd);
  if (g.dim == 3)
    k_energy_df<3><<<nb, 256, 0, st>>>(g, cast_mat<df>(m), xd, s.partials, s.counter, out);
  else
    k_energy_df<2><<<nb, 256, 0, st>>>(g, cast_mat<df>(m), xd, s.partials, s.counter, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------ assembled Hessian
// The lagged FP64 Hessian stored as a (3^d)-point block stencil: for node i,
// offset o (component k of the offset = o_k - 1 in {-1, 0, 1}) and fields
// f, g, the entry S[((o * F + f) * F + g) * N + i] couples dof (f, i) with
// dof (g, i + offset).  Assembled from the stored Gauss-point coefficients
// (A, M, B) of the up to 2^d elements around each node; each thread owns
// one node's row, so the sums need no atomics.
template <int D>
__device__ __forceinline__ void shape_tables(int a, int q, double& na, double (&da)[D]) {
  double n1[D];
#pragma unroll
  for (int k = 0; k < D; ++k) n1[k] = (((q >> k) & 1) == ((a >> k) & 1)) ? PF_XI1 : PF_XI0;
  na = 1.0;
#pragma unroll
  for (int k = 0; k < D; ++k) na *= n1[k];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double t = ((a >> k) & 1) ? 1.0 : -1.0;  // raw derivative of the 1D factor
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (j != k) t *= n1[j];
    da[k] = t;
  }
}

// One thread per (node i, stencil offset o): the 4x4 (3x3 in 2D) block of
// the lagged Hessian coupling node i with node i + o, summed over the corner
// pairs (a, b = a + o) of the elements that contain both and over their
// Gauss points.  Every entry of S is written once (no atomics, no clearing);
// per pair the Gauss-point sum is formed first, then added to the block.
template <int D>
__global__ void __launch_bounds__(128) k_assemble(Geom g, Mat<double> m,
                                                  const double* __restrict__ coef,
                                                  double* __restrict__ S) {
  constexpr int F = D + 1, NC = 1 << D, NCF = NCoef<D>::value, NO = D == 3 ? 27 : 9;
  const double kc = m.w * m.Gc * m.ls * m.inv_h * m.inv_h;
  const long long total = NO * g.N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int o = int(t / g.N);
    const long long i = t - (long long)o * g.N;
    const int ix = int(i % g.n[0]);
    const long long r = i / g.n[0];
    const int iy = int(r % g.n[1]);
    const int iz = int(r / g.n[1]);
    const int ic[3] = {ix, iy, iz};
    int dof[3] = {0, 0, 0};  // o = sum_k (d_k + 1) 3^k
    {
      int oo = o;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        dof[k] = oo % 3 - 1;
        oo /= 3;
      }
    }
    double tot[F][F];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int h = 0; h < F; ++h) tot[f][h] = 0.0;
    for (int a = 0; a < NC; ++a) {  // node i is corner a of element i - corner(a)
      int ec[3] = {0, 0, 0}, b = 0;
      bool ok = true;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int ak = (a >> k) & 1, bk = ak + dof[k];
        ec[k] = ic[k] - ak;
        ok = ok && ec[k] >= 0 && ec[k] < g.ne[k] && bk >= 0 && bk <= 1;
        b |= (bk & 1) << k;
      }
      if (!ok) continue;
      const long long e = ec[0] + (long long)g.ne[0] * (ec[1] + (long long)g.ne[1] * ec[2]);
      double blk[F][F];
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int h = 0; h < F; ++h) blk[f][h] = 0.0;
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        double na, nb, da[D], db[D];
        shape_tables<D>(a, q, na, da);
        shape_tables<D>(b, q, nb, db);
        const double A = coef[(q * NCF + 0) * g.NE + e];
        const double M = coef[(q * NCF + 1) * g.NE + e];
        double B[D][D];
#pragma unroll
        for (int ii = 0; ii < D; ++ii)
#pragma unroll
          for (int kk = 0; kk < D; ++kk) B[ii][kk] = coef[(q * NCF + 2 + sym_index<D>(ii, kk)) * g.NE + e];
        double dd = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) dd += da[k] * db[k];
#pragma unroll
        for (int ii = 0; ii < D; ++ii) {
#pragma unroll
          for (int jj = 0; jj < D; ++jj) {
            double v = m.lam * da[ii] * db[jj] + m.mu * da[jj] * db[ii];
            if (ii == jj) v += m.mu * dd;
            blk[ii][jj] += A * v;
          }
          double bu = 0.0, bc = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            bu += B[ii][k] * da[k];
            bc += B[ii][k] * db[k];
          }
          blk[ii][D] += bu * nb;  // u_i(a) - c(b)
          blk[D][ii] += na * bc;  // c(a) - u_i(b)
        }
        blk[D][D] += M * na * nb + kc * dd;
      }
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int h = 0; h < F; ++h) tot[f][h] += blk[f][h];
    }
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int h = 0; h < F; ++h) S[((long long)(o * F + f) * F + h) * g.N + i] = tot[f][h];
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_stencil_apply(Geom g, const double* __restrict__ S,
                                                       const double* __restrict__ v,
                                                       double* __restrict__ y,
                                                       const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int F = D + 1, NO = D == 3 ? 27 : 9;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = int(i % g.n[0]);
    const long long r = i / g.n[0];
    const int iy = int(r % g.n[1]);
    const int iz = int(r / g.n[1]);
    double acc[F];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = 0.0;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = D == 3 ? o / 9 - 1 : 0;
      const int jx = ix + ox, jy = iy + oy, jz = iz + oz;
      if (jx < 0 || jx >= g.n[0] || jy < 0 || jy >= g.n[1] || jz < 0 || jz >= g.n[2]) continue;
      const long long j = jx + g.n[0] * (jy + (long long)g.n[1] * jz);
      double vj[F];
#pragma unroll
      for (int h = 0; h < F; ++h) vj[h] = v[h * g.N + j];
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int h = 0; h < F; ++h) acc[f] += S[((long long)(o * F + f) * F + h) * g.N + i] * vj[h];
    }
#pragma unroll
    for (int f = 0; f < F; ++f) y[f * g.N + i] = acc[f];
  }
}

// The product on grids too small to fill the SMs with one thread per node:
// one thread per (node, output row), the same summation order per output.
template <int D>
__global__ void __launch_bounds__(128) k_stencil_apply_rows(Geom g, const double* __restrict__ S,
                                                            const double* __restrict__ v,
                                                            double* __restrict__ y,
                                                            const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int F = D + 1, NO = D == 3 ? 27 : 9;
  const long long total = F * g.N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int f = int(t / g.N);
    const long long i = t - (long long)f * g.N;
    const int ix = int(i % g.n[0]);
    const long long r = i / g.n[0];
    const int iy = int(r % g.n[1]);
    const int iz = int(r / g.n[1]);
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = D == 3 ? o / 9 - 1 : 0;
      const int jx = ix + ox, jy = iy + oy, jz = iz + oz;
      if (jx < 0 || jx >= g.n[0] || jy < 0 || jy >= g.n[1] || jz < 0 || jz >= g.n[2]) continue;
      const long long j = jx + g.n[0] * (jy + (long long)g.n[1] * jz);
#pragma unroll
      for (int h = 0; h < F; ++h) acc += S[((long long)(o * F + f) * F + h) * g.N + i] * v[h * g.N + j];
    }
    y[f * g.N + i] = acc;
  }
}

// Projected Gauss-Seidel on the nodes of one parity colour (i_k mod 2 =
// bit k of `colour`): nodes of one colour are not coupled by the 3^d-point
// stencil, so they update in parallel exactly as one after another.  Each
// node updates its fields in order (reverse: in reverse order), each with
// the latest values of the node's other fields:
// s_f <- clamp(s_f - (g_f + (S s)_f) / S_ff, lo_f, hi_f) where S_ff > 0.
template <int D>
__global__ void __launch_bounds__(128) k_pgs_colour(Geom g, const double* __restrict__ S,
                                                    const double* __restrict__ gv,
                                                    const double* __restrict__ lo,
                                                    const double* __restrict__ hi, double* s,
                                                    int colour, int reverse) {
  constexpr int F = D + 1, NO = D == 3 ? 27 : 9, CENTER = D == 3 ? 13 : 4;
  const int cx = colour & 1, cy = (colour >> 1) & 1, cz = D == 3 ? (colour >> 2) & 1 : 0;
  const int mx = (g.n[0] - cx + 1) / 2, my = (g.n[1] - cy + 1) / 2;
  const int mz = D == 3 ? (g.n[2] - cz + 1) / 2 : 1;
  const long long total = (long long)mx * my * mz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ix = 2 * int(t % mx) + cx;
    const int iy = 2 * int((t / mx) % my) + cy;
    const int iz = D == 3 ? 2 * int(t / ((long long)mx * my)) + cz : 0;
    const long long i = ix + (long long)g.n[0] * (iy + (long long)g.n[1] * iz);
    double own[F];
#pragma unroll
    for (int h = 0; h < F; ++h) own[h] = s[h * g.N + i];
    // r = g + S s without the node's own (centre) block, then each field
    // adds the centre block's row with the node's latest values
    double r[F];
#pragma unroll
    for (int f = 0; f < F; ++f) r[f] = gv[f * g.N + i];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      if (o == CENTER) continue;
      const int jx = ix + o % 3 - 1, jy = iy + (o / 3) % 3 - 1, jz = D == 3 ? iz + o / 9 - 1 : 0;
      if (jx < 0 || jx >= g.n[0] || jy < 0 || jy >= g.n[1] || jz < 0 || jz >= g.n[2]) continue;
      const long long j = jx + g.n[0] * (jy + (long long)g.n[1] * jz);
#pragma unroll
      for (int h = 0; h < F; ++h) {
        const double sj = s[h * g.N + j];
#pragma unroll
        for (int f = 0; f < F; ++f) r[f] += S[((long long)(o * F + f) * F + h) * g.N + i] * sj;
      }
    }
#pragma unroll
    for (int k = 0; k < F; ++k) {
      const int f = reverse ? F - 1 - k : k;
      double rf = r[f];
#pragma unroll
      for (int h = 0; h < F; ++h) rf += S[((long long)(CENTER * F + f) * F + h) * g.N + i] * own[h];
      const double d = S[((long long)(CENTER * F + f) * F + f) * g.N + i];
      if (d > 0.0) own[f] = fmin(fmax(own[f] - rf / d, lo[f * g.N + i]), hi[f * g.N + i]);
    }
#pragma unroll
    for (int h = 0; h < F; ++h) s[h * g.N + i] = own[h];
  }
}

cudaError_t pgs_sweep(const Geom& g, const double* S, const double* gv, const double* lo,
                      const double* hi, double* s, bool reverse, cudaStream_t st) {
  const int nc = 1 << g.dim;
  for (int k = 0; k < nc; ++k) {
    const int colour = reverse ? nc - 1 - k : k;
    const long long nodes = (g.N + nc - 1) / nc + g.n[0] * g.n[1];
    const int nb = int(std::min<long long>((nodes + 127) / 128, 16LL * 1216));
    if (g.dim == 3) k_pgs_colour<3><<<nb, 128, 0, st>>>(g, S, gv, lo, hi, s, colour, reverse ? 1 : 0);
    else k_pgs_colour<2><<<nb, 128, 0, st>>>(g, S, gv, lo, hi, s, colour, reverse ? 1 : 0);
  }
  return cudaGetLastError();
}

// Row sums of |D^-1/2 S D^-1/2| (D the positive diagonal of S, 1 where it is
// not): out[row] for every dof, whose maximum bounds the scaled operator's
// largest eigenvalue (Gershgorin).
template <int D>
__global__ void __launch_bounds__(128) k_scaled_rowsum(Geom g, const double* __restrict__ S,
                                                       double* __restrict__ out) {
  constexpr int F = D + 1, NO = D == 3 ? 27 : 9, CENTER = D == 3 ? 13 : 4;
  auto diag = [&](long long node, int f) {
    const double d = S[((long long)(CENTER * F + f) * F + f) * g.N + node];
    return d > 0.0 ? d : 1.0;
  };
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = int(i % g.n[0]);
    const long long rr = i / g.n[0];
    const int iy = int(rr % g.n[1]);
    const int iz = int(rr / g.n[1]);
    double acc[F];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = 0.0;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int jx = ix + o % 3 - 1, jy = iy + (o / 3) % 3 - 1, jz = D == 3 ? iz + o / 9 - 1 : 0;
      if (jx < 0 || jx >= g.n[0] || jy < 0 || jy >= g.n[1] || jz < 0 || jz >= g.n[2]) continue;
      const long long j = jx + g.n[0] * (jy + (long long)g.n[1] * jz);
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int h = 0; h < F; ++h)
          acc[f] += fabs(S[((long long)(o * F + f) * F + h) * g.N + i]) / sqrt(diag(i, f) * diag(j, h));
    }
#pragma unroll
    for (int f = 0; f < F; ++f) out[f * g.N + i] = acc[f];
  }
}

cudaError_t scaled_rowsum(const Geom& g, const double* S, double* out, cudaStream_t st) {
  const int nb = int(std::min<long long>((g.N + 127) / 128, 16LL * 1216));
  if (g.dim == 3) k_scaled_rowsum<3><<<nb, 128, 0, st>>>(g, S, out);
  else k_scaled_rowsum<2><<<nb, 128, 0, st>>>(g, S, out);
  return cudaGetLastError();
}

cudaError_t stencil_assemble(const Geom& g, const Mat<double>& m, const double* coef, double* S,
                             cudaStream_t st) {
  const long long total = (g.dim == 3 ? 27LL : 9LL) * g.N;
  const int nb = int(std::min<long long>((total + 127) / 128, 16LL * 1216));
  if (g.dim == 3) k_assemble<3><<<nb, 128, 0, st>>>(g, m, coef, S);
  else k_assemble<2><<<nb, 128, 0, st>>>(g, m, coef, S);
  return cudaGetLastError();
}

cudaError_t stencil_apply(const Geom& g, const double* S, const double* v, double* y,
                          cudaStream_t st, const int* skip) {
  if (g.N < 152LL * 512) {  // fewer nodes than two 256-thread CTAs per SM
    const long long total = (g.dim + 1) * g.N;
    const int nb = int(std::min<long long>((total + 127) / 128, 16LL * 1216));
    if (g.dim == 3) k_stencil_apply_rows<3><<<nb, 128, 0, st>>>(g, S, v, y, skip);
    else k_stencil_apply_rows<2><<<nb, 128, 0, st>>>(g, S, v, y, skip);
    return cudaGetLastError();
  }
  const int nb = int(std::min<long long>((g.N + 255) / 256, 16LL * 1216));
  if (g.dim == 3) k_stencil_apply<3><<<nb, 256, 0, st>>>(g, S, v, y, skip);
  else k_stencil_apply<2><<<nb, 256, 0, st>>>(g, S, v, y, skip);
  return cudaGetLastError();
}

cudaError_t elem_hessdiag(const Geom& g, const Mat<double>& m, const void* x, int prec,
                          double* y, cudaStream_t st) {
  if (g.dim == 3)
    return prec ? launch_scatter<3, float, double, OP_DIAG>(g, m, x, nullptr, y, nullptr, st)
                : launch_scatter<3, double, double, OP_DIAG>(g, m, x, nullptr, y, nullptr, st);
  return prec ? launch_scatter<2, float, double, OP_DIAG>(g, m, x, nullptr, y, nullptr, st)
              : launch_scatter<2, double, double, OP_DIAG>(g, m, x, nullptr, y, nullptr, st);
}

cudaError_t elem_hessvec_mixed(const Geom& g, const Mat<double>& m, const float* x32,
                               const double* v, double* y, cudaStream_t st, const int* skip,
                               void* part, const float* p_dev) {
  if (g.dim == 3) return launch_hess_tile3<double>(g, m, x32, v, y, skip, st, part, p_dev);
  return launch_scatter<2, float, double, OP_HESS>(g, m, x32, v, y, skip, st);
}

template <int D, class T>
static cudaError_t launch_energy(const Geom& g, const Mat<double>& m, const void* x,
                                 const Scratch& s, double* out, cudaStream_t st) {
  const int nb = reduce_grid(g.NE, 256);
  k_energy<D, T><<<nb, 256, 0, st>>>(g, m, static_cast<const T*>(x), s.partials, s.counter, out);
  return cudaGetLastError();
}

cudaError_t elem_energy(const Geom& g, const Mat<double>& m, const void* x, int prec,
                        const Scratch& s, double* out, cudaStream_t st) {
  if (g.dim == 3)
    return prec ? launch_energy<3, float>(g, m, x, s, out, st)
                : launch_energy<3, double>(g, m, x, s, out, st);
  return prec ? launch_energy<2, float>(g, m, x, s, out, st)
              : launch_energy<2, double>(g, m, x, s, out, st);
}

// The energy kernel with one element per thread (nblocks = ceil(NE / 256))
// and caller-provided partial sums (one per block) and counter.
template <int D, class T>
static cudaError_t launch_energy_blocks(const Geom& g, const Mat<double>& m, const void* x,
                                        double* partials, unsigned* counter, int nblocks,
                                        double* out, cudaStream_t st) {
  k_energy<D, T><<<nblocks, 256, 0, st>>>(g, m, static_cast<const T*>(x), partials, counter, out);
  return cudaGetLastError();
}

cudaError_t elem_energy_blocks(const Geom& g, const Mat<double>& m, const void* x, int prec,
                               double* partials, unsigned* counter, int nblocks, double* out,
                               cudaStream_t st) {
  if (g.dim == 3)
    return prec ? launch_energy_blocks<3, float>(g, m, x, partials, counter, nblocks, out, st)
                : launch_energy_blocks<3, double>(g, m, x, partials, counter, nblocks, out, st);
  return prec ? launch_energy_blocks<2, float>(g, m, x, partials, counter, nblocks, out, st)
              : launch_energy_blocks<2, double>(g, m, x, partials, counter, nblocks, out, st);
}

template <int D, class T>
static cudaError_t launch_energy_diff(const Geom& g, const Mat<double>& m, const void* x,
                                      const void* sv, const Scratch& s, double* out,
                                      cudaStream_t st) {
  const int nb = reduce_grid(g.NE, 256);
  k_energy_diff<D, T><<<nb, 256, 0, st>>>(g, m, static_cast<const T*>(x),
                                           static_cast<const T*>(sv), s.partials, s.counter, out);
  return cudaGetLastError();
}

cudaError_t elem_energy_diff(const Geom& g, const Mat<double>& m, const void* x, const void* sv,
                             int prec, const Scratch& s, double* out, cudaStream_t st) {
  if (g.dim == 3)
    return prec ? launch_energy_diff<3, float>(g, m, x, sv, s, out, st)
                : launch_energy_diff<3, double>(g, m, x, sv, s, out, st);
  return prec ? launch_energy_diff<2, float>(g, m, x, sv, s, out, st)
              : launch_energy_diff<2, double>(g, m, x, sv, s, out, st);
}

// 3D form of k_energy_diff_hi on element tiles: a block takes 8^3-element
// tiles in turn (each element once), stages the tile's 9^3 corner nodes of x
// and s in shared memory as float4, and adds the FP64 g . s of the nodes the
// tile owns ([o, o+8) per axis, the last tile of an axis also its end node).
// out = (gx . s, a2, a3, a4), deterministic (fixed tile order per block).
__global__ void __launch_bounds__(128, 4) k_energy_diff_hi_tile3(Geom g, Mat<float> m,
                                                              const double* __restrict__ x,
                                                              const double* __restrict__ s,
                                                              const double* __restrict__ gx,
                                                              double* partials, unsigned* counter,
                                                              double* out) {
  constexpr int T = 8, NN = T + 1, NH = NN * NN * NN, NT = 128;
  __shared__ float4 xs[NH], ss[NH];
  const int tx = (g.ne[0] + T - 1) / T, ty = (g.ne[1] + T - 1) / T, tz = (g.ne[2] + T - 1) / T;
  const long long ntiles = (long long)tx * ty * tz;
  const long long N = g.N;
  float acc[3] = {0.f, 0.f, 0.f};
  double dot = 0.0;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int bx = int(t % tx), by = int((t / tx) % ty), bz = int(t / ((long long)tx * ty));
    const int ox = bx * T, oy = by * T, oz = bz * T;
    __syncthreads();  // the previous tile's reads are done
    for (int j = threadIdx.x; j < NH; j += NT) {
      const int i = j % NN, jj = (j / NN) % NN, k = j / (NN * NN);
      const int nx = ox + i, ny = oy + jj, nz = oz + k;
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      if (nx < g.n[0] && ny < g.n[1] && nz < g.n[2]) {
        const long long idx = nx + (long long)g.n[0] * (ny + (long long)g.n[1] * nz);
        a = make_float4(float(x[idx]), float(x[N + idx]), float(x[2 * N + idx]), float(x[3 * N + idx]));
        b = make_float4(float(s[idx]), float(s[N + idx]), float(s[2 * N + idx]), float(s[3 * N + idx]));
        // g . s over the nodes this tile owns
        const bool own = (i < T || bx == tx - 1) && (jj < T || by == ty - 1) && (k < T || bz == tz - 1);
        if (gx && own)
#pragma unroll
          for (int f = 0; f < 4; ++f) dot += gx[f * N + idx] * s[f * N + idx];
      }
      xs[j] = a;
      ss[j] = b;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < T * T * T; e += NT) {
      const int lx = e % T, ly = (e / T) % T, lz = e / (T * T);
      if (ox + lx >= g.ne[0] || oy + ly >= g.ne[1] || oz + lz >= g.ne[2]) continue;
      const int c0 = lx + NN * (ly + NN * lz);
      float xe[4][8], se[4][8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int c = c0 + (a & 1) + NN * ((a >> 1) & 1) + NN * NN * ((a >> 2) & 1);
        const float4 xa = xs[c], sa = ss[c];
        xe[0][a] = xa.x; xe[1][a] = xa.y; xe[2][a] = xa.z; xe[3][a] = xa.w;
        se[0][a] = sa.x; se[1][a] = sa.y; se[2][a] = sa.z; se[3][a] = sa.w;
      }
      float a4[4];
      elem_energy_diff<3, float>(xe, se, m, a4);
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[k] += a4[k + 1];
    }
  }
  double d[4] = {dot, double(acc[0]), double(acc[1]), double(acc[2])};
  grid_finish<4, OpSum>(d, partials, counter, out);
}

cudaError_t elem_energy_diff_hi(const Geom& g, const Mat<double>& m, const double* x,
                                const double* sv, const double* gx, const Scratch& s,
                                double* out, cudaStream_t st) {
  const int nb = reduce_grid(g.NE, 256);
  const long long n = (long long)(g.dim + 1) * g.N;
  if (g.dim == 3) {
    const long long tiles = (long long)((g.ne[0] + 7) / 8) * ((g.ne[1] + 7) / 8) * ((g.ne[2] + 7) / 8);
    const int nt = int(std::min<long long>(tiles, kMaxBlocks));
    k_energy_diff_hi_tile3<<<nt, 128, 0, st>>>(g, cast_mat<float>(m), x, sv, gx, s.partials,
                                                s.counter, out);
  } else
    k_energy_diff_hi<2><<<nb, 256, 0, st>>>(g, cast_mat<float>(m), x, sv, gx, n, s.partials,
                                            s.counter, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------ rasterisation
// LINE2D device rows: [cx, cy, tx, ty, nx, ny, half_length]
// DISC3D device rows: [cx, cy, cz, nx, ny, nz, radius]
// Products and sums are rounded one by one (no contraction) so that the
// band test takes the same FP64 decisions as a plain evaluation.
__global__ void k_raster(Geom g, int kind, int nrows, const double* __restrict__ rows,
                         double band, double* __restrict__ c, double* __restrict__ cprev) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long ix = i % g.n[0];
    const long long r = i / g.n[0];
    const long long iy = r % g.n[1];
    const long long iz = r / g.n[1];
    const double X = __dmul_rn(double(ix), g.h), Y = __dmul_rn(double(iy), g.h),
                 Z = __dmul_rn(double(iz), g.h);
    bool in = false;
    for (int k = 0; k < nrows && !in; ++k) {
      const double* q = rows + kRasterRow * k;
      if (kind == 0) {
        const double dx = __dadd_rn(X, -q[0]), dy = __dadd_rn(Y, -q[1]);
        const double dn = fabs(__dadd_rn(__dmul_rn(q[4], dx), __dmul_rn(q[5], dy)));
        const double dt = fabs(__dadd_rn(__dmul_rn(q[2], dx), __dmul_rn(q[3], dy)));
        in = dn <= band && dt <= q[6];
      } else if (kind == 1) {
        const double dx = __dadd_rn(X, -q[0]), dy = __dadd_rn(Y, -q[1]), dz = __dadd_rn(Z, -q[2]);
        const double dn = __dadd_rn(__dadd_rn(__dmul_rn(q[3], dx), __dmul_rn(q[4], dy)),
                                    __dmul_rn(q[5], dz));
        const double px = __dadd_rn(dx, -__dmul_rn(dn, q[3]));
        const double py = __dadd_rn(dy, -__dmul_rn(dn, q[4]));
        const double pz = __dadd_rn(dz, -__dmul_rn(dn, q[5]));
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz));
        in = fabs(dn) <= band && r2 <= __dmul_rn(q[6], q[6]);
      } else if (kind == 2) {
        // rectangle: |d.n| <= band, |d.a| <= half_a, |d.b| <= half_b
        const double dx = __dadd_rn(X, -q[0]), dy = __dadd_rn(Y, -q[1]), dz = __dadd_rn(Z, -q[2]);
        const double dn = __dadd_rn(__dadd_rn(__dmul_rn(q[3], dx), __dmul_rn(q[4], dy)),
                                    __dmul_rn(q[5], dz));
        const double da = __dadd_rn(__dadd_rn(__dmul_rn(q[6], dx), __dmul_rn(q[7], dy)),
                                    __dmul_rn(q[8], dz));
        const double db = __dadd_rn(__dadd_rn(__dmul_rn(q[9], dx), __dmul_rn(q[10], dy)),
                                    __dmul_rn(q[11], dz));
        in = fabs(dn) <= band && fabs(da) <= q[12] && fabs(db) <= q[13];
      }
    }
    const double val = in ? 1.0 : 0.0;
    c[i] = val;
    cprev[i] = val;
  }
}

cudaError_t rasterize(const Geom& g, int kind, int n, const double* rows_dev, double band,
                      double* c_plane, double* c_prev, cudaStream_t st) {
  long long nb = (g.N + 255) / 256;
  if (nb > 4096) nb = 4096;
  k_raster<<<int(nb), 256, 0, st>>>(g, kind, n, rows_dev, band, c_plane, c_prev);
  return cudaGetLastError();
}

// ------------------------------------------------------------ transfers
// Q1 prolongation: a fine node on an even index coincides with a coarse
// node; on an odd index it averages its two coarse neighbours (per axis).
template <class T>
__global__ void k_prolong(Geom gc, Geom gf, int nf, const T* __restrict__ in, T* __restrict__ out,
                          const int* __restrict__ skip) {
  if (skip && *skip) return;
  const long long total = gf.N * nf;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int f = int(t / gf.N);
    const long long i = t - f * gf.N;
    const int ix = int(i % gf.n[0]);
    const long long r = i / gf.n[0];
    const int iy = int(r % gf.n[1]);
    const int iz = int(r / gf.n[1]);
    int c0[3] = {ix >> 1, iy >> 1, iz >> 1};
    int odd[3] = {ix & 1, iy & 1, iz & 1};
    const T* src = in + f * gc.N;
    T acc = T(0);
    for (int dz = 0; dz <= odd[2]; ++dz)
      for (int dy = 0; dy <= odd[1]; ++dy)
        for (int dx = 0; dx <= odd[0]; ++dx) {
          T wgt = T(1);
          if (odd[0]) wgt *= T(0.5);
          if (odd[1]) wgt *= T(0.5);
          if (odd[2]) wgt *= T(0.5);
          const long long j = (c0[0] + dx) + gc.n[0] * ((c0[1] + dy) + (long long)gc.n[1] * (c0[2] + dz));
          acc += wgt * src[j];
        }
    out[t] = acc;
  }
}

// Restriction R = I^T: a coarse node collects the fine nodes within one fine
// spacing, weight 1 on the coincident node and 1/2 per odd offset and axis.
// With normalise, the sum is divided by the sum of the weights (P).
template <class T>
__global__ void k_restrict(Geom gc, Geom gf, int nf, const T* __restrict__ in,
                           T* __restrict__ out, bool normalise, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const long long total = gc.N * nf;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int f = int(t / gc.N);
    const long long j = t - f * gc.N;
    const int jx = int(j % gc.n[0]);
    const long long r = j / gc.n[0];
    const int jy = int(r % gc.n[1]);
    const int jz = int(r / gc.n[1]);
    const T* src = in + f * gf.N;
    T acc = T(0), wsum = T(0);
    const int zlo = gf.dim == 3 ? -1 : 0, zhi = gf.dim == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
      const int iz = 2 * jz + dz;
      if (iz < 0 || iz >= gf.n[2]) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int iy = 2 * jy + dy;
        if (iy < 0 || iy >= gf.n[1]) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int ix = 2 * jx + dx;
          if (ix < 0 || ix >= gf.n[0]) continue;
          T wgt = T(1);
          if (dx) wgt *= T(0.5);
          if (dy) wgt *= T(0.5);
          if (dz) wgt *= T(0.5);
          acc += wgt * src[ix + gf.n[0] * (iy + (long long)gf.n[1] * iz)];
          wsum += wgt;
        }
      }
    }
    out[t] = normalise ? acc / wsum : acc;
  }
}

__global__ void k_bounds(Geom gc, Geom gf, int nf, const double* __restrict__ lo_f,
                         const double* __restrict__ hi_f, double* __restrict__ lo_c,
                         double* __restrict__ hi_c) {
  const long long total = gc.N * nf;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int f = int(t / gc.N);
    const long long j = t - f * gc.N;
    const int jx = int(j % gc.n[0]);
    const long long r = j / gc.n[0];
    const int jy = int(r % gc.n[1]);
    const int jz = int(r / gc.n[1]);
    double lo = -INFINITY, hi = INFINITY;
    const int zlo = gf.dim == 3 ? -1 : 0, zhi = gf.dim == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
      const int iz = 2 * jz + dz;
      if (iz < 0 || iz >= gf.n[2]) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int iy = 2 * jy + dy;
        if (iy < 0 || iy >= gf.n[1]) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int ix = 2 * jx + dx;
          if (ix < 0 || ix >= gf.n[0]) continue;
          const long long i = f * gf.N + ix + gf.n[0] * (iy + (long long)gf.n[1] * iz);
          lo = fmax(lo, lo_f[i]);
          hi = fmin(hi, hi_f[i]);
        }
      }
    }
    lo_c[t] = lo;
    hi_c[t] = hi;
  }
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 8192) b = 8192;
  if (b < 1) b = 1;
  return int(b);
}

cudaError_t xfer_prolong(const Geom& gc, const Geom& gf, int nf, const void* in, void* out,
                         int prec, cudaStream_t st, const int* skip) {
  const int nb = grid_for(gf.N * nf);
  if (prec)
    k_prolong<float><<<nb, 256, 0, st>>>(gc, gf, nf, static_cast<const float*>(in), static_cast<float*>(out), skip);
  else
    k_prolong<double><<<nb, 256, 0, st>>>(gc, gf, nf, static_cast<const double*>(in), static_cast<double*>(out), skip);
  return cudaGetLastError();
}

cudaError_t xfer_restrict(const Geom& gc, const Geom& gf, int nf, const void* in, void* out,
                          int prec, bool normalise, cudaStream_t st, const int* skip) {
  const int nb = grid_for(gc.N * nf);
  if (prec)
    k_restrict<float><<<nb, 256, 0, st>>>(gc, gf, nf, static_cast<const float*>(in), static_cast<float*>(out), normalise, skip);
  else
    k_restrict<double><<<nb, 256, 0, st>>>(gc, gf, nf, static_cast<const double*>(in), static_cast<double*>(out), normalise, skip);
  return cudaGetLastError();
}

cudaError_t xfer_bounds(const Geom& gc, const Geom& gf, int nf, const double* lo_f,
                        const double* hi_f, double* lo_c, double* hi_c, cudaStream_t st) {
  k_bounds<<<grid_for(gc.N * nf), 256, 0, st>>>(gc, gf, nf, lo_f, hi_f, lo_c, hi_c);
  return cudaGetLastError();
}

}  // namespace pf
