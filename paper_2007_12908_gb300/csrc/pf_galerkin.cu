// Stored Galerkin coarse operators (the second-order coherent level model of
// eq. (second_order_consistency) and eq. (delta_terms) under Hessian
// lagging, Sec. 4.2.1): the model Hessian of a coarse level l is
// G^l = R G^{l+1} I with G^{L-1} = H(x_lag) on the finest level.  Instead
// of applying that chain matrix-free (a finest-level product per coarse
// product), the operators are assembled once per lag into FP32 block
// stencils, 3^d points per node.
//
// Element-nested construction:
//  1. next-to-finest level: the element matrix of a coarse element E is the
//     sum over its 2^d fine children and their Gauss points of the Hessian
//     density at the fine Gauss point, with the coarse Q1 basis functions
//     (which lie in the fine space, so I maps them exactly) evaluated
//     there: K_E = sum_q B_E(q)^T D_q B_E(q).  D_q is the lagged Gauss-point
//     coefficient set (A, M, B) of the fine element, computed from x_lag.
//  2. coarser levels: K_E' = sum_children I_c^T K_c I_c with I_c the Q1
//     interpolation from the coarse element's corners to the child's.
//  3. each level's stencil: the (node, offset) block is the sum of the
//     element blocks of the elements that hold both nodes, in a fixed
//     element order (no atomics; deterministic).
// Element matrices are (2^d (d+1))^2 floats, row a*F + f, column b*F + h
// (corner a/b, field f/h).
#include <algorithm>
#include <string>

#include "../../include/pf.h"
#include "pf_element.cuh"
#include "pf_internal.h"

namespace pf {

namespace {

template <int D>
struct GalDims {
  static constexpr int NC = 1 << D, F = D + 1, R = NC * F, NQ = NC;
  static constexpr int NO = D == 3 ? 27 : 9;
};

// Coarse Q1 basis at the fine Gauss points of the 2^d children of a coarse
// element: value and raw derivatives (d/dt of the 1D factor = +-1, times the
// other factors), the derivatives halved so that they are raw derivatives
// of the fine element (the fine coefficients carry 1/h_fine).
// Index (child c, fine Gauss point q, coarse corner a).
template <int D>
__device__ __forceinline__ void coarse_shape(int c, int q, int a, float& na, float (&da)[3]) {
  float n1[3], d1[3];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float xi = ((q >> k) & 1) ? float(PF_XI1) : float(PF_XI0);
    const float t = 0.5f * (float((c >> k) & 1) + xi);  // coarse reference coordinate
    const int ak = (a >> k) & 1;
    n1[k] = ak ? t : 1.f - t;
    d1[k] = ak ? 0.5f : -0.5f;
  }
  na = 1.f;
#pragma unroll
  for (int k = 0; k < D; ++k) na *= n1[k];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    float t = d1[k];
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (j != k) t *= n1[j];
    da[k] = t;
  }
}

template <int D>
__device__ __forceinline__ long long node_index(const Geom& g, int ix, int iy, int iz) {
  return D == 3 ? ix + (long long)g.n[0] * (iy + (long long)g.n[1] * iz) : ix + (long long)g.n[0] * iy;
}

template <int D>
__device__ __forceinline__ void elem_xyz(const Geom& g, long long e, int& ex, int& ey, int& ez) {
  ex = int(e % g.ne[0]);
  const long long r = e / g.ne[0];
  ey = D == 3 ? int(r % g.ne[1]) : int(r);
  ez = D == 3 ? int(r / g.ne[1]) : 0;
}

// 1. Element matrices of the next-to-finest level gc from the finest lag
// (FP32 x on the finest grid gf).  One warp per coarse element; lane r =
// a*F + f accumulates row r over the 2^d children x 2^d Gauss points.
template <int D>
__global__ void __launch_bounds__(256) k_gal_fine(Geom gc, Geom gf, Mat<float> m,
                                                  const float* __restrict__ x,
                                                  float* __restrict__ K) {
  using G = GalDims<D>;
  constexpr int NC = G::NC, F = G::F, R = G::R, NCF = NCoef<D>::value;
  __shared__ float cf_s[8][NC][NC][NCF];  // per warp: [child][q][coef]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long e = blockIdx.x * 8LL + warp;
  const bool live = e < gc.NE;
  int ex = 0, ey = 0, ez = 0;
  if (live) elem_xyz<D>(gc, e, ex, ey, ez);
  // lanes 0 .. NC-1: the lagged coefficients of child c = lane
  if (live && lane < NC) {
    const int c = lane;
    const int fx = 2 * ex + (c & 1), fy = 2 * ey + ((c >> 1) & 1), fz = D == 3 ? 2 * ez + ((c >> 2) & 1) : 0;
    float xe[F][NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      const long long idx = node_index<D>(gf, fx + (a & 1), fy + ((a >> 1) & 1), D == 3 ? fz + ((a >> 2) & 1) : 0);
#pragma unroll
      for (int f = 0; f < F; ++f) xe[f][a] = x[f * gf.N + idx];
    }
    float cf[NC][NCF];
    hess_coef<D, float>(xe, m, cf);
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int k = 0; k < NCF; ++k) cf_s[warp][c][q][k] = cf[q][k];
  }
  __syncwarp();
  if (!live || lane >= R) return;
  const int a = lane / F, f = lane % F;
  const float kc = m.w * m.Gc * m.ls * m.inv_h * m.inv_h;
  float row[R];
#pragma unroll
  for (int j = 0; j < R; ++j) row[j] = 0.f;
  for (int c = 0; c < NC; ++c)
    for (int q = 0; q < NC; ++q) {
      const float* cq = cf_s[warp][c][q];
      const float A = cq[0], M = cq[1];
      float B[3][3];
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) B[i][k] = cq[2 + sym_index<D>(i, k)];
      float na, da[3];
      coarse_shape<D>(c, q, a, na, da);
      // this row's factors: for u_i rows B.da, for the c row na
      float bda = 0.f;
      if (f < D) {
#pragma unroll
        for (int k = 0; k < D; ++k) bda += B[f][k] * da[k];
      }
#pragma unroll
      for (int b = 0; b < NC; ++b) {
        float nb, db[3];
        coarse_shape<D>(c, q, b, nb, db);
        float dd = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) dd += da[k] * db[k];
        if (f < D) {
#pragma unroll
          for (int j = 0; j < D; ++j) {
            float v = m.lam * da[f] * db[j] + m.mu * da[j] * db[f];
            if (j == f) v += m.mu * dd;
            row[b * F + j] += A * v;
          }
          row[b * F + D] += bda * nb;  // u_f(a) - c(b)
        } else {
#pragma unroll
          for (int j = 0; j < D; ++j) {
            float bdb = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) bdb += B[j][k] * db[k];
            row[b * F + j] += na * bdb;  // c(a) - u_j(b)
          }
          row[b * F + D] += M * na * nb + kc * dd;
        }
      }
    }
  float* out = K + (e * R + lane) * R;
#pragma unroll
  for (int j = 0; j < R; ++j) out[j] = row[j];
}

// Interpolation weight of coarse corner ap (per axis 0/1, at position 2 ap)
// at fine position pos (0, 1, 2) of the coarse element.
__device__ __forceinline__ float interp_w(int pos, int ap) {
  return pos == 2 * ap ? 1.f : (pos == 1 ? 0.5f : 0.f);
}

// 2. K' of the coarse level gc from the element matrices Kf of the level
// above it (gf): K'_E = sum over children c of I_c^T K_c I_c.  One warp per
// coarse element, lane r' = a'*F + f.
template <int D>
__global__ void __launch_bounds__(256) k_gal_rap(Geom gc, Geom gf, const float* __restrict__ Kf,
                                                 float* __restrict__ Kc) {
  using G = GalDims<D>;
  constexpr int NC = G::NC, F = G::F, R = G::R;
  __shared__ float ks[8][R * R];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long e = blockIdx.x * 8LL + warp;
  const bool live = e < gc.NE;
  int ex = 0, ey = 0, ez = 0;
  if (live) elem_xyz<D>(gc, e, ex, ey, ez);
  const int ap = lane / F, f = lane % F;
  float row[R];
#pragma unroll
  for (int j = 0; j < R; ++j) row[j] = 0.f;
  for (int c = 0; c < NC; ++c) {
    __syncwarp();
    if (live) {
      const int fx = 2 * ex + (c & 1), fy = 2 * ey + ((c >> 1) & 1), fz = D == 3 ? 2 * ez + ((c >> 2) & 1) : 0;
      const long long ef = D == 3 ? fx + (long long)gf.ne[0] * (fy + (long long)gf.ne[1] * fz)
                                  : fx + (long long)gf.ne[0] * fy;
      const float* src = Kf + ef * R * R;
      for (int i = lane; i < R * R; i += 32) ks[warp][i] = src[i];
    }
    __syncwarp();
    if (!live || lane >= R) continue;
    // weights of this lane's coarse corner ap at the child's corners a
    float wa[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      float w = 1.f;
#pragma unroll
      for (int k = 0; k < D; ++k) w *= interp_w(((c >> k) & 1) + ((a >> k) & 1), (ap >> k) & 1);
      wa[a] = w;
    }
    // t[b h] = sum_a wa[a] Kc[a f][b h]
    float t[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      float s = 0.f;
#pragma unroll
      for (int a = 0; a < NC; ++a) s += wa[a] * ks[warp][(a * F + f) * R + j];
      t[j] = s;
    }
    // row[b' h] += sum_b t[b h] w(b, b')
#pragma unroll
    for (int bp = 0; bp < NC; ++bp) {
      float wb[NC];
#pragma unroll
      for (int b = 0; b < NC; ++b) {
        float w = 1.f;
#pragma unroll
        for (int k = 0; k < D; ++k) w *= interp_w(((c >> k) & 1) + ((b >> k) & 1), (bp >> k) & 1);
        wb[b] = w;
      }
#pragma unroll
      for (int h = 0; h < F; ++h) {
        float s = 0.f;
#pragma unroll
        for (int b = 0; b < NC; ++b) s += t[b * F + h] * wb[b];
        row[bp * F + h] += s;
      }
    }
  }
  if (!live || lane >= R) return;
  float* out = Kc + (e * R + lane) * R;
#pragma unroll
  for (int j = 0; j < R; ++j) out[j] = row[j];
}

// 3. Stencil of level g from its element matrices: one thread per (node,
// offset); the block sums the elements holding both nodes in ascending
// corner order.  S[((o F + f) F + h) N + i], as the FP64 stencil.
template <int D>
__global__ void __launch_bounds__(128) k_gal_assemble(Geom g, const float* __restrict__ K,
                                                      float* __restrict__ S) {
  using G = GalDims<D>;
  constexpr int NC = G::NC, F = G::F, R = G::R, NO = G::NO;
  const long long total = NO * g.N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int o = int(t / g.N);
    const long long i = t - (long long)o * g.N;
    const int ic[3] = {int(i % g.n[0]), int((i / g.n[0]) % g.n[1]),
                       D == 3 ? int(i / ((long long)g.n[0] * g.n[1])) : 0};
    int dof[3] = {0, 0, 0};
    {
      int oo = o;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        dof[k] = oo % 3 - 1;
        oo /= 3;
      }
    }
    float tot[F][F];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int h = 0; h < F; ++h) tot[f][h] = 0.f;
    for (int a = 0; a < NC; ++a) {
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
      const long long e = D == 3 ? ec[0] + (long long)g.ne[0] * (ec[1] + (long long)g.ne[1] * ec[2])
                                 : ec[0] + (long long)g.ne[0] * ec[1];
      const float* Ke = K + e * R * R;
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int h = 0; h < F; ++h) tot[f][h] += Ke[(a * F + f) * R + b * F + h];
    }
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int h = 0; h < F; ++h) S[((long long)(o * F + f) * F + h) * g.N + i] = tot[f][h];
  }
}

// 4. y = S v with an FP32 stencil; vectors float (FP32 sums) or double
// (FP64 sums of the FP32 entries).
template <int D, class TV>
__global__ void __launch_bounds__(256) k_gal_apply(Geom g, const float* __restrict__ S,
                                                   const TV* __restrict__ v, TV* __restrict__ y,
                                                   const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int F = D + 1, NO = D == 3 ? 27 : 9;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = int(i % g.n[0]);
    const long long r = i / g.n[0];
    const int iy = int(r % g.n[1]);
    const int iz = int(r / g.n[1]);
    TV acc[F];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = TV(0);
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int jx = ix + o % 3 - 1, jy = iy + (o / 3) % 3 - 1, jz = D == 3 ? iz + o / 9 - 1 : iz;
      if (jx < 0 || jx >= g.n[0] || jy < 0 || jy >= g.n[1] || jz < 0 || jz >= g.n[2]) continue;
      const long long j = jx + g.n[0] * (jy + (long long)g.n[1] * jz);
      TV vj[F];
#pragma unroll
      for (int h = 0; h < F; ++h) vj[h] = v[h * g.N + j];
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int h = 0; h < F; ++h) acc[f] += TV(S[((long long)(o * F + f) * F + h) * g.N + i]) * vj[h];
    }
#pragma unroll
    for (int f = 0; f < F; ++f) y[f * g.N + i] = acc[f];
  }
}

template <class T>
Mat<T> to_mat(const Mat<double>& m) {
  Mat<T> r;
  r.lam = T(m.lam); r.mu = T(m.mu); r.Gc = T(m.Gc); r.ls = T(m.ls); r.k = T(m.k);
  r.p = T(m.p); r.inv_h = T(m.inv_h); r.w = T(m.w);
  return r;
}

int blocks_for(long long n, int threads, long long cap) {
  return int(std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, cap)));
}

}  // namespace

long long galerkin_elem_count(const Geom& g) {
  const long long r = (1LL << g.dim) * (g.dim + 1);
  return g.NE * r * r;
}

long long galerkin_stencil_count(const Geom& g) {
  const int f = g.dim + 1;
  return (g.dim == 3 ? 27LL : 9LL) * f * f * g.N;
}

cudaError_t galerkin_fine(const Geom& gc, const Geom& gf, const Mat<double>& mf, const float* x_fine,
                          float* K, cudaStream_t st) {
  const int nb = int((gc.NE + 7) / 8);
  if (gc.dim == 3) k_gal_fine<3><<<nb, 256, 0, st>>>(gc, gf, to_mat<float>(mf), x_fine, K);
  else k_gal_fine<2><<<nb, 256, 0, st>>>(gc, gf, to_mat<float>(mf), x_fine, K);
  return cudaGetLastError();
}

cudaError_t galerkin_rap(const Geom& gc, const Geom& gf, const float* Kf, float* Kc, cudaStream_t st) {
  const int nb = int((gc.NE + 7) / 8);
  if (gc.dim == 3) k_gal_rap<3><<<nb, 256, 0, st>>>(gc, gf, Kf, Kc);
  else k_gal_rap<2><<<nb, 256, 0, st>>>(gc, gf, Kf, Kc);
  return cudaGetLastError();
}

cudaError_t galerkin_assemble(const Geom& g, const float* K, float* S, cudaStream_t st) {
  const long long total = (g.dim == 3 ? 27LL : 9LL) * g.N;
  const int nb = blocks_for(total, 128, 16LL * 1216);
  if (g.dim == 3) k_gal_assemble<3><<<nb, 128, 0, st>>>(g, K, S);
  else k_gal_assemble<2><<<nb, 128, 0, st>>>(g, K, S);
  return cudaGetLastError();
}

cudaError_t galerkin_apply(const Geom& g, const float* S, const void* v, void* y, int prec,
                           cudaStream_t st, const int* skip) {
  const int nb = blocks_for(g.N, 256, 16LL * 1216);
  if (prec == PF_FP32) {
    if (g.dim == 3)
      k_gal_apply<3, float><<<nb, 256, 0, st>>>(g, S, static_cast<const float*>(v), static_cast<float*>(y), skip);
    else
      k_gal_apply<2, float><<<nb, 256, 0, st>>>(g, S, static_cast<const float*>(v), static_cast<float*>(y), skip);
  } else {
    if (g.dim == 3)
      k_gal_apply<3, double><<<nb, 256, 0, st>>>(g, S, static_cast<const double*>(v), static_cast<double*>(y), skip);
    else
      k_gal_apply<2, double><<<nb, 256, 0, st>>>(g, S, static_cast<const double*>(v), static_cast<double*>(y), skip);
  }
  return cudaGetLastError();
}

}  // namespace pf
