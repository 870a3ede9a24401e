// Q1 element algebra of the pressurised AT2 functional (Sec. 2, eq.
// pressurized with the +p g(c) div u sign reading), evaluated per element at
// the 2^d Gauss points of a uniform cell.
//
// Interpolation to the Gauss points and the test-function contraction back to
// the corners are sum-factorised along the axes: one pass per axis, each a
// 2-point linear blend (values) or a difference (derivatives, constant along
// their own axis for Q1).  Corner a = ax + 2 ay + 4 az, Gauss point
// q = qx + 2 qy + 4 qz; 1D shape values at the Gauss points are
// N(q=0) = (XI1, XI0), N(q=1) = (XI0, XI1) with XI0 + XI1 = 1.
// Derivatives here are raw nodal differences; callers scale by 1/h.
#pragma once
#include <cuda_runtime.h>

namespace pf {

// (1 -+ 1/sqrt(3)) / 2
#define PF_XI0 0.21132486540518711775
#define PF_XI1 0.78867513459481288225

template <class T>
struct Mat {
  T lam, mu, Gc, ls, k, p;  // Lame, toughness, length scale, residual, pressure
  T inv_h;                  // 1/h
  T w;                      // Gauss weight times det J = h^d / 2^d
};

// ---------------------------------------------------------------- 3D passes
template <class T>
__device__ __forceinline__ void interp3(const T f[8], T val[8], T gx[8], T gy[8], T gz[8]) {
  const T x0 = T(PF_XI0), x1 = T(PF_XI1);
  T X[2][2][2], DX[2][2];
#pragma unroll
  for (int az = 0; az < 2; ++az)
#pragma unroll
    for (int ay = 0; ay < 2; ++ay) {
      const T v0 = f[2 * ay + 4 * az], d = f[1 + 2 * ay + 4 * az] - v0;
      DX[ay][az] = d;
      X[0][ay][az] = v0 + x0 * d;
      X[1][ay][az] = v0 + x1 * d;
    }
  T XY[2][2][2], DY[2][2], DXY[2][2];
#pragma unroll
  for (int az = 0; az < 2; ++az) {
#pragma unroll
    for (int qx = 0; qx < 2; ++qx) {
      const T v0 = X[qx][0][az], d = X[qx][1][az] - v0;
      DY[qx][az] = d;
      XY[qx][0][az] = v0 + x0 * d;
      XY[qx][1][az] = v0 + x1 * d;
    }
    const T v0 = DX[0][az], d = DX[1][az] - v0;
    DXY[0][az] = v0 + x0 * d;
    DXY[1][az] = v0 + x1 * d;
  }
#pragma unroll
  for (int qy = 0; qy < 2; ++qy)
#pragma unroll
    for (int qx = 0; qx < 2; ++qx) {
      const int q = qx + 2 * qy;
      const T v0 = XY[qx][qy][0], d = XY[qx][qy][1] - v0;
      val[q] = v0 + x0 * d;
      val[q + 4] = v0 + x1 * d;
      gz[q] = d;
      gz[q + 4] = d;
    }
#pragma unroll
  for (int qy = 0; qy < 2; ++qy) {
    const T v0 = DXY[qy][0], d = DXY[qy][1] - v0;
    const T a = v0 + x0 * d, b = v0 + x1 * d;
    gx[2 * qy] = a; gx[1 + 2 * qy] = a;
    gx[2 * qy + 4] = b; gx[1 + 2 * qy + 4] = b;
  }
#pragma unroll
  for (int qx = 0; qx < 2; ++qx) {
    const T v0 = DY[qx][0], d = DY[qx][1] - v0;
    const T a = v0 + x0 * d, b = v0 + x1 * d;
    gy[qx] = a; gy[qx + 2] = a;
    gy[qx + 4] = b; gy[qx + 6] = b;
  }
}

// r[a] = sum_q s0[q] N_a(q) + sx[q] Dx_a(q) + sy[q] Dy_a(q) + sz[q] Dz_a(q)
// (raw derivatives), the adjoint of interp3.  s0 == nullptr drops the value
// term (IEEE arithmetic cannot fold multiplications by a zero term away).
template <class T>
__device__ __forceinline__ void test3(const T* s0, const T sx[8], const T sy[8], const T sz[8],
                                      T r[8]) {
  const T x0 = T(PF_XI0), x1 = T(PF_XI1);
  T XYb[2][2][2], DXYb[2][2], DYb[2][2];
#pragma unroll
  for (int qy = 0; qy < 2; ++qy)
#pragma unroll
    for (int qx = 0; qx < 2; ++qx) {
      const int q = qx + 2 * qy;
      const T zs = sz[q] + sz[q + 4];
      if (s0) {
        XYb[qx][qy][0] = x1 * s0[q] + x0 * s0[q + 4] - zs;
        XYb[qx][qy][1] = x0 * s0[q] + x1 * s0[q + 4] + zs;
      } else {
        XYb[qx][qy][0] = -zs;
        XYb[qx][qy][1] = zs;
      }
    }
#pragma unroll
  for (int qy = 0; qy < 2; ++qy) {
    const T a = sx[2 * qy] + sx[1 + 2 * qy], b = sx[2 * qy + 4] + sx[1 + 2 * qy + 4];
    DXYb[qy][0] = x1 * a + x0 * b;
    DXYb[qy][1] = x0 * a + x1 * b;
  }
#pragma unroll
  for (int qx = 0; qx < 2; ++qx) {
    const T a = sy[qx] + sy[qx + 2], b = sy[qx + 4] + sy[qx + 6];
    DYb[qx][0] = x1 * a + x0 * b;
    DYb[qx][1] = x0 * a + x1 * b;
  }
  T Xb[2][2][2], DXb[2][2];
#pragma unroll
  for (int az = 0; az < 2; ++az) {
#pragma unroll
    for (int qx = 0; qx < 2; ++qx) {
      Xb[qx][0][az] = x1 * XYb[qx][0][az] + x0 * XYb[qx][1][az] - DYb[qx][az];
      Xb[qx][1][az] = x0 * XYb[qx][0][az] + x1 * XYb[qx][1][az] + DYb[qx][az];
    }
    DXb[0][az] = x1 * DXYb[0][az] + x0 * DXYb[1][az];
    DXb[1][az] = x0 * DXYb[0][az] + x1 * DXYb[1][az];
  }
#pragma unroll
  for (int az = 0; az < 2; ++az)
#pragma unroll
    for (int ay = 0; ay < 2; ++ay) {
      r[2 * ay + 4 * az] = x1 * Xb[0][ay][az] + x0 * Xb[1][ay][az] - DXb[ay][az];
      r[1 + 2 * ay + 4 * az] = x0 * Xb[0][ay][az] + x1 * Xb[1][ay][az] + DXb[ay][az];
    }
}

// ---------------------------------------------------------------- 2D passes
template <class T>
__device__ __forceinline__ void interp2(const T f[4], T val[4], T gx[4], T gy[4]) {
  const T x0 = T(PF_XI0), x1 = T(PF_XI1);
  T X[2][2], DX[2];
#pragma unroll
  for (int ay = 0; ay < 2; ++ay) {
    const T v0 = f[2 * ay], d = f[1 + 2 * ay] - v0;
    DX[ay] = d;
    X[0][ay] = v0 + x0 * d;
    X[1][ay] = v0 + x1 * d;
  }
#pragma unroll
  for (int qx = 0; qx < 2; ++qx) {
    const T v0 = X[qx][0], d = X[qx][1] - v0;
    val[qx] = v0 + x0 * d;
    val[qx + 2] = v0 + x1 * d;
    gy[qx] = d;
    gy[qx + 2] = d;
  }
  const T v0 = DX[0], d = DX[1] - v0;
  const T a = v0 + x0 * d, b = v0 + x1 * d;
  gx[0] = a; gx[1] = a; gx[2] = b; gx[3] = b;
}

template <class T>
__device__ __forceinline__ void test2(const T* s0, const T sx[4], const T sy[4], T r[4]) {
  const T x0 = T(PF_XI0), x1 = T(PF_XI1);
  T Xb[2][2];
#pragma unroll
  for (int qx = 0; qx < 2; ++qx) {
    const T ys = sy[qx] + sy[qx + 2];
    if (s0) {
      Xb[qx][0] = x1 * s0[qx] + x0 * s0[qx + 2] - ys;
      Xb[qx][1] = x0 * s0[qx] + x1 * s0[qx + 2] + ys;
    } else {
      Xb[qx][0] = -ys;
      Xb[qx][1] = ys;
    }
  }
  const T a = sx[0] + sx[1], b = sx[2] + sx[3];
  const T DXb0 = x1 * a + x0 * b, DXb1 = x0 * a + x1 * b;
#pragma unroll
  for (int ay = 0; ay < 2; ++ay) {
    const T dxb = ay ? DXb1 : DXb0;
    r[2 * ay] = x1 * Xb[0][ay] + x0 * Xb[1][ay] - dxb;
    r[1 + 2 * ay] = x0 * Xb[0][ay] + x1 * Xb[1][ay] + dxb;
  }
}

// ---------------------------------------------------------------- dispatch
template <int D, class T>
__device__ __forceinline__ void interp(const T* f, T* val, T (*g)[1 << D]) {
  if constexpr (D == 3) interp3<T>(f, val, g[0], g[1], g[2]);
  else interp2<T>(f, val, g[0], g[1]);
}

template <int D, class T>
__device__ __forceinline__ void test(const T* s0, T (*s1)[1 << D], T* r) {
  if constexpr (D == 3) test3<T>(s0, s1[0], s1[1], s1[2], r);
  else test2<T>(s0, s1[0], s1[1], r);
}

template <int D, class T>
__device__ __forceinline__ void zero_test(T* r) {
#pragma unroll
  for (int a = 0; a < (1 << D); ++a) r[a] = T(0);
}

// Strain of a displacement gradient G[i][k] = d u_i / d x_k.
template <int D, class T>
struct Strain {
  T eps[D][D];
  T tr;
  __device__ __forceinline__ void set(const T G[D][D]) {
    tr = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      tr += G[i][i];
#pragma unroll
      for (int k = 0; k < D; ++k) eps[i][k] = T(0.5) * (G[i][k] + G[k][i]);
    }
  }
  __device__ __forceinline__ T ddot(const Strain& o) const {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) s += eps[i][k] * o.eps[i][k];
    return s;
  }
};

template <int D>
struct NSym {
  static constexpr int value = D * (D + 1) / 2;  // B stored 00, 11, (22), 01, (02, 12)
};
template <int D>
struct NCoef {
  static constexpr int value = NSym<D>::value + 2;  // A, M, B
};

template <int D>
__device__ __forceinline__ constexpr int sym_index(int i, int k) {
  if (i == k) return i;
  if (D == 2) return 2;
  const int lo = i < k ? i : k, hi = i < k ? k : i;
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

// ---------------------------------------------------------------- element ops
// Every op takes the element's nodal values xe[f][a] (f = field plane,
// a = corner) and, for hessvec / energy_diff, a second vector ve[f][a].

// Energy of one element: sum_q w [g psi + Gc/2 (c^2/ls + ls |grad c|^2) + p g tr]
template <int D, class T>
__device__ __forceinline__ T elem_energy(const T (*xe)[1 << D], const Mat<T>& m) {
  constexpr int NQ = 1 << D;
  T gu[D][D][NQ], cv[NQ], gc[D][NQ], dummy[NQ];
#pragma unroll
  for (int i = 0; i < D; ++i) interp<D, T>(xe[i], dummy, gu[i]);
  interp<D, T>(xe[D], cv, gc);
  T e = T(0);
  const T ils = T(1) / m.ls;  // one division per element, not one per Gauss point
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T G[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) G[i][k] = gu[i][k][q] * m.inv_h;
    Strain<D, T> s;
    s.set(G);
    const T psi = T(0.5) * m.lam * s.tr * s.tr + m.mu * s.ddot(s);
    const T omc = T(1) - cv[q];
    const T g = (T(1) - m.k) * omc * omc + m.k;
    T gc2 = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const T t = gc[k][q] * m.inv_h;
      gc2 += t * t;
    }
    e += g * psi + T(0.5) * m.Gc * (cv[q] * cv[q] * ils + m.ls * gc2) + m.p * g * s.tr;
  }
  return m.w * e;
}

// Strain invariants of a displacement gradient G (physical units):
// tr = div u, ee = eps : eps, and the symmetric off-diagonal sums
// G_ik + G_ki (i < k) in sym order 01, (02, 12).
template <int D, class T>
struct StrainSym {
  T tr, ee, off[D == 3 ? 3 : 1];
  __device__ __forceinline__ void set(const T G[D][D]) {
    tr = T(0);
    ee = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      tr += G[i][i];
      ee += G[i][i] * G[i][i];
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = i + 1; k < D; ++k) {
        const T sik = G[i][k] + G[k][i];
        off[sym_index<D>(i, k) - D] = sik;
        ee += T(0.5) * sik * sik;
      }
  }
};

// Quartic coefficients of E_e(x + t s) - E_e(x).  Gradients stay raw nodal
// differences; 1/h and 1/h^2 are folded into the constants.
template <int D, class T>
__device__ __forceinline__ void elem_energy_diff(const T (*xe)[1 << D], const T (*se)[1 << D],
                                                 const Mat<T>& m, T a[4]) {
  constexpr int NQ = 1 << D;
  T gu[D][D][NQ], cv[NQ], gc[D][NQ], dummy[NQ];
  T gs[D][D][NQ], sc[NQ], gsc[D][NQ];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    interp<D, T>(xe[i], dummy, gu[i]);
    interp<D, T>(se[i], dummy, gs[i]);
  }
  interp<D, T>(xe[D], cv, gc);
  interp<D, T>(se[D], sc, gsc);
  T a1 = 0, a2 = 0, a3 = 0, a4 = 0;
  const T omk = T(1) - m.k;
  const T ih2 = m.inv_h * m.inv_h;
  const T hl = T(0.5) * m.lam * ih2, lam2 = m.lam * ih2, mu2 = m.mu * ih2, ph = m.p * m.inv_h;
  const T gls = m.Gc * m.ls * ih2, hgls = T(0.5) * gls, gcl = m.Gc / m.ls, hgcl = T(0.5) * gcl;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T G[D][D], Gs[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        G[i][k] = gu[i][k][q];
        Gs[i][k] = gs[i][k][q];
      }
    StrainSym<D, T> e0, e1;
    e0.set(G);
    e1.set(Gs);
    T e01 = T(0);  // eps(u) : eps(s), raw
#pragma unroll
    for (int i = 0; i < D; ++i) e01 += G[i][i] * Gs[i][i];
#pragma unroll
    for (int j = 0; j < (D == 3 ? 3 : 1); ++j) e01 += T(0.5) * e0.off[j] * e1.off[j];
    const T psi0 = hl * e0.tr * e0.tr + mu2 * e0.ee;
    const T psi2 = hl * e1.tr * e1.tr + mu2 * e1.ee;
    const T psi1 = lam2 * e0.tr * e1.tr + T(2) * mu2 * e01;
    const T omc = T(1) - cv[q], s = sc[q];
    const T g0 = omk * omc * omc + m.k;
    const T g1 = T(-2) * omk * omc * s;
    const T g2 = omk * s * s;
    T cg = 0, gg = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const T u = gc[k][q], v = gsc[k][q];
      cg += u * v;
      gg += v * v;
    }
    const T t0 = ph * e0.tr, t1 = ph * e1.tr;
    a1 += g0 * psi1 + g1 * psi0 + (g0 * t1 + g1 * t0) + gcl * cv[q] * s + gls * cg;
    a2 += g0 * psi2 + g1 * psi1 + g2 * psi0 + (g1 * t1 + g2 * t0) + hgcl * s * s + hgls * gg;
    a3 += g1 * psi2 + g2 * psi1 + g2 * t1;
    a4 += g2 * psi2;
  }
  a[0] = m.w * a1; a[1] = m.w * a2; a[2] = m.w * a3; a[3] = m.w * a4;
}

// Gradient: u-rows  int g (sigma + p I) : grad phi,
//           c-row   int [g'(psi + p tr) + Gc c/ls] phi + Gc ls grad c . grad phi
template <int D, class T>
__device__ __forceinline__ void elem_gradient(const T (*xe)[1 << D], const Mat<T>& m,
                                              T (*out)[1 << D]) {
  constexpr int NQ = 1 << D;
  T gu[D][D][NQ], cv[NQ], gc[D][NQ], dummy[NQ];
#pragma unroll
  for (int i = 0; i < D; ++i) interp<D, T>(xe[i], dummy, gu[i]);
  interp<D, T>(xe[D], cv, gc);
  T su[D][D][NQ], s0[NQ], sc[D][NQ];
  const T omk = T(1) - m.k;
  const T kc = m.w * m.Gc * m.ls * m.inv_h * m.inv_h;
  const T gcl = m.Gc / m.ls;  // one division per element, not one per Gauss point
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T G[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) G[i][k] = gu[i][k][q] * m.inv_h;
    StrainSym<D, T> e;
    e.set(G);
    const T psi = T(0.5) * m.lam * e.tr * e.tr + m.mu * e.ee;
    const T omc = T(1) - cv[q];
    const T g = omk * omc * omc + m.k;
    const T dg = T(-2) * omk * omc;
    // weight and 1/h of the test gradient folded into the coefficient
    const T wg = m.w * m.inv_h * g;
    const T dia = m.lam * e.tr + m.p, wgm = wg * m.mu;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      su[i][i][q] = wg * (dia + T(2) * m.mu * G[i][i]);
#pragma unroll
      for (int k = i + 1; k < D; ++k) {
        const T v = wgm * e.off[sym_index<D>(i, k) - D];
        su[i][k][q] = v;
        su[k][i][q] = v;
      }
    }
    s0[q] = m.w * (dg * (psi + m.p * e.tr) + gcl * cv[q]);
#pragma unroll
    for (int k = 0; k < D; ++k) sc[k][q] = kc * gc[k][q];
  }
#pragma unroll
  for (int i = 0; i < D; ++i) test<D, T>(nullptr, su[i], out[i]);
  test<D, T>(s0, sc, out[D]);
}

// Gradient difference grad E_e(x + s) - grad E_e(x), written so that every
// term is of order one or higher in s (no difference of two gradients is
// formed; for c' = c + s_c, u' = u + s_u):
//   u-rows  int [g(c') sigma(s_u) + (g(c') - g(c)) (sigma(u) + p I)] : grad phi
//   c-row   int [g'(c') (psi_1 + psi(s_u) + p tr s_u)
//                + (g'(c') - g'(c)) (psi(u) + p tr u) + Gc s_c/ls] phi
//               + Gc ls grad s_c . grad phi
// with psi_1 = lam tr(u) tr(s_u) + 2 mu eps(u) : eps(s_u),
// g(c') - g(c) = (1-k) s_c (s_c - 2 (1-c)) and g'(c') - g'(c) = 2 (1-k) s_c.
template <int D, class T>
__device__ __forceinline__ void elem_gradient_diff(const T (*xe)[1 << D], const T (*se)[1 << D],
                                                   const Mat<T>& m, T (*out)[1 << D]) {
  constexpr int NQ = 1 << D;
  T su[D][D][NQ], s0[NQ], sc[D][NQ];
  {
    T gu[D][D][NQ], cv[NQ], gcx[D][NQ], dummy[NQ];
    T gs[D][D][NQ], scv[NQ], gsc[D][NQ];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      interp<D, T>(xe[i], dummy, gu[i]);
      interp<D, T>(se[i], dummy, gs[i]);
    }
    interp<D, T>(xe[D], cv, gcx);
    interp<D, T>(se[D], scv, gsc);
    const T omk = T(1) - m.k;
    const T kc = m.w * m.Gc * m.ls * m.inv_h * m.inv_h;
    const T gcl = m.Gc / m.ls;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T G[D][D], Gs[D][D];
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          G[i][k] = gu[i][k][q] * m.inv_h;
          Gs[i][k] = gs[i][k][q] * m.inv_h;
        }
      StrainSym<D, T> e0, e1;
      e0.set(G);
      e1.set(Gs);
      T e01 = T(0);
#pragma unroll
      for (int i = 0; i < D; ++i) e01 += G[i][i] * Gs[i][i];
#pragma unroll
      for (int j = 0; j < (D == 3 ? 3 : 1); ++j) e01 += T(0.5) * e0.off[j] * e1.off[j];
      const T psi0 = T(0.5) * m.lam * e0.tr * e0.tr + m.mu * e0.ee;
      const T psi2 = T(0.5) * m.lam * e1.tr * e1.tr + m.mu * e1.ee;
      const T psi1 = m.lam * e0.tr * e1.tr + T(2) * m.mu * e01;
      const T omc = T(1) - cv[q], sq = scv[q], omc1 = omc - sq;
      const T g1 = omk * omc1 * omc1 + m.k;         // g(c')
      const T dg = omk * sq * (sq - T(2) * omc);      // g(c') - g(c)
      const T dp1 = T(-2) * omk * omc1;               // g'(c')
      const T wg1 = m.w * m.inv_h * g1, wdg = m.w * m.inv_h * dg;
      const T d0 = m.lam * e0.tr + m.p, d1 = m.lam * e1.tr;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        su[i][i][q] = wg1 * (d1 + T(2) * m.mu * Gs[i][i]) + wdg * (d0 + T(2) * m.mu * G[i][i]);
#pragma unroll
        for (int k = i + 1; k < D; ++k) {
          const int j = sym_index<D>(i, k) - D;
          const T v = m.mu * (wg1 * e1.off[j] + wdg * e0.off[j]);
          su[i][k][q] = v;
          su[k][i][q] = v;
        }
      }
      s0[q] = m.w * (dp1 * (psi1 + psi2 + m.p * e1.tr) + T(2) * omk * sq * (psi0 + m.p * e0.tr) +
                     gcl * sq);
#pragma unroll
      for (int k = 0; k < D; ++k) sc[k][q] = kc * gsc[k][q];
    }
  }
#pragma unroll
  for (int i = 0; i < D; ++i) test<D, T>(nullptr, su[i], out[i]);
  test<D, T>(s0, sc, out[D]);
}

// ---------------------------------------------------------------- Hessian
// The Hessian at x applied to v,
//   u-rows  int [g sigma(v_u) + g' v_c (sigma(u) + p I)] : grad phi
//   c-row   int [g' (sigma(u) + p I) : eps(v_u) + (g''(psi + p tr) + Gc/ls) v_c] phi
//               + Gc ls grad v_c . grad phi
// depends on x only through three Gauss-point coefficients (raw nodal
// differences for the gradients, 1/h and the weight folded in):
//   A = w g / h^2,   B = w g' (sigma(u) + p I) / h  (symmetric),
//   M = w (g''(psi + p tr) + Gc/ls).
// Under Hessian lagging they are computed once per lagged point and every
// Hessian-vector product then needs only the v-part below.
// cf[q][0] = A, cf[q][1] = M, cf[q][2 + s] = B_s
template <int D, class T>
__device__ __forceinline__ void hess_coef(const T (*xe)[1 << D], const Mat<T>& m,
                                          T (*cf)[NCoef<D>::value]) {
  constexpr int NQ = 1 << D;
  T gu[D][D][NQ], cv[NQ], gdummy[D][NQ], dummy[NQ];
#pragma unroll
  for (int i = 0; i < D; ++i) interp<D, T>(xe[i], dummy, gu[i]);
  interp<D, T>(xe[D], cv, gdummy);
  const T omk = T(1) - m.k;
  const T wh2 = m.w * m.inv_h * m.inv_h, wh = m.w * m.inv_h;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T G[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) G[i][k] = gu[i][k][q] * m.inv_h;
    T tr = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) tr += G[i][i];
    T ee = T(0);  // eps : eps
#pragma unroll
    for (int i = 0; i < D; ++i) {
      ee += G[i][i] * G[i][i];
#pragma unroll
      for (int k = i + 1; k < D; ++k) {
        const T e = T(0.5) * (G[i][k] + G[k][i]);
        ee += T(2) * e * e;
      }
    }
    const T psi = T(0.5) * m.lam * tr * tr + m.mu * ee;
    const T omc = T(1) - cv[q];
    const T g = omk * omc * omc + m.k;
    const T dgw = T(-2) * omk * omc * wh;
    cf[q][0] = wh2 * g;
    cf[q][1] = m.w * (T(2) * omk * (psi + m.p * tr) + m.Gc / m.ls);
    const T diag = m.lam * tr + m.p;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      cf[q][2 + i] = dgw * (diag + T(2) * m.mu * G[i][i]);
#pragma unroll
      for (int k = i + 1; k < D; ++k) cf[q][2 + sym_index<D>(i, k)] = dgw * m.mu * (G[i][k] + G[k][i]);
    }
  }
}

// The v-part: out = H v from the coefficients of the element's Gauss points.
template <int D, class T>
__device__ __forceinline__ void hess_apply(const T (*ve)[1 << D], const T (*cf)[NCoef<D>::value],
                                           const Mat<T>& m, T (*out)[1 << D]) {
  constexpr int NQ = 1 << D;
  T su[D][D][NQ], s0[NQ], sc[D][NQ];
  {
    T gv[D][D][NQ], vc[NQ], gvc[D][NQ], dummy[NQ];
#pragma unroll
    for (int i = 0; i < D; ++i) interp<D, T>(ve[i], dummy, gv[i]);
    interp<D, T>(ve[D], vc, gvc);
    const T kc = m.w * m.Gc * m.ls * m.inv_h * m.inv_h;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const T A = cf[q][0], M = cf[q][1];
      T trr = T(0);
#pragma unroll
      for (int i = 0; i < D; ++i) trr += gv[i][i][q];
      const T lt = m.lam * trr, am = A * m.mu;
      T c0 = M * vc[q];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const T Bii = cf[q][2 + i];
        su[i][i][q] = A * (lt + T(2) * m.mu * gv[i][i][q]) + vc[q] * Bii;
        c0 += Bii * gv[i][i][q];
#pragma unroll
        for (int k = i + 1; k < D; ++k) {
          const T Bik = cf[q][2 + sym_index<D>(i, k)];
          const T sik = gv[i][k][q] + gv[k][i][q];
          const T v = am * sik + vc[q] * Bik;
          su[i][k][q] = v;
          su[k][i][q] = v;
          c0 += Bik * sik;
        }
      }
      s0[q] = c0;
#pragma unroll
      for (int k = 0; k < D; ++k) sc[k][q] = kc * gvc[k][q];
    }
  }
#pragma unroll
  for (int i = 0; i < D; ++i) test<D, T>(nullptr, su[i], out[i]);
  test<D, T>(s0, sc, out[D]);
}

template <int D, class T>
__device__ __forceinline__ void elem_hessvec(const T (*xe)[1 << D], const T (*ve)[1 << D],
                                             const Mat<T>& m, T (*out)[1 << D]) {
  T cf[1 << D][NCoef<D>::value];
  hess_coef<D, T>(xe, m, cf);
  hess_apply<D, T>(ve, cf, m, out);
}

// Diagonal of the Hessian (Jacobi preconditioner):
//   u_i dof of corner a: sum_q w g [lam (d_i phi_a)^2 + mu (|grad phi_a|^2 + (d_i phi_a)^2)]
//   c dof:              sum_q w [(g''(psi + p tr) + Gc/ls) phi_a^2 + Gc ls |grad phi_a|^2]
template <int D, class T>
__device__ __forceinline__ void elem_hessdiag(const T (*xe)[1 << D], const Mat<T>& m,
                                              T (*out)[1 << D]) {
  constexpr int NQ = 1 << D;
  T gu[D][D][NQ], cv[NQ], gdummy[D][NQ], dummy[NQ];
#pragma unroll
  for (int i = 0; i < D; ++i) interp<D, T>(xe[i], dummy, gu[i]);
  interp<D, T>(xe[D], cv, gdummy);
  T gq[NQ], mq[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T G[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) G[i][k] = gu[i][k][q] * m.inv_h;
    Strain<D, T> e;
    e.set(G);
    const T psi = T(0.5) * m.lam * e.tr * e.tr + m.mu * e.ddot(e);
    const T omk = T(1) - m.k, omc = T(1) - cv[q];
    gq[q] = m.w * (omk * omc * omc + m.k);
    mq[q] = m.w * (T(2) * omk * (psi + m.p * e.tr) + m.Gc / m.ls);
  }
  const T h2 = m.inv_h * m.inv_h;
#pragma unroll
  for (int a = 0; a < NQ; ++a) {
    T du[D], dc = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) du[i] = T(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      // 1D factors: N(q, a) = XI1 if q == a along the axis, else XI0
      T n1[D];
#pragma unroll
      for (int k = 0; k < D; ++k) n1[k] = (((q >> k) & 1) == ((a >> k) & 1)) ? T(PF_XI1) : T(PF_XI0);
      T phi = T(1);
#pragma unroll
      for (int k = 0; k < D; ++k) phi *= n1[k];
      T d2[D], g2 = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        T t = T(1);
#pragma unroll
        for (int j = 0; j < D; ++j)
          if (j != k) t *= n1[j] * n1[j];
        d2[k] = t * h2;
        g2 += d2[k];
      }
#pragma unroll
      for (int i = 0; i < D; ++i) du[i] += gq[q] * (m.lam * d2[i] + m.mu * (g2 + d2[i]));
      dc += mq[q] * phi * phi + m.w * m.Gc * m.ls * g2;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) out[i][a] = du[i];
    out[D][a] = dc;
  }
}

}  // namespace pf
