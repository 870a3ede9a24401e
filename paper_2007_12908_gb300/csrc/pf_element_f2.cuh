// Packed FP32 variant of the 3D Q1 Hessian-vector element operation.  The
// two Gauss points of an element along x form one float2 (lane qx), so the
// sum-factorised interpolation, the Gauss-point algebra and the adjoint
// contraction run on the paired FP32 FMA/ADD/MUL instructions of sm_100+
// (__ffma2_rn etc.).  Pairs are indexed pp = qy + 2 qz; Gauss point
// q = qx + 2 qy + 4 qz of the scalar code is lane qx of pair pp.
#pragma once
#include <cuda_runtime.h>

#include "pf_element.cuh"

namespace pf {
namespace p2 {

__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
// a - b, exact: b * (-1) + a rounds once
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc(-1.f), a); }

// Values and raw-difference gradients of one field at the 8 Gauss points,
// as 4 pairs.  The x-derivative is constant along x and returned scalar.
struct Interp {
  float2 val[4], gy[4], gz[4];
  float gx[4];
};

__device__ __forceinline__ void interp(const float f[8], Interp& o) {
  const float x0 = float(PF_XI0), x1 = float(PF_XI1);
  const float2 xi = make_float2(x0, x1);
  float2 X[2][2];  // [ay][az], lanes qx
  float DX[2][2];
#pragma unroll
  for (int az = 0; az < 2; ++az)
#pragma unroll
    for (int ay = 0; ay < 2; ++ay) {
      const float v0 = f[2 * ay + 4 * az], d = f[1 + 2 * ay + 4 * az] - v0;
      DX[ay][az] = d;
      X[ay][az] = fma2(bc(d), xi, bc(v0));
    }
  float2 XY[2][2];  // [qy][az]
  float2 DY[2];     // [az]
  float DXY[2][2];  // [qy][az]
#pragma unroll
  for (int az = 0; az < 2; ++az) {
    const float2 d = sub2(X[1][az], X[0][az]);
    DY[az] = d;
    XY[0][az] = fma2(d, bc(x0), X[0][az]);
    XY[1][az] = fma2(d, bc(x1), X[0][az]);
    const float dd = DX[1][az] - DX[0][az];
    DXY[0][az] = fmaf(x0, dd, DX[0][az]);
    DXY[1][az] = fmaf(x1, dd, DX[0][az]);
  }
#pragma unroll
  for (int qy = 0; qy < 2; ++qy) {
    const float2 d = sub2(XY[qy][1], XY[qy][0]);
    o.val[qy] = fma2(d, bc(x0), XY[qy][0]);
    o.val[qy + 2] = fma2(d, bc(x1), XY[qy][0]);
    o.gz[qy] = d;
    o.gz[qy + 2] = d;
    const float dd = DXY[qy][1] - DXY[qy][0];
    o.gx[qy] = fmaf(x0, dd, DXY[qy][0]);
    o.gx[qy + 2] = fmaf(x1, dd, DXY[qy][0]);
  }
  const float2 d = sub2(DY[1], DY[0]);
  const float2 a = fma2(d, bc(x0), DY[0]), b = fma2(d, bc(x1), DY[0]);
  o.gy[0] = a; o.gy[1] = a;
  o.gy[2] = b; o.gy[3] = b;
}

// Adjoint of interp: r[a] = sum over Gauss points of s0 N_a + sx Dx_a +
// sy Dy_a + sz Dz_a (raw derivatives).  WITH_S0 = false skips the value term.
template <bool WITH_S0>
__device__ __forceinline__ void test(const float2 s0[4], const float2 sx[4], const float2 sy[4],
                                     const float2 sz[4], float r[8]) {
  const float x0 = float(PF_XI0), x1 = float(PF_XI1);
  // z pass: XYb[qy][az] (pairs), DXYb[qy][az] (scalar), DYb[az] (pairs)
  float2 XYb[2][2];
  float DXYb[2][2];
  float2 DYb[2];
#pragma unroll
  for (int qy = 0; qy < 2; ++qy) {
    const float2 zs = add2(sz[qy], sz[qy + 2]);
    if (WITH_S0) {
      XYb[qy][0] = sub2(fma2(bc(x1), s0[qy], mul2(bc(x0), s0[qy + 2])), zs);
      XYb[qy][1] = add2(fma2(bc(x0), s0[qy], mul2(bc(x1), s0[qy + 2])), zs);
    } else {
      XYb[qy][0] = sub2(make_float2(0.f, 0.f), zs);
      XYb[qy][1] = zs;
    }
    const float a = sx[qy].x + sx[qy].y, b = sx[qy + 2].x + sx[qy + 2].y;
    DXYb[qy][0] = fmaf(x1, a, x0 * b);
    DXYb[qy][1] = fmaf(x0, a, x1 * b);
  }
  {
    const float2 a = add2(sy[0], sy[1]), b = add2(sy[2], sy[3]);
    DYb[0] = fma2(bc(x1), a, mul2(bc(x0), b));
    DYb[1] = fma2(bc(x0), a, mul2(bc(x1), b));
  }
  // y pass: Xb[ay][az] (pairs), DXb[ay][az] (scalar)
  float2 Xb[2][2];
  float DXb[2][2];
#pragma unroll
  for (int az = 0; az < 2; ++az) {
    Xb[0][az] = sub2(fma2(bc(x1), XYb[0][az], mul2(bc(x0), XYb[1][az])), DYb[az]);
    Xb[1][az] = add2(fma2(bc(x0), XYb[0][az], mul2(bc(x1), XYb[1][az])), DYb[az]);
    DXb[0][az] = fmaf(x1, DXYb[0][az], x0 * DXYb[1][az]);
    DXb[1][az] = fmaf(x0, DXYb[0][az], x1 * DXYb[1][az]);
  }
  // x pass: lanes qx combine into the two corners along x
#pragma unroll
  for (int az = 0; az < 2; ++az)
#pragma unroll
    for (int ay = 0; ay < 2; ++ay) {
      const float2 v = Xb[ay][az];
      r[2 * ay + 4 * az] = fmaf(x1, v.x, fmaf(x0, v.y, -DXb[ay][az]));
      r[1 + 2 * ay + 4 * az] = fmaf(x0, v.x, fmaf(x1, v.y, DXb[ay][az]));
    }
}

// The lagged Gauss-point coefficients (see hess_coef) for the 4 pairs:
// A, M and the symmetric B in sym order 00, 11, 22, 01, 02, 12.
struct Coef {
  float2 A, M, B[6];
};

__device__ __forceinline__ void coef(const float (*xe)[8], const Mat<float>& m, Coef cf[4]) {
  Interp u[3], c;
#pragma unroll
  for (int i = 0; i < 3; ++i) interp(xe[i], u[i]);
  interp(xe[3], c);
  const float omk = 1.f - m.k;
  const float wh2 = m.w * m.inv_h * m.inv_h, wh = m.w * m.inv_h;
#pragma unroll
  for (int pp = 0; pp < 4; ++pp) {
    // G[i][k] = d u_i / d x_k (physical)
    float2 G[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      G[i][0] = mul2(bc(u[i].gx[pp]), bc(m.inv_h));
      G[i][1] = mul2(u[i].gy[pp], bc(m.inv_h));
      G[i][2] = mul2(u[i].gz[pp], bc(m.inv_h));
    }
    const float2 tr = add2(add2(G[0][0], G[1][1]), G[2][2]);
    const float2 s01 = add2(G[0][1], G[1][0]), s02 = add2(G[0][2], G[2][0]), s12 = add2(G[1][2], G[2][1]);
    float2 ee = mul2(G[0][0], G[0][0]);
    ee = fma2(G[1][1], G[1][1], ee);
    ee = fma2(G[2][2], G[2][2], ee);
    const float2 half = bc(0.5f);
    ee = fma2(mul2(half, s01), s01, ee);
    ee = fma2(mul2(half, s02), s02, ee);
    ee = fma2(mul2(half, s12), s12, ee);
    const float2 psi = fma2(mul2(bc(0.5f * m.lam), tr), tr, mul2(bc(m.mu), ee));
    const float2 omc = sub2(bc(1.f), c.val[pp]);
    const float2 g = fma2(mul2(bc(omk), omc), omc, bc(m.k));
    const float2 dgw = mul2(bc(-2.f * omk * wh), omc);
    cf[pp].A = mul2(bc(wh2), g);
    cf[pp].M = mul2(bc(m.w), fma2(bc(2.f * omk), fma2(bc(m.p), tr, psi), bc(m.Gc / m.ls)));
    const float2 diag = fma2(bc(m.lam), tr, bc(m.p));
    const float2 tmu = bc(2.f * m.mu);
    cf[pp].B[0] = mul2(dgw, fma2(tmu, G[0][0], diag));
    cf[pp].B[1] = mul2(dgw, fma2(tmu, G[1][1], diag));
    cf[pp].B[2] = mul2(dgw, fma2(tmu, G[2][2], diag));
    const float2 dgm = mul2(dgw, bc(m.mu));
    cf[pp].B[3] = mul2(dgm, s01);
    cf[pp].B[4] = mul2(dgm, s02);
    cf[pp].B[5] = mul2(dgm, s12);
  }
}

__device__ __forceinline__ void apply(const float (*ve)[8], const Coef cf[4], const Mat<float>& m,
                                      float (*out)[8]) {
  float2 su[3][3][4], s0[4], sc[3][4];
  {
    Interp v[3], vc;
#pragma unroll
    for (int i = 0; i < 3; ++i) interp(ve[i], v[i]);
    interp(ve[3], vc);
    const float kc = m.w * m.Gc * m.ls * m.inv_h * m.inv_h;
#pragma unroll
    for (int pp = 0; pp < 4; ++pp) {
      float2 G[3][3];  // raw differences of v_u
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        G[i][0] = bc(v[i].gx[pp]);
        G[i][1] = v[i].gy[pp];
        G[i][2] = v[i].gz[pp];
      }
      const float2 A = cf[pp].A, M = cf[pp].M, w = vc.val[pp];
      const float2 trr = add2(add2(G[0][0], G[1][1]), G[2][2]);
      const float2 lt = mul2(bc(m.lam), trr), am = mul2(A, bc(m.mu));
      const float2 tmu = bc(2.f * m.mu);
      float2 c0 = mul2(M, w);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float2 Bii = cf[pp].B[i];
        su[i][i][pp] = fma2(w, Bii, mul2(A, fma2(tmu, G[i][i], lt)));
        c0 = fma2(Bii, G[i][i], c0);
      }
      const int ii[3] = {0, 0, 1}, kk[3] = {1, 2, 2};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float2 Bik = cf[pp].B[3 + j];
        const float2 sik = add2(G[ii[j]][kk[j]], G[kk[j]][ii[j]]);
        const float2 val = fma2(am, sik, mul2(w, Bik));
        su[ii[j]][kk[j]][pp] = val;
        su[kk[j]][ii[j]][pp] = val;
        c0 = fma2(Bik, sik, c0);
      }
      s0[pp] = c0;
      sc[0][pp] = bc(kc * vc.gx[pp]);
      sc[1][pp] = mul2(bc(kc), vc.gy[pp]);
      sc[2][pp] = mul2(bc(kc), vc.gz[pp]);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) test<false>(nullptr, su[i][0], su[i][1], su[i][2], out[i]);
  test<true>(s0, sc[0], sc[1], sc[2], out[3]);
}

__device__ __forceinline__ void elem_hessvec(const float (*xe)[8], const float (*ve)[8],
                                             const Mat<float>& m, float (*out)[8]) {
  Coef cf[4];
  coef(xe, m, cf);
  apply(ve, cf, m, out);
}

}  // namespace p2
}  // namespace pf
