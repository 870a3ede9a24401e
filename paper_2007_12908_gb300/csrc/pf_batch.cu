// Batched operators over many 2D instances of uneven size (the batched
// workload: independent fracture networks, Sec. 5 scenarios drawn at
// several resolutions).  One persistent launch covers every instance's
// finest grid: the work list is the instances' node rows, cut into strips
// of 63 node columns, and each warp of the grid takes an equal contiguous
// range of (instance, strip, row) steps, so uneven instances need no
// per-instance launch and the grid ends together.
//
// A warp marches up its strip one element row at a time.  Lane j evaluates
// the elements of columns c0 + j and c0 + 32 + j as the two halves of
// float2 values (paired FP32 instructions), reading only node row y + 1 per
// step (the row below is still in registers); a node's right-hand element
// is in the next lane, reached by a shuffle.  Corner contributions are added per
// node in a fixed order -- left element before right, the element row
// below before the one above -- so the product is the same bit for bit for
// every grid size, strip cut and warp range (and across autotuned
// variants).  Nothing is staged in shared memory and there are no
// barriers.
//
// Per-instance reductions (v . Hv for the CG curvature, the energy) are
// segmented: one partial per node row (per element row for the energy),
// then per instance a fixed-order two-level sum.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pf_element_f2.cuh"
#include "pf_hier.h"

namespace pf {
namespace {

constexpr int kStripCols = 63;   // node columns a warp owns (64 element columns)
constexpr int kSegChunk = 2048;  // partials per block of the segmented sum
constexpr unsigned kFull = 0xffffffffu;
constexpr int kHessThreads = 128;  // 4 warps per block; 3 blocks per SM fit its 168 registers

struct BInst {
  Geom g;            // finest grid of the instance
  Mat<double> md;    // its material (FP64, energy)
  long long row0;    // first global row step (strips * n1 steps per instance)
  long long erow0;   // first global element row (energy)
  int strips;        // ceil(n0 / 63)
  // FP32 constants of the paired Hessian (Gauss-point algebra with the
  // 1/h scalings folded in; raw nodal differences in, see hess2_pair)
  float lam, mu2, mu, lam_h, mu2_h, mu_h, p;
  float cA, cAk, cdg, cpl, cpm, cpt, cM2, cM0, kc;
};

struct BVec {
  const float* x;
  const float* v;
  float* y;
};

using p2::add2;
using p2::bc;
using p2::fma2;
using p2::mul2;
using p2::sub2;

// Values and raw-difference gradients at the 4 Gauss points (q = qx + 2 qy)
// of a Q1 field given at corners a = ax + 2 ay.
struct I2 {
  float2 val[4], gx[4], gy[4];
};
__device__ __forceinline__ void interp_pair(const float2 f[4], I2& o) {
  const float x0 = float(PF_XI0), x1 = float(PF_XI1);
  float2 X[2][2], DX[2];  // X[qx][ay]
#pragma unroll
  for (int ay = 0; ay < 2; ++ay) {
    const float2 d = sub2(f[1 + 2 * ay], f[2 * ay]);
    DX[ay] = d;
    X[0][ay] = fma2(bc(x0), d, f[2 * ay]);
    X[1][ay] = fma2(bc(x1), d, f[2 * ay]);
  }
#pragma unroll
  for (int qx = 0; qx < 2; ++qx) {
    const float2 d = sub2(X[qx][1], X[qx][0]);
    o.val[qx] = fma2(bc(x0), d, X[qx][0]);
    o.val[qx + 2] = fma2(bc(x1), d, X[qx][0]);
    o.gy[qx] = d;
    o.gy[qx + 2] = d;
  }
  const float2 d = sub2(DX[1], DX[0]);
  const float2 a = fma2(bc(x0), d, DX[0]), b = fma2(bc(x1), d, DX[0]);
  o.gx[0] = a; o.gx[1] = a;
  o.gx[2] = b; o.gx[3] = b;
}

// Adjoint of interp_pair: r[a] = sum_q s0[q] N_a(q) + sx[q] Dx_a(q) +
// sy[q] Dy_a(q) with raw differences (s0 null: no value term).
template <bool S0>
__device__ __forceinline__ void test_pair(const float2* s0, const float2 sx[4], const float2 sy[4],
                                          float2 r[4]) {
  const float x0 = float(PF_XI0), x1 = float(PF_XI1);
  float2 Xb[2][2];  // [qx][ay]
#pragma unroll
  for (int qx = 0; qx < 2; ++qx) {
    const float2 ys = add2(sy[qx], sy[qx + 2]);
    if constexpr (S0) {
      const float2 lo = fma2(bc(x0), s0[qx + 2], mul2(bc(x1), s0[qx]));
      const float2 hi = fma2(bc(x1), s0[qx + 2], mul2(bc(x0), s0[qx]));
      Xb[qx][0] = sub2(lo, ys);
      Xb[qx][1] = add2(hi, ys);
    } else {
      Xb[qx][0] = mul2(bc(-1.f), ys);
      Xb[qx][1] = ys;
    }
  }
  const float2 a = add2(sx[0], sx[1]), b = add2(sx[2], sx[3]);
  const float2 dx0 = fma2(bc(x0), b, mul2(bc(x1), a));
  const float2 dx1 = fma2(bc(x1), b, mul2(bc(x0), a));
#pragma unroll
  for (int ay = 0; ay < 2; ++ay) {
    const float2 dxb = ay ? dx1 : dx0;
    const float2 l = fma2(bc(x0), Xb[1][ay], mul2(bc(x1), Xb[0][ay]));
    const float2 h = fma2(bc(x1), Xb[1][ay], mul2(bc(x0), Xb[0][ay]));
    r[2 * ay] = sub2(l, dxb);
    r[1 + 2 * ay] = add2(h, dxb);
  }
}

// Hessian of the pressurised AT2 element energy at xe applied to ve, for two
// elements at once (lanes .x and .y).  Fields 0, 1: displacement, 2: phase
// field.  Per Gauss point, with G = grad u, e = sym G, g(c) = (1-k)(1-c)^2 + k:
//   A = w g / h^2,  B = w g'(c) (sigma(u) + p I) / h,
//   M = w (g''(c) (psi(u) + p tr e) + Gc / l_s),
// and the product's Gauss-point stresses
//   u_i: A sigma(grad v_u)_ik + v_c B_ik,  c: M v_c + B : grad v_u,
//   grad c: w Gc l_s grad v_c,
// contracted with the test functions' gradients and values.
__device__ __forceinline__ void hess2_pair(const float2 xe[3][4], const float2 ve[3][4],
                                           const BInst& I, float2 out[3][4]) {
  I2 xu0, xu1, xc, vu0, vu1, vcf;
  interp_pair(xe[0], xu0);
  interp_pair(xe[1], xu1);
  interp_pair(xe[2], xc);
  interp_pair(ve[0], vu0);
  interp_pair(ve[1], vu1);
  interp_pair(ve[2], vcf);
  float2 su0x[4], su0y[4], su1x[4], su1y[4], s0[4], scx[4], scy[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    // coefficients at the lagged point (raw differences; 1/h folded in)
    const float2 g00 = xu0.gx[q], g01 = xu0.gy[q], g10 = xu1.gx[q], g11 = xu1.gy[q];
    const float2 omc = fma2(xc.val[q], bc(-1.f), bc(1.f));
    const float2 A = fma2(bc(I.cA), mul2(omc, omc), bc(I.cAk));
    const float2 dgw = mul2(bc(I.cdg), omc);
    const float2 tr = add2(g00, g11), s01 = add2(g01, g10);
    const float2 ee = fma2(mul2(bc(0.5f), s01), s01, fma2(g11, g11, mul2(g00, g00)));
    const float2 inner = fma2(bc(I.cpt), tr, fma2(bc(I.cpm), ee, mul2(bc(I.cpl), mul2(tr, tr))));
    const float2 M = fma2(bc(I.cM2), inner, bc(I.cM0));
    const float2 diag = fma2(bc(I.lam_h), tr, bc(I.p));
    const float2 B00 = mul2(dgw, fma2(bc(I.mu2_h), g00, diag));
    const float2 B11 = mul2(dgw, fma2(bc(I.mu2_h), g11, diag));
    const float2 B01 = mul2(dgw, mul2(bc(I.mu_h), s01));
    // the direction's Gauss-point values
    const float2 v00 = vu0.gx[q], v01 = vu0.gy[q], v10 = vu1.gx[q], v11 = vu1.gy[q];
    const float2 vc = vcf.val[q];
    const float2 lt = mul2(bc(I.lam), add2(v00, v11));
    const float2 vs = add2(v01, v10);
    su0x[q] = fma2(A, fma2(bc(I.mu2), v00, lt), mul2(vc, B00));
    su1y[q] = fma2(A, fma2(bc(I.mu2), v11, lt), mul2(vc, B11));
    const float2 off = fma2(mul2(A, bc(I.mu)), vs, mul2(vc, B01));
    su0y[q] = off;
    su1x[q] = off;
    s0[q] = fma2(B01, vs, fma2(B11, v11, fma2(B00, v00, mul2(M, vc))));
    scx[q] = mul2(bc(I.kc), vcf.gx[q]);
    scy[q] = mul2(bc(I.kc), vcf.gy[q]);
  }
  test_pair<false>(nullptr, su0x, su0y, out[0]);
  test_pair<false>(nullptr, su1x, su1y, out[1]);
  test_pair<true>(s0, scx, scy, out[2]);
}

// One row of node values of a vector (3 planes) as element-pair corners:
// lane j's elements are columns e1 = c0 + j and e2 = c0 + 32 + j, so
// L = (node e1, node e2) holds their left corners and R = (node e1 + 1,
// node e2 + 1) their right ones; no node value sits in two pairs of a lane.
// Interior rows of interior strips (every column and the row inside the
// grid, a warp-uniform test) load with no bounds checks; elsewhere values
// outside the grid read as 0 (they only enter elements outside the grid,
// whose outputs are dropped).  Indices are 32-bit: pf_batch_create refuses
// instances with 3 N >= 2^31.
struct Row2 {
  float2 L[3], R[3];
};
template <bool EDGE>
__device__ __forceinline__ void load_row(const float* __restrict__ src, int N, int n0, int n1,
                                         int e1, int y, Row2& r) {
  if constexpr (!EDGE) {
    const float* p = src + (y * n0 + e1);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      r.L[f] = make_float2(__ldg(p + f * N), __ldg(p + f * N + 32));
      r.R[f] = make_float2(__ldg(p + f * N + 1), __ldg(p + f * N + 33));
    }
  } else {
    const bool ry = y >= 0 && y < n1;
    const bool i0 = ry && e1 >= 0 && e1 < n0, i1 = ry && e1 + 1 < n0;
    const bool i32 = ry && e1 + 32 < n0, i33 = ry && e1 + 33 < n0;
    const int b = ry ? y * n0 + e1 : 0;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const float* p = src + f * N + b;
      r.L[f] = make_float2(i0 ? __ldg(p) : 0.f, i32 ? __ldg(p + 32) : 0.f);
      r.R[f] = make_float2(i1 ? __ldg(p + 1) : 0.f, i33 ? __ldg(p + 33) : 0.f);
    }
  }
}
__device__ __forceinline__ void load_row(bool interior, const float* __restrict__ src, int N,
                                         int n0, int n1, int e1, int y, Row2& r) {
  if (interior && y >= 0 && y < n1) load_row<false>(src, N, n0, n1, e1, y, r);
  else load_row<true>(src, N, n0, n1, e1, y, r);
}

// Rows [r0, r0 + rows) of strip `strip` of one instance: the Hessian at x
// applied to v, written to y; with DOT, the node rows' v . Hv to
// rowdot[0 .. rows).  The strip evaluates element columns c0 .. c0 + 63
// (c0 = 63 strip - 1) and owns node columns c0 + 1 .. c0 + 63: lane j the
// nodes c0 + 1 + j (right corner of e1 plus left corner of the next
// element) and, for j < 31, c0 + 33 + j.
template <bool DOT>
__device__ __forceinline__ void hess2_strip(const BInst& I, const BVec& V, int strip, int r0,
                                            int rows, int lane, double* __restrict__ rowdot) {
  const int n0 = I.g.n[0], n1 = I.g.n[1], N = int(I.g.N);
  const int c0 = strip * kStripCols - 1;
  const int e1 = c0 + lane;
  const bool interior = strip > 0 && c0 + 64 < n0;  // columns c0 .. c0 + 64 inside (warp-uniform)
  const bool ok1 = e1 >= 0 && e1 < n0 - 1, ok2 = e1 + 32 < n0 - 1;
  const bool all_el = __all_sync(kFull, ok1 && ok2);
  const bool own1 = e1 + 1 < n0, own2 = lane < 31 && e1 + 33 < n0;
  const int src_lane = (lane + 1) & 31;  // the lane holding the element right of e1 (lane 31: e2 of lane 0)
  Row2 bx, bv, tx, tv, px, pv;
  load_row(interior, V.x, N, n0, n1, e1, r0 - 1, bx);
  load_row(interior, V.v, N, n0, n1, e1, r0 - 1, bv);
  load_row(interior, V.x, N, n0, n1, e1, r0, px);  // the next row, loaded one step ahead
  load_row(interior, V.v, N, n0, n1, e1, r0, pv);
  float car1[3] = {0.f, 0.f, 0.f}, car2[3] = {0.f, 0.f, 0.f};
  for (int s = 0; s <= rows; ++s) {
    const int ey = r0 - 1 + s;  // element row; its top node row is ey + 1
    tx = px;
    tv = pv;
    if (s < rows) {
      load_row(interior, V.x, N, n0, n1, e1, ey + 2, px);
      load_row(interior, V.v, N, n0, n1, e1, ey + 2, pv);
    }
    float2 xe[3][4], ve[3][4];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      xe[f][0] = bx.L[f];
      xe[f][1] = bx.R[f];
      xe[f][2] = tx.L[f];
      xe[f][3] = tx.R[f];
      ve[f][0] = bv.L[f];
      ve[f][1] = bv.R[f];
      ve[f][2] = tv.L[f];
      ve[f][3] = tv.R[f];
    }
    float2 out[3][4];
    hess2_pair(xe, ve, I, out);
    const bool rowok = ey >= 0 && ey < n1 - 1;
    if (!(rowok && all_el)) {  // warp-uniform: drop elements outside the grid
      const bool a = rowok && ok1, b = rowok && ok2;
#pragma unroll
      for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (!a) out[f][k].x = 0.f;
          if (!b) out[f][k].y = 0.f;
        }
    }
    float dot = 0.f;
    float* yrow = V.y + (ey * n0 + e1 + 1);  // dereferenced only for ey in [r0, r0 + rows)
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      // per node the left element's corner comes first: right corner of
      // e1 (e2) plus the left corner of the element to its right
      const float sb = lane == 0 ? out[f][0].y : out[f][0].x;
      const float st = lane == 0 ? out[f][2].y : out[f][2].x;
      const float rb1 = __shfl_sync(kFull, sb, src_lane), rt1 = __shfl_sync(kFull, st, src_lane);
      const float rb2 = __shfl_down_sync(kFull, out[f][0].y, 1);
      const float rt2 = __shfl_down_sync(kFull, out[f][2].y, 1);
      const float bot1 = out[f][1].x + rb1, bot2 = out[f][1].y + rb2;
      const float top1 = out[f][3].x + rt1, top2 = out[f][3].y + rt2;
      if (s > 0) {
        const float h1 = car1[f] + bot1, h2 = car2[f] + bot2;
        if (own1) yrow[f * N] = h1;
        if (own2) yrow[f * N + 32] = h2;
        if constexpr (DOT) dot += (own1 ? h1 * bv.R[f].x : 0.f) + (own2 ? h2 * bv.R[f].y : 0.f);
      }
      car1[f] = top1;
      car2[f] = top2;
    }
    if constexpr (DOT) {
      if (s > 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(kFull, dot, o);
        if (lane == 0) rowdot[s - 1] = double(dot);
      }
    }
    bx = tx;
    bv = tv;
  }
}

__device__ __forceinline__ int find_inst(const BInst* __restrict__ inst, int n, long long s,
                                         bool elem_rows) {
  int lo = 0, hi = n - 1;  // largest i with start(i) <= s
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const long long st = elem_rows ? inst[mid].erow0 : inst[mid].row0;
    if (st <= s) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Persistent batched Hessian product: warp w takes the row steps
// [w T / W, (w + 1) T / W) of the whole batch.
template <bool DOT>
__global__ void __launch_bounds__(128, 3)
    k_batch_hess2(const BInst* __restrict__ inst, const BVec* __restrict__ vec, int n_inst,
                  long long T, double* __restrict__ rowdot) {
  const int lane = threadIdx.x & 31;
  const long long W = (long long)gridDim.x * (blockDim.x >> 5);
  const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  long long s = w * T / W;
  const long long s_end = (w + 1) * T / W;
  if (s >= s_end) return;
  int i = find_inst(inst, n_inst, s, false);
  while (s < s_end) {
    while (i + 1 < n_inst && inst[i + 1].row0 <= s) ++i;
    const BInst& I = inst[i];
    const int n1 = I.g.n[1];
    const long long local = s - I.row0;
    const int strip = int(local / n1), r0 = int(local % n1);
    const long long left = s_end - s;
    const int rows = left < (long long)(n1 - r0) ? int(left) : n1 - r0;
    hess2_strip<DOT>(I, vec[i], strip, r0, rows, lane, DOT ? rowdot + s : nullptr);
    s += rows;
  }
}

// Energy of every instance: warps take element rows from a shared counter;
// a row's elements are summed per lane in column order, then across the
// warp by a fixed butterfly, into erow[r].
__global__ void __launch_bounds__(256)
    k_batch_energy2(const BInst* __restrict__ inst, const double* const* __restrict__ xs,
                    int n_inst, long long TE, unsigned long long* counter,
                    double* __restrict__ erow) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long r = 0;
    if (lane == 0) r = atomicAdd(counter, 1ULL);
    r = __shfl_sync(kFull, r, 0);
    if ((long long)r >= TE) return;
    const int i = find_inst(inst, n_inst, (long long)r, true);
    const BInst& I = inst[i];
    const int ey = int((long long)r - I.erow0);
    const double* x = xs[i];
    double acc = 0.0;
    const long long row = (long long)ey * I.g.n[0];
    for (int ex = lane; ex < I.g.ne[0]; ex += 32) {
      double xe[3][4];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const double* pf = x + f * I.g.N + row + ex;
        xe[f][0] = pf[0];
        xe[f][1] = pf[1];
        xe[f][2] = pf[I.g.n[0]];
        xe[f][3] = pf[I.g.n[0] + 1];
      }
      acc += elem_energy<2, double>(xe, I.md);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane == 0) erow[r] = acc;
  }
}

// Segmented sums: out[i] = sum of vals[seg0[i] .. seg0[i+1]).  Block b sums
// chunk b (kSegChunk values of one segment, threads in a fixed stride
// order, then a fixed tree); the last block to finish adds each segment's
// chunk sums in chunk order.
__global__ void __launch_bounds__(256)
    k_segsum(const double* __restrict__ vals, const long long* __restrict__ seg0,
             const int* __restrict__ chunk0, int n_seg, double* __restrict__ part,
             unsigned* counter, double* __restrict__ out) {
  __shared__ double red[256];
  __shared__ bool last;
  const int b = blockIdx.x;
  int i = 0, lo = 0, hi = n_seg - 1;  // segment of chunk b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chunk0[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  i = lo;
  const long long a0 = seg0[i] + (long long)(b - chunk0[i]) * kSegChunk;
  const long long a1 = a0 + kSegChunk < seg0[i + 1] ? a0 + kSegChunk : seg0[i + 1];
  double acc = 0.0;
  for (long long t = a0 + threadIdx.x; t < a1; t += blockDim.x) acc += vals[t];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[b] = red[0];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int s = threadIdx.x; s < n_seg; s += blockDim.x) {
    double t = 0.0;
    for (int c = chunk0[s]; c < chunk0[s + 1]; ++c) t += ((volatile double*)part)[c];
    out[s] = t;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// One instance's FP32 Hessian product on the same strips (the 2D product's
// "marching strips" tile variant): the instance travels as a kernel
// argument; skip non-null and set makes the launch a no-op (a CG run that
// has stopped).
__global__ void __launch_bounds__(128, 3)
    k_hess2_march(const BInst I, const BVec V, long long T, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const long long W = (long long)gridDim.x * (blockDim.x >> 5);
  const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  long long s = w * T / W;
  const long long s_end = (w + 1) * T / W;
  const int n1 = I.g.n[1];
  while (s < s_end) {
    const int strip = int(s / n1), r0 = int(s % n1);
    const long long left = s_end - s;
    const int rows = left < (long long)(n1 - r0) ? int(left) : n1 - r0;
    hess2_strip<false>(I, V, strip, r0, rows, lane, nullptr);
    s += rows;
  }
}

}  // namespace
}  // namespace pf

using namespace pf;

struct pf_batch {
  int n = 0;
  std::vector<pf_hierarchy*> hs;
  cudaStream_t st = nullptr;
  int sms = 0, occ = 0;  // SMs, resident blocks per SM of the product kernel
  int bps = 0;           // blocks per SM used by the product (autotuned)
  long long T = 0, TE = 0, dofs = 0;
  std::vector<BInst> h_inst;
  std::vector<double> mat_p;  // pressure each instance's constants were built with
  BInst* d_inst = nullptr;
  BVec* d_vec = nullptr;
  const double** d_xs = nullptr;
  std::vector<BVec> h_vec;
  std::vector<const double*> h_xs;
  double* rowdot = nullptr;  // T partials (node rows)
  double* erow = nullptr;    // TE partials (element rows)
  long long* d_seg_rows = nullptr;   // n + 1 row-step offsets
  long long* d_seg_erows = nullptr;  // n + 1 element-row offsets
  int* d_chunk_rows = nullptr;       // n + 1 chunk offsets of the row partials
  int* d_chunk_erows = nullptr;
  int chunks_rows = 0, chunks_erows = 0;
  double* part = nullptr;       // chunk sums
  unsigned* counter = nullptr;  // segmented-sum completion ticket
  unsigned long long* ecount = nullptr;  // energy row counter
  double* d_E = nullptr;        // n energies
  double* h_E = nullptr;        // pinned mirror
  std::vector<void*> allocations;
};

namespace {

pf_status bad_b(const char* msg) {
  set_error(msg);
  return PF_EINVAL;
}

#define PF_B_TRY(call, what)                                                    \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      set_error(std::string(what) + ": " + cudaGetErrorString(e_));             \
      return e_ == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA;            \
    }                                                                           \
  } while (0)

// FP32 constants of hess2_pair from an instance's FP64 material.
void set_consts(BInst& I, const Mat<double>& m) {
  const double ih = m.inv_h, w = m.w, omk = 1.0 - m.k;
  I.lam = float(m.lam);
  I.mu = float(m.mu);
  I.mu2 = float(2.0 * m.mu);
  I.lam_h = float(m.lam * ih);
  I.mu2_h = float(2.0 * m.mu * ih);
  I.mu_h = float(m.mu * ih);
  I.p = float(m.p);
  const double wh2 = w * ih * ih, wh = w * ih;
  I.cA = float(wh2 * omk);                // A = cA (1-c)^2 + cAk
  I.cAk = float(wh2 * m.k);
  I.cdg = float(-2.0 * omk * wh);         // w g'(c) / h = cdg (1-c)
  I.cpl = float(0.5 * m.lam * ih * ih);   // psi = cpl tr^2 + cpm ee (raw differences)
  I.cpm = float(m.mu * ih * ih);
  I.cpt = float(m.p * ih);                // p tr e
  I.cM2 = float(2.0 * omk * w);           // M = cM2 (psi + p tr) + cM0
  I.cM0 = float(w * m.Gc / m.ls);
  I.kc = float(w * m.Gc * m.ls * ih * ih);
}

template <class T>
cudaError_t balloc(pf_batch* b, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) return e;
  b->allocations.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

void free_batch(pf_batch* b) {
  for (void* p : b->allocations) cudaFree(p);
  if (b->h_E) cudaFreeHost(b->h_E);
  delete b;
}

// Refreshes the device instance table where a hierarchy's pressure changed.
pf_status sync_consts(pf_batch* b) {
  bool dirty = false;
  for (int i = 0; i < b->n; ++i) {
    const pf_hierarchy* H = b->hs[i];
    const Mat<double>& m = H->mat[H->L - 1];
    if (m.p != b->mat_p[i]) {
      b->h_inst[i].md = m;
      set_consts(b->h_inst[i], m);
      b->mat_p[i] = m.p;
      dirty = true;
    }
  }
  if (dirty) {
    PF_B_TRY(cudaMemcpyAsync(b->d_inst, b->h_inst.data(), sizeof(BInst) * b->n,
                             cudaMemcpyHostToDevice, b->st),
             "batch: instance table");
    PF_B_TRY(cudaStreamSynchronize(b->st), "batch: instance table");
  }
  return PF_OK;
}

pf_status launch_hess(pf_batch* b, int bps, bool dot) {
  const int blocks = b->sms * bps;
  if (dot)
    k_batch_hess2<true><<<blocks, kHessThreads, 0, b->st>>>(b->d_inst, b->d_vec, b->n, b->T, b->rowdot);
  else
    k_batch_hess2<false><<<blocks, kHessThreads, 0, b->st>>>(b->d_inst, b->d_vec, b->n, b->T, nullptr);
  PF_B_TRY(cudaGetLastError(), "batch_hessvec");
  return PF_OK;
}

}  // namespace

namespace pf {
cudaError_t hess2_march(const Geom& g, const Mat<double>& m, const float* x, const float* v,
                        float* y, const int* skip, cudaStream_t st) {
  if (g.dim != 2 || 3 * g.N >= (1LL << 31)) return cudaErrorInvalidValue;
  BInst I;
  std::memset(&I, 0, sizeof(I));
  I.g = g;
  I.md = m;
  I.strips = (g.n[0] + kStripCols - 1) / kStripCols;
  set_consts(I, m);
  const long long T = (long long)I.strips * g.n[1];
  static const int sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 1;
    return n;
  }();
  // every warp at least 8 rows (one halo row each), at most 3 blocks per SM
  const long long warps = std::min<long long>(3LL * 4 * sms, (T + 7) / 8);
  const int blocks = int(std::max<long long>(1, (warps + 3) / 4));
  k_hess2_march<<<blocks, kHessThreads, 0, st>>>(I, BVec{x, v, y}, T, skip);
  return cudaGetLastError();
}
}  // namespace pf

extern "C" {

pf_status pf_batch_create(int n, pf_hierarchy* const* hs, void* stream, pf_batch** out) {
  if (!out || !hs || n < 1) return bad_b("batch_create: bad argument");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return bad_b("batch_create: null hierarchy");
    if (hs[i]->dim != 2) return bad_b("batch_create: the batched operators are 2D");
    if (3 * hs[i]->geo[hs[i]->L - 1].N >= (1LL << 31))
      return bad_b("batch_create: an instance has 3 N >= 2^31 dofs (32-bit indices)");
  }
  pf_batch* b = new pf_batch();
  b->n = n;
  b->hs.assign(hs, hs + n);
  b->st = static_cast<cudaStream_t>(stream);
  b->h_inst.resize(n);
  b->mat_p.assign(n, std::nan(""));
  b->h_vec.assign(n, BVec{nullptr, nullptr, nullptr});
  b->h_xs.assign(n, nullptr);
  std::vector<long long> seg_rows(n + 1, 0), seg_erows(n + 1, 0);
  std::vector<int> ch_rows(n + 1, 0), ch_erows(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const pf_hierarchy* H = hs[i];
    BInst& I = b->h_inst[i];
    std::memset(&I, 0, sizeof(I));
    I.g = H->geo[H->L - 1];
    I.md = H->mat[H->L - 1];
    set_consts(I, I.md);
    b->mat_p[i] = I.md.p;
    I.strips = (I.g.n[0] + kStripCols - 1) / kStripCols;
    I.row0 = seg_rows[i];
    I.erow0 = seg_erows[i];
    const long long steps = (long long)I.strips * I.g.n[1];
    seg_rows[i + 1] = seg_rows[i] + steps;
    seg_erows[i + 1] = seg_erows[i] + I.g.ne[1];
    ch_rows[i + 1] = ch_rows[i] + int((steps + kSegChunk - 1) / kSegChunk);
    ch_erows[i + 1] = ch_erows[i] + int((I.g.ne[1] + kSegChunk - 1) / kSegChunk);
    b->dofs += 3 * I.g.N;
  }
  b->T = seg_rows[n];
  b->TE = seg_erows[n];
  b->chunks_rows = ch_rows[n];
  b->chunks_erows = ch_erows[n];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ, k_batch_hess2<true>, kHessThreads, 0);
  if (e == cudaSuccess) {
    b->occ = std::max(1, std::min(b->occ, 4));
    b->bps = b->occ;
  }
  if (e == cudaSuccess) e = balloc(b, &b->d_inst, n);
  if (e == cudaSuccess) e = balloc(b, &b->d_vec, n);
  if (e == cudaSuccess) e = balloc(b, &b->d_xs, n);
  if (e == cudaSuccess) e = balloc(b, &b->rowdot, b->T);
  if (e == cudaSuccess) e = balloc(b, &b->erow, b->TE);
  if (e == cudaSuccess) e = balloc(b, &b->d_seg_rows, n + 1);
  if (e == cudaSuccess) e = balloc(b, &b->d_seg_erows, n + 1);
  if (e == cudaSuccess) e = balloc(b, &b->d_chunk_rows, n + 1);
  if (e == cudaSuccess) e = balloc(b, &b->d_chunk_erows, n + 1);
  if (e == cudaSuccess) e = balloc(b, &b->part, std::max(b->chunks_rows, b->chunks_erows));
  if (e == cudaSuccess) e = balloc(b, &b->counter, 1);
  if (e == cudaSuccess) e = balloc(b, &b->ecount, 1);
  if (e == cudaSuccess) e = balloc(b, &b->d_E, n);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_E, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->counter, 0, sizeof(unsigned), b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_inst, b->h_inst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_seg_rows, seg_rows.data(), sizeof(long long) * (n + 1),
                        cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_seg_erows, seg_erows.data(), sizeof(long long) * (n + 1),
                        cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_chunk_rows, ch_rows.data(), sizeof(int) * (n + 1),
                        cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_chunk_erows, ch_erows.data(), sizeof(int) * (n + 1),
                        cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) {
    set_error(std::string("batch_create: ") + cudaGetErrorString(e));
    free_batch(b);
    return e == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA;
  }
  *out = b;
  return PF_OK;
}

pf_status pf_batch_destroy(pf_batch* b) {
  if (!b) return PF_OK;
  cudaStreamSynchronize(b->st);
  free_batch(b);
  return PF_OK;
}

pf_status pf_batch_info(const pf_batch* b, long long* dofs, int* blocks_per_sm, int* sms) {
  if (!b) return bad_b("batch_info: null handle");
  if (dofs) *dofs = b->dofs;
  if (blocks_per_sm) *blocks_per_sm = b->bps;
  if (sms) *sms = b->sms;
  return PF_OK;
}

pf_status pf_batch_hessvec(pf_batch* b, const float* const* x_dev, const float* const* v_dev,
                           float* const* Hv_dev, double* vHv_dev) {
  if (!b || !x_dev || !v_dev || !Hv_dev) return bad_b("batch_hessvec: bad argument");
  bool changed = false;
  for (int i = 0; i < b->n; ++i) {
    if (!x_dev[i] || !v_dev[i] || !Hv_dev[i]) return bad_b("batch_hessvec: null vector");
    if ((const void*)Hv_dev[i] == (const void*)x_dev[i] ||
        (const void*)Hv_dev[i] == (const void*)v_dev[i])
      return bad_b("batch_hessvec: Hv must not alias x or v");
    const BVec nv{x_dev[i], v_dev[i], Hv_dev[i]};
    if (nv.x != b->h_vec[i].x || nv.v != b->h_vec[i].v || nv.y != b->h_vec[i].y) {
      b->h_vec[i] = nv;
      changed = true;
    }
  }
  pf_status s = sync_consts(b);
  if (s != PF_OK) return s;
  if (changed) {
    PF_B_TRY(cudaMemcpyAsync(b->d_vec, b->h_vec.data(), sizeof(BVec) * b->n,
                             cudaMemcpyHostToDevice, b->st),
             "batch_hessvec: vector table");
    PF_B_TRY(cudaStreamSynchronize(b->st), "batch_hessvec: vector table");
  }
  s = launch_hess(b, b->bps, vHv_dev != nullptr);
  if (s != PF_OK || !vHv_dev) return s;
  k_segsum<<<b->chunks_rows, 256, 0, b->st>>>(b->rowdot, b->d_seg_rows, b->d_chunk_rows, b->n,
                                               b->part, b->counter, vHv_dev);
  PF_B_TRY(cudaGetLastError(), "batch_hessvec: segmented sum");
  return PF_OK;
}

pf_status pf_batch_energy(pf_batch* b, const double* const* x_dev, double* E_host) {
  if (!b || !x_dev || !E_host) return bad_b("batch_energy: bad argument");
  bool changed = false;
  for (int i = 0; i < b->n; ++i) {
    if (!x_dev[i]) return bad_b("batch_energy: null vector");
    if (x_dev[i] != b->h_xs[i]) {
      b->h_xs[i] = x_dev[i];
      changed = true;
    }
  }
  pf_status s = sync_consts(b);
  if (s != PF_OK) return s;
  if (changed) {
    PF_B_TRY(cudaMemcpyAsync(b->d_xs, b->h_xs.data(), sizeof(double*) * b->n,
                             cudaMemcpyHostToDevice, b->st),
             "batch_energy: vector table");
    PF_B_TRY(cudaStreamSynchronize(b->st), "batch_energy: vector table");
  }
  PF_B_TRY(cudaMemsetAsync(b->ecount, 0, sizeof(unsigned long long), b->st), "batch_energy");
  k_batch_energy2<<<b->sms * 4, 256, 0, b->st>>>(b->d_inst, b->d_xs, b->n, b->TE, b->ecount,
                                                  b->erow);
  PF_B_TRY(cudaGetLastError(), "batch_energy");
  k_segsum<<<b->chunks_erows, 256, 0, b->st>>>(b->erow, b->d_seg_erows, b->d_chunk_erows, b->n,
                                                b->part, b->counter, b->d_E);
  PF_B_TRY(cudaGetLastError(), "batch_energy: segmented sum");
  PF_B_TRY(cudaMemcpyAsync(b->h_E, b->d_E, sizeof(double) * b->n, cudaMemcpyDeviceToHost, b->st),
           "batch_energy");
  PF_B_TRY(cudaStreamSynchronize(b->st), "batch_energy");
  bool finite = true;
  for (int i = 0; i < b->n; ++i) {
    E_host[i] = b->h_E[i];
    finite = finite && std::isfinite(b->h_E[i]);
  }
  if (!finite) {
    set_error("batch_energy: non-finite result");
    return PF_ENONFINITE;
  }
  return PF_OK;
}

pf_status pf_batch_autotune(pf_batch* b, const float* const* x_dev, const float* const* v_dev,
                            float* const* Hv_dev, int* bps_out, double* us_out) {
  if (!b) return bad_b("batch_autotune: null handle");
  pf_status s = pf_batch_hessvec(b, x_dev, v_dev, Hv_dev, nullptr);
  if (s != PF_OK) return s;
  cudaEvent_t e0, e1;
  PF_B_TRY(cudaEventCreate(&e0), "batch_autotune");
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    PF_B_TRY(ce, "batch_autotune");
  }
  int best = b->bps;
  double best_us = 1e300;
  for (int v = 1; v <= 4; ++v) {
    double us = -1.0;
    if (v <= b->occ) {
      s = launch_hess(b, v, false);  // warm-up
      for (int r = 0; r < 5 && s == PF_OK; ++r) {
        if (r == 0) cudaEventRecord(e0, b->st);
        s = launch_hess(b, v, false);
      }
      if (s != PF_OK) break;
      cudaEventRecord(e1, b->st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      us = 1e3 * ms / 5.0;
      if (us < best_us) {
        best_us = us;
        best = v;
      }
    }
    if (us_out) us_out[v - 1] = us;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != PF_OK) return s;
  b->bps = best;
  if (bps_out) *bps_out = best;
  return PF_OK;
}

pf_status pf_batch_variant_set(pf_batch* b, int blocks_per_sm) {
  if (!b) return bad_b("batch_variant_set: null handle");
  if (blocks_per_sm < 1 || blocks_per_sm > b->occ)
    return bad_b("batch_variant_set: blocks per SM outside 1 .. the kernel's occupancy");
  b->bps = blocks_per_sm;
  return PF_OK;
}

}  // extern "C"
