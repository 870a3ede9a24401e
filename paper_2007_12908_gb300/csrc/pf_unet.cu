// Learned initial iterate: a 2D U-Net (4 levels, two 3x3 convolutions +
// ReLU per level, 2x2 average pooling down, nearest 2x up, skip
// concatenation, 1x1 head).  BF16 weights and activations, FP32 master
// weights and Adam moments.  Every convolution (forward, data gradient,
// weight gradient) is an implicit GEMM on the tensor cores with BF16
// operands and FP32 accumulation; the data-gradient and weight-gradient
// operand dL/d(out) (FP32) is staged as a BF16 pair hi + lo and multiplied
// twice, keeping about 16 significant bits of the gradient.
//
// Convolutions read their input through a fused transform: the first
// operand may be pooled (it lives at twice the resolution) or upsampled (it
// lives at half the resolution), and a second operand (the encoder skip) is
// concatenated after it, so neither the pooled, the upsampled nor the
// concatenated tensor is ever stored.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pf.h"
#include "pf_internal.h"

namespace pf {
void set_error(const std::string& msg);
}
using namespace pf;

namespace {

enum { IN_PLAIN = 0, IN_POOL = 1, IN_UP = 2 };

struct ConvIn {
  const __nv_bfloat16* a;  // first operand (ca channels)
  int ca, mode;            // mode: IN_PLAIN / IN_POOL / IN_UP
  const __nv_bfloat16* b;  // concatenated operand (cb channels, same resolution), or null
  int cb;
};

// value of input channel c at (y, x) of the conv's H x W grid (0 outside)
__device__ __forceinline__ float conv_in(const ConvIn& in, int c, int y, int x, int H, int W) {
  if (y < 0 || y >= H || x < 0 || x >= W) return 0.f;
  if (c < in.ca) {
    if (in.mode == IN_PLAIN) return __bfloat162float(in.a[((long long)c * H + y) * W + x]);
    if (in.mode == IN_POOL) {
      const int W2 = 2 * W;
      const __nv_bfloat16* p = in.a + ((long long)c * 2 * H + 2 * y) * W2 + 2 * x;
      return 0.25f * (__bfloat162float(p[0]) + __bfloat162float(p[1]) + __bfloat162float(p[W2]) +
                      __bfloat162float(p[W2 + 1]));
    }
    const int Hh = H / 2, Wh = W / 2;
    return __bfloat162float(in.a[((long long)c * Hh + (y >> 1)) * Wh + (x >> 1)]);
  }
  return __bfloat162float(in.b[((long long)(c - in.ca) * H + y) * W + x]);
}

// ---------------------------------------------------------------- tensor cores
// The convolutions are implicit GEMMs on the tensor cores: BF16 operands,
// FP32 accumulation, mma.sync.m16n8k16 (one warp-wide 16x8x16 product per
// instruction).
//
// Forward:  out[co](p)  = sum_{ci, tap} w[co][ci][tap] in[ci](p + off(tap))
//           (M = co, N = pixels, K = ci for each tap)
// Data gradient: din[ci](p) = sum_{co, tap} w[co][ci][KK-1-tap] dpre[co](p + off(tap))
//           (the same form with the weights transposed and flipped)
// Weight gradient: dw[co][ci][tap] = sum_p dpre[co](p) in[ci](p + off(tap))
//           (M = co, N = ci, K = pixels)

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

// 16 channels of one pixel (or one GEMM row) are 8 32-bit words; words 4..7
// of rows whose bit 2 is set are swapped with words 0..3, so that the eight
// rows a fragment load touches fall in distinct banks.
__device__ __forceinline__ int swz(int row, int word) { return row * 8 + (word ^ (((row >> 2) & 1) << 2)); }

// Operand sources of the forward / data-gradient kernel.
struct MmaIn {
  ConvIn conv;                     // forward: the fused input transform
  const float* dout;               // data gradient: dL/d(out) (FP32) ...
  const __nv_bfloat16* out;        // ... masked by out > 0 when relu
  int relu;
};

template <bool DGRAD>
__device__ __forceinline__ float mma_in_value(const MmaIn& s, int c, int Kc, int y, int x, int H,
                                              int W) {
  if (c >= Kc) return 0.f;
  if constexpr (!DGRAD) {
    return conv_in(s.conv, c, y, x, H, W);
  } else {
    if (y < 0 || y >= H || x < 0 || x >= W) return 0.f;
    const long long o = ((long long)c * H + y) * W + x;
    float v = s.dout[o];
    if (s.relu && !(__bfloat162float(s.out[o]) > 0.f)) v = 0.f;
    return v;
  }
}

// grid: (W/16, H/16, ceil(M/MB)); 256 threads = 8 warps, warp w owns pixel
// rows 2w, 2w+1 of the 16 x 16 tile (four 8-pixel n-tiles) and all MB rows.
// Forward (DGRAD = false): M = CO rows co, Kc = CI, A[co][ci] =
// w[co][ci][tap]; epilogue bias + ReLU, BF16 and/or FP32 output.
// Data gradient: M = CI rows ci, Kc = CO, A[ci][co] = w[co][ci][KK-1-tap];
// FP32 output, no bias.
// The data gradient's operand dpre is FP32: it is staged as a BF16 pair
// hi + lo (hi = bf16(v), lo = bf16(v - hi), about 16 significant bits) and
// multiplied twice, so that the gradient keeps more than BF16 precision
// through the layers; activations and weights are BF16 already.
template <int K, int MB, bool DGRAD>
__global__ void __launch_bounds__(256) k_conv_mma(MmaIn src, int H, int W, int M, int Kc, int CIw,
                                                  const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ bias, int relu,
                                                  __nv_bfloat16* __restrict__ out_bf,
                                                  float* __restrict__ out_f) {
  constexpr int R = K / 2, T = 16 + 2 * R, KK = K * K, MT = MB / 16, NS = DGRAD ? 2 : 1;
  __shared__ unsigned s_in[NS][T * T * 8];  // [pixel][16 channels] BF16 pairs, swizzled
  __shared__ unsigned s_w[KK * MB * 8];     // [tap][row][16 channels]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const int x0 = blockIdx.x * 16, y0 = blockIdx.y * 16, m0 = blockIdx.z * MB;
  float acc[MT][4][4];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  for (int k0 = 0; k0 < Kc; k0 += 16) {
    for (int i = threadIdx.x; i < T * T * 8; i += 256) {
      const int q = i % (T * T), j = i / (T * T);
      const int yy = y0 - R + q / T, xx = x0 - R + q % T;
      const float v0 = mma_in_value<DGRAD>(src, k0 + 2 * j, Kc, yy, xx, H, W);
      const float v1 = mma_in_value<DGRAD>(src, k0 + 2 * j + 1, Kc, yy, xx, H, W);
      s_in[0][swz(q, j)] = pack_bf16(v0, v1);
      if constexpr (DGRAD)
        s_in[1][swz(q, j)] = pack_bf16(v0 - __bfloat162float(__float2bfloat16(v0)),
                                       v1 - __bfloat162float(__float2bfloat16(v1)));
    }
    for (int i = threadIdx.x; i < KK * MB * 8; i += 256) {
      const int j = i & 7, row = (i >> 3) % MB, tap = i / (8 * MB);
      const int m = m0 + row;
      float v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kc = k0 + 2 * j + h;
        v[h] = 0.f;
        if (m < M && kc < Kc) {
          // forward: w[m][kc][tap]; data gradient: w[kc][m][KK-1-tap]
          const long long o = DGRAD ? ((long long)kc * CIw + m) * KK + (KK - 1 - tap)
                                    : ((long long)m * CIw + kc) * KK + tap;
          v[h] = __bfloat162float(w[o]);
        }
      }
      s_w[tap * MB * 8 + swz(row, j)] = pack_bf16(v[0], v[1]);
    }
    __syncthreads();
#pragma unroll
    for (int tap = 0; tap < KK; ++tap) {
      const int ky = tap / K, kx = tap % K;
#pragma unroll
      for (int part = 0; part < NS; ++part) {
        unsigned bfr[4][2];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int py = 2 * warp + (nt >> 1), px = (nt & 1) * 8 + g;
          const int q = (py + ky) * T + px + kx;
          bfr[nt][0] = s_in[part][swz(q, t4)];
          bfr[nt][1] = s_in[part][swz(q, t4 + 4)];
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const unsigned* sw = s_w + tap * MB * 8;
          const int r0 = mt * 16 + g, r1 = r0 + 8;
          const unsigned a[4] = {sw[swz(r0, t4)], sw[swz(r1, t4)], sw[swz(r0, t4 + 4)],
                                 sw[swz(r1, t4 + 4)]};
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a, bfr[nt][0], bfr[nt][1]);
        }
      }
    }
    __syncthreads();
  }
  // epilogue: c0 (row g, pixel 2t), c1 (row g, 2t+1), c2 (row g+8, 2t), c3 (row g+8, 2t+1)
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int y = y0 + 2 * warp + (nt >> 1);
      const int xb = x0 + (nt & 1) * 8 + 2 * t4;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + mt * 16 + g + 8 * h;
        if (m >= M || y >= H) continue;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int x = xb + e;
          if (x >= W) continue;
          float v = acc[mt][nt][2 * h + e];
          if (!DGRAD) {
            v += bias[m];
            if (relu) v = fmaxf(v, 0.f);
          }
          const long long o = ((long long)m * H + y) * W + x;
          if (out_bf) out_bf[o] = __float2bfloat16(v);
          if (out_f) out_f[o] = v;
        }
      }
    }
}

// Weight gradient partials on the tensor cores.  grid: (ceil(CI/NB),
// ceil(CO/MB), P); the 16 x 16 pixel tiles of the layer (tx per row, T in
// all, row-major) are cut into P contiguous chunks, chunk p taking tiles
// [p T / P, (p+1) T / P) in order.
// The CTA stages, per 16 x 16 pixel tile, dpre for its MB output channels
// (A rows; K = the 16 pixels of a tile row) and the fused input for its NB
// input channels (three copies shifted by kx, so that every pixel pair a
// fragment reads is 4-byte aligned).  Per-channel strides are padded by 4
// words so the eight rows of a fragment fall in distinct banks.  Warp w
// accumulates the (m-tile, n-tile, tap) products w, w+8, ...; the bias
// gradient sums the FP32 dpre of each channel (warp w: channels w, w+8, ...)
// lane-wise and by a fixed shuffle tree.  Every sum runs over the pixels in
// a fixed order, so the partials are deterministic.
template <int K, int MB, int NB>
struct WgradSmem {
  static constexpr int R = K / 2, YT = 16 + 2 * R;
  static constexpr int SD = 16 * 8 + 4, SX = YT * 8 + 4;
  static constexpr size_t bytes = sizeof(unsigned) * (2 * size_t(MB) * SD + size_t(K) * NB * SX);
};

template <int K, int MB, int NB>
__global__ void __launch_bounds__(256) k_conv_wgrad_mma(const float* __restrict__ dout,
                                                        const __nv_bfloat16* __restrict__ out,
                                                        int relu, ConvIn in, int H, int W, int CO,
                                                        int P, float* __restrict__ part,
                                                        float* __restrict__ part_b) {
  using S = WgradSmem<K, MB, NB>;
  constexpr int R = S::R, YT = S::YT, SD = S::SD, SX = S::SX, KK = K * K;
  constexpr int MT = MB / 16, NT = NB / 8;
  constexpr int COMBOS = MT * NT * KK, PER = (COMBOS + 7) / 8, BPW = MB / 8;
  extern __shared__ unsigned smem_u[];
  unsigned* s_d = smem_u;             // [2][MB][SD] (hi, lo): row r, pixel pair wd at r * 8 + wd
  unsigned* s_x = s_d + 2 * MB * SD;  // [K][NB][SX]: row r, pixel pair wd at r * 8 + wd
  const int CI = in.ca + in.cb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const int n0 = blockIdx.x * NB, m0 = blockIdx.y * MB, p = blockIdx.z;
  const int tx = (W + 15) / 16;
  const long long T = (long long)tx * ((H + 15) / 16);
  const long long t_lo = p * T / P, t_hi = (p + 1) * T / P;
  float acc[PER][4];
#pragma unroll
  for (int i = 0; i < PER; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0.f;
  float accb[BPW];
#pragma unroll
  for (int j = 0; j < BPW; ++j) accb[j] = 0.f;
  auto dpre = [&](int c, int yy, int xx) -> float {
    if (m0 + c >= CO || yy >= H || xx >= W) return 0.f;
    const long long o = ((long long)(m0 + c) * H + yy) * W + xx;
    const float d = dout[o];
    return (relu && !(__bfloat162float(out[o]) > 0.f)) ? 0.f : d;
  };
  for (long long ti = t_lo; ti < t_hi; ++ti) {
    const int yb = int(ti / tx) * 16, xb = int(ti % tx) * 16;
    {
      for (int i = threadIdx.x; i < MB * 16 * 8; i += 256) {
        const int wd = i & 7, r = (i >> 3) & 15, c = i >> 7;
        const float v0 = dpre(c, yb + r, xb + 2 * wd), v1 = dpre(c, yb + r, xb + 2 * wd + 1);
        s_d[c * SD + r * 8 + wd] = pack_bf16(v0, v1);
        s_d[(MB + c) * SD + r * 8 + wd] = pack_bf16(v0 - __bfloat162float(__float2bfloat16(v0)),
                                                   v1 - __bfloat162float(__float2bfloat16(v1)));
      }
      for (int i = threadIdx.x; i < K * NB * YT * 8; i += 256) {
        const int wd = i & 7, r = (i >> 3) % YT, c = (i / (8 * YT)) % NB, kx = i / (8 * YT * NB);
        const int yy = yb - R + r, xx = xb - R + kx + 2 * wd;
        const float lo = (n0 + c < CI) ? conv_in(in, n0 + c, yy, xx, H, W) : 0.f;
        const float hi = (n0 + c < CI) ? conv_in(in, n0 + c, yy, xx + 1, H, W) : 0.f;
        s_x[(kx * NB + c) * SX + r * 8 + wd] = pack_bf16(lo, hi);
      }
      // bias (blocks of the first input-channel block only): FP32 sums of
      // dpre, lane-wise over the tile then a fixed tree
      if (blockIdx.x == 0)
#pragma unroll
      for (int j = 0; j < BPW; ++j) {
        const int c = warp + 8 * j;
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int px = lane + 32 * k;
          s += dpre(c, yb + px / 16, xb + px % 16);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        accb[j] += s;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int combo = warp + 8 * i;
        if (combo < COMBOS) {
          const int mt = combo % MT, nt = (combo / MT) % NT, tap = combo / (MT * NT);
          const int ky = tap / K, kx = tap % K;
          const unsigned* xb0 = s_x + (kx * NB + nt * 8 + g) * SX + ky * 8;
#pragma unroll
          for (int part = 0; part < 2; ++part) {  // dpre = hi + lo
            const unsigned* da0 = s_d + (part * MB + mt * 16 + g) * SD;
            const unsigned* da1 = da0 + 8 * SD;
#pragma unroll 4
            for (int r = 0; r < 16; ++r) {
              const unsigned a[4] = {da0[r * 8 + t4], da1[r * 8 + t4], da0[r * 8 + t4 + 4],
                                     da1[r * 8 + t4 + 4]};
              mma_bf16(acc[i], a, xb0[r * 8 + t4], xb0[r * 8 + t4 + 4]);
            }
          }
        }
      }
      __syncthreads();
    }
  }
  // c0 (m = g, n = 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1)
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int combo = warp + 8 * i;
    if (combo >= COMBOS) continue;
    const int mt = combo % MT, nt = (combo / MT) % NT, tap = combo / (MT * NT);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int co = m0 + mt * 16 + g + 8 * (e >> 1), ci = n0 + nt * 8 + 2 * t4 + (e & 1);
      if (co < CO && ci < CI) part[(((long long)p * CO + co) * CI + ci) * KK + tap] = acc[i][e];
    }
  }
  if (blockIdx.x == 0 && lane == 0)
#pragma unroll
    for (int j = 0; j < BPW; ++j) {
      const int c = warp + 8 * j;
      if (m0 + c < CO) part_b[(long long)p * CO + m0 + c] = accb[j];
    }
}


// Forward (DGRAD = false) or data-gradient convolution on the tensor cores;
// MB (GEMM rows per CTA) follows the row count M.
template <int K, bool DGRAD>
void launch_conv_mma(const MmaIn& src, int H, int W, int M, int Kc, int CIw,
                     const __nv_bfloat16* w, const float* bias, int relu, __nv_bfloat16* ob,
                     float* of, cudaStream_t st) {
  const int MB = M <= 16 ? 16 : (M <= 32 ? 32 : 64);
  const dim3 grid((W + 15) / 16, (H + 15) / 16, (M + MB - 1) / MB);
  if (MB == 16)
    k_conv_mma<K, 16, DGRAD><<<grid, 256, 0, st>>>(src, H, W, M, Kc, CIw, w, bias, relu, ob, of);
  else if (MB == 32)
    k_conv_mma<K, 32, DGRAD><<<grid, 256, 0, st>>>(src, H, W, M, Kc, CIw, w, bias, relu, ob, of);
  else
    k_conv_mma<K, 64, DGRAD><<<grid, 256, 0, st>>>(src, H, W, M, Kc, CIw, w, bias, relu, ob, of);
}

constexpr int WG_MB = 32, WG_NB = 16;

// Pixel-tile chunks of a weight-gradient launch: enough for two CTAs per SM
// over the (input block, output block) grid, at most one chunk per tile.
int wgrad_chunks(int H, int W, int CI, int CO, int sms) {
  const long long T = (long long)((W + 15) / 16) * ((H + 15) / 16);
  const long long base = (long long)((CI + WG_NB - 1) / WG_NB) * ((CO + WG_MB - 1) / WG_MB);
  const long long want = (2LL * sms + base - 1) / base;
  return int(std::max<long long>(1, std::min(T, want)));
}

template <int K>
cudaError_t launch_wgrad_mma(const float* dout, const __nv_bfloat16* out, int relu, const ConvIn& in,
                             int H, int W, int CO, int P, float* part, float* part_b, cudaStream_t st) {
  const int CI = in.ca + in.cb;
  const dim3 grid((CI + WG_NB - 1) / WG_NB, (CO + WG_MB - 1) / WG_MB, P);
  const size_t bytes = WgradSmem<K, WG_MB, WG_NB>::bytes;
  static_assert(WgradSmem<3, WG_MB, WG_NB>::bytes <= 100 * 1024, "wgrad shared memory above 100 KB");
  static thread_local int dev_done = -1;  // opt-in above 48 KB, once per device and thread
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev_done != dev) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_wgrad_mma<K, WG_MB, WG_NB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e != cudaSuccess) return e;
    dev_done = dev;
  }
  k_conv_wgrad_mma<K, WG_MB, WG_NB><<<grid, 256, bytes, st>>>(dout, out, relu, in, H, W, CO, P,
                                                             part, part_b);
  return cudaGetLastError();
}

// grad += sum_p part[p] in order p = 0 .. P-1 (deterministic)
__global__ void k_sum_parts(const float* __restrict__ part, int P, long long n,
                            float* __restrict__ grad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int p = 0; p < P; ++p) s += part[p * n + i];
    grad[i] += s;
  }
}

// Adjoint of the fused input transform: scatter dIn (conv grid H x W, CI
// channels) into the FP32 gradients of the two operands (accumulating).
__global__ void k_in_adjoint(const float* __restrict__ din, int H, int W, int ca, int mode,
                             int cb, float* __restrict__ ga, float* __restrict__ gb) {
  const long long total_a = (mode == IN_POOL ? 4LL : (mode == IN_UP ? 0 : 1)) * ca * H * W;
  // plain / pool: one thread per element of the operand's own grid
  if (mode == IN_PLAIN || mode == IN_POOL) {
    const int Hs = mode == IN_POOL ? 2 * H : H, Ws = mode == IN_POOL ? 2 * W : W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total_a;
         i += (long long)gridDim.x * blockDim.x) {
      const int c = int(i / ((long long)Hs * Ws));
      const long long r = i % ((long long)Hs * Ws);
      const int y = int(r / Ws), x = int(r % Ws);
      const float g = mode == IN_POOL ? 0.25f * din[((long long)c * H + y / 2) * W + x / 2]
                                      : din[((long long)c * H + y) * W + x];
      ga[i] += g;
    }
  } else {
    const int Hh = H / 2, Wh = W / 2;
    const long long n = (long long)ca * Hh * Wh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const int c = int(i / ((long long)Hh * Wh));
      const long long r = i % ((long long)Hh * Wh);
      const int y = int(r / Wh), x = int(r % Wh);
      const float* p = din + ((long long)c * H + 2 * y) * W + 2 * x;
      ga[i] += p[0] + p[1] + p[W] + p[W + 1];
    }
  }
  if (gb) {
    const long long nb = (long long)cb * H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb;
         i += (long long)gridDim.x * blockDim.x)
      gb[i] += din[(long long)ca * H * W + i];
  }
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}

// Adam (Kingma & Ba) on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, long long n,
                       float lr, float b1, float b2, float eps, float c1, float c2, float scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i] * scale;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
  }
}

// masked MSE: loss partials per block, dy = (y - t) mask / n
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ y, const float* __restrict__ t,
                                             const float* __restrict__ mask, int C, long long HW,
                                             double inv_n, float* __restrict__ dy,
                                             double* __restrict__ part) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < C * HW;
       i += (long long)gridDim.x * blockDim.x) {
    const float mk = mask ? mask[i % HW] : 1.f;
    const float d = (y[i] - t[i]) * mk;
    dy[i] = float(d * inv_n);
    acc += 0.5 * double(d) * double(d) * inv_n;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

int grid1(long long n) {
  long long b = (n + 255) / 256;
  if (b > 8192) b = 8192;
  return int(b < 1 ? 1 : b);
}

}  // namespace

// ------------------------------------------------------------------ network
struct ConvLayer {
  int co, ci, k;
  long long off_w, off_b;  // offsets into the parameter vector
  bool relu;
};

struct pf_unet {
  int H = 0, W = 0, nin = 0, nout = 0, L = 4;
  int sms = 1;  // SMs of the device (the weight-gradient chunking)
  int ch[4] = {16, 32, 64, 128};
  cudaStream_t st = nullptr;
  std::vector<ConvLayer> layers;  // enc0a, enc0b, ..., enc3b, dec2a, dec2b, dec1a, ..., head
  long long nparam = 0;
  float *w32 = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  __nv_bfloat16* wbf = nullptr;
  int adam_t = 0;
  // activations (BF16): input, and the output of every 3x3 layer
  __nv_bfloat16* xin = nullptr;
  std::vector<__nv_bfloat16*> act;  // one per layer (head excluded)
  std::vector<float*> gact;         // FP32 gradient of each activation
  float* gin = nullptr;             // gradient of the input (unused but kept for adjoint writes)
  float* dscratch = nullptr;        // dIn of one conv (largest layer)
  float* wpart = nullptr;           // weight-gradient partials
  long long wpart_n = 0;
  double* lpart = nullptr;
  double* h_loss = nullptr;
  std::vector<void*> allocs;
};

namespace {

pf_status ualloc(pf_unet* u, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    set_error("unet: cudaMalloc failed");
    return PF_ENOMEM;
  }
  u->allocs.push_back(*p);
  cudaMemsetAsync(*p, 0, bytes, u->st);
  return PF_OK;
}

// resolution of layer l's output: level of the layer
int layer_level(const pf_unet* u, int l) {
  if (l < 2 * u->L) return l / 2;
  const int d = l - 2 * u->L;  // decoder index 0 .. 2(L-1)-1 (+ head)
  if (d >= 2 * (u->L - 1)) return 0;
  return u->L - 2 - d / 2;
}

ConvIn layer_input(const pf_unet* u, int l) {
  ConvIn in{};
  const int L = u->L;
  if (l == 0) {
    in.a = u->xin; in.ca = u->nin; in.mode = IN_PLAIN;
  } else if (l < 2 * L) {
    in.a = u->act[l - 1];
    in.ca = u->layers[l - 1].co;
    in.mode = (l % 2 == 0) ? IN_POOL : IN_PLAIN;
  } else {
    const int d = l - 2 * L;
    if (d >= 2 * (L - 1)) {  // head
      in.a = u->act[l - 1]; in.ca = u->layers[l - 1].co; in.mode = IN_PLAIN;
    } else if (d % 2 == 0) {  // first conv of a decoder level: [up(below), skip]
      const int k = L - 2 - d / 2;
      in.a = u->act[l - 1]; in.ca = u->layers[l - 1].co; in.mode = IN_UP;
      in.b = u->act[2 * k + 1]; in.cb = u->ch[k];
    } else {
      in.a = u->act[l - 1]; in.ca = u->layers[l - 1].co; in.mode = IN_PLAIN;
    }
  }
  return in;
}

}  // namespace

extern "C" {

pf_status pf_unet_destroy(pf_unet* u) {
  if (!u) return PF_OK;
  if (u->st) cudaStreamSynchronize(u->st);
  else cudaDeviceSynchronize();
  for (void* p : u->allocs) cudaFree(p);
  if (u->h_loss) cudaFreeHost(u->h_loss);
  delete u;
  return PF_OK;
}

pf_status pf_unet_create(int height, int width, int n_in, int n_out, const int channels[4],
                         void* stream, pf_unet** out) {
  if (!out || !channels) {
    set_error("unet_create: null argument");
    return PF_EINVAL;
  }
  *out = nullptr;
  if (height < 8 || width < 8 || height % 8 || width % 8 || height > 16384 || width > 16384 ||
      n_in < 1 || n_in > 64 || n_out < 1 || n_out > 64) {
    set_error("unet_create: height and width must be multiples of 8 (8 .. 16384); 1 .. 64 channels in/out");
    return PF_EINVAL;
  }
  for (int k = 0; k < 4; ++k)
    if (channels[k] < 1 || channels[k] > 512) {
      set_error("unet_create: channels must be 1 .. 512");
      return PF_EINVAL;
    }
  pf_unet* u = new pf_unet();
  u->H = height; u->W = width; u->nin = n_in; u->nout = n_out;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&u->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      u->sms = 1;
  }
  for (int k = 0; k < 4; ++k) u->ch[k] = channels[k];
  u->st = static_cast<cudaStream_t>(stream);
  long long off = 0;
  auto add = [&](int co, int ci, int k, bool relu) {
    ConvLayer c{co, ci, k, off, off + (long long)co * ci * k * k, relu};
    off += (long long)co * ci * k * k + co;
    u->layers.push_back(c);
  };
  int cprev = n_in;
  for (int k = 0; k < 4; ++k) {
    add(u->ch[k], cprev, 3, true);
    add(u->ch[k], u->ch[k], 3, true);
    cprev = u->ch[k];
  }
  for (int k = 2; k >= 0; --k) {
    add(u->ch[k], u->ch[k + 1] + u->ch[k], 3, true);
    add(u->ch[k], u->ch[k], 3, true);
  }
  add(n_out, u->ch[0], 1, false);
  u->nparam = off;
  pf_status rc;
  const long long HW = (long long)height * width;
  if ((rc = ualloc(u, (void**)&u->w32, sizeof(float) * off)) ||
      (rc = ualloc(u, (void**)&u->m, sizeof(float) * off)) ||
      (rc = ualloc(u, (void**)&u->v, sizeof(float) * off)) ||
      (rc = ualloc(u, (void**)&u->g, sizeof(float) * off)) ||
      (rc = ualloc(u, (void**)&u->wbf, sizeof(__nv_bfloat16) * off)) ||
      (rc = ualloc(u, (void**)&u->xin, sizeof(__nv_bfloat16) * n_in * HW)) ||
      (rc = ualloc(u, (void**)&u->lpart, sizeof(double) * 8192))) {
    pf_unet_destroy(u);
    return rc;
  }
  long long max_din = 0, max_part = 0;
  const int nl = int(u->layers.size());
  u->act.assign(nl - 1, nullptr);
  u->gact.assign(nl - 1, nullptr);
  for (int l = 0; l < nl; ++l) {
    const int lev = layer_level(u, l);
    const long long hw = HW >> (2 * lev);
    const ConvLayer& c = u->layers[l];
    if (l < nl - 1) {
      if ((rc = ualloc(u, (void**)&u->act[l], sizeof(__nv_bfloat16) * c.co * hw)) ||
          (rc = ualloc(u, (void**)&u->gact[l], sizeof(float) * c.co * hw))) {
        pf_unet_destroy(u);
        return rc;
      }
    }
    max_din = std::max(max_din, (long long)c.ci * hw);
    const int P = wgrad_chunks(height >> lev, width >> lev, c.ci, c.co, u->sms);
    max_part = std::max(max_part, (long long)P * ((long long)c.co * c.ci * c.k * c.k + c.co));
  }
  if ((rc = ualloc(u, (void**)&u->dscratch, sizeof(float) * max_din)) ||
      (rc = ualloc(u, (void**)&u->wpart, sizeof(float) * max_part)) ||
      (rc = ualloc(u, (void**)&u->gin, sizeof(float) * n_in * HW))) {
    pf_unet_destroy(u);
    return rc;
  }
  if (cudaMallocHost((void**)&u->h_loss, sizeof(double) * 8192) != cudaSuccess) {
    pf_unet_destroy(u);
    set_error("unet_create: cudaMallocHost failed");
    return PF_ENOMEM;
  }
  if (cudaStreamSynchronize(u->st) != cudaSuccess) {
    pf_unet_destroy(u);
    set_error("unet_create: stream error");
    return PF_ECUDA;
  }
  *out = u;
  return PF_OK;
}

pf_status pf_unet_num_params(const pf_unet* u, long long* n) {
  if (!u || !n) {
    set_error("unet_num_params: null argument");
    return PF_EINVAL;
  }
  *n = u->nparam;
  return PF_OK;
}

pf_status pf_unet_set_params(pf_unet* u, const float* params) {
  if (!u || !params) {
    set_error("unet_set_params: null argument");
    return PF_EINVAL;
  }
  cudaError_t e = cudaMemcpyAsync(u->w32, params, sizeof(float) * u->nparam, cudaMemcpyHostToDevice, u->st);
  if (e == cudaSuccess) {
    k_to_bf16<<<grid1(u->nparam), 256, 0, u->st>>>(u->w32, u->wbf, u->nparam);
    cudaMemsetAsync(u->m, 0, sizeof(float) * u->nparam, u->st);
    cudaMemsetAsync(u->v, 0, sizeof(float) * u->nparam, u->st);
    cudaMemsetAsync(u->g, 0, sizeof(float) * u->nparam, u->st);
    u->adam_t = 0;
    e = cudaStreamSynchronize(u->st);
  }
  if (e != cudaSuccess) {
    set_error(std::string("unet_set_params: ") + cudaGetErrorString(e));
    return PF_ECUDA;
  }
  return PF_OK;
}

static pf_status copy_out(pf_unet* u, const float* src, float* dst, const char* what) {
  if (!u || !dst) {
    set_error(std::string(what) + ": null argument");
    return PF_EINVAL;
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(float) * u->nparam, cudaMemcpyDeviceToHost, u->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->st);
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return PF_ECUDA;
  }
  return PF_OK;
}

pf_status pf_unet_get_params(pf_unet* u, float* params) { return copy_out(u, u ? u->w32 : nullptr, params, "unet_get_params"); }
pf_status pf_unet_get_grads(pf_unet* u, float* grads) { return copy_out(u, u ? u->g : nullptr, grads, "unet_get_grads"); }

pf_status pf_unet_forward(pf_unet* u, const float* x, float* y) {
  if (!u || !x || !y) {
    set_error("unet_forward: null argument");
    return PF_EINVAL;
  }
  const long long HW = (long long)u->H * u->W;
  k_to_bf16<<<grid1(u->nin * HW), 256, 0, u->st>>>(x, u->xin, u->nin * HW);
  const int nl = int(u->layers.size());
  for (int l = 0; l < nl; ++l) {
    const ConvLayer& c = u->layers[l];
    const int lev = layer_level(u, l);
    const int H = u->H >> lev, W = u->W >> lev;
    const ConvIn in = layer_input(u, l);
    const __nv_bfloat16* w = u->wbf + c.off_w;
    const float* b = u->w32 + c.off_b;
    MmaIn src{};
    src.conv = in;
    if (c.k == 3)
      launch_conv_mma<3, false>(src, H, W, c.co, c.ci, c.ci, w, b, 1, u->act[l], nullptr, u->st);
    else
      launch_conv_mma<1, false>(src, H, W, c.co, c.ci, c.ci, w, b, 0, nullptr, y, u->st);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("unet_forward: ") + cudaGetErrorString(e));
    return PF_ECUDA;
  }
  return PF_OK;
}

// Backward from dL/dy (FP32, n_out x H x W); parameter gradients are added to
// the accumulated gradient (zeroed by pf_unet_adam or pf_unet_set_params).
pf_status pf_unet_backward(pf_unet* u, const float* dy) {
  if (!u || !dy) {
    set_error("unet_backward: null argument");
    return PF_EINVAL;
  }
  const int nl = int(u->layers.size());
  const long long HW = (long long)u->H * u->W;
  for (int l = 0; l < nl - 1; ++l) {
    const int lev = layer_level(u, l);
    cudaMemsetAsync(u->gact[l], 0, sizeof(float) * u->layers[l].co * (HW >> (2 * lev)), u->st);
  }
  for (int l = nl - 1; l >= 0; --l) {
    const ConvLayer& c = u->layers[l];
    const int lev = layer_level(u, l);
    const int H = u->H >> lev, W = u->W >> lev;
    const ConvIn in = layer_input(u, l);
    const float* dout = (l == nl - 1) ? dy : u->gact[l];
    const __nv_bfloat16* out = (l == nl - 1) ? nullptr : u->act[l];
    const int relu = c.relu ? 1 : 0;
    // weight and bias gradients
    const int P = wgrad_chunks(H, W, c.ci, c.co, u->sms);
    const long long nw = (long long)c.co * c.ci * c.k * c.k;
    float* part_b = u->wpart + (long long)P * nw;
    if (c.k == 3)
      launch_wgrad_mma<3>(dout, out, relu, in, H, W, c.co, P, u->wpart, part_b, u->st);
    else
      launch_wgrad_mma<1>(dout, out, relu, in, H, W, c.co, P, u->wpart, part_b, u->st);
    k_sum_parts<<<grid1(nw), 256, 0, u->st>>>(u->wpart, P, nw, u->g + c.off_w);
    k_sum_parts<<<grid1(c.co), 256, 0, u->st>>>(part_b, P, c.co, u->g + c.off_b);
    if (l == 0) continue;  // no gradient needed for the input features
    // data gradient on the conv grid, then the adjoint of the input transform
    const __nv_bfloat16* w = u->wbf + c.off_w;
    MmaIn src{};
    src.dout = dout;
    src.out = out;
    src.relu = relu;
    if (c.k == 3)
      launch_conv_mma<3, true>(src, H, W, c.ci, c.co, c.ci, w, nullptr, 0, nullptr, u->dscratch, u->st);
    else
      launch_conv_mma<1, true>(src, H, W, c.ci, c.co, c.ci, w, nullptr, 0, nullptr, u->dscratch, u->st);
    // operand a is the output of layer l-1; operand b (decoder) a skip
    float* ga = u->gact[l - 1];
    float* gb = nullptr;
    if (in.cb > 0) {
      const int d = l - 2 * u->L;
      const int k = u->L - 2 - d / 2;
      gb = u->gact[2 * k + 1];
    }
    k_in_adjoint<<<grid1((long long)c.ci * H * W * 4), 256, 0, u->st>>>(u->dscratch, H, W, in.ca, in.mode,
                                                                         in.cb, ga, gb);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("unet_backward: ") + cudaGetErrorString(e));
    return PF_ECUDA;
  }
  return PF_OK;
}

pf_status pf_unet_adam(pf_unet* u, float lr, float beta1, float beta2, float eps, float grad_scale) {
  if (!u || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0)) {
    set_error("unet_adam: bad argument");
    return PF_EINVAL;
  }
  u->adam_t += 1;
  const float c1 = 1.f - std::pow(beta1, float(u->adam_t)), c2 = 1.f - std::pow(beta2, float(u->adam_t));
  k_adam<<<grid1(u->nparam), 256, 0, u->st>>>(u->w32, u->m, u->v, u->g, u->wbf, u->nparam, lr, beta1,
                                               beta2, eps, c1, c2, grad_scale);
  cudaMemsetAsync(u->g, 0, sizeof(float) * u->nparam, u->st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("unet_adam: ") + cudaGetErrorString(e));
    return PF_ECUDA;
  }
  return PF_OK;
}

pf_status pf_unet_mse(pf_unet* u, const float* y, const float* t, const float* mask,
                      double n_valid, float* dy, double* loss) {
  if (!u || !y || !t || !dy || !loss || !(n_valid > 0)) {
    set_error("unet_mse: bad argument");
    return PF_EINVAL;
  }
  const long long HW = (long long)u->H * u->W;
  const double n = double(u->nout) * (mask ? n_valid : double(HW));
  const int nb = std::min(grid1(u->nout * HW), 8192);
  k_mse<<<nb, 256, 0, u->st>>>(y, t, mask, u->nout, HW, 1.0 / n, dy, u->lpart);
  cudaError_t e = cudaMemcpyAsync(u->h_loss, u->lpart, sizeof(double) * nb, cudaMemcpyDeviceToHost, u->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->st);
  if (e != cudaSuccess) {
    set_error(std::string("unet_mse: ") + cudaGetErrorString(e));
    return PF_ECUDA;
  }
  double s = 0;
  for (int i = 0; i < nb; ++i) s += u->h_loss[i];
  *loss = s;
  return PF_OK;
}

}  // extern "C"
