// Learned initial iterate: a 2D U-Net (4 levels, two 3x3 convolutions +
// ReLU per level, 2x2 average pooling down, nearest 2x up, skip
// concatenation, 1x1 head).  BF16 weights and activations, FP32 arithmetic
// and accumulation, FP32 master weights and Adam moments.
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

constexpr int TILE = 16, COB = 16, CIB = 8;

// y[co] = relu?(b[co] + sum_ci sum_k w[co][ci][k] in[ci](y + dy, x + dx))
// grid: (W/16, H/16, ceil(CO/16)), block 256 threads, one pixel each.
template <int K>
__global__ void __launch_bounds__(256) k_conv_fwd(ConvIn in, int H, int W, int CO,
                                                  const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ bias, int relu,
                                                  __nv_bfloat16* __restrict__ out_bf,
                                                  float* __restrict__ out_f) {
  constexpr int R = K / 2, T = TILE + 2 * R;
  __shared__ float tile[CIB][T][T];
  __shared__ float ws[COB][CIB][K * K];
  const int CI = in.ca + in.cb;
  const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
  const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE, co0 = blockIdx.z * COB;
  float acc[COB];
#pragma unroll
  for (int c = 0; c < COB; ++c) acc[c] = 0.f;
  for (int ci0 = 0; ci0 < CI; ci0 += CIB) {
    for (int i = threadIdx.x; i < CIB * T * T; i += 256) {
      const int c = i / (T * T), r = i % (T * T);
      const int yy = y0 + r / T - R, xx = x0 + r % T - R;
      tile[c][r / T][r % T] = (ci0 + c < CI) ? conv_in(in, ci0 + c, yy, xx, H, W) : 0.f;
    }
    for (int i = threadIdx.x; i < COB * CIB * K * K; i += 256) {
      const int co = i / (CIB * K * K), rem = i % (CIB * K * K);
      const int c = rem / (K * K), k = rem % (K * K);
      ws[co][c][k] = (co0 + co < CO && ci0 + c < CI)
                         ? __bfloat162float(w[((long long)(co0 + co) * CI + ci0 + c) * K * K + k])
                         : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CIB; ++c)
#pragma unroll
      for (int k = 0; k < K * K; ++k) {
        const float v = tile[c][ty + k / K][tx + k % K];
#pragma unroll
        for (int co = 0; co < COB; ++co) acc[co] = fmaf(ws[co][c][k], v, acc[co]);
      }
    __syncthreads();
  }
  const int y = y0 + ty, x = x0 + tx;
  if (y >= H || x >= W) return;
#pragma unroll
  for (int co = 0; co < COB; ++co) {
    if (co0 + co >= CO) break;
    float v = acc[co] + bias[co0 + co];
    if (relu) v = fmaxf(v, 0.f);
    const long long o = ((long long)(co0 + co) * H + y) * W + x;
    if (out_bf) out_bf[o] = __float2bfloat16(v);
    if (out_f) out_f[o] = v;
  }
}

// Data gradient: dIn[ci](y, x) = sum_co sum_k w[co][ci][k] dpre[co](y - dy, x - dx),
// dpre = dout * (out > 0) when the layer has a ReLU.  Written FP32 on the
// conv's own grid (the virtual concatenated input).
template <int K>
__global__ void __launch_bounds__(256) k_conv_dgrad(const float* __restrict__ dout,
                                                    const __nv_bfloat16* __restrict__ out, int relu,
                                                    int H, int W, int CO, int CI,
                                                    const __nv_bfloat16* __restrict__ w,
                                                    float* __restrict__ din) {
  constexpr int R = K / 2, T = TILE + 2 * R;
  __shared__ float tile[CIB][T][T];
  __shared__ float ws[COB][CIB][K * K];  // [ci][co][k], flipped taps
  const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
  const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE, ci0 = blockIdx.z * COB;
  float acc[COB];
#pragma unroll
  for (int c = 0; c < COB; ++c) acc[c] = 0.f;
  for (int co0 = 0; co0 < CO; co0 += CIB) {
    for (int i = threadIdx.x; i < CIB * T * T; i += 256) {
      const int c = i / (T * T), r = i % (T * T);
      const int yy = y0 + r / T - R, xx = x0 + r % T - R;
      float v = 0.f;
      if (co0 + c < CO && yy >= 0 && yy < H && xx >= 0 && xx < W) {
        const long long o = ((long long)(co0 + c) * H + yy) * W + xx;
        v = dout[o];
        if (relu && !(__bfloat162float(out[o]) > 0.f)) v = 0.f;
      }
      tile[c][r / T][r % T] = v;
    }
    for (int i = threadIdx.x; i < COB * CIB * K * K; i += 256) {
      const int ci = i / (CIB * K * K), rem = i % (CIB * K * K);
      const int c = rem / (K * K), k = rem % (K * K);
      ws[ci][c][k] = (ci0 + ci < CI && co0 + c < CO)
                         ? __bfloat162float(w[((long long)(co0 + c) * CI + ci0 + ci) * K * K + (K * K - 1 - k)])
                         : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CIB; ++c)
#pragma unroll
      for (int k = 0; k < K * K; ++k) {
        const float v = tile[c][ty + k / K][tx + k % K];
#pragma unroll
        for (int ci = 0; ci < COB; ++ci) acc[ci] = fmaf(ws[ci][c][k], v, acc[ci]);
      }
    __syncthreads();
  }
  const int y = y0 + ty, x = x0 + tx;
  if (y >= H || x >= W) return;
#pragma unroll
  for (int ci = 0; ci < COB; ++ci) {
    if (ci0 + ci >= CI) break;
    din[((long long)(ci0 + ci) * H + y) * W + x] = acc[ci];
  }
}

// Weight gradient partials: part[p][co][ci][k] = sum over the pixel rows of
// chunk p of dpre[co](y, x) in[ci](y + dy, x + dx), and part_b[p][co] = sum
// of dpre.  grid: (ceil(CI/8), ceil(CO/8), P) blocks of 256 threads; the
// 8 x 8 x K*K (co, ci, tap) triples of a block are dealt round-robin to the
// threads (up to NT each), and every sum runs over pixels in a fixed order.
constexpr int WG_C = 8;
template <int K>
__global__ void __launch_bounds__(256) k_conv_wgrad(const float* __restrict__ dout,
                                                    const __nv_bfloat16* __restrict__ out, int relu,
                                                    ConvIn in, int H, int W, int CO, int rows_per,
                                                    float* __restrict__ part, float* __restrict__ part_b) {
  constexpr int R = K / 2, T = TILE + 2 * R;
  constexpr int NTRI = WG_C * WG_C * K * K, NT = (NTRI + 255) / 256;
  const int CI = in.ca + in.cb;
  const int ci0 = blockIdx.x * WG_C, co0 = blockIdx.y * WG_C, p = blockIdx.z;
  const int y_lo = p * rows_per, y_hi = min(H, y_lo + rows_per);
  __shared__ float sd[WG_C][TILE * TILE];
  __shared__ float sx[WG_C][T * T];
  const int t = threadIdx.x;
  float acc[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j] = 0.f;
  float accb = 0.f;  // bias sum of output channel co0 + t (threads t < 8)
  for (int yb = y_lo; yb < y_hi; yb += TILE)
    for (int xb = 0; xb < W; xb += TILE) {
      for (int i = t; i < WG_C * TILE * TILE; i += 256) {
        const int c = i / (TILE * TILE), r = i % (TILE * TILE);
        const int yy = yb + r / TILE, xx = xb + r % TILE;
        float v = 0.f;
        if (co0 + c < CO && yy < y_hi && xx < W) {
          const long long o = ((long long)(co0 + c) * H + yy) * W + xx;
          v = dout[o];
          if (relu && !(__bfloat162float(out[o]) > 0.f)) v = 0.f;
        }
        sd[c][r] = v;
      }
      for (int i = t; i < WG_C * T * T; i += 256) {
        const int c = i / (T * T), r = i % (T * T);
        const int yy = yb + r / T - R, xx = xb + r % T - R;
        sx[c][r] = (ci0 + c < CI) ? conv_in(in, ci0 + c, yy, xx, H, W) : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int tri = t + 256 * j;
        if (tri < NTRI) {
          const int co = tri / (WG_C * K * K), rem = tri % (WG_C * K * K);
          const int ci = rem / (K * K), k = rem % (K * K);
          const int dy = k / K, dx = k % K;
          float a = acc[j];
          for (int r = 0; r < TILE * TILE; ++r)
            a = fmaf(sd[co][r], sx[ci][(r / TILE + dy) * T + r % TILE + dx], a);
          acc[j] = a;
        }
      }
      if (t < WG_C)
        for (int r = 0; r < TILE * TILE; ++r) accb += sd[t][r];
      __syncthreads();
    }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int tri = t + 256 * j;
    if (tri < NTRI) {
      const int co = tri / (WG_C * K * K), rem = tri % (WG_C * K * K);
      const int ci = rem / (K * K), k = rem % (K * K);
      if (co0 + co < CO && ci0 + ci < CI)
        part[(((long long)p * CO + co0 + co) * CI + ci0 + ci) * K * K + k] = acc[j];
    }
  }
  if (t < WG_C && blockIdx.x == 0 && co0 + t < CO) part_b[(long long)p * CO + co0 + t] = accb;
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
    const int H_l = height >> lev;
    const int P = (H_l + 31) / 32;
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
    dim3 grid((W + TILE - 1) / TILE, (H + TILE - 1) / TILE, (c.co + COB - 1) / COB);
    const __nv_bfloat16* w = u->wbf + c.off_w;
    const float* b = u->w32 + c.off_b;
    if (c.k == 3)
      k_conv_fwd<3><<<grid, 256, 0, u->st>>>(in, H, W, c.co, w, b, 1, u->act[l], nullptr);
    else
      k_conv_fwd<1><<<grid, 256, 0, u->st>>>(in, H, W, c.co, w, b, 0, nullptr, y);
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
    const int rows = 32, P = (H + rows - 1) / rows;
    dim3 gw((c.ci + WG_C - 1) / WG_C, (c.co + WG_C - 1) / WG_C, P);
    const long long nw = (long long)c.co * c.ci * c.k * c.k;
    float* part_b = u->wpart + (long long)P * nw;
    if (c.k == 3)
      k_conv_wgrad<3><<<gw, 256, 0, u->st>>>(dout, out, relu, in, H, W, c.co, rows, u->wpart, part_b);
    else
      k_conv_wgrad<1><<<gw, 256, 0, u->st>>>(dout, out, relu, in, H, W, c.co, rows, u->wpart, part_b);
    k_sum_parts<<<grid1(nw), 256, 0, u->st>>>(u->wpart, P, nw, u->g + c.off_w);
    k_sum_parts<<<grid1(c.co), 256, 0, u->st>>>(part_b, P, c.co, u->g + c.off_b);
    if (l == 0) continue;  // no gradient needed for the input features
    // data gradient on the conv grid, then the adjoint of the input transform
    dim3 gd((W + TILE - 1) / TILE, (H + TILE - 1) / TILE, (c.ci + COB - 1) / COB);
    const __nv_bfloat16* w = u->wbf + c.off_w;
    if (c.k == 3)
      k_conv_dgrad<3><<<gd, 256, 0, u->st>>>(dout, out, relu, H, W, c.co, c.ci, w, u->dscratch);
    else
      k_conv_dgrad<1><<<gd, 256, 0, u->st>>>(dout, out, relu, H, W, c.co, c.ci, w, u->dscratch);
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
