// Deterministic block and grid reductions.  A grid reduction writes one
// partial per block, and the last block to finish (counted with an atomic
// ticket) combines the partials in block order, so the result does not
// depend on block scheduling.
#pragma once
#include <cuda_runtime.h>

#include "pf_internal.h"

namespace pf {

// FP32 overloads serve per-thread partial results of FP32 vectors; blocks
// and the grid always combine in FP64.
struct OpSum {
  static __device__ __forceinline__ double id() { return 0.0; }
  static __device__ __forceinline__ double op(double a, double b) { return a + b; }
  static __device__ __forceinline__ float op(float a, float b) { return a + b; }
};
struct OpMax {
  static __device__ __forceinline__ double id() { return -INFINITY; }
  static __device__ __forceinline__ double op(double a, double b) { return fmax(a, b); }
  static __device__ __forceinline__ float op(float a, float b) { return fmaxf(a, b); }
};
struct OpMin {
  static __device__ __forceinline__ double id() { return INFINITY; }
  static __device__ __forceinline__ double op(double a, double b) { return fmin(a, b); }
  static __device__ __forceinline__ float op(float a, float b) { return fminf(a, b); }
};

template <int K, class Op>
__device__ __forceinline__ void block_reduce(double (&v)[K]) {
  __shared__ double sh[K][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = Op::op(v[k], __shfl_down_sync(0xffffffffu, v[k], o));
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][wid] = v[k];
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      v[k] = lane < nw ? sh[k][lane] : Op::id();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] = Op::op(v[k], __shfl_down_sync(0xffffffffu, v[k], o));
    }
  }
}

template <int K, class Op>
__device__ __forceinline__ void grid_finish(double (&v)[K], double* partials, unsigned* counter,
                                            double* out) {
  __shared__ bool last;
  block_reduce<K, Op>(v);
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[k * kMaxBlocks + blockIdx.x] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == unsigned(nb - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    acc[k] = Op::id();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      acc[k] = Op::op(acc[k], __ldcg(partials + k * kMaxBlocks + b));
  }
  block_reduce<K, Op>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = acc[k];
    *counter = 0u;
  }
}

// As grid_finish, but the last block's thread 0 hands the combined values to
// fin(acc) instead of storing them (device-side control logic).
template <int K, class Op, class Fin>
__device__ __forceinline__ void grid_finish_fn(double (&v)[K], double* partials, unsigned* counter,
                                               Fin& fin) {
  __shared__ bool last;
  block_reduce<K, Op>(v);
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[k * kMaxBlocks + blockIdx.x] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == unsigned(nb - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    acc[k] = Op::id();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      acc[k] = Op::op(acc[k], __ldcg(partials + k * kMaxBlocks + b));
  }
  block_reduce<K, Op>(acc);
  if (threadIdx.x == 0) {
    fin(acc);
    __threadfence();
    *counter = 0u;
  }
}

inline int reduce_grid(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  if (b > kMaxBlocks) b = kMaxBlocks;
  if (b < 1) b = 1;
  return int(b);
}

}  // namespace pf
