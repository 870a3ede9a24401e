// pf_energy_noalloc: the discrete energy for callers that must not allocate
// device memory.  Its reduction scratch (one partial sum per block and a
// completion counter) lives in a fixed array in the library's own device
// memory instead of a buffer obtained from cudaMalloc.
#include <cuda.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/pf.h"
#include "pf_internal.h"

namespace pf {
void set_error(const std::string& msg);
}

using namespace pf;

namespace {

// 65,536 block partials (512 KiB) plus a 256-byte slot for the counter.
// Each block of the energy kernel reduces 256 elements, so a grid may have
// at most 65,536 * 256 = 16,777,216 elements.
constexpr long long kNoAllocPartials = 65536;
constexpr long long kNoAllocMaxElements = kNoAllocPartials * 256;
constexpr size_t kNoAllocBytes = kNoAllocPartials * sizeof(double) + 256;

// Zero-initialised when the module loads on a device and kept until the
// process exits; every device that loads the library holds its own copy.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device addresses of g_noalloc_scratch, looked up once per device and
// context.  In host code the symbol names a host-side stand-in, never the
// device array.  The address belongs to the context that loaded the module:
// after cudaDeviceReset (or any teardown of the device's context) the next
// call sees a new context id and looks the address up again, so no call
// writes through the address of a context that is gone.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Id of the calling thread's current context (0 if none), through driver
// entry points obtained from the runtime (the library links no libcuda).
cudaError_t current_context_id(unsigned long long* id) {
  *id = 0;
  if (!g_ctx_get_current || !g_ctx_get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&g_ctx_get_current,
                                                     12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess)
      e = cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&g_ctx_get_id, 12000,
                                           cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
      g_ctx_get_current = nullptr;
      g_ctx_get_id = nullptr;
      return cudaErrorSymbolNotFound;
    }
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
  if (!ctx) return cudaSuccess;
  if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
  return cudaSuccess;
}

cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  unsigned long long ctx = 0;
  e = current_context_id(&ctx);
  if (e != cudaSuccess) return e;
  if (!g_scratch_dev[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the device's context current
    if (e != cudaSuccess) return e;
    e = current_context_id(&ctx);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" pf_status pf_energy_noalloc(int dim, const int n[3], double h, double E, double nu,
                                       double Gc, double ls, double k_res, double p,
                                       const void* x_dev, int prec, double* E_dev,
                                       void* stream) {
  if (dim != 2 && dim != 3) {
    set_error("energy_noalloc: dim must be 2 or 3");
    return PF_EINVAL;
  }
  if (!n || !x_dev || !E_dev) {
    set_error("energy_noalloc: null argument");
    return PF_EINVAL;
  }
  if (prec != PF_FP64 && prec != PF_FP32) {
    set_error("energy_noalloc: precision must be PF_FP64 or PF_FP32");
    return PF_EINVAL;
  }
  if (!(h > 0) || !(E > 0) || !(Gc > 0) || !(ls > 0) || !(nu > -1.0 && nu < 0.5) ||
      !(k_res >= 0 && k_res < 1) || !std::isfinite(p)) {
    set_error("energy_noalloc: invalid spacing, material or pressure");
    return PF_EINVAL;
  }
  long long ne = 1;
  for (int k = 0; k < dim; ++k) {
    if (n[k] < 2 || n[k] > (1 << 20)) {
      set_error("energy_noalloc: each axis needs 2 .. 2^20 nodes");
      return PF_EINVAL;
    }
    ne *= n[k] - 1;
    if (ne > kNoAllocMaxElements) {
      set_error("energy_noalloc: grid has more than 16,777,216 elements, the most its static "
                "reduction scratch (65,536 block partials) can hold; use pf_energy");
      return PF_EINVAL;
    }
  }
  unsigned char* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    set_error(std::string("energy_noalloc: device scratch lookup failed: ") + cudaGetErrorString(e));
    return PF_ECUDA;
  }
  double* partials = reinterpret_cast<double*>(scratch);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNoAllocPartials * sizeof(double));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Geom g = make_geom(dim, n, h);
  const Mat<double> m = make_mat(g, E, nu, Gc, ls, k_res, p);
  const int nblocks = int((g.NE + 255) / 256);
  // the counter must start at zero even if an earlier call was cut short
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = elem_energy_blocks(g, m, x_dev, prec, partials, counter, nblocks, E_dev, st);
  if (e != cudaSuccess) {
    set_error(std::string("energy_noalloc: ") + cudaGetErrorString(e));
    return PF_ECUDA;
  }
  return PF_OK;
}
