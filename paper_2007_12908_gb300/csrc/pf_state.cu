// Checkpoint and resume of a load-step sequence.  The paper's workflow
// (Sec. 4.1) exports the state after every pseudo-time step; here that state
// is written to a file that pf_state_load can later restore into a hierarchy
// of the same grid and material, so that a ramp resumes at the step after
// the checkpoint and reproduces the uninterrupted run bit for bit.
//
// File layout (host byte order, recorded in the header):
//   StateHeader, then the finest FP64 state x ((dim+1) N values), then c_prev
//   (N values).  The header's checksum is FNV-1a (64-bit) over the payload.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pf_hier.h"

namespace pf {
void set_error(const std::string& msg);
}

using namespace pf;

namespace {

constexpr char kMagic[8] = {'P', 'F', 'S', 'T', 'A', 'T', 'E', 0};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kByteOrder = 0x01020304u;

struct StateHeader {
  char magic[8];
  uint32_t version, byte_order;
  int32_t dim, levels, n[3], reserved;
  double h, E, nu, Gc, ls, k_res;
  double p, p_last;
  uint64_t n_x, n_c;
  uint64_t checksum;
};

uint64_t fnv1a(const void* data, size_t bytes, uint64_t h = 1469598103934665603ull) {
  const unsigned char* b = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < bytes; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

pf_status fail(pf_status rc, const std::string& msg) {
  set_error(msg);
  return rc;
}

void fill_header(const pf_hierarchy* H, StateHeader* hd) {
  std::memset(hd, 0, sizeof *hd);
  std::memcpy(hd->magic, kMagic, sizeof kMagic);
  hd->version = kVersion;
  hd->byte_order = kByteOrder;
  const Geom& g = H->geo.back();
  hd->dim = H->dim;
  hd->levels = H->L;
  for (int k = 0; k < 3; ++k) hd->n[k] = g.n[k];
  hd->h = g.h;
  hd->E = H->E;
  hd->nu = H->nu;
  hd->Gc = H->Gc;
  hd->ls = H->ls;
  hd->k_res = H->k_res;
  hd->p = H->p;
  hd->p_last = H->p_last;
  hd->n_x = uint64_t(H->dim + 1) * uint64_t(g.N);
  hd->n_c = uint64_t(g.N);
}

}  // namespace

extern "C" {

pf_status pf_state_save(pf_hierarchy* H, const double* x_dev, const char* path) {
  if (!H || !x_dev || !path) return fail(PF_EINVAL, "state_save: null argument");
  StateHeader hd;
  fill_header(H, &hd);
  std::vector<double> buf(hd.n_x + hd.n_c);
  cudaError_t e = cudaMemcpyAsync(buf.data(), x_dev, sizeof(double) * hd.n_x,
                                  cudaMemcpyDeviceToHost, H->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(buf.data() + hd.n_x, H->c_prev, sizeof(double) * hd.n_c,
                        cudaMemcpyDeviceToHost, H->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(H->st);
  if (e != cudaSuccess) return fail(PF_ECUDA, std::string("state_save: ") + cudaGetErrorString(e));
  for (double v : buf)
    if (!std::isfinite(v)) return fail(PF_ENONFINITE, "state_save: the state holds a non-finite value");
  hd.checksum = fnv1a(buf.data(), sizeof(double) * buf.size());
  // write beside the target and rename, so that a reader never sees half a file
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(PF_EIO, "state_save: cannot open " + tmp + " for writing");
  bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1 &&
            std::fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  ok = (std::fflush(f) == 0) && ok;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(PF_EIO, std::string("state_save: writing ") + path + " failed");
  }
  return PF_OK;
}

pf_status pf_state_load(pf_hierarchy* H, double* x_dev, const char* path) {
  if (!H || !x_dev || !path) return fail(PF_EINVAL, "state_load: null argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(PF_EIO, std::string("state_load: cannot open ") + path);
  StateHeader hd;
  if (std::fread(&hd, sizeof hd, 1, f) != 1) {
    std::fclose(f);
    return fail(PF_EIO, "state_load: file shorter than its header");
  }
  StateHeader want;
  fill_header(H, &want);
  if (std::memcmp(hd.magic, kMagic, sizeof kMagic) != 0 || hd.version != kVersion ||
      hd.byte_order != kByteOrder) {
    std::fclose(f);
    return fail(PF_EINVAL, "state_load: not a libpf state file of this version and byte order");
  }
  if (hd.dim != want.dim || hd.levels != want.levels || hd.n[0] != want.n[0] ||
      hd.n[1] != want.n[1] || hd.n[2] != want.n[2] || hd.h != want.h || hd.n_x != want.n_x ||
      hd.n_c != want.n_c) {
    std::fclose(f);
    return fail(PF_EINVAL, "state_load: the file was written for another grid hierarchy");
  }
  if (hd.E != want.E || hd.nu != want.nu || hd.Gc != want.Gc || hd.ls != want.ls ||
      hd.k_res != want.k_res) {
    std::fclose(f);
    return fail(PF_EINVAL, "state_load: the file was written for another material");
  }
  std::vector<double> buf(hd.n_x + hd.n_c);
  const size_t got = std::fread(buf.data(), sizeof(double), buf.size(), f);
  const bool trailing = std::fgetc(f) != EOF;
  std::fclose(f);
  if (got != buf.size() || trailing)
    return fail(PF_EIO, "state_load: payload size does not match the header");
  if (fnv1a(buf.data(), sizeof(double) * buf.size()) != hd.checksum)
    return fail(PF_EINVAL, "state_load: checksum mismatch (the file is corrupt)");
  for (double v : buf)
    if (!std::isfinite(v)) return fail(PF_ENONFINITE, "state_load: non-finite value in the file");
  if (!std::isfinite(hd.p) || !std::isfinite(hd.p_last))
    return fail(PF_ENONFINITE, "state_load: non-finite pressure in the file");
  // every check passed: only now is anything changed
  cudaError_t e = cudaMemcpyAsync(x_dev, buf.data(), sizeof(double) * hd.n_x,
                                  cudaMemcpyHostToDevice, H->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(H->c_prev, buf.data() + hd.n_x, sizeof(double) * hd.n_c,
                        cudaMemcpyHostToDevice, H->st);
  const float p32 = float(hd.p);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(H->p_dev, &p32, sizeof(float), cudaMemcpyHostToDevice, H->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(H->st);
  if (e != cudaSuccess) return fail(PF_ECUDA, std::string("state_load: ") + cudaGetErrorString(e));
  H->p = hd.p;
  for (auto& m : H->mat) m.p = hd.p;
  H->p_last = hd.p_last;
  H->bounds_set = false;
  H->have_fractures = true;
  return PF_OK;
}

}  // extern "C"
