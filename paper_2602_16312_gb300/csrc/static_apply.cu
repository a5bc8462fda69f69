// agg_operator_apply_static: the level-operator product of agg_operator_apply
// for callers that must not allocate device memory. The two unit-permuted
// work vectors live in one file-scope device array instead of the
// hierarchy's work buffers; the entry point itself calls no allocator.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/aggmg.h"
#include "engine.h"
#include "handles.h"

namespace {

// Two vectors of up to AGG_STATIC_APPLY_MAX_ENTRIES doubles each (16 MiB in
// total), held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_static_apply_scratch[2 * AGG_STATIC_APPLY_MAX_ENTRIES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host symbol is not a device address).
agg_status scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    aggmg::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return AGG_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    aggmg::set_last_error("device ordinal out of range for the static scratch table");
    return AGG_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_apply_scratch);
    if (e != cudaSuccess || !p) {
      aggmg::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return AGG_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return AGG_OK;
}

}  // namespace

extern "C" agg_status agg_operator_apply_static(agg_hier_t h, int level, const double* x, double* y, void* stream) {
  if (!h || !x || !y) {
    aggmg::set_last_error("NULL argument");
    return AGG_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) {
    aggmg::set_last_error("current device differs from the hierarchy's device");
    return AGG_EINVAL;
  }
  const int64_t need = h->eng->level_scratch_entries(level);
  if (need < 0 || level >= h->L - 1) {
    aggmg::set_last_error("level out of range (levels 0 .. n_levels-2 have a stored operator)");
    return AGG_EINVAL;
  }
  if (need > AGG_STATIC_APPLY_MAX_ENTRIES) {
    aggmg::set_last_error("level " + std::to_string(level) + " needs " + std::to_string(need) +
                          " scratch entries per vector; agg_operator_apply_static supports at most " +
                          std::to_string((long long)AGG_STATIC_APPLY_MAX_ENTRIES));
    return AGG_EINVAL;
  }
  void* base = nullptr;
  agg_status s = scratch_address(&base);
  if (s) return s;
  double* s_in = static_cast<double*>(base);
  double* s_out = s_in + AGG_STATIC_APPLY_MAX_ENTRIES;
  std::string err;
  int rc = h->eng->apply_level_scratch(level, x, y, s_in, s_out, (cudaStream_t)stream, err);
  if (rc) {
    aggmg::set_last_error(err);
    return (agg_status)rc;
  }
  return AGG_OK;
}
