// agg_theta_gradient: per-element log-conductivity gradients reduced to the
// mesh's conductivity parameters (D_e = theta_k D0_e for k = theta_map[e]):
// dL/dtheta_k = sum_{e in k} dL/dlog s_e / theta_k. The elements of each
// parameter are grouped on the host once (CSR in increasing element order)
// and uploaded on the first call; the device sums each group with one warp,
// lane-strided then by shuffles, so the result does not depend on timing.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/aggmg.h"
#include "engine.h"
#include "handles.h"
#include "kernels.cuh"

namespace aggmg {

static __global__ void k_theta_reduce(const int32_t* __restrict__ ptr, const int32_t* __restrict__ mem,
                                      const double* __restrict__ theta, const double* __restrict__ g,
                                      double* __restrict__ out, int64_t nk) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= nk) return;
  double s = 0.0;
  for (int32_t i = ptr[k] + lane; i < ptr[k + 1]; i += 32) s += g[mem[i]];
  s = warp_sum(s);
  if (lane == 0) out[k] += s / theta[k];
}

}  // namespace aggmg

namespace {

agg_status theta_fail(agg_status s, const std::string& msg) {
  aggmg::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" agg_status agg_theta_gradient(agg_hier_t h, const double* g, double* out, void* stream) {
  if (!h || !g || !out) return theta_fail(AGG_EINVAL, "NULL argument");
  const aggmg::Mesh& m = h->mesh->m;
  if (m.theta.empty()) return theta_fail(AGG_EINVAL, "the hierarchy's mesh has no conductivity parameters (theta)");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
    return theta_fail(AGG_EINVAL, "current device differs from the hierarchy's device");
  const int64_t nk = (int64_t)m.theta.size();
  if (!h->d_tptr) {
    std::vector<int32_t> ptr(nk + 1, 0), mem(m.ne);
    for (int64_t e = 0; e < m.ne; ++e) ptr[m.theta_map[e] + 1] += 1;
    for (int64_t k = 0; k < nk; ++k) ptr[k + 1] += ptr[k];
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t e = 0; e < m.ne; ++e) mem[fill[m.theta_map[e]]++] = (int32_t)e;
    int32_t *dp = nullptr, *dm = nullptr;
    double* dt = nullptr;
    if (cudaMalloc(&dp, sizeof(int32_t) * ptr.size()) != cudaSuccess ||
        cudaMalloc(&dm, sizeof(int32_t) * mem.size()) != cudaSuccess ||
        cudaMalloc(&dt, sizeof(double) * nk) != cudaSuccess) {
      cudaFree(dp);
      cudaFree(dm);
      cudaFree(dt);
      cudaGetLastError();
      return theta_fail(AGG_ENOMEM, "cudaMalloc for the theta groups failed");
    }
    if (cudaMemcpy(dp, ptr.data(), sizeof(int32_t) * ptr.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dm, mem.data(), sizeof(int32_t) * mem.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dt, m.theta.data(), sizeof(double) * nk, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(dp);
      cudaFree(dm);
      cudaFree(dt);
      return theta_fail(AGG_ECUDA, "upload of the theta groups failed");
    }
    h->d_tptr = dp;
    h->d_tmem = dm;
    h->d_theta = dt;
  }
  const int64_t threads = nk * 32;
  aggmg::k_theta_reduce<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      h->d_tptr, h->d_tmem, h->d_theta, g, out, nk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return theta_fail(AGG_ECUDA, std::string("k_theta_reduce: ") + cudaGetErrorString(e));
  return AGG_OK;
}
