// Interface between the C ABI (capi.cu) and the per-block-size device
// engines (engine_b*.cu). One engine owns the device copy of a hierarchy
// and the CUDA graphs of the solver.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/aggmg.h"
#include "setup.h"

namespace aggmg {

struct SolveOpts {
  double rtol = 1e-8, atol = 0.0;
  int max_it = 500, flexible = 0;
};

struct SolveResult {
  int iterations = 0, status = 0;
  double r0 = 0, rn = 0;
};

struct SimParams {
  int model = 0;
  double k = 0, a = 0, eps = 0, gamma = 0, mu1 = 0, mu2 = 0;
  agg_bueno_orovio_params bo{};
  double dt = 0, chi = 1, cm = 1;
  double iapp_value = 0;
  int64_t iapp_steps = 0;
  int scheme = 0;              // 0 IMEX backward Euler, 1 BDF2 with extrapolation
  SolveOpts pcg;
};

class EngineBase {
 public:
  virtual ~EngineBase() {}
  // upload the host hierarchy (and element mass blocks) and capture graphs
  virtual int init(const HostHierarchy& h, const Mesh& m, int precision, int fine_operator, int coarse_persistent,
                   int coarse_cluster, cudaStream_t s,
                   std::string& err) = 0;
  virtual int pcg_solve(const double* b_user, double* x_user, const SolveOpts& o, SolveResult& res,
                        cudaStream_t s, std::string& err) = 0;
  virtual int apply_level(int level, const double* x_user, double* y_user, cudaStream_t s, std::string& err) = 0;
  virtual int vcycle_apply(const double* r_user, double* z_user, cudaStream_t s, std::string& err) = 0;
  // time stepping: one simulation per engine at a time
  virtual int sim_create(const SimParams& p, const double* mask_user, cudaStream_t s, std::string& err) = 0;
  virtual int sim_step(int n_steps, double* u_user, double* w_user, int* iters_host, int64_t& clock,
                       cudaStream_t s, std::string& err) = 0;
  virtual int sim_destroy() = 0;
  virtual void sim_invalidate_history() = 0;
  // one reverse time step (discrete adjoint), vectors in the caller's order
  virtual int adjoint_step(const double* u_n, const double* w_n, const double* u_np1, double* ubar, double* wbar,
                           double* grad, SolveResult& res, cudaStream_t s, std::string& err) = 0;
  virtual bool uses_conditional_graph() const = 0;
  // instrumentation: launch one hot kernel `reps` times on the internal
  // buffers, and its algorithmic bytes / flops per launch
  virtual int kernel_loop(int id, int reps, cudaStream_t s, std::string& err) = 0;
  virtual int kernel_cost(int id, double& bytes, double& flops) const = 0;
  // kernel launches of one V-cycle, one solve-body iteration and one solve
  // set-up; whether the coarse levels run in the persistent kernel
  virtual void launch_counts(int& per_vcycle, int& per_iteration, int& per_setup, int& persistent,
                             int& cluster_level, int& cluster_ctas) const = 0;
  // y = A_l x with the permuted copies of x and y in caller-provided device
  // scratch (s_in, s_out: at least level_scratch_entries(l) doubles each)
  virtual int64_t level_scratch_entries(int level) const = 0;
  virtual int apply_level_scratch(int level, const double* x_user, double* y_user, void* s_in, void* s_out,
                                  cudaStream_t s, std::string& err) = 0;
};

EngineBase* make_engine(int B, int precision);
// records the calling thread's last error message (read by agg_last_error)
void set_last_error(const std::string& msg);

}  // namespace aggmg
