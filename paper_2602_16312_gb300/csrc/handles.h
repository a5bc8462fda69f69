// Definitions of the C ABI's opaque handles, shared by the C ABI files.
#pragma once
#include <cstdint>
#include <vector>

#include "engine.h"
#include "setup.h"

struct agg_mesh {
  aggmg::Mesh m;
};

struct agg_hier {
  agg_mesh* mesh = nullptr;
  int device = 0;
  int L = 0, B = 0, precision = 0;
  double mass_coeff = 0;
  std::vector<int64_t> units, nnzb, perm0;
  std::vector<double> lam_max;
  aggmg::EngineBase* eng = nullptr;
  bool sim_active = false;
  // conductivity parameters on the device (uploaded by the first
  // agg_theta_gradient): elements grouped by parameter (CSR) and theta
  int32_t* d_tptr = nullptr;
  int32_t* d_tmem = nullptr;
  double* d_theta = nullptr;
};
