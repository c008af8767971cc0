// Internal definition of the LBM handle, shared by the LBM and hybrid units.
#pragma once

#include <vector>

#include "common.cuh"

namespace lbmfno {

struct Handle {
  std::vector<lbm_grid> grids;
  std::vector<GridDev> gd;
  GridDev* gd_d = nullptr;  // in the caller's workspace
  int ngrids = 0;
  int nblk_total = 0;
  int nrblk_total = 0;  // blocks of the residual kernel
  int nsm = 0;
  int variant = 0;                             // step-kernel tile shape in use
  int ntiles_v[LBM_STEP_VARIANTS] = {};        // tiles of the batch per shape
  int blocks_per_sm_v[LBM_STEP_VARIANTS] = {};  // resident CTAs per SM per shape
  int4* tiles_d[LBM_STEP_VARIANTS] = {};      // per-shape tile descriptors (workspace)
  unsigned* status_d = nullptr;
  unsigned status_h = 0;
  const uint32_t* mask = nullptr;
  float* f[2] = {nullptr, nullptr};
  int cur = 0;  // buffer holding the current state
  float* ux_prev = nullptr;
  float* uy_prev = nullptr;
  double* partial = nullptr;
  double* stats_d = nullptr;
  std::vector<double> stats_h;
  lbm_layout layout{};
  float u_max2 = 0.04f;
  long long steps = 0;
};

}  // namespace lbmfno

struct lbm_handle : lbmfno::Handle {};
