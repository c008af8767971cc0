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
  int nrblk_total = 0;  // blocks of the statistics reduction
  int nsm = 0;
  int variant = 0;                             // step-kernel tile shape in use
  int ntiles_v[LBM_STEP_VARIANTS] = {};        // tiles of the batch per shape
  int blocks_per_sm_v[LBM_STEP_VARIANTS] = {};  // resident CTAs per SM per shape
  int blocks_per_sm_vm[LBM_STEP_VARIANTS][5] = {};  // ... per shape and kernel mode
  bool persistent = false;     // lbm_step runs nsteps > 1 in one multi-step launch
  unsigned* bar_count = nullptr;  // grid-barrier counter of the multi-step launch
  int4* tiles_d[LBM_STEP_VARIANTS] = {};      // per-shape tile descriptors (workspace)
  unsigned* status_d = nullptr;
  unsigned status_h = 0;
  const uint32_t* mask = nullptr;
  float* f[2] = {nullptr, nullptr};
  int cur = 0;  // buffer holding the current state
  float* ux_prev = nullptr;
  float* uy_prev = nullptr;
  char* scratch = nullptr;  // statistics scratch in the workspace: FP32 row-segment
                            // partials, FP64 block sums, FP64 per-grid sums
  std::vector<double> stats_h;
  lbm_layout layout{};
  float u_max2 = 0.04f;
  long long steps = 0;
};

// Statistics of the current time level (what lbm_residual returns) computed by the
// step kernel while it writes the next time level into the other buffer.  The handle's
// current buffer is NOT switched: the caller either keeps the state (nothing to do) or
// accepts the step with accept_step().  Synchronises `s`.
int residual_step(Handle* h, double* out_h, int update_prev, cudaStream_t s);

// f = f^eq(rho, u) (+ f^neq) of every grid into the current buffer (reinit.cu), one CTA
// a tile of the step-kernel tile table with kReinitRows rows a tile.
constexpr int kReinitRows = 6;
int reinit_init(Handle* h);  // sets the kernel's shared-memory limit (once per handle)
int reinit_launch(Handle* h, const int4* tiles, int ntiles, const float* rho_d,
                  const float* ux_d, const float* uy_d, int neq_mode, cudaStream_t s);
inline void accept_step(Handle* h) {
  h->cur ^= 1;
  h->steps += 1;
}

}  // namespace lbmfno

struct lbm_handle : lbmfno::Handle {};
