// Per-cell device helpers of the D2Q9 kernels, shared by the forward kernels
// (lbm.cu) and the adjoint kernels (lbm_adjoint.cu): the pull of one cell with
// halfway bounce-back and Zou-He completion, the moments of shifted populations,
// the BGK collision with the Guo source (Sec. 2.1), and the cell owned by a thread
// of the per-cell launch decomposition.
#pragma once

#include "common.cuh"

namespace lbmfno {

// ------------------------------------------------------------ cell pull ---
// Gather the post-stream shifted populations of fluid cell (x, y) from the
// post-collision state `src` (streaming with halfway bounce-back), then apply
// the Zou-He completion on open end columns.  Returns false for solid cells.
__device__ __forceinline__ bool pull_cell(const GridDev& G, const uint32_t* __restrict__ mask,
                                          const float* __restrict__ src, int x, int y,
                                          float g[kQ]) {
  const uint32_t* m = mask + G.mask_off;
  if (mask_bit(m, G.wpr, x, y)) return false;
  const float* b = src + G.f_off;
  const long long P = G.plane;
  const int pitch = G.pitch;
  const int ym = (y == 0) ? G.ny - 1 : y - 1;
  const int yp = (y == G.ny - 1) ? 0 : y + 1;
  int xm = x - 1, xp = x + 1;
  bool xm_out = false, xp_out = false;
  if (xm < 0) {
    if (G.periodic_x) xm = G.nx - 1; else xm_out = true;
  }
  if (xp >= G.nx) {
    if (G.periodic_x) xp = 0; else xp_out = true;
  }
  const long long here = (long long)y * pitch + x;
  g[0] = __ldg(b + here);
#define LBM_PULL(i, XS, YS, OUT)                                              \
  if (OUT) {                                                                  \
    g[i] = 0.0f;                                                              \
  } else if (mask_bit(m, G.wpr, XS, YS)) {                                    \
    g[i] = __ldg(b + (long long)opp_of(i) * P + here);                        \
  } else {                                                                    \
    g[i] = __ldg(b + (long long)(i) * P + (long long)(YS) * pitch + (XS));    \
  }
  LBM_PULL(1, xm, y, xm_out)
  LBM_PULL(2, x, ym, false)
  LBM_PULL(3, xp, y, xp_out)
  LBM_PULL(4, x, yp, false)
  LBM_PULL(5, xm, ym, xm_out)
  LBM_PULL(6, xp, ym, xp_out)
  LBM_PULL(7, xp, yp, xp_out)
  LBM_PULL(8, xm, yp, xm_out)
#undef LBM_PULL
  if (xm_out) {  // west column, unknown i = 1, 5, 8 (Zou-He, shifted form)
    const float G0 = g[0] + g[2] + g[4] + 2.0f * (g[3] + g[6] + g[7]);
    float ru;  // rho * u_x
    if (G.bc_west == LBM_BC_PRESSURE) {
      ru = G.west_d - G0;  // rho_in u_x = (rho_in - 1) - G0
    } else {
      const float U = G.west_d;
      ru = (1.0f + G0) / (1.0f - U) * U;
    }
    const float t = 0.5f * (g[2] - g[4]);
    g[1] = g[3] + (2.0f / 3.0f) * ru;
    g[5] = g[7] - t + (1.0f / 6.0f) * ru;
    g[8] = g[6] + t + (1.0f / 6.0f) * ru;
  }
  if (xp_out) {  // east column, unknown i = 3, 6, 7
    const float G0 = g[0] + g[2] + g[4] + 2.0f * (g[1] + g[5] + g[8]);
    float ru;
    if (G.bc_east == LBM_BC_PRESSURE) {
      ru = G0 - G.east_d;  // rho_out u_x = G0 - (rho_out - 1)
    } else {
      const float U = G.east_d;
      ru = (1.0f + G0) / (1.0f + U) * U;
    }
    const float t = 0.5f * (g[2] - g[4]);
    g[3] = g[1] - (2.0f / 3.0f) * ru;
    g[7] = g[5] + t - (1.0f / 6.0f) * ru;
    g[6] = g[8] - t - (1.0f / 6.0f) * ru;
  }
  return true;
}

// Moments of shifted populations: drho = rho - 1, u with the Guo half-force shift.
__device__ __forceinline__ void moments(const GridDev& G, const float g[kQ], float& drho,
                                        float& rho, float& ux, float& uy) {
  drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  rho = 1.0f + drho;
  const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]) + 0.5f * G.fx;
  const float jy = (g[2] - g[4]) + (g[5] - g[8]) + (g[6] - g[7]) + 0.5f * G.fy;
  const float inv = 1.0f / rho;
  ux = jx * inv;
  uy = jy * inv;
}

// BGK relaxation towards the shifted equilibrium, plus the Guo source.  Opposite
// directions (i, opp(i)) share the even part of f^eq and of the source and differ
// in the sign of the odd part, so the nine updates are written per pair.
__device__ __forceinline__ void collide_pair(float& gi, float& go, float w, float cu, float cf,
                                             float drho, float rho, float usq, float om,
                                             float sym_f, float guo) {
  // shifted equilibrium: w (drho + rho (3 cu + 4.5 cu^2 - 1.5 u^2))
  const float even = w * (drho + rho * (4.5f * cu * cu - usq));
  const float odd = w * rho * 3.0f * cu;
  // Guo source: guo w [3 (c - u).F + 9 (c.u)(c.F)]; even part -3 u.F + 9 cu cF, odd 3 cF
  const float s_even = guo * w * (sym_f + 9.0f * cu * cf);
  const float s_odd = guo * w * 3.0f * cf;
  gi = gi + om * (even + odd - gi) + (s_even + s_odd);
  go = go + om * (even - odd - go) + (s_even - s_odd);
}

// Unforced pair update (no source term).  Every multiply-add that is fused is written as
// fmaf: the LBM kernels are compiled without automatic contraction, so each variant of
// the step kernel rounds identically.
__device__ __forceinline__ void relax_pair(float& gi, float& go, float wr3, float wcu, float cu,
                                           float base, float rho, float om) {
  // even part w (drho + rho (4.5 cu^2 - 1.5 u^2)) = w drho - w rho usq + 4.5 w rho cu^2
  const float even = fmaf(4.5f * wcu * cu, cu, base);
  gi = fmaf(om, fmaf(wr3, cu, even) - gi, gi);    // even + odd, odd = wr3 cu
  go = fmaf(om, fmaf(-wr3, cu, even) - go, go);   // even - odd
}

// One BGK collision of a cell's nine shifted populations (Sec. 2.1), with the Guo
// source when the grid carries a body force.
__device__ __forceinline__ void collide(const GridDev& G, float g[kQ]) {
  if (G.fx != 0.0f || G.fy != 0.0f) {
    float drho, rho, ux, uy;
    moments(G, g, drho, rho, ux, uy);
    const float usq = 1.5f * (ux * ux + uy * uy);
    const float om = G.omega, guo = G.guo, fx = G.fx, fy = G.fy;
    const float sym_f = -3.0f * (ux * fx + uy * fy);
    g[0] = g[0] + om * (kW0 * (drho - rho * usq) - g[0]) + guo * kW0 * sym_f;
    collide_pair(g[1], g[3], kW1, ux, fx, drho, rho, usq, om, sym_f, guo);
    collide_pair(g[2], g[4], kW1, uy, fy, drho, rho, usq, om, sym_f, guo);
    collide_pair(g[5], g[7], kW2, ux + uy, fx + fy, drho, rho, usq, om, sym_f, guo);
    collide_pair(g[6], g[8], kW2, uy - ux, fy - fx, drho, rho, usq, om, sym_f, guo);
    return;
  }
  const float drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  const float rho = 1.0f + drho;
  const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
  const float jy = (g[2] - g[4]) + (g[5] - g[8]) + (g[6] - g[7]);
  const float inv = __frcp_rn(rho);
  const float ux = jx * inv, uy = jy * inv;
  const float om = G.omega;
  const float rusq = rho * 1.5f * fmaf(ux, ux, uy * uy);   // rho * 1.5 u^2
  const float e1 = kW1 * (drho - rusq), e2 = kW2 * (drho - rusq);
  const float r1 = kW1 * rho, r2 = kW2 * rho;
  g[0] = fmaf(om, fmaf(kW0, drho - rusq, -g[0]), g[0]);
  relax_pair(g[1], g[3], 3.0f * r1, r1, ux, e1, rho, om);
  relax_pair(g[2], g[4], 3.0f * r1, r1, uy, e1, rho, om);
  relax_pair(g[5], g[7], 3.0f * r2, r2, ux + uy, e2, rho, om);
  relax_pair(g[6], g[8], 3.0f * r2, r2, uy - ux, e2, rho, om);
}

__device__ __forceinline__ bool cell_of_thread(const GridDev* __restrict__ grids, int ngrids,
                                               int& gi, int& x, int& y) {
  gi = grid_of_block(grids, ngrids, blockIdx.x);
  const GridDev& G = grids[gi];
  const int p = (blockIdx.x - G.blk_start) * kBlock + threadIdx.x;
  y = p / G.pitch;
  x = p - y * G.pitch;
  return y < G.ny && x < G.nx;
}

// Derivative of field v at fluid cell (x, y) along axis 0 (x) or 1 (y): central
// where both neighbours are fluid cells of the domain, one-sided where one is, zero
// where none is (the velocity-gradient estimate of the re-initialisation).
__device__ __forceinline__ float dfield(const GridDev& G, const uint32_t* __restrict__ m,
                                        const float* __restrict__ v, int x, int y, int axis) {
  int xp = x, xm = x, yp = y, ym = y;
  bool okp = true, okm = true;
  if (axis == 0) {
    xp = x + 1;
    xm = x - 1;
    if (G.periodic_x) {
      if (xp >= G.nx) xp = 0;
      if (xm < 0) xm = G.nx - 1;
    } else {
      okp = xp < G.nx;
      okm = xm >= 0;
    }
  } else {
    yp = (y == G.ny - 1) ? 0 : y + 1;
    ym = (y == 0) ? G.ny - 1 : y - 1;
  }
  if (okp && mask_bit(m, G.wpr, xp, yp)) okp = false;
  if (okm && mask_bit(m, G.wpr, xm, ym)) okm = false;
  const float vc = v[(long long)y * G.nx + x];
  if (okp && okm) return 0.5f * (v[(long long)yp * G.nx + xp] - v[(long long)ym * G.nx + xm]);
  if (okp) return v[(long long)yp * G.nx + xp] - vc;
  if (okm) return vc - v[(long long)ym * G.nx + xm];
  return 0.0f;
}

}  // namespace lbmfno
