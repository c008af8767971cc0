// Reverse-mode (adjoint) kernels of the LBM part of the hybrid pipeline and their
// C ABI: the vector-Jacobian products of the moments (Sec. 2.1), of one fused
// time step (pull streaming with halfway bounce-back, Zou-He completion, BGK
// collision with the Guo source, Sec. 2.1), and of the re-initialisation of the
// populations from macroscopic fields (f^eq + Chapman-Enskog f^neq, Sec. 2.3).
//
// Notation.  s_n is the stored state of the library (shifted post-collision
// populations of time level n-1), P the pull that turns it into the populations
// f_n of level n (gather with bounce-back, then Zou-He completion of the unknown
// populations of open end columns), C the per-cell collision, M the moments:
//   lbm_step:  s_{n+1} = C(P(s_n)),   lbm_macro: (rho, u)_n = M(P(s_n)).
// The adjoint variable mu_n is the gradient of the loss with respect to the
// *pulled known* populations of every fluid cell at level n, i.e. to the values
// gathered by P before the Zou-He completion (unknown slots hold 0, solid cells
// hold 0).  Then
//   mu_N     = Z^T (dM/df)^T (drho, du)                 lbm_adjoint_macro
//   mu_{n-1} = Z^T J_C(f_{n-1})^T G^T mu_n               lbm_adjoint_step
//   (drho, du)_0 = R^T mu_0                              lbm_adjoint_reinit
// with Z the Zou-He completion (linear in the known populations), J_C the 9x9
// collision Jacobian of each cell at f_{n-1} = P(s_{n-1}), G the gather of the
// pull (a permutation of the fluid slots with bounce-back), and R the
// re-initialisation followed by the pull, whose known populations are exactly
// f^eq + f^neq of each cell.
//
// Every buffer here is in the canonical state layout of lbm_get_state: per grid,
// 9 planes of ny x nx floats at 9 * cell offset.  All kernels are per-cell and
// read only the cell's own stencil, so there are no atomics and the results are
// deterministic.
#include <math.h>

#include "common.cuh"
#include "lbm_cell.cuh"
#include "lbm_internal.cuh"

namespace lbmfno {

namespace {

inline cudaStream_t AS(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// A copy of the grid descriptor that addresses the canonical layout.
__device__ __forceinline__ GridDev canonical(const GridDev& G) {
  GridDev C = G;
  C.pitch = G.nx;
  C.plane = (long long)G.nx * G.ny;
  C.f_off = 9LL * G.cell_off;
  return C;
}

// Transpose of the Zou-He completion at an open end cell: the gradients of the
// completed unknown populations are distributed onto the known ones they were
// computed from, and the unknown slots are cleared.  rho u_x = a + beta * G0
// with G0 the sum of the known populations (2x those pointing outwards).
__device__ __forceinline__ void zou_he_transpose(const GridDev& G, bool west, bool east,
                                                 float m[kQ]) {
  if (west) {  // unknown 1, 5, 8
    const float beta = (G.bc_west == LBM_BC_PRESSURE) ? -1.0f : G.west_d / (1.0f - G.west_d);
    const float bs = beta * ((2.0f / 3.0f) * m[1] + (1.0f / 6.0f) * (m[5] + m[8]));
    m[0] += bs;
    m[2] += bs - 0.5f * m[5] + 0.5f * m[8];
    m[4] += bs + 0.5f * m[5] - 0.5f * m[8];
    m[3] += m[1] + 2.0f * bs;
    m[7] += m[5] + 2.0f * bs;
    m[6] += m[8] + 2.0f * bs;
    m[1] = m[5] = m[8] = 0.0f;
  }
  if (east) {  // unknown 3, 6, 7
    const float beta = (G.bc_east == LBM_BC_PRESSURE) ? 1.0f : G.east_d / (1.0f + G.east_d);
    const float bs = -beta * ((2.0f / 3.0f) * m[3] + (1.0f / 6.0f) * (m[7] + m[6]));
    m[0] += bs;
    m[2] += bs + 0.5f * m[7] - 0.5f * m[6];
    m[4] += bs - 0.5f * m[7] + 0.5f * m[6];
    m[1] += m[3] + 2.0f * bs;
    m[5] += m[7] + 2.0f * bs;
    m[8] += m[6] + 2.0f * bs;
    m[3] = m[6] = m[7] = 0.0f;
  }
}

// lam <- J_C(f)^T lam for the BGK collision with the Guo source:
//   (J^T l)_j = (1 - om) l_j + om [A + V.(c_j - u)] + Gv.(c_j - u) / rho
//   A   = sum_i l_i f^eq_i / rho
//   V_a = sum_i l_i w_i (3 c_ia + 9 (c_i.u) c_ia - 3 u_a)
//   Gv_b = (1 - om/2) sum_i l_i w_i (-3 F_b + 9 c_ib (c_i.F))
__device__ __forceinline__ void collision_transpose(const GridDev& G, const float f[kQ],
                                                    float l[kQ]) {
  float drho, rho, ux, uy;
  moments(G, f, drho, rho, ux, uy);
  const float usq = 1.5f * (ux * ux + uy * uy);
  const float om = G.omega;
  float A = 0.f, Vx = 0.f, Vy = 0.f, Gx = 0.f, Gy = 0.f;
  const bool forced = (G.fx != 0.0f || G.fy != 0.0f);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float cx = (float)cx_of(i), cy = (float)cy_of(i);
    const float cu = cx * ux + cy * uy;
    const float wl = w_of(i) * l[i];
    A += wl * (1.0f + 3.0f * cu + 4.5f * cu * cu - usq);
    const float t = 3.0f + 9.0f * cu;
    Vx += wl * (t * cx - 3.0f * ux);
    Vy += wl * (t * cy - 3.0f * uy);
    if (forced) {
      const float cf = 9.0f * (cx * G.fx + cy * G.fy);
      Gx += wl * (cf * cx - 3.0f * G.fx);
      Gy += wl * (cf * cy - 3.0f * G.fy);
    }
  }
  const float ginv = G.guo / rho;  // guo = 1 - om / 2
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    const float dx = (float)cx_of(j) - ux, dy = (float)cy_of(j) - uy;
    l[j] = (1.0f - om) * l[j] + om * (A + Vx * dx + Vy * dy) + ginv * (Gx * dx + Gy * dy);
  }
}

__device__ __forceinline__ void store9(const GridDev& Gc, float* buf, int x, int y,
                                       const float v[kQ]) {
  float* o = buf + Gc.f_off + (long long)y * Gc.pitch + x;
#pragma unroll
  for (int i = 0; i < kQ; ++i) o[i * Gc.plane] = v[i];
}

__global__ void __launch_bounds__(kBlock) k_adj_macro(const GridDev* __restrict__ grids,
                                                      int ngrids, const uint32_t* __restrict__ mask,
                                                      const float* __restrict__ state,
                                                      const float* __restrict__ drho_i,
                                                      const float* __restrict__ dux_i,
                                                      const float* __restrict__ duy_i,
                                                      float* __restrict__ mu) {
  int gidx, x, y;
  if (!cell_of_thread(grids, ngrids, gidx, x, y)) return;
  const GridDev Gc = canonical(grids[gidx]);
  float f[kQ], m[kQ];
  if (!pull_cell(Gc, mask, state, x, y, f)) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) m[i] = 0.0f;
    store9(Gc, mu, x, y, m);
    return;
  }
  float drho, rho, ux, uy;
  moments(Gc, f, drho, rho, ux, uy);
  const long long c = Gc.cell_off + (long long)y * Gc.nx + x;
  const float dr = drho_i[c], inv = 1.0f / rho;
  const float ax = dux_i[c] * inv, ay = duy_i[c] * inv;
#pragma unroll
  for (int j = 0; j < kQ; ++j)
    m[j] = dr + ax * ((float)cx_of(j) - ux) + ay * ((float)cy_of(j) - uy);
  zou_he_transpose(Gc, !Gc.periodic_x && x == 0, !Gc.periodic_x && x == Gc.nx - 1, m);
  store9(Gc, mu, x, y, m);
}

__global__ void __launch_bounds__(kBlock) k_adj_step(const GridDev* __restrict__ grids,
                                                     int ngrids, const uint32_t* __restrict__ mask,
                                                     const float* __restrict__ state_prev,
                                                     const float* __restrict__ mu_in,
                                                     float* __restrict__ mu_out) {
  int gidx, x, y;
  if (!cell_of_thread(grids, ngrids, gidx, x, y)) return;
  const GridDev Gc = canonical(grids[gidx]);
  float f[kQ], l[kQ];
  if (!pull_cell(Gc, mask, state_prev, x, y, f)) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) l[i] = 0.0f;
    store9(Gc, mu_out, x, y, l);
    return;
  }
  // G^T: slot (j, x) of the stored state was read by cell x + c_j as its population j
  // when that cell is a fluid cell of the domain, by this cell's population opp(j)
  // (bounce-back) when it is solid, and by nobody when it lies beyond an open end.
  const uint32_t* m = mask + Gc.mask_off;
  const float* b = mu_in + Gc.f_off;
  const long long P = Gc.plane;
  const long long here = (long long)y * Gc.pitch + x;
  const int yp = (y == Gc.ny - 1) ? 0 : y + 1;
  const int ym = (y == 0) ? Gc.ny - 1 : y - 1;
  l[0] = b[here];
#pragma unroll
  for (int j = 1; j < kQ; ++j) {
    int tx = x + cx_of(j);
    const int ty = cy_of(j) == 0 ? y : (cy_of(j) > 0 ? yp : ym);
    if (tx < 0 || tx >= Gc.nx) {
      if (!Gc.periodic_x) {
        l[j] = 0.0f;
        continue;
      }
      tx = tx < 0 ? Gc.nx - 1 : 0;
    }
    if (mask_bit(m, Gc.wpr, tx, ty))
      l[j] = b[(long long)opp_of(j) * P + here];
    else
      l[j] = b[(long long)j * P + (long long)ty * Gc.pitch + tx];
  }
  collision_transpose(Gc, f, l);
  zou_he_transpose(Gc, !Gc.periodic_x && x == 0, !Gc.periodic_x && x == Gc.nx - 1, l);
  store9(Gc, mu_out, x, y, l);
}

// R^T, local part: per fluid cell the gradient with respect to rho and u of the
// cell's own f^eq + f^neq, and the gradients with respect to the four velocity
// derivatives (d_x u_x, d_y u_y, and the shared coefficient of d_x u_y and d_y u_x)
// that the stencil kernel below distributes to the neighbours.
__global__ void __launch_bounds__(kBlock) k_adj_reinit_local(
    const GridDev* __restrict__ grids, int ngrids, const uint32_t* __restrict__ mask,
    const float* __restrict__ mu, const float* __restrict__ rho_i,
    const float* __restrict__ ux_i, const float* __restrict__ uy_i, int neq_mode,
    float* __restrict__ drho_o, float* __restrict__ dux_o, float* __restrict__ duy_o,
    float* __restrict__ dgrad) {
  int gidx, x, y;
  if (!cell_of_thread(grids, ngrids, gidx, x, y)) return;
  const GridDev G = grids[gidx];
  const GridDev Gc = canonical(G);
  const long long cells = (long long)G.nx * G.ny;
  const long long c = G.cell_off + (long long)y * G.nx + x;
  const uint32_t* m = mask + G.mask_off;
  float* dg = dgrad + 3LL * G.cell_off + (long long)y * G.nx + x;
  if (mask_bit(m, G.wpr, x, y)) {
    drho_o[c] = dux_o[c] = duy_o[c] = 0.0f;
    dg[0] = dg[cells] = dg[2 * cells] = 0.0f;
    return;
  }
  float l[kQ];
  const float* b = mu + Gc.f_off + (long long)y * Gc.pitch + x;
#pragma unroll
  for (int i = 0; i < kQ; ++i) l[i] = b[i * Gc.plane];
  // unknown populations of open end cells are not taken from the reinit
  if (!G.periodic_x && x == 0) l[1] = l[5] = l[8] = 0.0f;
  if (!G.periodic_x && x == G.nx - 1) l[3] = l[6] = l[7] = 0.0f;
  const float rho = rho_i[c], ux = ux_i[c], uy = uy_i[c];
  float dxux = 0.f, dxuy = 0.f, dyux = 0.f, dyuy = 0.f;
  if (neq_mode) {
    const float* UX = ux_i + G.cell_off;
    const float* UY = uy_i + G.cell_off;
    dxux = dfield(G, m, UX, x, y, 0);
    dxuy = dfield(G, m, UY, x, y, 0);
    dyux = dfield(G, m, UX, x, y, 1);
    dyuy = dfield(G, m, UY, x, y, 1);
  }
  const float usq = 1.5f * (ux * ux + uy * uy);
  const float div = dxux + dyuy;
  const float k3 = -3.0f * G.tau;
  float gr = 0.f, gx = 0.f, gy = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float cx = (float)cx_of(i), cy = (float)cy_of(i);
    const float cu = cx * ux + cy * uy;
    const float wl = w_of(i) * l[i];
    const float qd = cx * cx * dxux + cx * cy * (dxuy + dyux) + cy * cy * dyuy - div / 3.0f;
    gr += wl * (1.0f + 3.0f * cu + 4.5f * cu * cu - usq + k3 * qd);
    const float t = 3.0f + 9.0f * cu;
    gx += wl * (t * cx - 3.0f * ux);
    gy += wl * (t * cy - 3.0f * uy);
    sxx += wl * (cx * cx - 1.0f / 3.0f);
    syy += wl * (cy * cy - 1.0f / 3.0f);
    sxy += wl * (cx * cy);
  }
  drho_o[c] = gr;
  dux_o[c] = rho * gx;
  duy_o[c] = rho * gy;
  const float kr = k3 * rho;
  dg[0] = kr * sxx;          // d loss / d (d_x u_x)
  dg[cells] = kr * syy;      // d loss / d (d_y u_y)
  dg[2 * cells] = kr * sxy;  // d loss / d (d_x u_y) = d loss / d (d_y u_x)
}

// Stencil of the derivative of a field at fluid cell (x, y) along `axis`: flags for
// the + and - neighbours (fluid cells of the domain), mirroring dfield.
__device__ __forceinline__ void stencil_flags(const GridDev& G, const uint32_t* m, int x, int y,
                                              int axis, bool& okp, bool& okm) {
  int xp = x, xm = x, yp = y, ym = y;
  okp = okm = true;
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
}

// Transpose of the derivative stencil along `axis` applied to the field D (the
// gradient with respect to that derivative), gathered at fluid cell (x, y).
__device__ __forceinline__ float stencil_transpose(const GridDev& G, const uint32_t* m,
                                                   const float* D, int x, int y, int axis) {
  float acc = 0.0f;
  bool okp, okm;
  stencil_flags(G, m, x, y, axis, okp, okm);  // the cell's own derivative
  if (okp != okm) acc += (okp ? -1.0f : 1.0f) * D[(long long)y * G.nx + x];
  // the - neighbour uses this cell as its + neighbour, the + neighbour as its -
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    int nx_ = x, ny_ = y;
    if (axis == 0) {
      nx_ = side == 0 ? x - 1 : x + 1;
      if (nx_ < 0 || nx_ >= G.nx) {
        if (!G.periodic_x) continue;
        nx_ = nx_ < 0 ? G.nx - 1 : 0;
      }
    } else {
      ny_ = side == 0 ? (y == 0 ? G.ny - 1 : y - 1) : (y == G.ny - 1 ? 0 : y + 1);
    }
    if (mask_bit(m, G.wpr, nx_, ny_)) continue;
    bool np, nm;
    stencil_flags(G, m, nx_, ny_, axis, np, nm);
    const float d = D[(long long)ny_ * G.nx + nx_];
    if (side == 0)  // this cell is the + neighbour of (nx_, ny_): np is true
      acc += (nm ? 0.5f : 1.0f) * d;
    else  // this cell is the - neighbour of (nx_, ny_): nm is true
      acc -= (np ? 0.5f : 1.0f) * d;
  }
  return acc;
}

__global__ void __launch_bounds__(kBlock) k_adj_reinit_stencil(
    const GridDev* __restrict__ grids, int ngrids, const uint32_t* __restrict__ mask,
    const float* __restrict__ dgrad, float* __restrict__ dux_o, float* __restrict__ duy_o) {
  int gidx, x, y;
  if (!cell_of_thread(grids, ngrids, gidx, x, y)) return;
  const GridDev G = grids[gidx];
  const uint32_t* m = mask + G.mask_off;
  if (mask_bit(m, G.wpr, x, y)) return;
  const long long cells = (long long)G.nx * G.ny;
  const float* Dxx = dgrad + 3LL * G.cell_off;
  const float* Dyy = Dxx + cells;
  const float* Dxy = Dxx + 2 * cells;
  const long long c = G.cell_off + (long long)y * G.nx + x;
  // u_x enters d_x u_x (axis 0) and d_y u_x (axis 1); u_y enters d_x u_y and d_y u_y
  dux_o[c] += stencil_transpose(G, m, Dxx, x, y, 0) + stencil_transpose(G, m, Dxy, x, y, 1);
  duy_o[c] += stencil_transpose(G, m, Dxy, x, y, 0) + stencil_transpose(G, m, Dyy, x, y, 1);
}

}  // namespace

}  // namespace lbmfno

using namespace lbmfno;

extern "C" {

int lbm_adjoint_macro(lbm_handle* h, const float* gstar_d, const float* drho_d,
                      const float* dux_d, const float* duy_d, float* mu_d, void* stream) {
  LBM_REQUIRE(h != nullptr && gstar_d != nullptr && drho_d != nullptr && dux_d != nullptr &&
                  duy_d != nullptr && mu_d != nullptr,
              "lbm_adjoint_macro: null argument");
  k_adj_macro<<<h->nblk_total, kBlock, 0, AS(stream)>>>(h->gd_d, h->ngrids, h->mask, gstar_d,
                                                        drho_d, dux_d, duy_d, mu_d);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int lbm_adjoint_step(lbm_handle* h, const float* gstar_prev_d, const float* mu_d,
                     float* mu_prev_d, void* stream) {
  LBM_REQUIRE(h != nullptr && gstar_prev_d != nullptr && mu_d != nullptr && mu_prev_d != nullptr,
              "lbm_adjoint_step: null argument");
  LBM_REQUIRE(mu_d != mu_prev_d, "lbm_adjoint_step: mu and mu_prev must not alias");
  k_adj_step<<<h->nblk_total, kBlock, 0, AS(stream)>>>(h->gd_d, h->ngrids, h->mask,
                                                       gstar_prev_d, mu_d, mu_prev_d);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int lbm_adjoint_reinit(lbm_handle* h, const float* mu_d, const float* rho_d, const float* ux_d,
                       const float* uy_d, int neq_mode, float* scratch_d, float* drho_d,
                       float* dux_d, float* duy_d, void* stream) {
  LBM_REQUIRE(h != nullptr && mu_d != nullptr && rho_d != nullptr && ux_d != nullptr &&
                  uy_d != nullptr && scratch_d != nullptr && drho_d != nullptr &&
                  dux_d != nullptr && duy_d != nullptr,
              "lbm_adjoint_reinit: null argument");
  k_adj_reinit_local<<<h->nblk_total, kBlock, 0, AS(stream)>>>(
      h->gd_d, h->ngrids, h->mask, mu_d, rho_d, ux_d, uy_d, neq_mode, drho_d, dux_d, duy_d,
      scratch_d);
  LBM_CHECK_LAUNCH();
  if (neq_mode) {
    k_adj_reinit_stencil<<<h->nblk_total, kBlock, 0, AS(stream)>>>(h->gd_d, h->ngrids,
                                                                   h->mask, scratch_d, dux_d,
                                                                   duy_d);
    LBM_CHECK_LAUNCH();
  }
  return LBM_OK;
}

}  // extern "C"
