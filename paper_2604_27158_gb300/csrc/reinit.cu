// Re-initialisation of the LBM populations from macroscopic fields (Sec. 2.3 of
// arXiv 2604.27158): f = f^eq(rho, u), optionally plus the Chapman-Enskog
// non-equilibrium part f^neq_i = -(w_i tau rho / c_s^2) Q_iab d_a u_b, laid out for the
// pull step of lbm.cu.  Compiled with the default FMA contraction (the step kernels'
// file is not): the values agree with the per-cell definition to FP32 rounding.
//
// Layout.  The state holds post-collision populations, shifted by the weights, so the
// re-initialised values go where the next pull reads them: the pull of population j at
// a fluid cell n reads plane j at n - c_j when that cell is fluid, else (halfway
// bounce-back) plane opp(j) at n itself.  So plane j at a fluid location p holds
// g_j(p + c_j) when p + c_j is a fluid cell, g_opp(j)(p) when it is a solid cell, and 0
// when it lies outside a non-periodic grid (an open-boundary unknown, completed by the
// next pull); solid locations hold 0.  None of the zeros is ever read by a pull.
//
// Kernel.  One CTA per tile of kReinitRows rows x 128 columns.
//  0. rho, u and the cell kinds of the tile and a two-cell halo are staged in shared
//     memory, every load of a thread issued before the first is used.
//  1. The populations of the tile and a one-cell halo are evaluated (derivatives central
//     where both neighbours along an axis are fluid cells of the grid, one-sided where
//     one is, zero otherwise; y periodic, x periodic for periodic grids) and written
//     *pre-shifted*: g_j(n) of a fluid cell n into the slot of plane j at n - c_j; a
//     fluid cell p of the tile whose neighbour p + c_j is solid or outside puts
//     g_opp(j)(p) or 0 into its own slot of plane j (that slot's other writer would be
//     the non-fluid cell, which writes nothing).
//  2. Every plane of the tile is copied out as aligned 16-byte chunks, masked to 0 at
//     solid cells.
#include "common.cuh"
#include "lbm_cell.cuh"
#include "lbm_internal.cuh"

namespace lbmfno {

namespace {

enum : unsigned char { kRiFluid = 0, kRiSolid = 1, kRiOutside = 2 };
constexpr int kTR = kReinitRows;
constexpr int kRiThreads = 256;  // threads a CTA (a tile's rows, columns and planes are shared out)
constexpr int kSW = 132;      // staged row: columns x0 - 2 .. x0 + 129 (sx = 0 .. 131)
constexpr int kOW = 136;      // slot row: hx = 0 .. 129 at hx + 3, so that hx = 1 (the
                              // tile's first column) is 16-byte aligned; 133 .. 135 unread
constexpr int kOOff = 3;
constexpr int kKOff = 2;      // kind row: sx at sx + 2, so that sx = 2 is 4-byte aligned
constexpr int kDummy = kOW - 1;
struct Smem {
  float out[kQ][kTR + 2][kOW];                  // pre-shifted planes of the tile and halo
  float fs[3][kTR + 4][kSW];                    // rho, u_x, u_y of the tile and two halo cells
  __align__(4) unsigned char ks[kTR + 4][kOW];  // cell kinds of the same cells
};
static_assert(sizeof(Smem) <= 57 * 1024, "four CTAs a multiprocessor");

__device__ __forceinline__ unsigned char& kind_at(Smem& S, int sy, int sx) {
  return S.ks[sy][sx + kKOff];
}
__device__ __forceinline__ unsigned char kind_of(const Smem& S, int sy, int sx) {
  return S.ks[sy][sx + kKOff];
}

// One-axis difference: central, one-sided or zero as dfield, without branches (the values
// of cells that are not selected may be anything).
__device__ __forceinline__ float dsel(bool okp, bool okm, float vp, float vc, float vm) {
  const float central = 0.5f * (vp - vm), fwd = vp - vc, bwd = vc - vm;
  return okp ? (okm ? central : fwd) : (okm ? bwd : 0.0f);
}

// Populations of staged cell (hy, hx) (hy = 0 .. rows + 1, hx = 0 .. 129; the tile's
// cells are hy = 1 .. rows, hx = 1 .. 128).  Evaluated branch-free for every cell; a
// store that must not happen goes to the unread column kDummy of its row instead.
// Opposite directions share the even part of f^eq + f^neq (c_a c_b is even in c).
template <bool kOwn>
__device__ __forceinline__ void eval_cell(Smem& S, int hy, int hx, int rows, int neq_mode,
                                          float kneq_tau) {
  const int sy = hy + 1, sx = hx + 1;
  unsigned char kn[kQ];  // kind of the neighbour n + c_i (kn[0]: the cell itself)
#pragma unroll
  for (int i = 0; i < kQ; ++i) kn[i] = kind_of(S, sy + cy_of(i), sx + cx_of(i));
  const bool fluid = kn[0] == kRiFluid;
  const float rho = S.fs[0][sy][sx], ux = S.fs[1][sy][sx], uy = S.fs[2][sy][sx];
  float dxux = 0.f, dxuy = 0.f, dyux = 0.f, dyuy = 0.f;
  if (neq_mode) {
    const bool xp = kn[1] == kRiFluid, xm = kn[3] == kRiFluid;
    const bool yp = kn[2] == kRiFluid, ym = kn[4] == kRiFluid;
    dxux = dsel(xp, xm, S.fs[1][sy][sx + 1], ux, S.fs[1][sy][sx - 1]);
    dxuy = dsel(xp, xm, S.fs[2][sy][sx + 1], uy, S.fs[2][sy][sx - 1]);
    dyux = dsel(yp, ym, S.fs[1][sy + 1][sx], ux, S.fs[1][sy - 1][sx]);
    dyuy = dsel(yp, ym, S.fs[2][sy + 1][sx], uy, S.fs[2][sy - 1][sx]);
  }
  const float drho = rho - 1.0f;
  const float usq = 1.5f * (ux * ux + uy * uy);
  const float div3 = (1.0f / 3.0f) * (dxux + dyuy);
  const float kneq = kneq_tau * rho;  // -(tau rho / c_s^2)
  const float shear = dxuy + dyux;
  float g[kQ];
  // Q_iab d_a u_b = c_ia c_ib d_a u_b - c_s^2 div u, per direction pair
  g[0] = kW0 * (drho - rho * usq - kneq * div3);
  auto pair = [&](int i, float w, float cu, float qd) {
    const float even = w * (drho + rho * (4.5f * cu * cu - usq) + kneq * qd);
    const float odd = (3.0f * w) * (rho * cu);
    g[i] = even + odd;
    g[opp_of(i)] = even - odd;
  };
  pair(1, kW1, ux, dxux - div3);                        // c = (1, 0)
  pair(2, kW1, uy, dyuy - div3);                        // c = (0, 1)
  pair(5, kW2, ux + uy, (dxux + dyuy) + shear - div3);  // c = (1, 1)
  pair(6, kW2, uy - ux, (dxux + dyuy) - shear - div3);  // c = (-1, 1)
  // g_j(n) into the slot of plane j at n - c_j (inside the slot array)
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    const int ty = hy - cy_of(j), tx = hx - cx_of(j);
    bool ok = fluid;
    if (!kOwn) ok = ok && ty >= 0 && ty <= rows + 1 && tx >= 0 && tx <= 129;
    S.out[j][ok ? ty : hy][ok ? tx + kOOff : kDummy] = g[j];
  }
  if (kOwn) {  // bounce-back (solid n + c_j) or open-boundary (outside) value of plane j
#pragma unroll
    for (int j = 1; j < kQ; ++j) {
      const bool b = fluid && kn[j] != kRiFluid;
      S.out[j][hy][b ? hx + kOOff : kDummy] = kn[j] == kRiSolid ? g[opp_of(j)] : 0.0f;
    }
  }
}

__global__ void __launch_bounds__(kRiThreads, 1024 / kRiThreads) k_reinit(const GridDev* __restrict__ grids,
                                                   const int4* __restrict__ tiles,
                                                   const uint32_t* __restrict__ mask,
                                                   const float* __restrict__ rho_i,
                                                   const float* __restrict__ ux_i,
                                                   const float* __restrict__ uy_i, int neq_mode,
                                                   float* __restrict__ state,
                                                   float* __restrict__ ux_prev,
                                                   float* __restrict__ uy_prev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const int4 tile = __ldg(&tiles[blockIdx.x]);  // (grid, x0, y0, rows)
  const GridDev G = grids[tile.x];              // registers: stores below cannot alias it
  const int x0 = tile.y, y0 = tile.z, rows = tile.w;
  const uint32_t* m = mask + G.mask_off;
  const float* F[3] = {rho_i + G.cell_off, ux_i + G.cell_off, uy_i + G.cell_off};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // 0. stage rows y0 - 2 .. y0 + rows + 1 (wrapped in y) and columns x0 - 2 .. x0 + 129
  //    (wrapped in x for periodic grids, outside otherwise): a warp a row
  constexpr int kSlotsY = (kTR + 4 + kRiThreads / 32 - 1) / (kRiThreads / 32);
  constexpr int kSlotsX = (kSW + 31) / 32;
  float fv[kSlotsY][kSlotsX][3];
  uint32_t mw[kSlotsY][kSlotsX];
  int gxs[kSlotsX];
#pragma unroll
  for (int q = 0; q < kSlotsX; ++q) {  // column of slot q, -1 when outside the grid
    int gx = x0 - 2 + lane + 32 * q;
    if (G.periodic_x && (gx < 0 || gx >= G.nx)) gx = (gx % G.nx + G.nx) % G.nx;
    gxs[q] = (gx >= 0 && gx < G.nx && lane + 32 * q < kSW) ? gx : -1;
  }
#pragma unroll
  for (int r = 0; r < kSlotsY; ++r) {
    const int sy = warp + r * (kRiThreads / 32);
    int gy = y0 - 2 + sy;
    if (gy < 0 || gy >= G.ny) gy = (gy % G.ny + G.ny) % G.ny;
    const uint32_t* mrow = m + (long long)gy * G.wpr;
    const long long crow = (long long)gy * G.nx;
#pragma unroll
    for (int q = 0; q < kSlotsX; ++q) {
      if (sy < rows + 4 && gxs[q] >= 0) {
        mw[r][q] = __ldg(&mrow[gxs[q] >> 5]);
#pragma unroll
        for (int f = 0; f < 3; ++f) fv[r][q][f] = __ldg(&F[f][crow + gxs[q]]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kSlotsY; ++r) {
    const int sy = warp + r * (kRiThreads / 32);
#pragma unroll
    for (int q = 0; q < kSlotsX; ++q) {
      const int sx = lane + 32 * q;
      if (sy < rows + 4 && sx < kSW) {
        unsigned char k = kRiOutside;
        if (gxs[q] >= 0) {
          k = (mw[r][q] >> (gxs[q] & 31)) & 1u ? kRiSolid : kRiFluid;
#pragma unroll
          for (int f = 0; f < 3; ++f) S.fs[f][sy][sx] = fv[r][q][f];
        }
        kind_at(S, sy, sx) = k;
      }
    }
  }
  __syncthreads();
  // 1. columns x0 .. x0 + 127 of rows y0 - 1 .. y0 + rows (cell e: row e / 128, so whether
  //    a warp's cells belong to the tile is warp-uniform) and the halo columns x0 - 1,
  //    x0 + 128; the tile's cells also store the current velocity (0 at solid cells) for
  //    the next steady-state check
  const float kneq_tau = -3.0f * G.tau;
  for (int e = threadIdx.x; e < (rows + 2) * 128; e += kRiThreads) {
    const int hy = e >> 7, hx = 1 + (e & 127);
    if (hy >= 1 && hy <= rows) {
      const int gx = x0 + hx - 1;
      if (gx < G.nx) {
        const bool fluid = kind_of(S, hy + 1, hx + 1) == kRiFluid;
        const long long at = G.f_off + (long long)(y0 + hy - 1) * G.pitch + gx;
        ux_prev[at] = fluid ? S.fs[1][hy + 1][hx + 1] : 0.0f;
        uy_prev[at] = fluid ? S.fs[2][hy + 1][hx + 1] : 0.0f;
      }
      eval_cell<true>(S, hy, hx, rows, neq_mode, kneq_tau);
    } else {
      eval_cell<false>(S, hy, hx, rows, neq_mode, kneq_tau);
    }
  }
  if (warp == kRiThreads / 32 - 1 && lane < 2 * (rows + 2))  // halo columns x0 - 1, x0 + 128
    eval_cell<false>(S, lane >> 1, (lane & 1) ? 129 : 0, rows, neq_mode, kneq_tau);
  __syncthreads();
  // 2. a thread a (row, 4 columns), all nine planes: aligned 16-byte chunks, 0 at solid
  //    cells (four cell kinds in one 4-byte load)
  const int ncols = min(128, G.nx - x0);
  for (int u = threadIdx.x; u < rows * 32; u += kRiThreads) {
    const int r = u >> 5, c0 = (u & 31) * 4;
    if (c0 >= ncols) continue;
    const uint32_t k4 = *reinterpret_cast<const uint32_t*>(&S.ks[r + 2][c0 + 2 + kKOff]);
    const bool f0 = (k4 & 0xffu) == kRiFluid, f1 = ((k4 >> 8) & 0xffu) == kRiFluid;
    const bool f2 = ((k4 >> 16) & 0xffu) == kRiFluid, f3 = (k4 >> 24) == kRiFluid;
    float* dst = state + G.f_off + (long long)(y0 + r) * G.pitch + x0 + c0;
#pragma unroll
    for (int j = 0; j < kQ; ++j) {
      const float4 v = *reinterpret_cast<const float4*>(&S.out[j][r + 1][c0 + 1 + kOOff]);
      const float4 o = make_float4(f0 ? v.x : 0.0f, f1 ? v.y : 0.0f, f2 ? v.z : 0.0f,
                                   f3 ? v.w : 0.0f);
      float* d = dst + (long long)j * G.plane;
      if (c0 + 4 <= ncols) {
        *reinterpret_cast<float4*>(d) = o;
      } else {
        d[0] = o.x;
        if (c0 + 1 < ncols) d[1] = o.y;
        if (c0 + 2 < ncols) d[2] = o.z;
      }
    }
  }
}


}  // namespace

int reinit_init(Handle*) {
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_reinit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(Smem)));
  return LBM_OK;
}

int reinit_launch(Handle* h, const int4* tiles, int ntiles, const float* rho_d,
                  const float* ux_d, const float* uy_d, int neq_mode, cudaStream_t s) {
  if (ntiles == 0) return LBM_OK;
  k_reinit<<<ntiles, kRiThreads, sizeof(Smem), s>>>(h->gd_d, tiles, h->mask, rho_d, ux_d, uy_d,
                                                neq_mode, h->f[h->cur], h->ux_prev,
                                                h->uy_prev);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

}  // namespace lbmfno
