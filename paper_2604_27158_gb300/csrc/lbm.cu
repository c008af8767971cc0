// D2Q9 BGK lattice Boltzmann kernels for GB300 (sm_103a) and their C ABI.
//
// Method: Sec. 2.1 of arXiv 2604.27158 (equilibrium, SRT collision, streaming,
// moments) with halfway bounce-back on a bit-packed solid mask, Zou-He
// inlet/outlet columns, Guo body force, and the re-initialisation of the
// populations from macroscopic fields used by the hybrid framework (Sec. 2.3).
//
// State and data layout (all FP32, HBM resident, caller-owned):
//   * Two state buffers A/B (ping-pong).  The current buffer holds the
//     *post-collision* populations of the previous time level, shifted by the
//     lattice weights (g*_i = f*_i - w_i), structure of arrays over the whole
//     batch: plane i holds population i of every grid, grid g's rows starting at
//     f_off inside the plane, rows `pitch` floats apart (pitch = nx rounded up to
//     32 so each warp's 32 lanes read one aligned 128-byte line per population).
//     A batch of small grids is thus nine contiguous streams, like one tall grid.
//   * One step is a *pull*: cell x gathers g*_i(x - c_i) (bounce-back
//     g*_opp(i)(x) when x - c_i is solid), completes the Zou-He unknowns on the
//     open end columns, takes moments, relaxes, and stores its own nine g*
//     at aligned addresses of the other buffer.  72 B of HBM traffic per fluid
//     cell and step, plus the 1-bit mask.
//   * Solid cells are never read by the step; it stores 0 into their slots.
#include <math.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "lbm_cell.cuh"
#include "lbm_internal.cuh"
#include "sm100.cuh"

namespace lbmfno {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

// raw per-block reduction slots of the residual kernel
enum {
  R_DU2 = 0,
  R_U2,
  R_RHO_W,
  R_N_W,
  R_RHO_E,
  R_N_E,
  R_DRHO,  // sum of (rho - 1) over fluid cells
  R_MOMX,
  R_MOMY,
  R_BAD,
  R_FLUID,
  R_COUNT
};

// --------------------------------------------------------------- kernels ---
__device__ __forceinline__ float f4get(const float4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Sums of 16 per-lane values over the warp in one butterfly: at the level with lane bit
// b (16, 8, 4, 2) every lane keeps one half of its remaining slots (the upper half if its
// bit b is set) and adds the partner's copy of that half, so each level moves half as
// many values as the one before (8 + 4 + 2 + 1 shuffles, then one more for the last lane
// bit).  On return lanes 2s and 2s + 1 hold the total of slot s in v[0].  Fixed lane and
// slot order: deterministic.
__device__ __forceinline__ float warp_sum16(float v[16], int lane) {
#pragma unroll
  for (int half = 8, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
    const bool up = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = up ? v[i] : v[i + half];
      const float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// ------------------------------------------------------ the fused step ---
// One time step of every grid of the batch in one launch: pull streaming with
// halfway bounce-back, Zou-He completion, moments, BGK collision (Sec. 2.1).
//
// Work decomposition: tiles of kTY rows x 128 cells.  A persistent grid of CTAs
// (several per SM) walks the tiles.  Each CTA has one producer warp and kTY
// consumer warps sharing a kStages-deep ring of shared-memory stages:
//  * the producer issues one cp.async.bulk per (population i, staged row): the
//    row segment x0-4 .. x0+131 of population i's *source* rows y0 + r - c_iy,
//    plus one own row for the six populations with c_iy != 0 (bounce-back reads
//    the own cell's opposite population).  Every population is fetched at its
//    own source rows, so a tile needs no y-halo.  The producer also stages the
//    tile's metadata (the grid descriptor) and the packed mask words of rows
//    y0-1 .. y0+kTY, then arrives on the stage's mbarrier;
//  * consumer warp w owns tile row y0 + w; lane l owns cells x0+4l .. x0+4l+3.
//    The nine pulled values are aligned 16-byte shared loads (the +-1 x-shift is
//    a neighbouring 16-byte chunk), bounce-back takes the own cell's opposite
//    population from the stage, Zou-He completes open ends, and the collision
//    result is stored as float4 rows straight to global memory (solid cells
//    store 0, so every 32-byte sector is written whole).
// DRAM traffic: 36 B read + 36 B written per cell; the 8-float x-halo only costs
// shared-memory bandwidth.  Every mbarrier wait is bounded: on expiry the kernel
// records LBM_ERR_TIMEOUT in `status` and stops.
constexpr int kVec = 4;
constexpr int kSeg = 32 * kVec;
constexpr int kRowF = kSeg + 8;  // floats per staged row segment
constexpr int kWords = kVec + 2;  // mask words per row around a segment
// Staged rows of population i: the TY rows it is pulled from plus, for c_iy != 0,
// the tile's own last (c_iy = +1) or first (c_iy = -1) row, so that bounce-back always
// finds the own cell's opposite population in the stage.  Stage row 0 of population i
// holds source row y0 + stage_first(i).
template <int TY>
__host__ __device__ constexpr int stage_rows(int i) { return TY + (cy_of(i) != 0 ? 1 : 0); }
// first stage row of population i = sum of stage_rows(j) for j < i (closed form:
// the populations with c_jy != 0 are j = 2, 4, 5, 6, 7, 8)
template <int TY>
__host__ __device__ constexpr int stage_row0(int i) {
  return i * TY + (i > 2 ? 1 : 0) + (i > 4 ? 1 : 0) + (i > 5 ? i - 5 : 0);
}
__host__ __device__ constexpr int stage_first(int i) { return cy_of(i) > 0 ? -1 : 0; }

// A tile shape of the step kernel: TY rows per tile (= consumer warps per CTA),
// ST stages in the shared-memory ring, MB CTAs requested per SM.
template <int TY, int ST, int MB>
struct StepShape {
  static constexpr int kStageRows = stage_row0<TY>(kQ);  // 9 TY + 6
  static constexpr int kStageFloats = kStageRows * kRowF;
  // statistics modes: the stage also holds the tile's rows of the previous residual's
  // velocity (u_x rows, then u_y rows, 128 floats each)
  static constexpr int kStageFloatsStats = kStageFloats + 2 * TY * kSeg;
  static constexpr int kMaskWords = (TY + 2) * kWords;  // rows y0-1 .. y0+TY
  struct __align__(16) Meta {
    GridDev g;
    int x0, y0, rows, pad;
    uint32_t mask[kMaskWords];
  };
  static constexpr size_t kSmem =
      (size_t)ST * kStageFloats * sizeof(float) + (size_t)ST * sizeof(Meta);
  static constexpr size_t kSmemStats =
      (size_t)ST * kStageFloatsStats * sizeof(float) + (size_t)ST * sizeof(Meta);
  static_assert(stage_row0<TY>(3) == 3 * TY + 1 && stage_row0<TY>(kQ) == 9 * TY + 6 &&
                    stage_row0<TY>(8) + stage_rows<TY>(8) == stage_row0<TY>(kQ),
                "stage row offsets");
};

// Tiles are described by an int4 per tile and shape, built at lbm_init: (grid, first
// column x0, first row y0, rows covered -- the last tile row of a grid can be short).

// What one launch of the step kernel does with the pulled populations of a cell (the
// gather -- streaming, halfway bounce-back, Zou-He completion -- is the same code in
// every mode):
//  * kModeStep:   BGK collision, store: one time step (Sec. 2.1).
//  * kModeStream: store the pulled populations unchanged (collision replaced by the
//                 identity): the state becomes its streamed populations, so the gather's
//                 index map can be compared bit for bit with the oracle's streaming.
//  * kModeStats:  no collision, no population store: the FP32 statistics of the pulled
//                 time level (velocity residual, |u|^2, end-column densities, mass,
//                 momentum, unstable cells) per 128-cell row segment, and optionally the
//                 velocity stored for the next residual.
//  * kModeStepStats: both kModeStep and kModeStats in one pass.
//  * kModeMulti:  kModeStep for ma.nsteps time steps in one persistent launch: the CTAs
//                 stay resident (cooperative launch) and meet at a grid-wide barrier
//                 between steps; the source and destination buffers swap every step.
enum StepMode { kModeStep = 0, kModeStream = 1, kModeStats = 2, kModeStepStats = 3, kModeMulti = 4 };
// floats per row-segment statistics slot (R_COUNT values, padded)
constexpr int kSegStride = 12;
static_assert(R_COUNT <= kSegStride, "segment statistics slot");

// Extra arguments of the statistics modes (unused by the others).
struct StatsArgs {
  float* ux_prev;      // velocity of the previous residual, pitched like a population plane
  float* uy_prev;      // (read; written if update_prev)
  float* seg_partial;  // kSegStride floats per row segment (slot of GridDev)
  float u_max2;
  int update_prev;
};

// Extra arguments of the persistent multi-step mode (unused by the others).
struct MultiArgs {
  int nsteps;                   // time steps of this launch
  unsigned* bar_count;          // grid-barrier arrivals, 0 at launch
  unsigned expected_ctas;       // CTAs arriving at every barrier (gridDim.x)
  unsigned long long limit_ns;  // bound of one barrier wait
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// All threads of the CTA, whatever code path they are on (named barrier 1).
__device__ __forceinline__ void cta_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(blockDim.x) : "memory");
}
// Grid-wide barrier between two steps of the multi-step mode, called by every thread.
// Stores of the step are made visible to the bulk copies (async proxy) and device-wide
// before the CTA's arrival (a release add); thread 0 spins on an acquire load (checking
// the limit every 64 polls) until every CTA has arrived.  An expired wait, here or earlier in any CTA, sets kStatusTimeout and the
// function returns false in every thread of the CTA.
__device__ __forceinline__ bool grid_barrier(const MultiArgs& ma, int sstep, unsigned* status,
                                             int* abort_s) {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  cta_sync();
  if (threadIdx.x == 0) {
    // release: the CTA's stores (ordered before this thread by the CTA barrier) become
    // visible device-wide no later than the arrival; acquire on the polling load
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ma.bar_count) : "memory");
    const unsigned target = (unsigned)(sstep + 1) * ma.expected_ctas;
    const unsigned long long t0 = global_ns();
    int abort = 0;
    for (unsigned it = 0;; ++it) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ma.bar_count) : "memory");
      if (v >= target) break;
      if ((it & 63u) == 63u && global_ns() - t0 > ma.limit_ns) {
        atomicOr(status, kStatusTimeout);
        abort = 1;
        break;
      }
    }
    unsigned st;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(st) : "l"(status) : "memory");
    *abort_s = abort || (st & kStatusTimeout) != 0;
  }
  cta_sync();
  asm volatile("fence.proxy.async.global;" ::: "memory");
  return *abort_s == 0;
}

// Population loads outside the staged rows: read-only path for a single step; for the
// multi-step mode, which reads buffers that other CTAs wrote earlier in the same launch,
// the L2 (coherent) path.
template <bool kCoherent>
__device__ __forceinline__ float ldpop(const float* p) {
  return kCoherent ? __ldcg(p) : __ldg(p);
}

// The statistics modes hold eleven more lane partials and four velocities; they are
// compiled for one CTA per SM fewer than the shape's time step (no spills).
__host__ __device__ constexpr int step_min_blocks(int mb, int mode) {
  return (mode == kModeStats || mode == kModeStepStats) && mb > 1 ? mb - 1 : mb;
}

template <int TY, int ST, int MB, int MODE>
__global__ void __launch_bounds__((TY + 1) * 32, step_min_blocks(MB, MODE))
    k_step_tma(const GridDev* __restrict__ grids, const int4* __restrict__ tiles, int ntiles,
               const uint32_t* __restrict__ mask, const float* __restrict__ src0,
               float* __restrict__ dst0, unsigned* __restrict__ status, StatsArgs sa,
               MultiArgs ma) {
  constexpr bool kMulti = MODE == kModeMulti;
  constexpr bool kCollide = MODE == kModeStep || MODE == kModeStepStats || kMulti;
  constexpr bool kStore = MODE != kModeStats;
  constexpr bool kStats = MODE == kModeStats || MODE == kModeStepStats;
  const int nst = kMulti ? ma.nsteps : 1;
  __shared__ int abort_s;
  using SS = StepShape<TY, ST, MB>;
  using TileMeta = typename SS::Meta;
  constexpr int kTY = TY, kStages = ST,
                kStageFloats = kStats ? SS::kStageFloatsStats : SS::kStageFloats,
                kUOff = SS::kStageFloats,  // statistics modes: u rows after the populations
                kMaskWords = SS::kMaskWords;
  extern __shared__ __align__(128) float stage_mem[];
  TileMeta* metas = reinterpret_cast<TileMeta*>(stage_mem + (size_t)kStages * kStageFloats);
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], kTY);
    }
    mbar_init_fence();
  }
  __syncthreads();
  // Programmatic dependent launch: the next step may be scheduled as this grid drains;
  // no thread touches the populations before the previous step has completed and its
  // writes are visible (its source is this step's destination and vice versa).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");

  if (warp == kTY) {
    // ------------------------------------------------------------ producer
    // Everything a tile needs from global memory besides the populations (its
    // descriptor, the grid descriptor words, the mask words) is loaded into registers
    // before waiting for the stage to drain, and the next tile's descriptor one
    // iteration ahead, so these dependent loads stay off the consumers' path.  The
    // grid's fields the producer itself needs come from the descriptor words by warp
    // shuffles.
    constexpr int kMetaWords = (int)(sizeof(GridDev) / 4);
    constexpr int kMaskRegs = (kMaskWords + 31) / 32;
    static_assert(kMetaWords <= 32, "grid descriptor copied by one warp pass");
    constexpr int kWNy = (int)(offsetof(GridDev, ny) / 4);
    constexpr int kWPitch = (int)(offsetof(GridDev, pitch) / 4);
    constexpr int kWWpr = (int)(offsetof(GridDev, wpr) / 4);
    constexpr int kWFoff = (int)(offsetof(GridDev, f_off) / 4);
    constexpr int kWPlane = (int)(offsetof(GridDev, plane) / 4);
    constexpr int kWMask = (int)(offsetof(GridDev, mask_off) / 4);
    auto word64 = [](uint32_t w, int at) {
      const uint32_t lo = __shfl_sync(0xffffffffu, w, at);
      const uint32_t hi = __shfl_sync(0xffffffffu, w, at + 1);
      return (long long)(((unsigned long long)hi << 32) | lo);
    };
    int k = 0;
    bool ok = true;
    for (int sstep = 0; sstep < nst; ++sstep) {
    const float* src = (kMulti && (sstep & 1)) ? dst0 : src0;
    int4 next = blockIdx.x < (unsigned)ntiles ? __ldg(&tiles[blockIdx.x]) : make_int4(0, 0, 0, 0);
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++k) {
      const int s = k % kStages;
      const int4 d = next;
      if (t + (int)gridDim.x < ntiles) next = __ldg(&tiles[t + gridDim.x]);
      const int gi = d.x, x0 = d.y, y0 = d.z, rows = d.w;
      const uint32_t* gw = reinterpret_cast<const uint32_t*>(grids + gi);
      const uint32_t meta_w = lane < kMetaWords ? __ldg(gw + lane) : 0u;
      const int ny = (int)__shfl_sync(0xffffffffu, meta_w, kWNy);
      const int pitch = (int)__shfl_sync(0xffffffffu, meta_w, kWPitch);
      const int wpr = (int)__shfl_sync(0xffffffffu, meta_w, kWWpr);
      const float* b = src + word64(meta_w, kWFoff);
      const long long plane = word64(meta_w, kWPlane);
      const uint32_t* m = mask + word64(meta_w, kWMask);
      const int xs = max(x0 - 4, 0);
      const int xe = min(x0 + kSeg + 4, pitch);
      const unsigned seg_bytes = (unsigned)(xe - xs) * 4u;
      uint32_t mask_w[kMaskRegs];
#pragma unroll
      for (int q = 0; q < kMaskRegs; ++q) {
        const int w = lane + 32 * q;
        mask_w[q] = 0u;
        if (w < kMaskWords) {
          const int r = w / kWords;
          int yy = y0 - 1 + r;
          yy = yy < 0 ? yy + ny : (yy >= ny ? yy % ny : yy);
          const int wi = (x0 >> 5) - 1 + (w - r * kWords);
          if (wi >= 0 && wi < wpr) mask_w[q] = __ldg(&m[yy * wpr + wi]);
        }
      }
      if (k >= kStages) ok = mbar_wait(&empty_bar[s], ((k / kStages) - 1) & 1, status);
      if (!ok) break;
      float* st = stage_mem + (size_t)s * kStageFloats;
      if (lane == 0)
        mbar_expect_tx(&full_bar[s], seg_bytes * (unsigned)(kQ * rows + 6) +
                                         (kStats ? 2u * (unsigned)rows * (unsigned)min(kSeg, pitch - x0) * 4u
                                                 : 0u));
      static_assert(kStageFloats > 0 && kMaskWords > 0, "shape");
      __syncwarp();
#pragma unroll
      for (int i = 0; i < kQ; ++i) {  // compile-time population index
        const int nr = rows + (cy_of(i) != 0 ? 1 : 0);  // rows past the last grid row skipped
        for (int r = lane; r < nr; r += 32) {
          int ys = y0 + stage_first(i) + r;
          ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
          bulk_g2s(st + (stage_row0<TY>(i) + r) * kRowF + (xs - (x0 - 4)),
                   b + (size_t)i * plane + (size_t)ys * pitch + xs, seg_bytes, &full_bar[s]);
        }
      }
      if constexpr (kStats) {
        // the tile's rows of the previous residual's velocity (pitched planes, so every
        // row segment is 16-byte aligned): u_x rows, then u_y rows
        const unsigned u_bytes = (unsigned)min(kSeg, pitch - x0) * 4u;
        const long long foff = word64(meta_w, kWFoff);
        for (int q = lane; q < 2 * rows; q += 32) {
          const int f = q / rows, r = q - f * rows;
          bulk_g2s(st + kUOff + (f * kTY + r) * kSeg,
                   (f ? sa.uy_prev : sa.ux_prev) + foff + (size_t)(y0 + r) * pitch + x0, u_bytes,
                   &full_bar[s]);
        }
      }
      // tile metadata and mask words (generic-proxy stores, released by the arrive)
      TileMeta* tm = metas + s;
      if (lane < kMetaWords) reinterpret_cast<uint32_t*>(&tm->g)[lane] = meta_w;
#pragma unroll
      for (int q = 0; q < kMaskRegs; ++q)
        if (lane + 32 * q < kMaskWords) tm->mask[lane + 32 * q] = mask_w[q];
      if (lane == 0) {
        tm->x0 = x0;
        tm->y0 = y0;
        tm->rows = rows;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_bar[s]);
    }
    if constexpr (kMulti) {
      if (!grid_barrier(ma, sstep, status, &abort_s)) break;
    }
    }  // steps
    // never leave with bulk copies in flight: wait (bounded) for the issued stages
    const int issued = k;
    for (int q = max(0, issued - kStages); q < issued; ++q)
      mbar_wait(&full_bar[q % kStages], (q / kStages) & 1, status);
    return;
  }

  // -------------------------------------------------------------- consumers
  int k = 0;
  bool alive = true;
  for (int sstep = 0; sstep < nst; ++sstep) {
  const float* src = (kMulti && (sstep & 1)) ? dst0 : src0;
  float* dst = (kMulti && (sstep & 1)) ? const_cast<float*>(src0) : dst0;
  for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x, ++k) {
    const int s = k % kStages;
    if (!mbar_wait(&full_bar[s], (k / kStages) & 1, status)) {
      alive = false;
      break;
    }
    const TileMeta* tm = metas + s;
    const GridDev G = tm->g;
    const int x0 = tm->x0, y0 = tm->y0;
    const bool row_ok = warp < tm->rows;  // warp-uniform
    if (!row_ok) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty_bar[s]);
      continue;
    }
    const int nx = G.nx, ny = G.ny;
    const int y = y0 + warp;
    const int x = x0 + kVec * lane;
    const bool active = x < nx;
    const bool periodic = G.periodic_x != 0;
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;
    const float* b = src + G.f_off;
    const unsigned P = (unsigned)G.plane;
    // solid bits: window bit b of row r (r = 0: y-1, 1: y, 2: y+1) <-> cell x - 1 + b
    const int bitpos = 31 + kVec * lane;
    const int k0 = bitpos >> 5, sh = bitpos & 31;
    uint32_t win[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const uint32_t* mw = tm->mask + (warp + r) * kWords;
      win[r] = __funnelshift_r(mw[k0], mw[k0 + 1], sh) & ((1u << (kVec + 2)) - 1u);
    }
    const int jw = nx - 1 - x;  // lane-local index of the cell x = nx-1, if 0..3
    const float* st = stage_mem + (size_t)s * kStageFloats;
    float g[kQ][kVec];
    uint32_t own_solid = 0;
    if (active) {
      const uint32_t* m = mask + G.mask_off;
      if (x == 0) {  // west neighbour of the first column
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          win[r] &= ~1u;
          if (periodic) win[r] |= (uint32_t)mask_bit(m, G.wpr, nx - 1, r == 0 ? ym : (r == 1 ? y : yp));
        }
      }
      if (jw >= 0 && jw < kVec) {  // east neighbour of the last column
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          win[r] &= ~(1u << (jw + 2));
          if (periodic)
            win[r] |= (uint32_t)mask_bit(m, G.wpr, 0, r == 0 ? ym : (r == 1 ? y : yp)) << (jw + 2);
        }
      }
      own_solid = (win[1] >> 1) & 0xFu;
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const float* rowp =
            st + (stage_row0<TY>(i) + warp - cy_of(i) - stage_first(i)) * kRowF + 4 + kVec * lane;
        const float4 c0 = *reinterpret_cast<const float4*>(rowp);
        const int ys = cy_of(i) > 0 ? ym : (cy_of(i) == 0 ? y : yp);
        if (cx_of(i) == 0) {
          g[i][0] = c0.x; g[i][1] = c0.y; g[i][2] = c0.z; g[i][3] = c0.w;
        } else if (cx_of(i) > 0) {  // source x - 1
          const float4 cm = *reinterpret_cast<const float4*>(rowp - 4);
          g[i][0] = cm.w; g[i][1] = c0.x; g[i][2] = c0.y; g[i][3] = c0.z;
          if (x == 0) g[i][0] = periodic ? ldpop<kMulti>(b + i * P + ys * G.pitch + nx - 1) : 0.0f;
        } else {  // source x + 1
          const float4 cp = *reinterpret_cast<const float4*>(rowp + 4);
          g[i][0] = c0.y; g[i][1] = c0.z; g[i][2] = c0.w; g[i][3] = cp.x;
          if (jw >= 0 && jw < kVec) {
            const float wrap = periodic ? ldpop<kMulti>(b + i * P + ys * G.pitch) : 0.0f;
#pragma unroll
            for (int j = 0; j < kVec; ++j)
              if (j == jw) g[i][j] = wrap;
          }
        }
      }
      // halfway bounce-back: the own cell's opposite population, from the stage
#pragma unroll
      for (int i = 1; i < kQ; ++i) {
        const int r = cy_of(i) > 0 ? 0 : (cy_of(i) == 0 ? 1 : 2);
        const uint32_t bb = ((win[r] >> (1 - cx_of(i))) & 0xFu) & ~own_solid;
        if (bb) {
          const int o = opp_of(i);
          const float4 v = *reinterpret_cast<const float4*>(
              st + (stage_row0<TY>(o) + warp - stage_first(o)) * kRowF + 4 + kVec * lane);
          if (bb & 1u) g[i][0] = v.x;
          if (bb & 2u) g[i][1] = v.y;
          if (bb & 4u) g[i][2] = v.z;
          if (bb & 8u) g[i][3] = v.w;
        }
      }
    }
    float4 pu = make_float4(0.f, 0.f, 0.f, 0.f), pv = pu;
    if constexpr (kStats) {  // the previous residual's velocity of this lane's four cells
      pu = *reinterpret_cast<const float4*>(st + kUOff + warp * kSeg + kVec * lane);
      pv = *reinterpret_cast<const float4*>(st + kUOff + (kTY + warp) * kSeg + kVec * lane);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty_bar[s]);  // this warp no longer reads the stage
    if constexpr (!kStats) {
      if (!active) continue;
    }
    // statistics of this lane's four cells (kStats): FP32 lane partials; the difference
    // to the previous residual's velocity is taken after the loop
    float acc[kStats ? R_COUNT : 1];
    float ux4[kVec], uy4[kVec];
    if constexpr (kStats) {
#pragma unroll
      for (int k = 0; k < R_COUNT; ++k) acc[k] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < kVec; ++j) {
      ux4[j] = 0.0f;
      uy4[j] = 0.0f;
      if constexpr (kStats) {
        if (!active) continue;
      }
      float c[kQ];
#pragma unroll
      for (int i = 0; i < kQ; ++i) c[i] = g[i][j];
      if (!periodic) {
        if (x + j == 0) {
          const float G0 = c[0] + c[2] + c[4] + 2.0f * (c[3] + c[6] + c[7]);
          const float ru = (G.bc_west == LBM_BC_PRESSURE)
                               ? G.west_d - G0
                               : (1.0f + G0) / (1.0f - G.west_d) * G.west_d;
          const float tt = 0.5f * (c[2] - c[4]);
          c[1] = c[3] + (2.0f / 3.0f) * ru;
          c[5] = c[7] - tt + (1.0f / 6.0f) * ru;
          c[8] = c[6] + tt + (1.0f / 6.0f) * ru;
        }
        if (x + j == nx - 1) {
          const float G0 = c[0] + c[2] + c[4] + 2.0f * (c[1] + c[5] + c[8]);
          const float ru = (G.bc_east == LBM_BC_PRESSURE)
                               ? G0 - G.east_d
                               : (1.0f + G0) / (1.0f + G.east_d) * G.east_d;
          const float tt = 0.5f * (c[2] - c[4]);
          c[3] = c[1] - (2.0f / 3.0f) * ru;
          c[7] = c[5] + tt - (1.0f / 6.0f) * ru;
          c[6] = c[8] - tt - (1.0f / 6.0f) * ru;
        }
      }
      const bool keep = !((own_solid >> j) & 1u);  // solid cells store 0
      if constexpr (kStats) {
        if (keep && x + j < nx) {
          float drho, rho, ux, uy;
          moments(G, c, drho, rho, ux, uy);
          const float u2 = ux * ux + uy * uy;
          acc[R_U2] += u2;
          if (!periodic && x + j == 0) {
            acc[R_RHO_W] += drho;
            acc[R_N_W] += 1.0f;
          }
          if (!periodic && x + j == nx - 1) {
            acc[R_RHO_E] += drho;
            acc[R_N_E] += 1.0f;
          }
          acc[R_DRHO] += drho;
          acc[R_MOMX] += rho * ux;
          acc[R_MOMY] += rho * uy;
          acc[R_BAD] += (!isfinite(drho) || !isfinite(u2) || u2 > sa.u_max2) ? 1.0f : 0.0f;
          acc[R_FLUID] += 1.0f;
          ux4[j] = ux;
          uy4[j] = uy;
        }
      }
      if constexpr (!kStats) {
        if constexpr (kCollide) collide(G, c);
        if constexpr (kStore) {
#pragma unroll
          for (int i = 0; i < kQ; ++i) g[i][j] = keep ? c[i] : 0.0f;
        }
      } else if constexpr (kStore) {
        // statistics modes: keep the completed populations; the collision runs after the
        // statistics are reduced, so the lane partials are dead by then
#pragma unroll
        for (int i = 0; i < kQ; ++i) g[i][j] = c[i];
      }
    }
    if constexpr (kStats) {
      if (active) {
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
          if (((own_solid >> j) & 1u) || x + j >= nx) continue;
          const float dux = ux4[j] - f4get(pu, j);
          const float duy = uy4[j] - f4get(pv, j);
          acc[R_DU2] += dux * dux + duy * duy;
        }
      }
      if (active && sa.update_prev) {
        // pitched rows: the four cells (and any row padding past nx, which stays 0) are
        // one aligned float4; solid cells keep 0, as set by the re-initialisation
        const size_t pc = (size_t)G.f_off + (size_t)y * G.pitch + x;
        *reinterpret_cast<float4*>(sa.ux_prev + pc) = make_float4(ux4[0], ux4[1], ux4[2], ux4[3]);
        *reinterpret_cast<float4*>(sa.uy_prev + pc) = make_float4(uy4[0], uy4[1], uy4[2], uy4[3]);
      }
      // FP32 sums over the segment's 128 cells, all statistics in one warp butterfly
      float v16[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) v16[k] = k < R_COUNT ? acc[k] : 0.0f;
      const float tot = warp_sum16(v16, lane);
      const long long slot = (long long)G.rblk_start * kSegsPerRblk + (long long)y * G.nseg + x0 / kSeg;
      if ((lane & 1) == 0 && (lane >> 1) < R_COUNT)
        sa.seg_partial[slot * kSegStride + (lane >> 1)] = tot;
      if (!active) continue;
      if constexpr (kStore) {
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
          float c[kQ];
#pragma unroll
          for (int i = 0; i < kQ; ++i) c[i] = g[i][j];
          if constexpr (kCollide) collide(G, c);
          const bool keep = !((own_solid >> j) & 1u);  // solid cells store 0
#pragma unroll
          for (int i = 0; i < kQ; ++i) g[i][j] = keep ? c[i] : 0.0f;
        }
      }
    }
    if constexpr (kStore) {
      float* o = dst + G.f_off + (size_t)y * G.pitch + x;
      if (x + kVec <= nx) {
#pragma unroll
        for (int i = 0; i < kQ; ++i)
          *reinterpret_cast<float4*>(o + i * P) = make_float4(g[i][0], g[i][1], g[i][2], g[i][3]);
      } else {
#pragma unroll
        for (int j = 0; j < kVec; ++j)
          if (x + j < nx) {
#pragma unroll
            for (int i = 0; i < kQ; ++i) o[i * P + j] = g[i][j];
          }
      }
    }
  }
  if constexpr (kMulti) {
    if (!grid_barrier(ma, sstep, status, &abort_s)) break;
  }
  }  // steps
}

// Tile shapes compiled into the library (rows per tile, stages, CTAs per SM).
// Every shape performs the same arithmetic per cell in the same order, so the
// choice changes speed only; lbm_autotune times them on the caller's batch.
using StepKernel = void (*)(const GridDev*, const int4*, int, const uint32_t*, const float*,
                           float*, unsigned*, StatsArgs, MultiArgs);
constexpr int kStepModes = 5;
struct StepVariant {
  int ty, stages, minb;
  StepKernel kernel[kStepModes];  // by StepMode
  size_t smem;        // dynamic shared memory of the modes without statistics
  size_t smem_stats;  // ... of kModeStats and kModeStepStats
  size_t smem_of(int mode) const {
    return mode == kModeStats || mode == kModeStepStats ? smem_stats : smem;
  }
};
#define LBM_STEP_VARIANT(TY, ST, MB)                                                       \
  StepVariant {                                                                            \
    TY, ST, MB,                                                                            \
        {k_step_tma<TY, ST, MB, kModeStep>, k_step_tma<TY, ST, MB, kModeStream>,           \
         k_step_tma<TY, ST, MB, kModeStats>, k_step_tma<TY, ST, MB, kModeStepStats>,       \
         k_step_tma<TY, ST, MB, kModeMulti>},                                              \
        StepShape<TY, ST, MB>::kSmem, StepShape<TY, ST, MB>::kSmemStats                    \
  }
static const StepVariant kStepVariants[LBM_STEP_VARIANTS] = {
    LBM_STEP_VARIANT(3, 2, 5), LBM_STEP_VARIANT(4, 2, 4), LBM_STEP_VARIANT(2, 2, 7),
    LBM_STEP_VARIANT(5, 2, 4), LBM_STEP_VARIANT(3, 3, 4), LBM_STEP_VARIANT(6, 2, 3)};
#undef LBM_STEP_VARIANT

__global__ void __launch_bounds__(kBlock) k_export(const GridDev* __restrict__ grids, int ngrids,
                                                   const uint32_t* __restrict__ mask,
                                                   const float* __restrict__ src,
                                                   float* __restrict__ out) {
  int gidx, x, y;
  if (!cell_of_thread(grids, ngrids, gidx, x, y)) return;
  const GridDev G = grids[gidx];  // registers: stores below cannot alias it
  float g[kQ];
  if (!pull_cell(G, mask, src, x, y, g)) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] = 0.0f;
  }
  const long long cells = (long long)G.nx * G.ny;
  float* o = out + 9 * G.cell_off + (long long)y * G.nx + x;
#pragma unroll
  for (int i = 0; i < kQ; ++i) o[i * cells] = g[i];
}

// copy canonical <-> pitched state (dir 0: canonical -> state, 1: state -> canonical)
__global__ void __launch_bounds__(kBlock) k_copy_state(const GridDev* __restrict__ grids,
                                                       int ngrids, float* state,
                                                       float* canon, int dir) {
  int gidx, x, y;
  if (!cell_of_thread(grids, ngrids, gidx, x, y)) return;
  const GridDev G = grids[gidx];  // registers: stores below cannot alias it
  const long long cells = (long long)G.nx * G.ny;
  float* s = state + G.f_off + (long long)y * G.pitch + x;
  float* c = canon + 9 * G.cell_off + (long long)y * G.nx + x;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    if (dir == 0)
      s[i * G.plane] = c[i * cells];
    else
      c[i * cells] = s[i * G.plane];
  }
}

__global__ void __launch_bounds__(kBlock) k_macro(const GridDev* __restrict__ grids, int ngrids,
                                                  const uint32_t* __restrict__ mask,
                                                  const float* __restrict__ src,
                                                  float* __restrict__ rho_o,
                                                  float* __restrict__ ux_o,
                                                  float* __restrict__ uy_o) {
  int gidx, x, y;
  if (!cell_of_thread(grids, ngrids, gidx, x, y)) return;
  const GridDev G = grids[gidx];  // registers: stores below cannot alias it
  float g[kQ];
  float rho = 1.0f, ux = 0.0f, uy = 0.0f, drho;
  if (pull_cell(G, mask, src, x, y, g)) moments(G, g, drho, rho, ux, uy);
  const long long c = G.cell_off + (long long)y * G.nx + x;
  if (rho_o) rho_o[c] = rho;
  if (ux_o) ux_o[c] = ux;
  if (uy_o) uy_o[c] = uy;
}

// Deterministic FP64 block reduction of R_COUNT values; thread 0 writes the result.
__device__ __forceinline__ void block_reduce_store(double v[R_COUNT], double* out) {
  __shared__ double red[kBlock / 32][R_COUNT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < R_COUNT; ++k) {
    double a = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) red[warp][k] = a;
  }
  __syncthreads();
  if (threadIdx.x < R_COUNT) {
    double a = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) a += red[w][threadIdx.x];
    out[threadIdx.x] = a;
  }
}

// Steady-state statistics of the current time level, stage 1: the step kernel in a
// statistics mode leaves FP32 sums (a warp tree over the 128 cells of one row segment)
// per row segment; block b of grid g sums the segments b * kSegsPerRblk .. +kSegsPerRblk
// of the grid in FP64, four consecutive segments per thread, then in a fixed FP64 tree.  Stage 2
// (k_residual_final) adds a grid's blocks.  Fixed maps and trees: deterministic.
__global__ void __launch_bounds__(kBlock) k_stats_reduce(const GridDev* __restrict__ grids,
                                                         int ngrids,
                                                         const float* __restrict__ seg_partial,
                                                         double* __restrict__ partial) {
  constexpr int kPerThread = kSegsPerRblk / kBlock;
  static_assert(kPerThread * kBlock == kSegsPerRblk, "whole segments per thread");
  const int gidx = grid_of<&GridDev::rblk_start>(grids, ngrids, blockIdx.x);
  const GridDev& G = grids[gidx];
  const long long nsegs = (long long)G.nseg * G.ny;
  const long long task0 =
      (long long)(blockIdx.x - G.rblk_start) * kSegsPerRblk + (long long)threadIdx.x * kPerThread;
  double v[R_COUNT];
#pragma unroll
  for (int k = 0; k < R_COUNT; ++k) v[k] = 0.0;
  for (int q = 0; q < kPerThread; ++q) {  // consecutive segments, in order
    const long long task = task0 + q;
    if (task < nsegs) {
      const float* sp = seg_partial + ((long long)G.rblk_start * kSegsPerRblk + task) * kSegStride;
#pragma unroll
      for (int k = 0; k < R_COUNT; ++k) v[k] += (double)sp[k];
    }
  }
  block_reduce_store(v, partial + (size_t)blockIdx.x * R_COUNT);
}

__global__ void __launch_bounds__(kBlock) k_residual_final(const GridDev* __restrict__ grids,
                                                           const double* __restrict__ partial,
                                                           double* __restrict__ stats) {
  const GridDev& G = grids[blockIdx.x];
  double v[R_COUNT];
#pragma unroll
  for (int k = 0; k < R_COUNT; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < G.nrblk; b += kBlock) {
    const double* s = partial + (size_t)(G.rblk_start + b) * R_COUNT;
#pragma unroll
    for (int k = 0; k < R_COUNT; ++k) v[k] += s[k];
  }
  block_reduce_store(v, stats + (size_t)blockIdx.x * R_COUNT);
}

// Vorticity omega = d_x u_y - d_y u_x of dense velocity fields (the accuracy metric of
// the unsteady results, Sec. 3.2.2), with the re-initialisation's difference stencils;
// solid cells get 0.
__global__ void __launch_bounds__(kBlock) k_vorticity(const GridDev* __restrict__ grids,
                                                      int ngrids, const uint32_t* __restrict__ mask,
                                                      const float* __restrict__ ux_i,
                                                      const float* __restrict__ uy_i,
                                                      float* __restrict__ omega) {
  int gidx, x, y;
  if (!cell_of_thread(grids, ngrids, gidx, x, y)) return;
  const GridDev G = grids[gidx];
  const uint32_t* m = mask + G.mask_off;
  const long long c = G.cell_off + (long long)y * G.nx + x;
  if (mask_bit(m, G.wpr, x, y)) {
    omega[c] = 0.0f;
    return;
  }
  omega[c] = dfield(G, m, uy_i + G.cell_off, x, y, 0) - dfield(G, m, ux_i + G.cell_off, x, y, 1);
}

// ------------------------------------------------------------ host side ---
struct WsPlan {
  size_t grids_off, uprev_off, seg_off, partial_off, stats_off, status_off, bar_off, tiles_off,
      total;
};

// Scratch of one statistics evaluation: FP32 row-segment partials, FP64 block sums,
// FP64 per-grid sums, laid out one after the other at 256-byte boundaries.
struct StatsScratch {
  size_t seg_off, partial_off, stats_off, total;
};
static StatsScratch stats_scratch(long long nrblk_total, int ngrids) {
  StatsScratch r{};
  r.seg_off = 0;
  r.partial_off = align_up((size_t)nrblk_total * kSegsPerRblk * kSegStride * sizeof(float), 256);
  r.stats_off = align_up(r.partial_off + (size_t)nrblk_total * R_COUNT * sizeof(double), 256);
  r.total = align_up(r.stats_off + (size_t)ngrids * R_COUNT * sizeof(double), 256);
  return r;
}

static int plan_layout(const lbm_grid* grids, int ngrids, lbm_layout* lay,
                       std::vector<GridDev>* gd, WsPlan* wp) {
  LBM_REQUIRE(grids != nullptr && ngrids > 0, "lbm: need at least one grid");
  size_t f = 0, words = 0, cells = 0;
  long long blk = 0, tiles = 0, rblk = 0;
  if (gd) gd->clear();
  // Population-major batch layout: plane i holds population i of every grid, grid after
  // grid (each grid ny rows of pitch floats), so a batch of small grids streams nine
  // contiguous planes exactly like one tall grid.
  size_t plane_all = 0;
  for (int k = 0; k < ngrids; ++k) {
    LBM_REQUIRE(grids[k].nx >= 2 && grids[k].ny >= 2 && grids[k].nx <= (1 << 20) &&
                    grids[k].ny <= (1 << 20),
                "lbm: grid %d has invalid size %d x %d", k, grids[k].nx, grids[k].ny);
    plane_all += (size_t)grids[k].ny * align_up((size_t)grids[k].nx, 32);
  }
  LBM_REQUIRE((size_t)kQ * plane_all < (1ull << 31),
              "lbm: batch too large (9 * padded cells >= 2^31)");
  for (int k = 0; k < ngrids; ++k) {
    const lbm_grid& g = grids[k];
    LBM_REQUIRE(g.nx >= 2 && g.ny >= 2 && g.nx <= (1 << 20) && g.ny <= (1 << 20),
                "lbm: grid %d has invalid size %d x %d", k, g.nx, g.ny);
    LBM_REQUIRE(g.tau > 0.5 && g.tau < 100.0, "lbm: grid %d tau %g not in (0.5, 100)", k,
                g.tau);
    const bool pw = g.bc_west == LBM_BC_PERIODIC, pe = g.bc_east == LBM_BC_PERIODIC;
    LBM_REQUIRE(pw == pe, "lbm: grid %d: periodic x needs both ends periodic", k);
    LBM_REQUIRE(g.bc_west >= 0 && g.bc_west <= 2 && g.bc_east >= 0 && g.bc_east <= 2,
                "lbm: grid %d: unknown boundary kind", k);
    if (g.bc_west == LBM_BC_VELOCITY)
      LBM_REQUIRE(fabs(g.west_value) < 0.5, "lbm: grid %d: |inlet velocity| >= 0.5", k);
    if (g.bc_east == LBM_BC_VELOCITY)
      LBM_REQUIRE(fabs(g.east_value) < 0.5, "lbm: grid %d: |outlet velocity| >= 0.5", k);
    if (g.bc_west == LBM_BC_PRESSURE)
      LBM_REQUIRE(g.west_value > 0.5 && g.west_value < 2.0, "lbm: grid %d: inlet rho", k);
    if (g.bc_east == LBM_BC_PRESSURE)
      LBM_REQUIRE(g.east_value > 0.5 && g.east_value < 2.0, "lbm: grid %d: outlet rho", k);
    GridDev d{};
    d.nx = g.nx;
    d.ny = g.ny;
    d.pitch = (int)align_up((size_t)g.nx, 32);
    d.wpr = (g.nx + 31) / 32;
    d.f_off = (long long)f;  // offset of the grid's first row inside each plane
    d.plane = (long long)plane_all;
    d.mask_off = (long long)words;
    d.cell_off = (long long)cells;
    d.nblk = (int)(((long long)g.ny * d.pitch + kBlock - 1) / kBlock);
    d.blk_start = (int)blk;
    d.nseg = (g.nx + kSeg - 1) / kSeg;
    d.nrblk = (int)(((long long)d.nseg * g.ny + kSegsPerRblk - 1) / kSegsPerRblk);
    d.rblk_start = (int)rblk;


    d.tau = (float)g.tau;
    d.omega = (float)(1.0 / g.tau);
    d.guo = (float)(1.0 - 0.5 / g.tau);
    d.fx = (float)g.fx;
    d.fy = (float)g.fy;
    d.periodic_x = pw ? 1 : 0;
    d.bc_west = g.bc_west;
    d.bc_east = g.bc_east;
    d.west_d = (float)(g.bc_west == LBM_BC_PRESSURE ? g.west_value - 1.0 : g.west_value);
    d.east_d = (float)(g.bc_east == LBM_BC_PRESSURE ? g.east_value - 1.0 : g.east_value);
    f += (size_t)g.ny * d.pitch;
    words += (size_t)d.wpr * g.ny;
    cells += (size_t)g.nx * g.ny;
    blk += d.nblk;
    tiles += (long long)d.nseg * g.ny;
    rblk += d.nrblk;
    LBM_REQUIRE(blk < (1LL << 30) && tiles < (1LL << 30),
                "lbm: batch too large");
    if (gd) gd->push_back(d);
  }
  WsPlan w{};
  w.grids_off = 0;
  w.uprev_off = align_up(sizeof(GridDev) * ngrids, 256);
  const StatsScratch sc = stats_scratch(rblk, ngrids);
  w.seg_off = align_up(w.uprev_off + 2 * plane_all * sizeof(float), 256);
  w.partial_off = w.seg_off + sc.partial_off;
  w.stats_off = w.seg_off + sc.stats_off;
  w.status_off = w.seg_off + sc.total;
  w.bar_off = align_up(w.status_off + sizeof(unsigned), 256);
  w.tiles_off = align_up(w.bar_off + sizeof(unsigned), 256);
  size_t tiles_all = 0;  // descriptors of every tile shape
  for (int v = 0; v < LBM_STEP_VARIANTS; ++v)
    for (int k = 0; k < ngrids; ++k)
      tiles_all += (size_t)((grids[k].nx + kSeg - 1) / kSeg) *
                   ((grids[k].ny + kStepVariants[v].ty - 1) / kStepVariants[v].ty);
  w.total = align_up(w.tiles_off + tiles_all * sizeof(int4), 256);
  lay->f_elems = (size_t)kQ * plane_all;
  lay->mask_words = words;
  lay->cells = cells;
  lay->ws_bytes = w.total;
  if (wp) *wp = w;
  return LBM_OK;
}

static inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }
constexpr double kBarrierLimitMs = 2000.0;  // bound of one grid-barrier wait

// One launch of the step kernel in `mode` over every grid with tile shape `v`: reads
// `src`, writes `dst` (modes that store populations).
static int launch_step(Handle* h, int v, int mode, const float* src, float* dst, cudaStream_t s,
                       const StatsArgs& sa = StatsArgs{}) {
  const StepVariant& sv = kStepVariants[v];
  const int ctas = std::min(h->ntiles_v[v], h->nsm * std::max(1, h->blocks_per_sm_vm[v][mode]));
  // launched with programmatic stream serialisation: consecutive steps overlap the
  // launch of the next grid with the tail of the previous one (see griddepcontrol above)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3((unsigned)((sv.ty + 1) * 32));
  cfg.dynamicSmemBytes = sv.smem_of(mode);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  LBM_CHECK_CUDA(cudaLaunchKernelEx(&cfg, sv.kernel[mode], (const GridDev*)h->gd_d,
                                    (const int4*)h->tiles_d[v], h->ntiles_v[v],
                                    (const uint32_t*)h->mask, src, dst, h->status_d, sa,
                                    MultiArgs{}));
  return LBM_OK;
}

// nsteps time steps in one cooperative launch of the multi-step mode (every CTA resident;
// grid-wide barrier between steps).  expected_extra > 0 makes every barrier wait for CTAs
// that do not exist (the self-test of the bounded wait); status: the word the kernel
// reports an expired wait in.
static int launch_multi(Handle* h, int v, int nsteps, const float* src, float* dst,
                        unsigned* status, unsigned expected_extra, double limit_ms,
                        cudaStream_t s) {
  const StepVariant& sv = kStepVariants[v];
  const int ctas = std::min(h->ntiles_v[v], h->nsm * std::max(1, h->blocks_per_sm_vm[v][kModeMulti]));
  LBM_CHECK_CUDA(cudaMemsetAsync(h->bar_count, 0, sizeof(unsigned), s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3((unsigned)((sv.ty + 1) * 32));
  cfg.dynamicSmemBytes = sv.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MultiArgs ma{nsteps, h->bar_count, (unsigned)ctas + expected_extra,
               (unsigned long long)(limit_ms * 1.0e6)};
  LBM_CHECK_CUDA(cudaLaunchKernelEx(&cfg, sv.kernel[kModeMulti], (const GridDev*)h->gd_d,
                                    (const int4*)h->tiles_d[v], h->ntiles_v[v],
                                    (const uint32_t*)h->mask, src, dst, status, StatsArgs{}, ma));
  return LBM_OK;
}

// Per-grid statistics (enum lbm_stat_index) from the FP64 sums of R_COUNT raw values;
// returns LBM_ERR_UNSTABLE if a grid has non-finite values or |u| > u_max.
static int finish_stats(const Handle* h, double* out_h, const char* name) {
  bool bad = false;
  for (int g = 0; g < h->ngrids; ++g) {
    const double* r = &h->stats_h[(size_t)g * R_COUNT];
    double* o = out_h + (size_t)g * LBM_NSTAT;
    o[LBM_STAT_RESIDUAL] = r[R_U2] > 0 ? sqrt(r[R_DU2] / r[R_U2]) : INFINITY;
    o[LBM_STAT_UNORM] = sqrt(r[R_U2]);
    const double rw = r[R_N_W] > 0 ? r[R_RHO_W] / r[R_N_W] : 0.0;
    const double re = r[R_N_E] > 0 ? r[R_RHO_E] / r[R_N_E] : 0.0;
    o[LBM_STAT_DP] = (rw - re) / 3.0;
    o[LBM_STAT_MASS] = r[R_FLUID] + r[R_DRHO];
    o[LBM_STAT_MOMX] = r[R_MOMX];
    o[LBM_STAT_MOMY] = r[R_MOMY];
    o[LBM_STAT_BAD] = r[R_BAD];
    o[LBM_STAT_FLUID] = r[R_FLUID];
    if (r[R_BAD] > 0 || !std::isfinite(r[R_DU2]) || !std::isfinite(r[R_U2])) bad = true;
  }
  if (bad) {
    set_error("%s: non-finite values or |u| > u_max detected", name);
    return LBM_ERR_UNSTABLE;
  }
  return LBM_OK;
}

// Statistics of the current time level into out_h, with the scratch at `scratch`
// (layout of stats_scratch): the step kernel in kModeStats (nothing else written) or
// kModeStepStats (the next time level written to the other buffer, which the caller
// may accept), the two reduction stages, one copy back.  Synchronises `s`.
static int residual_run(Handle* h, int mode, char* scratch, double* out_h, int update_prev,
                        cudaStream_t s, const char* name) {
  const StatsScratch sc = stats_scratch(h->nrblk_total, h->ngrids);
  float* seg = reinterpret_cast<float*>(scratch + sc.seg_off);
  double* partial = reinterpret_cast<double*>(scratch + sc.partial_off);
  double* stats = reinterpret_cast<double*>(scratch + sc.stats_off);
  StatsArgs sa{h->ux_prev, h->uy_prev, seg, h->u_max2, update_prev ? 1 : 0};
  LBM_TRY(launch_step(h, h->variant, mode, h->f[h->cur], h->f[h->cur ^ 1], s, sa));
  if (h->nrblk_total == h->ngrids) {
    // every grid's segments fit one first-stage block: its sum is the grid's total
    k_stats_reduce<<<h->nrblk_total, kBlock, 0, s>>>(h->gd_d, h->ngrids, seg, stats);
    LBM_CHECK_LAUNCH();
  } else {
    k_stats_reduce<<<h->nrblk_total, kBlock, 0, s>>>(h->gd_d, h->ngrids, seg, partial);
    LBM_CHECK_LAUNCH();
    k_residual_final<<<h->ngrids, kBlock, 0, s>>>(h->gd_d, partial, stats);
    LBM_CHECK_LAUNCH();
  }
  LBM_CHECK_CUDA(cudaMemcpyAsync(h->stats_h.data(), stats, sizeof(double) * R_COUNT * h->ngrids,
                                 cudaMemcpyDeviceToHost, s));
  LBM_CHECK_CUDA(cudaMemcpyAsync(&h->status_h, h->status_d, sizeof(unsigned),
                                 cudaMemcpyDeviceToHost, s));
  LBM_CHECK_CUDA(cudaStreamSynchronize(s));
  if (h->status_h & kStatusTimeout) {
    set_error("lbm: a device-side wait expired (status 0x%x)", h->status_h);
    return LBM_ERR_TIMEOUT;
  }
  return finish_stats(h, out_h, name);
}

int residual_step(Handle* h, double* out_h, int update_prev, cudaStream_t s) {
  return residual_run(h, kModeStepStats, h->scratch, out_h, update_prev, s,
                      "lbm_step_residual");
}

}  // namespace lbmfno

using namespace lbmfno;


extern "C" {

const char* lbm_last_error(void) { return lbmfno::g_err; }

int lbm_query_layout(const lbm_grid* grids_h, int ngrids, lbm_layout* out_h) {
  LBM_REQUIRE(out_h != nullptr, "lbm_query_layout: null output");
  return plan_layout(grids_h, ngrids, out_h, nullptr, nullptr);
}

int lbm_init(const lbm_grid* grids_h, int ngrids, const uint32_t* mask_d, float* f_a_d,
             float* f_b_d, void* ws_d, double u_max, void* stream, lbm_handle** out) {
  LBM_REQUIRE(out != nullptr, "lbm_init: null handle output");
  *out = nullptr;
  LBM_REQUIRE(mask_d && f_a_d && f_b_d && ws_d, "lbm_init: null device pointer");
  LBM_REQUIRE(((uintptr_t)f_a_d % 16) == 0 && ((uintptr_t)f_b_d % 16) == 0 &&
                  ((uintptr_t)ws_d % 256) == 0,
              "lbm_init: f buffers need 16-byte and workspace 256-byte alignment");
  LBM_REQUIRE(u_max > 0.0 && u_max < 1.0, "lbm_init: u_max must be in (0, 1)");
  lbm_handle* h = new lbm_handle();
  WsPlan wp;
  int st = plan_layout(grids_h, ngrids, &h->layout, &h->gd, &wp);
  if (st != LBM_OK) {
    delete h;
    return st;
  }
  h->grids.assign(grids_h, grids_h + ngrids);
  h->ngrids = ngrids;
  h->nblk_total = h->gd.back().blk_start + h->gd.back().nblk;
  h->nrblk_total = h->gd.back().rblk_start + h->gd.back().nrblk;
  h->mask = mask_d;
  h->f[0] = f_a_d;
  h->f[1] = f_b_d;
  char* ws = static_cast<char*>(ws_d);
  h->gd_d = reinterpret_cast<GridDev*>(ws + wp.grids_off);
  h->ux_prev = reinterpret_cast<float*>(ws + wp.uprev_off);
  h->uy_prev = h->ux_prev + h->layout.f_elems / kQ;  // one pitched plane per field
  h->scratch = ws + wp.seg_off;
  h->status_d = reinterpret_cast<unsigned*>(ws + wp.status_off);
  h->bar_count = reinterpret_cast<unsigned*>(ws + wp.bar_off);
  // tile descriptors of every shape: grid after grid, row of tiles after row of tiles
  std::vector<int4> tiles;
  std::vector<size_t> tiles_at(LBM_STEP_VARIANTS);
  for (int v = 0; v < LBM_STEP_VARIANTS; ++v) {
    tiles_at[v] = tiles.size();
    const int ty = kStepVariants[v].ty;
    for (int k = 0; k < ngrids; ++k) {
      const GridDev& d = h->gd[k];
      for (int y0 = 0; y0 < d.ny; y0 += ty)
        for (int sg = 0; sg < d.nseg; ++sg)
          tiles.push_back(make_int4(k, sg * kSeg, y0, std::min(ty, d.ny - y0)));
    }
    h->ntiles_v[v] = (int)(tiles.size() - tiles_at[v]);
  }
  for (int v = 0; v < LBM_STEP_VARIANTS; ++v)
    h->tiles_d[v] = reinterpret_cast<int4*>(ws + wp.tiles_off) + tiles_at[v];
  h->stats_h.assign((size_t)ngrids * R_COUNT, 0.0);
  h->u_max2 = (float)(u_max * u_max);
  cudaStream_t s = S(stream);
  {
    int dev = 0;
    bool ok = cudaGetDevice(&dev) == cudaSuccess &&
              cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    for (int v = 0; ok && v < LBM_STEP_VARIANTS; ++v) {
      const StepVariant& sv = kStepVariants[v];
      for (int m = 0; ok && m < kStepModes; ++m)
        ok = cudaFuncSetAttribute(sv.kernel[m], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sv.smem_of(m)) == cudaSuccess;
      // each mode's persistent grid holds the CTAs that fit at once
      for (int m = 0; ok && m < kStepModes; ++m)
        ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->blocks_per_sm_vm[v][m],
                                                           sv.kernel[m], (sv.ty + 1) * 32,
                                                           sv.smem_of(m)) == cudaSuccess;
      h->blocks_per_sm_v[v] = h->blocks_per_sm_vm[v][kModeStep];
    }
    if (ok) ok = reinit_init(h) == LBM_OK;
    if (!ok) {
      set_error("lbm_init: %s", cudaGetErrorString(cudaGetLastError()));
      delete h;
      return LBM_ERR_CUDA;
    }
    h->variant = 0;
  }
  auto fail = [&](int code) {
    delete h;
    return code;
  };
  if (cudaMemcpyAsync(h->gd_d, h->gd.data(), sizeof(GridDev) * ngrids, cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      cudaMemsetAsync(f_a_d, 0, h->layout.f_elems * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(f_b_d, 0, h->layout.f_elems * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(h->ux_prev, 0, 2 * (h->layout.f_elems / kQ) * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(h->status_d, 0, sizeof(unsigned), s) != cudaSuccess ||
      cudaMemcpyAsync(h->tiles_d[0], tiles.data(), tiles.size() * sizeof(int4),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("lbm_init: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(LBM_ERR_CUDA);
  }
  *out = h;
  return LBM_OK;
}

int lbm_step(lbm_handle* h, int nsteps, void* stream) {
  LBM_REQUIRE(h != nullptr && nsteps >= 0, "lbm_step: bad arguments");
  cudaStream_t s = S(stream);
  if (h->persistent && nsteps > 1) {
    LBM_TRY(launch_multi(h, h->variant, nsteps, h->f[h->cur], h->f[h->cur ^ 1], h->status_d, 0u,
                         kBarrierLimitMs, s));
    if (nsteps & 1) h->cur ^= 1;
    h->steps += nsteps;
    return LBM_OK;
  }
  for (int k = 0; k < nsteps; ++k) {
    LBM_TRY(launch_step(h, h->variant, kModeStep, h->f[h->cur], h->f[h->cur ^ 1], s));
    h->cur ^= 1;
  }
  h->steps += nsteps;
  return LBM_OK;
}

int lbm_macro(lbm_handle* h, float* rho_d, float* ux_d, float* uy_d, void* stream) {
  LBM_REQUIRE(h != nullptr, "lbm_macro: null handle");
  k_macro<<<h->nblk_total, kBlock, 0, S(stream)>>>(h->gd_d, h->ngrids, h->mask, h->f[h->cur],
                                                   rho_d, ux_d, uy_d);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int lbm_residual(lbm_handle* h, double* out_h, int update_prev, void* stream) {
  LBM_REQUIRE(h != nullptr && out_h != nullptr, "lbm_residual: bad arguments");
  return residual_run(h, kModeStats, h->scratch, out_h, update_prev, S(stream), "lbm_residual");
}

int lbm_step_residual(lbm_handle* h, double* out_h, int update_prev, void* stream) {
  LBM_REQUIRE(h != nullptr && out_h != nullptr, "lbm_step_residual: bad arguments");
  const int rc = residual_step(h, out_h, update_prev, S(stream));
  if (rc == LBM_OK || rc == LBM_ERR_UNSTABLE) accept_step(h);
  return rc;
}

int lbm_set_persistent(lbm_handle* h, int on) {
  LBM_REQUIRE(h != nullptr, "lbm_set_persistent: null handle");
  h->persistent = on != 0;
  return LBM_OK;
}

int lbm_barrier_selftest(lbm_handle* h, unsigned* status_d, int arrive_all, double limit_ms,
                         void* stream) {
  LBM_REQUIRE(h != nullptr && status_d != nullptr, "lbm_barrier_selftest: bad arguments");
  LBM_REQUIRE(limit_ms > 0.0 && limit_ms <= 2000.0,
              "lbm_barrier_selftest: limit_ms must be in (0, 2000]");
  cudaStream_t s = S(stream);
  LBM_CHECK_CUDA(cudaMemsetAsync(status_d, 0, sizeof(unsigned), s));
  // two steps from the current state into the other buffer and back: the second step
  // only runs after the barrier, so with arrive_all == 0 the state is left unchanged
  LBM_TRY(launch_multi(h, h->variant, 2, h->f[h->cur], h->f[h->cur ^ 1], status_d,
                       arrive_all ? 0u : 1u, limit_ms, s));
  unsigned st = 0;
  LBM_CHECK_CUDA(cudaMemcpyAsync(&st, status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  LBM_CHECK_CUDA(cudaStreamSynchronize(s));
  if (st & kStatusTimeout) {
    set_error("lbm_barrier_selftest: the grid barrier wait expired after %.3f ms (status 0x%x)",
              limit_ms, st);
    return LBM_ERR_TIMEOUT;
  }
  h->steps += 2;  // two steps taken: the state is back in the current buffer
  return LBM_OK;
}

int lbm_stream_probe(lbm_handle* h, int variant, void* stream) {
  LBM_REQUIRE(h != nullptr && variant >= 0 && variant < LBM_STEP_VARIANTS,
              "lbm_stream_probe: bad arguments");
  LBM_REQUIRE(h->blocks_per_sm_v[variant] > 0, "lbm_stream_probe: shape %d does not fit",
              variant);
  LBM_TRY(launch_step(h, variant, kModeStream, h->f[h->cur], h->f[h->cur ^ 1], S(stream)));
  h->cur ^= 1;
  return LBM_OK;
}

int lbm_reinit_from_macro(lbm_handle* h, const float* rho_d, const float* ux_d,
                          const float* uy_d, int neq_mode, void* stream) {
  LBM_REQUIRE(h != nullptr && rho_d && ux_d && uy_d, "lbm_reinit_from_macro: bad arguments");
  int v = 0;  // the tiles of the step-kernel shape with kReinitRows rows
  while (v < LBM_STEP_VARIANTS && kStepVariants[v].ty != kReinitRows) ++v;
  LBM_REQUIRE(v < LBM_STEP_VARIANTS, "lbm_reinit_from_macro: no tile table of %d rows",
              kReinitRows);
  h->steps = 0;
  return reinit_launch(h, h->tiles_d[v], h->ntiles_v[v], rho_d, ux_d, uy_d, neq_mode, S(stream));
}

int lbm_vorticity(lbm_handle* h, const float* ux_d, const float* uy_d, float* omega_d,
                  void* stream) {
  LBM_REQUIRE(h != nullptr && ux_d && uy_d && omega_d, "lbm_vorticity: bad arguments");
  k_vorticity<<<h->nblk_total, kBlock, 0, S(stream)>>>(h->gd_d, h->ngrids, h->mask, ux_d, uy_d,
                                                       omega_d);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int lbm_export_f(lbm_handle* h, float* g_d, void* stream) {
  LBM_REQUIRE(h != nullptr && g_d != nullptr, "lbm_export_f: bad arguments");
  k_export<<<h->nblk_total, kBlock, 0, S(stream)>>>(h->gd_d, h->ngrids, h->mask, h->f[h->cur],
                                                    g_d);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int lbm_set_state(lbm_handle* h, const float* gstar_d, void* stream) {
  LBM_REQUIRE(h != nullptr && gstar_d != nullptr, "lbm_set_state: bad arguments");
  k_copy_state<<<h->nblk_total, kBlock, 0, S(stream)>>>(h->gd_d, h->ngrids, h->f[h->cur],
                                                        const_cast<float*>(gstar_d), 0);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int lbm_get_state(lbm_handle* h, float* gstar_d, void* stream) {
  LBM_REQUIRE(h != nullptr && gstar_d != nullptr, "lbm_get_state: bad arguments");
  k_copy_state<<<h->nblk_total, kBlock, 0, S(stream)>>>(h->gd_d, h->ngrids, h->f[h->cur],
                                                        gstar_d, 1);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int lbm_autotune(lbm_handle* h, int reps, float* ms_h, int* chosen_h, void* stream) {
  LBM_REQUIRE(h != nullptr && reps >= 1, "lbm_autotune: bad arguments");
  cudaStream_t s = S(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LBM_CHECK_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    set_error("lbm_autotune: cudaEventCreate failed");
    return LBM_ERR_CUDA;
  }
  // timing launches read the current state and overwrite only the other buffer,
  // which the next step overwrites anyway: the simulation state is unchanged
  const float* src = h->f[h->cur];
  float* scratch = h->f[h->cur ^ 1];
  int best = h->variant;
  float best_ms = INFINITY;
  int rc = LBM_OK;
  for (int v = 0; v < LBM_STEP_VARIANTS && rc == LBM_OK; ++v) {
    float ms = INFINITY;
    if (h->blocks_per_sm_v[v] > 0) {
      for (int w = 0; w < 2 && rc == LBM_OK; ++w) rc = launch_step(h, v, kModeStep, src, scratch, s);
      if (rc == LBM_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = LBM_ERR_CUDA;
      for (int k = 0; k < reps && rc == LBM_OK; ++k) rc = launch_step(h, v, kModeStep, src, scratch, s);
      if (rc == LBM_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                           cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = LBM_ERR_CUDA;
      ms /= (float)reps;
    }
    if (ms_h) ms_h[v] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LBM_OK) {
    if (rc == LBM_ERR_CUDA) set_error("lbm_autotune: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  h->variant = best;
  if (chosen_h) *chosen_h = best;
  return LBM_OK;
}

int lbm_set_step_variant(lbm_handle* h, int variant) {
  LBM_REQUIRE(h != nullptr && variant >= 0 && variant < LBM_STEP_VARIANTS,
              "lbm_set_step_variant: bad arguments");
  LBM_REQUIRE(h->blocks_per_sm_v[variant] > 0, "lbm_set_step_variant: shape %d does not fit",
              variant);
  h->variant = variant;
  return LBM_OK;
}

int lbm_get_step_variant(const lbm_handle* h, int* variant_h, int* rows_per_tile_h,
                         int* stages_h, int* ctas_per_sm_h) {
  LBM_REQUIRE(h != nullptr, "lbm_get_step_variant: null handle");
  const StepVariant& sv = kStepVariants[h->variant];
  if (variant_h) *variant_h = h->variant;
  if (rows_per_tile_h) *rows_per_tile_h = sv.ty;
  if (stages_h) *stages_h = sv.stages;
  if (ctas_per_sm_h) *ctas_per_sm_h = h->blocks_per_sm_v[h->variant];
  return LBM_OK;
}

int lbm_steps_done(const lbm_handle* h, long long* out_h) {
  LBM_REQUIRE(h != nullptr && out_h != nullptr, "lbm_steps_done: bad arguments");
  *out_h = h->steps;
  return LBM_OK;
}

int lbm_destroy(lbm_handle* h) {
  delete h;
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Residual statistics without caller-provided scratch memory.
//
// lbm_residual keeps its FP32 row-segment partials, FP64 block sums and per-grid
// sums in the workspace the caller allocated for lbm_init.  Some callers cannot
// allocate device memory when they want these statistics: for example a host program
// whose device memory is entirely handed out by another allocator (a framework's
// caching allocator that already owns the budget), or a runtime that forbids device
// allocation once it has started.  lbm_residual_static gives them the same numbers
// with the scratch held in a fixed array compiled into this library.
//
// The array is file-scope device memory of kResidualStaticBytes; every GPU that
// loads the library holds it until the process exits.  Host code may not use the
// array's name as a device address, so every call looks the address up with
// cudaGetSymbolAddress for the device that is current (a lookup allocates nothing;
// looking it up every call also stays correct after the context has been destroyed
// and created again, when the module, and with it the array, is loaded anew).
// Every call shares the array and it keeps the previous call's contents: every slot
// a call reads is written by that call first (each row segment's partial by the
// step kernel, each block sum by the first reduction stage, each grid sum by the
// second), so nothing has to start at zero.  Calls whose kernels overlap on the
// GPU (two streams, two threads) race on the array.
// ---------------------------------------------------------------------------
namespace lbmfno {
constexpr size_t kResidualStaticBytes = 4u << 20;  // 4 MiB
static __device__ __align__(256) unsigned char g_residual_static[kResidualStaticBytes];
}  // namespace lbmfno

extern "C" int lbm_residual_static(lbm_handle* h, double* out_h, int update_prev, void* stream) {
  LBM_REQUIRE(h != nullptr && out_h != nullptr, "lbm_residual_static: bad arguments");
  const size_t need = stats_scratch(h->nrblk_total, h->ngrids).total;
  LBM_REQUIRE(need <= kResidualStaticBytes,
              "lbm_residual_static: batch needs %zu bytes of scratch, the static array holds "
              "%zu (at most about %zu row segments of 128 cells); use lbm_residual",
              need, kResidualStaticBytes,
              kResidualStaticBytes / (kSegStride * sizeof(float) + R_COUNT * sizeof(double) /
                                                                       kSegsPerRblk));
  void* base = nullptr;
  LBM_CHECK_CUDA(cudaGetSymbolAddress(&base, g_residual_static));
  return residual_run(h, kModeStats, static_cast<char*>(base), out_h, update_prev, S(stream),
                      "lbm_residual_static");
}
