// Shared device/host helpers of the lbmfno library (status handling, D2Q9
// constants, per-grid metadata).  Used only by the CUDA path.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/lbmfno.h"

namespace lbmfno {

// ---------------------------------------------------------------- status ---
void set_error(const char* fmt, ...);

#define LBM_CHECK_CUDA(expr)                                                       \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ::lbmfno::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,               \
                          cudaGetErrorString(e_));                                 \
      return LBM_ERR_CUDA;                                                         \
    }                                                                              \
  } while (0)

#define LBM_REQUIRE(cond, ...)                                                     \
  do {                                                                             \
    if (!(cond)) {                                                                 \
      ::lbmfno::set_error(__VA_ARGS__);                                            \
      return LBM_ERR_INVALID_ARG;                                                  \
    }                                                                              \
  } while (0)

#define LBM_CHECK_LAUNCH()                                                         \
  do {                                                                             \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess) {                                                       \
      ::lbmfno::set_error("%s:%d kernel launch: %s", __FILE__, __LINE__,           \
                          cudaGetErrorString(e_));                                 \
      return LBM_ERR_CUDA;                                                         \
    }                                                                              \
  } while (0)

#define LBM_TRY(expr)              \
  do {                             \
    int s_ = (expr);               \
    if (s_ != LBM_OK) return s_;   \
  } while (0)

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ------------------------------------------------------------- lattice ---
// D2Q9: i = 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
constexpr int kQ = 9;
constexpr float kW0 = 4.0f / 9.0f;
constexpr float kW1 = 1.0f / 9.0f;
constexpr float kW2 = 1.0f / 36.0f;

__host__ __device__ constexpr int cx_of(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int i) {
  return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
__host__ __device__ constexpr float w_of(int i) { return i == 0 ? kW0 : (i <= 4 ? kW1 : kW2); }

// ----------------------------------------------------------- per grid ---
// Metadata of one lattice in a batch, resident in device memory.
struct GridDev {
  int nx, ny;
  int pitch;        // floats between rows of a population plane (multiple of 32)
  int wpr;          // mask words per row = ceil(nx/32)
  long long f_off;  // offset (floats) of the grid's first row inside each population plane
  long long plane;  // floats per population plane of the batch (every grid's rows)
  long long mask_off;
  long long cell_off;  // offset of the grid in dense fields
  int blk_start;       // first block of the grid in flat 256-cell block launches
  int nblk;            // blocks of the grid
  int nseg;            // 128-cell row segments per row (step kernel)
  int rblk_start;      // first block of the grid in the statistics reduction (each
                       // block sums kSegsPerRblk row-segment partials)
  int nrblk;           // statistics-reduction blocks of the grid
  float omega;         // 1 / tau
  float tau;
  float guo;           // 1 - 1/(2 tau)
  float fx, fy;
  int periodic_x;
  int bc_west, bc_east;
  float west_d;  // west: rho - 1 (pressure) or u_x (velocity)
  float east_d;
};

constexpr int kBlock = 256;  // threads per block of the flat cell launches
// Row segments (128 cells) whose statistics partials one reduction block sums; a
// grid's segment (y, s) has partial slot rblk_start * kSegsPerRblk + y * nseg + s.
constexpr int kSegsPerRblk = 4 * kBlock;

// Grid of a block index: binary search over a per-grid prefix of first blocks.
template <int GridDev::*START>
__device__ __forceinline__ int grid_of(const GridDev* __restrict__ grids, int ngrids, int blk) {
  int lo = 0, hi = ngrids - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&(grids[mid].*START)) <= blk)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int grid_of_block(const GridDev* __restrict__ grids, int ngrids,
                                             int blk) {
  return grid_of<&GridDev::blk_start>(grids, ngrids, blk);
}

__device__ __forceinline__ int mask_bit(const uint32_t* __restrict__ m, int wpr, int x, int y) {
  return (__ldg(&m[(size_t)y * wpr + (x >> 5)]) >> (x & 31)) & 1u;
}

}  // namespace lbmfno
