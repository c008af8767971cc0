// Tensor-core (tcgen05) path of the FNO forward pass (Sec. 2.2 of arXiv 2604.27158).
//
// Latent field layout ("channel-blocked"): theta[b][y][c/8][x][c%8] bfloat16, so a
// run of x positions of one 8-channel group is contiguous and every operand tile
// is a set of contiguous 128-byte core matrices (no swizzle).
//
// One Fourier layer  theta' = act(W theta + F^-1(R . F(theta)) + bias):
//  1. k_fwd_x_tc   X1[b][y][kx][c] = sum_x theta[x][c] e^{-2 pi i kx x / W}
//                  tcgen05: D[(row, c)][kx re|im] = A[(row, c)][x] * Fw[x][kx re|im]
//                  (M = 128 = 128/C rows x C channels, N = 32, K = W; A MN-major)
//  2. k_ydft_tc    Xh[a, kx][b][c] = sum_y X1[b][y][kx][c] e^{-2 pi i ky(a) y / H}
//                  tcgen05: D[(kx, c)][(a, re|im)] = X1b[(kx, c)][(y, re|im)] * Fy
//                  (M = 128, N = 4m rounded up to 16, K = 2H; X1 carried in bfloat16)
//  3. k_mix4 / k_mix  per mode: Y[b][o] = sum_c Xh[b][c] R[c][o] (CUDA cores, FP32),
//                  written as the bfloat16 operand Yb of the inverse y-DFT (k_mix4: a
//                  block per group of four modes sharing Yb's 16-byte entries, C <= 32)
//     k_iydft_tc   Zt[b][y][k'/8][o][k'%8] = Ty[y][(a, re|im)] * Yb[(a, re|im)][(k', o)]
//                  (k' < m real parts, m <= k' < 2m imaginary parts, M = 128 rows y)
//  4. k_inv_x_tc   theta'[x][o] = act( sum_k' T[x][k'] Zt[k'][o] + sum_i theta[x][i] W[o][i] + b[o] )
//                  tcgen05: D[x][o] = [T | theta][x][k] * [Zt ; W^T][k][o]
//                  (M = 128 x positions, N = C, K = K2 + C; both operands K-major;
//                  the CTA's slice of T and W^T stay in shared memory; for C <= 32
//                  a tile covers several grid rows, side by side in the accumulator)
// T folds 1/(H W) and the real-input inverse weights (1 for kx = 0, 2 otherwise).
// Around the layers: k_lift_tc (layer 1 of P on CUDA cores in producer warps, layer 2 as
// MMAs) and k_decoder_tc (Q1 as an MMA, activation and Q2 in the epilogue).
//
// The layer and projection kernels are persistent and warp-specialised: epilogue warps
// (four, or two groups of four that take alternate tiles) drain the TMEM accumulators,
// one producer warp streams operand tiles with cp.async.bulk into a ring of
// shared-memory stages, one warp issues the MMAs.  Two TMEM accumulators let the
// epilogue of one tile overlap the MMAs of the next.  Every wait is bounded (the
// waiting warp suspends in try_wait) and records a timeout in the status word.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "fno_tc.cuh"
#include "gelu.cuh"
#include "sm100.cuh"

namespace lbmfno {

// Programmatic dependent launch across the kernels of one forward (and from one forward
// to the next): every kernel lets its successor be scheduled as soon as it has started
// (pdl_trigger) and waits for its predecessor to complete, with its memory visible, before
// it reads or writes any buffer a predecessor uses (pdl_wait).  What runs in between is
// set-up that touches only this kernel's shared memory, TMEM and the read-only
// parameters, and it overlaps the predecessor's tail.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ float act_tc(float v, int act) {
  return act == FNO_ACT_GELU ? gelu_poly(v) : fmaxf(v, 0.0f);
}
template <int kAct>
__device__ __forceinline__ float act_c(float v) {
  return kAct == FNO_ACT_GELU ? gelu_poly(v) : fmaxf(v, 0.0f);
}
template <int kAct>
__device__ __forceinline__ float2 act_c2(float2 v) {
  return kAct == FNO_ACT_GELU ? gelu_poly2(v) : make_float2(fmaxf(v.x, 0.0f), fmaxf(v.y, 0.0f));
}
__device__ __forceinline__ int kept_ky_tc(int a, int H, int m) { return a < m ? a : H - 2 * m + a; }

// ------------------------------------------------------------------ tables
// Grid sizes of the tensor-core path.  The Fourier layers run on the (padded) grid
// Hv x Wv (the input grid plus the padding); the latent field is stored on Hs x Ws
// (Hs = Hv rounded up to 8 rows, Ws = Wv rounded up to 64 columns; the lift and the
// inverse x-DFT work in tiles of 128 columns, the last of which may cover storage columns
// Ws .. +63 that do not exist: their loads read the workspace that follows, their results
// are not stored).  Every DFT table
// uses the true periods Hv and Wv and is zero on the storage padding, and the storage
// padding of the latent field is kept at zero, so the contractions over the padded
// extents equal the DFTs of the Hv x Wv grid.  K2: the kept x-frequencies as MMA
// columns, 2m rounded up to 32 or 64.
struct TcGrid {
  int H0, W0;  // input / output grid
  int Hv, Wv;  // grid of the Fourier layers (H0 + padding, W0 + padding)
  int Hs, Ws;  // storage of the latent field
};
__host__ __device__ inline int tc_k2(int m) { return 2 * m <= 32 ? 32 : 64; }

// Fw[x/8][n][x%8] (n < K2): n < K2/2: cos(2 pi n x / Wv) for n < m; K2/2 <= n: -sin(2 pi
// (n - K2/2) x / Wv) for n - K2/2 < m; 0 elsewhere and for x >= Wv.
__device__ void table_fw(int t, __nv_bfloat16* __restrict__ fw, int Wv, int m, int k2) {
  const int xl = t & 7, n = (t >> 3) % k2, xh = (t >> 3) / k2;
  const int x = xh * 8 + xl;
  const int k = n < k2 / 2 ? n : n - k2 / 2;
  float v = 0.0f;
  if (k < m && x < Wv) {
    float s, c;
    sincospif(2.0f * (float)((long long)k * x % Wv) / (float)Wv, &s, &c);
    v = n < k2 / 2 ? c : -s;
  }
  fw[t] = __float2bfloat16_rn(v);
}
// Ti[k'/8][x][k'%8] (k' < K2, x < Ws): k' < m: c_k cos(2 pi k' x / Wv) / (Hv Wv);
// m <= k' < 2m: -c_k sin(2 pi (k'-m) x / Wv) / (Hv Wv); else 0, and 0 for x >= Wv;
// c_0 = 1, c_k = 2 (k > 0).
__device__ void table_ti(int t, __nv_bfloat16* __restrict__ ti, int Hv, int Wv, int Ws, int m) {
  const int kl = t & 7, x = (t >> 3) % Ws, kh = (t >> 3) / Ws;
  const int kp = kh * 8 + kl;
  float v = 0.0f;
  if (kp < 2 * m && x < Wv) {
    const int k = kp < m ? kp : kp - m;
    float s, c;
    sincospif(2.0f * (float)((long long)k * x % Wv) / (float)Wv, &s, &c);
    const float w = (k == 0 ? 1.0f : 2.0f) / ((float)Hv * (float)Wv);
    v = kp < m ? w * c : -w * s;
  }
  ti[t] = __float2bfloat16_rn(v);
}
// Sizes of the spectral stage.  The forward y-DFT's N (= the inverse y-DFT's K) runs
// over (a, re|im) for the 2m kept ky, rounded up to a multiple of 16; the inverse's N
// runs over (k', o) in chunks of knk consecutive k' (8, or 4 for C = 64 so that a
// chunk is at most 256 accumulator columns).
struct SpecDims {
  int nf;      // 4m rounded up to 16
  int kg;      // nf / 8: K groups of the inverse y-DFT
  int knk;     // k' per inverse N chunk
  int nc;      // inverse N chunks: ceil(2m / knk)
  int nchunk;  // columns per inverse chunk: knk * C
  int nn;      // nc * nchunk
};
__host__ __device__ inline SpecDims spec_dims(int C, int m) {
  SpecDims d;
  d.nf = (4 * m + 15) / 16 * 16;
  d.kg = d.nf / 8;
  d.knk = C <= 32 ? 8 : 4;
  d.nc = (2 * m + d.knk - 1) / d.knk;
  d.nchunk = d.knk * C;
  d.nn = d.nc * d.nchunk;
  return d;
}
// Fy[y/4][n][(y%4) * 2 + p], n = 2a + q: the real form of e^{-2 pi i ky(a) y / Hv} that
// maps the pair (Re, Im) (p) of X1[y] to (Re, Im) (q) of the kept mode a; 0 for a >= 2m
// and for y >= Hv.
__device__ void table_fy(int t, __nv_bfloat16* __restrict__ fy, int Hv, int m, int nf) {
  const int j = t & 7, n = (t >> 3) % nf, yg = (t >> 3) / nf;
  const int y = yg * 4 + (j >> 1), p = j & 1, a = n >> 1, q = n & 1;
  float v = 0.0f;
  if (a < 2 * m && y < Hv) {
    float sn, cs;
    sincospif(2.0f * (float)((long long)kept_ky_tc(a, Hv, m) * y % Hv) / (float)Hv, &sn, &cs);
    v = p == 0 ? (q == 0 ? cs : -sn) : (q == 0 ? sn : cs);
  }
  fy[t] = __float2bfloat16_rn(v);
}
// Ty[a/4][y][(a%4) * 2 + p]: cos (p = 0) and sin (p = 1) of 2 pi ky(a) y / Hv for the
// inverse y-DFT; rows padded to hp (a multiple of 128) and a >= 2m are 0.
__device__ void table_ty(int t, __nv_bfloat16* __restrict__ ty, int Hv, int hp, int m, int kg) {
  const int j = t & 7, y = (t >> 3) % hp, g = (t >> 3) / hp;
  const int a = g * 4 + (j >> 1), p = j & 1;
  float v = 0.0f;
  if (a < 2 * m && y < Hv) {
    float sn, cs;
    sincospif(2.0f * (float)((long long)kept_ky_tc(a, Hv, m) * y % Hv) / (float)Hv, &sn, &cs);
    v = p == 0 ? cs : sn;
  }
  ty[t] = __float2bfloat16_rn(v);
}

// All four DFT tables of one forward in one launch (FP32 sines and cosines of exactly
// reduced integer phases; the tables are stored in bfloat16).
__global__ void k_tables(__nv_bfloat16* __restrict__ fw, __nv_bfloat16* __restrict__ ti,
                         __nv_bfloat16* __restrict__ fy, __nv_bfloat16* __restrict__ ty,
                         TcGrid g, int m, int hp, int nf, int kg) {
  pdl_trigger();
  pdl_wait();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int k2 = tc_k2(m);
  const int n_fw = g.Ws * k2, n_fy = (g.Hs / 4) * nf * 8, n_ty = kg * hp * 8;
  if (t < n_fw) return table_fw(t, fw, g.Wv, m, k2);
  t -= n_fw;
  if (t < n_fw) return table_ti(t, ti, g.Hv, g.Wv, g.Ws, m);
  t -= n_fw;
  if (t < n_fy) return table_fy(t, fy, g.Hv, m, nf);
  t -= n_fy;
  if (t < n_ty) return table_ty(t, ty, g.Hv, hp, m, kg);
}

// ---------------------------------------------------- lifting / projection
// Lifting network P on the tensor cores: layer 1 ((c_in + 2) -> C/2, activation) on
// CUDA cores with one thread per pixel, its outputs rounded to bfloat16 into the K-major
// A operand in shared memory; layer 2 (C/2 -> C) as one tcgen05 MMA per 128-pixel tile
// (M = 128 x positions of one row, N = C, K = C/2 padded to 16) with the bias added in
// the epilogue.  Warp-specialised: four producer warps compute layer 1 of successive
// tiles into a ring of A stages, one warp issues the MMAs into two TMEM accumulators,
// four epilogue warps drain them — no CTA-wide barrier in the loop.
// The tiles cover the storage grid Hs x Ws: pixels outside the input grid H0 x W0 (the
// zero padding of the lifted field and the storage padding) are written as 0 without an
// MMA, and rows y >= Hv of the second latent buffer `theta_alt` are zeroed too (no layer
// writes them).
// The tiles t = t0, t0 + G, t0 + 2G, ... (G = gridDim.x) of a (b, y, x tile) raster with
// xt tiles a row and Hs rows an image, stepped without a division per tile.
struct TileWalk {
  int xt, Hs, dq, dr, dy0, dy1, db0, db1;  // a step moves dq (+1 on a carry) rows
  int t, row, b, y, xi;
  __device__ TileWalk(int t0, int xt_, int Hs_) : xt(xt_), Hs(Hs_), t(t0) {
    dq = gridDim.x / xt;
    dr = gridDim.x - dq * xt;
    dy0 = dq % Hs;
    db0 = dq / Hs;
    dy1 = (dq + 1) % Hs;
    db1 = (dq + 1) / Hs;
    row = t0 / xt;
    xi = t0 - row * xt;
    b = row / Hs;
    y = row - b * Hs;
  }
  __device__ void next() {
    t += gridDim.x;
    xi += dr;
    const bool c = xi >= xt;
    if (c) xi -= xt;
    row += dq + (c ? 1 : 0);
    y += c ? dy1 : dy0;
    b += c ? db1 : db0;
    if (y >= Hs) {
      y -= Hs;
      ++b;
    }
  }
};
constexpr int kLiftStages = 4;
constexpr int kLiftInStages = 6;  // input ring (dynamic shared memory, cin x 512 B a stage)
constexpr int kLiftThreads = 9 * 32;  // warps 0-3 producer, 4 MMA, 5-8 epilogue
// three CTAs per SM; two for width 64 with a runtime input width (the producers then hold
// 16 input channels and their prefetch, which would spill at three)
constexpr int lift_ctas_per_sm(int cin, int C) { return cin > 0 || C < 64 ? 3 : 2; }
// Grid rows a tile: two for C = 16 (the second row fills the other 16 columns of the
// 32-column accumulator, halving the tiles' fixed costs), else one (two rows of a wider
// latent spill the producers at this occupancy).
__host__ __device__ constexpr int lift_rows(int C) { return C == 16 ? 2 : 1; }
template <int kC, int kCin, int kAct>
__global__ void __launch_bounds__(kLiftThreads, lift_ctas_per_sm(kCin, kC))
    k_lift_tc(const float* __restrict__ in, __nv_bfloat16* __restrict__ theta,
              __nv_bfloat16* __restrict__ theta_alt, const float* __restrict__ w0,
              const float* __restrict__ b0, const float* __restrict__ w1,
              const float* __restrict__ b1, int B, TcGrid gd, int cin_rt,
              unsigned* __restrict__ status) {
  pdl_trigger();
  constexpr int kHid = kC / 2;
  constexpr int kK = kHid < 16 ? 16 : kHid;  // MMA K (zero-padded hidden units)
  constexpr int kKG = kK / 8;
  constexpr int kX = kCin > 0 ? kCin + 2 : 18;  // inputs and the two coordinates
  constexpr int kR = lift_rows(kC);  // grid rows a tile
  constexpr int kAccCols = kR * kC < 32 ? 32 : kR * kC;  // the rows side by side
  const int cin = kCin > 0 ? kCin : cin_rt;
  const int cin2 = cin + 2;
  __shared__ __align__(1024) unsigned char a_s[kLiftStages][kR][kKG * 2048];  // [k group][x][8]
  __shared__ __align__(1024) unsigned char b_s[kKG * kC * 16];  // W1^T: [k group][o][8]
  __shared__ float2 w0p_s[(kHid / 2) * 18];  // (w0[j][c], w0[j+1][c]) for hidden pairs
  __shared__ __align__(16) float b0_s[kHid], b1_s[kC];
  __shared__ __align__(8) uint64_t a_full[kLiftStages], a_empty[kLiftStages];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  extern __shared__ __align__(16) float in_s[];  // [kLiftInStages][kR rows][cin][128 pixels]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < kKG * kC * 8; e += blockDim.x) {
    const int g = e / (kC * 8), o = (e / 8) % kC, il = e % 8, j = g * 8 + il;
    reinterpret_cast<__nv_bfloat16*>(b_s)[e] = __float2bfloat16_rn(j < kHid ? w1[o * kHid + j] : 0.f);
  }
  for (int e = threadIdx.x; e < (kHid / 2) * cin2; e += blockDim.x) {
    const int jp = e / cin2, c = e - jp * cin2;
    w0p_s[e] = make_float2(w0[(2 * jp) * cin2 + c], w0[(2 * jp + 1) * cin2 + c]);
  }
  for (int j = threadIdx.x; j < kHid; j += blockDim.x) b0_s[j] = b0[j];
  for (int o = threadIdx.x; o < kC; o += blockDim.x) b1_s[o] = b1[o];
  if (kHid < kK)  // padded hidden units stay zero
    for (int e = threadIdx.x; e < kLiftStages * kR * 128 * 8; e += blockDim.x)
      reinterpret_cast<__nv_bfloat16*>(&a_s[0][0][0] + (size_t)(e / 1024) * kKG * 2048 +
                                       2048)[e % 1024] = __float2bfloat16_rn(0.f);
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kLiftStages; ++s) {
      mbar_init(&a_full[s], 4);
      mbar_init(&a_empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
    }
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_base, 2 * kAccCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // everything below may touch buffers of the previous kernels
  const uint32_t tmem = tmem_base;
  const int H = gd.H0, W = gd.W0, Hs = gd.Hs, Ws = gd.Ws;
  const int xt = (Ws + 127) / 128;
  const int Hp = Hs / kR;  // row groups an image (Hs is a multiple of 8)
  const int ntiles = B * Hp * xt;
  // CTA-uniform: the whole tile is padding (no MMA); TileWalk rows are row groups
  auto is_pad = [&](const TileWalk& w) { return w.y * kR >= H || w.xi * 128 >= W; };

  if (warp < 4) {
    // ---------------------------------------------------------- producers
    // inputs of the next kLiftInStages - 1 tiles in flight: each thread copies and later
    // reads only its own pixel's channels, so the per-thread commit groups order them
    constexpr int kCinR = kCin > 0 ? kCin : 16;
    TileWalk ahead(blockIdx.x, xt, Hp);
    auto issue = [&](int i) {  // the CTA's i-th tile, at `ahead`
      const int xx = ahead.xi * 128 + threadIdx.x;
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const int yy = ahead.y * kR + r;
        const bool ok = ahead.t < ntiles && yy < H && xx < W;
        const float* src = ok ? in + (((size_t)ahead.b * cin) * H + yy) * W + xx : in;
        float* dst = in_s + ((size_t)(i % kLiftInStages) * kR + r) * (cin * 128) + threadIdx.x;
#pragma unroll
        for (int c = 0; c < kCinR; ++c)
          if (c < cin) cp_async4(dst + c * 128, ok ? src + (size_t)c * H * W : in, ok ? 4u : 0u);
      }
      cp_async_commit();
      ahead.next();
    };
#pragma unroll 1
    for (int i = 0; i < kLiftInStages - 1; ++i) issue(i);
    int k = 0, i = 0;
    for (TileWalk w(blockIdx.x, xt, Hp); w.t < ntiles; w.next(), ++i) {
      const int y0 = w.y * kR, x = w.xi * 128 + threadIdx.x;
      issue(i + kLiftInStages - 1);  // its stage was last read in iteration i - 1
      cp_async_wait<kLiftInStages - 1>();
      if (is_pad(w)) {
        if (x < Ws) {
#pragma unroll
          for (int r = 0; r < kR; ++r)
#pragma unroll
            for (int g = 0; g < kC / 8; ++g) {
              const size_t at = (((size_t)(w.row * kR + r) * (kC / 8) + g) * Ws + x) * 8;
              *reinterpret_cast<uint4*>(theta + at) = make_uint4(0, 0, 0, 0);
              if (y0 + r >= gd.Hv)
                *reinterpret_cast<uint4*>(theta_alt + at) = make_uint4(0, 0, 0, 0);
            }
        }
        continue;
      }
      const int s = k % kLiftStages;
      if (k >= kLiftStages && !mbar_wait_sleep(&a_empty[s], ((k / kLiftStages) - 1) & 1, status))
        break;
#pragma unroll 1
      for (int r = 0; r < kR; ++r) {
      const int y = y0 + r;
      const float* cur =
          in_s + ((size_t)(i % kLiftInStages) * kR + r) * cin * 128 + threadIdx.x;
      // layer 1 for this thread's pixel (inputs and coordinates rounded to bfloat16)
      const float xc = (float)x / (float)max(W - 1, 1), yc = (float)y / (float)max(H - 1, 1);
      float xin[kX];  // inputs then the two coordinates, all indices compile-time
#pragma unroll
      for (int c = 0; c < kX; ++c) {
        const float v = c < kCinR && c < cin ? cur[(c < kCinR ? c : 0) * 128]  // 0 off the grid
                        : c == cin           ? xc
                        : c == cin + 1       ? yc
                                             : 0.0f;
        xin[c] = __bfloat162float(__float2bfloat16_rn(v));
      }
#pragma unroll
      for (int g = 0; g < kHid / 8; ++g) {  // eight hidden units at a time into the A stage
        __align__(16) __nv_bfloat16 h[8];
#pragma unroll
        for (int jq = 0; jq < 4; ++jq) {
          const int jp = g * 4 + jq;
          float2 a = *reinterpret_cast<const float2*>(&b0_s[2 * jp]);
#pragma unroll
          for (int c = 0; c < kX; ++c)
            if (c < cin2) a = __ffma2_rn(w0p_s[jp * cin2 + c], make_float2(xin[c], xin[c]), a);
          const float2 r = act_c2<kAct>(a);
          h[2 * jq] = __float2bfloat16_rn(r.x);
          h[2 * jq + 1] = __float2bfloat16_rn(r.y);
        }
        *reinterpret_cast<uint4*>(a_s[s][r] + g * 2048 + threadIdx.x * 16) =
            *reinterpret_cast<const uint4*>(h);
      }
      }  // rows of the tile
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&a_full[s]);
      ++k;
    }
    cp_async_wait<0>();  // the zero-filled copies issued past the last tile
  } else if (warp == 4) {
    // --------------------------------------------------------------- MMA
    constexpr uint32_t idesc = idesc_bf16(128, kC, false, false);
    int j = 0;
    for (TileWalk w(blockIdx.x, xt, Hp); w.t < ntiles; w.next()) {
      if (is_pad(w)) continue;
      const int s = j % kLiftStages, acc = j & 1;
      bool ok = mbar_wait_sleep(&a_full[s], (j / kLiftStages) & 1, status);
      if (ok && j >= 2) ok = mbar_wait_sleep(&acc_empty[acc], ((j >> 1) - 1) & 1, status);
      if (!ok) break;
      tc_fence_after();
      if (lane == 0) {
#pragma unroll
        for (int r = 0; r < kR; ++r)  // row r into accumulator columns r C ..
#pragma unroll
          for (int kk = 0; kk < kKG / 2; ++kk)
            mma_bf16(tmem + acc * kAccCols + r * kC, smem_desc(a_s[s][r] + kk * 4096, 2048, 128),
                     smem_desc(b_s + kk * 2 * kC * 16, kC * 16, 128), idesc, kk > 0);
        mma_commit(&a_empty[s]);
        mma_commit(&acc_full[acc]);
      }
      __syncwarp();
      ++j;
    }
  } else {
    // ----------------------------------------------------------- epilogue
    const int quad = warp & 3;  // a warp reads TMEM lanes 32 (warp % 4) .. +31: pixels x0 + 32 quad + lane
    int j = 0;
    for (TileWalk w(blockIdx.x, xt, Hp); w.t < ntiles; w.next()) {
      if (is_pad(w)) continue;
      const int acc = j & 1;
      if (!mbar_wait_sleep(&acc_full[acc], (j >> 1) & 1, status)) break;
      tc_fence_after();
      const int x = w.xi * 128 + quad * 32 + lane;
#pragma unroll
      for (int r = 0; r < kR; ++r) {
      // a row past the input grid (the second row of a tile) is zero padding
      const int row = w.row * kR + r, y = w.y * kR + r;
      const bool valid = x < W && y < H, in_storage = x < Ws;
      if (y >= gd.Hv && in_storage)
#pragma unroll
        for (int g = 0; g < kC / 8; ++g)
          *reinterpret_cast<uint4*>(theta_alt + (((size_t)row * (kC / 8) + g) * Ws + x) * 8) =
              make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int cb = 0; cb < kC / 16; ++cb) {
        float v[16];
        tmem_ld16(tmem + acc * kAccCols + r * kC + cb * 16 + ((uint32_t)(quad * 32) << 16), v);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const int o0 = cb * 16 + g * 8;
          __align__(16) __nv_bfloat16 o8[8];
#pragma unroll
          for (int q = 0; q < 8; q += 2) {
            const float2 r = __fadd2_rn(make_float2(v[g * 8 + q], v[g * 8 + q + 1]),
                                        *reinterpret_cast<const float2*>(&b1_s[o0 + q]));
            o8[q] = __float2bfloat16_rn(valid ? r.x : 0.0f);
            o8[q + 1] = __float2bfloat16_rn(valid ? r.y : 0.0f);
          }
          if (in_storage)
            *reinterpret_cast<uint4*>(theta + (((size_t)row * (kC / 8) + o0 / 8) * Ws + x) * 8) =
                *reinterpret_cast<const uint4*>(o8);
        }
      }
      }  // rows of the tile
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[acc]);
      ++j;
    }
  }
  // all MMAs of this CTA have completed once the epilogue has drained (or timed out)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 2 * kAccCols);
}

// Projection Q from the channel-blocked field, any decoder shape (the common shape
// runs in k_decoder_tc); one thread per pixel of the output grid H0 x W0 (the padded
// grid is cropped), decoder weights staged in shared memory.
template <int kC>
__global__ void __launch_bounds__(128)
    k_decoder_blk(const __nv_bfloat16* __restrict__ theta, float* __restrict__ out,
                  const float* __restrict__ params, const unsigned* __restrict__ offs,
                  int nlayers, int B, TcGrid gd, int S, int cout, int act) {
  pdl_trigger();
  pdl_wait();
  const int H = gd.H0, W = gd.W0;
  extern __shared__ float dec_s[];
  // layout: for each layer l: w [S][fan] then b [S]; then out.w [cout][fan], out.b [cout]
  int at = 0, fan = kC;
  for (int l = 0; l <= nlayers; ++l) {
    const int rows = l < nlayers ? S : cout;
    const float* w = params + offs[2 * l];
    const float* bb = params + offs[2 * l + 1];
    for (int t = threadIdx.x; t < rows * fan; t += blockDim.x) dec_s[at + t] = w[t];
    for (int t = threadIdx.x; t < rows; t += blockDim.x) dec_s[at + rows * fan + t] = bb[t];
    at += rows * fan + rows;
    fan = S;
  }
  __syncthreads();
  const size_t pix = (size_t)B * H * W;
  const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p >= pix) return;
  const int x = (int)(p % W);
  const int y = (int)((p / W) % H);
  const int b = (int)(p / ((size_t)W * H));
  const size_t row = (size_t)b * gd.Hs + y;  // storage row
  float a[kC];
#pragma unroll
  for (int g = 0; g < kC / 8; ++g) {
    const uint4 v = *reinterpret_cast<const uint4*>(theta + ((row * (kC / 8) + g) * gd.Ws + x) * 8);
    const __nv_bfloat16* hv = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
    for (int q = 0; q < 8; ++q) a[g * 8 + q] = __bfloat162float(hv[q]);
  }
  {
    float h[64], t[64];
#pragma unroll
    for (int c = 0; c < kC; ++c) h[c] = a[c];
    at = 0;
    fan = kC;
    for (int l = 0; l < nlayers; ++l) {
      const float* w = dec_s + at;
      const float* bb = w + S * fan;
      for (int j = 0; j < S; ++j) {
        float v = bb[j];
        for (int c = 0; c < fan; ++c) v = fmaf(w[j * fan + c], h[c], v);
        t[j] = act_tc(v, act);
      }
      for (int j = 0; j < S; ++j) h[j] = t[j];
      at += S * fan + S;
      fan = S;
    }
    const float* w = dec_s + at;
    const float* bb = w + cout * fan;
    for (int q = 0; q < cout; ++q) {
      float v = bb[q];
      for (int c = 0; c < fan; ++c) v = fmaf(w[q * fan + c], h[c], v);
      out[(((size_t)b * cout + q) * H + y) * W + x] = v;
    }
  }
}

// --------------------------------------------------- 1. forward x-DFT (tcgen05)
constexpr int kTcThreads = 192;  // warps 0-3 epilogue, 4 producer, 5 MMA
constexpr int kFwdChunk = 64;    // x positions per stage
constexpr int kFwdMaxStages = 6;  // stages: as many as two CTAs a multiprocessor hold
constexpr int kFwdStageBytes = 128 * kFwdChunk * 2;  // 16 KB: 128 (row, channel) x 64 x

template <int kC, int kK2>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_fwd_x_tc(const __nv_bfloat16* __restrict__ theta, const __nv_bfloat16* __restrict__ fw,
               __nv_bfloat16* __restrict__ x1b, int B, int H, int W, int m, int nst,
               unsigned* __restrict__ status) {
  pdl_trigger();
  // H, W: the storage grid Hs x Ws (the table is zero beyond the layers' grid); nst stages
  constexpr int kRows = 128 / kC;  // image rows per tile
  constexpr int kG = kC / 8;       // 8-channel groups
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* fw_s = smem;                                // W * kK2 * 2 bytes
  unsigned char* stages = smem + (size_t)W * kK2 * 2;        // nst * 16 KB
  __shared__ __align__(8) uint64_t full_bar[kFwdMaxStages], empty_bar[kFwdMaxStages];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], fw_bar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ytiles = (H + kRows - 1) / kRows;
  const int ntiles = B * ytiles;
  const int nchunks = W / kFwdChunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
    }
    mbar_init(&fw_bar, 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_base, 2 * kK2);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // everything below may touch buffers of the previous kernels
  const uint32_t tmem = tmem_base;

  if (warp == 4) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      mbar_arrive_expect_tx(&fw_bar, (unsigned)(W * kK2 * 2));
      bulk_g2s(fw_s, fw, (unsigned)(W * kK2 * 2), &fw_bar);
    }
    __syncwarp();
    int k = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int b = t / ytiles, y0 = (t - b * ytiles) * kRows;
      const int rows = min(kRows, H - y0);
      for (int ch = 0; ch < nchunks; ++ch, ++k) {
        const int s = k % nst;
        if (k >= nst) ok = mbar_wait_sleep(&empty_bar[s], ((k / nst) - 1) & 1, status);
        if (!ok) break;
        unsigned char* st = stages + (size_t)s * kFwdStageBytes;
        if (lane == 0) mbar_arrive_expect_tx(&full_bar[s], (unsigned)(rows * kG * kFwdChunk * 16));
        __syncwarp();
        for (int q = lane; q < rows * kG; q += 32) {
          const int r = q / kG, g = q - r * kG;
          const __nv_bfloat16* src =
              theta + ((((size_t)b * H + y0 + r) * kG + g) * W + (size_t)ch * kFwdChunk) * 8;
          bulk_g2s(st + (size_t)q * kFwdChunk * 16, src, kFwdChunk * 16, &full_bar[s]);
        }
      }
    }
    // no copy may still be in flight when the CTA exits
    mbar_wait_sleep(&fw_bar, 0, status);
    for (int q = max(0, k - nst); q < k; ++q)
      mbar_wait_sleep(&full_bar[q % nst], (q / nst) & 1, status);
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA
    constexpr uint32_t idesc = idesc_bf16(128, kK2, /*a_mn=*/true, /*b_mn=*/false);
    bool ok = mbar_wait_sleep(&fw_bar, 0, status);
    int k = 0, j = 0;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++j) {
      const int acc = j & 1;
      if (j >= 2) ok = mbar_wait_sleep(&acc_empty[acc], ((j >> 1) - 1) & 1, status);
      if (!ok) break;
      tc_fence_after();
      for (int ch = 0; ch < nchunks; ++ch, ++k) {
        const int s = k % nst;
        ok = mbar_wait_sleep(&full_bar[s], (k / nst) & 1, status);
        if (!ok) break;
        tc_fence_after();
        if (lane == 0) {
          const unsigned char* st = stages + (size_t)s * kFwdStageBytes;
#pragma unroll
          for (int kk = 0; kk < kFwdChunk / 16; ++kk) {
            // A: MN-major, K-adjacent core matrices 128 B apart, MN-adjacent 1024 B
            const uint64_t ad = smem_desc(st + kk * 256, 128, kFwdChunk * 16);
            // B: K-major, K-adjacent core matrices kK2 * 16 B apart, N-adjacent 128 B
            const uint64_t bd = smem_desc(
                fw_s + (size_t)((ch * kFwdChunk + kk * 16) / 8) * (kK2 * 16), kK2 * 16, 128);
            mma_bf16(tmem + acc * kK2, ad, bd, idesc, ch > 0 || kk > 0);
          }
          mma_commit(&empty_bar[s]);  // stage reusable once these MMAs have read it
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(&acc_full[acc]);
      __syncwarp();
    }
  } else {
    // ----------------------------------------------------------- epilogue
    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      const int acc = j & 1;
      if (!mbar_wait_sleep(&acc_full[acc], (j >> 1) & 1, status)) break;
      tc_fence_after();
      float v[kK2];
#pragma unroll
      for (int q = 0; q < kK2 / 32; ++q)
        tmem_ld32(tmem + acc * kK2 + q * 32 + ((uint32_t)(warp * 32) << 16), v + q * 32);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[acc]);
      const int b = t / ytiles, y0 = (t - b * ytiles) * kRows;
      const int mi = warp * 32 + lane;  // accumulator row = r * C + c
      const int r = mi / kC, c = mi - r * kC;
      const int y = y0 + r;
      if (y < H) {
        // X1b[b][y/4][kx][c][(y%4) * 2 + re|im]: the K-major operand of the y-DFT; column
        // kx holds the cosine sum, column kK2/2 + kx the negated sine sum
        uint32_t* o = reinterpret_cast<uint32_t*>(x1b) +
                      ((((size_t)b * (H / 4) + (y >> 2)) * m) * kC + c) * 4 + (y & 3);
#pragma unroll
        for (int kx = 0; kx < kK2 / 2; ++kx) {
          if (kx < m) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[kx], v[kK2 / 2 + kx]);
            o[(size_t)kx * kC * 4] = *reinterpret_cast<const uint32_t*>(&h2);
          }
        }
      }
    }
  }
  // all MMAs of this CTA have completed once the epilogue has drained (or timed out)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 2 * kK2);
}

// ------------------------------------------------------ 2. y-DFT (tcgen05)
// Xh[a * m + kx][b][c] = sum_y X1[b][y][kx][c] e^{-2 pi i ky(a) y / H} for the 2m kept ky:
// D[(kx, c)][(a, re|im)] = X1b[(kx, c)][(y, re|im)] * Fy[(y, re|im)][(a, re|im)]
// (M = 128 (kx, c) rows of one batch item, N = nf, K = 2H; both operands K-major).
// The Fy table stays in shared memory; X1b streams through a ring of kYChunk y groups.
constexpr int kYStagesMax = 8;
constexpr int kYChunk = 8;                   // y groups of 4 rows per stage
constexpr int kYStageBytes = kYChunk * 2048;  // [group][row (128)][8]
constexpr int kYSmemMax = 200 * 1024;
// As many stages as fit next to the Fy table (a tile's whole K extent is in flight for
// the workloads' heights, so a CTA's single tile is not paced by stage round trips).
__host__ __device__ inline int ydft_stages(int Hs, int nf) {
  const int fy = ((Hs / 4) * nf * 16 + 1023) / 1024 * 1024;
  const int n = (kYSmemMax - fy) / kYStageBytes;
  return n < 2 ? 2 : (n > kYStagesMax ? kYStagesMax : n);
}

template <int kC>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_ydft_tc(const __nv_bfloat16* __restrict__ x1b, const __nv_bfloat16* __restrict__ fy,
              float2* __restrict__ xh, int B, int H, int m, unsigned* __restrict__ status) {
  pdl_trigger();
  const SpecDims d = spec_dims(kC, m);
  const int rows = m * kC;  // (kx, c) rows of one batch item
  const int mt = (rows + 127) / 128;
  const int ntiles = B * mt;
  const int ngroups = H / 4;
  const int nchunks = (ngroups + kYChunk - 1) / kYChunk;
  const unsigned fy_bytes = (unsigned)ngroups * d.nf * 16;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* fy_s = smem;
  unsigned char* stages = smem + ((fy_bytes + 1023) & ~1023u);
  const int kYStages = ydft_stages(H, d.nf);
  __shared__ __align__(8) uint64_t full_bar[kYStagesMax], empty_bar[kYStagesMax];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], fy_bar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kYStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
    }
    mbar_init(&fy_bar, 1);
    mbar_init_fence();
  }
  const int acc_cols = d.nf <= 64 ? 64 : 128;  // two accumulators of nf <= 128 columns
  if (warp == 0) tmem_alloc(&tmem_base, 2 * acc_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // everything below may touch buffers of the previous kernels
  const uint32_t tmem = tmem_base;

  if (warp == 4) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      mbar_arrive_expect_tx(&fy_bar, fy_bytes);
      bulk_g2s(fy_s, fy, fy_bytes, &fy_bar);
    }
    __syncwarp();
    int k = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int b = t / mt, m0 = (t - b * mt) * 128;
      const int nv = min(128, rows - m0);
      for (int ch = 0; ch < nchunks; ++ch, ++k) {
        const int s = k % kYStages;
        if (k >= kYStages) ok = mbar_wait_sleep(&empty_bar[s], ((k / kYStages) - 1) & 1, status);
        if (!ok) break;
        const int g0 = ch * kYChunk, gn = min(kYChunk, ngroups - g0);
        unsigned char* st = stages + (size_t)s * kYStageBytes;
        if (lane == 0) mbar_arrive_expect_tx(&full_bar[s], (unsigned)(gn * nv * 16));
        __syncwarp();
        for (int q = lane; q < gn; q += 32)
          bulk_g2s(st + q * 2048, x1b + (((size_t)b * ngroups + g0 + q) * rows + m0) * 8,
                   (unsigned)(nv * 16), &full_bar[s]);
      }
    }
    mbar_wait_sleep(&fy_bar, 0, status);
    for (int q = max(0, k - kYStages); q < k; ++q)
      mbar_wait_sleep(&full_bar[q % kYStages], (q / kYStages) & 1, status);
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA
    const uint32_t idesc = idesc_bf16(128, d.nf, false, false);
    bool ok = mbar_wait_sleep(&fy_bar, 0, status);
    int k = 0, j = 0;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++j) {
      const int acc = j & 1;
      if (j >= 2) ok = mbar_wait_sleep(&acc_empty[acc], ((j >> 1) - 1) & 1, status);
      if (!ok) break;
      tc_fence_after();
      for (int ch = 0; ch < nchunks; ++ch, ++k) {
        const int s = k % kYStages;
        ok = mbar_wait_sleep(&full_bar[s], (k / kYStages) & 1, status);
        if (!ok) break;
        tc_fence_after();
        if (lane == 0) {
          const unsigned char* st = stages + (size_t)s * kYStageBytes;
          const int g0 = ch * kYChunk, gn = min(kYChunk, ngroups - g0);
          for (int kk = 0; kk < gn / 2; ++kk) {
            const uint64_t ad = smem_desc(st + kk * 4096, 2048, 128);
            const uint64_t bd = smem_desc(fy_s + (size_t)(g0 + 2 * kk) * d.nf * 16, d.nf * 16, 128);
            mma_bf16(tmem + acc * acc_cols, ad, bd, idesc, ch > 0 || kk > 0);
          }
          mma_commit(&empty_bar[s]);
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(&acc_full[acc]);
      __syncwarp();
    }
  } else {
    // ----------------------------------------------------------- epilogue
    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      const int acc = j & 1;
      if (!mbar_wait_sleep(&acc_full[acc], (j >> 1) & 1, status)) break;
      tc_fence_after();
      const int b = t / mt, row = (t - b * mt) * 128 + warp * 32 + lane;
      const int kx = row / kC, c = row - kx * kC;
      for (int cb = 0; cb < d.nf / 16; ++cb) {
        float v[16];
        tmem_ld16(tmem + acc * acc_cols + cb * 16 + ((uint32_t)(warp * 32) << 16), v);
        if (row < rows) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int a = cb * 8 + i;
            if (a < 2 * m) xh[(((size_t)a * m + kx) * B + b) * kC + c] = make_float2(v[2 * i], v[2 * i + 1]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[acc]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 2 * acc_cols);
}

// ----------------------------------------- 3. per-mode channel mixing (CUDA cores)
// Y[b][a][kx][o] = sum_c Xh[a * m + kx][b][c] R[a * m + kx][c][o]; one block per (mode,
// batch chunk).  Y is written as the K-major B operand of the inverse y-DFT:
// Yb[b][a/4][n][(a%4) * 2 + p] with n = n(k', o) and, for k' = kx (real part of the
// inverse) (Re Y, -Im Y), for k' = m + kx (imaginary part) (Im Y, Re Y).
constexpr int kMixB = 32;
template <int kC>
__global__ void __launch_bounds__(256)
    k_mix(const float2* __restrict__ xh, const float2* __restrict__ rt,
          __nv_bfloat16* __restrict__ yb, int B, int m) {
  pdl_trigger();
  pdl_wait();
  const SpecDims d = spec_dims(kC, m);
  extern __shared__ float2 mix_s[];
  float2* r_s = mix_s;             // [c][o]
  float2* x_s = mix_s + kC * kC;   // [b][c]
  const int md = blockIdx.x;
  const int b0 = blockIdx.y * kMixB, nb = min(kMixB, B - b0);
  {  // all of this thread's loads in flight before the first shared-memory store
    constexpr int kR = (kC * kC + 255) / 256, kXn = (kMixB * kC + 255) / 256;
    float2 rv[kR], xv[kXn];
#pragma unroll
    for (int u = 0; u < kR; ++u) {
      const int t = threadIdx.x + u * 256;
      rv[u] = t < kC * kC ? rt[(size_t)md * kC * kC + t] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kXn; ++u) {
      const int t = threadIdx.x + u * 256;
      xv[u] = t < nb * kC ? xh[((size_t)md * B + b0) * kC + t] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kR; ++u)
      if (threadIdx.x + u * 256 < kC * kC) r_s[threadIdx.x + u * 256] = rv[u];
#pragma unroll
    for (int u = 0; u < kXn; ++u)
      if (threadIdx.x + u * 256 < nb * kC) x_s[threadIdx.x + u * 256] = xv[u];
  }
  __syncthreads();
  const int a = md / m, kx = md - a * m;
  auto ncol = [&](int kp, int o) { return (kp / d.knk) * d.nchunk + o * d.knk + kp % d.knk; };
  // thread: channel o and four batch items bl, bl + kBl, bl + 2 kBl, bl + 3 kBl (one read
  // of R[c][o] serves four outputs)
  constexpr int kBl = 256 / kC;
  const int o = threadIdx.x % kC;
  for (int bl0 = threadIdx.x / kC; bl0 < nb; bl0 += 4 * kBl) {
    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int i = 0; i < kC; ++i) {
      const float2 w = r_s[i * kC + o];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int bl = min(bl0 + k * kBl, nb - 1);
        const float2 xv = x_s[bl * kC + i];
        re[k] = fmaf(xv.x, w.x, fmaf(-xv.y, w.y, re[k]));
        im[k] = fmaf(xv.x, w.y, fmaf(xv.y, w.x, im[k]));
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int bl = bl0 + k * kBl;
      if (bl >= nb) break;
      uint32_t* base = reinterpret_cast<uint32_t*>(yb) +
                       ((size_t)(b0 + bl) * d.kg + a / 4) * d.nn * 4 + (a % 4);
      const __nv_bfloat162 lo = __floats2bfloat162_rn(re[k], -im[k]);
      const __nv_bfloat162 hi = __floats2bfloat162_rn(im[k], re[k]);
      base[(size_t)ncol(kx, o) * 4] = *reinterpret_cast<const uint32_t*>(&lo);
      base[(size_t)ncol(m + kx, o) * 4] = *reinterpret_cast<const uint32_t*>(&hi);
    }
  }
}

// The same mixing for C <= 32, one block per (group of four modes a = 4 g .. 4 g + 3 with
// the same kx, batch chunk): the four modes share one 16-byte entry of Yb
// ([b][a/4][n][(a%4) * 2 + p]), so a thread writes whole entries (one store where the
// per-mode kernel makes four 4-byte ones).  Modes a >= 2m of the last group get 0.  The
// batch chunk bc (<= kMixB) is chosen so that the grid covers the multiprocessors.
template <int kC>
__global__ void __launch_bounds__(256)
    k_mix4(const float2* __restrict__ xh, const float2* __restrict__ rt,
           __nv_bfloat16* __restrict__ yb, int B, int m, int bc) {
  static_assert(kC <= 32, "shared memory");
  pdl_trigger();
  pdl_wait();
  const SpecDims d = spec_dims(kC, m);
  extern __shared__ float2 mix_s[];
  float2* r_s = mix_s;                  // [q][c][o]
  float2* x_s = mix_s + 4 * kC * kC;    // [q][b][c]
  const int ag = blockIdx.x / m, kx = blockIdx.x - ag * m;  // modes a = 4 ag + q
  const int b0 = blockIdx.y * bc, nb = min(bc, B - b0);  // batch chunk bc <= kMixB
  {  // all of this thread's loads in flight before the first shared-memory store
    constexpr int kR = (4 * kC * kC + 255) / 256, kXn = (4 * kMixB * kC + 255) / 256;
    float2 rv[kR], xv[kXn];
#pragma unroll
    for (int u = 0; u < kR; ++u) {
      const int t = threadIdx.x + u * 256;
      const int q = t / (kC * kC), e = t - q * (kC * kC), a = 4 * ag + q;
      rv[u] = (t < 4 * kC * kC && a < 2 * m) ? rt[((size_t)a * m + kx) * kC * kC + e]
                                             : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kXn; ++u) {
      const int t = threadIdx.x + u * 256;
      const int q = t / (kMixB * kC), e = t - q * (kMixB * kC), a = 4 * ag + q;
      xv[u] = (t < 4 * kMixB * kC && e < nb * kC && a < 2 * m)
                  ? xh[(((size_t)a * m + kx) * B + b0) * kC + e]
                  : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kR; ++u)
      if (threadIdx.x + u * 256 < 4 * kC * kC) r_s[threadIdx.x + u * 256] = rv[u];
#pragma unroll
    for (int u = 0; u < kXn; ++u)
      if (threadIdx.x + u * 256 < 4 * kMixB * kC) x_s[threadIdx.x + u * 256] = xv[u];
  }
  __syncthreads();
  const int n_re = (kx / d.knk) * d.nchunk + kx % d.knk;            // ncol(kx, 0)
  const int n_im = ((m + kx) / d.knk) * d.nchunk + (m + kx) % d.knk;  // ncol(m + kx, 0)
  // thread: channel o of batch items bl = tid / C, + 256 / C, ...; four modes each
  for (int e = threadIdx.x; e < nb * kC; e += 256) {
    const int bl = e / kC, o = e - bl * kC;
    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int i = 0; i < kC; ++i) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 w = r_s[(q * kC + i) * kC + o];
        const float2 xv = x_s[(q * kMixB + bl) * kC + i];
        re[q] = fmaf(xv.x, w.x, fmaf(-xv.y, w.y, re[q]));
        im[q] = fmaf(xv.x, w.y, fmaf(xv.y, w.x, im[q]));
      }
    }
    // entry (b, ag, n): (a%4) * 2 + p; real part of the inverse (Re Y, -Im Y) at
    // n = ncol(kx, o), imaginary part (Im Y, Re Y) at n = ncol(m + kx, o)
    __align__(16) __nv_bfloat162 lo[4], hi[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      lo[q] = __floats2bfloat162_rn(re[q], -im[q]);
      hi[q] = __floats2bfloat162_rn(im[q], re[q]);
    }
    uint4* base = reinterpret_cast<uint4*>(yb) + ((size_t)(b0 + bl) * d.kg + ag) * d.nn;
    base[n_re + o * d.knk] = *reinterpret_cast<const uint4*>(lo);
    base[n_im + o * d.knk] = *reinterpret_cast<const uint4*>(hi);
  }
}

// ---------------------------------------------- 3b. inverse y-DFT (tcgen05)
// Zt[b][y][k'/8][o][k'%8] (bf16, kK2 slots k') = D[y][n(k', o)] = Ty[y][(a, re|im)] *
// Yb[(a, re|im)][n]: k' < m gives Re Z(kx = k'), m <= k' < 2m gives Im Z(kx = k' - m)
// with Z[kx][o] = sum_a Y[a][kx][o] e^{+2 pi i ky(a) y / H}; k' in [2m, kK2) is written
// as 0.  One tile = (b, 128 rows, one chunk of knk k'); M = 128, N = knk * C, K = nf.
// H: the layers' grid rows Hv (rows y >= Hv are not written).
constexpr int kIyStagesMax = 4;
constexpr int kIyMinSmem = 120 * 1024;  // one CTA per SM: the accumulators fill the TMEM
constexpr int kTcSmemMax = 200 * 1024;
constexpr int kTcSmemSm = 228 * 1024;  // shared memory of one multiprocessor
__host__ __device__ inline int iy_stage_bytes(int C, int m) {
  const SpecDims d = spec_dims(C, m);
  return d.kg * 2048 + d.kg * d.nchunk * 16;
}
__host__ __device__ inline int iy_stages(int C, int m) {
  const int n = kTcSmemMax / iy_stage_bytes(C, m);
  return n < kIyStagesMax ? n : kIyStagesMax;
}

constexpr int kIyEpiWarps = 8;  // two per TMEM lane quadrant, each draining half the columns
constexpr int kIyThreads = (kIyEpiWarps + 2) * 32;

template <int kC, int kK2>
__global__ void __launch_bounds__(kIyThreads, 1)
    k_iydft_tc(const __nv_bfloat16* __restrict__ ty, const __nv_bfloat16* __restrict__ yb,
               __nv_bfloat16* __restrict__ zt, int B, int H, int m,
               unsigned* __restrict__ status) {
  pdl_trigger();
  constexpr int kKnk = kC <= 32 ? 8 : 4;
  constexpr int kN = kKnk * kC;  // accumulator columns per tile (128 or 256)
  const SpecDims d = spec_dims(kC, m);
  const int hp = (H + 127) / 128 * 128;
  const int yt_n = hp / 128;
  const int ntiles = B * yt_n * d.nc;
  const int a_bytes = d.kg * 2048, b_bytes = d.kg * kN * 16;
  const int stage_bytes = a_bytes + b_bytes;
  const int kIyStages = iy_stages(kC, m);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kIyStagesMax], empty_bar[kIyStagesMax];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kIyStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], kIyEpiWarps);
    }
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_base, 2 * kN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // everything below may touch buffers of the previous kernels
  const uint32_t tmem = tmem_base;

  if (warp == kIyEpiWarps) {
    // ------------------------------------------------------------ producer
    int k = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int s = k % kIyStages;
      if (k >= kIyStages) ok = mbar_wait_sleep(&empty_bar[s], ((k / kIyStages) - 1) & 1, status);
      if (!ok) break;
      const int b = t / (yt_n * d.nc), rem = t - b * yt_n * d.nc;
      const int yt = rem / d.nc, ci = rem - yt * d.nc;
      unsigned char* st = smem + (size_t)s * stage_bytes;
      if (lane == 0) mbar_arrive_expect_tx(&full_bar[s], (unsigned)stage_bytes);
      __syncwarp();
      for (int q = lane; q < 2 * d.kg; q += 32) {
        if (q < d.kg)
          bulk_g2s(st + q * 2048, ty + ((size_t)q * hp + yt * 128) * 8, 2048, &full_bar[s]);
        else
          bulk_g2s(st + a_bytes + (q - d.kg) * kN * 16,
                   yb + (((size_t)b * d.kg + (q - d.kg)) * d.nn + (size_t)ci * kN) * 8,
                   (unsigned)(kN * 16), &full_bar[s]);
      }
    }
    for (int q = max(0, k - kIyStages); q < k; ++q)
      mbar_wait_sleep(&full_bar[q % kIyStages], (q / kIyStages) & 1, status);
  } else if (warp == kIyEpiWarps + 1) {
    // ---------------------------------------------------------------- MMA
    constexpr uint32_t idesc = idesc_bf16(128, kN, false, false);
    int j = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      const int acc = j & 1;
      if (j >= 2) ok = mbar_wait_sleep(&acc_empty[acc], ((j >> 1) - 1) & 1, status);
      if (ok) ok = mbar_wait_sleep(&full_bar[j % kIyStages], (j / kIyStages) & 1, status);
      if (!ok) break;
      tc_fence_after();
      if (lane == 0) {
        const unsigned char* st = smem + (size_t)(j % kIyStages) * stage_bytes;
        for (int kk = 0; kk < d.kg / 2; ++kk) {
          const uint64_t ad = smem_desc(st + kk * 4096, 2048, 128);
          const uint64_t bd = smem_desc(st + a_bytes + kk * 2 * kN * 16, kN * 16, 128);
          mma_bf16(tmem + acc * kN, ad, bd, idesc, kk > 0);
        }
        mma_commit(&empty_bar[j % kIyStages]);
        mma_commit(&acc_full[acc]);
      }
      __syncwarp();
    }
  } else {
    // ----------------------------------------------------------- epilogue
    // 32 accumulator columns = 32 / knk channels o, each with knk consecutive k'
    constexpr int kOpl = 32 / kKnk;
    const int quad = warp & 3, half = warp >> 2;  // TMEM lanes 32 quad.., column half
    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      const int acc = j & 1;
      if (!mbar_wait_sleep(&acc_full[acc], (j >> 1) & 1, status)) break;
      tc_fence_after();
      const int b = t / (yt_n * d.nc), rem = t - b * yt_n * d.nc;
      const int yt = rem / d.nc, ci = rem - yt * d.nc;
      const int y = yt * 128 + quad * 32 + lane;
      const int kp0 = ci * kKnk;
      __nv_bfloat16* zrow = zt + ((size_t)b * H + y) * kK2 * kC + (kp0 / 8) * kC * 8 + (kp0 % 8);
#pragma unroll 1
      for (int cb = half * (kN / 64); cb < (half + 1) * (kN / 64); ++cb) {
        float v[32];
        tmem_ld32(tmem + acc * kN + cb * 32 + ((uint32_t)(quad * 32) << 16), v);
        if (y < H) {
#pragma unroll
          for (int oo = 0; oo < kOpl; ++oo) {
            const int o = cb * kOpl + oo;
            __align__(16) __nv_bfloat16 h[kKnk];
#pragma unroll
            for (int q = 0; q < kKnk; ++q) h[q] = __float2bfloat16_rn(v[oo * kKnk + q]);
            if constexpr (kKnk == 8)
              *reinterpret_cast<uint4*>(zrow + o * 8) = *reinterpret_cast<const uint4*>(h);
            else
              *reinterpret_cast<uint2*>(zrow + o * 8) = *reinterpret_cast<const uint2*>(h);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[acc]);
      if (half == 0 && ci == d.nc - 1 && y < H) {  // k' in [nc * knk, kK2): zero
        __nv_bfloat16* zr = zt + ((size_t)b * H + y) * kK2 * kC;
        for (int kp = d.nc * kKnk; kp < kK2; kp += kKnk)
          for (int o = 0; o < kC; ++o) {
            if constexpr (kKnk == 8)
              *reinterpret_cast<uint4*>(zr + ((kp / 8) * kC + o) * 8) = make_uint4(0, 0, 0, 0);
            else
              *reinterpret_cast<uint2*>(zr + ((kp / 8) * kC + o) * 8 + kp % 8) = make_uint2(0, 0);
          }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 2 * kN);
}

// ------------------------ 4. inverse x-DFT + W theta + bias + activation (tcgen05)
constexpr int kInvMaxStages = 8;
// CTAs per SM: three for C <= 32 (their epilogue warps hide the activation's latency),
// two for C = 64 (shared memory)
template <int kC>
constexpr int inv_ctas_per_sm() { return kC <= 32 ? 3 : 2; }
constexpr int kInvEpiWarps = 8;  // two groups of four: each drains alternate tiles
constexpr int kInvAccs = 2;      // TMEM accumulators, one a warp group
constexpr int kInvThreads = (kInvEpiWarps + 2) * 32;
// Shared memory: a resident part (the CTA's 128-column slice of the inverse-DFT table
// and W^T) and `stages` stages of (latent tile, Zt row), each 1024-byte aligned.
__host__ __device__ constexpr size_t inv_res_bytes(int C, int k2) {
  return (size_t)(k2 / 8) * 2048 + ((size_t)(C / 8) * C * 16 + 1023) / 1024 * 1024;
}
// Grid rows a tile: four for C = 16 and two for C = 32 (each row's MMA fills C columns of
// a 64-column accumulator, spreading the tiles' fixed costs), one for C = 64.
__host__ __device__ constexpr int inv_rows(int C) { return C == 16 ? 4 : (C == 32 ? 2 : 1); }
__host__ __device__ constexpr size_t inv_stage_bytes(int C, int k2) {
  return (size_t)inv_rows(C) * ((size_t)(C / 8) * 2048 + (size_t)(k2 / 8) * C * 16);
}

// Tiles: inv_rows(C) consecutive rows (b, y < Hv) of the layers' grid, 128 storage columns
// each; columns x >= Wv (the storage padding) are written as 0.  Zt rows are indexed on the Hv grid, latent rows on
// the Hs storage.  The grid is a multiple of the tiles a row, so that a CTA's tiles all
// have the same 128 columns and their table slice stays in shared memory.
template <int kC, int kAct, int kK2>
__global__ void __launch_bounds__(kInvThreads, inv_ctas_per_sm<kC>())
    k_inv_x_tc(const __nv_bfloat16* __restrict__ theta, const __nv_bfloat16* __restrict__ ti,
               const __nv_bfloat16* __restrict__ zt, const float* __restrict__ wmat,
               const float* __restrict__ bias, __nv_bfloat16* __restrict__ out, int B, TcGrid gd,
               int stages, unsigned* __restrict__ status) {
  pdl_trigger();
  constexpr int kG = kC / 8;
  constexpr int kSG = kK2 / 8;  // spectral K groups (k' < kK2)
  constexpr int kThetaBytes = kG * 128 * 16;  // A, channel part: [group][x (128)][8]
  constexpr size_t kResBytes = inv_res_bytes(kC, kK2);
  constexpr size_t kStageBytes = inv_stage_bytes(kC, kK2);
  constexpr int kR = inv_rows(kC);                              // grid rows a tile
  constexpr int kPartBytes = kThetaBytes + kSG * kC * 16;      // one row's part of a stage
  static_assert(kStageBytes % 1024 == 0, "stage alignment");
  constexpr int kAccCols = kR * kC < 32 ? 32 : kR * kC;  // the rows' columns side by side
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* ti_s = smem;                      // A, spectral part: [group][x][8]
  unsigned char* w_s = smem + kSG * 2048;          // B, channel part: W^T as [group][o][8]
  unsigned char* stage0 = smem + kResBytes;        // stage s, part r: latent tile, Zt row
  __shared__ __align__(8) uint64_t full_bar[kInvMaxStages], empty_bar[kInvMaxStages];
  __shared__ __align__(8) uint64_t acc_full[kInvAccs], acc_empty[kInvAccs], res_bar;
  __shared__ uint32_t tmem_base;
  __shared__ __align__(16) float bias_s[kC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int H = gd.Hv, W = gd.Ws;
  const int xt = (W + 127) / 128;
  const int nrows = B * H;
  const int ntiles = (nrows + kR - 1) / kR * xt;
  const int x0 = (blockIdx.x % xt) * 128;  // this CTA's columns (gridDim.x % xt == 0)

  for (int e = threadIdx.x; e < kG * kC * 8; e += blockDim.x) {  // W^T, once
    const int g = e / (kC * 8), o = (e / 8) % kC, il = e % 8;
    reinterpret_cast<__nv_bfloat16*>(w_s)[e] = __float2bfloat16_rn(wmat[o * kC + g * 8 + il]);
  }
  for (int o = threadIdx.x; o < kC; o += blockDim.x) bias_s[o] = bias[o];
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < kInvAccs; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], kInvEpiWarps / 2);
    }
    mbar_init(&res_bar, 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_base, kInvAccs * kAccCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // everything below may touch buffers of the previous kernels
  const uint32_t tmem = tmem_base;

  if (warp == kInvEpiWarps) {
    // ------------------------------------------------------------ producer
    if (lane == 0) mbar_arrive_expect_tx(&res_bar, (unsigned)(kSG * 2048));
    __syncwarp();
    if (lane < kSG)  // the table slice of this CTA's columns, group = lane
      bulk_g2s(ti_s + lane * 2048, ti + ((size_t)lane * W + x0) * 8, 2048, &res_bar);
    int k = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int s = k % stages;
      if (k >= stages) ok = mbar_wait_sleep(&empty_bar[s], ((k / stages) - 1) & 1, status);
      if (!ok) break;
      const int row0 = t / xt * kR;  // first row b * Hv + y of the tile
      const int nr = min(kR, nrows - row0);
      unsigned char* st = stage0 + (size_t)s * kStageBytes;
      if (lane == 0) mbar_arrive_expect_tx(&full_bar[s], (unsigned)(nr * kPartBytes));
      __syncwarp();
      if (lane < nr * (kG + 1)) {  // row r = lane / (kG + 1): kG latent groups, Zt row
        const int r = lane / (kG + 1), q = lane - r * (kG + 1), row = row0 + r;
        const int b = row / H, y = row - b * H;
        const size_t srow = (size_t)b * gd.Hs + y;  // latent storage row
        unsigned char* part = st + r * kPartBytes;
        if (q < kG)
          bulk_g2s(part + q * 2048, theta + ((srow * kG + q) * W + x0) * 8, 2048, &full_bar[s]);
        else
          bulk_g2s(part + kThetaBytes, zt + (size_t)row * kK2 * kC, kSG * kC * 16, &full_bar[s]);
      }
    }
    for (int q = max(0, k - stages); q < k; ++q)
      mbar_wait_sleep(&full_bar[q % stages], (q / stages) & 1, status);
    mbar_wait_sleep(&res_bar, 0, status);
  } else if (warp == kInvEpiWarps + 1) {
    // ---------------------------------------------------------------- MMA
    constexpr uint32_t idesc = idesc_bf16(128, kC, false, false);
    int j = 0;
    bool ok = mbar_wait_sleep(&res_bar, 0, status);  // the table slice
    for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++j) {
      const int acc = j % kInvAccs;
      if (j >= kInvAccs) ok = mbar_wait_sleep(&acc_empty[acc], ((j / kInvAccs) - 1) & 1, status);
      if (ok) ok = mbar_wait_sleep(&full_bar[j % stages], (j / stages) & 1, status);
      if (!ok) break;
      tc_fence_after();
      if (lane == 0) {
        const int nr = min(kR, nrows - t / xt * kR);
        // per row r, into accumulator columns r C ..: K = [spectral k' (table slice x Zt
        // row) | channels (latent tile x W^T)]
        for (int r = 0; r < nr; ++r) {
          const unsigned char* part = stage0 + (size_t)(j % stages) * kStageBytes + r * kPartBytes;
          const uint32_t d = tmem + acc * kAccCols + r * kC;
#pragma unroll
          for (int kk = 0; kk < kSG / 2; ++kk) {
            const uint64_t ad = smem_desc(ti_s + kk * 2 * 2048, 2048, 128);
            const uint64_t bd = smem_desc(part + kThetaBytes + kk * 2 * kC * 16, kC * 16, 128);
            mma_bf16(d, ad, bd, idesc, kk > 0);
          }
#pragma unroll
          for (int kk = 0; kk < kG / 2; ++kk) {
            const uint64_t ad = smem_desc(part + kk * 2 * 2048, 2048, 128);
            const uint64_t bd = smem_desc(w_s + kk * 2 * kC * 16, kC * 16, 128);
            mma_bf16(d, ad, bd, idesc, true);
          }
        }
        mma_commit(&empty_bar[j % stages]);
        mma_commit(&acc_full[acc]);
      }
      __syncwarp();
    }
  } else {
    // ----------------------------------------------------------- epilogue
    // warp w drains TMEM lanes 32 (w % 4) .. +31 (x positions), all C columns, of the
    // tiles whose accumulator is w / 4 (the two warp groups take alternate tiles)
    const int quad = warp & 3, grp = warp >> 2;
    for (int t = blockIdx.x + grp * gridDim.x, j = grp; t < ntiles; t += 2 * gridDim.x, j += 2) {
      const int acc = j % kInvAccs;
      if (!mbar_wait_sleep(&acc_full[acc], (j / kInvAccs) & 1, status)) break;
      tc_fence_after();
      const int rp = t / xt, row0 = rp * kR, nr = min(kR, nrows - row0);
      const int xw = (t - rp * xt) * 128 + quad * 32;  // this warp's first column
      const int x = xw + lane;
      const bool valid = x < gd.Wv;
      auto srow_of = [&](int r) {  // latent storage row of the tile's row r
        const int row = row0 + r, b = row / H;
        return (size_t)b * gd.Hs + (row - b * H);
      };
      if (xw >= gd.Wv) {  // warp-uniform: every column of this warp is storage padding
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[acc]);
        if (x < W) {
          for (int r = 0; r < nr; ++r) {
            const size_t srow = srow_of(r);
#pragma unroll
            for (int g = 0; g < kG; ++g)
              *reinterpret_cast<uint4*>(out + ((srow * kG + g) * W + x) * 8) =
                  make_uint4(0, 0, 0, 0);
          }
        }
        continue;
      }
      for (int r = 0; r < nr; ++r) {
        const size_t srow = srow_of(r);
#pragma unroll
        for (int cb = 0; cb < (kC + 31) / 32; ++cb) {
          constexpr int kCols = kC < 32 ? kC : 32;
          float v[32];
          const uint32_t ta =
              tmem + acc * kAccCols + r * kC + cb * 32 + ((uint32_t)(quad * 32) << 16);
          if (kCols == 32) tmem_ld32(ta, v);
          else tmem_ld16(ta, v);
          if (r == nr - 1 && cb == (kC + 31) / 32 - 1) {  // the accumulator is free
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[acc]);
          }
#pragma unroll
          for (int g = 0; g < kCols / 8; ++g) {
            const int o0 = cb * 32 + g * 8;
            __align__(16) __nv_bfloat16 o8[8];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
              const float2 rr = act_c2<kAct>(
                  __fadd2_rn(make_float2(v[g * 8 + q], v[g * 8 + q + 1]),
                             *reinterpret_cast<const float2*>(&bias_s[o0 + q])));
              o8[q] = __float2bfloat16_rn(valid ? rr.x : 0.0f);
              o8[q + 1] = __float2bfloat16_rn(valid ? rr.y : 0.0f);
            }
            if (x < W)
              *reinterpret_cast<uint4*>(out + ((srow * kG + o0 / 8) * W + x) * 8) =
                  *reinterpret_cast<const uint4*>(o8);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kInvAccs * kAccCols);
}

// ------------------------------------------ 5. projection Q (tcgen05 + CUDA cores)
// One hidden layer of width S (32 or 64) and cout <= 3 outputs:
// out = Q2 act(Q1 theta + q1) + q2.  The C x S contraction runs on the tensor cores
// (M = 128 x positions of one image row, N = S, K = C; theta and Q1 both K-major, no
// swizzle); the epilogue adds q1, applies the activation and contracts with Q2 in FP32.  Several CTAs share an SM so
// that enough epilogue warps hide the activation's latency.
constexpr int kDecStages = 4;
constexpr int kDecCtasPerSm = 2;
constexpr int kDecEpiWarps = 8;  // two groups of four: each drains alternate tiles
constexpr int kDecThreads = (kDecEpiWarps + 2) * 32;
// Output rows a tile: two for C <= 32 (their hidden layers side by side in one
// accumulator, spreading the tiles' fixed costs), else one.
__host__ __device__ constexpr int dec_rows(int C) { return C <= 32 ? 2 : 1; }

// Tiles: dec_rows(C) consecutive rows (b, y) of the output grid H0 x W0, 128 columns each
// (W0 a multiple of 128), read from the latent storage (the padded grid is cropped).
template <int kC, int kS, int kAct>
__global__ void __launch_bounds__(kDecThreads, kDecCtasPerSm)
    k_decoder_tc(const __nv_bfloat16* __restrict__ theta, float* __restrict__ out,
                 const float* __restrict__ params, const unsigned* __restrict__ offs, int B,
                 TcGrid gd, int cout, unsigned* __restrict__ status) {
  pdl_trigger();
  const int H = gd.H0, W = gd.W0;
  constexpr int kG = kC / 8;
  constexpr int kR = dec_rows(kC);                 // output rows a tile
  constexpr int kPartBytes = kG * 128 * 16;        // one row: [channel group][x (128)][8]
  constexpr int kStageBytes = kR * kPartBytes;
  constexpr int kAccCols = kR * kS;                // the rows' hidden layers side by side
  static_assert(kS == 32 || kS == 64, "hidden width");
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* q1_s = smem;                       // Q1 as [k group][s][8] bf16
  unsigned char* stages = smem + kG * kS * 16;      // kDecStages * kStageBytes
  // per hidden pair (j, j + 1): {q1[j], q1[j+1], Q2[0][j], Q2[0][j+1]},
  //                            {Q2[1][j], Q2[1][j+1], Q2[2][j], Q2[2][j+1]}
  __shared__ __align__(16) float4 ep_s[kS];
  __shared__ float q2_s[3];
  __shared__ __align__(8) uint64_t full_bar[kDecStages], empty_bar[kDecStages];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  // cout <= 3: the epilogue packs Q2 rows into a float4 with the hidden bias
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int xt = W / 128;
  const int nrows = B * H;
  const int ntiles = (nrows + kR - 1) / kR * xt;
  const float* w1 = params + offs[0];
  const float* b1 = params + offs[1];
  const float* w2 = params + offs[2];
  const float* b2 = params + offs[3];

  for (int e = threadIdx.x; e < kS * kC; e += blockDim.x) {
    const int g = e / (kS * 8), sl = (e / 8) % kS, il = e % 8;
    reinterpret_cast<__nv_bfloat16*>(q1_s)[e] = __float2bfloat16_rn(w1[sl * kC + g * 8 + il]);
  }
  for (int jp = threadIdx.x; jp < kS / 2; jp += blockDim.x) {
    const int j = 2 * jp;
    auto q2w = [&](int q, int jj) { return q < cout ? w2[q * kS + jj] : 0.f; };
    ep_s[2 * jp] = make_float4(b1[j], b1[j + 1], q2w(0, j), q2w(0, j + 1));
    ep_s[2 * jp + 1] = make_float4(q2w(1, j), q2w(1, j + 1), q2w(2, j), q2w(2, j + 1));
  }
  for (int q = threadIdx.x; q < 3; q += blockDim.x) q2_s[q] = q < cout ? b2[q] : 0.f;
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kDecStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
    }
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_base, 2 * kAccCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // everything below may touch buffers of the previous kernels
  const uint32_t tmem = tmem_base;

  if (warp == kDecEpiWarps) {
    // ------------------------------------------------------------ producer
    int k = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int s = k % kDecStages;
      if (k >= kDecStages) ok = mbar_wait_sleep(&empty_bar[s], ((k / kDecStages) - 1) & 1, status);
      if (!ok) break;
      const int rp = t / xt, row0 = rp * kR;  // first row b * H0 + y of the tile
      const int nr = min(kR, nrows - row0);
      const int x0 = (t - rp * xt) * 128;
      unsigned char* st = stages + (size_t)s * kStageBytes;
      if (lane == 0) mbar_arrive_expect_tx(&full_bar[s], (unsigned)(nr * kPartBytes));
      __syncwarp();
      if (lane < nr * kG) {  // row r = lane / kG, channel group lane % kG
        const int r = lane / kG, g = lane - r * kG, row = row0 + r, b = row / H;
        const size_t srow = (size_t)b * gd.Hs + (row - b * H);  // latent storage row
        bulk_g2s(st + r * kPartBytes + g * 2048, theta + ((srow * kG + g) * gd.Ws + x0) * 8,
                 2048, &full_bar[s]);
      }
    }
    for (int q = max(0, k - kDecStages); q < k; ++q)
      mbar_wait_sleep(&full_bar[q % kDecStages], (q / kDecStages) & 1, status);
  } else if (warp == kDecEpiWarps + 1) {
    // ---------------------------------------------------------------- MMA
    constexpr uint32_t idesc = idesc_bf16(128, kS, false, false);
    int j = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      const int acc = j & 1;
      if (j >= 2) ok = mbar_wait_sleep(&acc_empty[acc], ((j >> 1) - 1) & 1, status);
      if (ok) ok = mbar_wait_sleep(&full_bar[j % kDecStages], (j / kDecStages) & 1, status);
      if (!ok) break;
      tc_fence_after();
      if (lane == 0) {
        const unsigned char* st = stages + (size_t)(j % kDecStages) * kStageBytes;
        const int nr = min(kR, nrows - t / xt * kR);
        for (int r = 0; r < nr; ++r)  // row r into accumulator columns r S ..
#pragma unroll
          for (int kk = 0; kk < kG / 2; ++kk) {
            const uint64_t ad = smem_desc(st + r * kPartBytes + kk * 2 * 2048, 2048, 128);
            const uint64_t bd = smem_desc(q1_s + kk * 2 * kS * 16, kS * 16, 128);
            mma_bf16(tmem + acc * kAccCols + r * kS, ad, bd, idesc, kk > 0);
          }
        mma_commit(&empty_bar[j % kDecStages]);
        mma_commit(&acc_full[acc]);
      }
      __syncwarp();
    }
  } else {
    // ----------------------------------------------------------- epilogue
    // warp w holds TMEM lanes 32 (w % 4) .. +31 (x positions x0 + 32 (w % 4) + lane) of
    // the tiles whose accumulator is w / 4 (the two warp groups take alternate tiles)
    const int quad = warp & 3, acc = warp >> 2;
    for (int t = blockIdx.x + acc * gridDim.x, j = acc; t < ntiles; t += 2 * gridDim.x, j += 2) {
      if (!mbar_wait_sleep(&acc_full[acc], (j >> 1) & 1, status)) break;
      tc_fence_after();
      const int rp = t / xt, row0 = rp * kR, nr = min(kR, nrows - row0);
      const int x = (t - rp * xt) * 128 + quad * 32 + lane;
      for (int r = 0; r < nr; ++r) {
        // Q2 contraction on packed pairs: oq[q] = (sum over even j, sum over odd j)
        float2 oq[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
        for (int cb = 0; cb < kS / 32; ++cb) {
          float v[32];
          tmem_ld32(tmem + acc * kAccCols + r * kS + cb * 32 + ((uint32_t)(quad * 32) << 16), v);
          if (r == nr - 1 && cb == kS / 32 - 1) {  // the accumulator is free
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[acc]);
          }
#pragma unroll
          for (int i = 0; i < 32; i += 2) {
            const float4 e0 = ep_s[cb * 32 + i], e1 = ep_s[cb * 32 + i + 1];
            const float2 h =
                act_c2<kAct>(__fadd2_rn(make_float2(v[i], v[i + 1]), make_float2(e0.x, e0.y)));
            oq[0] = __ffma2_rn(make_float2(e0.z, e0.w), h, oq[0]);
            oq[1] = __ffma2_rn(make_float2(e1.x, e1.y), h, oq[1]);
            oq[2] = __ffma2_rn(make_float2(e1.z, e1.w), h, oq[2]);
          }
        }
        float o[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) o[q] = q2_s[q] + (oq[q].x + oq[q].y);
        const int row = row0 + r, b = row / H, y = row - b * H;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (q < cout) out[(((size_t)b * cout + q) * H + y) * W + x] = o[q];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 2 * kAccCols);
}

// ------------------------------------------------------------------- host
int fno_tc_width(int C) { return C <= 16 ? 16 : (C <= 32 ? 32 : 64); }

// Launch with programmatic stream serialisation (see pdl_trigger / pdl_wait).
template <typename... KArgs, typename... Args>
static int launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                      cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  LBM_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
  return LBM_OK;
}

static TcGrid tc_grid(const fno_config& c, int H, int W) {
  TcGrid g;
  g.H0 = H;
  g.W0 = W;
  g.Hv = H + c.padding;
  g.Wv = W + c.padding;
  g.Hs = (g.Hv + 7) / 8 * 8;
  g.Ws = (g.Wv + 63) / 64 * 64;
  return g;
}
// Shared memory of the kernels whose footprint depends on the shape.
// Stages and CTAs a multiprocessor of the forward x-DFT: two CTAs with as many stages as
// fit half a multiprocessor's shared memory beside the table (at most kFwdMaxStages),
// else (wide storage grids) one CTA; 0 stages when fewer than two fit.
struct FwdPlan {
  int stages, ctas_per_sm;
};
static FwdPlan fwd_plan(int Ws, int k2) {
  const long long table = (long long)Ws * k2 * 2;
  for (int ctas = 2; ctas >= 1; --ctas) {
    const long long room =
        std::min<long long>(kTcSmemMax, (long long)kTcSmemSm / ctas - 2048) - table;
    const int n = room > 0 ? (int)std::min<long long>(kFwdMaxStages, room / kFwdStageBytes) : 0;
    if (n >= 2) return {n, ctas};
  }
  return {0, 1};
}
static int fwd_stages(int Ws, int k2) { return fwd_plan(Ws, k2).stages; }
static size_t fwd_smem(int Ws, int k2) {
  return (size_t)Ws * k2 * 2 + (size_t)std::max(fwd_stages(Ws, k2), 2) * kFwdStageBytes;
}
static size_t ydft_smem(int C, int Hs, int m) {
  const SpecDims d = spec_dims(C, m);
  return align_up((size_t)(Hs / 4) * d.nf * 16, 1024) +
         (size_t)ydft_stages(Hs, d.nf) * kYStageBytes;
}
static size_t iydft_smem(int C, int m) {
  return std::max((size_t)iy_stages(C, m) * iy_stage_bytes(C, m), (size_t)kIyMinSmem);
}
// Stages of the inverse x-DFT kernel: as many as fit the CTAs a multiprocessor holds
// (inv_ctas_per_sm), at most kInvMaxStages.
static int inv_stages(int C, int k2) {
  const size_t per_cta = (size_t)kTcSmemSm / (C <= 32 ? 3 : 2) - 2048;  // static + reserved
  const size_t res = inv_res_bytes(C, k2), st = inv_stage_bytes(C, k2);
  if (per_cta <= res) return 0;
  return (int)std::min<size_t>(kInvMaxStages, (per_cta - res) / st);
}
static size_t inv_smem(int C, int k2) {
  return inv_res_bytes(C, k2) + (size_t)std::max(inv_stages(C, k2), 2) * inv_stage_bytes(C, k2);
}

bool fno_tc_supported(const fno_config& c, int H, int W) {
  const int C = fno_tc_width(c.width), m = c.modes;
  const TcGrid g = tc_grid(c, H, W);
  if (m < 1 || m > 32 || 2 * m > g.Hv || 2 * m >= g.Wv || g.Ws > 2048 || c.c_in > 16 || H < 1 ||
      W < 1)
    return false;
  const int k2 = tc_k2(m);
  return fwd_stages(g.Ws, k2) >= 2 && ydft_smem(C, g.Hs, m) <= (size_t)kTcSmemMax &&
         iy_stages(C, m) >= 2 && inv_stages(C, k2) >= 2 && inv_smem(C, k2) <= (size_t)kTcSmemMax;
}

FnoTcWs fno_tc_ws_plan(const fno_config& c, int B, int H, int W) {
  FnoTcWs w{};
  const size_t C = fno_tc_width(c.width), m = c.modes, k2 = tc_k2(c.modes);
  const SpecDims d = spec_dims((int)C, (int)m);
  const TcGrid g = tc_grid(c, H, W);
  size_t p = 0;
  auto take = [&](size_t bytes) {
    const size_t a = p;
    p = align_up(p + bytes, 256);
    return a;
  };
  const size_t spix = (size_t)B * g.Hs * g.Ws;
  const size_t hp = ((size_t)g.Hv + 127) / 128 * 128;
  const size_t tail = 128 * 16;  // a last 128-column tile reads up to 64 columns past the end
  w.theta0 = take(spix * C * 2 + tail);
  w.theta1 = take(spix * C * 2 + tail);
  w.x1b = take((size_t)B * g.Hs * m * C * 4);
  w.xh = take((size_t)2 * m * m * B * C * sizeof(float2));
  w.yb = take((size_t)B * d.kg * d.nn * 16);
  w.zt = take((size_t)B * g.Hv * k2 * C * 2);
  w.fw = take((size_t)g.Ws * k2 * 2);
  w.ti = take((size_t)g.Ws * k2 * 2 + tail);
  w.fy = take((size_t)(g.Hs / 4) * d.nf * 16);
  w.ty = take((size_t)d.kg * hp * 16);
  w.status = take(sizeof(unsigned));
  w.total = p;
  return w;
}

template <int kC, int kAct, int kK2>
static int fno_forward_tc_impl(const fno_config& c, const FnoTcParams& P, const float* in,
                               float* out, int B, int H, int W, char* ws, cudaStream_t s) {
  const FnoTcWs wp = fno_tc_ws_plan(c, B, H, W);
  const TcGrid gd = tc_grid(c, H, W);
  __nv_bfloat16* th[2] = {reinterpret_cast<__nv_bfloat16*>(ws + wp.theta0),
                          reinterpret_cast<__nv_bfloat16*>(ws + wp.theta1)};
  __nv_bfloat16* x1b = reinterpret_cast<__nv_bfloat16*>(ws + wp.x1b);
  float2* xh = reinterpret_cast<float2*>(ws + wp.xh);
  __nv_bfloat16* yb = reinterpret_cast<__nv_bfloat16*>(ws + wp.yb);
  __nv_bfloat16* zt = reinterpret_cast<__nv_bfloat16*>(ws + wp.zt);
  __nv_bfloat16* fw = reinterpret_cast<__nv_bfloat16*>(ws + wp.fw);
  __nv_bfloat16* ti = reinterpret_cast<__nv_bfloat16*>(ws + wp.ti);
  __nv_bfloat16* fy = reinterpret_cast<__nv_bfloat16*>(ws + wp.fy);
  __nv_bfloat16* ty = reinterpret_cast<__nv_bfloat16*>(ws + wp.ty);
  unsigned* status = reinterpret_cast<unsigned*>(ws + wp.status);
  const int m = c.modes;
  const SpecDims d = spec_dims(kC, m);
  const int hp = (gd.Hv + 127) / 128 * 128;
  int dev = 0, nsm = 0;
  LBM_CHECK_CUDA(cudaGetDevice(&dev));
  LBM_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  LBM_CHECK_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), s));
  // padding entries of Yb (k' >= 2m, a >= 2m) are never written by the mixing kernel
  LBM_CHECK_CUDA(cudaMemsetAsync(yb, 0, (size_t)B * d.kg * d.nn * 16, s));
  const int n_tables = 2 * gd.Ws * kK2 + (gd.Hs / 4) * d.nf * 8 + d.kg * hp * 8;
  LBM_TRY(launch_pdl(k_tables, dim3((n_tables + 255) / 256), dim3(256), 0, s, fw, ti, fy, ty, gd, m, hp, d.nf, d.kg));
  const size_t lift_smem = (size_t)kLiftInStages * lift_rows(kC) * c.c_in * 128 * 4;
  const size_t lift_tiles = (size_t)B * (gd.Hs / lift_rows(kC)) * ((gd.Ws + 127) / 128);
  auto lift = [&](auto kern, int cin_c) {
    const int ctas = (int)std::min<size_t>(lift_tiles, (size_t)lift_ctas_per_sm(cin_c, kC) * nsm);
    return launch_pdl(kern, dim3(ctas), dim3(kLiftThreads), lift_smem, s, in, th[0], th[1],
                      P.lift0_w, P.lift0_b, P.lift1_w, P.lift1_b, B, gd, c.c_in, status);
  };
  switch (c.c_in) {  // the input widths of the paper's models get their own instances
    case 1: LBM_TRY(lift(k_lift_tc<kC, 1, kAct>, 1)); break;
    case 2: LBM_TRY(lift(k_lift_tc<kC, 2, kAct>, 2)); break;
    case 4: LBM_TRY(lift(k_lift_tc<kC, 4, kAct>, 4)); break;
    default: LBM_TRY(lift(k_lift_tc<kC, 0, kAct>, 0)); break;
  }
  const size_t f_smem = fwd_smem(gd.Ws, kK2), i_smem = inv_smem(kC, kK2);
  const size_t y_smem = ydft_smem(kC, gd.Hs, m), iy_smem = iydft_smem(kC, m);
  const size_t mix_smem = (size_t)(kC * kC + kMixB * kC) * sizeof(float2);
  LBM_REQUIRE(y_smem <= (size_t)kTcSmemMax && iy_smem <= (size_t)kTcSmemMax &&
                  f_smem <= (size_t)kTcSmemMax && i_smem <= (size_t)kTcSmemMax,
              "fno_forward: spectral working set too large for shared memory");
  const int fwd_ctas = std::min(B * (gd.Hs / (128 / kC)), fwd_plan(gd.Ws, kK2).ctas_per_sm * nsm);
  const int inv_xt = (gd.Ws + 127) / 128;  // a CTA keeps one column slice: grid % inv_xt == 0
  const int inv_ctas = std::max(
      inv_xt, std::min(B * gd.Hv * inv_xt, inv_ctas_per_sm<kC>() * nsm) / inv_xt * inv_xt);
  const int inv_st = inv_stages(kC, kK2);
  const int ydft_ctas = std::min(B * ((m * kC + 127) / 128), 2 * nsm);
  const int iydft_ctas = std::min(B * (hp / 128) * d.nc, nsm);
  const dim3 mix_grid((unsigned)(2 * m * m), (unsigned)((B + kMixB - 1) / kMixB));
  int mix4_bc = kMixB;  // batch chunk: halved while the grid would not cover the SMs twice
  while (mix4_bc > 4 && (2 * m + 3) / 4 * m * ((B + mix4_bc - 1) / mix4_bc) < 2 * nsm)
    mix4_bc /= 2;
  const dim3 mix4_grid((unsigned)((2 * m + 3) / 4 * m), (unsigned)((B + mix4_bc - 1) / mix4_bc));
  const size_t mix4_smem = (size_t)4 * (kC * kC + kMixB * kC) * sizeof(float2);
  int cur = 0;
  for (int n = 0; n < c.layers; ++n) {
    LBM_TRY(launch_pdl((k_fwd_x_tc<kC, kK2>), dim3(fwd_ctas), dim3(kTcThreads), f_smem, s, th[cur],
                       fw, x1b, B, gd.Hs, gd.Ws, m, fwd_stages(gd.Ws, kK2), status));
    LBM_TRY(launch_pdl((k_ydft_tc<kC>), dim3(ydft_ctas), dim3(kTcThreads), y_smem, s, x1b, fy, xh, B, gd.Hs, m, status));
    if constexpr (kC <= 32)  // a block per group of four modes
      LBM_TRY(launch_pdl((k_mix4<kC>), dim3(mix4_grid), dim3(256), mix4_smem, s, xh, P.rt[n], yb,
                         B, m, mix4_bc));
    else
      LBM_TRY(launch_pdl((k_mix<kC>), dim3(mix_grid), dim3(256), mix_smem, s, xh, P.rt[n], yb, B,
                         m));
    LBM_TRY(launch_pdl((k_iydft_tc<kC, kK2>), dim3(iydft_ctas), dim3(kIyThreads), iy_smem, s, ty, yb, zt, B, gd.Hv, m, status));
    LBM_TRY(launch_pdl((k_inv_x_tc<kC, kAct, kK2>), dim3(inv_ctas), dim3(kInvThreads), i_smem, s, 
        th[cur], ti, zt, P.w[n], P.b[n], th[cur ^ 1], B, gd, inv_st, status));
    cur ^= 1;
  }
  const size_t pix = (size_t)B * H * W;
  if (c.dec_layers == 1 && (c.dec_size == 32 || c.dec_size == 64) && c.c_out <= 3 &&
      W % 128 == 0) {
    const size_t smem_tc = (size_t)kC * c.dec_size * 2 +
                           (size_t)kDecStages * dec_rows(kC) * (kC / 8) * 128 * 16;
    const int ntiles = (B * H + dec_rows(kC) - 1) / dec_rows(kC) * (W / 128);
    const int ctas = std::min(ntiles, kDecCtasPerSm * nsm);
    if (c.dec_size == 32)
      LBM_TRY(launch_pdl((k_decoder_tc<kC, 32, kAct>), dim3(ctas), dim3(kDecThreads), smem_tc, s,
                         th[cur], out, P.params, P.dec_offs, B, gd, c.c_out, status));
    else
      LBM_TRY(launch_pdl((k_decoder_tc<kC, 64, kAct>), dim3(ctas), dim3(kDecThreads), smem_tc, s,
                         th[cur], out, P.params, P.dec_offs, B, gd, c.c_out, status));
  } else {
    const size_t dec_smem =
        ((size_t)c.dec_layers * (c.dec_size * 64 + c.dec_size) + c.c_out * 64 + c.c_out) *
        sizeof(float);
    LBM_TRY(launch_pdl((k_decoder_blk<kC>), dim3((unsigned)((pix + 127) / 128)), dim3(128), dec_smem, s, 
        th[cur], out, P.params, P.dec_offs, c.dec_layers, B, gd, c.dec_size, c.c_out,
        c.activation));
  }
  return LBM_OK;
}

template <int kC, int kAct, int kK2>
static int tc_set_smem_attrs_k2() {
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_inv_x_tc<kC, kAct, kK2>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax));
  if (kAct == FNO_ACT_GELU) {
    LBM_CHECK_CUDA(cudaFuncSetAttribute(k_fwd_x_tc<kC, kK2>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax));
    LBM_CHECK_CUDA(cudaFuncSetAttribute(k_iydft_tc<kC, kK2>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax));
  }
  return LBM_OK;
}
template <int kC, int kAct>
static int tc_set_smem_attrs_act() {
  constexpr int lift_in_max = kLiftInStages * lift_rows(kC) * 16 * 128 * 4;  // c_in <= 16
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_lift_tc<kC, 1, kAct>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, lift_in_max));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_lift_tc<kC, 2, kAct>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, lift_in_max));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_lift_tc<kC, 4, kAct>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, lift_in_max));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_lift_tc<kC, 0, kAct>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, lift_in_max));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_decoder_tc<kC, 32, kAct>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_decoder_tc<kC, 64, kAct>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax));
  LBM_TRY((tc_set_smem_attrs_k2<kC, kAct, 32>()));
  return tc_set_smem_attrs_k2<kC, kAct, 64>();
}
template <int kC>
static int tc_set_smem_attrs() {
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_ydft_tc<kC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_mix<kC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax));
  if constexpr (kC <= 32)
    LBM_CHECK_CUDA(cudaFuncSetAttribute(k_mix4<kC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kTcSmemMax));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_decoder_blk<kC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemMax));
  LBM_TRY((tc_set_smem_attrs_act<kC, FNO_ACT_GELU>()));
  return tc_set_smem_attrs_act<kC, FNO_ACT_RELU>();
}

int fno_tc_prepare(const fno_config& c) {
  switch (fno_tc_width(c.width)) {
    case 16: return tc_set_smem_attrs<16>();
    case 32: return tc_set_smem_attrs<32>();
    default: return tc_set_smem_attrs<64>();
  }
}

template <int kC, int kAct>
static int fno_forward_tc_k2(const fno_config& c, const FnoTcParams& P, const float* in, float* out,
                             int B, int H, int W, char* ws, cudaStream_t s) {
  return tc_k2(c.modes) == 32 ? fno_forward_tc_impl<kC, kAct, 32>(c, P, in, out, B, H, W, ws, s)
                              : fno_forward_tc_impl<kC, kAct, 64>(c, P, in, out, B, H, W, ws, s);
}
template <int kC>
static int fno_forward_tc_act(const fno_config& c, const FnoTcParams& P, const float* in, float* out,
                              int B, int H, int W, char* ws, cudaStream_t s) {
  return c.activation == FNO_ACT_GELU
             ? fno_forward_tc_k2<kC, FNO_ACT_GELU>(c, P, in, out, B, H, W, ws, s)
             : fno_forward_tc_k2<kC, FNO_ACT_RELU>(c, P, in, out, B, H, W, ws, s);
}

int fno_forward_tc(const fno_config& c, const FnoTcParams& P, const float* in, float* out, int B,
                   int H, int W, char* ws, cudaStream_t s) {
  switch (fno_tc_width(c.width)) {
    case 16: return fno_forward_tc_act<16>(c, P, in, out, B, H, W, ws, s);
    case 32: return fno_forward_tc_act<32>(c, P, in, out, B, H, W, ws, s);
    default: return fno_forward_tc_act<64>(c, P, in, out, B, H, W, ws, s);
  }
}

// Element-wise activation of the tensor-core kernels, for tests: element pairs go
// through the packed form the kernels use, an odd last element through the scalar one.
template <int kAct>
__global__ void k_act_eval(const float* __restrict__ x, float* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; 2 * i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    if (2 * i + 1 < n) {
      const float2 r = act_c2<kAct>(make_float2(x[2 * i], x[2 * i + 1]));
      y[2 * i] = r.x;
      y[2 * i + 1] = r.y;
    } else {
      y[2 * i] = act_c<kAct>(x[2 * i]);
    }
  }
}

}  // namespace lbmfno

using namespace lbmfno;

extern "C" int fno_activation_eval(int act, const float* x_d, float* y_d, size_t n, void* stream) {
  LBM_REQUIRE(act == FNO_ACT_GELU || act == FNO_ACT_RELU, "fno_activation_eval: unknown activation");
  LBM_REQUIRE(n == 0 || (x_d != nullptr && y_d != nullptr), "fno_activation_eval: null buffer");
  if (n == 0) return LBM_OK;
  const unsigned grid = (unsigned)std::min<size_t>((n / 2 + 256) / 256, 4096);
  if (act == FNO_ACT_GELU)
    k_act_eval<FNO_ACT_GELU><<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x_d, y_d, n);
  else
    k_act_eval<FNO_ACT_RELU><<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x_d, y_d, n);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}
