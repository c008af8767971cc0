// Fourier Neural Operator forward pass (Sec. 2.2, Fig. 2 of arXiv 2604.27158)
// for GB300 (sm_103a) and its C ABI.
//
// Data layout (caller-owned workspace, HBM resident):
//   theta   [B][H][W][C]  bfloat16 latent field (channels innermost)
//   X1      [B][H][m][C]  float2  forward x-DFT of each row (kx < m)
//   Xh, Yh  [B][2m][m][C] float2  kept spectral coefficients before / after mixing
//   Z       [B][H][m][C]  float2  inverse y-DFT of the mixed coefficients
// The spectral convolution is separable: forward x-DFT per row, forward y-DFT per
// column over the kept kx, per-mode complex channel mixing, inverse y-DFT, and a
// fused "inverse x-DFT + W theta + bias + activation" row kernel that writes the
// next latent field.  All sums accumulate in FP32; twiddles e^{+-2 pi i k n / N}
// come from FP32 tables indexed by (k n mod N).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "fno_tc.cuh"
#include "gelu.cuh"
#include "sm100.cuh"

namespace lbmfno {

struct FnoOffsets {
  size_t lift0_w, lift0_b, lift1_w, lift1_b;
  std::vector<size_t> r1re, r1im, r2re, r2im, w, b;
  std::vector<size_t> dec_w, dec_b;
  size_t out_w, out_b;
  size_t n_params;
  size_t rt_off;     // float offset of the transposed spectral filters
  size_t rt_layer;   // floats per layer of transposed filters
  // Copies for the tensor-core kernels with the channel dimensions zero-padded to
  // tcw = fno_tc_width(C), present when tcw != C (tc_pad): lift, per layer the
  // transposed filters [mode][tcw][tcw], W [tcw][tcw] and b [tcw], decoder layer 0 [S][tcw].
  bool tc_pad = false;
  int tcw = 0;
  size_t tp_lift0_w = 0, tp_lift0_b = 0, tp_lift1_w = 0, tp_lift1_b = 0, tp_q1 = 0;
  std::vector<size_t> tp_rt, tp_w, tp_b;
  size_t total_floats;
};

static int fno_offsets(const fno_config& c, FnoOffsets* o) {
  LBM_REQUIRE(c.c_in >= 1 && c.c_in <= 16 && c.c_out >= 1 && c.c_out <= 16,
              "fno: channel counts out of range");
  LBM_REQUIRE(c.width >= 2 && c.width <= 64 && c.width % 2 == 0, "fno: width must be even, <= 64");
  LBM_REQUIRE(c.layers >= 1 && c.layers <= 16 && c.modes >= 1 && c.modes <= 64,
              "fno: layers / modes out of range");
  LBM_REQUIRE(c.dec_layers >= 1 && c.dec_layers <= 8 && c.dec_size >= 1 && c.dec_size <= 64,
              "fno: decoder shape out of range");
  LBM_REQUIRE(c.activation == FNO_ACT_GELU || c.activation == FNO_ACT_RELU,
              "fno: unknown activation");
  LBM_REQUIRE(c.padding >= 0 && c.padding <= 64, "fno: padding must be in 0..64");
  const size_t C = c.width, h = C / 2, m = c.modes, cin2 = c.c_in + 2;
  size_t p = 0;
  auto take = [&](size_t n) {
    const size_t at = p;
    p += n;
    return at;
  };
  o->lift0_w = take(h * cin2);
  o->lift0_b = take(h);
  o->lift1_w = take(C * h);
  o->lift1_b = take(C);
  o->r1re.clear(); o->r1im.clear(); o->r2re.clear(); o->r2im.clear(); o->w.clear(); o->b.clear();
  for (int n = 0; n < c.layers; ++n) {
    o->r1re.push_back(take(C * C * m * m));
    o->r1im.push_back(take(C * C * m * m));
    o->r2re.push_back(take(C * C * m * m));
    o->r2im.push_back(take(C * C * m * m));
    o->w.push_back(take(C * C));
    o->b.push_back(take(C));
  }
  o->dec_w.clear(); o->dec_b.clear();
  size_t fan = C;
  for (int l = 0; l < c.dec_layers; ++l) {
    o->dec_w.push_back(take((size_t)c.dec_size * fan));
    o->dec_b.push_back(take(c.dec_size));
    fan = c.dec_size;
  }
  o->out_w = take((size_t)c.c_out * fan);
  o->out_b = take(c.c_out);
  o->n_params = p;
  o->rt_off = align_up(p, 64);
  o->rt_layer = 2 * m * m * C * C * 2;  // float2 per (mode, i, o)
  o->total_floats = o->rt_off + o->rt_layer * c.layers;
  o->tcw = fno_tc_width(c.width);
  o->tc_pad = (size_t)o->tcw != C;
  o->tp_rt.clear(); o->tp_w.clear(); o->tp_b.clear();
  if (o->tc_pad) {
    const size_t T = o->tcw, th = T / 2;
    p = align_up(o->total_floats, 64);
    auto take2 = [&](size_t n) {  // 2-float aligned for float2 arrays
      p = align_up(p, 2);
      return take(n);
    };
    o->tp_lift0_w = take(th * cin2);
    o->tp_lift0_b = take(th);
    o->tp_lift1_w = take(T * th);
    o->tp_lift1_b = take(T);
    for (int n = 0; n < c.layers; ++n) {
      o->tp_rt.push_back(take2(2 * m * m * T * T * 2));
      o->tp_w.push_back(take(T * T));
      o->tp_b.push_back(take(T));
    }
    o->tp_q1 = take((size_t)c.dec_size * T);
    o->total_floats = p;
  }
  return LBM_OK;
}

struct FnoWs {
  size_t theta0, theta1, x1, xh, yh, z, twx, twy, total;
};
// Workspace of the CUDA-core path for an input of B x H x W: the latent field and the
// spectral buffers live on the padded grid (H + padding) x (W + padding).
static FnoWs fno_ws_plan(const fno_config& c, int B, int H0, int W0) {
  FnoWs w{};
  const size_t C = c.width, m = c.modes;
  const int H = H0 + c.padding, W = W0 + c.padding;
  size_t p = 0;
  auto take = [&](size_t bytes) {
    const size_t at = p;
    p = align_up(p + bytes, 256);
    return at;
  };
  const size_t pix = (size_t)B * H * W;
  w.theta0 = take(pix * C * 2);
  w.theta1 = take(pix * C * 2);
  w.x1 = take((size_t)B * H * m * C * sizeof(float2));
  w.xh = take((size_t)B * 2 * m * m * C * sizeof(float2));
  w.yh = take((size_t)B * 2 * m * m * C * sizeof(float2));
  w.z = take((size_t)B * H * m * C * sizeof(float2));
  w.twx = take((size_t)W * sizeof(float2));
  w.twy = take((size_t)H * sizeof(float2));
  w.total = p;
  return w;
}

// ---------------------------------------------------------------- kernels ---
__device__ __forceinline__ float act_fn(float v, int act) {
  return act == FNO_ACT_GELU ? gelu_poly(v) : fmaxf(v, 0.0f);
}
__device__ __forceinline__ float bf16r(float v) {  // round to the nearest bfloat16 value
  return __bfloat162float(__float2bfloat16_rn(v));
}

__global__ void k_bf16_to_f32(const uint16_t* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t u = (uint32_t)in[i] << 16;
    out[i] = __uint_as_float(u);
  }
}

// Rt[(mode * C + i) * C + o] = (re, im) with mode = a * m + kx, a < m from r1, a >= m from r2
__global__ void k_transpose_r(const float* __restrict__ r1re, const float* __restrict__ r1im,
                              const float* __restrict__ r2re, const float* __restrict__ r2im,
                              float2* __restrict__ rt, int C, int m) {
  const size_t n = (size_t)2 * m * m * C * C;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(t % C);
    const int i = (int)((t / C) % C);
    const int mode = (int)(t / ((size_t)C * C));
    const int a = mode / m, kx = mode % m;
    const bool lo = a < m;
    const int ky = lo ? a : a - m;
    const size_t src = (((size_t)i * C + o) * m + ky) * m + kx;
    rt[t] = lo ? make_float2(r1re[src], r1im[src]) : make_float2(r2re[src], r2im[src]);
  }
}

// dst [drows][dcols] = src [srows][scols] zero-padded (drows >= srows, dcols >= scols)
__global__ void k_pad2d(const float* __restrict__ src, int srows, int scols,
                        float* __restrict__ dst, int drows, int dcols) {
  const size_t n = (size_t)drows * dcols;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / dcols), c = (int)(t % dcols);
    dst[t] = (r < srows && c < scols) ? src[(size_t)r * scols + c] : 0.0f;
  }
}
// dst[(mode * T + i) * T + o] = src[(mode * C + i) * C + o] for i, o < C, else 0
__global__ void k_pad_rt(const float2* __restrict__ src, int C, float2* __restrict__ dst, int T,
                         int modes) {
  const size_t n = (size_t)modes * T * T;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(t % T), i = (int)((t / T) % T);
    const size_t mode = t / ((size_t)T * T);
    dst[t] = (i < C && o < C) ? src[(mode * C + i) * C + o] : make_float2(0.0f, 0.0f);
  }
}

// tw[t] = (cos(2 pi t / N), sin(2 pi t / N))
__global__ void k_twiddle(float2* __restrict__ tw, int N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < N) {
    double s, c;
    sincospi(2.0 * (double)t / (double)N, &s, &c);
    tw[t] = make_float2((float)c, (float)s);
  }
}


// Twiddles by recurrence: e^{i k (n+1) phi} = e^{i k n phi} e^{i k phi}, a complex product
// in registers instead of a shared-memory table load per term; the product is re-seeded
// from the exact table every kReseed steps, which bounds the FP32 drift to ~kReseed ulps.
constexpr int kReseed = 32;
constexpr int kAccMaxV0 = 16;  // most accumulators per thread of the row / column DFTs
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Forward x-DFT of one row (b, y): X1[kx][c] = sum_x theta[x][c] e^{-2 pi i kx x / W}.
// Threads: c = tid % C, kx group g = tid / C owns kx = g, g + G, ... (G = blockDim / C),
// one pass of up to kAccX frequencies (a template: the launch picks the smallest power of
// two covering ceil(m / G)); each staged value feeds all of them.
template <int kAccX>
__global__ void k_fwd_x(const __nv_bfloat16* __restrict__ theta, float2* __restrict__ x1,
                        const float2* __restrict__ twx, int H, int W, int C, int m) {
  extern __shared__ float smem_f[];
  float* row = smem_f;                                  // W * C
  float2* tw = reinterpret_cast<float2*>(row + (size_t)W * C);  // W
  const size_t r = blockIdx.x;  // row index b * H + y
  const __nv_bfloat16* src = theta + r * (size_t)W * C;
  for (int t = threadIdx.x; t < W * C; t += blockDim.x) row[t] = __bfloat162float(src[t]);
  for (int t = threadIdx.x; t < W; t += blockDim.x) tw[t] = twx[t];
  __syncthreads();
  const int groups = blockDim.x / C;
  const int c = threadIdx.x % C, g0 = threadIdx.x / C;
  if (g0 >= groups) return;
  for (int k0 = 0; k0 < m; k0 += kAccX * groups) {
    float2 acc[kAccX], e[kAccX], step[kAccX];
#pragma unroll
    for (int k = 0; k < kAccX; ++k) {
      const int kx = k0 + g0 + k * groups;
      acc[k] = make_float2(0.f, 0.f);
      step[k] = tw[kx < m ? kx : 0];
    }
    for (int x0 = 0; x0 < W; x0 += kReseed) {
#pragma unroll
      for (int k = 0; k < kAccX; ++k) {
        const int kx = k0 + g0 + k * groups;
        e[k] = tw[kx < m ? (int)(((long long)kx * x0) % W) : 0];
      }
      const int xe = min(W, x0 + kReseed);
      for (int x = x0; x < xe; ++x) {
        const float v = row[x * C + c];
#pragma unroll
        for (int k = 0; k < kAccX; ++k) {
          const int kx = k0 + g0 + k * groups;
          if (kx < m) {
            acc[k].x = fmaf(v, e[k].x, acc[k].x);   // v e^{-i phi}: (v cos, -v sin)
            acc[k].y = fmaf(-v, e[k].y, acc[k].y);
            e[k] = cmul(e[k], step[k]);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kAccX; ++k) {
      const int kx = k0 + g0 + k * groups;
      if (kx < m) x1[(r * m + kx) * C + c] = acc[k];
    }
  }
}

// Forward x-DFT, one warp per row (b, y) and one lane per frequency kx (32 at a time):
// each lane advances its own twiddle e^{-i kx x phi} once per x and applies it to all
// C channels of the staged row, so the twiddle work is shared by the channels (the
// kernel above shares a staged value among frequencies instead).  C <= kMaxC <= 32.
constexpr int kFxRowsPerBlock = 4;
constexpr int kFxChunk = 64;  // x positions staged per pass
template <int kMaxC>
__global__ void __launch_bounds__(32 * kFxRowsPerBlock)
    k_fwd_x_row(const __nv_bfloat16* __restrict__ theta, float2* __restrict__ x1,
                const float2* __restrict__ twx, int rows, int W, int C, int m) {
  extern __shared__ float smem_f[];
  float2* tw = reinterpret_cast<float2*>(smem_f);                              // W
  float* rs = smem_f + 2 * (size_t)W + (size_t)(threadIdx.x >> 5) * kFxChunk * kMaxC;
  for (int t = threadIdx.x; t < W; t += blockDim.x) tw[t] = twx[t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const size_t r = (size_t)blockIdx.x * kFxRowsPerBlock + (threadIdx.x >> 5);
  if (r >= (size_t)rows) return;
  const __nv_bfloat16* src = theta + r * (size_t)W * C;
  for (int kx0 = 0; kx0 < m; kx0 += 32) {
    const int kx = min(kx0 + lane, m - 1);
    const float2 step = tw[kx];
    float2 e = make_float2(1.f, 0.f);
    float2 acc[kMaxC];
#pragma unroll
    for (int c = 0; c < kMaxC; ++c) acc[c] = make_float2(0.f, 0.f);
    for (int x0 = 0; x0 < W; x0 += kFxChunk) {
      const int nx = min(kFxChunk, W - x0);
      __syncwarp();
      for (int t = lane; t < nx * C; t += 32) rs[t] = __bfloat162float(src[(size_t)x0 * C + t]);
      __syncwarp();
      for (int xl = 0; xl < nx; ++xl) {
        const int x = x0 + xl;
        if (x % kReseed == 0) e = tw[(int)(((long long)kx * x) % W)];
        const float* v = rs + xl * C;
#pragma unroll
        for (int c = 0; c < kMaxC; ++c)
          if (c < C) {
            acc[c].x = fmaf(v[c], e.x, acc[c].x);   // v e^{-i phi}: (v cos, -v sin)
            acc[c].y = fmaf(-v[c], e.y, acc[c].y);
          }
        e = cmul(e, step);
      }
    }
    if (kx0 + lane < m) {
#pragma unroll
      for (int c = 0; c < kMaxC; ++c)
        if (c < C) x1[(r * m + kx) * C + c] = acc[c];
    }
  }
}

__device__ __forceinline__ int kept_ky(int a, int H, int m) { return a < m ? a : H - 2 * m + a; }

// Forward y-DFT over the kept ky for one (b, kx): Xh[b][a][kx][c].  The column
// X1[b][.][kx][.] is staged through shared memory 32 rows at a time; each thread keeps
// the accumulators of its kept rows a = g, g + G, ... (G = blockDim / C) in registers and
// advances each phase index (ky y mod H) by ky per row.
constexpr int kFwdYRows = 32;
template <int kFwdYAcc>
__global__ void k_fwd_y(const float2* __restrict__ x1, float2* __restrict__ xh,
                        const float2* __restrict__ twy, int H, int C, int m) {
  extern __shared__ float2 fy_s[];  // twiddles [H], then a [kFwdYRows][C] tile
  float2* tile = fy_s + H;
  const int b = blockIdx.x / m, kx = blockIdx.x % m;
  for (int t = threadIdx.x; t < H; t += blockDim.x) fy_s[t] = twy[t];
  const int groups = blockDim.x / C;
  const int c = threadIdx.x % C, g0 = threadIdx.x / C;
  // kept rows handled per pass; more than kFwdYAcc * groups rows take several passes
  for (int a0 = 0; a0 < 2 * m; a0 += kFwdYAcc * groups) {
  float2 acc[kFwdYAcc];
#pragma unroll
  for (int k = 0; k < kFwdYAcc; ++k) acc[k] = make_float2(0.f, 0.f);
  for (int y0 = 0; y0 < H; y0 += kFwdYRows) {
    const int ny = min(kFwdYRows, H - y0);
    __syncthreads();
    for (int t = threadIdx.x; t < ny * C; t += blockDim.x) {
      const int yy = t / C, cc = t - yy * C;
      tile[t] = x1[(((size_t)b * H + y0 + yy) * m + kx) * C + cc];
    }
    __syncthreads();
    if (g0 < groups) {
      float2 e[kFwdYAcc], step[kFwdYAcc];  // e^{+i ky y phi}, advanced by e^{+i ky phi}
#pragma unroll
      for (int k = 0; k < kFwdYAcc; ++k) {
        const int a = a0 + g0 + k * groups;
        const int ky = a < 2 * m ? kept_ky(a, H, m) : 0;
        e[k] = fy_s[(int)(((long long)ky * y0) % H)];
        step[k] = fy_s[ky];
      }
      for (int yy = 0; yy < ny; ++yy) {
        const float2 v = tile[yy * C + c];
#pragma unroll
        for (int k = 0; k < kFwdYAcc; ++k) {
          const int a = a0 + g0 + k * groups;
          if (a < 2 * m) {
            // v e^{-i phi} = v conj(e)
            acc[k].x += v.x * e[k].x + v.y * e[k].y;
            acc[k].y += v.y * e[k].x - v.x * e[k].y;
            e[k] = cmul(e[k], step[k]);
          }
        }
      }
    }
  }
  if (g0 < groups) {
#pragma unroll
    for (int k = 0; k < kFwdYAcc; ++k) {
      const int a = a0 + g0 + k * groups;
      if (a < 2 * m) xh[(((size_t)b * 2 * m + a) * m + kx) * C + c] = acc[k];
    }
  }
  __syncthreads();  // the next pass restages the tile
  }
}

// Forward y-DFT with one thread per kept row a and all C channels in registers: each
// thread advances its twiddle e^{+i ky y phi} once per row and applies it to every
// channel of the staged tile (broadcast reads).  C <= kMaxC <= 32.
template <int kMaxC>
__global__ void k_fwd_y_row(const float2* __restrict__ x1, float2* __restrict__ xh,
                            const float2* __restrict__ twy, int H, int C, int m) {
  extern __shared__ float2 fy_s[];  // twiddles [H], then a [kFwdYRows][C] tile
  // tile entries (Re v, Im v, Im v, -Re v): v conj(e) = (Re v, Im v) e.x + (Im v, -Re v) e.y
  float4* tile = reinterpret_cast<float4*>(fy_s + H + (H & 1));
  const int b = blockIdx.x / m, kx = blockIdx.x % m;
  for (int t = threadIdx.x; t < H; t += blockDim.x) fy_s[t] = twy[t];
  const int a = min((int)threadIdx.x, 2 * m - 1);
  const int ky = kept_ky(a, H, m);
  float2 acc[kMaxC];
#pragma unroll
  for (int c = 0; c < kMaxC; ++c) acc[c] = make_float2(0.f, 0.f);
  for (int y0 = 0; y0 < H; y0 += kFwdYRows) {
    const int ny = min(kFwdYRows, H - y0);
    __syncthreads();
    for (int t = threadIdx.x; t < ny * C; t += blockDim.x) {
      const int yy = t / C, cc = t - yy * C;
      const float2 v = x1[(((size_t)b * H + y0 + yy) * m + kx) * C + cc];
      tile[t] = make_float4(v.x, v.y, v.y, -v.x);
    }
    __syncthreads();
    float2 e = fy_s[(int)(((long long)ky * y0) % H)];
    const float2 step = fy_s[ky];
    for (int yy = 0; yy < ny; ++yy) {
      const float4* v = tile + yy * C;
      const float2 ex = make_float2(e.x, e.x), ey = make_float2(e.y, e.y);
#pragma unroll
      for (int c = 0; c < kMaxC; ++c)
        if (c < C) {
          const float4 q = v[c];
          acc[c] = __ffma2_rn(make_float2(q.z, q.w), ey, __ffma2_rn(make_float2(q.x, q.y), ex, acc[c]));
        }
      e = cmul(e, step);
    }
  }
  if ((int)threadIdx.x < 2 * m) {
#pragma unroll
    for (int c = 0; c < kMaxC; ++c)
      if (c < C) xh[(((size_t)b * 2 * m + a) * m + kx) * C + c] = acc[c];
  }
}

// Inverse y-DFT with one thread per row y and all C channels in registers (the twiddle
// advanced once per kept row and applied to every channel).  C <= kMaxC <= 32.
template <int kMaxC>
__global__ void k_inv_y_row(const float2* __restrict__ yh, float2* __restrict__ z,
                            const float2* __restrict__ twy, int H, int C, int m) {
  // entries (Re v, Re v, -Im v, Im v): v e = (Re v, Re v)(e.x, e.y) + (-Im v, Im v)(e.y, e.x)
  extern __shared__ float4 ys4[];  // 2m * C
  const int b = blockIdx.x / m, kx = blockIdx.x % m;
  for (int t = threadIdx.x; t < 2 * m * C; t += blockDim.x) {
    const int a = t / C, o = t % C;
    const float2 v = yh[(((size_t)b * 2 * m + a) * m + kx) * C + o];
    ys4[t] = make_float4(v.x, v.x, -v.y, v.y);
  }
  __syncthreads();
  for (int y = threadIdx.x; y < H; y += blockDim.x) {
    float2 acc[kMaxC];
#pragma unroll
    for (int o = 0; o < kMaxC; ++o) acc[o] = make_float2(0.f, 0.f);
    const float2 step = twy[y];
    float2 e = make_float2(1.f, 0.f);
    for (int a = 0; a < 2 * m; ++a) {
      if (a % kReseed == 0 || a == m) e = twy[(int)(((long long)kept_ky(a, H, m) * y) % H)];
      const float4* v = ys4 + a * C;
      const float2 e1 = e, e2 = make_float2(e.y, e.x);
#pragma unroll
      for (int o = 0; o < kMaxC; ++o)
        if (o < C) {
          const float4 q = v[o];
          acc[o] = __ffma2_rn(make_float2(q.z, q.w), e2, __ffma2_rn(make_float2(q.x, q.y), e1, acc[o]));
        }
      e = cmul(e, step);
    }
#pragma unroll
    for (int o = 0; o < kMaxC; ++o)
      if (o < C) z[(((size_t)b * H + y) * m + kx) * C + o] = acc[o];
  }
}

// Per-mode complex channel mixing: Yh[b][mode][o] = sum_i Xh[b][mode][i] R[mode][i][o].
__global__ void k_mix(const float2* __restrict__ xh, float2* __restrict__ yh,
                      const float2* __restrict__ rt, int B, int C, int modes) {
  extern __shared__ float2 rs[];  // C * C
  const int mode = blockIdx.x;
  for (int t = threadIdx.x; t < C * C; t += blockDim.x) rs[t] = rt[(size_t)mode * C * C + t];
  __syncthreads();
  const int o = threadIdx.x % C, bg = threadIdx.x / C, groups = blockDim.x / C;
  if (bg >= groups) return;
  for (int b = bg; b < B; b += groups) {
    const float2* xv = xh + ((size_t)b * modes + mode) * C;
    float re = 0.f, im = 0.f;
    for (int i = 0; i < C; ++i) {
      const float2 a = xv[i], r = rs[i * C + o];
      re += a.x * r.x - a.y * r.y;
      im += a.x * r.y + a.y * r.x;
    }
    yh[((size_t)b * modes + mode) * C + o] = make_float2(re, im);
  }
}

// Inverse y-DFT over the kept ky for one (b, kx): Z[b][y][kx][o].
__global__ void k_inv_y(const float2* __restrict__ yh, float2* __restrict__ z,
                        const float2* __restrict__ twy, int H, int C, int m) {
  extern __shared__ float2 ys[];  // 2m * C
  const int b = blockIdx.x / m, kx = blockIdx.x % m;
  for (int t = threadIdx.x; t < 2 * m * C; t += blockDim.x) {
    const int a = t / C, o = t % C;
    ys[t] = yh[(((size_t)b * 2 * m + a) * m + kx) * C + o];
  }
  __syncthreads();
  const int o = threadIdx.x % C, g0 = threadIdx.x / C, groups = blockDim.x / C;
  if (g0 >= groups) return;
  for (int y = g0; y < H; y += groups) {
    float re = 0.f, im = 0.f;
    const float2 step = twy[y];  // ky -> ky + 1 multiplies e^{+i ky y phi} by e^{+i y phi}
    float2 e = make_float2(1.f, 0.f);
    for (int a = 0; a < 2 * m; ++a) {
      if (a % kReseed == 0 || a == m)  // exact restart (and the jump to ky = H - m)
        e = twy[(int)(((long long)kept_ky(a, H, m) * y) % H)];
      const float2 v = ys[a * C + o];
      re += v.x * e.x - v.y * e.y;
      im += v.x * e.y + v.y * e.x;
      e = cmul(e, step);
    }
    z[(((size_t)b * H + y) * m + kx) * C + o] = make_float2(re, im);
  }
}

// Row kernel: theta'[x][o] = act( (1/HW) sum_kx c_kx Re(Z[kx][o] e^{+2 pi i kx x/W})
//                                 + sum_i Wt[o][i] theta[x][i] + bias[o] ).
// One thread per x position computes all C outputs: the twiddle e^{+i kx x phi} is
// advanced once per frequency and applied to every channel; Z is staged pre-scaled by
// c_kx / (H W).  C <= kMaxC, C even.
template <int kMaxC>
__global__ void k_inv_x_row(const __nv_bfloat16* __restrict__ theta, const float2* __restrict__ z,
                            const float* __restrict__ wmat, const float* __restrict__ bias,
                            __nv_bfloat16* __restrict__ out, const float2* __restrict__ twx,
                            int H, int W, int C, int m, int act) {
  extern __shared__ float smem_f[];
  // channel pairs (o, o + 1) on packed FP32: wt2[i][o/2] = (W[o][i], W[o+1][i]),
  // zs4[kx][o/2] = (Re Z[o], Re Z[o+1], -Im Z[o], -Im Z[o+1]) * c_kx / (H W)
  const int C2 = C / 2;
  float4* zs4 = reinterpret_cast<float4*>(smem_f);          // m * C2
  float2* wt2 = reinterpret_cast<float2*>(zs4 + m * C2);   // C * C2
  float2* bs2 = wt2 + C * C2;                               // C2
  float2* tw = bs2 + C2;                                    // W
  const size_t r = blockIdx.x;
  for (int t = threadIdx.x; t < C * C2; t += blockDim.x) {
    const int i = t / C2, o = 2 * (t % C2);
    wt2[t] = make_float2(wmat[o * C + i], wmat[(o + 1) * C + i]);
  }
  for (int t = threadIdx.x; t < C2; t += blockDim.x) bs2[t] = make_float2(bias[2 * t], bias[2 * t + 1]);
  const float inv_hw = 1.0f / ((float)H * (float)W);
  for (int t = threadIdx.x; t < m * C2; t += blockDim.x) {
    const int kx = t / C2, o = 2 * (t % C2);
    const float2 v0 = z[(r * m + kx) * C + o], v1 = z[(r * m + kx) * C + o + 1];
    const float w = (kx == 0 ? 1.0f : 2.0f) * inv_hw;
    zs4[t] = make_float4(v0.x * w, v1.x * w, -v0.y * w, -v1.y * w);
  }
  for (int t = threadIdx.x; t < W; t += blockDim.x) tw[t] = twx[t];
  __syncthreads();
  const __nv_bfloat16* src = theta + r * (size_t)W * C;
  __nv_bfloat16* dst = out + r * (size_t)W * C;
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    float2 acc[kMaxC / 2];
#pragma unroll
    for (int q = 0; q < kMaxC / 2; ++q) acc[q] = q < C2 ? bs2[q] : make_float2(0.f, 0.f);
    const float2 step = tw[x];
    float2 e = make_float2(1.f, 0.f);
    for (int kx = 0; kx < m; ++kx) {
      if (kx % kReseed == 0 && kx > 0) e = tw[(int)(((long long)kx * x) % W)];
      const float4* zk = zs4 + kx * C2;
      const float2 ex = make_float2(e.x, e.x), ey = make_float2(e.y, e.y);
#pragma unroll
      for (int q = 0; q < kMaxC / 2; ++q)
        if (q < C2) {
          const float4 v = zk[q];
          acc[q] = __ffma2_rn(make_float2(v.z, v.w), ey, __ffma2_rn(make_float2(v.x, v.y), ex, acc[q]));
        }
      e = cmul(e, step);
    }
    const __nv_bfloat162* tv = reinterpret_cast<const __nv_bfloat162*>(src + (size_t)x * C);
    for (int i2 = 0; i2 < C2; ++i2) {
      const float2 t = __bfloat1622float2(tv[i2]);
      const float2 tx = make_float2(t.x, t.x), ty = make_float2(t.y, t.y);
      const float2* w0 = wt2 + (2 * i2) * C2;
      const float2* w1 = w0 + C2;
#pragma unroll
      for (int q = 0; q < kMaxC / 2; ++q)
        if (q < C2) acc[q] = __ffma2_rn(w1[q], ty, __ffma2_rn(w0[q], tx, acc[q]));
    }
    __nv_bfloat162* dv = reinterpret_cast<__nv_bfloat162*>(dst + (size_t)x * C);
#pragma unroll
    for (int q = 0; q < kMaxC / 2; ++q)
      if (q < C2) dv[q] = __floats2bfloat162_rn(act_fn(acc[q].x, act), act_fn(acc[q].y, act));
  }
}

// Lifting network with register-resident inputs and hidden units (C <= kMaxC): zero
// for the padding pixels, else P = 1x1 (c_in + 2) -> C/2 -> act -> C.
template <int kMaxC>
__global__ void k_lift_reg(const float* __restrict__ in, __nv_bfloat16* __restrict__ theta,
                           const float* __restrict__ w0, const float* __restrict__ b0,
                           const float* __restrict__ w1, const float* __restrict__ b1, int B,
                           int H, int W, int Hp, int Wp, int cin, int C, int act) {
  const size_t pix = (size_t)B * Hp * Wp;
  const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p >= pix) return;
  const int x = (int)(p % Wp);
  const int y = (int)((p / Wp) % Hp);
  const int b = (int)(p / ((size_t)Wp * Hp));
  __nv_bfloat162* out = reinterpret_cast<__nv_bfloat162*>(theta + p * C);  // C even
  if (x >= W || y >= H) {
    for (int o = 0; o < C / 2; ++o) out[o] = __floats2bfloat162_rn(0.0f, 0.0f);
    return;
  }
  float xin[18];
#pragma unroll
  for (int c = 0; c < 16; ++c)
    if (c < cin) xin[c] = bf16r(in[(((size_t)b * cin + c) * H + y) * W + x]);
  const float gx = bf16r((float)x / (float)max(W - 1, 1));
  const float gy = bf16r((float)y / (float)max(H - 1, 1));
  const int h = C / 2, cin2 = cin + 2;
  float hid[kMaxC / 2];
#pragma unroll
  for (int j = 0; j < kMaxC / 2; ++j) {
    float a = 0.f;
    if (j < h) {
      a = b0[j];
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < cin) a = fmaf(w0[j * cin2 + c], xin[c], a);
      a = fmaf(w0[j * cin2 + cin], gx, a);
      a = fmaf(w0[j * cin2 + cin + 1], gy, a);
      a = act_fn(a, act);
    }
    hid[j] = a;
  }
#pragma unroll
  for (int o = 0; o < kMaxC; o += 2)
    if (o < C) {
      float a0 = b1[o], a1 = b1[o + 1];
#pragma unroll
      for (int j = 0; j < kMaxC / 2; ++j)
        if (j < h) {
          a0 = fmaf(w1[o * h + j], hid[j], a0);
          a1 = fmaf(w1[(o + 1) * h + j], hid[j], a1);
        }
      out[o / 2] = __floats2bfloat162_rn(a0, a1);
    }
}

// Projection Q with one hidden layer, register-resident (C <= kMaxC, c_out <= 4): each
// hidden unit is computed, activated and folded into the outputs at once; the weights
// are staged in shared memory (broadcast reads).
template <int kMaxC>
__global__ void k_decoder1_reg(const __nv_bfloat16* __restrict__ theta, float* __restrict__ out,
                               const float* __restrict__ params, const unsigned* __restrict__ offs,
                               int B, int H, int W, int Hp, int Wp, int C, int S, int cout,
                               int act) {
  extern __shared__ float dec_s[];
  float* w1 = dec_s;           // S * C
  float* b1 = w1 + S * C;      // S
  float* w2 = b1 + S;          // cout * S
  float* b2 = w2 + cout * S;   // cout
  for (int t = threadIdx.x; t < S * C; t += blockDim.x) w1[t] = params[offs[0] + t];
  for (int t = threadIdx.x; t < S; t += blockDim.x) b1[t] = params[offs[1] + t];
  for (int t = threadIdx.x; t < cout * S; t += blockDim.x) w2[t] = params[offs[2] + t];
  for (int t = threadIdx.x; t < cout; t += blockDim.x) b2[t] = params[offs[3] + t];
  __syncthreads();
  const size_t pix = (size_t)B * H * W;
  const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p >= pix) return;
  const int x = (int)(p % W);
  const int y = (int)((p / W) % H);
  const int b = (int)(p / ((size_t)W * H));
  const __nv_bfloat162* src =
      reinterpret_cast<const __nv_bfloat162*>(theta + (((size_t)b * Hp + y) * Wp + x) * C);
  float a[kMaxC];
#pragma unroll
  for (int c = 0; c < kMaxC; c += 2) {
    const float2 v = c < C ? __bfloat1622float2(src[c / 2]) : make_float2(0.f, 0.f);
    a[c] = v.x;
    a[c + 1] = v.y;
  }
  float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q < cout) o[q] = b2[q];
  for (int j = 0; j < S; ++j) {
    float v = b1[j];
#pragma unroll
    for (int c = 0; c < kMaxC; ++c)
      if (c < C) v = fmaf(w1[j * C + c], a[c], v);
    v = act_fn(v, act);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < cout) o[q] = fmaf(w2[q * S + j], v, o[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q < cout) out[(((size_t)b * cout + q) * H + y) * W + x] = o[q];
}

// Projection Q: hidden layers with the activation, then the linear output layer.
// Reads the H x W corner of the padded latent field (the crop after the last layer).
__global__ void k_decoder(const __nv_bfloat16* __restrict__ theta, float* __restrict__ out,
                          const float* __restrict__ params, const unsigned* __restrict__ offs,
                          int nlayers, int B, int H, int W, int Hp, int Wp, int C, int S, int cout,
                          int act) {
  const size_t pix = (size_t)B * H * W;
  const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p >= pix) return;
  float a[64], t[64];
  {
    const int x = (int)(p % W);
    const int y = (int)((p / W) % H);
    const int b = (int)(p / ((size_t)W * H));
    const size_t q = ((size_t)b * Hp + y) * Wp + x;
    for (int c = 0; c < C; ++c) a[c] = __bfloat162float(theta[q * C + c]);
  }
  int fan = C;
  for (int l = 0; l < nlayers; ++l) {
    const float* w = params + offs[2 * l];
    const float* bb = params + offs[2 * l + 1];
    for (int j = 0; j < S; ++j) {
      float v = bb[j];
      for (int c = 0; c < fan; ++c) v = fmaf(w[j * fan + c], a[c], v);
      t[j] = act_fn(v, act);
    }
    for (int j = 0; j < S; ++j) a[j] = t[j];
    fan = S;
  }
  const float* w = params + offs[2 * nlayers];
  const float* bb = params + offs[2 * nlayers + 1];
  const int x = (int)(p % W);
  const int y = (int)((p / W) % H);
  const int b = (int)(p / ((size_t)W * H));
  for (int o = 0; o < cout; ++o) {
    float v = bb[o];
    for (int c = 0; c < fan; ++c) v = fmaf(w[o * fan + c], a[c], v);
    out[(((size_t)b * cout + o) * H + y) * W + x] = v;
  }
}

}  // namespace lbmfno

using namespace lbmfno;

static constexpr size_t kRowSmemMax = 200 * 1024;

// Accumulators per thread for `count` outputs spread over `groups` thread groups: the
// smallest power of two covering ceil(count / groups), at most kAccMaxV0 (more take passes).
static int acc_per_thread(int count, int groups) {
  const int need = (count + groups - 1) / groups;
  int k = 1;
  while (k < need && k < kAccMaxV0) k *= 2;
  return k;
}

static int launch_fwd_x(int rows, int threads, size_t smem, cudaStream_t s,
                        const __nv_bfloat16* th, float2* x1, const float2* twx, int H, int W,
                        int C, int m) {
  switch (acc_per_thread(m, threads / C)) {
    case 1: k_fwd_x<1><<<rows, threads, smem, s>>>(th, x1, twx, H, W, C, m); break;
    case 2: k_fwd_x<2><<<rows, threads, smem, s>>>(th, x1, twx, H, W, C, m); break;
    case 4: k_fwd_x<4><<<rows, threads, smem, s>>>(th, x1, twx, H, W, C, m); break;
    case 8: k_fwd_x<8><<<rows, threads, smem, s>>>(th, x1, twx, H, W, C, m); break;
    default: k_fwd_x<16><<<rows, threads, smem, s>>>(th, x1, twx, H, W, C, m); break;
  }
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

static int launch_fwd_y(int blocks, int threads, size_t smem, cudaStream_t s, const float2* x1,
                        float2* xh, const float2* twy, int H, int C, int m) {
  switch (acc_per_thread(2 * m, threads / C)) {
    case 1: k_fwd_y<1><<<blocks, threads, smem, s>>>(x1, xh, twy, H, C, m); break;
    case 2: k_fwd_y<2><<<blocks, threads, smem, s>>>(x1, xh, twy, H, C, m); break;
    case 4: k_fwd_y<4><<<blocks, threads, smem, s>>>(x1, xh, twy, H, C, m); break;
    case 8: k_fwd_y<8><<<blocks, threads, smem, s>>>(x1, xh, twy, H, C, m); break;
    default: k_fwd_y<16><<<blocks, threads, smem, s>>>(x1, xh, twy, H, C, m); break;
  }
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

static size_t fwd_x_row_smem(int W, int C) {
  const int kmax = C <= 16 ? 16 : 32;
  return (size_t)W * sizeof(float2) + (size_t)kFxRowsPerBlock * kFxChunk * kmax * sizeof(float);
}
static int launch_fwd_x_row(int rows, cudaStream_t s, const __nv_bfloat16* th, float2* x1,
                            const float2* twx, int W, int C, int m) {
  const unsigned blocks = (unsigned)((rows + kFxRowsPerBlock - 1) / kFxRowsPerBlock);
  const size_t smem = fwd_x_row_smem(W, C);
  if (C <= 16)
    k_fwd_x_row<16><<<blocks, 32 * kFxRowsPerBlock, smem, s>>>(th, x1, twx, rows, W, C, m);
  else
    k_fwd_x_row<32><<<blocks, 32 * kFxRowsPerBlock, smem, s>>>(th, x1, twx, rows, W, C, m);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}
static size_t inv_x_row_smem(int W, int C, int m) {
  return (size_t)m * (C / 2) * sizeof(float4) + (size_t)(C * (C / 2) + C / 2 + W) * sizeof(float2);
}
static int launch_inv_x_row(int rows, cudaStream_t s, const __nv_bfloat16* th, const float2* z,
                            const float* w, const float* b, __nv_bfloat16* out,
                            const float2* twx, int H, int W, int C, int m, int act) {
  const int threads = std::min(256, (W + 31) / 32 * 32);
  const size_t smem = inv_x_row_smem(W, C, m);
  if (C <= 16)
    k_inv_x_row<16><<<rows, threads, smem, s>>>(th, z, w, b, out, twx, H, W, C, m, act);
  else if (C <= 32)
    k_inv_x_row<32><<<rows, threads, smem, s>>>(th, z, w, b, out, twx, H, W, C, m, act);
  else
    k_inv_x_row<64><<<rows, threads, smem, s>>>(th, z, w, b, out, twx, H, W, C, m, act);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

// The y-DFT pair for C <= 32: the forward one (x1 -> xh) when x1 is given, else the
// inverse one (yh -> z).
static int launch_y_rows(int B, cudaStream_t s, const float2* x1, float2* xh, const float2* yh,
                         float2* z, const float2* twy, int H, int C, int m) {
  const unsigned blocks = (unsigned)(B * m);
  if (x1 != nullptr) {
    const int threads = (2 * m + 31) / 32 * 32;
    const size_t smem = ((size_t)H + 1) * sizeof(float2) + (size_t)kFwdYRows * C * sizeof(float4);
    if (C <= 16) k_fwd_y_row<16><<<blocks, threads, smem, s>>>(x1, xh, twy, H, C, m);
    else k_fwd_y_row<32><<<blocks, threads, smem, s>>>(x1, xh, twy, H, C, m);
  } else {
    const int threads = std::min(256, (H + 31) / 32 * 32);
    const size_t smem = (size_t)2 * m * C * sizeof(float4);
    if (C <= 16) k_inv_y_row<16><<<blocks, threads, smem, s>>>(yh, z, twy, H, C, m);
    else k_inv_y_row<32><<<blocks, threads, smem, s>>>(yh, z, twy, H, C, m);
  }
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

template <typename K>
static bool raise_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kRowSmemMax) == cudaSuccess;
}

constexpr size_t kDecOffsSlots = 32;  // decoder offsets per table (2 per layer, <= 9 layers)

struct fno_handle {
  fno_config cfg;
  FnoOffsets off;
  float* packed = nullptr;  // caller-owned
  unsigned* dec_offs = nullptr;  // inside packed: decoder offsets table (as floats' bits)
  unsigned* tc_dec_offs = nullptr;  // the same for the tensor-core kernels (padded layer 0)
  bool force_cuda_cores = false;  // use the CUDA-core kernels even where tensor cores apply
};

static inline cudaStream_t SS(void* s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

int fno_query(const fno_config* cfg_h, int B, int H, int W, fno_sizes* out_h) {
  LBM_REQUIRE(cfg_h && out_h, "fno_query: null argument");
  FnoOffsets o;
  LBM_TRY(fno_offsets(*cfg_h, &o));
  LBM_REQUIRE(B >= 0 && H >= 1 && W >= 1, "fno_query: bad shape");
  LBM_REQUIRE(2 * cfg_h->modes <= H + cfg_h->padding && 2 * cfg_h->modes < W + cfg_h->padding,
              "fno_query: need 2m <= H + padding and m < (W + padding)/2 (m=%d, H=%d, W=%d)",
              cfg_h->modes, H, W);
  out_h->n_params = o.n_params;
  out_h->packed_bytes = align_up((o.total_floats + 2 * kDecOffsSlots) * sizeof(float), 256);
  out_h->ws_bytes = std::max(fno_ws_plan(*cfg_h, std::max(B, 1), H, W).total,
                             fno_tc_supported(*cfg_h, H, W)
                                 ? fno_tc_ws_plan(*cfg_h, std::max(B, 1), H, W).total
                                 : (size_t)0);
  return LBM_OK;
}

int fno_create(const fno_config* cfg_h, const uint16_t* params_d, void* packed_d, void* stream,
               fno_handle** out) {
  LBM_REQUIRE(out != nullptr, "fno_create: null handle output");
  *out = nullptr;
  LBM_REQUIRE(cfg_h && params_d && packed_d, "fno_create: null argument");
  LBM_REQUIRE(((uintptr_t)packed_d % 256) == 0, "fno_create: packed buffer must be 256-byte aligned");
  fno_handle* h = new fno_handle();
  h->cfg = *cfg_h;
  int st = fno_offsets(*cfg_h, &h->off);
  if (st != LBM_OK) {
    delete h;
    return st;
  }
  h->packed = static_cast<float*>(packed_d);
  cudaStream_t s = SS(stream);
  // row kernels size their shared memory by W; opt in once (not allowed inside graph capture)
  if (!raise_smem(k_fwd_x<1>) || !raise_smem(k_fwd_x<2>) || !raise_smem(k_fwd_x<4>) ||
      !raise_smem(k_fwd_x<8>) || !raise_smem(k_fwd_x<16>) || !raise_smem(k_fwd_y<1>) ||
      !raise_smem(k_fwd_y<2>) || !raise_smem(k_fwd_y<4>) || !raise_smem(k_fwd_y<8>) ||
      !raise_smem(k_fwd_y<16>) || !raise_smem(k_fwd_x_row<16>) || !raise_smem(k_fwd_x_row<32>) ||
      !raise_smem(k_inv_x_row<16>) || !raise_smem(k_inv_x_row<32>) ||
      !raise_smem(k_inv_x_row<64>) || !raise_smem(k_fwd_y_row<16>) ||
      !raise_smem(k_fwd_y_row<32>) || !raise_smem(k_inv_y_row<16>) ||
      !raise_smem(k_inv_y_row<32>) ||
      fno_tc_prepare(*cfg_h) != LBM_OK) {
    set_error("fno_create: %s", cudaGetErrorString(cudaGetLastError()));
    delete h;
    return LBM_ERR_CUDA;
  }
  const FnoOffsets& o = h->off;
  k_bf16_to_f32<<<1024, 256, 0, s>>>(params_d, h->packed, o.n_params);
  for (int n = 0; n < cfg_h->layers; ++n) {
    k_transpose_r<<<512, 256, 0, s>>>(h->packed + o.r1re[n], h->packed + o.r1im[n],
                                      h->packed + o.r2re[n], h->packed + o.r2im[n],
                                      reinterpret_cast<float2*>(h->packed + o.rt_off + o.rt_layer * n),
                                      cfg_h->width, cfg_h->modes);
  }
  if (o.tc_pad) {  // zero-padded copies for the tensor-core kernels
    const int C = cfg_h->width, T = o.tcw, cin2 = cfg_h->c_in + 2;
    float* P = h->packed;
    k_pad2d<<<64, 256, 0, s>>>(P + o.lift0_w, C / 2, cin2, P + o.tp_lift0_w, T / 2, cin2);
    k_pad2d<<<64, 256, 0, s>>>(P + o.lift0_b, 1, C / 2, P + o.tp_lift0_b, 1, T / 2);
    k_pad2d<<<64, 256, 0, s>>>(P + o.lift1_w, C, C / 2, P + o.tp_lift1_w, T, T / 2);
    k_pad2d<<<64, 256, 0, s>>>(P + o.lift1_b, 1, C, P + o.tp_lift1_b, 1, T);
    for (int n = 0; n < cfg_h->layers; ++n) {
      k_pad_rt<<<512, 256, 0, s>>>(reinterpret_cast<const float2*>(P + o.rt_off + o.rt_layer * n),
                                   C, reinterpret_cast<float2*>(P + o.tp_rt[n]), T,
                                   2 * cfg_h->modes * cfg_h->modes);
      k_pad2d<<<64, 256, 0, s>>>(P + o.w[n], C, C, P + o.tp_w[n], T, T);
      k_pad2d<<<64, 256, 0, s>>>(P + o.b[n], 1, C, P + o.tp_b[n], 1, T);
    }
    k_pad2d<<<64, 256, 0, s>>>(P + o.dec_w[0], cfg_h->dec_size, C, P + o.tp_q1, cfg_h->dec_size, T);
  }
  // decoder offset tables after the transposed filters: the CUDA-core kernels', then the
  // tensor-core kernels' (layer 0's weights zero-padded to the tensor-core width)
  std::vector<unsigned> offs;
  for (int l = 0; l < cfg_h->dec_layers; ++l) {
    offs.push_back((unsigned)o.dec_w[l]);
    offs.push_back((unsigned)o.dec_b[l]);
  }
  offs.push_back((unsigned)o.out_w);
  offs.push_back((unsigned)o.out_b);
  offs.resize(kDecOffsSlots, 0u);
  const std::vector<unsigned> first(offs);
  offs.insert(offs.end(), first.begin(), first.end());
  if (o.tc_pad) offs[kDecOffsSlots] = (unsigned)o.tp_q1;
  h->dec_offs = reinterpret_cast<unsigned*>(h->packed + o.total_floats);
  h->tc_dec_offs = h->dec_offs + kDecOffsSlots;
  if (cudaMemcpyAsync(h->dec_offs, offs.data(), offs.size() * sizeof(unsigned),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("fno_create: %s", cudaGetErrorString(cudaGetLastError()));
    delete h;
    return LBM_ERR_CUDA;
  }
  *out = h;
  return LBM_OK;
}

int fno_forward(fno_handle* h, const float* in_d, float* out_d, int B, int H, int W, void* ws_d,
                size_t ws_bytes, void* stream) {
  LBM_REQUIRE(h && in_d && out_d && ws_d, "fno_forward: null argument");
  const fno_config& c = h->cfg;
  LBM_REQUIRE(B >= 1 && 2 * c.modes <= H + c.padding && 2 * c.modes < W + c.padding,
              "fno_forward: need B >= 1, 2m <= H + padding, m < (W + padding)/2");
  const FnoWs wp = fno_ws_plan(c, B, H, W);
  LBM_REQUIRE(ws_bytes >= wp.total, "fno_forward: workspace too small (%zu < %zu)", ws_bytes,
              wp.total);
  LBM_REQUIRE(((uintptr_t)ws_d % 256) == 0, "fno_forward: workspace must be 256-byte aligned");
  if (fno_tc_supported(c, H, W) && !h->force_cuda_cores) {
    LBM_REQUIRE(ws_bytes >= fno_tc_ws_plan(c, B, H, W).total, "fno_forward: workspace too small");
    FnoTcParams tp{};
    const float* P0 = h->packed;
    const FnoOffsets& o0 = h->off;
    const bool pd = o0.tc_pad;
    tp.lift0_w = P0 + (pd ? o0.tp_lift0_w : o0.lift0_w);
    tp.lift0_b = P0 + (pd ? o0.tp_lift0_b : o0.lift0_b);
    tp.lift1_w = P0 + (pd ? o0.tp_lift1_w : o0.lift1_w);
    tp.lift1_b = P0 + (pd ? o0.tp_lift1_b : o0.lift1_b);
    for (int n = 0; n < c.layers; ++n) {
      tp.rt[n] = reinterpret_cast<const float2*>(P0 + (pd ? o0.tp_rt[n] : o0.rt_off + o0.rt_layer * n));
      tp.w[n] = P0 + (pd ? o0.tp_w[n] : o0.w[n]);
      tp.b[n] = P0 + (pd ? o0.tp_b[n] : o0.b[n]);
    }
    tp.params = P0;
    tp.dec_offs = h->tc_dec_offs;
    return fno_forward_tc(c, tp, in_d, out_d, B, H, W, static_cast<char*>(ws_d), SS(stream));
  }
  char* ws = static_cast<char*>(ws_d);
  __nv_bfloat16* th[2] = {reinterpret_cast<__nv_bfloat16*>(ws + wp.theta0),
                          reinterpret_cast<__nv_bfloat16*>(ws + wp.theta1)};
  float2* x1 = reinterpret_cast<float2*>(ws + wp.x1);
  float2* xh = reinterpret_cast<float2*>(ws + wp.xh);
  float2* yh = reinterpret_cast<float2*>(ws + wp.yh);
  float2* z = reinterpret_cast<float2*>(ws + wp.z);
  float2* twx = reinterpret_cast<float2*>(ws + wp.twx);
  float2* twy = reinterpret_cast<float2*>(ws + wp.twy);
  cudaStream_t s = SS(stream);
  const int C = c.width, m = c.modes;
  const float* P = h->packed;
  const FnoOffsets& o = h->off;
  const int H0 = H, W0 = W;  // input / output grid; the layers run on the padded grid
  H = H0 + c.padding;
  W = W0 + c.padding;
  k_twiddle<<<(W + 255) / 256, 256, 0, s>>>(twx, W);
  k_twiddle<<<(H + 255) / 256, 256, 0, s>>>(twy, H);
  const size_t pix_p = (size_t)B * H * W;
  {
    const unsigned blocks = (unsigned)((pix_p + 127) / 128);
    if (C <= 16)
      k_lift_reg<16><<<blocks, 128, 0, s>>>(in_d, th[0], P + o.lift0_w, P + o.lift0_b,
                                            P + o.lift1_w, P + o.lift1_b, B, H0, W0, H, W, c.c_in,
                                            C, c.activation);
    else if (C <= 32)
      k_lift_reg<32><<<blocks, 128, 0, s>>>(in_d, th[0], P + o.lift0_w, P + o.lift0_b,
                                            P + o.lift1_w, P + o.lift1_b, B, H0, W0, H, W, c.c_in,
                                            C, c.activation);
    else
      k_lift_reg<64><<<blocks, 128, 0, s>>>(in_d, th[0], P + o.lift0_w, P + o.lift0_b,
                                            P + o.lift1_w, P + o.lift1_b, B, H0, W0, H, W, c.c_in,
                                            C, c.activation);
  }
  LBM_CHECK_LAUNCH();
  const int rows = B * H;
  const size_t smem_fx = (size_t)W * C * sizeof(float) + (size_t)W * sizeof(float2);
  const size_t smem_ix = inv_x_row_smem(W, C, m);
  LBM_REQUIRE(((size_t)H + kFwdYRows * C) * sizeof(float2) <= kRowSmemMax,
              "fno_forward: H too large for the y-DFT kernel");
  LBM_REQUIRE(smem_fx <= kRowSmemMax && smem_ix <= kRowSmemMax &&
                  fwd_x_row_smem(W, C) <= kRowSmemMax,
              "fno_forward: W * C too large for the row kernels");
  const int cur_threads = 256;
  int cur = 0;
  for (int n = 0; n < c.layers; ++n) {
    if (C <= 32)
      LBM_TRY(launch_fwd_x_row(rows, s, th[cur], x1, twx, W, C, m));
    else
      LBM_TRY(launch_fwd_x(rows, cur_threads, smem_fx, s, th[cur], x1, twx, H, W, C, m));
    if (C <= 32 && 2 * m >= 32)  // one thread per kept row: worth it from a full warp of rows
      LBM_TRY(launch_y_rows(B, s, x1, xh, nullptr, nullptr, twy, H, C, m));
    else
      LBM_TRY(launch_fwd_y(B * m, cur_threads, ((size_t)H + kFwdYRows * C) * sizeof(float2), s,
                           x1, xh, twy, H, C, m));
    k_mix<<<2 * m * m, cur_threads, (size_t)C * C * sizeof(float2), s>>>(
        xh, yh, reinterpret_cast<const float2*>(P + o.rt_off + o.rt_layer * n), B, C, 2 * m * m);
    if (C <= 32)
      LBM_TRY(launch_y_rows(B, s, nullptr, nullptr, yh, z, twy, H, C, m));
    else
      k_inv_y<<<B * m, cur_threads, (size_t)2 * m * C * sizeof(float2), s>>>(yh, z, twy, H, C, m);
    LBM_TRY(launch_inv_x_row(rows, s, th[cur], z, P + o.w[n], P + o.b[n], th[cur ^ 1], twx, H,
                             W, C, m, c.activation));
    cur ^= 1;
  }
  const size_t pix = (size_t)B * H0 * W0;
  const unsigned dblocks = (unsigned)((pix + 127) / 128);
  const size_t dsmem = ((size_t)c.dec_size * C + c.dec_size + (size_t)c.c_out * c.dec_size + c.c_out) * sizeof(float);
  if (c.dec_layers == 1 && c.c_out <= 4 && C <= 32) {
    if (C <= 16)
      k_decoder1_reg<16><<<dblocks, 128, dsmem, s>>>(th[cur], out_d, P, h->dec_offs, B, H0, W0, H,
                                                     W, C, c.dec_size, c.c_out, c.activation);
    else
      k_decoder1_reg<32><<<dblocks, 128, dsmem, s>>>(th[cur], out_d, P, h->dec_offs, B, H0, W0, H,
                                                     W, C, c.dec_size, c.c_out, c.activation);
  } else {
    k_decoder<<<dblocks, 128, 0, s>>>(th[cur], out_d, P, h->dec_offs, c.dec_layers, B, H0, W0, H,
                                      W, C, c.dec_size, c.c_out, c.activation);
  }
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int fno_set_path(fno_handle* h, int path) {
  LBM_REQUIRE(h != nullptr && (path == FNO_PATH_AUTO || path == FNO_PATH_CUDA_CORES),
              "fno_set_path: bad arguments");
  h->force_cuda_cores = path == FNO_PATH_CUDA_CORES;
  return LBM_OK;
}

int fno_uses_tensor_cores(const fno_handle* h, int H, int W, int* out_h) {
  LBM_REQUIRE(h != nullptr && out_h != nullptr, "fno_uses_tensor_cores: bad arguments");
  *out_h = (!h->force_cuda_cores && fno_tc_supported(h->cfg, H, W)) ? 1 : 0;
  return LBM_OK;
}

int fno_check(const fno_handle* h, const void* ws_d, int B, int H, int W, void* stream) {
  LBM_REQUIRE(h != nullptr && ws_d != nullptr, "fno_check: bad arguments");
  cudaStream_t s = SS(stream);
  LBM_CHECK_CUDA(cudaStreamSynchronize(s));
  if (!h->force_cuda_cores && fno_tc_supported(h->cfg, H, W)) {
    const FnoTcWs wp = fno_tc_ws_plan(h->cfg, B, H, W);
    unsigned st = 0;
    LBM_CHECK_CUDA(cudaMemcpy(&st, static_cast<const char*>(ws_d) + wp.status, sizeof(unsigned),
                              cudaMemcpyDeviceToHost));
    if (st & kStatusTimeout) {
      set_error("fno: a device-side wait expired (status 0x%x)", st);
      return LBM_ERR_TIMEOUT;
    }
  }
  return LBM_OK;
}

int fno_get_config(const fno_handle* h, fno_config* out_h) {
  LBM_REQUIRE(h && out_h, "fno_get_config: null argument");
  *out_h = h->cfg;
  return LBM_OK;
}

int fno_destroy(fno_handle* h) {
  delete h;
  return LBM_OK;
}

}  // extern "C"
