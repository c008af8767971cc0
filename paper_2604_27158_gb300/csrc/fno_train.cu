// FNO training kernels (Sec. 2.2 forward with saved activations, and its exact
// reverse mode) for GB300 (sm_103a) and their C ABI.
//
// The training path keeps FP32 master parameters and FP32 activations: the forward
// pass saves, per layer, the latent field theta_n, the pre-activation z_n and the
// kept spectral coefficients X_n = F(theta_n); the backward pass is the chain rule
// through the same operators, with the spectral layer's adjoint written out:
//   z = W theta + b + F^-1(R . F(theta)),   theta' = sigma(z)
//   dz      = dtheta' * sigma'(z)
//   dW      = sum_pixels dz theta^T,  db = sum_pixels dz
//   dY[k]   = (c_kx / (H W)) * F(dz)[k]           (transpose of the real inverse)
//   dR[k]   = sum_batch conj(X[k]) dY[k]          (per-mode complex channel mixing)
//   dX[k]   = dY[k] conj(R[k])^T
//   dtheta  = W^T dz + Re sum_k dX[k] e^{+i phi_k}  (transpose of the forward DFT)
// with F the truncated forward DFT over ky in [0, m) U [H-m, H), kx in [0, m),
// c_0 = 1, c_kx = 2 for kx > 0, phi_k = 2 pi (ky y / H + kx x / W).
//
// Layout: latent fields channels-last, [B][H][W][C] FP32 (pixel p = (b H + y) W + x);
// spectral buffers [B][rows][m][C] float2.  Every reduction is in a fixed order (block
// partials, then one ordered pass), so gradients are deterministic.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace lbmfno {

namespace {

inline cudaStream_t TS(void* s) { return reinterpret_cast<cudaStream_t>(s); }

constexpr int kPwPix = 128;      // pixels per block of the pointwise kernel
constexpr int kWgThreads = 256;  // threads of the weight-gradient kernel
constexpr int kWgPairs = 17;     // (o, i) pairs per thread: 64 x (64 + 1) <= 256 * 17
constexpr int kWgTile = 32;      // pixels staged per iteration
constexpr int kSpecThreads = 256;
constexpr int kAccMax = 16;      // spectral accumulators per thread
constexpr int kTrModesMax = 32;

struct TrOff {
  size_t lift0_w, lift0_b, lift1_w, lift1_b;
  std::vector<size_t> r1re, r1im, r2re, r2im, w, b, dec_w, dec_b;
  size_t out_w, out_b, n;
};

int tr_offsets(const fno_config& c, TrOff* o) {
  LBM_REQUIRE(c.c_in >= 1 && c.c_in <= 16 && c.c_out >= 1 && c.c_out <= 16,
              "fno_train: channel counts out of range");
  LBM_REQUIRE(c.width >= 2 && c.width <= 64 && c.width % 2 == 0,
              "fno_train: width must be even, <= 64");
  LBM_REQUIRE(c.layers >= 1 && c.layers <= 16 && c.modes >= 1 && c.modes <= kTrModesMax,
              "fno_train: layers in 1..16, modes in 1..%d", kTrModesMax);
  LBM_REQUIRE(c.dec_layers >= 1 && c.dec_layers <= 8 && c.dec_size >= 1 && c.dec_size <= 64,
              "fno_train: decoder shape out of range");
  LBM_REQUIRE(c.activation == FNO_ACT_GELU || c.activation == FNO_ACT_RELU,
              "fno_train: unknown activation");
  LBM_REQUIRE(c.padding == 0, "fno_train: padding is not supported by the training path");
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
  for (int n = 0; n < c.layers; ++n) {
    o->r1re.push_back(take(C * C * m * m));
    o->r1im.push_back(take(C * C * m * m));
    o->r2re.push_back(take(C * C * m * m));
    o->r2im.push_back(take(C * C * m * m));
    o->w.push_back(take(C * C));
    o->b.push_back(take(C));
  }
  size_t fan = C;
  for (int l = 0; l < c.dec_layers; ++l) {
    o->dec_w.push_back(take((size_t)c.dec_size * fan));
    o->dec_b.push_back(take(c.dec_size));
    fan = c.dec_size;
  }
  o->out_w = take((size_t)c.c_out * fan);
  o->out_b = take(c.c_out);
  o->n = p;
  return LBM_OK;
}

// Saved activations (floats) and workspace (bytes) of one (config, B, H, W).
struct TrPlan {
  size_t P, C, S, h, cin2, m;
  // saved, in floats
  size_t xin, h1pre, theta, zpre, xh, hdpre, saved_floats;
  // workspace, in bytes
  size_t rt, x1, yh, dyh, z, s, ta, tb, dz, part, twx, twy, ycl, ws_bytes;
  int wg_blocks;
};

TrPlan tr_plan(const fno_config& c, int B, int H, int W) {
  TrPlan t{};
  t.P = (size_t)B * H * W;
  t.C = c.width;
  t.S = c.dec_size;
  t.h = c.width / 2;
  t.cin2 = c.c_in + 2;
  t.m = c.modes;
  const size_t N = c.layers, L = c.dec_layers, P = t.P, C = t.C, m = t.m;
  const size_t spec = (size_t)B * 2 * m * m * C;  // float2 per layer
  size_t f = 0;
  auto takef = [&](size_t n) {
    const size_t at = f;
    f += (n + 63) / 64 * 64;
    return at;
  };
  t.xin = takef(P * t.cin2);
  t.h1pre = takef(P * t.h);
  t.theta = takef((N + 1) * P * C);
  t.zpre = takef(N * P * C);
  t.xh = takef(N * spec * 2);
  t.hdpre = takef(L * P * t.S);
  t.saved_floats = f;
  size_t b = 0;
  auto take = [&](size_t bytes) {
    const size_t at = b;
    b = align_up(b + bytes, 256);
    return at;
  };
  const size_t wide = std::max(std::max(C, t.S), std::max(t.cin2, (size_t)c.c_out));
  t.rt = take(N * 2 * m * m * C * C * sizeof(float2));
  t.x1 = take((size_t)B * H * m * C * sizeof(float2));
  t.yh = take(spec * sizeof(float2));
  t.dyh = take(spec * sizeof(float2));
  t.z = take((size_t)B * H * m * C * sizeof(float2));
  t.s = take(P * C * sizeof(float));
  t.ta = take(P * wide * sizeof(float));
  t.tb = take(P * wide * sizeof(float));
  t.dz = take(P * wide * sizeof(float));
  t.wg_blocks = (int)std::min<size_t>(1024, (P + 511) / 512);
  t.part = take((size_t)t.wg_blocks * 64 * 65 * sizeof(float));
  t.twx = take((size_t)W * sizeof(float2));
  t.twy = take((size_t)H * sizeof(float2));
  t.ycl = take(P * c.c_out * sizeof(float));
  t.ws_bytes = b;
  return t;
}

__device__ __forceinline__ float tr_act(float v, int act) {
  return act == FNO_ACT_GELU ? 0.5f * v * (1.0f + erff(v * 0.70710678118654752f))
                             : fmaxf(v, 0.0f);
}
// sigma'(v): GELU Phi(v) + v phi(v); ReLU the step function
__device__ __forceinline__ float tr_dact(float v, int act) {
  if (act != FNO_ACT_GELU) return v > 0.0f ? 1.0f : 0.0f;
  const float cdf = 0.5f * (1.0f + erff(v * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * v * v);
  return cdf + v * pdf;
}
__device__ __forceinline__ float bf16r(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

__global__ void k_tr_twiddle(float2* __restrict__ tw, int N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < N) {
    double s, c;
    sincospi(2.0 * (double)t / (double)N, &s, &c);
    tw[t] = make_float2((float)c, (float)s);
  }
}

// Rt[layer][mode][i][o] = R[i][o][ky][kx] (mode = a m + kx; a < m: r1 at ky = a,
// a >= m: r2 at ky = a - m).
struct RtOffs {
  unsigned long long v[4 * 16];  // r1re, r1im, r2re, r2im of each layer
};
__global__ void k_tr_rt(const float* __restrict__ params, const RtOffs offs,
                        float2* __restrict__ rt, int layers, int C, int m) {
  const size_t per = (size_t)2 * m * m * C * C;
  const size_t n = per * layers;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int layer = (int)(t / per);
    const size_t r = t - layer * per;
    const int o = (int)(r % C);
    const int i = (int)((r / C) % C);
    const int mode = (int)(r / ((size_t)C * C));
    const int a = mode / m, kx = mode % m;
    const bool lo = a < m;
    const int ky = lo ? a : a - m;
    const size_t src = (((size_t)i * C + o) * m + ky) * m + kx;
    const unsigned long long* ol = offs.v + 4 * layer;
    rt[t] = lo ? make_float2(params[ol[0] + src], params[ol[1] + src])
               : make_float2(params[ol[2] + src], params[ol[3] + src]);
  }
}

// Lifting network input: xin[p] = (in channels, x/(W-1), y/(H-1)) with the coordinate
// channels rounded to bfloat16 as in the inference path.
__global__ void k_tr_xin(const float* __restrict__ in, float* __restrict__ xin, int B, int H,
                         int W, int cin) {
  const size_t P = (size_t)B * H * W;
  const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int x = (int)(p % W);
  const int y = (int)((p / W) % H);
  const int b = (int)(p / ((size_t)W * H));
  const int cin2 = cin + 2;
  for (int c = 0; c < cin; ++c) xin[p * cin2 + c] = in[(((size_t)b * cin + c) * H + y) * W + x];
  xin[p * cin2 + cin] = bf16r((float)x / (float)max(W - 1, 1));
  xin[p * cin2 + cin + 1] = bf16r((float)y / (float)max(H - 1, 1));
}

// Pointwise linear layer over kPwPix pixels per block:
//   v[p][o] = add[p][o] + bias[o] + sum_i Wm(o, i) * A(in[p][i]),
//   Wm(o, i) = trans ? w[i * cout + o] : w[o * cin + i],  A = sigma if in_act else identity;
//   pre[p][o] = v (if pre != null);  out[p][o] = out_act ? sigma(v) : v.
__global__ void __launch_bounds__(kPwPix) k_tr_pw(const float* __restrict__ in, int cin,
                                                  const float* __restrict__ w, int trans,
                                                  const float* __restrict__ bias,
                                                  const float* __restrict__ add, int cout,
                                                  float* __restrict__ pre, float* __restrict__ out,
                                                  int in_act, int out_act, int act, size_t P) {
  extern __shared__ float sm[];
  float* ws = sm;                               // [cout][cin]
  float* is = ws + cout * cin;                  // [kPwPix][cin + 1]
  float* os = is + kPwPix * (cin + 1);          // [kPwPix][cout + 1]
  const size_t p0 = (size_t)blockIdx.x * kPwPix;
  const int np = (int)min((size_t)kPwPix, P - p0);
  for (int j = threadIdx.x; j < cout * cin; j += kPwPix) {
    const int o = j / cin, i = j - o * cin;
    ws[j] = trans ? w[(size_t)i * cout + o] : w[j];
  }
  for (int j = threadIdx.x; j < np * cin; j += kPwPix) {
    const int t = j / cin, i = j - t * cin;
    const float v = in[p0 * cin + j];
    is[t * (cin + 1) + i] = in_act ? tr_act(v, act) : v;
  }
  for (int j = threadIdx.x; j < np * cout; j += kPwPix) {
    const int t = j / cout, o = j - t * cout;
    os[t * (cout + 1) + o] = (add ? add[p0 * cout + j] : 0.0f) + (bias ? bias[o] : 0.0f);
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < np) {
    const float* ir = is + t * (cin + 1);
    float* orow = os + t * (cout + 1);
    for (int o = 0; o < cout; ++o) {
      const float* wr = ws + o * cin;
      float acc = 0.0f;
      for (int i = 0; i < cin; ++i) acc = fmaf(wr[i], ir[i], acc);
      orow[o] += acc;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < np * cout; j += kPwPix) {
    const int tt = j / cout, o = j - tt * cout;
    const float v = os[tt * (cout + 1) + o];
    if (pre) pre[p0 * cout + j] = v;
    out[p0 * cout + j] = out_act ? tr_act(v, act) : v;
  }
}

// dz = g * sigma'(z), elementwise
__global__ void k_tr_act_bwd(const float* __restrict__ g, const float* __restrict__ z,
                             float* __restrict__ dz, size_t n, int act) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dz[i] = g[i] * tr_dact(z[i], act);
}

// Block partials of dW[o][i] = sum_p dz[p][o] A(in[p][i]) and db[o] = sum_p dz[p][o]
// (pair (o, cin) of the partial is db).  Block k covers a contiguous pixel range.
__global__ void __launch_bounds__(kWgThreads) k_tr_wgrad(const float* __restrict__ dz, int cout,
                                                         const float* __restrict__ in, int cin,
                                                         int in_act, int act, size_t P,
                                                         float* __restrict__ part) {
  __shared__ float ds[kWgTile][65];
  __shared__ float is[kWgTile][66];
  const int npairs = cout * (cin + 1);
  const size_t per = (P + gridDim.x - 1) / gridDim.x;
  const size_t pa = (size_t)blockIdx.x * per;
  const size_t pb = min(P, pa + per);
  float acc[kWgPairs];
#pragma unroll
  for (int k = 0; k < kWgPairs; ++k) acc[k] = 0.0f;
  for (size_t q0 = pa; q0 < pb; q0 += kWgTile) {
    const int nt = (int)min((size_t)kWgTile, pb - q0);
    __syncthreads();
    for (int j = threadIdx.x; j < kWgTile * cout; j += kWgThreads) {
      const int t = j / cout, o = j - t * cout;
      ds[t][o] = t < nt ? dz[(q0 + t) * cout + o] : 0.0f;
    }
    for (int j = threadIdx.x; j < kWgTile * (cin + 1); j += kWgThreads) {
      const int t = j / (cin + 1), i = j - t * (cin + 1);
      float v = 0.0f;
      if (t < nt) {
        if (i == cin) {
          v = 1.0f;
        } else {
          v = in[(q0 + t) * cin + i];
          if (in_act) v = tr_act(v, act);
        }
      }
      is[t][i] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kWgPairs; ++k) {
      const int pr = threadIdx.x + k * kWgThreads;
      if (pr < npairs) {
        const int o = pr / (cin + 1), i = pr - o * (cin + 1);
        float a = acc[k];
        for (int t = 0; t < kWgTile; ++t) a = fmaf(ds[t][o], is[t][i], a);
        acc[k] = a;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kWgPairs; ++k) {
    const int pr = threadIdx.x + k * kWgThreads;
    if (pr < npairs) part[(size_t)blockIdx.x * npairs + pr] = acc[k];
  }
}

// Ordered sum of the block partials into dW (cout x cin) and db (cout).
__global__ void k_tr_wgrad_reduce(const float* __restrict__ part, int nblk, int cout, int cin,
                                  float* __restrict__ dw, float* __restrict__ db) {
  const int npairs = cout * (cin + 1);
  const int pr = blockIdx.x * blockDim.x + threadIdx.x;
  if (pr >= npairs) return;
  float s = 0.0f;
  for (int k = 0; k < nblk; ++k) s += part[(size_t)k * npairs + pr];
  const int o = pr / (cin + 1), i = pr - o * (cin + 1);
  if (i == cin)
    db[o] = s;
  else
    dw[o * cin + i] = s;
}

// Forward x-DFT of each row: X1[row][kx][c] = sum_x f[row][x][c] e^{-2 pi i kx x / W}.
__global__ void __launch_bounds__(kSpecThreads) k_tr_dft_x(const float* __restrict__ f,
                                                           float2* __restrict__ x1,
                                                           const float2* __restrict__ twx,
                                                           int W, int C, int m) {
  extern __shared__ float sm[];
  float2* tw = reinterpret_cast<float2*>(sm);  // W
  float* tile = sm + 2 * W;                     // [32][C]
  const size_t row = blockIdx.x;
  for (int t = threadIdx.x; t < W; t += kSpecThreads) tw[t] = twx[t];
  const int G = kSpecThreads / C;
  const int c = threadIdx.x % C, g = threadIdx.x / C;
  float2 acc[kAccMax];
#pragma unroll
  for (int k = 0; k < kAccMax; ++k) acc[k] = make_float2(0.f, 0.f);
  for (int x0 = 0; x0 < W; x0 += 32) {
    const int nx = min(32, W - x0);
    __syncthreads();
    for (int j = threadIdx.x; j < nx * C; j += kSpecThreads)
      tile[j] = f[(row * W + x0) * C + j];
    __syncthreads();
    if (g < G) {
#pragma unroll
      for (int k = 0; k < kAccMax; ++k) {
        const int kx = g + k * G;
        if (kx < m) {
          int idx = (kx * x0) % W;  // phase index (kx x) mod W, advanced by kx per x
          for (int xx = 0; xx < nx; ++xx) {
            const float2 e = tw[idx];
            const float v = tile[xx * C + c];
            acc[k].x = fmaf(v, e.x, acc[k].x);
            acc[k].y = fmaf(-v, e.y, acc[k].y);
            idx += kx;
            if (idx >= W) idx -= W;
          }
        }
      }
    }
  }
  if (g < G) {
#pragma unroll
    for (int k = 0; k < kAccMax; ++k) {
      const int kx = g + k * G;
      if (kx < m) x1[(row * m + kx) * C + c] = acc[k];
    }
  }
}

// Forward y-DFT over the kept rows: Xh[b][a][kx][c] = scale(kx) sum_y X1[b][y][kx][c]
// e^{-2 pi i ky(a) y / H}, ky(a) = a (a < m) or H - 2m + a; scale = 1, or c_kx / (H W)
// for the adjoint of the real inverse transform.
__global__ void __launch_bounds__(kSpecThreads) k_tr_dft_y(const float2* __restrict__ x1,
                                                           float2* __restrict__ xh,
                                                           const float2* __restrict__ twy,
                                                           int H, int W, int C, int m,
                                                           int adjoint_scale) {
  extern __shared__ float sm[];
  float2* tw = reinterpret_cast<float2*>(sm);  // H
  float2* tile = tw + H;                        // [32][C]
  const int b = blockIdx.x / m, kx = blockIdx.x % m;
  for (int t = threadIdx.x; t < H; t += kSpecThreads) tw[t] = twy[t];
  const int G = kSpecThreads / C;
  const int c = threadIdx.x % C, g = threadIdx.x / C;
  float2 acc[kAccMax];
#pragma unroll
  for (int k = 0; k < kAccMax; ++k) acc[k] = make_float2(0.f, 0.f);
  for (int y0 = 0; y0 < H; y0 += 32) {
    const int ny = min(32, H - y0);
    __syncthreads();
    for (int j = threadIdx.x; j < ny * C; j += kSpecThreads) {
      const int yy = j / C, cc = j - yy * C;
      tile[j] = x1[(((size_t)b * H + y0 + yy) * m + kx) * C + cc];
    }
    __syncthreads();
    if (g < G) {
#pragma unroll
      for (int k = 0; k < kAccMax; ++k) {
        const int a = g + k * G;
        if (a < 2 * m) {
          const int ky = a < m ? a : H - 2 * m + a;
          int idx = (int)(((long long)ky * y0) % H);  // (ky y) mod H, advanced by ky per y
          for (int yy = 0; yy < ny; ++yy) {
            const float2 e = tw[idx];  // e^{+i}: use conj
            idx += ky;
            if (idx >= H) idx -= H;
            const float2 v = tile[yy * C + c];
            // v * conj(e)
            acc[k].x = fmaf(v.x, e.x, fmaf(v.y, e.y, acc[k].x));
            acc[k].y = fmaf(v.y, e.x, fmaf(-v.x, e.y, acc[k].y));
          }
        }
      }
    }
  }
  const float sc = adjoint_scale ? (kx == 0 ? 1.0f : 2.0f) / ((float)H * (float)W) : 1.0f;
  if (g < G) {
#pragma unroll
    for (int k = 0; k < kAccMax; ++k) {
      const int a = g + k * G;
      if (a < 2 * m)
        xh[(((size_t)b * 2 * m + a) * m + kx) * C + c] = make_float2(acc[k].x * sc, acc[k].y * sc);
    }
  }
}

// Per-mode channel mixing and its two adjoints (modes = 2 m m, Rt[mode][i][o]).
__global__ void k_tr_mix(const float2* __restrict__ xh, const float2* __restrict__ rt,
                         float2* __restrict__ yh, int B, int C, int modes) {
  const size_t n = (size_t)B * modes * C;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int o = (int)(t % C);
  const size_t bm = t / C;  // b * modes + mode
  const int mode = (int)(bm % modes);
  const float2* xr = xh + bm * C;
  const float2* rr = rt + (size_t)mode * C * C + o;
  float re = 0.f, im = 0.f;
  for (int i = 0; i < C; ++i) {
    const float2 x = xr[i], r = rr[(size_t)i * C];
    re = fmaf(x.x, r.x, fmaf(-x.y, r.y, re));
    im = fmaf(x.x, r.y, fmaf(x.y, r.x, im));
  }
  yh[t] = make_float2(re, im);
}
__global__ void k_tr_mix_bwd_x(const float2* __restrict__ dyh, const float2* __restrict__ rt,
                               float2* __restrict__ dxh, int B, int C, int modes) {
  const size_t n = (size_t)B * modes * C;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = (int)(t % C);
  const size_t bm = t / C;
  const int mode = (int)(bm % modes);
  const float2* dy = dyh + bm * C;
  const float2* rr = rt + ((size_t)mode * C + i) * C;
  float re = 0.f, im = 0.f;
  for (int o = 0; o < C; ++o) {  // dy * conj(r)
    const float2 d = dy[o], r = rr[o];
    re = fmaf(d.x, r.x, fmaf(d.y, r.y, re));
    im = fmaf(d.y, r.x, fmaf(-d.x, r.y, im));
  }
  dxh[t] = make_float2(re, im);
}
// dR[i][o][ky][kx] (re into r?re, im into r?im) = sum_b conj(X[b][mode][i]) dY[b][mode][o]
__global__ void k_tr_mix_bwd_r(const float2* __restrict__ xh, const float2* __restrict__ dyh,
                               float* __restrict__ dparams, size_t r1re, size_t r1im, size_t r2re,
                               size_t r2im, int B, int C, int m) {
  const int modes = 2 * m * m;
  const size_t n = (size_t)modes * C * C;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int o = (int)(t % C);
  const int i = (int)((t / C) % C);
  const int mode = (int)(t / ((size_t)C * C));
  float re = 0.f, im = 0.f;
  for (int b = 0; b < B; ++b) {
    const float2 x = xh[((size_t)b * modes + mode) * C + i];
    const float2 d = dyh[((size_t)b * modes + mode) * C + o];
    re = fmaf(x.x, d.x, fmaf(x.y, d.y, re));
    im = fmaf(x.x, d.y, fmaf(-x.y, d.x, im));
  }
  const int a = mode / m, kx = mode % m;
  const bool lo = a < m;
  const int ky = lo ? a : a - m;
  const size_t dst = (((size_t)i * C + o) * m + ky) * m + kx;
  dparams[(lo ? r1re : r2re) + dst] = re;
  dparams[(lo ? r1im : r2im) + dst] = im;
}

// Inverse y-DFT: Z[b][y][kx][c] = sum_a Yh[b][a][kx][c] e^{+2 pi i ky(a) y / H}.
__global__ void __launch_bounds__(kSpecThreads) k_tr_inv_y(const float2* __restrict__ yh,
                                                           float2* __restrict__ z,
                                                           const float2* __restrict__ twy,
                                                           int H, int C, int m) {
  extern __shared__ float sm[];
  float2* tw = reinterpret_cast<float2*>(sm);  // H
  float2* col = tw + H;                         // [2m][C]
  const int b = blockIdx.x / m, kx = blockIdx.x % m;
  for (int t = threadIdx.x; t < H; t += kSpecThreads) tw[t] = twy[t];
  for (int j = threadIdx.x; j < 2 * m * C; j += kSpecThreads) {
    const int a = j / C, c = j - a * C;
    col[j] = yh[(((size_t)b * 2 * m + a) * m + kx) * C + c];
  }
  __syncthreads();
  const int G = kSpecThreads / C;
  const int c = threadIdx.x % C, g = threadIdx.x / C;
  if (g >= G) return;
  for (int y = g; y < H; y += G) {
    float re = 0.f, im = 0.f;
    int idx = 0;  // (ky y) mod H for ky = 0 .. m-1, then H-m .. H-1
    for (int a = 0; a < 2 * m; ++a) {
      if (a == m) idx = (int)(((long long)(H - m) * y) % H);
      const float2 e = tw[idx];
      idx += y;
      if (idx >= H) idx -= H;
      const float2 v = col[a * C + c];
      re = fmaf(v.x, e.x, fmaf(-v.y, e.y, re));
      im = fmaf(v.x, e.y, fmaf(v.y, e.x, im));
    }
    z[(((size_t)b * H + y) * m + kx) * C + c] = make_float2(re, im);
  }
}

// Inverse x-DFT with real output: S[row][x][c] = scale sum_kx w(kx) Re(Z[row][kx][c]
// e^{+2 pi i kx x / W}); w(kx) = c_kx (forward) or 1 (adjoint of the forward DFT).
__global__ void __launch_bounds__(kSpecThreads) k_tr_inv_x(const float2* __restrict__ z,
                                                           float* __restrict__ s,
                                                           const float2* __restrict__ twx,
                                                           int W, int C, int m, float scale,
                                                           int hermitian) {
  extern __shared__ float sm[];
  float2* tw = reinterpret_cast<float2*>(sm);  // W
  float2* zr = tw + W;                          // [m][C]
  const size_t row = blockIdx.x;
  for (int t = threadIdx.x; t < W; t += kSpecThreads) tw[t] = twx[t];
  for (int j = threadIdx.x; j < m * C; j += kSpecThreads) {
    const int kx = j / C;
    float2 v = z[row * m * C + j];
    const float wk = (hermitian && kx > 0) ? 2.0f * scale : scale;
    zr[j] = make_float2(v.x * wk, v.y * wk);
  }
  __syncthreads();
  const int G = kSpecThreads / C;
  const int c = threadIdx.x % C, g = threadIdx.x / C;
  if (g >= G) return;
  for (int x = g; x < W; x += G) {
    float acc = 0.f;
    int idx = 0;  // (kx x) mod W
    for (int kx = 0; kx < m; ++kx) {
      const float2 e = tw[idx];
      idx += x;
      if (idx >= W) idx -= W;
      const float2 v = zr[kx * C + c];
      acc = fmaf(v.x, e.x, fmaf(-v.y, e.y, acc));
    }
    s[(row * W + x) * C + c] = acc;
  }
}

// NCHW <-> channels-last for the decoder output / its gradient
__global__ void k_tr_cl_to_nchw(const float* __restrict__ cl, float* __restrict__ out, int B,
                                int H, int W, int C) {
  const size_t n = (size_t)B * C * H * W;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const size_t hw = (size_t)H * W;
  const int b = (int)(t / (C * hw));
  const int c = (int)((t / hw) % C);
  const size_t q = t % hw;
  out[t] = cl[((size_t)b * hw + q) * C + c];
}
__global__ void k_tr_nchw_to_cl(const float* __restrict__ in, float* __restrict__ cl, int B, int H,
                                int W, int C) {
  const size_t n = (size_t)B * C * H * W;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const size_t hw = (size_t)H * W;
  const int b = (int)(t / (C * hw));
  const int c = (int)((t / hw) % C);
  const size_t q = t % hw;
  cl[((size_t)b * hw + q) * C + c] = in[t];
}
// din[b][c][y][x] = dxin[p][c] for the physical input channels
__global__ void k_tr_din(const float* __restrict__ dxin, float* __restrict__ din, int B, int H,
                         int W, int cin) {
  const size_t n = (size_t)B * cin * H * W;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const size_t hw = (size_t)H * W;
  const int b = (int)(t / (cin * hw));
  const int c = (int)((t / hw) % cin);
  const size_t q = t % hw;
  din[t] = dxin[((size_t)b * hw + q) * (cin + 2) + c];
}

inline unsigned nb(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

struct TrCtx {
  const fno_config* c;
  TrOff off;
  TrPlan pl;
  int B, H, W;
  cudaStream_t st;
  unsigned char* ws;
};

size_t pw_smem(int cin, int cout) {
  return sizeof(float) * ((size_t)cout * cin + (size_t)kPwPix * (cin + 1) + (size_t)kPwPix * (cout + 1));
}

int pw(const TrCtx& x, const float* in, int cin, const float* w, int trans, const float* bias,
       const float* add, int cout, float* pre, float* out, int in_act, int out_act) {
  const size_t smem = pw_smem(cin, cout);
  k_tr_pw<<<nb(x.pl.P, kPwPix), kPwPix, smem, x.st>>>(in, cin, w, trans, bias, add, cout, pre, out,
                                                      in_act, out_act, x.c->activation, x.pl.P);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int wgrad(const TrCtx& x, const float* dz, int cout, const float* in, int cin, int in_act,
          float* dw, float* db) {
  float* part = reinterpret_cast<float*>(x.ws + x.pl.part);
  k_tr_wgrad<<<x.pl.wg_blocks, kWgThreads, 0, x.st>>>(dz, cout, in, cin, in_act,
                                                      x.c->activation, x.pl.P, part);
  LBM_CHECK_LAUNCH();
  k_tr_wgrad_reduce<<<nb((size_t)cout * (cin + 1)), 256, 0, x.st>>>(part, x.pl.wg_blocks, cout,
                                                                    cin, dw, db);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

// X (or the adjoint-scaled dY) of a field: forward x-DFT then y-DFT over the kept rows.
int spectral_fwd(const TrCtx& x, const float* f, float2* out, int adjoint_scale) {
  const int C = x.c->width, m = x.c->modes;
  float2* x1 = reinterpret_cast<float2*>(x.ws + x.pl.x1);
  const float2* twx = reinterpret_cast<const float2*>(x.ws + x.pl.twx);
  const float2* twy = reinterpret_cast<const float2*>(x.ws + x.pl.twy);
  k_tr_dft_x<<<x.B * x.H, kSpecThreads, (2 * x.W + 32 * C) * sizeof(float), x.st>>>(f, x1, twx, x.W,
                                                                                    C, m);
  LBM_CHECK_LAUNCH();
  k_tr_dft_y<<<x.B * m, kSpecThreads, (x.H + 32 * C) * sizeof(float2), x.st>>>(
      x1, out, twy, x.H, x.W, C, m, adjoint_scale);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

// Real field from kept coefficients: inverse y-DFT then inverse x-DFT.
int spectral_inv(const TrCtx& x, const float2* coef, float* s, float scale, int hermitian) {
  const int C = x.c->width, m = x.c->modes;
  float2* z = reinterpret_cast<float2*>(x.ws + x.pl.z);
  const float2* twx = reinterpret_cast<const float2*>(x.ws + x.pl.twx);
  const float2* twy = reinterpret_cast<const float2*>(x.ws + x.pl.twy);
  k_tr_inv_y<<<x.B * m, kSpecThreads, (x.H + 2 * m * C) * sizeof(float2), x.st>>>(coef, z, twy,
                                                                                  x.H, C, m);
  LBM_CHECK_LAUNCH();
  k_tr_inv_x<<<x.B * x.H, kSpecThreads, (x.W + m * C) * sizeof(float2), x.st>>>(z, s, twx, x.W, C, m,
                                                                                scale, hermitian);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int set_smem_limits() {
  static bool done = false;
  if (done) return LBM_OK;
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_tr_pw, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)pw_smem(64, 64)));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_tr_dft_x, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((2 * 2048 + 32 * 64) * sizeof(float))));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_tr_dft_y, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((8192 + 32 * 64) * sizeof(float2))));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_tr_inv_y, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((8192 + 2 * kTrModesMax * 64) * sizeof(float2))));
  LBM_CHECK_CUDA(cudaFuncSetAttribute(k_tr_inv_x, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((2048 + kTrModesMax * 64) * sizeof(float2))));
  done = true;
  return LBM_OK;
}

int tr_setup(const fno_config* cfg, const float* params, int B, int H, int W, void* ws,
             void* stream, TrCtx* x) {
  LBM_REQUIRE(cfg != nullptr && params != nullptr && ws != nullptr, "fno_train: null argument");
  LBM_TRY(tr_offsets(*cfg, &x->off));
  LBM_REQUIRE(B >= 1 && H >= 2 && W >= 2 && H <= 8192 && W <= 2048,
              "fno_train: need B >= 1, 2 <= H <= 8192, 2 <= W <= 2048");
  LBM_REQUIRE(2 * cfg->modes <= H && cfg->modes <= W / 2, "fno_train: need 2m <= H and m <= W/2");
  LBM_REQUIRE((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "fno_train: ws must be 256-byte aligned");
  LBM_TRY(set_smem_limits());
  x->c = cfg;
  x->pl = tr_plan(*cfg, B, H, W);
  x->B = B;
  x->H = H;
  x->W = W;
  x->st = TS(stream);
  x->ws = static_cast<unsigned char*>(ws);
  k_tr_twiddle<<<nb(W), 256, 0, x->st>>>(reinterpret_cast<float2*>(x->ws + x->pl.twx), W);
  LBM_CHECK_LAUNCH();
  k_tr_twiddle<<<nb(H), 256, 0, x->st>>>(reinterpret_cast<float2*>(x->ws + x->pl.twy), H);
  LBM_CHECK_LAUNCH();
  // spectral filters per layer, transposed to [mode][i][o]
  RtOffs offs{};
  for (int n = 0; n < cfg->layers; ++n) {
    offs.v[4 * n + 0] = x->off.r1re[n];
    offs.v[4 * n + 1] = x->off.r1im[n];
    offs.v[4 * n + 2] = x->off.r2re[n];
    offs.v[4 * n + 3] = x->off.r2im[n];
  }
  const size_t nrt = (size_t)cfg->layers * 2 * cfg->modes * cfg->modes * cfg->width * cfg->width;
  k_tr_rt<<<(unsigned)std::min<size_t>(nb(nrt), 65535), 256, 0, x->st>>>(
      params, offs, reinterpret_cast<float2*>(x->ws + x->pl.rt), cfg->layers, cfg->width,
      cfg->modes);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

}  // namespace

}  // namespace lbmfno

using namespace lbmfno;

extern "C" {

int fno_train_query(const fno_config* cfg_h, int B, int H, int W, fno_train_sizes* out_h) {
  LBM_REQUIRE(cfg_h != nullptr && out_h != nullptr, "fno_train_query: null argument");
  TrOff off;
  LBM_TRY(tr_offsets(*cfg_h, &off));
  LBM_REQUIRE(B >= 1 && H >= 2 && W >= 2, "fno_train_query: bad shape");
  const TrPlan pl = tr_plan(*cfg_h, B, H, W);
  out_h->n_params = off.n;
  out_h->saved_bytes = pl.saved_floats * sizeof(float);
  out_h->ws_bytes = pl.ws_bytes;
  return LBM_OK;
}

int fno_train_forward(const fno_config* cfg_h, const float* params_d, const float* in_d,
                      float* out_d, int B, int H, int W, float* saved_d, void* ws_d,
                      void* stream) {
  LBM_REQUIRE(in_d != nullptr && out_d != nullptr && saved_d != nullptr,
              "fno_train_forward: null argument");
  TrCtx x;
  LBM_TRY(tr_setup(cfg_h, params_d, B, H, W, ws_d, stream, &x));
  const fno_config& c = *cfg_h;
  const TrPlan& pl = x.pl;
  const TrOff& o = x.off;
  const int C = c.width, h = C / 2, S = c.dec_size, m = c.modes;
  const size_t P = pl.P, spec = (size_t)B * 2 * m * m * C;
  float* xin = saved_d + pl.xin;
  float* h1pre = saved_d + pl.h1pre;
  auto theta = [&](int n) { return saved_d + pl.theta + (size_t)n * P * C; };
  auto zpre = [&](int n) { return saved_d + pl.zpre + (size_t)n * P * C; };
  auto xh = [&](int n) { return reinterpret_cast<float2*>(saved_d + pl.xh) + (size_t)n * spec; };
  auto hdpre = [&](int l) { return saved_d + pl.hdpre + (size_t)l * P * S; };
  float* ta = reinterpret_cast<float*>(x.ws + pl.ta);
  float* tb = reinterpret_cast<float*>(x.ws + pl.tb);
  float* s = reinterpret_cast<float*>(x.ws + pl.s);
  float2* yh = reinterpret_cast<float2*>(x.ws + pl.yh);
  const float2* rt = reinterpret_cast<const float2*>(x.ws + pl.rt);
  const float* p = params_d;

  k_tr_xin<<<nb(P), 256, 0, x.st>>>(in_d, xin, B, H, W, c.c_in);
  LBM_CHECK_LAUNCH();
  LBM_TRY(pw(x, xin, c.c_in + 2, p + o.lift0_w, 0, p + o.lift0_b, nullptr, h, h1pre, ta, 0, 1));
  LBM_TRY(pw(x, ta, h, p + o.lift1_w, 0, p + o.lift1_b, nullptr, C, nullptr, theta(0), 0, 0));
  for (int n = 0; n < c.layers; ++n) {
    LBM_TRY(spectral_fwd(x, theta(n), xh(n), 0));
    k_tr_mix<<<nb(spec), 256, 0, x.st>>>(xh(n), rt + (size_t)n * 2 * m * m * C * C, yh, B, C,
                                         2 * m * m);
    LBM_CHECK_LAUNCH();
    LBM_TRY(spectral_inv(x, yh, s, 1.0f / ((float)H * (float)W), 1));
    LBM_TRY(pw(x, theta(n), C, p + o.w[n], 0, p + o.b[n], s, C, zpre(n), theta(n + 1), 0, 1));
  }
  const float* hin = theta(c.layers);
  int fan = C;
  for (int l = 0; l < c.dec_layers; ++l) {
    float* hout = (l % 2 == 0) ? ta : tb;
    LBM_TRY(pw(x, hin, fan, p + o.dec_w[l], 0, p + o.dec_b[l], nullptr, S, hdpre(l), hout, 0, 1));
    hin = hout;
    fan = S;
  }
  float* ycl = reinterpret_cast<float*>(x.ws + pl.ycl);
  LBM_TRY(pw(x, hin, fan, p + o.out_w, 0, p + o.out_b, nullptr, c.c_out, nullptr, ycl, 0, 0));
  k_tr_cl_to_nchw<<<nb(P * c.c_out), 256, 0, x.st>>>(ycl, out_d, B, H, W, c.c_out);
  LBM_CHECK_LAUNCH();
  return LBM_OK;
}

int fno_train_backward(const fno_config* cfg_h, const float* params_d, const float* dout_d,
                       const float* saved_d, float* dparams_d, float* din_d, int B, int H, int W,
                       void* ws_d, void* stream) {
  LBM_REQUIRE(dout_d != nullptr && saved_d != nullptr && dparams_d != nullptr,
              "fno_train_backward: null argument");
  TrCtx x;
  LBM_TRY(tr_setup(cfg_h, params_d, B, H, W, ws_d, stream, &x));
  const fno_config& c = *cfg_h;
  const TrPlan& pl = x.pl;
  const TrOff& o = x.off;
  const int C = c.width, h = C / 2, S = c.dec_size, m = c.modes, act = c.activation;
  const size_t P = pl.P, spec = (size_t)B * 2 * m * m * C;
  const float* xin = saved_d + pl.xin;
  const float* h1pre = saved_d + pl.h1pre;
  auto theta = [&](int n) { return saved_d + pl.theta + (size_t)n * P * C; };
  auto zpre = [&](int n) { return saved_d + pl.zpre + (size_t)n * P * C; };
  auto xh = [&](int n) {
    return reinterpret_cast<const float2*>(saved_d + pl.xh) + (size_t)n * spec;
  };
  auto hdpre = [&](int l) { return saved_d + pl.hdpre + (size_t)l * P * S; };
  float* ta = reinterpret_cast<float*>(x.ws + pl.ta);
  float* tb = reinterpret_cast<float*>(x.ws + pl.tb);
  float* dz = reinterpret_cast<float*>(x.ws + pl.dz);
  float* s = reinterpret_cast<float*>(x.ws + pl.s);
  float2* dyh = reinterpret_cast<float2*>(x.ws + pl.dyh);
  float2* dxh = reinterpret_cast<float2*>(x.ws + pl.yh);
  const float2* rt = reinterpret_cast<const float2*>(x.ws + pl.rt);
  const float* p = params_d;
  float* dp = dparams_d;

  // decoder: output layer, then the hidden layers in reverse
  float* ycl = reinterpret_cast<float*>(x.ws + pl.ycl);
  k_tr_nchw_to_cl<<<nb(P * c.c_out), 256, 0, x.st>>>(dout_d, ycl, B, H, W, c.c_out);
  LBM_CHECK_LAUNCH();
  const int L = c.dec_layers;
  const int fan_last = S;
  LBM_TRY(wgrad(x, ycl, c.c_out, hdpre(L - 1), fan_last, 1, dp + o.out_w, dp + o.out_b));
  LBM_TRY(pw(x, ycl, c.c_out, p + o.out_w, 1, nullptr, nullptr, fan_last, nullptr, ta, 0, 0));
  float* g = ta;  // gradient with respect to the output of decoder layer L-1
  for (int l = L - 1; l >= 0; --l) {
    k_tr_act_bwd<<<nb(P * S), 256, 0, x.st>>>(g, hdpre(l), dz, P * S, act);
    LBM_CHECK_LAUNCH();
    const float* lin = (l == 0) ? theta(c.layers) : hdpre(l - 1);
    const int fan = (l == 0) ? C : S;
    LBM_TRY(wgrad(x, dz, S, lin, fan, l == 0 ? 0 : 1, dp + o.dec_w[l], dp + o.dec_b[l]));
    float* gn = (g == ta) ? tb : ta;
    LBM_TRY(pw(x, dz, S, p + o.dec_w[l], 1, nullptr, nullptr, fan, nullptr, gn, 0, 0));
    g = gn;
  }
  // Fourier layers in reverse: g = dL/dtheta_{n+1}
  for (int n = c.layers - 1; n >= 0; --n) {
    k_tr_act_bwd<<<nb(P * C), 256, 0, x.st>>>(g, zpre(n), dz, P * C, act);
    LBM_CHECK_LAUNCH();
    LBM_TRY(wgrad(x, dz, C, theta(n), C, 0, dp + o.w[n], dp + o.b[n]));
    LBM_TRY(spectral_fwd(x, dz, dyh, 1));
    k_tr_mix_bwd_r<<<nb((size_t)2 * m * m * C * C), 256, 0, x.st>>>(
        xh(n), dyh, dp, o.r1re[n], o.r1im[n], o.r2re[n], o.r2im[n], B, C, m);
    LBM_CHECK_LAUNCH();
    k_tr_mix_bwd_x<<<nb(spec), 256, 0, x.st>>>(dyh, rt + (size_t)n * 2 * m * m * C * C, dxh, B, C,
                                               2 * m * m);
    LBM_CHECK_LAUNCH();
    LBM_TRY(spectral_inv(x, dxh, s, 1.0f, 0));
    float* gn = (g == ta) ? tb : ta;
    LBM_TRY(pw(x, dz, C, p + o.w[n], 1, nullptr, s, C, nullptr, gn, 0, 0));
    g = gn;
  }
  // lifting network: g = dL/dtheta_0
  LBM_TRY(wgrad(x, g, C, h1pre, h, 1, dp + o.lift1_w, dp + o.lift1_b));
  float* gh = (g == ta) ? tb : ta;
  LBM_TRY(pw(x, g, C, p + o.lift1_w, 1, nullptr, nullptr, h, nullptr, gh, 0, 0));
  k_tr_act_bwd<<<nb(P * h), 256, 0, x.st>>>(gh, h1pre, dz, P * h, act);
  LBM_CHECK_LAUNCH();
  LBM_TRY(wgrad(x, dz, h, xin, c.c_in + 2, 0, dp + o.lift0_w, dp + o.lift0_b));
  if (din_d) {
    float* gx = (gh == ta) ? tb : ta;
    LBM_TRY(pw(x, dz, h, p + o.lift0_w, 1, nullptr, nullptr, c.c_in + 2, nullptr, gx, 0, 0));
    k_tr_din<<<nb(P * c.c_in), 256, 0, x.st>>>(gx, din_d, B, H, W, c.c_in);
    LBM_CHECK_LAUNCH();
  }
  return LBM_OK;
}

}  // extern "C"
