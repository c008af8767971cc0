// Interface between the FNO front end (fno.cu) and its tensor-core path (fno_tc.cu).
#pragma once

#include "common.cuh"

namespace lbmfno {

// Workspace layout of the tensor-core path (byte offsets).
struct FnoTcWs {
  size_t theta0, theta1, x1b, xh, yb, zt, fw, ti, fy, ty, status, total;
};

// FP32 parameters of one FNO, already repacked on the device (channel dimensions padded
// to fno_tc_width with zeros when the width is not 16, 32 or 64).
struct FnoTcParams {
  const float *lift0_w, *lift0_b, *lift1_w, *lift1_b;
  const float2* rt[16];  // per layer: spectral filters [mode][C_in][C_out]
  const float* w[16];    // per layer: 1x1 weights [C_out][C_in]
  const float* b[16];    // per layer: bias
  const float* params;   // base of the FP32 parameter mirror (decoder offsets index it)
  const unsigned* dec_offs;
};

// Latent width of the tensor-core kernels for c.width channels (16, 32 or 64): the extra
// channels carry zero weights and stay exactly 0.
int fno_tc_width(int C);
bool fno_tc_supported(const fno_config& c, int H, int W);
FnoTcWs fno_tc_ws_plan(const fno_config& c, int B, int H, int W);
int fno_tc_prepare(const fno_config& c);
int fno_forward_tc(const fno_config& c, const FnoTcParams& P, const float* in, float* out, int B,
                   int H, int W, char* ws, cudaStream_t s);

}  // namespace lbmfno
