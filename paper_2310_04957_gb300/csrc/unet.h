// unet.h -- internal interface of the learned preconditioner's kernels.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace pic {
namespace unet {

// 3x3 convolution over an H x W NHWC image (p = y*W + x), zero padding.
// Input channels [in_off, in_off+Cin) of a tensor with in_cs channels per pixel.
// Weights w[cout][tap][cin], tap = 3*(dy+1) + (dx+1).
// Output: BF16 (out_bf, bias + optional ReLU) or FP32 (out_f, optionally
// accumulated and masked by mask > 0).
struct ConvArgs {
  const __nv_bfloat16 *in;
  int in_cs, in_off, Cin;
  __nv_bfloat16 *out_bf;
  float *out_f;
  int out_cs, out_off, Cout;
  const __nv_bfloat16 *w;
  const float *bias;
  const __nv_bfloat16 *mask;
  int mask_cs, mask_off;
  int H, W;
  int relu, accumulate;
  int *err;
};

// Weight gradient: dw[(tap*Cin + cin)*Cout + cout] += sum_p x[p+off(tap)][cin] dy[p][cout].
struct WgradArgs {
  const __nv_bfloat16 *x;
  int x_cs, x_off, Cin;
  const __nv_bfloat16 *dy;
  int dy_cs, dy_off, Cout;
  float *dw;
  int H, W, pix_per_cta;
  int *err;
};

cudaError_t launch_conv3x3(const ConvArgs &a, cudaStream_t st);
cudaError_t launch_wgrad(const WgradArgs &a, cudaStream_t st);

}  // namespace unet
}  // namespace pic
