// unet.h -- internal interface of the learned preconditioner's kernels.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/pic.h"

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

// Tiling of the TMA-fed convolution.  A CTA computes `nmma` accumulators of
// 128 pixels x N output channels; each accumulator covers q = 128 / Wt image
// rows of a Wt-pixel-wide column strip, so a CTA covers R = nmma * q rows.
//   halo mode (nvar = 1, Wt = 128): one box of Bx = 130 pixels x By = R + 2 rows
//     per 8-channel group; tap (dy, dx) is the same box shifted by dy rows and
//     dx pixels (the MMA reads 128 contiguous pixels of one row).
//   column-copy mode (nvar = 3, Wt <= 64): three boxes of Bx = Wt pixels, read at
//     x0 - 1, x0, x0 + 1, so that tap (dy, dx) is box dx shifted by whole rows.
struct ConvGeom {
  int N, nmma, Wt, q, R, nvar, Bx, By;
  int slot;         // shared-memory bytes per box (128-byte multiple)
  int a_bytes;      // A bytes per stage: 2 groups x nvar boxes
  int stage_bytes;  // A + B (B = 2 groups x 9 taps x N rows x 16 bytes)
  int tx_bytes;     // bytes the TMA delivers per stage
  int S;            // pipeline stages
  int tiles_x, tiles_y, nsplit;
  int tcols, smem;
};

// Chooses a tiling for an H x W convolution with Cin -> Cout channels.  tile_n
// and tile_mma force N and nmma when nonzero.  Returns false when the shape has
// no TMA tiling (W not a multiple of 8, Cin or Cout not multiples of 16/32).
bool plan_conv(int H, int W, int Cin, int Cout, int tile_n, int tile_mma, ConvGeom *g);
// Tensor map of the BF16 NHWC input (cs channels per pixel) for tiling g.
cudaError_t make_input_map(CUtensorMap *m, const __nv_bfloat16 *base, int cs, int H, int W, const ConvGeom &g);
// w [Cout][9][Cin] -> packed [Cout/N][Cin/16][2][9][N][8], the per-stage shared-memory image.
cudaError_t pack_weights(const __nv_bfloat16 *w, int Cin, int Cout, int N, __nv_bfloat16 *dst, cudaStream_t st);
cudaError_t launch_conv_tma(const CUtensorMap &tin, const ConvArgs &a, const ConvGeom &g,
                            const __nv_bfloat16 *wpk, cudaStream_t st);

// Network forward (as pic_unet_forward) enqueued on stream s instead of the
// network's own stream (used to capture it into the solver's graph).
int forward_on_stream(pic_unet *u, const float *in, float *out, cudaStream_t s);
// Grid of the network.
void net_dims(const pic_unet *u, int *H, int *W);

// cp.async gather kernel (any W; Cin multiple of 16, Cout <= 256).
cudaError_t launch_conv3x3(const ConvArgs &a, cudaStream_t st);
cudaError_t launch_wgrad(const WgradArgs &a, cudaStream_t st);

}  // namespace unet
}  // namespace pic
