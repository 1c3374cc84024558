// unet.cu -- the learned field-solve preconditioner: a 4-level U-Net (32 base
// channels, BF16 weights and activations, FP32 accumulation) mapping
// (rho~, chi, boundary-voltage mask) on an H x W node grid to phi, with its
// forward and backward passes and an Adam optimiser, all on the GPU.
//
// Network (every conv 3x3 + bias + ReLU, except the final 1x1):
//   enc0: 16->32, 32->32 (e0)   pool2x2  enc1: 32->64, 64->64 (e1)   pool
//   enc2: 64->128, 128->128 (e2) pool    bottom: 128->256, 256->256 (b)
//   up(b)|e2: 384->128, 128->128 (d2)   up(d2)|e1: 192->64, 64->64 (d1)
//   up(d1)|e0: 96->32, 32->32 (d0)      out = 1x1 32->1
// Concatenation is free: encoders write into the channel slice of the
// decoder's input buffer.  Input channels: 0 = the scaled Jacobi value D^-1 r / s
// of the residual it is applied to, 1 = chi, 2 = Dirichlet mask, 3..15 = 0.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pic.h"
#include "unet.h"

using namespace pic::unet;

namespace {

constexpr int kNConv = 14;
constexpr int kCin[kNConv] = {16, 32, 32, 64, 64, 128, 128, 256, 384, 128, 192, 64, 96, 32};
constexpr int kCout[kNConv] = {32, 32, 64, 64, 128, 128, 256, 256, 128, 128, 64, 64, 32, 32};
constexpr int kLevel[kNConv] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};

struct Tensor {
  __nv_bfloat16 *p = nullptr;
  int cs = 0;  // channels per pixel
};

}  // namespace

struct pic_unet {
  int H = 0, W = 0;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  // parameters (per conv): bf16 W [cout][9][cin], flipped Wt [cin][9][cout], FP32 master, bias
  __nv_bfloat16 *w[kNConv], *wt[kNConv];
  float *wm[kNConv], *b[kNConv], *gw[kNConv], *gb[kNConv];
  float *mw[kNConv], *vw[kNConv], *mb[kNConv], *vb[kNConv];
  float *w_out = nullptr, *b_out = nullptr, *gw_out = nullptr, *m_out = nullptr, *v_out = nullptr;  // 33 values
  // activations
  Tensor in0, a0, cat0, pool0, a1, cat1, pool1, a2, cat2, pool2, b1, b2, d2a, d2, d1a, d1, d0a, d0;
  float *out = nullptr;
  // gradients (FP32) and the BF16 pre-activation gradient scratch
  float *g_d0, *g_d0a, *g_cat0, *g_d1, *g_d1a, *g_cat1, *g_d2, *g_d2a, *g_cat2, *g_b2, *g_b1, *g_pool2, *g_a2,
      *g_pool1, *g_a1, *g_pool0, *g_a0;
  __nv_bfloat16 *dpre = nullptr;
  int *err = nullptr;
  size_t nparams = 0;
  // TMA tilings, input tensor maps and packed weights of each forward conv (f)
  // and input-gradient conv (g); use_* false -> the cp.async gather kernel
  ConvGeom geo_f[kNConv], geo_g[kNConv];
  CUtensorMap map_f[kNConv], map_g[kNConv];
  bool use_f[kNConv] = {}, use_g[kNConv] = {};
  __nv_bfloat16 *wpk[kNConv], *wtpk[kNConv];
  bool tuning = false;  // set while pic_unet_create times the candidate tilings
  const float *last_out = nullptr;  // output of the last forward
  float *gout = nullptr;            // loss gradient scratch [H*W]
  double *loss_sums = nullptr;      // [2]
};

namespace {

#define UK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      fprintf(stderr, "pic_unet: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      return PIC_ECUDA;                                                           \
    }                                                                             \
  } while (0)

template <typename P>
int ualloc(pic_unet *u, P **ptr, size_t bytes) {
  void *p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    return PIC_ENOMEM;
  }
  cudaMemsetAsync(p, 0, bytes ? bytes : 16, u->stream);
  u->allocs.push_back(p);
  *ptr = reinterpret_cast<P *>(p);
  return PIC_OK;
}

#define UA(ptr, bytes)                     \
  do {                                     \
    int st_ = ualloc(u, &(ptr), (bytes));  \
    if (st_) return st_;                   \
  } while (0)

int pixels(const pic_unet *u, int level) { return (u->H >> level) * (u->W >> level); }

// ---- elementwise kernels ------------------------------------------------------------
__global__ void k_pack_input(const float *src, int HW, __nv_bfloat16 *dst) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    __align__(16) __nv_bfloat16 h[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) h[c] = __float2bfloat16(c < 3 ? src[(size_t)c * HW + p] : 0.0f);
    uint4 *o = reinterpret_cast<uint4 *>(dst + (size_t)p * 16);
    o[0] = reinterpret_cast<const uint4 *>(h)[0];
    o[1] = reinterpret_cast<const uint4 *>(h)[1];
  }
}

// 2x2 average pool: src (h x w, channels [off, off+C) of cs) -> dst (h/2 x w/2 x C).
// One thread per 8 channels of an output pixel (16-byte loads and stores).
__global__ void k_pool(const __nv_bfloat16 *src, int cs, int off, int C, int h, int w, __nv_bfloat16 *dst) {
  const int ho = h / 2, wo = w / 2, C8 = C / 8;
  const int n = ho * wo * C8;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = (i % C8) * 8, q = i / C8, y = q / wo, x = q - y * wo;
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        __align__(16) __nv_bfloat16 v[8];
        *reinterpret_cast<uint4 *>(v) =
            *reinterpret_cast<const uint4 *>(src + ((size_t)(2 * y + dy) * w + 2 * x + dx) * cs + off + c);
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] += __bfloat162float(v[k]);
      }
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16(0.25f * s[k]);
    *reinterpret_cast<uint4 *>(dst + (size_t)q * C + c) = *reinterpret_cast<const uint4 *>(o);
  }
}

// Nearest 2x upsample of src (h x w x C) into channels [0, C) of dst (2h x 2w, cs).
// One thread per 8 channels of an output pixel.
__global__ void k_upsample(const __nv_bfloat16 *src, int C, int h, int w, __nv_bfloat16 *dst, int cs) {
  const int C8 = C / 8, W2 = 2 * w;
  const int n = 4 * h * w * C8;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = (i % C8) * 8, q = i / C8, y = q / W2, x = q - y * W2;
    *reinterpret_cast<uint4 *>(dst + (size_t)q * cs + c) =
        *reinterpret_cast<const uint4 *>(src + ((size_t)(y / 2) * w + x / 2) * C + c);
  }
}

// Upsample backward: g_src[y][x][c] = sum of the 4 children g[2y+dy][2x+dx][c] (channels [0,C) of gcs).
__global__ void k_upsample_bwd(const float *g, int gcs, int C, int h, int w, float *g_src) {
  int n = h * w * C;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c = i % C, q = i / C, y = q / w, x = q - y * w;
    float s = 0.0f;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) s += g[((size_t)(2 * y + dy) * (2 * w) + 2 * x + dx) * gcs + c];
    g_src[i] = s;
  }
}

// Pool backward into a slice: g[child][off+c] += g_pool/4 * (act[child][off+c] > 0).
__global__ void k_pool_bwd(const float *gp, int C, int h, int w, float *g, const __nv_bfloat16 *act, int cs, int off) {
  int ho = h / 2, wo = w / 2, n = ho * wo * C;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c = i % C, q = i / C, y = q / wo, x = q - y * wo;
    float v = 0.25f * gp[i];
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        size_t k = ((size_t)(2 * y + dy) * w + 2 * x + dx) * cs + off + c;
        if (__bfloat162float(act[k]) > 0.0f) g[k] += v;
      }
  }
}

// Gradient (FP32 slice) -> BF16 dense pre-activation gradient, with the bias
// gradient.  One thread per 8 channels; the grid stride is a multiple of C/8,
// so each thread keeps one channel group and sums it in registers.
__global__ void k_to_bf16_bias(const float *g, int cs, int off, int C, int HW, __nv_bfloat16 *dst, float *gb) {
  extern __shared__ float sb[];
  for (int c = threadIdx.x; c < C; c += blockDim.x) sb[c] = 0.0f;
  __syncthreads();
  const int C8 = C / 8, n = HW * C8;
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = i0; i < n; i += gridDim.x * blockDim.x) {
    const int c = (i % C8) * 8, p = i / C8;
    const float4 *src = reinterpret_cast<const float4 *>(g + (size_t)p * cs + off + c);
    const float4 a = src[0], b = src[1];
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      h[k] = __float2bfloat16(v[k]);
      acc[k] += __bfloat162float(h[k]);
    }
    *reinterpret_cast<uint4 *>(dst + (size_t)p * C + c) = *reinterpret_cast<const uint4 *>(h);
  }
  if (i0 < n) {
    const int c = (i0 % C8) * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) atomicAdd(&sb[c + k], acc[k]);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&gb[c], sb[c]);
}

// 1x1 output conv: out[p] = b + sum_c w[c] d0[p][c].
__global__ void k_out_fwd(const __nv_bfloat16 *d0, int HW, const float *w, const float *b, float *out) {
  __shared__ float sw[33];
  if (threadIdx.x < 33) sw[threadIdx.x] = w[threadIdx.x];  // w[32] is the bias
  __syncthreads();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    float s = sw[32];
    const uint4 *src = reinterpret_cast<const uint4 *>(d0 + (size_t)p * 32);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __align__(16) __nv_bfloat16 v[8];
      *reinterpret_cast<uint4 *>(v) = src[q];
#pragma unroll
      for (int k = 0; k < 8; ++k) s += sw[8 * q + k] * __bfloat162float(v[k]);
    }
    out[p] = s;
  }
}

// 1x1 backward: g_d0[p][c] = gout[p] w[c] (d0 > 0); gw[c] += sum gout d0; gw[32] += sum gout.
__global__ void k_out_bwd(const float *gout, const __nv_bfloat16 *d0, int HW, const float *w, float *g_d0, float *gw) {
  __shared__ float s[33];
  __shared__ float sw[32];
  if (threadIdx.x < 33) s[threadIdx.x] = 0.0f;
  if (threadIdx.x < 32) sw[threadIdx.x] = w[threadIdx.x];
  __syncthreads();
  float acc[33];
#pragma unroll
  for (int c = 0; c < 33; ++c) acc[c] = 0.0f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    const float go = gout[p];
    const uint4 *src = reinterpret_cast<const uint4 *>(d0 + (size_t)p * 32);
    float4 *dst = reinterpret_cast<float4 *>(g_d0 + (size_t)p * 32);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __align__(16) __nv_bfloat16 v[8];
      *reinterpret_cast<uint4 *>(v) = src[q];
      float o[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float a = __bfloat162float(v[k]);
        o[k] = a > 0.0f ? go * sw[8 * q + k] : 0.0f;
        acc[8 * q + k] += go * a;
      }
      dst[2 * q] = make_float4(o[0], o[1], o[2], o[3]);
      dst[2 * q + 1] = make_float4(o[4], o[5], o[6], o[7]);
    }
    acc[32] += go;
  }
#pragma unroll
  for (int c = 0; c < 33; ++c) {
    float v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s[c], v);
  }
  __syncthreads();
  if (threadIdx.x < 33) atomicAdd(&gw[threadIdx.x], s[threadIdx.x]);
}

// Relative L2 loss over free pixels (mask channel == 0): sums t^2 and (o-t)^2.
__global__ void k_loss_sums(const float *o, const float *t, const float *mask, int HW, double *sums) {
  double a = 0.0, b = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    if (mask[p] != 0.0f) continue;
    const double tv = t[p], d = (double)o[p] - tv;
    a += tv * tv;
    b += d * d;
  }
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], b);
  }
}

// dL/do = 2 (o - t) / sum t^2 on free pixels; adds L to *loss.
__global__ void k_loss_grad(const float *o, const float *t, const float *mask, int HW, const double *sums, float *g,
                            float *loss) {
  const double t2 = sums[0] > 0.0 ? sums[0] : 1.0;
  const float sc = (float)(2.0 / t2);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x)
    g[p] = mask[p] != 0.0f ? 0.0f : sc * (o[p] - t[p]);
  if (loss && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(loss, (float)(sums[1] / t2));
}

// Adam on one conv layer: master W [cout][9][cin] from gradient gWt [(tap*cin+ci)*cout+co];
// writes BF16 W and the flipped transpose Wt[ci][8-tap][co] used by the input gradient.
__global__ void k_adam_conv(int Cin, int Cout, float *wm, const float *gwt, float *m, float *v, __nv_bfloat16 *w,
                            __nv_bfloat16 *wt, float lr, float b1, float b2, float eps, float c1, float c2) {
  int n = Cout * 9 * Cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int ci = i % Cin, t = (i / Cin) % 9, co = i / (9 * Cin);
    float g = gwt[((size_t)t * Cin + ci) * Cout + co];
    if (lr > 0.0f) {
      float mi = b1 * m[i] + (1.0f - b1) * g, vi = b2 * v[i] + (1.0f - b2) * g * g;
      m[i] = mi;
      v[i] = vi;
      wm[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
    __nv_bfloat16 h = __float2bfloat16(wm[i]);
    w[i] = h;
    wt[((size_t)ci * 9 + (8 - t)) * Cout + co] = h;
  }
}

__global__ void k_adam_vec(int n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

ConvArgs conv_args(pic_unet *u, const Tensor &in, int in_off, int Cin, int level) {
  ConvArgs a;
  memset(&a, 0, sizeof(a));
  a.in = in.p;
  a.in_cs = in.cs;
  a.in_off = in_off;
  a.Cin = Cin;
  a.H = u->H >> level;
  a.W = u->W >> level;
  a.err = u->err;
  return a;
}

// Autotuner: times every TMA tiling of one convolution (two warm-up and five
// timed launches on the network's own buffers) and keeps the fastest.
template <class Launch>
int tune_conv(pic_unet *u, int h, int w, int Cin, int Cout, const __nv_bfloat16 *inp, int in_cs, ConvGeom *geo,
              CUtensorMap *map, Launch launch) {
  cudaEvent_t e0, e1;
  UK(cudaEventCreate(&e0));
  UK(cudaEventCreate(&e1));
  float best = 1e30f;
  const int ns[4] = {32, 64, 128, 256};
  for (int ni = 0; ni < 4; ++ni)
    for (int m = 1; m <= 8; m *= 2) {
      ConvGeom g;
      CUtensorMap mp;
      if (!plan_conv(h, w, Cin, Cout, ns[ni], m, &g)) continue;
      if (make_input_map(&mp, inp, in_cs, h, w, g) != cudaSuccess) continue;
      for (int r = 0; r < 2; ++r) UK(launch(mp, g));
      UK(cudaEventRecord(e0, u->stream));
      for (int r = 0; r < 5; ++r) UK(launch(mp, g));
      UK(cudaEventRecord(e1, u->stream));
      UK(cudaEventSynchronize(e1));
      float ms = 0.0f;
      UK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        *geo = g;
        *map = mp;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return PIC_OK;
}

int conv_fwd(pic_unet *u, int l, const Tensor &in, int in_off, const Tensor &out, int out_off) {
  ConvArgs a = conv_args(u, in, in_off, kCin[l], kLevel[l]);
  a.out_bf = out.p;
  a.out_cs = out.cs;
  a.out_off = out_off;
  a.Cout = kCout[l];
  a.w = u->w[l];
  a.bias = u->b[l];
  a.relu = 1;
  if (u->use_f[l] && u->tuning) {
    int st = tune_conv(u, a.H, a.W, a.Cin, a.Cout, in.p, in.cs, &u->geo_f[l], &u->map_f[l],
                       [&](const CUtensorMap &m, const ConvGeom &g) { return launch_conv_tma(m, a, g, u->wpk[l], u->stream); });
    if (st) return st;
  }
  if (u->use_f[l])
    UK(launch_conv_tma(u->map_f[l], a, u->geo_f[l], u->wpk[l], u->stream));
  else
    UK(launch_conv3x3(a, u->stream));
  return PIC_OK;
}

// Backward of conv l: dPre (BF16) from the FP32 gradient slice of its output,
// bias gradient, weight gradient, and (if g_in) the input gradient masked by
// in > 0 when `mask_in`.
int conv_bwd(pic_unet *u, int l, const Tensor &in, int in_off, const float *g_out, int g_cs, int g_off, float *g_in,
             int g_in_cs, int g_in_off, bool mask_in, bool accumulate) {
  const int level = kLevel[l], HW = pixels(u, level), Cin = kCin[l], Cout = kCout[l];
  k_to_bf16_bias<<<grid_for((long long)HW * Cout / 8), 256, Cout * sizeof(float), u->stream>>>(g_out, g_cs, g_off, Cout, HW,
                                                                                         u->dpre, u->gb[l]);
  UK(cudaGetLastError());
  WgradArgs wa;
  memset(&wa, 0, sizeof(wa));
  wa.x = in.p;
  wa.x_cs = in.cs;
  wa.x_off = in_off;
  wa.Cin = Cin;
  wa.dy = u->dpre;
  wa.dy_cs = Cout;
  wa.dy_off = 0;
  wa.Cout = Cout;
  wa.dw = u->gw[l];
  wa.H = u->H >> level;
  wa.W = u->W >> level;
  wa.pix_per_cta = HW >= 65536 ? 1024 : (HW >= 8192 ? 512 : 256);
  wa.err = u->err;
  UK(launch_wgrad(wa, u->stream));
  if (g_in && u->use_g[l]) {
    // input gradient = conv with the flipped transposed weights Wt[cin][9][cout]
    Tensor dp{u->dpre, Cout};
    ConvArgs a = conv_args(u, dp, 0, Cout, level);
    a.out_f = g_in;
    a.out_cs = g_in_cs;
    a.out_off = g_in_off;
    a.Cout = Cin;
    a.w = u->wt[l];
    a.mask = mask_in ? in.p : nullptr;
    a.mask_cs = in.cs;
    a.mask_off = in_off;
    a.accumulate = accumulate ? 1 : 0;
    if (u->tuning) {
      int st = tune_conv(u, a.H, a.W, a.Cin, a.Cout, u->dpre, Cout, &u->geo_g[l], &u->map_g[l],
                         [&](const CUtensorMap &m, const ConvGeom &g) { return launch_conv_tma(m, a, g, u->wtpk[l], u->stream); });
      if (st) return st;
    }
    UK(launch_conv_tma(u->map_g[l], a, u->geo_g[l], u->wtpk[l], u->stream));
  } else if (g_in) {
    // gather kernel, in output-channel chunks of at most 256 (the accumulator width)
    Tensor dp{u->dpre, Cout};
    for (int c0 = 0; c0 < Cin; c0 += 256) {
      const int nc = Cin - c0 < 256 ? Cin - c0 : 256;
      ConvArgs a = conv_args(u, dp, 0, Cout, level);
      a.out_f = g_in;
      a.out_cs = g_in_cs;
      a.out_off = g_in_off + c0;
      a.Cout = nc;
      a.w = u->wt[l] + (size_t)c0 * 9 * Cout;
      a.mask = mask_in ? in.p : nullptr;
      a.mask_cs = in.cs;
      a.mask_off = in_off + c0;
      a.accumulate = accumulate ? 1 : 0;
      UK(launch_conv3x3(a, u->stream));
    }
  }
  return PIC_OK;
}

int refresh_weights(pic_unet *u, float lr, float b1, float b2, float eps, int t) {
  float c1 = lr > 0 ? 1.0f - powf(b1, (float)t) : 1.0f, c2 = lr > 0 ? 1.0f - powf(b2, (float)t) : 1.0f;
  for (int l = 0; l < kNConv; ++l) {
    int n = kCout[l] * 9 * kCin[l];
    k_adam_conv<<<grid_for(n), 256, 0, u->stream>>>(kCin[l], kCout[l], u->wm[l], u->gw[l], u->mw[l], u->vw[l], u->w[l],
                                                     u->wt[l], lr, b1, b2, eps, c1, c2);
    UK(cudaGetLastError());
    if (u->use_f[l]) UK(pack_weights(u->w[l], kCin[l], kCout[l], u->geo_f[l].N, u->wpk[l], u->stream));
    if (u->use_g[l]) UK(pack_weights(u->wt[l], kCout[l], kCin[l], u->geo_g[l].N, u->wtpk[l], u->stream));
    if (lr > 0) {
      k_adam_vec<<<1, 256, 0, u->stream>>>(kCout[l], u->b[l], u->gb[l], u->mb[l], u->vb[l], lr, b1, b2, eps, c1, c2);
      UK(cudaGetLastError());
    }
  }
  if (lr > 0) {
    k_adam_vec<<<1, 64, 0, u->stream>>>(33, u->w_out, u->gw_out, u->m_out, u->v_out, lr, b1, b2, eps, c1, c2);
    UK(cudaGetLastError());
  }
  return PIC_OK;
}

}  // namespace

extern "C" {

int pic_unet_create(int H, int W, void *cuda_stream, pic_unet **out) {
  if (!out || H < 16 || W < 16 || H % 8 || W % 8 || (long long)H * W > (1 << 24)) return PIC_EINVAL;
  *out = nullptr;
  pic_unet *u = new (std::nothrow) pic_unet();
  if (!u) return PIC_ENOMEM;
  u->H = H;
  u->W = W;
  u->stream = (cudaStream_t)cuda_stream;
  int st = [&]() -> int {
    size_t np = 0;
    for (int l = 0; l < kNConv; ++l) {
      size_t n = (size_t)kCout[l] * 9 * kCin[l];
      np += n + kCout[l];
      UA(u->w[l], n * 2);
      UA(u->wt[l], n * 2);
      UA(u->wm[l], n * 4);
      UA(u->gw[l], n * 4);
      UA(u->mw[l], n * 4);
      UA(u->vw[l], n * 4);
      UA(u->b[l], kCout[l] * 4);
      UA(u->gb[l], kCout[l] * 4);
      UA(u->mb[l], kCout[l] * 4);
      UA(u->vb[l], kCout[l] * 4);
    }
    np += 33;
    u->nparams = np;
    UA(u->w_out, 33 * 4);
    u->b_out = u->w_out + 32;
    UA(u->gw_out, 33 * 4);
    UA(u->m_out, 33 * 4);
    UA(u->v_out, 33 * 4);
    auto T = [&](Tensor &t, int level, int C) -> int {
      t.cs = C;
      return ualloc(u, &t.p, (size_t)pixels(u, level) * C * 2);
    };
    int e = 0;
    e |= T(u->in0, 0, 16); e |= T(u->a0, 0, 32); e |= T(u->cat0, 0, 96); e |= T(u->pool0, 1, 32);
    e |= T(u->a1, 1, 64); e |= T(u->cat1, 1, 192); e |= T(u->pool1, 2, 64); e |= T(u->a2, 2, 128);
    e |= T(u->cat2, 2, 384); e |= T(u->pool2, 3, 128); e |= T(u->b1, 3, 256); e |= T(u->b2, 3, 256);
    e |= T(u->d2a, 2, 128); e |= T(u->d2, 2, 128); e |= T(u->d1a, 1, 64); e |= T(u->d1, 1, 64);
    e |= T(u->d0a, 0, 32); e |= T(u->d0, 0, 32);
    if (e) return PIC_ENOMEM;
    size_t p0 = pixels(u, 0), p1 = pixels(u, 1), p2 = pixels(u, 2), p3 = pixels(u, 3);
    UA(u->out, p0 * 4);
    UA(u->g_d0, p0 * 32 * 4); UA(u->g_d0a, p0 * 32 * 4); UA(u->g_cat0, p0 * 96 * 4); UA(u->g_d1, p1 * 64 * 4);
    UA(u->g_d1a, p1 * 64 * 4); UA(u->g_cat1, p1 * 192 * 4); UA(u->g_d2, p2 * 128 * 4); UA(u->g_d2a, p2 * 128 * 4);
    UA(u->g_cat2, p2 * 384 * 4); UA(u->g_b2, p3 * 256 * 4); UA(u->g_b1, p3 * 256 * 4); UA(u->g_pool2, p3 * 128 * 4);
    UA(u->g_a2, p2 * 128 * 4); UA(u->g_pool1, p2 * 64 * 4); UA(u->g_a1, p1 * 64 * 4); UA(u->g_pool0, p1 * 32 * 4);
    UA(u->g_a0, p0 * 32 * 4);
    UA(u->dpre, p0 * 64 * 2);  // largest Cout x pixels among the layers
    UA(u->gout, p0 * 4);
    UA(u->loss_sums, 2 * sizeof(double));
    UA(u->err, 16);
    // TMA tilings and tensor maps (input buffers are fixed for the network's life)
    const Tensor *fin[kNConv] = {&u->in0, &u->a0, &u->pool0, &u->a1, &u->pool1, &u->a2, &u->pool2,
                                 &u->b1, &u->cat2, &u->d2a, &u->cat1, &u->d1a, &u->cat0, &u->d0a};
    for (int l = 0; l < kNConv; ++l) {
      const int h = H >> kLevel[l], w = W >> kLevel[l];
      size_t n = (size_t)kCout[l] * 9 * kCin[l];
      if (plan_conv(h, w, kCin[l], kCout[l], 0, 0, &u->geo_f[l]) &&
          make_input_map(&u->map_f[l], fin[l]->p, fin[l]->cs, h, w, u->geo_f[l]) == cudaSuccess) {
        u->use_f[l] = true;
        UA(u->wpk[l], n * 2);
      }
      if (l > 0 && plan_conv(h, w, kCout[l], kCin[l], 0, 0, &u->geo_g[l]) &&
          make_input_map(&u->map_g[l], u->dpre, kCout[l], h, w, u->geo_g[l]) == cudaSuccess) {
        u->use_g[l] = true;
        UA(u->wtpk[l], n * 2);
      }
    }
    if (cudaStreamSynchronize(u->stream) != cudaSuccess) return PIC_ECUDA;
    // choose each convolution's tiling by timing (all weights and inputs are zero here)
    float *zero = nullptr;
    if (cudaMalloc(&zero, (size_t)p0 * 3 * 4) != cudaSuccess) return PIC_ENOMEM;
    cudaMemsetAsync(zero, 0, (size_t)p0 * 3 * 4, u->stream);
    u->tuning = true;
    int t = pic_unet_forward(u, zero, nullptr);
    if (!t) t = pic_unet_backward(u, zero);
    u->tuning = false;
    if (cudaStreamSynchronize(u->stream) != cudaSuccess) t = PIC_ECUDA;
    cudaFree(zero);
    if (!t) t = pic_unet_zero_grads(u);
    if (!t && cudaMemsetAsync(u->err, 0, 16, u->stream) != cudaSuccess) t = PIC_ECUDA;
    if (!t && cudaStreamSynchronize(u->stream) != cudaSuccess) t = PIC_ECUDA;
    return t;
  }();
  if (st) {
    for (void *p : u->allocs) cudaFree(p);
    delete u;
    return st;
  }
  *out = u;
  return PIC_OK;
}

void pic_unet_destroy(pic_unet *u) {
  if (!u) return;
  if (u->stream) cudaStreamSynchronize(u->stream);
  for (void *p : u->allocs) cudaFree(p);
  delete u;
}

int pic_unet_param_count(const pic_unet *u, int64_t *n) {
  if (!u || !n) return PIC_EINVAL;
  *n = (int64_t)u->nparams;
  return PIC_OK;
}

// Parameters in order: for each conv l, W[cout][9][cin] then bias[cout]; then the
// 1x1 output weights [32] and bias [1].
int pic_unet_set_params(pic_unet *u, const float *host, int64_t n) {
  if (!u || !host || n != (int64_t)u->nparams) return PIC_EINVAL;
  size_t o = 0;
  for (int l = 0; l < kNConv; ++l) {
    size_t nw = (size_t)kCout[l] * 9 * kCin[l];
    UK(cudaMemcpyAsync(u->wm[l], host + o, nw * 4, cudaMemcpyHostToDevice, u->stream));
    o += nw;
    UK(cudaMemcpyAsync(u->b[l], host + o, kCout[l] * 4, cudaMemcpyHostToDevice, u->stream));
    o += kCout[l];
  }
  UK(cudaMemcpyAsync(u->w_out, host + o, 33 * 4, cudaMemcpyHostToDevice, u->stream));
  int st = refresh_weights(u, 0.0f, 0.9f, 0.999f, 1e-8f, 1);
  if (st) return st;
  UK(cudaStreamSynchronize(u->stream));
  return PIC_OK;
}

static int copy_params(pic_unet *u, float *host, int64_t n, bool grads) {
  if (!u || !host || n != (int64_t)u->nparams) return PIC_EINVAL;
  UK(cudaStreamSynchronize(u->stream));
  size_t o = 0;
  std::vector<float> tmp;
  for (int l = 0; l < kNConv; ++l) {
    size_t nw = (size_t)kCout[l] * 9 * kCin[l];
    if (grads) {
      // device holds dWt[(tap*cin+ci)*cout+co]; return dW[co][tap][ci]
      tmp.resize(nw);
      UK(cudaMemcpy(tmp.data(), u->gw[l], nw * 4, cudaMemcpyDeviceToHost));
      for (int co = 0; co < kCout[l]; ++co)
        for (int t = 0; t < 9; ++t)
          for (int ci = 0; ci < kCin[l]; ++ci)
            host[o + ((size_t)co * 9 + t) * kCin[l] + ci] = tmp[((size_t)t * kCin[l] + ci) * kCout[l] + co];
    } else {
      UK(cudaMemcpy(host + o, u->wm[l], nw * 4, cudaMemcpyDeviceToHost));
    }
    o += nw;
    UK(cudaMemcpy(host + o, grads ? u->gb[l] : u->b[l], kCout[l] * 4, cudaMemcpyDeviceToHost));
    o += kCout[l];
  }
  UK(cudaMemcpy(host + o, grads ? u->gw_out : u->w_out, 33 * 4, cudaMemcpyDeviceToHost));
  return PIC_OK;
}

int pic_unet_get_params(pic_unet *u, float *host, int64_t n) { return copy_params(u, host, n, false); }
int pic_unet_get_grads(pic_unet *u, float *host, int64_t n) { return copy_params(u, host, n, true); }

int pic_unet_zero_grads(pic_unet *u) {
  if (!u) return PIC_EINVAL;
  for (int l = 0; l < kNConv; ++l) {
    UK(cudaMemsetAsync(u->gw[l], 0, (size_t)kCout[l] * 9 * kCin[l] * 4, u->stream));
    UK(cudaMemsetAsync(u->gb[l], 0, kCout[l] * 4, u->stream));
  }
  UK(cudaMemsetAsync(u->gw_out, 0, 33 * 4, u->stream));
  return PIC_OK;
}

// Forward: in = device FP32 [3][H*W] (channel-major), out = device FP32 [H*W].
int pic_unet_forward(pic_unet *u, const float *in, float *out) {
  if (!u || !in) return PIC_EINVAL;
  const int H = u->H, W = u->W;
  cudaStream_t s = u->stream;
  k_pack_input<<<grid_for(H * W), 256, 0, s>>>(in, H * W, u->in0.p);
  UK(cudaGetLastError());
  int st = 0;
  st |= conv_fwd(u, 0, u->in0, 0, u->a0, 0);
  st |= conv_fwd(u, 1, u->a0, 0, u->cat0, 64);
  k_pool<<<grid_for((long long)pixels(u, 1) * 4), 256, 0, s>>>(u->cat0.p, 96, 64, 32, H, W, u->pool0.p);
  st |= conv_fwd(u, 2, u->pool0, 0, u->a1, 0);
  st |= conv_fwd(u, 3, u->a1, 0, u->cat1, 128);
  k_pool<<<grid_for((long long)pixels(u, 2) * 8), 256, 0, s>>>(u->cat1.p, 192, 128, 64, H >> 1, W >> 1, u->pool1.p);
  st |= conv_fwd(u, 4, u->pool1, 0, u->a2, 0);
  st |= conv_fwd(u, 5, u->a2, 0, u->cat2, 256);
  k_pool<<<grid_for((long long)pixels(u, 3) * 16), 256, 0, s>>>(u->cat2.p, 384, 256, 128, H >> 2, W >> 2, u->pool2.p);
  st |= conv_fwd(u, 6, u->pool2, 0, u->b1, 0);
  st |= conv_fwd(u, 7, u->b1, 0, u->b2, 0);
  k_upsample<<<grid_for((long long)pixels(u, 2) * 32), 256, 0, s>>>(u->b2.p, 256, H >> 3, W >> 3, u->cat2.p, 384);
  st |= conv_fwd(u, 8, u->cat2, 0, u->d2a, 0);
  st |= conv_fwd(u, 9, u->d2a, 0, u->d2, 0);
  k_upsample<<<grid_for((long long)pixels(u, 1) * 16), 256, 0, s>>>(u->d2.p, 128, H >> 2, W >> 2, u->cat1.p, 192);
  st |= conv_fwd(u, 10, u->cat1, 0, u->d1a, 0);
  st |= conv_fwd(u, 11, u->d1a, 0, u->d1, 0);
  k_upsample<<<grid_for((long long)pixels(u, 0) * 8), 256, 0, s>>>(u->d1.p, 64, H >> 1, W >> 1, u->cat0.p, 96);
  st |= conv_fwd(u, 12, u->cat0, 0, u->d0a, 0);
  st |= conv_fwd(u, 13, u->d0a, 0, u->d0, 0);
  k_out_fwd<<<grid_for(H * W), 256, 0, s>>>(u->d0.p, H * W, u->w_out, u->b_out, out ? out : u->out);
  UK(cudaGetLastError());
  u->last_out = out ? out : u->out;
  return st ? PIC_ECUDA : PIC_OK;
}

// Backward of the last forward: gout = device FP32 [H*W] = dLoss/dout.  Adds the
// parameter gradients to the accumulators (zero them with pic_unet_zero_grads).
int pic_unet_backward(pic_unet *u, const float *gout) {
  if (!u || !gout) return PIC_EINVAL;
  const int H = u->H, W = u->W;
  cudaStream_t s = u->stream;
  const size_t p0 = pixels(u, 0), p1 = pixels(u, 1), p2 = pixels(u, 2);
  k_out_bwd<<<grid_for(H * W), 256, 0, s>>>(gout, u->d0.p, H * W, u->w_out, u->g_d0, u->gw_out);
  UK(cudaGetLastError());
  int st = 0;
  st |= conv_bwd(u, 13, u->d0a, 0, u->g_d0, 32, 0, u->g_d0a, 32, 0, true, false);
  st |= conv_bwd(u, 12, u->cat0, 0, u->g_d0a, 32, 0, u->g_cat0, 96, 0, true, false);
  k_upsample_bwd<<<grid_for((long long)p1 * 64), 256, 0, s>>>(u->g_cat0, 96, 64, H >> 1, W >> 1, u->g_d1);
  st |= conv_bwd(u, 11, u->d1a, 0, u->g_d1, 64, 0, u->g_d1a, 64, 0, true, false);
  st |= conv_bwd(u, 10, u->cat1, 0, u->g_d1a, 64, 0, u->g_cat1, 192, 0, true, false);
  k_upsample_bwd<<<grid_for((long long)p2 * 128), 256, 0, s>>>(u->g_cat1, 192, 128, H >> 2, W >> 2, u->g_d2);
  st |= conv_bwd(u, 9, u->d2a, 0, u->g_d2, 128, 0, u->g_d2a, 128, 0, true, false);
  st |= conv_bwd(u, 8, u->cat2, 0, u->g_d2a, 128, 0, u->g_cat2, 384, 0, true, false);
  k_upsample_bwd<<<grid_for((long long)pixels(u, 3) * 256), 256, 0, s>>>(u->g_cat2, 384, 256, H >> 3, W >> 3, u->g_b2);
  st |= conv_bwd(u, 7, u->b1, 0, u->g_b2, 256, 0, u->g_b1, 256, 0, true, false);
  st |= conv_bwd(u, 6, u->pool2, 0, u->g_b1, 256, 0, u->g_pool2, 128, 0, false, false);
  k_pool_bwd<<<grid_for((long long)pixels(u, 3) * 128), 256, 0, s>>>(u->g_pool2, 128, H >> 2, W >> 2, u->g_cat2,
                                                                      u->cat2.p, 384, 256);
  st |= conv_bwd(u, 5, u->a2, 0, u->g_cat2, 384, 256, u->g_a2, 128, 0, true, false);
  st |= conv_bwd(u, 4, u->pool1, 0, u->g_a2, 128, 0, u->g_pool1, 64, 0, false, false);
  k_pool_bwd<<<grid_for((long long)p2 * 64), 256, 0, s>>>(u->g_pool1, 64, H >> 1, W >> 1, u->g_cat1, u->cat1.p, 192,
                                                          128);
  st |= conv_bwd(u, 3, u->a1, 0, u->g_cat1, 192, 128, u->g_a1, 64, 0, true, false);
  st |= conv_bwd(u, 2, u->pool0, 0, u->g_a1, 64, 0, u->g_pool0, 32, 0, false, false);
  k_pool_bwd<<<grid_for((long long)p1 * 32), 256, 0, s>>>(u->g_pool0, 32, H, W, u->g_cat0, u->cat0.p, 96, 64);
  st |= conv_bwd(u, 1, u->a0, 0, u->g_cat0, 96, 64, u->g_a0, 32, 0, true, false);
  st |= conv_bwd(u, 0, u->in0, 0, u->g_a0, 32, 0, nullptr, 0, 0, false, false);
  (void)p0;
  UK(cudaGetLastError());
  return st ? PIC_ECUDA : PIC_OK;
}

}  // extern "C"

namespace pic {
namespace unet {
int forward_on_stream(pic_unet *u, const float *in, float *out, cudaStream_t s) {
  if (!u) return PIC_EINVAL;
  cudaStream_t keep = u->stream;
  u->stream = s;
  int st = pic_unet_forward(u, in, out);
  u->stream = keep;
  return st;
}
void net_dims(const pic_unet *u, int *H, int *W) {
  *H = u ? u->H : 0;
  *W = u ? u->W : 0;
}
}  // namespace unet
}  // namespace pic

extern "C" {

int pic_unet_loss_backward(pic_unet *u, const float *in3, const float *target, float *loss) {
  if (!u || !in3 || !target || !u->last_out) return PIC_EINVAL;
  const int HW = u->H * u->W;
  const float *mask = in3 + 2 * (size_t)HW;
  UK(cudaMemsetAsync(u->loss_sums, 0, 2 * sizeof(double), u->stream));
  k_loss_sums<<<grid_for(HW), 256, 0, u->stream>>>(u->last_out, target, mask, HW, u->loss_sums);
  k_loss_grad<<<grid_for(HW), 256, 0, u->stream>>>(u->last_out, target, mask, HW, u->loss_sums, u->gout, loss);
  UK(cudaGetLastError());
  return pic_unet_backward(u, u->gout);
}

int pic_unet_adam(pic_unet *u, float lr, float beta1, float beta2, float eps, int t) {
  if (!u || !(lr > 0) || t < 1) return PIC_EINVAL;
  return refresh_weights(u, lr, beta1, beta2, eps, t);
}

// One convolution operation on caller-owned device tensors (dense NHWC BF16):
//   op 0: out_f32[H*W][Cout] = conv3x3(in, w)            (no bias, no ReLU)
//   op 1: out_bf16[H*W][Cout] = bf16(ReLU(conv3x3(in, w) + bias))
//   op 2: out_f32[9*Cin][Cout] = weight gradient sum_p in[p+off][cin] dy[p][cout]
//         (in = x [H*W][Cin], w = dy [H*W][Cout] for this op)
// tile_n / tile_mma choose the tiling of ops 0 and 1 (0 = automatic; tile_n = -1
// = the cp.async gather kernel).
int pic_conv3x3_op_ex(int op, int H, int W, const void *in, int Cin, const void *w, const float *bias, void *out,
                      int Cout, int tile_n, int tile_mma, void *cuda_stream) {
  if (H < 1 || W < 1 || !in || !w || !out || Cin % 16 || Cout % 16 || op < 0 || op > 2) return PIC_EINVAL;
  if (tile_n != 0 && tile_n != -1 && tile_n != 32 && tile_n != 64 && tile_n != 128 && tile_n != 256) return PIC_EINVAL;
  if (tile_mma != 0 && tile_mma != 1 && tile_mma != 2 && tile_mma != 4 && tile_mma != 8) return PIC_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  ConvGeom geo;
  const bool tma = op < 2 && tile_n != -1 && plan_conv(H, W, Cin, Cout, tile_n > 0 ? tile_n : 0, tile_mma, &geo);
  if (op < 2 && !tma && (tile_n > 0 || tile_mma > 0)) return PIC_EINVAL;  // forced tiling not possible
  if (!tma && Cout > 256) return PIC_EINVAL;
  int *err = nullptr;
  __nv_bfloat16 *wpk = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return PIC_ENOMEM;
  if (tma && cudaMalloc(&wpk, (size_t)Cout * 9 * Cin * 2) != cudaSuccess) {
    cudaFree(err);
    return PIC_ENOMEM;
  }
  cudaMemsetAsync(err, 0, sizeof(int), s);
  cudaError_t e;
  if (op < 2) {
    ConvArgs a;
    memset(&a, 0, sizeof(a));
    a.in = (const __nv_bfloat16 *)in;
    a.in_cs = Cin;
    a.Cin = Cin;
    a.out_cs = Cout;
    a.Cout = Cout;
    a.w = (const __nv_bfloat16 *)w;
    a.H = H;
    a.W = W;
    a.err = err;
    if (op == 0) {
      a.out_f = (float *)out;
    } else {
      a.out_bf = (__nv_bfloat16 *)out;
      a.bias = bias;
      a.relu = 1;
    }
    if (tma) {
      CUtensorMap map;
      e = make_input_map(&map, a.in, Cin, H, W, geo);
      if (e == cudaSuccess) e = pack_weights(a.w, Cin, Cout, geo.N, wpk, s);
      if (e == cudaSuccess) e = launch_conv_tma(map, a, geo, wpk, s);
    } else {
      e = launch_conv3x3(a, s);
    }
  } else {
    WgradArgs a;
    memset(&a, 0, sizeof(a));
    a.x = (const __nv_bfloat16 *)in;
    a.x_cs = Cin;
    a.Cin = Cin;
    a.dy = (const __nv_bfloat16 *)w;
    a.dy_cs = Cout;
    a.Cout = Cout;
    a.dw = (float *)out;
    a.H = H;
    a.W = W;
    a.pix_per_cta = 256;
    a.err = err;
    cudaMemsetAsync(out, 0, sizeof(float) * 9 * Cin * Cout, s);
    e = launch_wgrad(a, s);
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  else cudaStreamSynchronize(s);
  cudaFree(err);
  if (wpk) cudaFree(wpk);
  if (e != cudaSuccess) return PIC_ECUDA;
  return herr ? PIC_ETIMEOUT : PIC_OK;
}

int pic_conv3x3_op(int op, int H, int W, const void *in, int Cin, const void *w, const float *bias, void *out, int Cout,
                   void *cuda_stream) {
  return pic_conv3x3_op_ex(op, H, W, in, Cin, w, bias, out, Cout, 0, 0, cuda_stream);
}

int pic_unet_status(pic_unet *u, int *err) {
  if (!u || !err) return PIC_EINVAL;
  UK(cudaStreamSynchronize(u->stream));
  UK(cudaMemcpy(err, u->err, sizeof(int), cudaMemcpyDeviceToHost));
  int z = 0;
  UK(cudaMemcpy(u->err, &z, sizeof(int), cudaMemcpyHostToDevice));
  return PIC_OK;
}

}  // extern "C"
