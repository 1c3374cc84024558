// unet_conv.cu -- 3x3 convolutions of the learned field-solve preconditioner on
// the 5th-generation tensor cores (tcgen05.mma, BF16 operands, FP32 accumulators
// in tensor memory).
//
// Forward and input-gradient (dgrad) are implicit GEMMs: M = 128 pixels of an
// NHWC activation, N = output channels, K = 9 taps x input channels.  Operands
// are staged by cp.async (16-byte chunks, zero-filled outside the image) into
// shared memory in the K-major canonical layout (8-row x 16-byte core matrices)
// through a three-stage pipeline; one thread issues the MMAs and commits them
// to an mbarrier per stage; the epilogue reads the accumulator with tcgen05.ld.
// The weight gradient (wgrad) is a GEMM over pixels (K) with both operands in
// the MN-major canonical layout, split over CTAs and summed with FP32 atomics.
// Every wait is bounded; on a timeout a kernel flags the error, stops issuing,
// and still releases its tensor memory.
#include <cstdint>
#include <cuda_bf16.h>

#include "unet.h"

namespace pic {
namespace unet {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start, leading-dimension offset
// (between core matrices adjacent along K), stride offset (adjacent along M/N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, int a_mn_major, int b_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn_major << 15) | ((uint32_t)b_mn_major << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

__device__ __forceinline__ void mma_bf16(uint32_t taddr, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

// Bounded wait on an mbarrier phase; returns false after ~2^26 polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int spin = 0; spin < (1 << 26); ++spin) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_u32(mbar)), "r"(parity));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t a, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(a));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

constexpr int kStages = 3;

// TMEM allocation of `cols` columns by warp 0; address published via shared memory.
__device__ __forceinline__ void tmem_alloc(uint32_t *s_taddr, uint32_t cols) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_taddr)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
  if ((threadIdx.x >> 5) == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols));
}

// ---------------------------------------------------------------------------------
// Forward / dgrad 3x3 convolution.  N = output channels (32..256), KC = input
// channels per K step (16, 32 or 64; divides Cin).
// ---------------------------------------------------------------------------------
template <int N, int KC>
__global__ void __launch_bounds__(128, 1) k_conv3x3(const ConvArgs a) {
  constexpr int M = 128;
  constexpr int A_BYTES = M * KC * 2, B_BYTES = N * KC * 2, STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t TCOLS = N < 32 ? 32 : N;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[kStages];
  __shared__ uint32_t s_taddr;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int HW = a.H * a.W;
  const int p0 = blockIdx.x * M;
  const int csteps = a.Cin / KC, nsteps = 9 * csteps;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  tmem_alloc(&s_taddr, TCOLS);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = s_taddr;
  const uint32_t idesc = instr_desc(M, N, 0, 0);
  const uint32_t sbase = smem_u32(smem);

  auto load_stage = [&](int buf, int step) {
    const int tap = step / csteps, c0 = (step - tap * csteps) * KC;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const uint32_t sA = sbase + buf * STAGE, sB = sA + A_BYTES;
    constexpr int CH = KC / 8;  // 16-byte chunks per row
    for (int c = tid; c < M * CH; c += 128) {
      int r = c / CH, kb = c - r * CH;
      int p = p0 + r;
      int y = p / a.W, x = p - y * a.W;
      int yy = y + dy, xx = x + dx;
      bool valid = p < HW && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
      const __nv_bfloat16 *src = a.in + (valid ? ((size_t)(yy * a.W + xx) * a.in_cs + a.in_off + c0 + kb * 8) : 0);
      cp_async16(sA + kb * (M / 8) * 128 + (r >> 3) * 128 + (r & 7) * 16, src, valid);
    }
    for (int c = tid; c < N * CH; c += 128) {
      int n = c / CH, kb = c - n * CH;
      bool valid = n < a.Cout;
      const __nv_bfloat16 *src = a.w + (valid ? ((size_t)(n * 9 + tap) * a.Cin + c0 + kb * 8) : 0);
      cp_async16(sB + kb * (N / 8) * 128 + (n >> 3) * 128 + (n & 7) * 16, src, valid);
    }
  };

  // prologue
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nsteps) load_stage(s, s);
    cp_async_commit();
  }
  bool ok = true;
  for (int step = 0; step < nsteps; ++step) {
    const int buf = step % kStages;
    cp_async_wait<kStages - 2>();
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sA = sbase + buf * STAGE, sB = sA + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < KC / 16; ++kk) {
        uint64_t da = smem_desc(sA + kk * 2 * (M / 8) * 128, (M / 8) * 128, 128);
        uint64_t db = smem_desc(sB + kk * 2 * (N / 8) * 128, (N / 8) * 128, 128);
        mma_bf16(taddr, da, db, idesc, (step > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&mbar[buf]);
    }
    const int next = step + kStages - 1;
    if (next < nsteps) {
      const int nbuf = next % kStages;
      if (next >= kStages && !mbar_wait(&mbar[nbuf], (uint32_t)((next / kStages - 1) & 1))) {
        ok = false;
        s_fail = 1;
      }
      if (ok) load_stage(nbuf, next);
    }
    cp_async_commit();
  }
  cp_async_wait<0>();
  if (nsteps > 0 && ok) {
    const int last = nsteps - 1;
    if (!mbar_wait(&mbar[last % kStages], (uint32_t)((last / kStages) & 1))) s_fail = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (s_fail) {
    if (tid == 0) atomicExch(a.err, 1);
  } else {
    const int row = warp * 32 + lane;
    const int p = p0 + row;
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (p < HW && c0 < a.Cout) {
        if (a.out_f) {
          // input gradient: mask by the forward activation of this conv's input
          float *o = a.out_f + (size_t)p * a.out_cs + a.out_off + c0;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float g = v[j];
            if (a.mask) g = __bfloat162float(a.mask[(size_t)p * a.mask_cs + a.mask_off + c0 + j]) > 0.0f ? g : 0.0f;
            o[j] = a.accumulate ? o[j] + g : g;
          }
        } else {
          __align__(16) __nv_bfloat16 h[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float y = v[j] + (a.bias ? a.bias[c0 + j] : 0.0f);
            if (a.relu) y = fmaxf(y, 0.0f);
            h[j] = __float2bfloat16(y);
          }
          uint4 *o = reinterpret_cast<uint4 *>(a.out_bf + (size_t)p * a.out_cs + a.out_off + c0);
          o[0] = reinterpret_cast<const uint4 *>(h)[0];
          o[1] = reinterpret_cast<const uint4 *>(h)[1];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  tmem_free(taddr, TCOLS);
}

// ---------------------------------------------------------------------------------
// Weight gradient: dWt[(tap,cin)][cout] += sum_p x[p + off(tap)][cin] * dy[p][cout].
// M = 128 rows of (tap, cin), N = Cout, K = pixels (64 per step), MN-major operands.
// ---------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128, 1) k_wgrad(const WgradArgs a) {
  constexpr int M = 128, KC = 64;
  constexpr int A_BYTES = M * KC * 2, B_BYTES = N * KC * 2, STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t TCOLS = N < 32 ? 32 : N;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[kStages];
  __shared__ uint32_t s_taddr;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int HW = a.H * a.W;
  const int rows = 9 * a.Cin;
  const int m0 = blockIdx.x * M;
  const int pbeg = blockIdx.y * a.pix_per_cta, pend = min(HW, pbeg + a.pix_per_cta);
  const int nsteps = pend > pbeg ? (pend - pbeg + KC - 1) / KC : 0;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  tmem_alloc(&s_taddr, TCOLS);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = s_taddr;
  const uint32_t idesc = instr_desc(M, N, 1, 1);
  const uint32_t sbase = smem_u32(smem);

  auto load_stage = [&](int buf, int step) {
    const uint32_t sA = sbase + buf * STAGE, sB = sA + A_BYTES;
    const int k0 = pbeg + step * KC;
    // A: for pixel k and 8 consecutive (tap, cin) rows
    for (int c = tid; c < KC * (M / 8); c += 128) {
      int k = c / (M / 8), mb = c - k * (M / 8);
      int p = k0 + k;
      int row = m0 + mb * 8;
      bool valid = p < pend && row < rows;
      size_t off = 0;
      if (valid) {
        int tap = row / a.Cin, cin = row - tap * a.Cin;
        int y = p / a.W, x = p - y * a.W;
        int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
        valid = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
        off = valid ? (size_t)(yy * a.W + xx) * a.x_cs + a.x_off + cin : 0;
      }
      cp_async16(sA + ((k >> 3) * (M / 8) + mb) * 128 + (k & 7) * 16, a.x + off, valid);
    }
    for (int c = tid; c < KC * (N / 8); c += 128) {
      int k = c / (N / 8), nb = c - k * (N / 8);
      int p = k0 + k;
      bool valid = p < pend && nb * 8 < a.Cout;
      const __nv_bfloat16 *src = a.dy + (valid ? (size_t)p * a.dy_cs + a.dy_off + nb * 8 : 0);
      cp_async16(sB + ((k >> 3) * (N / 8) + nb) * 128 + (k & 7) * 16, src, valid);
    }
  };

  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nsteps) load_stage(s, s);
    cp_async_commit();
  }
  bool ok = true;
  for (int step = 0; step < nsteps; ++step) {
    const int buf = step % kStages;
    cp_async_wait<kStages - 2>();
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sA = sbase + buf * STAGE, sB = sA + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < KC / 16; ++kk) {
        uint64_t da = smem_desc(sA + kk * 2 * (M / 8) * 128, (M / 8) * 128, 128);
        uint64_t db = smem_desc(sB + kk * 2 * (N / 8) * 128, (N / 8) * 128, 128);
        mma_bf16(taddr, da, db, idesc, (step > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&mbar[buf]);
    }
    const int next = step + kStages - 1;
    if (next < nsteps) {
      const int nbuf = next % kStages;
      if (next >= kStages && !mbar_wait(&mbar[nbuf], (uint32_t)((next / kStages - 1) & 1))) {
        ok = false;
        s_fail = 1;
      }
      if (ok) load_stage(nbuf, next);
    }
    cp_async_commit();
  }
  cp_async_wait<0>();
  if (nsteps > 0 && ok) {
    const int last = nsteps - 1;
    if (!mbar_wait(&mbar[last % kStages], (uint32_t)((last / kStages) & 1))) s_fail = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (s_fail) {
    if (tid == 0) atomicExch(a.err, 1);
  } else if (nsteps > 0) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < rows && c0 < a.Cout) {
        float *o = a.dw + (size_t)row * a.Cout + c0;
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(o + j, v[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  tmem_free(taddr, TCOLS);
}

// ---- host launchers ------------------------------------------------------------------
// Dynamic shared memory is padded so that at most 512 / columns CTAs fit on an
// SM: the CTAs resident on an SM never ask for more tensor-memory columns than
// the SM has (228 KB of shared memory per SM).
static int smem_for_tmem(int smem, int tcols) {
  int max_ctas = 512 / tcols;
  int cap = 233472 / (max_ctas + 1) + 1024;
  return smem > cap ? smem : cap;
}

template <int N, int KC>
static cudaError_t conv_launch(const ConvArgs &a, cudaStream_t st) {
  constexpr int STAGE = 128 * KC * 2 + N * KC * 2;
  const int smem = smem_for_tmem(kStages * STAGE, N < 32 ? 32 : N);
  static bool attr_set = false;  // per template instance
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3<N, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int tiles = (a.H * a.W + 127) / 128;
  k_conv3x3<N, KC><<<tiles, 128, smem, st>>>(a);
  return cudaGetLastError();
}

template <int N>
static cudaError_t conv_launch_kc(const ConvArgs &a, cudaStream_t st) {
  if (a.Cin % 64 == 0) return conv_launch<N, 64>(a, st);
  if (a.Cin % 32 == 0) return conv_launch<N, 32>(a, st);
  if (a.Cin % 16 == 0) return conv_launch<N, 16>(a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_conv3x3(const ConvArgs &a, cudaStream_t st) {
  int n = a.Cout <= 32 ? 32 : a.Cout <= 64 ? 64 : a.Cout <= 128 ? 128 : a.Cout <= 256 ? 256 : 0;
  if (n == 0 || a.Cout % 16 != 0) return cudaErrorInvalidValue;
  switch (n) {
    case 32: return conv_launch_kc<32>(a, st);
    case 64: return conv_launch_kc<64>(a, st);
    case 128: return conv_launch_kc<128>(a, st);
    default: return conv_launch_kc<256>(a, st);
  }
}

template <int N>
static cudaError_t wgrad_launch(const WgradArgs &a, cudaStream_t st) {
  constexpr int STAGE = 128 * 64 * 2 + N * 64 * 2;
  const int smem = smem_for_tmem(kStages * STAGE, N < 32 ? 32 : N);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_wgrad<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((9 * a.Cin + 127) / 128, (a.H * a.W + a.pix_per_cta - 1) / a.pix_per_cta);
  k_wgrad<N><<<grid, 128, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const WgradArgs &a, cudaStream_t st) {
  if (a.Cout % 16 != 0 || a.Cin % 8 != 0 || a.pix_per_cta < 64) return cudaErrorInvalidValue;
  if (a.Cout <= 32) return wgrad_launch<32>(a, st);
  if (a.Cout <= 64) return wgrad_launch<64>(a, st);
  if (a.Cout <= 128) return wgrad_launch<128>(a, st);
  if (a.Cout <= 256) return wgrad_launch<256>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace unet
}  // namespace pic
