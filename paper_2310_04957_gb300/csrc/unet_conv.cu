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
#include <cstring>
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

// ---------------------------------------------------------------------------------
// TMA-fed forward / dgrad convolution (warp-specialised).  Warp 0 lane 0 loads
// each stage (16 input channels: 2 groups x nvar boxes by TMA, zero-filled
// outside the image, plus the packed weights by one bulk copy); warp 1 lane 0
// issues 9 taps x nmma MMAs per stage and releases the stage with a commit; all
// four warps then drain the accumulators (tensor-memory lane = pixel).
// ---------------------------------------------------------------------------------
constexpr int kMaxStages = 8;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of the given parity; false after about two seconds.
__device__ __forceinline__ bool mbar_wait_timed(uint64_t *mbar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_u32(mbar)), "r"(parity));
    if (done) return true;
    if ((i & 63) == 63 && global_ns() - t0 > 2000000000ull) return false;
  }
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                           uint64_t *mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

template <int N>
__global__ void __launch_bounds__(128, 1)
    k_conv_tma(const __grid_constant__ CUtensorMap tin, const ConvArgs a, const ConvGeom g,
               const __nv_bfloat16 *__restrict__ wpk) {
  extern __shared__ __align__(128) uint8_t smem_tma[];
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], accum;
  __shared__ uint32_t s_taddr;
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tx = blockIdx.x % g.tiles_x, ty = blockIdx.x / g.tiles_x;
  const int x0 = tx * g.Wt, y0 = ty * g.R, n0 = blockIdx.y * N;
  const int nk = a.Cin / 16, S = g.S;
  const uint32_t sbase = (smem_u32(smem_tma) + 127u) & ~127u;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  if (tid == 32) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tin)) : "memory");
  tmem_alloc(&s_taddr, (uint32_t)g.tcols);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = s_taddr;

  if (tid == 0) {
    // producer
    int issued = 0;
    const uint8_t *wsrc = reinterpret_cast<const uint8_t *>(wpk) + (size_t)blockIdx.y * nk * (288 * N);
    for (int k = 0; k < nk; ++k) {
      const int s = k % S;
      if (k >= S && !mbar_wait_timed(&empty[s], (uint32_t)((k / S - 1) & 1))) {
        s_fail = 1;
        break;
      }
      if (s_fail) break;
      const uint32_t sA = sbase + s * g.stage_bytes, sB = sA + g.a_bytes;
      mbar_expect_tx(&full[s], (uint32_t)g.tx_bytes);
      const int c = a.in_off + 16 * k;
      for (int gi = 0; gi < 2; ++gi)
        for (int v = 0; v < g.nvar; ++v)
          tma_load3d(sA + (gi * g.nvar + v) * g.slot, &tin, c + 8 * gi, g.nvar == 1 ? x0 - 1 : x0 + v - 1, y0 - 1,
                     &full[s]);
      bulk_load(sB, wsrc + (size_t)k * (288 * N), 288 * N, &full[s]);
      issued = k + 1;
    }
    // the copies this thread started have all landed before the CTA moves on
    for (int k = issued > S ? issued - S : 0; k < issued; ++k)
      if (!mbar_wait_timed(&full[k % S], (uint32_t)((k / S) & 1))) s_fail = 1;
  } else if (tid == 32) {
    // MMA issuer
    const uint32_t idesc = instr_desc(128, N, 0, 0);
    const uint32_t lbo_a = (uint32_t)(g.nvar * g.slot), lbo_b = 144u * N;
    for (int k = 0; k < nk; ++k) {
      const int s = k % S;
      if (s_fail || !mbar_wait_timed(&full[s], (uint32_t)((k / S) & 1))) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sA = sbase + s * g.stage_bytes, sB = sA + g.a_bytes;
      for (int j = 0; j < g.nmma; ++j) {
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const int dy = t / 3 - 1, dx = t % 3 - 1;
          uint32_t aoff;
          if (g.nvar == 1)
            aoff = (uint32_t)(((j + dy + 1) * g.Bx + dx + 1) * 16);
          else
            aoff = (uint32_t)((dx + 1) * g.slot + (j * g.q + dy + 1) * g.Wt * 16);
          const uint64_t da = smem_desc(sA + aoff, lbo_a, 128);
          const uint64_t db = smem_desc(sB + t * N * 16, lbo_b, 128);
          mma_bf16(taddr + (uint32_t)(j * N), da, db, idesc, (k > 0 || t > 0) ? 1u : 0u);
        }
      }
      mma_commit(&empty[s]);
    }
    // arrives once every MMA issued above has completed
    mma_commit(&accum);
  }
  __syncwarp();
  if (!mbar_wait_timed(&accum, 0)) s_fail = 1;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool fail = s_fail != 0;
  if (!fail) {
    const int m = warp * 32 + lane;
    for (int j = 0; j < g.nmma; ++j) {
      int y, x;
      if (g.nvar == 1) {
        y = y0 + j;
        x = x0 + m;
      } else {
        y = y0 + j * g.q + m / g.Wt;
        x = x0 + m % g.Wt;
      }
      const bool valid = y < a.H;
      const size_t p = (size_t)y * a.W + x;
#pragma unroll 1
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * N + c0), v);
        if (!valid) continue;
        const int c = n0 + c0;
        if (a.out_f) {
          float *o = a.out_f + p * a.out_cs + a.out_off + c;
          if (a.mask) {
            const uint4 *mk = reinterpret_cast<const uint4 *>(a.mask + p * a.mask_cs + a.mask_off + c);
            __align__(16) __nv_bfloat16 mh[16];
            reinterpret_cast<uint4 *>(mh)[0] = mk[0];
            reinterpret_cast<uint4 *>(mh)[1] = mk[1];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = __bfloat162float(mh[i]) > 0.0f ? v[i] : 0.0f;
          }
          float4 *o4 = reinterpret_cast<float4 *>(o);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float4 r = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            if (a.accumulate) {
              const float4 q = o4[i];
              r.x += q.x;
              r.y += q.y;
              r.z += q.z;
              r.w += q.w;
            }
            o4[i] = r;
          }
        } else {
          __align__(16) __nv_bfloat16 h[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float yv = v[i] + (a.bias ? a.bias[c + i] : 0.0f);
            if (a.relu) yv = fmaxf(yv, 0.0f);
            h[i] = __float2bfloat16(yv);
          }
          uint4 *o = reinterpret_cast<uint4 *>(a.out_bf + p * a.out_cs + a.out_off + c);
          o[0] = reinterpret_cast<const uint4 *>(h)[0];
          o[1] = reinterpret_cast<const uint4 *>(h)[1];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (fail && tid == 0) atomicExch(a.err, 1);
  tmem_free(taddr, (uint32_t)g.tcols);
}

// w [Cout][9][Cin] -> [Cout/N][Cin/16][2][9][N][8]
__global__ void k_pack_weights(const __nv_bfloat16 *w, int Cin, int Cout, int N, __nv_bfloat16 *dst) {
  const int n = Cout * 9 * Cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ci = i % Cin, t = (i / Cin) % 9, co = i / (9 * Cin);
    const int b = co / N, r = co - b * N, ks = ci >> 4, gi = (ci >> 3) & 1, e = ci & 7;
    const size_t o = ((((size_t)b * (Cin >> 4) + ks) * 2 + gi) * 9 + t) * N + r;
    dst[o * 8 + e] = w[i];
  }
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

// ---- TMA convolution: tiling, tensor maps, packing, launch ------------------------------
static int round_up(int v, int m) { return (v + m - 1) / m * m; }

static bool geom_for(int H, int W, int Cin, int Cout, int N, int nmma, ConvGeom *g) {
  if (Cin % 16 || Cout % N || N * nmma > 256) return false;
  ConvGeom r;
  memset(&r, 0, sizeof(r));
  r.N = N;
  r.nmma = nmma;
  if (W % 128 == 0) {
    r.Wt = 128;
    r.nvar = 1;
  } else {
    r.Wt = W % 64 == 0 ? 64 : W % 32 == 0 ? 32 : W % 16 == 0 ? 16 : W % 8 == 0 ? 8 : 0;
    if (!r.Wt) return false;
    r.nvar = 3;
  }
  r.q = 128 / r.Wt;
  r.R = nmma * r.q;
  r.By = r.R + 2;
  r.Bx = r.nvar == 1 ? r.Wt + 2 : r.Wt;
  if (r.By > 256) return false;
  r.slot = round_up(16 * r.Bx * r.By, 128);
  r.a_bytes = 2 * r.nvar * r.slot;
  r.stage_bytes = round_up(r.a_bytes + 288 * N, 128);
  r.tx_bytes = 2 * r.nvar * 16 * r.Bx * r.By + 288 * N;
  int S = (110 * 1024) / r.stage_bytes;
  S = S > kMaxStages ? kMaxStages : S;
  if (S < 2) S = 2;
  r.S = S;
  r.tiles_x = W / r.Wt;
  r.tiles_y = (H + r.R - 1) / r.R;
  r.nsplit = Cout / N;
  int cols = N * nmma;
  r.tcols = cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : 256;
  r.smem = smem_for_tmem(S * r.stage_bytes + 128, r.tcols);
  if (r.smem > 227 * 1024) return false;
  *g = r;
  return true;
}

bool plan_conv(int H, int W, int Cin, int Cout, int tile_n, int tile_mma, ConvGeom *g) {
  if (H < 1 || W < 1) return false;
  if (tile_n || tile_mma) {
    const int n = tile_n ? tile_n : (Cout % 64 == 0 ? 64 : 32);
    return geom_for(H, W, Cin, Cout, n, tile_mma ? tile_mma : 1, g);
  }
  // Largest accumulator footprint (nmma x N) that still gives >= 256 CTAs
  // (two per SM on most of the 152 SMs); else the tiling with the most CTAs.
  ConvGeom best;
  bool have = false;
  long best_ctas = -1, best_cols = -1;
  int best_n = 0;
  const int ns[4] = {256, 128, 64, 32};
  for (int ni = 0; ni < 4; ++ni)
    for (int m = 1; m <= 8; m *= 2) {
      ConvGeom c;
      if (!geom_for(H, W, Cin, Cout, ns[ni], m, &c)) continue;
      const long ctas = (long)c.tiles_x * c.tiles_y * c.nsplit, cols = (long)ns[ni] * m;
      bool better;
      if (!have) {
        better = true;
      } else {
        const bool ok_new = ctas >= 256, ok_old = best_ctas >= 256;
        if (ok_new != ok_old)
          better = ok_new;
        else if (ok_new)
          better = cols > best_cols || (cols == best_cols && ns[ni] > best_n);
        else
          better = ctas > best_ctas || (ctas == best_ctas && ns[ni] > best_n);
      }
      if (better) {
        best = c;
        have = true;
        best_ctas = ctas;
        best_cols = cols;
        best_n = ns[ni];
      }
    }
  if (have) *g = best;
  return have;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

cudaError_t make_input_map(CUtensorMap *m, const __nv_bfloat16 *base, int cs, int H, int W, const ConvGeom &g) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || cs % 8) return cudaErrorInvalidValue;
  const cuuint64_t dims[3] = {(cuuint64_t)cs, (cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[2] = {(cuuint64_t)cs * 2, (cuuint64_t)W * cs * 2};
  const cuuint32_t box[3] = {8, (cuuint32_t)g.Bx, (cuuint32_t)g.By};
  const cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t pack_weights(const __nv_bfloat16 *w, int Cin, int Cout, int N, __nv_bfloat16 *dst, cudaStream_t st) {
  if (Cin % 16 || Cout % N) return cudaErrorInvalidValue;
  const int n = Cout * 9 * Cin;
  int blocks = (n + 255) / 256;
  blocks = blocks > 2048 ? 2048 : blocks;
  k_pack_weights<<<blocks, 256, 0, st>>>(w, Cin, Cout, N, dst);
  return cudaGetLastError();
}

template <int N>
static cudaError_t conv_tma_launch(const CUtensorMap &tin, const ConvArgs &a, const ConvGeom &g,
                                   const __nv_bfloat16 *wpk, cudaStream_t st) {
  static int attr = 0;  // largest dynamic shared memory granted so far (per instance)
  if (g.smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem);
    if (e != cudaSuccess) return e;
    attr = g.smem;
  }
  dim3 grid(g.tiles_x * g.tiles_y, g.nsplit);
  k_conv_tma<N><<<grid, 128, g.smem, st>>>(tin, a, g, wpk);
  return cudaGetLastError();
}

cudaError_t launch_conv_tma(const CUtensorMap &tin, const ConvArgs &a, const ConvGeom &g, const __nv_bfloat16 *wpk,
                            cudaStream_t st) {
  if (a.Cin % 16 || a.Cout % g.N || g.S < 2 || g.S > kMaxStages || a.in_off % 8 || a.out_off % 16) return cudaErrorInvalidValue;
  switch (g.N) {
    case 32: return conv_tma_launch<32>(tin, a, g, wpk, st);
    case 64: return conv_tma_launch<64>(tin, a, g, wpk, st);
    case 128: return conv_tma_launch<128>(tin, a, g, wpk, st);
    case 256: return conv_tma_launch<256>(tin, a, g, wpk, st);
    default: return cudaErrorInvalidValue;
  }
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
