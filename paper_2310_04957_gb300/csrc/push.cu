// push.cu -- host side of the particle phase (dispatch of the fused particle
// kernel of push_kernels.cuh, unweighted instances), the bin layout of the
// next write store, the start-up deposit and the Philox test kernel.
#include <cstdint>

#include "push_kernels.cuh"

namespace pic {

// ---------------------------------------------------------------------------
// Bin layout of the next write store, both species at once: room of a bin =
// fill + slack*fill + 8 for bins of plasma cells (0 elsewhere), or exactly the
// fill if that does not fit in 90 % of the capacity; start = exclusive scan of
// the rooms (clamped to the capacity); fill counters of the write store zeroed.
// Three launches: block sums, one scan of the block sums, block scans + writes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long room_of(int f, int plasma, int use_slack, float slack) {
  if (!plasma) return 0;
  return use_slack ? (long long)f + (long long)(slack * (float)f) + 8 : (long long)f;
}

template <int K>
__device__ __forceinline__ void block_sum_ll(long long v[K], long long *sh /* [K][32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    long long x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k * 32 + wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      long long x = lane < (int)(blockDim.x >> 5) ? sh[k * 32 + lane] : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) sh[k * 32] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sh[k * 32];
}

// Exclusive scan over the block (blockDim.x = 1024); returns the block total.
__device__ __forceinline__ long long block_exscan_ll(long long v, long long &excl, long long *sh /* [32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= d) t += y;
    }
    sh[lane] = t;  // inclusive warp totals
  }
  __syncthreads();
  long long before = wid > 0 ? sh[wid - 1] : 0;
  excl = before + x - v;
  long long total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(1024) k_layout_sums(const LayoutParams L) {
  __shared__ long long sh[3 * 32];
  const int s = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  long long v[3] = {0, 0, 0};
  if (b < L.nbins) {
    int f = L.fill_in[s][b], pl = L.bin_plasma[b];
    v[0] = room_of(f, pl, 1, L.slack);
    v[1] = room_of(f, pl, 0, L.slack);
    v[2] = f;
  }
  block_sum_ll<3>(v, sh);
  if (threadIdx.x < 3) L.part[((size_t)s * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = v[threadIdx.x];
}

__global__ void __launch_bounds__(1024) k_layout_scan(const LayoutParams L, int nblk) {
  __shared__ long long sh[3 * 32];
  __shared__ int s_use;
  const int s = blockIdx.x;
  const long long *part = L.part + (size_t)s * nblk * 4;
  long long v[3] = {0, 0, 0};
  if ((int)threadIdx.x < nblk) {
    v[0] = part[threadIdx.x * 4 + 0];
    v[1] = part[threadIdx.x * 4 + 1];
    v[2] = part[threadIdx.x * 4 + 2];
  }
  long long tot[3] = {v[0], v[1], v[2]};
  block_sum_ll<3>(tot, sh);
  if (threadIdx.x == 0) s_use = tot[0] <= (long long)(0.9 * (double)L.capacity[s]) ? 1 : 0;
  __syncthreads();
  int use = s_use;
  long long mine = use ? v[0] : v[1];
  long long excl;
  long long total = block_exscan_ll(mine, excl, sh);
  if ((int)threadIdx.x < nblk) L.boff[(size_t)s * nblk + threadIdx.x] = excl;
  if (threadIdx.x == 0) {
    L.use_slack[s] = use;
    L.meta_out[s]->ovf_base = (int)(total < L.capacity[s] ? total : L.capacity[s]);
    L.meta_out[s]->ovf_n = 0;
    L.meta_out[s]->total = 0;
    L.meta_in[s]->total = tot[2];
  }
}

__global__ void __launch_bounds__(1024) k_layout_write(const LayoutParams L) {
  __shared__ long long sh[32];
  const int s = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int use = L.use_slack[s];
  long long c = 0;
  if (b < L.nbins) c = room_of(L.fill_in[s][b], L.bin_plasma[b], use, L.slack);
  long long excl;
  block_exscan_ll(c, excl, sh);
  if (b < L.nbins) {
    long long run = L.boff[(size_t)s * gridDim.x + blockIdx.x] + excl;
    long long cap = L.capacity[s];
    if (run + c > cap) c = run < cap ? cap - run : 0;  // never hand out room past the buffer
    L.start[s][b] = (int)(run < cap ? run : cap);
    L.cap[s][b] = (int)c;
    L.fill_out[s][b] = 0;
  }
}

// Deposit of the read store's particles at their current x~ (start-up).
template <typename T, bool WT>
__global__ void k_deposit_only(const PushParams<T> P) {
  const int s = blockIdx.y;
  const StoreView<T> &A = P.in[s];
  const int nb = P.map.nbins();
  // one warp per bin, then the overflow region
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int b = warp; b < nb; b += nwarps) {
    int f = A.fill[b], c = A.cap[b];
    int n = f < c ? f : c;
    int ci, cj;
    P.map.cell(b, ci, cj);
    for (int k = lane; k < n; k += 32) {
      Part<T> p;
      load_particle<WT>(A, A.start[b] + k, p);
      p.ci = ci; p.cj = cj;
      deposit_global<WT>(P, s, p);
    }
  }
  int novf = min(A.meta->ovf_n, A.capacity - A.meta->ovf_base);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < novf; k += gridDim.x * blockDim.x) {
    int slot = A.meta->ovf_base + k;
    Part<T> p;
    load_particle<WT>(A, slot, p);
    int c = A.cell[slot];
    p.cj = c / P.nr;
    p.ci = c - p.cj * P.nr;
    deposit_global<WT>(P, s, p);
  }
}

__global__ void k_philox(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x[4];
    philox10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], key[2 * i], key[2 * i + 1], x);
    out[4 * i] = x[0]; out[4 * i + 1] = x[1]; out[4 * i + 2] = x[2]; out[4 * i + 3] = x[3];
  }
}

// Tile shapes compiled in (cells in r x z); others are rejected at pic_init.
bool tile_supported(int tx, int ty) {
  return (tx == 2 && ty == 2) || (tx == 4 && ty == 2) || (tx == 2 && ty == 4) || (tx == 4 && ty == 4) ||
         (tx == 8 && ty == 4) || (tx == 8 && ty == 8) || (tx == 16 && ty == 4) || (tx == 16 && ty == 8) ||
         (tx == 32 && ty == 4) || (tx == 4 && ty == 8) || (tx == 8 && ty == 2);
}

// Unweighted particles run the kernels compiled here; weighted ones (weight
// ratios, splitting) those of push_w.cu, a translation unit of its own so the
// two sets compile in parallel.
template <typename T>
cudaError_t launch_particles(const PushParams<T> &P, cudaStream_t st) {
  if (P.weighted) return launch_particles_weighted<T>(P, st);
  return launch_particles_tiles<T, false>(P, st);
}

template <typename T>
cudaError_t launch_deposit_only(const PushParams<T> &P, cudaStream_t st) {
  dim3 grid(1024, 2);
  if (P.weighted) k_deposit_only<T, true><<<grid, 256, 0, st>>>(P);
  else k_deposit_only<T, false><<<grid, 256, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_layout(const LayoutParams &L, cudaStream_t st) {
  int nblk = (L.nbins + 1023) / 1024;
  if (nblk > 1024) return cudaErrorInvalidValue;
  k_layout_sums<<<dim3(nblk, 2), 1024, 0, st>>>(L);
  k_layout_scan<<<2, 1024, 0, st>>>(L, nblk);
  k_layout_write<<<dim3(nblk, 2), 1024, 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_philox(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_philox<<<blocks, 256, 0, st>>>(n, ctr, key, out);
  return cudaGetLastError();
}

template cudaError_t launch_particles<float>(const PushParams<float> &, cudaStream_t);

template cudaError_t launch_particles<double>(const PushParams<double> &, cudaStream_t);
template cudaError_t launch_deposit_only<float>(const PushParams<float> &, cudaStream_t);
template cudaError_t launch_deposit_only<double>(const PushParams<double> &, cudaStream_t);

}  // namespace pic
