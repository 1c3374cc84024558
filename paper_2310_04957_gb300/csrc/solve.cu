// solve.cu -- field solve of the finite-volume implicit Poisson system
// sum_b G_ab (phi_a - phi_b) = qrhs_a on the free nodes (Eq. 1 of
// arXiv:2310.04957), Dirichlet metal nodes held fixed.
//
// Both solvers are Jacobi-preconditioned conjugate gradients in the
// Chronopoulos-Gear arrangement: the inner products of an iteration are
// formed together, so each iteration needs one grid-wide reduction and one
// barrier.  That barrier also publishes the vectors the next matrix-vector
// product reads at neighbouring nodes; r, w and s are double-buffered so a
// block rebuilds its neighbours' next preconditioned residual
// u = M^-1 (r - alpha (w + beta s)) on the fly without a second barrier.
//
//   plain: FP64 throughout, warm start from phi, stop at ||r|| <= tol ||b||
//          (b = node charge + Dirichlet lift), confirmed on the recomputed
//          residual.
//   mixed: FP64 residual and iterative refinement around FP32 inner solves of
//          the normalised residual equation (all inner arithmetic, products and
//          reductions in FP32).
//
// GB300 executes FP64 at 1/58 of the FP32 rate (one FP64 warp instruction
// holds a sub-partition for ~68 cycles), so the FP64 work is kept to the
// per-node arithmetic: nodes are spread evenly over all SMs, the scalar
// recurrences run in one thread per block, convergence is tested on squared
// norms.  One persistent cooperative launch; bounded barrier waits.
#include <cooperative_groups.h>
#include <cstdint>
#include <cstring>

#include "pic_device.cuh"
#include "pic_kernels.h"

namespace cg = cooperative_groups;

namespace pic {

__device__ bool grid_barrier(unsigned *bar, unsigned nblocks, long long limit, uint32_t *flags) {
  // One release-add per block and nothing after the last arrival: block 0 adds
  // 2^31 - (nblocks - 1), the others 1, so the arrivals of all blocks together
  // flip bit 31 and leave the low bits as they were (the host zeroes the word
  // before each launch).  Each block waits, with an acquire load, for the flip.
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (nblocks - 1u) : 1u;
    unsigned old, cur;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(bar), "r"(add) : "memory");
    int ok = 1;
    const long long t0 = clock64();
    while (true) {
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(bar) : "memory");
      if ((old ^ cur) & 0x80000000u) break;
      if (clock64() - t0 > limit) {
        ok = 0;
        atomicOr(flags, 0x2u);
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sum K per-thread values of type A over the block; result returned to all threads.
template <typename A, int K>
__device__ __forceinline__ void block_sum(A v[K]) {
  __shared__ A s[K][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s[k][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      A x = lane < nw ? s[k][lane] : (A)0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) s[k][0] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = s[k][0];
  __syncthreads();
}

// Grid reduction: block partials -> barrier -> every block sums all partials
// in the same order (bit-identical totals in every block).  Partials are
// double-buffered by parity so one barrier suffices.
template <typename A, int K>
__device__ __forceinline__ bool grid_sum(A v[K], A *partial, int parity, const PcgParams &P) {
  block_sum<A, K>(v);
  A *part = partial + parity * 4 * gridDim.x;
  if (threadIdx.x < K) part[blockIdx.x * 4 + threadIdx.x] = v[threadIdx.x];
  if (!grid_barrier(P.bar, gridDim.x, P.spin_limit, P.flags)) return false;
  A w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = (A)0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] += __ldcg(part + b * 4 + k);
  }
  block_sum<A, K>(w);
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = w[k];
  return true;
}

// Contiguous chunk of nodes owned by this block.
struct Range {
  int lo, hi;
};
__device__ __forceinline__ Range block_range(int nn) {
  int chunk = (nn + gridDim.x - 1) / gridDim.x;
  int lo = blockIdx.x * chunk;
  int hi = min(nn, lo + chunk);
  return {lo, hi};
}

template <typename T>
struct CgView {
  T *r[2], *w[2], *s[2], *p, *x;
  const T *Gr, *Gz, *dinv;
};

// u_{i+1} at node b from the buffers of iteration i (parity q).
template <typename T>
__device__ __forceinline__ T u_next(const CgView<T> &V, int q, int b, T alpha, T beta) {
  T sv = __ldcg(V.w[q] + b) + beta * __ldcg(V.s[q] + b);
  T rv = __ldcg(V.r[q] + b) - alpha * sv;
  return __ldcg(V.dinv + b) * rv;
}

// One Chronopoulos-Gear iteration at this block's free nodes, reading parity q
// and writing parity q^1; accumulates gamma = r.u, delta = w.u, rho = r.r.
template <typename T>
__device__ __forceinline__ void cg_iteration(const PcgParams &P, const CgView<T> &V, int q, T alpha, T beta,
                                             T acc[3]) {
  const int nr = P.nr, W = nr + 1;
  const Range R = block_range(P.nn);
  for (int a = R.lo + threadIdx.x; a < R.hi; a += blockDim.x) {
    if (P.node_kind[a] != 0) continue;
    int j = a / W, i = a - j * W;
    T ra = __ldcg(V.r[q] + a), wa = __ldcg(V.w[q] + a), sa = __ldcg(V.s[q] + a), da = __ldcg(V.dinv + a);
    T pa = da * ra + beta * __ldcg(V.p + a);
    T snew = wa + beta * sa;
    T rnew = ra - alpha * snew;
    T unew = da * rnew;
    T wnew = (T)0;
    if (i > 0) wnew += __ldcg(V.Gr + j * nr + i - 1) * (unew - u_next(V, q, a - 1, alpha, beta));
    if (i < nr) wnew += __ldcg(V.Gr + j * nr + i) * (unew - u_next(V, q, a + 1, alpha, beta));
    if (j > 0) wnew += __ldcg(V.Gz + (j - 1) * W + i) * (unew - u_next(V, q, a - W, alpha, beta));
    if (j < P.nz) wnew += __ldcg(V.Gz + j * W + i) * (unew - u_next(V, q, a + W, alpha, beta));
    V.x[a] = V.x[a] + alpha * pa;
    V.p[a] = pa;
    V.r[q ^ 1][a] = rnew;
    V.w[q ^ 1][a] = wnew;
    V.s[q ^ 1][a] = snew;
    acc[0] += rnew * unew;
    acc[1] += wnew * unew;
    acc[2] += rnew * rnew;
  }
}

// w_0 = A M^-1 r_0 from buffer 0 (r_0 complete), plus the first products.
template <typename T>
__device__ __forceinline__ void cg_start(const PcgParams &P, const CgView<T> &V, T acc[3]) {
  const int nr = P.nr, W = nr + 1;
  const Range R = block_range(P.nn);
  for (int a = R.lo + threadIdx.x; a < R.hi; a += blockDim.x) {
    if (P.node_kind[a] != 0) continue;
    int j = a / W, i = a - j * W;
    T ra = __ldcg(V.r[0] + a);
    T ua = __ldcg(V.dinv + a) * ra;
    T w = (T)0;
    if (i > 0) w += __ldcg(V.Gr + j * nr + i - 1) * (ua - __ldcg(V.dinv + a - 1) * __ldcg(V.r[0] + a - 1));
    if (i < nr) w += __ldcg(V.Gr + j * nr + i) * (ua - __ldcg(V.dinv + a + 1) * __ldcg(V.r[0] + a + 1));
    if (j > 0) w += __ldcg(V.Gz + (j - 1) * W + i) * (ua - __ldcg(V.dinv + a - W) * __ldcg(V.r[0] + a - W));
    if (j < P.nz) w += __ldcg(V.Gz + j * W + i) * (ua - __ldcg(V.dinv + a + W) * __ldcg(V.r[0] + a + W));
    V.w[0][a] = w;
    acc[0] += ra * ua;
    acc[1] += w * ua;
    acc[2] += ra * ra;
  }
}

// FP64 residual r = qrhs - A phi at this block's free nodes, with ||b||^2 and
// ||r||^2 (b = qrhs + Dirichlet lift).
__device__ __forceinline__ void residual64(const PcgParams &P, double *r64, double acc[2]) {
  const int nr = P.nr, W = nr + 1;
  const Range R = block_range(P.nn);
  for (int a = R.lo + threadIdx.x; a < R.hi; a += blockDim.x) {
    if (P.node_kind[a] != 0) continue;
    int j = a / W, i = a - j * W;
    double pa = __ldcg(P.phi + a), ax = 0.0, lift = 0.0;
    if (i > 0) {
      double g = __ldg(P.Gr + j * nr + i - 1), pb = __ldcg(P.phi + a - 1);
      ax += g * (pa - pb);
      if (P.node_kind[a - 1] != 0) lift += g * pb;
    }
    if (i < nr) {
      double g = __ldg(P.Gr + j * nr + i), pb = __ldcg(P.phi + a + 1);
      ax += g * (pa - pb);
      if (P.node_kind[a + 1] != 0) lift += g * pb;
    }
    if (j > 0) {
      double g = __ldg(P.Gz + (j - 1) * W + i), pb = __ldcg(P.phi + a - W);
      ax += g * (pa - pb);
      if (P.node_kind[a - W] != 0) lift += g * pb;
    }
    if (j < P.nz) {
      double g = __ldg(P.Gz + j * W + i), pb = __ldcg(P.phi + a + W);
      ax += g * (pa - pb);
      if (P.node_kind[a + W] != 0) lift += g * pb;
    }
    double q = __ldg(P.qrhs + a);
    double r = q - ax, b = q + lift;
    r64[a] = r;
    acc[0] += b * b;
    acc[1] += r * r;
  }
}

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }
__device__ __forceinline__ bool finite(float x) { return isfinite(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

// Inner CG loop.  Entry: parity-0 buffers hold r_0, w_0 (s = p = 0) and tot =
// (gamma_0, delta_0, rho_0).  Runs until rho <= stop2 or *it reaches cap.
// The scalar recurrence runs in thread 0 and is broadcast through shared
// memory.  Returns 0 ok, -5 timeout, -7 non-finite, 1 stopped at the cap.
template <typename T>
__device__ int cg_loop(const PcgParams &P, const CgView<T> &V, T *partial, T tot[3], T stop2, int cap, int *it,
                       int *parity) {
  __shared__ T s_ab[2];
  __shared__ int s_state;
  T gamma = tot[0], delta = tot[1], rho = tot[2];
  T gamma_prev = (T)1, alpha_prev = (T)1;
  int q = 0, k = 0;
  while (true) {
    if (threadIdx.x == 0) {
      int state = 0;
      if (!finite(rho) || !finite(gamma) || !finite(delta)) state = -7;
      else if (rho <= stop2) state = 2;
      else if (*it >= cap) state = 1;
      else {
        T beta = k == 0 ? (T)0 : gamma * recip(gamma_prev);
        T den = k == 0 ? delta : delta - beta * gamma * recip(alpha_prev);
        T alpha = gamma * recip(den);
        s_ab[0] = alpha;
        s_ab[1] = beta;
      }
      s_state = state;
    }
    __syncthreads();
    int state = s_state;
    if (state == 2) return 0;
    if (state != 0) return state;
    T alpha = s_ab[0], beta = s_ab[1];
    T acc[3] = {(T)0, (T)0, (T)0};
    cg_iteration<T>(P, V, q, alpha, beta, acc);
    if (!grid_sum<T, 3>(acc, partial, *parity, P)) return -5;
    *parity ^= 1;
    q ^= 1;
    ++k;
    ++*it;
    gamma_prev = gamma;
    alpha_prev = alpha;
    gamma = acc[0];
    delta = acc[1];
    rho = acc[2];
  }
}

// ---- plain FP64 ------------------------------------------------------------------
__global__ void __launch_bounds__(kPcgThreads) k_pcg(const PcgParams P) {
  const int nn = P.nn;
  CgView<double> V;
  for (int k = 0; k < 2; ++k) {
    V.r[k] = P.work + (size_t)k * nn;
    V.w[k] = P.work + (size_t)(2 + k) * nn;
    V.s[k] = P.work + (size_t)(4 + k) * nn;
  }
  V.p = P.work + (size_t)6 * nn;
  V.x = P.phi;
  V.Gr = P.Gr;
  V.Gz = P.Gz;
  V.dinv = P.dinv;
  const Range R = block_range(nn);
  int it = 0, parity = 0, status = -4;
  double b2 = 0.0, r2 = 0.0;
  for (int pass = 0; pass < 32; ++pass) {
    for (int a = R.lo + threadIdx.x; a < R.hi; a += blockDim.x) {
      for (int k = 0; k < 2; ++k) { V.r[k][a] = 0.0; V.w[k][a] = 0.0; V.s[k][a] = 0.0; }
      V.p[a] = 0.0;
    }
    if (!grid_barrier(P.bar, gridDim.x, P.spin_limit, P.flags)) { status = -5; break; }
    double acc2[2] = {0.0, 0.0};
    residual64(P, V.r[0], acc2);
    if (!grid_sum<double, 2>(acc2, P.partial, parity, P)) { status = -5; break; }
    parity ^= 1;
    b2 = acc2[0];
    r2 = acc2[1];
    double target2 = b2 > 0.0 ? P.tol * P.tol * b2 : 1e-60;
    if (!isfinite(r2)) { status = -7; break; }
    if (r2 <= target2) { status = 0; break; }
    if (it >= P.maxit) { status = -4; break; }
    double tot[3] = {0.0, 0.0, 0.0};
    cg_start<double>(P, V, tot);
    if (!grid_sum<double, 3>(tot, P.partial, parity, P)) { status = -5; break; }
    parity ^= 1;
    int st = cg_loop<double>(P, V, P.partial, tot, target2, P.maxit, &it, &parity);
    if (st == -5 || st == -7) { status = st; break; }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.out[0] = (double)it;
    P.out[1] = b2 > 0.0 ? sqrt(r2 / b2) : sqrt(r2);
    P.out[2] = (double)status;
    P.out[3] = 0.0;
    if (status == -4) atomicOr(P.flags, 0x4u);
    if (status == -7) atomicOr(P.flags, 0x8u);
  }
}

// ---- mixed: FP64 refinement around FP32 inner CG ---------------------------------------
__global__ void __launch_bounds__(kPcgThreads) k_pcg_mixed(const PcgParams P) {
  const int nn = P.nn, nr = P.nr, W = nr + 1;
  float *f = P.work32;
  CgView<float> V;
  for (int k = 0; k < 2; ++k) {
    V.r[k] = f + (size_t)k * nn;
    V.w[k] = f + (size_t)(2 + k) * nn;
    V.s[k] = f + (size_t)(4 + k) * nn;
  }
  V.p = f + (size_t)6 * nn;
  V.x = f + (size_t)7 * nn;
  float *gr32 = f + (size_t)8 * nn, *gz32 = f + (size_t)9 * nn, *dinv32 = f + (size_t)10 * nn;
  float *part32 = reinterpret_cast<float *>(P.partial + 8 * gridDim.x);  // FP32 partials after the FP64 ones
  V.Gr = gr32;
  V.Gz = gz32;
  V.dinv = dinv32;
  double *r64 = P.work;
  const Range R = block_range(nn);
  // FP32 operator, scaled by the largest diagonal so its entries are O(1)
  for (int a = R.lo + threadIdx.x; a < R.hi; a += blockDim.x) {
    int j = a / W, i = a - j * W;
    if (i < nr) gr32[j * nr + i] = (float)(__ldg(P.Gr + j * nr + i) * P.gscale);
    if (j < P.nz) gz32[j * W + i] = (float)(__ldg(P.Gz + j * W + i) * P.gscale);
    dinv32[a] = (float)(__ldg(P.dinv + a) / P.gscale);
  }
  int it = 0, parity = 0, status = -4, outer = 0;
  double b2 = 0.0, r2 = 0.0;
  for (outer = 0; outer < 64; ++outer) {
    for (int a = R.lo + threadIdx.x; a < R.hi; a += blockDim.x) {
      for (int k = 0; k < 2; ++k) { V.r[k][a] = 0.0f; V.w[k][a] = 0.0f; V.s[k][a] = 0.0f; }
      V.p[a] = 0.0f;
      V.x[a] = 0.0f;
    }
    if (!grid_barrier(P.bar, gridDim.x, P.spin_limit, P.flags)) { status = -5; break; }
    double acc2[2] = {0.0, 0.0};
    residual64(P, r64, acc2);
    if (!grid_sum<double, 2>(acc2, P.partial, parity, P)) { status = -5; break; }
    parity ^= 1;
    b2 = acc2[0];
    r2 = acc2[1];
    double target2 = b2 > 0.0 ? P.tol * P.tol * b2 : 1e-60;
    if (!isfinite(r2)) { status = -7; break; }
    if (r2 <= target2) { status = 0; break; }
    if (it >= P.maxit) { status = -4; break; }
    // inner right-hand side = residual / ||residual|| (unit 2-norm, FP32-safe)
    double inv = rsqrt(r2);
    for (int a = R.lo + threadIdx.x; a < R.hi; a += blockDim.x)
      if (P.node_kind[a] == 0) V.r[0][a] = (float)(r64[a] * inv);
    if (!grid_barrier(P.bar, gridDim.x, P.spin_limit, P.flags)) { status = -5; break; }
    float tot[3] = {0.0f, 0.0f, 0.0f};
    cg_start<float>(P, V, tot);
    if (!grid_sum<float, 3>(tot, part32, parity, P)) { status = -5; break; }
    parity ^= 1;
    // inner reduction: inner_tol, or just what the outer target still needs
    float stop = P.inner_tol;
    float need = (float)sqrt(target2 / r2);
    if (need > stop) stop = need;
    int st = cg_loop<float>(P, V, part32, tot, stop * stop, P.maxit, &it, &parity);
    if (st == -5 || st == -7) { status = st; break; }
    // phi += ||residual|| x (the operator was scaled by gscale, so x carries 1/gscale)
    double back = sqrt(r2) * P.gscale;
    for (int a = R.lo + threadIdx.x; a < R.hi; a += blockDim.x)
      if (P.node_kind[a] == 0) P.phi[a] += (double)V.x[a] * back;
    if (!grid_barrier(P.bar, gridDim.x, P.spin_limit, P.flags)) { status = -5; break; }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.out[0] = (double)it;
    P.out[1] = b2 > 0.0 ? sqrt(r2 / b2) : sqrt(r2);
    P.out[2] = (double)status;
    P.out[3] = (double)outer;
    if (status == -4) atomicOr(P.flags, 0x4u);
    if (status == -7) atomicOr(P.flags, 0x8u);
  }
}

// ---- multigrid-preconditioned mixed solve ----------------------------------------------
// Same FP64 residual and refinement as k_pcg_mixed; the FP32 inner solve is CG
// preconditioned by one symmetric V(2,2)-cycle over a hierarchy of 2x2 node
// aggregates.  Level 0 -> 1 uses the smoothed-aggregation prolongation
// P = (I - omega_s D^-1 A) P0 (P0: aggregation of the free nodes, omega_s =
// 4 / (3 lambda_max) with lambda_max(D^-1 A) <= 2): level 1 is the Galerkin
// product P^T A P, whose entries two aggregates apart (a few % of the
// diagonal) are moved onto the diagonal with row sums kept, leaving 9 points;
// coarser levels aggregate the 9-point operator plainly (it stays 9-point).
// Smoother: damped Jacobi (omega); coarse corrections scaled by alpha0 into
// level 0 and alpha below (piecewise-constant aggregation over-estimates the
// coarse energy); coarsest level (at most kMgDenseMax nodes): its inverse,
// formed at setup by Gauss-Jordan elimination in shared memory,
// applied as one matrix-vector product (Jacobi sweeps from zero on larger
// coarsest levels).  Every piece is a fixed linear symmetric map, so the
// preconditioner is SPD.
// Threads per block of the multigrid solve (one block per SM; the coarse
// levels run within one block, so its width sets their speed).
constexpr int kMgThreads = 512;

// Synchronisation scope of the multigrid solve: the whole grid (one
// cooperative launch, bounded grid barrier) or one thread-block cluster
// (hardware cluster barrier).
struct GridScope {
  __device__ int nblk() const { return (int)gridDim.x; }
  __device__ int bid() const { return (int)blockIdx.x; }
  __device__ bool sync(const PcgParams &P) const { return grid_barrier(P.bar, gridDim.x, P.spin_limit, P.flags); }
};
template <int CL>
struct ClusterScope {
  __device__ int nblk() const { return CL; }
  __device__ int bid() const { return (int)cg::this_cluster().block_rank(); }
  __device__ bool sync(const PcgParams &) const {
    cg::this_cluster().sync();
    return true;
  }
};

// grid_sum and residual64 over a scope's blocks.
template <typename A, int K, class S>
__device__ __forceinline__ bool grid_sum_s(const S &sc, A v[K], A *partial, int parity, const PcgParams &P) {
  block_sum<A, K>(v);
  A *part = partial + parity * 4 * sc.nblk();
  if (threadIdx.x < K) part[sc.bid() * 4 + threadIdx.x] = v[threadIdx.x];
  if (!sc.sync(P)) return false;
  A w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = (A)0;
  for (int b = threadIdx.x; b < sc.nblk(); b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] += __ldcg(part + b * 4 + k);
  }
  block_sum<A, K>(w);
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = w[k];
  return true;
}

template <class S>
__device__ __forceinline__ void residual64_s(const S &sc, const PcgParams &P, double *r64, double acc[2]) {
  const int nr = P.nr, W = nr + 1;
  const int chunk = (P.nn + sc.nblk() - 1) / sc.nblk();
  const int lo = sc.bid() * chunk, hi = min(P.nn, lo + chunk);
  for (int a = lo + threadIdx.x; a < hi; a += blockDim.x) {
    if (P.node_kind[a] != 0) continue;
    const int j = a / W, i = a - j * W;
    const double pa = __ldcg(P.phi + a);
    double ax = 0.0, lift = 0.0;
    if (i > 0) { const double g = __ldg(P.Gr + j * nr + i - 1), pb = __ldcg(P.phi + a - 1); ax += g * (pa - pb); if (P.node_kind[a - 1] != 0) lift += g * pb; }
    if (i < nr) { const double g = __ldg(P.Gr + j * nr + i), pb = __ldcg(P.phi + a + 1); ax += g * (pa - pb); if (P.node_kind[a + 1] != 0) lift += g * pb; }
    if (j > 0) { const double g = __ldg(P.Gz + (j - 1) * W + i), pb = __ldcg(P.phi + a - W); ax += g * (pa - pb); if (P.node_kind[a - W] != 0) lift += g * pb; }
    if (j < P.nz) { const double g = __ldg(P.Gz + j * W + i), pb = __ldcg(P.phi + a + W); ax += g * (pa - pb); if (P.node_kind[a + W] != 0) lift += g * pb; }
    const double q = __ldg(P.qrhs + a);
    const double r = q - ax, b = q + lift;
    r64[a] = r;
    acc[0] += b * b;
    acc[1] += r * r;
  }
}

// One multigrid level.  Level 0 is the fine operator in conductance form:
// (A v)_a = diag_a v_a - sum_b G_ab v_b with c0 = G to i+1, c1 = G to j+1 (0
// across non-free nodes), and c2..c4 = the smoothed-prolongation weights of
// the node (phs: its own aggregate; phx, phy: the aggregate across the
// aggregate boundary in i, in j).  Coarser levels hold 9-point matrix entries:
// c0 to (i+1, j), c1 to (i, j+1), c2 to (i+1, j+1), c3 to (i-1, j+1); the
// entries towards lower indices are the neighbour's.
struct MgLv {
  int ni, nj, n;
  float *c0, *c1, *c2, *c3, *c4, *diag, *dinv, *X, *Y, *B;
};

__device__ __forceinline__ MgLv mg_view(float *b, int ni, int nj) {
  MgLv v;
  v.ni = ni;
  v.nj = nj;
  v.n = ni * nj;
  const size_t n = (size_t)v.n;
  v.c0 = b; v.c1 = b + n; v.c2 = b + 2 * n; v.c3 = b + 3 * n; v.c4 = b + 4 * n;
  v.diag = b + 5 * n; v.dinv = b + 6 * n; v.X = b + 7 * n; v.Y = b + 8 * n; v.B = b + 9 * n;
  return v;
}

// Level l's arrays: the levels from M.smem_from on live in the shared memory
// of the blocks that run them (sm != nullptr only there); everything else in
// the global workspace.
__device__ __forceinline__ MgLv mg_level(const MgLevels &M, int l, float *sm) {
  float *b = (sm != nullptr && l >= M.smem_from) ? sm + M.soff[l] : M.ws + M.off[l];
  return mg_view(b, M.ni[l], M.nj[l]);
}

__device__ __forceinline__ MgLv mg_level(const MgLevels &M, int l) { return mg_view(M.ws + M.off[l], M.ni[l], M.nj[l]); }

// Level 0: (A v)_a with conductances.
__device__ __forceinline__ float mg_apply(const MgLv &L, const float *v, int a, int i, int j) {
  float s = L.diag[a] * v[a];
  if (i > 0) s -= L.c0[a - 1] * v[a - 1];
  if (i < L.ni - 1) s -= L.c0[a] * v[a + 1];
  if (j > 0) s -= L.c1[a - L.ni] * v[a - L.ni];
  if (j < L.nj - 1) s -= L.c1[a] * v[a + L.ni];
  return s;
}

// Level 0: (A v)_a with v_a = va and the neighbours' values from a functor of
// (node, i, j).
template <class V>
__device__ __forceinline__ float mg_apply_f(const MgLv &L, int a, int i, int j, float va, V v) {
  float s = L.diag[a] * va;
  if (i > 0) s -= L.c0[a - 1] * v(a - 1, i - 1, j);
  if (i < L.ni - 1) s -= L.c0[a] * v(a + 1, i + 1, j);
  if (j > 0) s -= L.c1[a - L.ni] * v(a - L.ni, i, j - 1);
  if (j < L.nj - 1) s -= L.c1[a] * v(a + L.ni, i, j + 1);
  return s;
}

// Coarser levels: (A v)_a over the 9-point stencil, neighbours from a functor.
template <class V>
__device__ __forceinline__ float mg_apply9_f(const MgLv &L, int a, int i, int j, float va, V v) {
  const int ni = L.ni;
  const bool w = i > 0, e = i < ni - 1, s = j > 0, nn = j < L.nj - 1;
  float r = L.diag[a] * va;
  if (e) r += L.c0[a] * v(a + 1, i + 1, j);
  if (w) r += L.c0[a - 1] * v(a - 1, i - 1, j);
  if (nn) r += L.c1[a] * v(a + ni, i, j + 1);
  if (s) r += L.c1[a - ni] * v(a - ni, i, j - 1);
  if (nn && e) r += L.c2[a] * v(a + ni + 1, i + 1, j + 1);
  if (s && w) r += L.c2[a - ni - 1] * v(a - ni - 1, i - 1, j - 1);
  if (nn && w) r += L.c3[a] * v(a + ni - 1, i - 1, j + 1);
  if (s && e) r += L.c3[a - ni + 1] * v(a - ni + 1, i + 1, j - 1);
  return r;
}

// (A v)_a on level l (l == 0: conductance form; else 9-point).
__device__ __forceinline__ float mg_apply_l(const MgLv &L, bool l0, const float *v, int a, int i, int j) {
  if (l0) return mg_apply(L, v, a, i, j);
  return mg_apply9_f(L, a, i, j, v[a], [&](int b, int, int) { return v[b]; });
}

// Matrix entry A(r, c) of level L for two nodes at most one step apart in i and
// j (0 otherwise).
__device__ __forceinline__ float mg_entry(const MgLv &L, bool l0, int r, int c) {
  const int jr = r / L.ni, ir = r - jr * L.ni, jc = c / L.ni, ic = c - jc * L.ni;
  const int di = ic - ir, dj = jc - jr;
  if (di < -1 || di > 1 || dj < -1 || dj > 1) return 0.0f;
  if (di == 0 && dj == 0) return L.diag[r];
  if (l0) {
    if (dj == 0) return -L.c0[min(r, c)];
    if (di == 0) return -L.c1[min(r, c)];
    return 0.0f;
  }
  if (dj == 0) return L.c0[min(r, c)];
  if (di == 0) return L.c1[min(r, c)];
  if (di == dj) return L.c2[min(r, c)];  // (1,1) or (-1,-1)
  return L.c3[di < 0 ? r : c];            // (-1,1) stored at r, (1,-1) stored at c
}

// f(a, i, j) for the nodes a = first, first + stride, ... of an ni-wide grid of
// n nodes, with (i, j) stepped along instead of divided out at every node (the
// block-local passes run on one SM, where the divisions would dominate).
template <class F>
__device__ __forceinline__ void mg_nodes(int first, int stride, int n, int ni, F f) {
  if (first >= n) return;
  int j = first / ni, i = first - j * ni;
  const int sj = stride / ni, si = stride - sj * ni;
  for (int a = first; a < n; a += stride) {
    f(a, i, j);
    i += si;
    j += sj;
    if (i >= ni) { i -= ni; ++j; }
  }
}

// Does this block run the block-local levels?  Block 0 alone, or, when those
// levels live in shared memory, every block on its own copy (the same
// arithmetic in each, so no block has to publish them to the others).
template <class S>
__device__ __forceinline__ bool mg_runs_local(const S &sc, const MgLevels &M) {
  return M.redundant || sc.bid() == 0;
}

// One pass over an ni-wide level of n nodes: grid-wide with a grid barrier
// after it, or (local) by the blocks that run the local levels, with a block
// barrier.  Returns false on a barrier timeout.
template <class S, class F>
__device__ __forceinline__ bool mg_pass(const S &sc, const PcgParams &P, const MgLevels &M, bool local, int n, int ni,
                                        F f) {
  if (local) {
    if (mg_runs_local(sc, M)) {
      mg_nodes(threadIdx.x, blockDim.x, n, ni, f);
      __syncthreads();
    }
    return true;
  }
  mg_nodes(sc.bid() * blockDim.x + threadIdx.x, sc.nblk() * blockDim.x, n, ni, f);
  return sc.sync(P);
}

// Operator hierarchy from the FP64 conductances (scaled by gscale): level 0
// with its smoothed-prolongation weights, level 1 = P^T A P with the smoothed
// prolongation (its entries two aggregates apart moved onto the diagonal, row
// sums kept), coarser levels by plain 2x2 aggregation of the 9-point operator.
template <class S>
__device__ bool mg_setup(const S &sc, const PcgParams &P, const MgLevels &M, float *sm) {
  const int nr = P.nr, nz = P.nz, W1 = nr + 1;
  const int8_t *kind = P.node_kind;
  const float oms = M.omega_s;
  {
    const MgLv L0 = mg_level(M, 0);
    if (!mg_pass(sc, P, M, false, L0.n, W1, [&](int a, int i, int j) {
          const bool fa = kind[a] == 0;
          // conductance to a neighbour, 0 unless both nodes are free
          auto gf = [&](int i2, int j2) {
            if (i2 < 0 || j2 < 0 || i2 > nr || j2 > nz) return 0.0f;
            const int b = j2 * W1 + i2;
            if (!fa || kind[b] != 0) return 0.0f;
            return j2 == j ? (float)(P.Gr[j * nr + min(i, i2)] * P.gscale) : (float)(P.Gz[min(j, j2) * W1 + i] * P.gscale);
          };
          float dg = 0.0f;
          if (fa) {
            // all four neighbours count in the diagonal, Dirichlet ones included
            if (i > 0) dg += (float)(P.Gr[j * nr + i - 1] * P.gscale);
            if (i < nr) dg += (float)(P.Gr[j * nr + i] * P.gscale);
            if (j > 0) dg += (float)(P.Gz[(j - 1) * W1 + i] * P.gscale);
            if (j < nz) dg += (float)(P.Gz[j * W1 + i] * P.gscale);
          }
          const float di = dg > 0.0f ? 1.0f / dg : 0.0f;
          L0.c0[a] = gf(i + 1, j);
          L0.c1[a] = gf(i, j + 1);
          // smoothed-prolongation weights: partner inside the 2x2 aggregate
          // and neighbour across its boundary, in i and in j
          const int ip = (i & 1) ? i - 1 : i + 1, jp = (j & 1) ? j - 1 : j + 1;
          const int ix = (i & 1) ? i + 1 : i - 1, jx = (j & 1) ? j + 1 : j - 1;
          L0.c2[a] = fa ? 1.0f - oms * di * (dg - gf(ip, j) - gf(i, jp)) : 0.0f;
          L0.c3[a] = oms * di * gf(ix, j);
          L0.c4[a] = oms * di * gf(i, jx);
          L0.diag[a] = dg;
          L0.dinv[a] = di;
        }))
      return false;
  }
  // Level 0 (the inner CG's operator and the smoother's) is always current.
  // The coarse hierarchy below it changes little from one step to the next:
  // it is rebuilt every rebuild_every-th solve of the discharge and reused in
  // between, its shared-memory part reloaded from the copy kept in global
  // memory.  A coarse correction from a slightly older operator leaves the
  // V-cycle symmetric positive definite, so the CG stays valid.
  if (M.rebuild_every > 1 && *M.solves % M.rebuild_every != 0) {
    if (sm != nullptr) {
      for (int a = threadIdx.x; a < M.smem_floats; a += blockDim.x) sm[a] = __ldcg(M.persist + a);
      __syncthreads();
    }
    return true;
  }
  for (int l = 0; l + 1 < M.L; ++l) {
    const MgLv F = mg_level(M, l, sm), C = mg_level(M, l + 1, sm);
    const bool local = l + 1 >= M.local_from;
    if (l == 0) {
      // Galerkin product with the smoothed prolongation: A1(I, K) = sum over
      // level-0 pairs (a, b) of phi_I(a) A0(a, b) phi_K(b).  Sixteen lanes per
      // coarse node, one per position of the 4x4 box of level-0 nodes around
      // its aggregate (the corners, outside phi_I's support, idle); the lanes'
      // sums are reduced with shuffles within the half-warp.
      auto body = [&](int first, int stride) {
        const int total = C.n * 16;
        // first is congruent to the lane mod 16 and stride a multiple of 16:
        // the 16 lanes of a half-warp always work on the same coarse node
        for (int task = first; task < total; task += stride) {
          const int c = task >> 4, pos = task & 15;
          const int J = c / C.ni, I = c - J * C.ni;
          const int di = (pos & 3) - 1, dj = (pos >> 2) - 1;
          // acc: to (I, J), (I+1, J), (I, J+1), (I+1, J+1), (I-1, J+1); acc[5]:
          // to the aggregates two steps away along i or j
          float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
          auto add = [&](int K, int L, float v) {
            const int dk = K - I, dl = L - J;
            acc[0] += (dk == 0 && dl == 0) ? v : 0.0f;
            acc[1] += (dk == 1 && dl == 0) ? v : 0.0f;
            acc[2] += (dk == 0 && dl == 1) ? v : 0.0f;
            acc[3] += (dk == 1 && dl == 1) ? v : 0.0f;
            acc[4] += (dk == -1 && dl == 1) ? v : 0.0f;
            acc[5] += ((dl == 0 && (dk == 2 || dk == -2)) || (dk == 0 && (dl == 2 || dl == -2))) ? v : 0.0f;
          };
          const bool ri = di == -1 || di == 2, rj = dj == -1 || dj == 2;
          const int i = 2 * I + di, j = 2 * J + dj;
          if (!(ri && rj) && i >= 0 && j >= 0 && i < F.ni && j < F.nj) {
            const int a = j * F.ni + i;
            // the aggregate's own nodes weigh phs, the ring across i phx, across j phy
            const float pa = ri ? F.c3[a] : (rj ? F.c4[a] : F.c2[a]);
#pragma unroll
            for (int t = 0; t < 5; ++t) {
              const int bi = t == 1 ? i - 1 : (t == 2 ? i + 1 : i), bj = t == 3 ? j - 1 : (t == 4 ? j + 1 : j);
              if (bi < 0 || bj < 0 || bi >= F.ni || bj >= F.nj) continue;
              const int b = bj * F.ni + bi;
              const float av = pa * (t == 0 ? F.diag[a]
                                            : (t <= 2 ? -F.c0[j * F.ni + min(i, bi)] : -F.c1[min(j, bj) * F.ni + i]));
              // node b belongs to its own aggregate (weight phs) and to the
              // aggregates across its boundaries in i (phx) and in j (phy)
              const int bx = (bi & 1) ? bi + 1 : bi - 1, by = (bj & 1) ? bj + 1 : bj - 1;
              add(bi >> 1, bj >> 1, av * F.c2[b]);
              if (bx >= 0) add(bx >> 1, bj >> 1, av * F.c3[b]);
              if (by >= 0) add(bi >> 1, by >> 1, av * F.c4[b]);
            }
          }
          const unsigned half = 0xffffu << (threadIdx.x & 16);
#pragma unroll
          for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(half, acc[k], o);
          if (pos == 0) {
            const float dg = acc[0] + acc[5];
            C.c0[c] = acc[1]; C.c1[c] = acc[2]; C.c2[c] = acc[3]; C.c3[c] = acc[4]; C.c4[c] = 0.0f;
            C.diag[c] = dg;
            C.dinv[c] = dg > 0.0f ? 1.0f / dg : 0.0f;
          }
        }
      };
      if (local) {
        if (mg_runs_local(sc, M)) {
          body(threadIdx.x, blockDim.x);
          __syncthreads();
        }
      } else {
        body(sc.bid() * blockDim.x + threadIdx.x, sc.nblk() * blockDim.x);
        if (!sc.sync(P)) return false;
      }
    } else {
      // plain aggregation of the 9-point operator
      if (!mg_pass(sc, P, M, local, C.n, C.ni, [&](int c, int I, int J) {
            const int i0 = 2 * I, j0 = 2 * J;
            auto g = [&](const float *x, int i, int j) {
              return (i >= 0 && j >= 0 && i < F.ni && j < F.nj) ? x[j * F.ni + i] : 0.0f;
            };
            float dg = g(F.diag, i0, j0) + g(F.diag, i0 + 1, j0) + g(F.diag, i0, j0 + 1) + g(F.diag, i0 + 1, j0 + 1);
            dg += 2.0f * (g(F.c0, i0, j0) + g(F.c0, i0, j0 + 1) + g(F.c1, i0, j0) + g(F.c1, i0 + 1, j0) +
                          g(F.c2, i0, j0) + g(F.c3, i0 + 1, j0));
            C.c0[c] = g(F.c0, i0 + 1, j0) + g(F.c0, i0 + 1, j0 + 1) + g(F.c2, i0 + 1, j0) + g(F.c3, i0 + 2, j0);
            C.c1[c] = g(F.c1, i0, j0 + 1) + g(F.c1, i0 + 1, j0 + 1) + g(F.c2, i0, j0 + 1) + g(F.c3, i0 + 1, j0 + 1);
            C.c2[c] = g(F.c2, i0 + 1, j0 + 1);
            C.c3[c] = g(F.c3, i0, j0 + 1);
            C.c4[c] = 0.0f;
            C.diag[c] = dg;
            C.dinv[c] = dg > 0.0f ? 1.0f / dg : 0.0f;
          }))
        return false;
    }
  }
  // dense inverse of the coarsest operator (SPD: no pivoting), in place, with
  // column k and row k staged so that each elimination step is one pass
  if (M.cinv_off >= 0 && mg_runs_local(sc, M)) {
    // warps take rows, lanes columns; column k and row k of the next step are
    // staged by the owners of those elements into the other buffer, so each
    // elimination step is one pass and one block barrier
    __shared__ float colk[2][kMgDenseMax], rowk[2][kMgDenseMax];
    const MgLv C = mg_level(M, M.L - 1, sm);
    const bool l0 = M.L == 1;
    const int n = C.n, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float *Ai = sm + M.cinv_off;
    for (int r = wid; r < n; r += nw)
      for (int c = lane; c < n; c += 32) {
        float v;
        if (C.diag[r] == 0.0f || C.diag[c] == 0.0f) v = r == c ? 1.0f : 0.0f;  // no unknowns: identity row
        else v = mg_entry(C, l0, r, c);
        Ai[r * n + c] = v;
        if (c == 0) colk[0][r] = v;
        if (r == 0) rowk[0][c] = v;
      }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      const int cur = k & 1, nxt = cur ^ 1;
      const float ip = 1.0f / colk[cur][k];
      for (int r = wid; r < n; r += nw)
        for (int c = lane; c < n; c += 32) {
          const float rk = (c == k ? 1.0f : rowk[cur][c]) * ip;  // row k after scaling
          const float v = r == k ? rk : (c == k ? 0.0f : Ai[r * n + c]) - colk[cur][r] * rk;
          Ai[r * n + c] = v;
          if (c == k + 1) colk[nxt][r] = v;
          if (r == k + 1) rowk[nxt][c] = v;
        }
      __syncthreads();
    }
  }
  // keep the shared-memory part for the solves that reuse the hierarchy
  if (sm != nullptr && sc.bid() == 0) {
    for (int a = threadIdx.x; a < M.smem_floats; a += blockDim.x) M.persist[a] = sm[a];
  }
  // the local levels were built block-locally: everyone waits for them
  return M.local_from >= M.L ? true : sc.sync(P);
}

// Level 0's right-hand side as the V-cycle's first pass reads it: r itself
// (RhsPlain), or the CG update r - alpha q (RhsUpdate), formed on the fly at
// the neighbours while the owner of each node writes it to the next r buffer
// and advances x there.
struct RhsPlain {
  const float *b;
  __device__ __forceinline__ float own(int a) const { return b[a]; }
  __device__ __forceinline__ float nb(int a) const { return b[a]; }
};
struct RhsUpdate {
  const float *r, *q, *p;
  float *rn, *x;
  float alpha;
  __device__ __forceinline__ float own(int a) const {
    const float v = r[a] - alpha * q[a];
    rn[a] = v;
    x[a] += alpha * p[a];
    return v;
  }
  __device__ __forceinline__ float nb(int a) const { return r[a] - alpha * q[a]; }
};

// z = V(b0): b0 is level 0's right-hand side (the first pass reads it through
// rhs), the result is left in level 0's X (each level's result in its X).  The
// last level-0 pass also forms (b0.z, b0.b0) and sums them over the scope into
// dots: the sum's barrier ends that pass.
template <class S, class R>
__device__ bool mg_vcycle(const S &sc, const PcgParams &P, const MgLevels &M, float *sm, float *b0, const R &rhs,
                          float dots[2], float *part32, int parity) {
  const float w = M.omega, al = M.alpha, al0 = M.alpha0;
  const int lf = M.local_from;
  // grid-wide coarse levels smooth once before and once after their coarse
  // correction (each sweep there is a grid barrier); their result is left in Y
  auto single = [&](int l) { return M.single_sweep && l >= 1 && l < lf; };
  // each block that runs the local levels takes the first local level's
  // right-hand side (restricted grid-wide into the global copy) into its
  // shared memory
  auto take_in = [&]() {
    if (sm == nullptr || lf < M.smem_from || lf >= M.L) return;
    const MgLv G = mg_level(M, lf, nullptr), Sh = mg_level(M, lf, sm);
    for (int a = threadIdx.x; a < G.n; a += blockDim.x) Sh.B[a] = __ldcg(G.B + a);
    __syncthreads();
  };
  // down
  for (int l = 0; l + 1 < M.L; ++l) {
    const bool local = l >= lf;
    if (local && !mg_runs_local(sc, M)) break;
    if (l == lf) take_in();
    // the grid-wide restriction into the first local level writes its global copy
    MgLv F = mg_level(M, l, sm);
    const MgLv C = mg_level(M, l + 1, l + 1 == lf ? nullptr : sm);
    // two Jacobi sweeps from zero; the first sweep's values (w D^-1 B) are
    // formed on the fly, so one pass and one barrier suffice
    if (l == 0) {
      F.B = b0;
      if (!mg_pass(sc, P, M, local, F.n, F.ni, [&](int a, int i, int j) {
            auto y = [&](int b, int, int) { return w * F.dinv[b] * rhs.nb(b); };
            const float ba = rhs.own(a), da = w * F.dinv[a], ya = da * ba;
            F.X[a] = ya + da * (ba - mg_apply_f(F, a, i, j, ya, y));
          }))
        return false;
      // restriction with the smoothed prolongation: sum over the aggregate
      // and its ring of phi_IJ times the residual
      if (!mg_pass(sc, P, M, local, C.n, C.ni, [&](int c, int I, int J) {
            float s = 0.0f;
#pragma unroll
            for (int dj = -1; dj <= 2; ++dj)
#pragma unroll
              for (int di = -1; di <= 2; ++di) {
                const bool ri = di == -1 || di == 2, rj = dj == -1 || dj == 2;
                if (ri && rj) continue;  // corners: outside the column's support
                const int i = 2 * I + di, j = 2 * J + dj;
                if (i < 0 || j < 0 || i >= F.ni || j >= F.nj) continue;
                const int a = j * F.ni + i;
                // the aggregate's own nodes weigh phs, the ring across i phx, across j phy
                const float ph = ri ? F.c3[a] : (rj ? F.c4[a] : F.c2[a]);
                s += ph * (F.B[a] - mg_apply(F, F.X, a, i, j));
              }
            C.B[c] = s;
          }))
        return false;
    } else if (single(l)) {
      // one sweep from zero, x = w D^-1 B, formed on the fly by the restriction,
      // which also stores it for the correction on the way up
      if (!mg_pass(sc, P, M, false, C.n, C.ni, [&](int c, int I, int J) {
            auto y = [&](int b, int, int) { return w * F.dinv[b] * F.B[b]; };
            float s = 0.0f;
            for (int dj = 0; dj < 2; ++dj)
              for (int di = 0; di < 2; ++di) {
                const int i = 2 * I + di, j = 2 * J + dj;
                if (i >= F.ni || j >= F.nj) continue;
                const int a = j * F.ni + i;
                const float xa = w * F.dinv[a] * F.B[a];
                F.X[a] = xa;
                if (F.dinv[a] != 0.0f) s += F.B[a] - mg_apply9_f(F, a, i, j, xa, y);
              }
            C.B[c] = s;
          }))
        return false;
    } else {
      if (local) {
        // one block's pass is bound by instructions, not barriers: the first
        // sweep is stored instead of being re-formed at every neighbour
        mg_pass(sc, P, M, true, F.n, F.ni, [&](int a, int, int) { F.Y[a] = w * F.dinv[a] * F.B[a]; });
        mg_pass(sc, P, M, true, F.n, F.ni, [&](int a, int i, int j) {
          F.X[a] = F.Y[a] + w * F.dinv[a] * (F.B[a] - mg_apply_l(F, false, F.Y, a, i, j));
        });
      } else if (!mg_pass(sc, P, M, false, F.n, F.ni, [&](int a, int i, int j) {
                   auto y = [&](int b, int, int) { return w * F.dinv[b] * F.B[b]; };
                   const float ba = F.B[a], da = w * F.dinv[a], ya = da * ba;
                   F.X[a] = ya + da * (ba - mg_apply9_f(F, a, i, j, ya, y));
                 })) {
        return false;
      }
      if (!mg_pass(sc, P, M, local, C.n, C.ni, [&](int c, int I, int J) {
            float s = 0.0f;
            for (int dj = 0; dj < 2; ++dj)
              for (int di = 0; di < 2; ++di) {
                const int i = 2 * I + di, j = 2 * J + dj;
                if (i >= F.ni || j >= F.nj) continue;
                const int a = j * F.ni + i;
                if (F.dinv[a] == 0.0f) continue;
                s += F.B[a] - mg_apply_l(F, false, F.X, a, i, j);
              }
            C.B[c] = s;
          }))
        return false;
    }
  }
  if (lf == M.L - 1) take_in();  // the coarsest level is the only local one
  // coarsest (dense inverse, or Jacobi from zero with an even number of sweeps
  // ending in X) and up, block-locally for the local levels
  if (M.cinv_off >= 0) {
    if (mg_runs_local(sc, M)) {
      const MgLv C = mg_level(M, M.L - 1, sm);
      const float *Ai = sm + M.cinv_off;
      const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int r = threadIdx.x >> 5; r < C.n; r += nw) {
        float v = 0.0f;
        for (int c = lane; c < C.n; c += 32) v += Ai[r * C.n + c] * C.B[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) C.X[r] = v;
      }
      __syncthreads();
    }
  } else if (mg_runs_local(sc, M) || M.local_from >= M.L) {
    const int lc = M.L - 1;
    const MgLv C = mg_level(M, lc, sm);
    const bool local = lc >= M.local_from, l0 = lc == 0;
    if (!local || mg_runs_local(sc, M)) {
      mg_pass(sc, P, M, local, C.n, C.ni, [&](int a, int, int) { C.X[a] = w * C.dinv[a] * C.B[a]; });
      for (int k = 0; k < M.coarse_sweeps; ++k) {  // an even count ends in X
        const float *src = (k & 1) ? C.Y : C.X;
        float *dst = (k & 1) ? C.X : C.Y;
        mg_pass(sc, P, M, local, C.n, C.ni, [&](int a, int i, int j) {
          dst[a] = src[a] + w * C.dinv[a] * (C.B[a] - mg_apply_l(C, l0, src, a, i, j));
        });
      }
    }
  }
  float t[2] = {0.0f, 0.0f};
  for (int l = M.L - 2; l >= 0; --l) {
    const bool local = l >= lf;
    if (!local && l + 1 >= lf && lf < M.L && !M.redundant) {
      // leaving the block-local levels: block 0 publishes the first local
      // level's result, and everyone waits for it
      if (sm != nullptr && lf >= M.smem_from) {
        const MgLv G = mg_level(M, lf, nullptr), Sh = mg_level(M, lf, sm);
        for (int a = threadIdx.x; a < G.n; a += blockDim.x) G.X[a] = Sh.X[a];
      }
      if (!sc.sync(P)) return false;
    }
    MgLv F = mg_level(M, l, sm);
    // the first local level's result: the global copy block 0 published, or
    // this block's own
    MgLv C = mg_level(M, l + 1, (l + 1 == lf && !M.redundant) ? nullptr : sm);
    if (l == 0) F.B = b0;
    if (single(l + 1)) {  // that level's result is in its Y
      float *const t = C.X;
      C.X = C.Y;
      C.Y = t;
    }
    if (local && !mg_runs_local(sc, M)) continue;
    // coarse correction folded into the first post-smoothing sweep: the
    // corrected values are formed on the fly at the node and its neighbours
    if (l == 0) {
      // smoothed prolongation: the node's own aggregate and the two across
      // its boundary, with the node's weights
      if (!mg_pass(sc, P, M, local, F.n, F.ni, [&](int a, int i, int j) {
            auto y = [&](int b, int ib, int jb) {
              const int I = ib >> 1, J = jb >> 1;
              const int ix = (ib & 1) ? ib + 1 : ib - 1, jx = (jb & 1) ? jb + 1 : jb - 1;
              const int cx = (ix >= 0 && ix < F.ni) ? (ix >> 1) : I, cy = (jx >= 0 && jx < F.nj) ? (jx >> 1) : J;
              // (the weights are 0 where the neighbour across is missing or not free)
              const float c = F.c2[b] * C.X[J * C.ni + I] + F.c3[b] * C.X[J * C.ni + cx] + F.c4[b] * C.X[cy * C.ni + I];
              return F.dinv[b] != 0.0f ? F.X[b] + al0 * c : 0.0f;
            };
            const float ya = y(a, i, j);
            F.Y[a] = ya + w * F.dinv[a] * (F.B[a] - mg_apply_f(F, a, i, j, ya, y));
          }))
        return false;
    } else if (local) {
      // block-local: the corrected values are stored once (in place in X),
      // then the first sweep reads them
      mg_pass(sc, P, M, true, F.n, F.ni, [&](int a, int i, int j) {
        F.X[a] = F.dinv[a] != 0.0f ? F.X[a] + al * C.X[(j >> 1) * C.ni + (i >> 1)] : 0.0f;
      });
      mg_pass(sc, P, M, true, F.n, F.ni, [&](int a, int i, int j) {
        F.Y[a] = F.X[a] + w * F.dinv[a] * (F.B[a] - mg_apply_l(F, false, F.X, a, i, j));
      });
    } else {
      if (!mg_pass(sc, P, M, false, F.n, F.ni, [&](int a, int i, int j) {
            auto y = [&](int b, int ib, int jb) {
              return F.dinv[b] != 0.0f ? F.X[b] + al * C.X[(jb >> 1) * C.ni + (ib >> 1)] : 0.0f;
            };
            const float ya = y(a, i, j);
            F.Y[a] = ya + w * F.dinv[a] * (F.B[a] - mg_apply9_f(F, a, i, j, ya, y));
          }))
        return false;
    }
    // second post-smoothing sweep: the level's result, in X (at level 0 with
    // the dot products, whose sum below ends the pass)
    const bool l0 = l == 0;
    auto sweep = [&](int a, int i, int j) {
      const float x = F.Y[a] + w * F.dinv[a] * (F.B[a] - mg_apply_l(F, l0, F.Y, a, i, j));
      F.X[a] = x;
      return x;
    };
    if (l == 0) {
      mg_nodes(local ? (int)threadIdx.x : sc.bid() * (int)blockDim.x + (int)threadIdx.x,
               local ? (int)blockDim.x : sc.nblk() * (int)blockDim.x, F.n, F.ni, [&](int a, int i, int j) {
                 const float x = sweep(a, i, j), b = F.B[a];
                 t[0] += b * x;
                 t[1] += b * b;
               });
    } else if (!single(l) && !mg_pass(sc, P, M, local, F.n, F.ni, [&](int a, int i, int j) { sweep(a, i, j); })) {
      return false;
    }
  }
  // every block joins the sum (a hierarchy entirely in block 0, the case of
  // small grids: the others add 0)
  if (!grid_sum_s<float, 2>(sc, t, part32, parity, P)) return false;
  dots[0] = t[0];
  dots[1] = t[1];
  return true;
}

template <class S>
__device__ void pcg_mg_body(const S &sc, const PcgParams &P, const MgLevels &M) {
  extern __shared__ __align__(16) float mg_sm[];
  float *sm = (mg_runs_local(sc, M) && M.smem_floats > 0) ? mg_sm : nullptr;
  const int nn = P.nn;
  float *part32 = reinterpret_cast<float *>(P.partial + 8 * sc.nblk());
  double *r64 = P.work;
  const MgLv L0 = mg_level(M, 0);
  // r and p buffers k = 0, 1
  auto rb = [&](int k) { return k ? M.r2 : L0.B; };
  auto pb = [&](int k) { return k ? M.p2 : M.p; };
  int it = 0, parity = 0, status = -4, outer = 0;
  double b2 = 0.0, r2 = 0.0;
  const int gtid = sc.bid() * blockDim.x + threadIdx.x, gstride = sc.nblk() * blockDim.x;
  if (!mg_setup(sc, P, M, sm)) status = -5;
  for (outer = 0; outer < 64 && status != -5; ++outer) {
    double acc2[2] = {0.0, 0.0};
    residual64_s(sc, P, r64, acc2);
    if (!grid_sum_s<double, 2>(sc, acc2, P.partial, parity, P)) { status = -5; break; }
    parity ^= 1;
    b2 = acc2[0];
    r2 = acc2[1];
    const double target2 = b2 > 0.0 ? P.tol * P.tol * b2 : 1e-60;
    if (!isfinite(r2)) { status = -7; break; }
    if (r2 <= target2) { status = 0; break; }
    if (it >= P.maxit) { status = -4; break; }
    const double inv = rsqrt(r2);
    for (int a = gtid; a < nn; a += gstride) {
      rb(0)[a] = P.node_kind[a] == 0 ? (float)(r64[a] * inv) : 0.0f;
      M.x[a] = 0.0f;
    }
    if (!sc.sync(P)) { status = -5; break; }
    float t2[2];
    if (!mg_vcycle(sc, P, M, sm, rb(0), RhsPlain{rb(0)}, t2, part32, parity)) { status = -5; break; }
    parity ^= 1;
    float rz = t2[0];
    // the V-cycle makes a deeper FP32 inner solve cheap: one outer step fewer
    float stop = fminf(P.inner_tol, 1e-5f);
    const float need = (float)sqrt(target2 / r2);
    if (need > stop) stop = need;
    const float stop2 = stop * stop;
    bool bad = false, fail = false;
    // r and p alternate between two buffers: a pass forms the new values of
    // the neighbours on the fly from the old ones, so no barrier is needed
    // between an update and its first use
    int rc = 0, pc = 0;
    float beta = 0.0f;
    while (it < P.maxit) {
      // p <- z + beta p (into the other buffer), q = A p, p.q
      const float *pold = pb(pc);
      float *pnew = pb(pc ^ 1);
      float pq[1] = {0.0f};
      mg_nodes(gtid, gstride, nn, L0.ni, [&](int a, int i, int j) {
        auto pv = [&](int b, int, int) { return beta != 0.0f ? L0.X[b] + beta * pold[b] : L0.X[b]; };
        const float pa = pv(a, i, j);
        pnew[a] = pa;
        const float qa = L0.dinv[a] != 0.0f ? mg_apply_f(L0, a, i, j, pa, pv) : 0.0f;
        M.q[a] = qa;
        pq[0] += pa * qa;
      });
      if (!grid_sum_s<float, 1>(sc, pq, part32, parity, P)) { fail = true; break; }
      parity ^= 1;
      const float alpha = rz / pq[0];
      ++it;
      // z = V(r - alpha q): the V-cycle's first pass also writes the new r and
      // advances x, its last one forms r.z and r.r
      float t[2];
      const RhsUpdate upd{rb(rc), M.q, pnew, rb(rc ^ 1), M.x, alpha};
      if (!mg_vcycle(sc, P, M, sm, rb(rc ^ 1), upd, t, part32, parity)) { fail = true; break; }
      parity ^= 1;
      rc ^= 1;
      pc ^= 1;
      if (!isfinite(t[0]) || !isfinite(t[1])) { bad = true; break; }
      if (t[1] <= stop2) break;
      beta = t[0] / rz;
      rz = t[0];
    }
    if (fail) { status = -5; break; }
    if (bad) { status = -7; break; }
    const double back = sqrt(r2) * P.gscale;
    for (int a = gtid; a < nn; a += gstride)
      if (P.node_kind[a] == 0) P.phi[a] += (double)M.x[a] * back;
    if (!sc.sync(P)) { status = -5; break; }
  }
  if (sc.bid() == 0 && threadIdx.x == 0) {
    P.out[0] = (double)it;
    P.out[1] = b2 > 0.0 ? sqrt(r2 / b2) : sqrt(r2);
    P.out[2] = (double)status;
    P.out[3] = (double)outer;
    if (status == -4) atomicOr(P.flags, 0x4u);
    if (status == -7) atomicOr(P.flags, 0x8u);
    // Every block read the counter at setup, before its first barrier.  A
    // failed solve may have left the global coarse levels half rebuilt: the
    // next solve then rebuilds the hierarchy (counter 0).
    if (status == 0) *M.solves += 1;
    else *M.solves = 0;
  }
}

__global__ void __launch_bounds__(kMgThreads, 1) k_pcg_mg(const PcgParams P, const MgLevels M) {
  GridScope sc;
  pcg_mg_body(sc, P, M);
}

// One discharge per cluster of CL CTAs (the batched sweep): the same solve with
// hardware cluster barriers in place of the grid barrier, so many solves run
// at once without waiting on one another.
template <int CL>
__global__ void __launch_bounds__(kMgThreads, 1) k_pcg_mg_cluster(const PcgParams P, const MgLevels M) {
  ClusterScope<CL> sc;
  pcg_mg_body(sc, P, M);
}

long long mg_plan(int nr, int nz, MgLevels *M) {
  memset(M, 0, sizeof(*M));
  int ni = nr + 1, nj = nz + 1;
  long long off = 0;
  M->local_from = kMgMaxLevels;
  for (int l = 0; l < kMgMaxLevels; ++l) {
    M->ni[l] = ni;
    M->nj[l] = nj;
    M->off[l] = off;
    off += (long long)kMgArrays * ni * nj;
    M->L = l + 1;
    if (M->local_from == kMgMaxLevels && (long long)ni * nj <= 4096) M->local_from = l;
    if ((long long)ni * nj <= 64 || ni < 3 || nj < 3) break;
    ni = (ni + 1) / 2;
    nj = (nj + 1) / 2;
  }
  // the block-local levels (below level 0) live in shared memory for the
  // whole solve when they fit, one copy per block
  M->smem_from = M->L;
  M->smem_floats = 0;
  if (M->local_from >= 1 && M->local_from < M->L) {
    long long sf = 0;
    for (int l = M->local_from; l < M->L; ++l) {
      M->soff[l] = sf;
      sf += (long long)kMgArrays * M->ni[l] * M->nj[l];
    }
    if (sf <= kMgSmemFloats - kMgDenseMax * kMgDenseMax) {
      M->smem_from = M->local_from;
      M->smem_floats = (int)sf;
      M->redundant = 1;  // every block runs the local levels on its own copy
    }
  }
  // the coarsest level is block-local (at most kMgDenseMax nodes is at most
  // 4096): its dense inverse follows the levels in shared memory
  const int nc = M->ni[M->L - 1] * M->nj[M->L - 1];
  M->cinv_off = -1;
  if (nc <= kMgDenseMax && M->local_from < M->L) {
    M->cinv_off = M->smem_floats;
    M->smem_floats += nc * nc;
  }
  M->omega = 0.8f;
  M->alpha = 1.8f;
  M->alpha0 = 1.0f;
  M->single_sweep = 1;
  M->rebuild_every = 8;
  M->omega_s = 2.0f / 3.0f;  // 4 / (3 lambda_max) with lambda_max(D^-1 A) <= 2
  M->coarse_sweeps = 10;
  return off + 5LL * (nr + 1) * (nz + 1);
}

template <int CL>
static cudaError_t launch_mg_cluster(const PcgParams &P, const MgLevels &M, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(kMgThreads);
  cfg.dynamicSmemBytes = sizeof(float) * (size_t)M.smem_floats;
  cfg.stream = st;
  static bool smem_set = false;
  if (!smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k_pcg_mg_cluster<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float) * kMgSmemFloats));
    if (e != cudaSuccess) return e;
    smem_set = true;
  }
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_pcg_mg_cluster<CL>, P, M);
}

int mg_cluster_size(int nn) { return nn <= 4096 ? 1 : nn <= 9000 ? 2 : nn <= 20000 ? 4 : 8; }

cudaError_t launch_pcg_mg_cluster(const PcgParams &P, const MgLevels &M, int cluster, cudaStream_t st) {
  switch (cluster) {
    case 1: return launch_mg_cluster<1>(P, M, st);
    case 2: return launch_mg_cluster<2>(P, M, st);
    case 4: return launch_mg_cluster<4>(P, M, st);
    case 8: return launch_mg_cluster<8>(P, M, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pcg_mg(const PcgParams &P, const MgLevels &M, int grid, cudaStream_t st) {
  static bool smem_set = false;
  if (!smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k_pcg_mg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float) * kMgSmemFloats));
    if (e != cudaSuccess) return e;
    smem_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kMgThreads);
  cfg.dynamicSmemBytes = sizeof(float) * (size_t)M.smem_floats;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_pcg_mg, P, M);
}

int pcg_grid_size(int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return sms;  // one block per SM (kPcgThreads threads)
}

static cudaError_t launch_coop(void (*kern)(PcgParams), const PcgParams &P, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPcgThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, P);
}

cudaError_t launch_pcg(const PcgParams &P, int grid, cudaStream_t st) { return launch_coop(k_pcg, P, grid, st); }

cudaError_t launch_pcg_mixed(const PcgParams &P, int grid, cudaStream_t st) {
  return launch_coop(k_pcg_mixed, P, grid, st);
}

}  // namespace pic
