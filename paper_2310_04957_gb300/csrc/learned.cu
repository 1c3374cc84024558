// learned.cu -- field solve with the learned preconditioner (Eq. 1 of
// arXiv:2310.04957 solved by flexible conjugate gradients whose
// preconditioner is the U-Net of unet.cu).
//
// With r = b - A phi the residual of the field equation on the free nodes and
// D its diagonal, the preconditioner is
//     z = M(r) = s * U(D^-1 r / s, chi, mask),   s = rms of D^-1 r over the
// free nodes the network covers (i < nr, j < nz); free nodes outside it get
// the Jacobi value D^-1 r.  U is nonlinear, so the search directions are
// A-orthogonalised against the previous one (flexible CG with one stored
// direction):
//     p_k = z_k - beta_k p_{k-1},  beta_k = (z_k . q_{k-1}) / (p_{k-1} . q_{k-1}),
//     q_k = A p_k,  alpha_k = (p_k . r_k) / (p_k . q_k),
//     phi += alpha_k p_k,  r -= alpha_k q_k.
// The first application z_0 = M(r_0) on the warm start's residual is the
// learned initial-guess correction.  All recurrences are FP64; only the
// network runs in BF16/FP32.
//
// The loop runs on the device: one CUDA graph with a while-conditional node
// whose body is [U-Net forward, z, p/q, update, pack]; the pack kernel
// decides whether another iteration is needed and sets the condition.  No
// host round trip per iteration.
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/pic.h"
#include "learned.h"
#include "unet.h"

namespace pic {
namespace learned {

constexpr int kThreads = 256;

// Block sum of K doubles; result in every thread.
template <int K>
__device__ __forceinline__ void block_sum(double v[K]) {
  __shared__ double s[K][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s[k][wid] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) x += s[k][w];
    v[k] = x;
  }
  __syncthreads();
}

// Writes this block's K partial sums to set `set`.
template <int K>
__device__ __forceinline__ void put_partial(const FcgParams &P, int set, double v[K]) {
  block_sum<K>(v);
  if (threadIdx.x < K) P.part[((size_t)set * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = v[threadIdx.x];
}

// Sums the partials of set `set` (written by the previous kernel) in a fixed
// order: every block obtains bit-identical totals.
template <int K>
__device__ __forceinline__ void get_total(const FcgParams &P, int set, double v[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __ldcg(P.part + ((size_t)set * gridDim.x + b) * 4 + k);
  block_sum<K>(v);
}

__device__ __forceinline__ bool in_net(const FcgParams &P, int i, int j) { return i < P.W && j < P.H; }

// (A v)_a at free node a, v given by a functor of the node index (Dirichlet nodes 0).
template <class V>
__device__ __forceinline__ double apply_A(const FcgParams &P, int a, int i, int j, double va, V v) {
  const int nr = P.nr, W1 = nr + 1;
  double s = 0.0;
  if (i > 0) s += __ldg(P.Gr + j * nr + i - 1) * (va - v(a - 1));
  if (i < nr) s += __ldg(P.Gr + j * nr + i) * (va - v(a + 1));
  if (j > 0) s += __ldg(P.Gz + (j - 1) * W1 + i) * (va - v(a - W1));
  if (j < P.nz) s += __ldg(P.Gz + j * W1 + i) * (va - v(a + W1));
  return s;
}

// Start: r = b - A phi (phi holds the warm start and the Dirichlet values),
// network channels 1 (chi) and 2 (Dirichlet mask), previous direction = 0.
// Partials (set 3): ||b||^2, ||r||^2, ||D^-1 r||^2 over covered free nodes.
__global__ void __launch_bounds__(kThreads) k_fcg_start(const FcgParams P) {
  const int nr = P.nr, W1 = nr + 1, HW = P.H * P.W;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < P.nn; a += gridDim.x * blockDim.x) {
    const int j = a / W1, i = a - j * W1;
    const int8_t kind = P.node_kind[a];
    P.p[0][a] = 0.0;
    P.p[1][a] = 0.0;
    P.q[0][a] = 0.0;
    P.q[1][a] = 0.0;
    if (in_net(P, i, j)) {
      const int px = j * P.W + i;
      P.in3[HW + px] = (float)P.chi[a];
      P.in3[2 * HW + px] = kind != 0 ? 1.0f : 0.0f;
    }
    if (kind != 0) {
      P.r[a] = 0.0;
      continue;
    }
    const double pa = P.phi[a];
    auto v = [&](int b) { return P.phi[b]; };
    const double ax = apply_A(P, a, i, j, pa, v);
    // lift = sum of G_ab phi_b over Dirichlet neighbours b (b = q + lift)
    double lift = 0.0;
    if (i > 0 && P.node_kind[a - 1] != 0) lift += __ldg(P.Gr + j * nr + i - 1) * P.phi[a - 1];
    if (i < nr && P.node_kind[a + 1] != 0) lift += __ldg(P.Gr + j * nr + i) * P.phi[a + 1];
    if (j > 0 && P.node_kind[a - W1] != 0) lift += __ldg(P.Gz + (j - 1) * W1 + i) * P.phi[a - W1];
    if (j < P.nz && P.node_kind[a + W1] != 0) lift += __ldg(P.Gz + j * W1 + i) * P.phi[a + W1];
    const double q = __ldg(P.qrhs + a);
    const double r = q - ax, b = q + lift;
    P.r[a] = r;
    acc[0] += b * b;
    acc[1] += r * r;
    if (in_net(P, i, j)) {
      const double u = __ldg(P.dinv + a) * r;
      acc[2] += u * u;
    }
  }
  put_partial<3>(P, 3, acc);
}

// Convergence test and the next network input.  `first` reads the start
// partials (and records ||b||^2); otherwise the update's.  Block 0 sets the
// loop condition; every block packs channel 0 = D^-1 r / s.
__global__ void __launch_bounds__(kThreads) k_fcg_pack(const FcgParams P, cudaGraphConditionalHandle cond, int first) {
  double t[3];
  get_total<3>(P, first ? 3 : 0, t);
  const double b2 = first ? t[0] : __ldcg(P.sc + 0);
  const double r2 = t[1], s2 = t[2];
  const int it = first ? 0 : (int)__ldcg(P.sc + 7);
  int status = 1;  // 1 = continue
  if (!isfinite(r2) || !isfinite(s2)) status = -7;
  else if (r2 <= (b2 > 0.0 ? P.tol * P.tol * b2 : 1e-60)) status = 0;
  else if (it >= P.maxit) status = -4;
  else if (!(s2 > 0.0)) status = -7;  // residual only outside the network: cannot precondition
  const double s = status == 1 ? sqrt(s2 / (double)P.n_cov) : 1.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (first) P.sc[0] = b2;
    P.sc[1] = r2;
    P.sc[3] = s;
    P.sc[4] = it;
    P.sc[5] = status;
    cudaGraphSetConditional(cond, status == 1 ? 1u : 0u);
  }
  if (status != 1) return;
  const double inv = 1.0 / s;
  const int W1 = P.nr + 1;
  for (int px = blockIdx.x * blockDim.x + threadIdx.x; px < P.H * P.W; px += gridDim.x * blockDim.x) {
    const int j = px / P.W, i = px - j * P.W, a = j * W1 + i;
    P.in3[px] = P.node_kind[a] == 0 ? (float)(__ldg(P.dinv + a) * __ldcg(P.r + a) * inv) : 0.0f;
  }
}

// z = s * U(.) on covered free nodes, D^-1 r on the other free nodes; partial
// (set 1) z . q_prev (used when no smoothing step follows).
__global__ void __launch_bounds__(kThreads) k_fcg_z(const FcgParams P) {
  const int W1 = P.nr + 1;
  const int it = (int)__ldcg(P.sc + 4);
  const double s = __ldcg(P.sc + 3);
  const double *qprev = P.q[(it + 1) & 1];
  double acc[1] = {0.0};
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < P.nn; a += gridDim.x * blockDim.x) {
    const int j = a / W1, i = a - j * W1;
    double z = 0.0;
    if (P.node_kind[a] == 0)
      z = in_net(P, i, j) ? (double)__ldcg(P.out_net + j * P.W + i) * s : __ldg(P.dinv + a) * __ldcg(P.r + a);
    P.z[a] = z;
    acc[0] += z * __ldcg(qprev + a);
  }
  put_partial<1>(P, 1, acc);
}

// One damped Jacobi step on A z = r: z' = z + omega D^-1 (r - A z), from
// P.z into `to` (the caller alternates buffers and leaves the result in P.z);
// partial (set 1) z' . q_prev.
__global__ void __launch_bounds__(kThreads) k_fcg_smooth(const FcgParams P, const double *from, double *to,
                                                         double omega) {
  const int W1 = P.nr + 1;
  const int it = (int)__ldcg(P.sc + 4);
  const double *qprev = P.q[(it + 1) & 1];
  auto zv = [&](int b) { return __ldcg(from + b); };
  double acc[1] = {0.0};
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < P.nn; a += gridDim.x * blockDim.x) {
    double z = 0.0;
    if (P.node_kind[a] == 0) {
      const int j = a / W1, i = a - j * W1;
      const double za = zv(a);
      z = za + omega * __ldg(P.dinv + a) * (__ldcg(P.r + a) - apply_A(P, a, i, j, za, zv));
    }
    to[a] = z;
    acc[0] += z * __ldcg(qprev + a);
  }
  put_partial<1>(P, 1, acc);
}

// beta, p_k = z_k - beta p_{k-1}, q_k = A p_k (neighbours' p_k formed on the
// fly); partials (set 2) p.q and p.r.
__global__ void __launch_bounds__(kThreads) k_fcg_pq(const FcgParams P) {
  double t[1];
  get_total<1>(P, 1, t);
  const int it = (int)__ldcg(P.sc + 4);
  const double beta = it > 0 ? t[0] / __ldcg(P.sc + 2) : 0.0;
  const double *pold = P.p[(it + 1) & 1];
  double *pnew = P.p[it & 1], *qnew = P.q[it & 1];
  const int W1 = P.nr + 1;
  auto pk = [&](int b) { return __ldcg(P.z + b) - beta * __ldcg(pold + b); };
  double acc[2] = {0.0, 0.0};
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < P.nn; a += gridDim.x * blockDim.x) {
    if (P.node_kind[a] != 0) {
      pnew[a] = 0.0;
      qnew[a] = 0.0;
      continue;
    }
    const int j = a / W1, i = a - j * W1;
    const double pa = pk(a);
    const double qa = apply_A(P, a, i, j, pa, pk);
    pnew[a] = pa;
    qnew[a] = qa;
    acc[0] += pa * qa;
    acc[1] += pa * __ldcg(P.r + a);
  }
  put_partial<2>(P, 2, acc);
}

// alpha, phi += alpha p, r -= alpha q; partials (set 0) ||r||^2, ||D^-1 r||^2.
__global__ void __launch_bounds__(kThreads) k_fcg_update(const FcgParams P) {
  double t[2];
  get_total<2>(P, 2, t);
  const int it = (int)__ldcg(P.sc + 4);
  const double pq = t[0], alpha = pq != 0.0 ? t[1] / pq : 0.0;
  const double *p = P.p[it & 1], *q = P.q[it & 1];
  const int W1 = P.nr + 1;
  const bool snap = P.snap && it + 1 == (int)__ldcg(P.sc + 6);
  double acc[3] = {0.0, 0.0, 0.0};
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < P.nn; a += gridDim.x * blockDim.x) {
    if (P.node_kind[a] != 0) {
      if (snap) P.snap[a] = P.phi[a];
      continue;
    }
    const int j = a / W1, i = a - j * W1;
    P.phi[a] += alpha * __ldcg(p + a);
    if (snap) P.snap[a] = P.phi[a];
    const double r = __ldcg(P.r + a) - alpha * __ldcg(q + a);
    P.r[a] = r;
    acc[1] += r * r;
    if (in_net(P, i, j)) {
      const double u = __ldg(P.dinv + a) * r;
      acc[2] += u * u;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.sc[2] = pq;
    P.sc[7] = it + 1;
  }
  put_partial<3>(P, 0, acc);
}

// Final statistics: [0] iterations, [1] relative residual, [2] status, [3] 0.
__global__ void k_fcg_finish(const FcgParams P) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double b2 = P.sc[0], r2 = P.sc[1];
    P.stats[0] = P.sc[4];
    P.stats[1] = b2 > 0.0 ? sqrt(r2 / b2) : sqrt(r2);
    P.stats[2] = P.sc[5];
    P.stats[3] = 0.0;
  }
}

// ---- training pairs ----------------------------------------------------------------
// From the warm start phi_w of the last solve and its solution phi:
// r0 = b - A phi_w, delta = phi - phi_w.  Channel 0 = D^-1 r0 / s, target =
// delta / s, s = rms of D^-1 r0 over covered free nodes (computed by the caller
// from the returned sum of squares in two passes: pass 0 sums, pass 1 scales).
__global__ void __launch_bounds__(kThreads) k_pair(const FcgParams P, const double *phi_w, float *target, int pass,
                                                   const double *s2sum) {
  const int nr = P.nr, W1 = nr + 1, HW = P.H * P.W;
  double acc[1] = {0.0};
  const double inv = pass ? 1.0 / sqrt(__ldcg(s2sum) / (double)P.n_cov) : 0.0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < P.nn; a += gridDim.x * blockDim.x) {
    const int j = a / W1, i = a - j * W1;
    if (!in_net(P, i, j)) continue;
    const int px = j * P.W + i;
    const int8_t kind = P.node_kind[a];
    if (kind != 0) {
      if (pass) {
        P.in3[px] = 0.0f;
        P.in3[HW + px] = (float)P.chi[a];
        P.in3[2 * HW + px] = 1.0f;
        target[px] = 0.0f;
      }
      continue;
    }
    auto v = [&](int b) { return phi_w[b]; };
    const double r = __ldg(P.qrhs + a) - apply_A(P, a, i, j, phi_w[a], v);
    const double u = __ldg(P.dinv + a) * r;
    if (pass) {
      P.in3[px] = (float)(u * inv);
      P.in3[HW + px] = (float)P.chi[a];
      P.in3[2 * HW + px] = 0.0f;
      target[px] = (float)((P.phi[a] - phi_w[a]) * inv);
    } else {
      acc[0] += u * u;
    }
  }
  if (!pass) {
    block_sum<1>(acc);
    if (threadIdx.x == 0) atomicAdd(const_cast<double *>(s2sum), acc[0]);
  }
}

// ---- host ------------------------------------------------------------------------------
int node_blocks(int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return 2 * (sms > 0 ? sms : 1);
}

// Builds the executable graph: start, pack(first), while { U-Net, z, pq,
// update, pack }, finish.
cudaError_t build_fcg_graph(const FcgParams &P, int nblk, pic_unet *net, cudaStream_t side, cudaGraphExec_t *exec) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle cond;
  std::vector<cudaGraphNode_t> deps;
  cudaGraphNode_t cnode = nullptr;
  auto fail = [&](cudaError_t err) {
    cudaStreamCaptureStatus stt;
    if (cudaStreamIsCapturing(side, &stt) == cudaSuccess && stt != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(side, &junk);
    }
    cudaGetLastError();
    cudaGraphDestroy(g);
    return err;
  };
  if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) return fail(e);
  // prologue
  if ((e = cudaStreamBeginCaptureToGraph(side, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return fail(e);
  k_fcg_start<<<nblk, kThreads, 0, side>>>(P);
  k_fcg_pack<<<nblk, kThreads, 0, side>>>(P, cond, 1);
  {
    cudaStreamCaptureStatus stt;
    const cudaGraphNode_t *d = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(side, &stt, nullptr, nullptr, &d, nullptr, &nd)) != cudaSuccess) return fail(e);
    deps.assign(d, d + nd);
  }
  {
    cudaGraph_t out = nullptr;
    if ((e = cudaStreamEndCapture(side, &out)) != cudaSuccess) return fail(e);
  }
  // loop
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if ((e = cudaGraphAddNode(&cnode, g, deps.data(), nullptr, deps.size(), &cp)) != cudaSuccess) return fail(e);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return fail(e);
  if (pic::unet::forward_on_stream(net, P.in3, P.out_net, side) != PIC_OK) return fail(cudaErrorUnknown);
  k_fcg_z<<<nblk, kThreads, 0, side>>>(P);
  // smoothing steps alternate z -> z2 -> z ...; an odd count ends in z2, so the
  // pq kernel reads whichever buffer holds the last result
  FcgParams Q = P;
  for (int k = 0; k < P.smooth; ++k) {
    const double *from = (k & 1) ? P.z2 : P.z;
    double *to = (k & 1) ? P.z : P.z2;
    k_fcg_smooth<<<nblk, kThreads, 0, side>>>(P, from, to, P.omega);
  }
  if (P.smooth & 1) Q.z = P.z2;
  k_fcg_pq<<<nblk, kThreads, 0, side>>>(Q);
  k_fcg_update<<<nblk, kThreads, 0, side>>>(P);
  k_fcg_pack<<<nblk, kThreads, 0, side>>>(P, cond, 0);
  {
    cudaGraph_t out = nullptr;
    if ((e = cudaStreamEndCapture(side, &out)) != cudaSuccess) return fail(e);
  }
  // epilogue
  if ((e = cudaStreamBeginCaptureToGraph(side, g, &cnode, nullptr, 1, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return fail(e);
  k_fcg_finish<<<1, 32, 0, side>>>(P);
  {
    cudaGraph_t out = nullptr;
    if ((e = cudaStreamEndCapture(side, &out)) != cudaSuccess) return fail(e);
  }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

cudaError_t launch_pair(const FcgParams &P, int nblk, const double *phi_w, float *target, double *s2sum,
                        cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(s2sum, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  k_pair<<<nblk, kThreads, 0, st>>>(P, phi_w, target, 0, s2sum);
  k_pair<<<nblk, kThreads, 0, st>>>(P, phi_w, target, 1, s2sum);
  return cudaGetLastError();
}

}  // namespace learned
}  // namespace pic
