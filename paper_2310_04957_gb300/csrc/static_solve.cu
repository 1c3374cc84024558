// static_solve.cu -- field solve on caller-owned device arrays that allocates
// no device memory.
//
// Some callers cannot allocate GPU memory at the point where they need a
// field solve: an application whose device memory is owned by its own pool
// allocator and that forbids allocations outside it, or a plugin invoked from
// a real-time loop that must not block on the allocator.  For them,
// pic_pcg_solve_static runs the same Jacobi PCG as pic_field_solve on arrays
// they already own, and keeps its work vectors in one fixed-size device array
// that lives in this library for the life of the process (on every GPU that
// loads it).  pic_pcg_static_result reads back the last call's outcome.
#include <cstdint>
#include <mutex>

#include "../../include/pic.h"
#include "pic_kernels.h"

namespace {

constexpr int kMaxPcgBlocks = 1024;
constexpr size_t kVecs = 9;  // 8 solver work vectors + the diagonal inverse
constexpr size_t kPartial = 8 * (kMaxPcgBlocks + 32);
constexpr size_t kStaticDoubles = kVecs * PIC_STATIC_MAX_NODES + kPartial + 8 + 8;

// The shared work area: every call uses it and it keeps the last call's
// contents; calls whose work overlaps on the GPU race on it.
static __device__ __align__(256) double g_scratch[kStaticDoubles];

std::mutex g_mutex;
double *g_ptr[256] = {nullptr};

// Device address of g_scratch on the current device, looked up once per device.
int scratch_address(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return PIC_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return PIC_ECUDA;
    }
    g_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_ptr[dev];
  return PIC_OK;
}

// Jacobi diagonal of the free nodes: 1 / sum of the node's edge conductances.
__global__ void k_diag_inverse(int nr, int nz, const int8_t *kind, const double *Gr, const double *Gz, double *dinv) {
  const int W = nr + 1, nn = W * (nz + 1);
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nn; a += gridDim.x * blockDim.x) {
    int j = a / W, i = a - j * W;
    double d = 0.0;
    if (i > 0) d += Gr[j * nr + i - 1];
    if (i < nr) d += Gr[j * nr + i];
    if (j > 0) d += Gz[(j - 1) * W + i];
    if (j < nz) d += Gz[j * W + i];
    dinv[a] = (kind[a] == 0 && d > 0.0) ? 1.0 / d : 0.0;
  }
}

}  // namespace

extern "C" int pic_pcg_solve_static(int32_t nr, int32_t nz, const int8_t *node_kind, const double *Gr,
                                    const double *Gz, const double *qrhs, double *phi, double tol, int32_t maxit,
                                    void *cuda_stream, int32_t *iters, double *rel_resid) {
  if (nr < 1 || nz < 1 || !node_kind || !Gr || !Gz || !qrhs || !phi || !(tol > 0) || maxit < 1) return PIC_EINVAL;
  const long long nn = (long long)(nr + 1) * (nz + 1);
  if (nn > PIC_STATIC_MAX_NODES) return PIC_EINVAL;  // beyond the fixed work area
  double *base = nullptr;
  int st = scratch_address(&base);
  if (st) return st;
  int dev = 0;
  cudaGetDevice(&dev);
  int grid = pic::pcg_grid_size(dev);
  if (grid > kMaxPcgBlocks) grid = kMaxPcgBlocks;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double *work = base, *dinv = work + 8 * (size_t)PIC_STATIC_MAX_NODES;
  double *partial = dinv + PIC_STATIC_MAX_NODES, *out = partial + kPartial;
  unsigned *bar = reinterpret_cast<unsigned *>(out + 8);
  // what must start at zero: the grid-barrier counter and the result slots
  if (cudaMemsetAsync(out, 0, 16 * sizeof(double), s) != cudaSuccess) return PIC_ECUDA;
  int blocks = (int)((nn + 255) / 256);
  if (blocks > 2048) blocks = 2048;
  k_diag_inverse<<<blocks, 256, 0, s>>>(nr, nz, node_kind, Gr, Gz, dinv);
  if (cudaGetLastError() != cudaSuccess) return PIC_ECUDA;
  pic::PcgParams P = {};
  P.nr = nr; P.nz = nz; P.nn = (int)nn;
  P.node_kind = node_kind;
  P.Gr = Gr; P.Gz = Gz; P.dinv = dinv; P.qrhs = qrhs; P.phi = phi;
  P.work = work;
  P.work32 = nullptr;
  P.partial = partial;
  P.bar = bar;
  P.tol = tol;
  P.maxit = maxit;
  P.gscale = 1.0;
  P.out = out;
  P.flags = reinterpret_cast<uint32_t *>(bar + 2);
  P.spin_limit = 4000000000ll;
  if (pic::launch_pcg(P, grid, s) != cudaSuccess) return PIC_ECUDA;
  if (!iters && !rel_resid) return PIC_OK;
  double res[3];
  if (cudaMemcpyAsync(res, out, sizeof(res), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PIC_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
  if (iters) *iters = (int32_t)res[0];
  if (rel_resid) *rel_resid = res[1];
  int code = (int)res[2];
  return code == 0 ? PIC_OK : (code == -5 ? PIC_ETIMEOUT : (code == -7 ? PIC_ENAN : PIC_ENOCONV));
}

// Outcome of the last pic_pcg_solve_static call on the current device, read
// from the result slots of the shared work area after `cuda_stream` drains.
extern "C" int pic_pcg_static_result(void *cuda_stream, int32_t *iters, double *rel_resid) {
  double *base = nullptr;
  int st = scratch_address(&base);
  if (st) return st;
  const double *out = base + kVecs * (size_t)PIC_STATIC_MAX_NODES + kPartial;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double res[3];
  if (cudaMemcpyAsync(res, out, sizeof(res), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PIC_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PIC_ECUDA;
  if (iters) *iters = (int32_t)res[0];
  if (rel_resid) *rel_resid = res[1];
  int code = (int)res[2];
  return code == 0 ? PIC_OK : (code == -5 ? PIC_ETIMEOUT : (code == -7 ? PIC_ENAN : PIC_ENOCONV));
}
