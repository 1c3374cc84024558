// upload.cu -- binning of uploaded particles on the device (pic_set_particles).
#include <cstdint>

#include "pic_device.cuh"
#include "pic_kernels.h"

namespace pic {

// ---------------------------------------------------------------------------
// Upload of one species from its raw FP64 columns (already on the device).
// Pass 1: each particle's cell (checked: r, z >= 0, inside the grid, a plasma
// cell; a weight ratio in (0, 1]), its cell-relative offsets in the store's
// precision (below 1) and its
// rank within its bin (one atomic per particle: the order inside a bin is
// arbitrary, which nothing downstream depends on).  Pass 2, after the bins'
// starts are known: the scatter into the binned store.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_upload_bin(UploadParams<T> U) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < U.n; k += stride) {
    const double r = U.r[k], z = U.z[k];
    int bin = -1;
    const bool w_ok = !U.w || (U.w[k] > 0.0 && U.w[k] <= 1.0);
    if (w_ok && r >= 0.0 && z >= 0.0) {
      const double x = r / U.dr, y = z / U.dz;
      const double fx = floor(x), fy = floor(y);
      const int i = fx < 2.0e9 ? (int)fx : U.map.nr, j = fy < 2.0e9 ? (int)fy : U.map.nz;
      if (i < U.map.nr && j < U.map.nz && U.cell_kind[(size_t)j * U.map.nr + i] == 0) {  // plasma cell
        T a = (T)(x - i), b = (T)(y - j);
        const T below1 = (T)1 - (T)(sizeof(T) == 4 ? 5.9604645e-8 : 1.1102230246251565e-16);
        if (a >= (T)1) a = below1;
        if (b >= (T)1) b = below1;
        if (a < (T)0) a = (T)0;
        if (b < (T)0) b = (T)0;
        U.fr_tmp[k] = a;
        U.fz_tmp[k] = b;
        bin = U.map.bin(i, j);
      }
    }
    if (bin < 0) {
      atomicOr(U.err, 1u);
      U.bin_rank[k] = make_int2(0, 0);
      continue;
    }
    U.bin_rank[k] = make_int2(bin, atomicAdd(U.count + bin, 1));
  }
}

template <typename T>
__global__ void k_upload_scatter(UploadParams<T> U) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < U.n; k += stride) {
    const int2 br = U.bin_rank[k];
    const int d = U.start[br.x] + br.y;
    const StoreView<T> &S = U.out;
    S.pa[d] = Vec4<T>{U.fr_tmp[k], U.fz_tmp[k], (T)U.vr[k], (T)U.vt[k]};
    S.pb[d] = Vec4<T>{(T)U.vz[k], (T)U.ar[k], (T)U.at[k], (T)U.az[k]};
    S.id[d] = U.id[k];
    if (S.w) S.w[d] = U.w ? (T)U.w[k] : (T)1;
  }
}

template <typename T>
cudaError_t launch_upload_bin(const UploadParams<T> &U, cudaStream_t st) {
  int64_t blocks = (U.n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  k_upload_bin<T><<<(int)blocks, 256, 0, st>>>(U);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_upload_scatter(const UploadParams<T> &U, cudaStream_t st) {
  int64_t blocks = (U.n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  k_upload_scatter<T><<<(int)blocks, 256, 0, st>>>(U);
  return cudaGetLastError();
}

template cudaError_t launch_upload_bin<float>(const UploadParams<float> &, cudaStream_t);
template cudaError_t launch_upload_bin<double>(const UploadParams<double> &, cudaStream_t);
template cudaError_t launch_upload_scatter<float>(const UploadParams<float> &, cudaStream_t);
template cudaError_t launch_upload_scatter<double>(const UploadParams<double> &, cudaStream_t);

}  // namespace pic
