// push_w.cu -- the fused particle kernel for weighted particles (per-particle
// weight ratios, splitting near the axis), in a translation unit of its own.
#include "push_kernels.cuh"

namespace pic {

template <typename T>
cudaError_t launch_particles_weighted(const PushParams<T> &P, cudaStream_t st) {
  return launch_particles_tiles<T, true>(P, st);
}

template cudaError_t launch_particles_weighted<float>(const PushParams<float> &, cudaStream_t);
template cudaError_t launch_particles_weighted<double>(const PushParams<double> &, cudaStream_t);

}  // namespace pic
