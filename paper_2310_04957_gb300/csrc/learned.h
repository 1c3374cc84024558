// learned.h -- internal interface of the learned-preconditioner field solve.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pic.h"

namespace pic {
namespace learned {

struct FcgParams {
  int nr, nz, nn;
  int H, W;        // network grid: nodes i < W, j < H (W = nr, H = nz)
  int n_cov;       // free nodes the network covers
  const int8_t *node_kind;
  const double *Gr, *Gz, *dinv, *qrhs, *chi;
  double *phi;     // warm start in, solution out (Dirichlet values fixed)
  double *r, *z, *z2;  // [nn]
  int smooth;      // damped Jacobi steps after each network application
  double omega;    // their damping
  double *p[2], *q[2];
  double *part;    // [4 sets][blocks][4] partial sums
  double *sc;      // [8] scalars: ||b||^2, ||r||^2, p.q, s, it, status, snapshot iteration, it+1
  double *snap;    // phi after the snapshot iteration (sc[6] > 0), for training pairs
  float *in3;      // network input [3][H*W]
  float *out_net;  // network output [H*W]
  double tol;
  int maxit;
  double *stats;   // [4] iterations, relative residual, status (0 ok, -4 cap, -7 non-finite), 0
};

int node_blocks(int device);
cudaError_t build_fcg_graph(const FcgParams &P, int nblk, pic_unet *net, cudaStream_t side, cudaGraphExec_t *exec);
cudaError_t launch_pair(const FcgParams &P, int nblk, const double *phi_w, float *target, double *s2sum,
                        cudaStream_t st);

}  // namespace learned
}  // namespace pic
