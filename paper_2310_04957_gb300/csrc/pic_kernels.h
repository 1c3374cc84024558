// pic_kernels.h -- parameter blocks and launchers of the library's kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pic_device.cuh"

namespace pic {

constexpr int kMaxTileCells = 256;

// Voltage-driven electrodes: electrode k (node kind 3 + k) at V[k] sin(2 pi f[k] t + phase[k]).
struct Drive {
  int n;
  double V[3], f[3], phase[3];
  __device__ __forceinline__ double voltage(int k, double t) const {
    return V[k] * sin(6.283185307179586476925286766559 * f[k] * t + phase[k]);
  }
};

template <typename T>
struct PushParams {
  BinMap map;
  int nr, nz;
  T dt, hdt, hdt2, dr, dz, inv_dr, inv_dz;
  const int8_t *cell_kind;  // [nz*nr]
  const int8_t *node_kind;  // [(nz+1)*(nr+1)]
  const void *E;            // node (E_r, E_z) as float2 / double2
  T qm[2];
  T pcoll[2], numax[2], n_gas;
  const T *xs_E, *xs_S;     // [n_xs], [5*n_xs]
  const float4 *xs_g;       // FP32 lookup groups: per interval k, electrons (sigma_el,
                            // sigma_ex, sigma_iz at E_k, 0) then their slopes per eV,
                            // then ions (sigma_iso, sigma_cx, slopes): [3*(n_xs-1)]
  int n_xs;
  T log2E0, inv_dlog2;
  T thr_ex, thr_iz, B_ej;
  T e_per_v2[2];            // table energy per v^2 (eV s^2/m^2): electron 1/2 m_e/e; ion 1/2 M_gas/e
  T v2_per_e[2];            // electron 2e/m_e
  T two_me_over_M;
  T vth_gas;                // sqrt(k T_gas / M_gas)
  T mi_frac;                // m_ion / (m_ion + M_gas)
  uint32_t seed;
  const uint32_t *step_ptr; // device step counter (Philox counter word 0)
  StoreView<T> in[2], out[2];
  unsigned long long *dep[2];
  unsigned long long *surf[2];
  unsigned long long *counters;
  T dep_scale;
  unsigned long long dep_one;
  uint32_t *flags;
  int weighted;             // particles carry weight ratios (store column w)
  int split_cells;          // split heavy particles in the first split_cells radial cells (0: off)
};

struct FieldParams {
  int nr, nz, nn;
  const int8_t *node_kind;
  const double *Gvac_r, *Gpl_r, *Gvac_z, *Gpl_z;
  const double *vnode;
  const unsigned long long *dep[2];
  const unsigned long long *surf[2];
  double surf_scale;        // macro particles per surface-tally unit (1, or 2^-32 weighted)
  double dep_inv_scale;
  double qw[2];             // q_s w_s
  double chi_coef[2];       // dt^2/(2 eps0) q_s^2/m_s w_s
  double *chi, *qrhs, *phi, *Gr, *Gz, *dinv;
  double *scalars;
  int vahedi;               // phi is phi_P: every electrode at 0
  Drive drive;              // voltage-driven electrodes (node kinds 3..)
};

// Unit-voltage boundary of electrode kind `e`: 1 on it, 0 on every other metal node.
cudaError_t launch_set_dirichlet_unit(int nn, const int8_t *kind, double *phi, int e, cudaStream_t st);
// Eq. 2: phi = phi_P + U_E phi_L0 + sum_k U_k phi_Lk (U_E and t from the scalars).
struct VahediParams {
  int nn;
  const double *phiP, *phiL[4];
  double *phi;
  const double *scalars;
  Drive drive;
};
cudaError_t launch_vahedi_combine(const VahediParams &V, cudaStream_t st);

// Field solve on the free nodes of sum_b G_ab (phi_a - phi_b) = qrhs_a.
// work: [8*nn] doubles (plain) -- r[2], w[2], s[2], p, spare;
// work32: [11*nn] floats (mixed) -- r[2], w[2], s[2], p, x, Gr, Gz, dinv.
struct PcgParams {
  int nr, nz, nn;
  const int8_t *node_kind;
  const double *Gr, *Gz, *dinv, *qrhs;
  double *phi;
  double *work;
  float *work32;
  double *partial;          // [16 * gridDim.x]: FP64 partials, then FP32 partials (mixed)
  unsigned *bar;            // [2]: arrival count, generation
  double tol;               // relative residual target ||b - A phi|| <= tol ||b||
  float inner_tol;          // mixed: relative reduction of each FP32 inner solve
  double gscale;            // mixed: scale making the FP32 operator entries O(1)
  int maxit;                // iteration cap (total inner iterations for mixed)
  double *out;              // [0] iterations, [1] relative residual, [2] status, [3] outer steps
  uint32_t *flags;
  long long spin_limit;     // clock cycles per barrier wait
};

struct EfieldParams {
  int nr, nz;
  double dr, dz;
  const int8_t *node_kind;
  const double *phi;
  double *Er, *Ez;
  float2 *E32;
  double2 *E64;
};

struct CircuitParams {
  int kind, nsub;
  double c[8];
  double V, f, phase, dt;
  double qw[2];
  const unsigned long long *counters;
  int weighted;             // absorbed charge from the weighted tallies
  const uint32_t *step_ptr;
  double *scalars;
  int n_run;                // steps to advance (1 inside the step graph)
  double *U_hist;           // optional U_E history [n_run]
  uint32_t *step_inc;       // if non-null, incremented once per advanced step
  double *prop;             // [64] step propagator (k_circuit_prepare)
};

struct DiagParams {
  int nn;
  int kind;                 // circuit (PIC_CIRCUIT_*) and its parameters, for the
  double c[8];              // circuit post-processing of the window
  double V, phase;
  const double *vnode;
  const unsigned long long *dep[2];
  double dep_inv_scale;
  double w[2];
  double qw_ion;
  double f, dt;
  int window;
  const unsigned long long *counters;
  int weighted;             // absorbed charge from the weighted tallies
  const uint32_t *step_ptr;
  uint32_t *step_mut;
  double *dens_sum[2], *dens_avg[2];
  double *scalars;
};

template <typename T> cudaError_t launch_particles(const PushParams<T> &P, cudaStream_t st);
template <typename T> cudaError_t launch_particles_weighted(const PushParams<T> &P, cudaStream_t st);
bool tile_supported(int tx, int ty);
template <typename T> cudaError_t launch_deposit_only(const PushParams<T> &P, cudaStream_t st);
struct LayoutParams {
  const int *fill_in[2];
  const int8_t *bin_plasma;
  int nbins;
  float slack;
  int capacity[2];
  int *start[2], *cap[2], *fill_out[2];
  BinMeta *meta_out[2], *meta_in[2];
  long long *part;          // [2 * nblk * 4]
  long long *boff;          // [2 * nblk]
  int *use_slack;           // [2]
};
cudaError_t launch_layout(const LayoutParams &L, cudaStream_t st);

// Upload of one species from raw FP64 device columns into the binned store.
template <typename T>
struct UploadParams {
  int64_t n;
  const double *r, *z, *vr, *vt, *vz, *ar, *at, *az;
  const unsigned long long *id;
  const double *w;   // weight ratios (weighted stores; nullptr: all 1)
  double dr, dz;
  BinMap map;
  const int8_t *cell_kind;
  int *count;        // [nbins] particles per bin (pass 1 adds)
  const int *start;  // [nbins] first slot of each bin (pass 2)
  int2 *bin_rank;    // [n] bin and rank within it
  T *fr_tmp, *fz_tmp;
  unsigned *err;     // set to 1 if any particle is outside the plasma or has a ratio outside (0, 1]
  StoreView<T> out;
};
template <typename T> cudaError_t launch_upload_bin(const UploadParams<T> &U, cudaStream_t st);
template <typename T> cudaError_t launch_upload_scatter(const UploadParams<T> &U, cudaStream_t st);
cudaError_t launch_philox(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, cudaStream_t st);

cudaError_t launch_assemble(const FieldParams &F, cudaStream_t st);
cudaError_t launch_assemble_edges_only(const FieldParams &F, cudaStream_t st);
cudaError_t launch_set_dirichlet(int nn, const int8_t *kind, double *phi, double U, cudaStream_t st);
cudaError_t launch_pcg(const PcgParams &P, int grid, cudaStream_t st);
cudaError_t launch_pcg_mixed(const PcgParams &P, int grid, cudaStream_t st);
int pcg_grid_size(int device);
constexpr int kPcgThreads = 256;

// Multigrid-preconditioned mixed solve: 2x2 aggregation hierarchy of the
// operator (levels 0..L-1), FP32 workspace ws holding per level the arrays
// gr, gz, gd (conductance to Dirichlet nodes), diag, dinv, X, Y, B (each
// ni*nj floats), then the level-0 CG vectors p, q, x.
constexpr int kMgMaxLevels = 12;
constexpr int kMgArrays = 10;  // per level: 5 stencil / prolongation arrays, diag, dinv, X, Y, B
constexpr int kMgSmemFloats = 52 * 1024;  // at most 208 KB of shared memory for the local levels
constexpr int kMgDenseMax = 64;           // coarsest levels up to this many nodes are inverted
struct MgLevels {
  int L;
  int ni[kMgMaxLevels], nj[kMgMaxLevels];
  long long off[kMgMaxLevels];  // first float of level l's arrays in ws
  int local_from;               // levels >= local_from run within a block (block 0, or each block)
  int smem_from;                // levels >= smem_from live in shared memory (L: none)
  long long soff[kMgMaxLevels]; // their offsets (floats) in it
  int smem_floats;              // its size
  int redundant;                // 1: every block runs the local levels in its own shared memory
  float omega;                  // Jacobi damping
  float alpha;                  // coarse-correction scale below level 1
  float alpha0;                 // coarse-correction scale of level 1 into level 0
  float omega_s;                // prolongation smoothing of level 0
  int single_sweep;             // grid-wide levels below 0 smooth once before and after
  int rebuild_every;            // the coarse hierarchy is rebuilt every n-th solve (1: always)
  int *solves;                  // solves so far (device counter)
  float *persist;               // [smem_floats] the shared-memory part of the last build
  int coarse_sweeps;            // Jacobi sweeps on the coarsest level (when not dense)
  int cinv_off;                 // dense inverse of the coarsest operator in the block's
                                // shared memory at this offset (floats); -1: Jacobi
  float *ws;
  float *p, *p2, *q, *x, *r2;  // CG vectors (p and r alternate between two buffers)
};
// Levels and workspace size (floats) for an (nr+1) x (nz+1) node grid.
long long mg_plan(int nr, int nz, MgLevels *M);
cudaError_t launch_pcg_mg(const PcgParams &P, const MgLevels &M, int grid, cudaStream_t st);
// The same solve on one thread-block cluster (1, 2, 4, 8 CTAs; mg_cluster_size
// picks it from the node count): for many discharges solved at once.
int mg_cluster_size(int nn);
cudaError_t launch_pcg_mg_cluster(const PcgParams &P, const MgLevels &M, int cluster, cudaStream_t st);
cudaError_t launch_efield(const EfieldParams &E, cudaStream_t st);
cudaError_t launch_energy(int nr, int nz, const int8_t *node_kind, const double *Gr, const double *Gz,
                          const double *phi, double *out2, cudaStream_t st);
cudaError_t launch_circuit(const CircuitParams &C, cudaStream_t st);
cudaError_t launch_circuit_prepare(const CircuitParams &C, cudaStream_t st);
cudaError_t launch_diag(const DiagParams &D, cudaStream_t st);
cudaError_t launch_diag_window(const DiagParams &D, cudaStream_t st);

}  // namespace pic
