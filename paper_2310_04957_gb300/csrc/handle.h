// handle.h -- private definition of the library's handles (a discharge,
// a batch of discharges), shared by the translation units that implement the
// C ABI of include/pic.h.  Not part of the public interface.
#pragma once
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pic.h"
#include "learned.h"
#include "pic_device.cuh"
#include "pic_kernels.h"
#include "unet.h"

namespace pic {

// Device buffers of one particle store (one species, one of the two buffers).
struct Store {
  void *pa = nullptr, *pb = nullptr;  // Vec4 (fr, fz, vr, vt) and (vz, ar, at, az)
  unsigned long long *id = nullptr;
  void *w = nullptr;                  // weight ratios (weighted handles only)
  int *cell = nullptr, *start = nullptr, *cap = nullptr, *fill = nullptr;
  BinMeta *meta = nullptr;
};

}  // namespace pic

struct pic_handle {
  pic_config cfg{};
  std::vector<int8_t> node_kind, cell_kind;
  std::vector<double> cell_eps, xs_E, xs_S;
  int device = 0;
  cudaStream_t stream = nullptr;
  int nr = 0, nz = 0, nn = 0, nc = 0;
  int prec = PIC_FP32;
  size_t esz = 4;
  pic::BinMap map{};
  int nbins = 0, ntiles = 0;
  float slack = 0.25f;
  int64_t capacity[2] = {0, 0};
  bool weighted = false;  // particles carry weight ratios (cfg.weighted)
  bool vahedi = false;    // field composed by Eq. 2 (cfg.field_mode)
  double *d_phiP = nullptr;                            // phi_P, the zero-boundary part
  double *d_phiLd[3] = {nullptr, nullptr, nullptr};    // unit Laplace solutions of the driven electrodes
  // device: geometry, operator, fields
  int8_t *d_node_kind = nullptr, *d_cell_kind = nullptr, *d_bin_plasma = nullptr;
  double *d_Gvac_r = nullptr, *d_Gpl_r = nullptr, *d_Gvac_z = nullptr, *d_Gpl_z = nullptr, *d_vnode = nullptr;
  double *d_chi = nullptr, *d_zero = nullptr, *d_qrhs = nullptr, *d_phi = nullptr, *d_Gr = nullptr, *d_Gz = nullptr,
         *d_dinv = nullptr, *d_Er = nullptr, *d_Ez = nullptr;
  void *d_E = nullptr;
  // PCG scratch
  double *d_work = nullptr, *d_partial = nullptr, *d_pcg_out = nullptr;
  float *d_work32 = nullptr;
  unsigned *d_bar = nullptr;
  // C_eq solve
  double *d_phiL = nullptr, *d_Grc = nullptr, *d_Gzc = nullptr, *d_dinvc = nullptr, *d_energy = nullptr,
         *d_ceq_out = nullptr;
  double *d_scal_pack = nullptr;  // the PIC_NSCALARS scalars of pic_diag, packed on the device
  // particles, deposits, counters
  unsigned long long *d_dep[2] = {nullptr, nullptr}, *d_surf[2] = {nullptr, nullptr}, *d_counters = nullptr;
  pic::Store st[2][2];  // [buffer][species]
  int cur = 0;
  void *d_xsE = nullptr, *d_xsS = nullptr;
  float4 *d_xsG = nullptr;  // FP32 cross-section lookup groups (PushParams::xs_g)
  double *d_scalars = nullptr, *d_prop = nullptr;
  long long *d_lay_part = nullptr, *d_lay_boff = nullptr;
  int *d_lay_use = nullptr;
  uint32_t *d_step = nullptr, *d_flags = nullptr;
  double *d_dens_sum[2] = {nullptr, nullptr}, *d_dens_avg[2] = {nullptr, nullptr};
  // host mirrors
  uint32_t step = 0;
  double numax[2] = {0, 0}, pcoll[2] = {0, 0};
  int pcg_grid = 0;
  bool started = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graph_failed = false;
  bool timing = false;
  double timing_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> tev;  // 8 events per timed step
  std::vector<void *> allocs;
  // learned preconditioner (PIC_SOLVER_LEARNED)
  pic_unet *net = nullptr;
  cudaGraphExec_t fcg_exec = nullptr;
  cudaStream_t side = nullptr;
  pic::learned::FcgParams fcg{};
  int fcg_nblk = 0;
  double *d_phi_warm = nullptr, *d_lstats = nullptr, *d_pair_s2 = nullptr;
  bool keep_warm = false;
  int learned_finish = PIC_SOLVER_PLAIN;  // solver that confirms / finishes a learned solve
  pic::MgLevels mg{};                          // multigrid hierarchy of PIC_SOLVER_MG (workspace in mg.ws)
  std::vector<void *> lallocs;  // learned-solver buffers (freed on re-attach)
};

// A sweep of independent discharges stepped together (see pic_batch_create).
struct pic_batch {
  std::vector<pic_handle *> hs;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;  // recorded after each pic_batch_step; the handles' streams wait on it
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
};
