// capi.cu -- the C ABI declared in include/pic.h: handle life cycle, particle
// upload/download, the per-step CUDA graph, field solve, C_eq, diagnostics.
//
// Per step (arXiv:2310.04957, Sec. 2): particle phase (push + MCC + re-bin +
// deposit of rho~ and chi), circuit and electrode charge (Eqs. 5, 8-10),
// assembly and solve of the implicit field equation (Eq. 1), node E field,
// diagnostics.  The step is captured once per buffer parity as a CUDA graph.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "handle.h"

using namespace pic;

namespace {

const double kEps0 = 8.8541878128e-12;   // F/m
const double kQe = 1.602176634e-19;      // C
const double kKB = 1.380649e-23;         // J/K
const double kPi = 3.141592653589793238462643383279;

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      fprintf(stderr, "pic: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      return PIC_ECUDA;                            \
    }                                              \
  } while (0)

template <typename P>
int dalloc(pic_handle *h, P **ptr, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return PIC_ENOMEM;
  }
  if (cudaMemsetAsync(p, 0, bytes, h->stream) != cudaSuccess) return PIC_ECUDA;
  h->allocs.push_back(p);
  *ptr = reinterpret_cast<P *>(p);
  return PIC_OK;
}

#define DA(ptr, bytes)                    \
  do {                                    \
    int st_ = dalloc(h, &(ptr), (bytes)); \
    if (st_) return st_;                  \
  } while (0)

int nidx(const pic_handle *h, int i, int j) { return j * (h->nr + 1) + i; }

// Vacuum and plasma parts of the edge conductances and plasma node volumes,
// from the finite-volume control volumes of the axisymmetric grid: a radial
// face at r_{i+1/2} has area 2 pi r_{i+1/2} dz split half into each adjacent
// cell row; an axial face is the annulus [r_{i-1/2}, r_{i+1/2}] split at r_i
// between the two adjacent cell columns.  Each cell contributes
// eps0 eps_r,cell x (its face part) / (edge length) to the vacuum part and, if
// it is plasma, eps0 x (its face part) / (edge length) to the chi part.
void build_geometry(const pic_handle *h, std::vector<double> &Gvr, std::vector<double> &Gpr, std::vector<double> &Gvz,
                    std::vector<double> &Gpz, std::vector<double> &vnode) {
  const int nr = h->nr, nz = h->nz;
  const double dr = h->cfg.dr, dz = h->cfg.dz;
  Gvr.assign((size_t)(nz + 1) * nr, 0.0);
  Gpr.assign((size_t)(nz + 1) * nr, 0.0);
  Gvz.assign((size_t)nz * (nr + 1), 0.0);
  Gpz.assign((size_t)nz * (nr + 1), 0.0);
  vnode.assign((size_t)h->nn, 0.0);
  for (int j = 0; j < nz; ++j)
    for (int i = 0; i < nr; ++i) {
      int c = j * nr + i;
      double eps = h->cell_eps[c];
      bool pl = h->cell_kind[c] == PIC_CELL_PLASMA;
      double ri = i * dr, rh = (i + 0.5) * dr, ri1 = (i + 1) * dr;
      // radial edges at rows j and j+1, each gets the half face inside this cell
      double ar = 2.0 * kPi * rh * 0.5 * dz / dr;
      for (int jj = j; jj <= j + 1; ++jj) {
        Gvr[(size_t)jj * nr + i] += kEps0 * eps * ar;
        if (pl) Gpr[(size_t)jj * nr + i] += kEps0 * ar;
      }
      // axial edges at columns i (annulus [r_i, r_{i+1/2}]) and i+1 ([r_{i+1/2}, r_{i+1}])
      double azl = kPi * (rh * rh - ri * ri) / dz;
      double azr = kPi * (ri1 * ri1 - rh * rh) / dz;
      Gvz[(size_t)j * (nr + 1) + i] += kEps0 * eps * azl;
      Gvz[(size_t)j * (nr + 1) + i + 1] += kEps0 * eps * azr;
      if (pl) {
        Gpz[(size_t)j * (nr + 1) + i] += kEps0 * azl;
        Gpz[(size_t)j * (nr + 1) + i + 1] += kEps0 * azr;
        double q = 0.25 * kPi * (ri1 * ri1 - ri * ri) * dz;
        vnode[nidx(h, i, j)] += q;
        vnode[nidx(h, i + 1, j)] += q;
        vnode[nidx(h, i, j + 1)] += q;
        vnode[nidx(h, i + 1, j + 1)] += q;
      }
    }
}

// Null-collision bound per species: n_g x max over table intervals of the
// larger node sigma_T times the speed at the interval's upper energy.
void null_bounds(pic_handle *h) {
  const pic_config &c = h->cfg;
  int n = c.n_xs;
  for (int s = 0; s < 2; ++s) {
    double mass = s == 0 ? c.m[0] : c.m_gas;
    int p0 = s == 0 ? 0 : 3, p1 = s == 0 ? 3 : 5;
    double best = 0.0;
    for (int k = 0; k + 1 < n; ++k) {
      double sa = 0.0, sb = 0.0;
      for (int p = p0; p < p1; ++p) {
        sa += h->xs_S[(size_t)p * n + k];
        sb += h->xs_S[(size_t)p * n + k + 1];
      }
      double v = std::sqrt(2.0 * h->xs_E[k + 1] * kQe / mass);
      double nu = c.n_gas * (sa > sb ? sa : sb) * v;
      if (nu > best) best = nu;
    }
    h->numax[s] = best;
    h->pcoll[s] = 1.0 - std::exp(-best * c.dt);
  }
}

template <typename T>
StoreView<T> view(pic_handle *h, int buf, int s) {
  Store &S = h->st[buf][s];
  StoreView<T> v;
  v.pa = (Vec4<T> *)S.pa; v.pb = (Vec4<T> *)S.pb;
  v.id = S.id; v.w = (T *)S.w; v.cell = S.cell; v.start = S.start; v.cap = S.cap; v.fill = S.fill; v.meta = S.meta;
  v.capacity = (int)h->capacity[s];
  return v;
}

template <typename T>
PushParams<T> push_params(pic_handle *h, int in_buf) {
  const pic_config &c = h->cfg;
  PushParams<T> P;
  memset(&P, 0, sizeof(P));
  P.map = h->map;
  P.nr = h->nr; P.nz = h->nz;
  P.dt = (T)c.dt; P.hdt = (T)(0.5 * c.dt); P.hdt2 = (T)(0.5 * c.dt * c.dt);
  P.dr = (T)c.dr; P.dz = (T)c.dz; P.inv_dr = (T)(1.0 / c.dr); P.inv_dz = (T)(1.0 / c.dz);
  P.cell_kind = h->d_cell_kind; P.node_kind = h->d_node_kind;
  P.E = h->d_E;
  for (int s = 0; s < 2; ++s) {
    P.qm[s] = (T)(c.q[s] / c.m[s]);
    P.pcoll[s] = (T)h->pcoll[s];
    P.numax[s] = (T)h->numax[s];
    P.in[s] = view<T>(h, in_buf, s);
    P.out[s] = view<T>(h, in_buf ^ 1, s);
    P.dep[s] = h->d_dep[s];
    P.surf[s] = h->d_surf[s];
  }
  P.n_gas = (T)c.n_gas;
  P.xs_E = (const T *)h->d_xsE; P.xs_S = (const T *)h->d_xsS; P.n_xs = c.n_xs;
  P.xs_g = h->d_xsG;
  double l0 = std::log2(h->xs_E[0]), l1 = std::log2(h->xs_E[c.n_xs - 1]);
  P.log2E0 = (T)l0; P.inv_dlog2 = (T)((c.n_xs - 1) / (l1 - l0));
  P.thr_ex = (T)c.thr_ex; P.thr_iz = (T)c.thr_iz; P.B_ej = (T)c.B_ej;
  P.e_per_v2[0] = (T)(0.5 * c.m[0] / kQe);
  P.e_per_v2[1] = (T)(0.5 * c.m_gas / kQe);
  P.v2_per_e[0] = (T)(2.0 * kQe / c.m[0]);
  P.v2_per_e[1] = (T)(2.0 * kQe / c.m[1]);
  P.two_me_over_M = (T)(2.0 * c.m[0] / c.m_gas);
  P.vth_gas = (T)std::sqrt(kKB * c.T_gas / c.m_gas);
  P.mi_frac = (T)(c.m[1] / (c.m[1] + c.m_gas));
  P.seed = c.seed;
  P.step_ptr = h->d_step;
  P.counters = h->d_counters;
  P.dep_scale = (T)(h->prec == PIC_FP32 ? 67108864.0 : 1099511627776.0);
  P.dep_one = h->prec == PIC_FP32 ? (1ull << 26) : (1ull << 40);
  P.flags = h->d_flags;
  P.weighted = h->weighted ? 1 : 0;
  P.split_cells = c.split_cells;
  return P;
}

Drive drive_of(const pic_config &c) {
  Drive d;
  memset(&d, 0, sizeof(d));
  d.n = c.n_drive;
  for (int k = 0; k < c.n_drive && k < 3; ++k) {
    d.V[k] = c.drive_V[k];
    d.f[k] = c.drive_f[k];
    d.phase[k] = c.drive_phase[k];
  }
  return d;
}

// The array the field solve works on: phi itself, or phi_P in the Vahedi composition.
double *field_target(pic_handle *h) { return h->vahedi ? h->d_phiP : h->d_phi; }

double dep_inv_scale(const pic_handle *h) { return h->prec == PIC_FP32 ? 1.0 / 67108864.0 : 1.0 / 1099511627776.0; }

FieldParams field_params(pic_handle *h, const double *chi, double *Gr, double *Gz, double *dinv) {
  const pic_config &c = h->cfg;
  FieldParams F;
  memset(&F, 0, sizeof(F));
  F.nr = h->nr; F.nz = h->nz; F.nn = h->nn;
  F.node_kind = h->d_node_kind;
  F.Gvac_r = h->d_Gvac_r; F.Gpl_r = h->d_Gpl_r; F.Gvac_z = h->d_Gvac_z; F.Gpl_z = h->d_Gpl_z;
  F.vnode = h->d_vnode;
  for (int s = 0; s < 2; ++s) {
    F.dep[s] = h->d_dep[s];
    F.surf[s] = h->d_surf[s];
    F.qw[s] = c.q[s] * c.w[s];
    F.chi_coef[s] = c.dt * c.dt / (2.0 * kEps0) * c.q[s] * c.q[s] / c.m[s] * c.w[s];
  }
  F.dep_inv_scale = dep_inv_scale(h);
  F.surf_scale = h->weighted ? 1.0 / kCreditOne : 1.0;
  F.chi = const_cast<double *>(chi);
  F.qrhs = h->d_qrhs; F.phi = field_target(h); F.Gr = Gr; F.Gz = Gz; F.dinv = dinv;
  F.scalars = h->d_scalars;
  F.vahedi = h->vahedi ? 1 : 0;
  F.drive = drive_of(c);
  return F;
}

// Eq. 2 from the last solve's phi_P and the Laplace parts of the last refresh.
VahediParams vahedi_params(pic_handle *h) {
  VahediParams V;
  memset(&V, 0, sizeof(V));
  V.nn = h->nn;
  V.phiP = h->d_phiP;
  V.phiL[0] = h->d_phiL;
  for (int k = 0; k < 3; ++k) V.phiL[k + 1] = h->d_phiLd[k];
  V.phi = h->d_phi;
  V.scalars = h->d_scalars;
  V.drive = drive_of(h->cfg);
  return V;
}

PcgParams pcg_params(pic_handle *h, const double *Gr, const double *Gz, const double *dinv, const double *qrhs, double *phi,
                     double tol, double *out) {
  PcgParams P;
  memset(&P, 0, sizeof(P));
  P.nr = h->nr; P.nz = h->nz; P.nn = h->nn;
  P.node_kind = h->d_node_kind;
  P.Gr = Gr; P.Gz = Gz; P.dinv = dinv; P.qrhs = qrhs; P.phi = phi;
  P.work = h->d_work;
  P.work32 = h->d_work32;
  P.partial = h->d_partial;
  P.inner_tol = 1e-4f;
  P.gscale = 1.0 / (kEps0 * h->cfg.dr);
  P.bar = h->d_bar;
  P.tol = tol;
  P.maxit = h->cfg.pcg_maxit;
  P.out = out;
  P.flags = h->d_flags;
  P.spin_limit = h->cfg.spin_limit > 0 ? h->cfg.spin_limit : 4000000000ll;  // ~2 s at 2 GHz per barrier wait
  return P;
}

EfieldParams efield_params(pic_handle *h) {
  EfieldParams E;
  E.nr = h->nr; E.nz = h->nz; E.dr = h->cfg.dr; E.dz = h->cfg.dz;
  E.node_kind = h->d_node_kind; E.phi = h->d_phi; E.Er = h->d_Er; E.Ez = h->d_Ez;
  E.E32 = h->prec == PIC_FP32 ? (float2 *)h->d_E : nullptr;
  E.E64 = h->prec == PIC_FP64 ? (double2 *)h->d_E : nullptr;
  return E;
}

CircuitParams circuit_params(pic_handle *h, int n_run, double *U_hist, uint32_t *step_inc) {
  const pic_config &c = h->cfg;
  CircuitParams C;
  memset(&C, 0, sizeof(C));
  C.kind = c.circuit; C.nsub = c.n_sub;
  for (int k = 0; k < 8; ++k) C.c[k] = c.circ[k];
  C.V = c.V_src; C.f = c.f_src; C.phase = c.phase_src; C.dt = c.dt;
  C.qw[0] = c.q[0] * c.w[0]; C.qw[1] = c.q[1] * c.w[1];
  C.counters = h->d_counters;
  C.weighted = h->weighted ? 1 : 0;
  C.step_ptr = h->d_step;
  C.scalars = h->d_scalars;
  C.n_run = n_run; C.U_hist = U_hist; C.step_inc = step_inc;
  C.prop = h->d_prop;
  return C;
}

DiagParams diag_params(pic_handle *h) {
  const pic_config &c = h->cfg;
  DiagParams D;
  memset(&D, 0, sizeof(D));
  D.nn = h->nn; D.vnode = h->d_vnode;
  D.kind = c.circuit;
  for (int k = 0; k < 8; ++k) D.c[k] = c.circ[k];
  D.V = c.V_src; D.phase = c.phase_src;
  D.dep[0] = h->d_dep[0]; D.dep[1] = h->d_dep[1];
  D.dep_inv_scale = dep_inv_scale(h);
  D.w[0] = c.w[0]; D.w[1] = c.w[1];
  D.qw_ion = c.q[1] * c.w[1];
  D.f = c.f_src; D.dt = c.dt; D.window = c.steps_per_rf;
  D.counters = h->d_counters;
  D.weighted = h->weighted ? 1 : 0;
  D.step_ptr = h->d_step; D.step_mut = h->d_step;
  for (int s = 0; s < 2; ++s) { D.dens_sum[s] = h->d_dens_sum[s]; D.dens_avg[s] = h->d_dens_avg[s]; }
  D.scalars = h->d_scalars;
  return D;
}

LayoutParams layout_params(pic_handle *h, int in_buf) {
  LayoutParams L;
  memset(&L, 0, sizeof(L));
  int out = in_buf ^ 1;
  for (int s = 0; s < 2; ++s) {
    Store &A = h->st[in_buf][s], &B = h->st[out][s];
    L.fill_in[s] = A.fill;
    L.capacity[s] = (int)h->capacity[s];
    L.start[s] = B.start; L.cap[s] = B.cap; L.fill_out[s] = B.fill;
    L.meta_out[s] = B.meta; L.meta_in[s] = A.meta;
  }
  L.bin_plasma = h->d_bin_plasma;
  L.nbins = h->nbins;
  L.slack = h->slack;
  L.part = h->d_lay_part;
  L.boff = h->d_lay_boff;
  L.use_slack = h->d_lay_use;
  return L;
}

int launch_push(pic_handle *h, int in_buf) {
  cudaError_t e;
  if (h->prec == PIC_FP32) e = launch_particles<float>(push_params<float>(h, in_buf), h->stream);
  else e = launch_particles<double>(push_params<double>(h, in_buf), h->stream);
  return e == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

// Layout of the write buffer from the read buffer's fill counts, then zeroed
// deposits and counters, then the particle kernel.
int enqueue_particle_phase(pic_handle *h, int in_buf) {
  CK(launch_layout(layout_params(h, in_buf), h->stream));
  CK(cudaMemsetAsync(h->d_dep[0], 0, sizeof(unsigned long long) * h->nn, h->stream));
  CK(cudaMemsetAsync(h->d_dep[1], 0, sizeof(unsigned long long) * h->nn, h->stream));
  CK(cudaMemsetAsync(h->d_counters, 0, sizeof(unsigned long long) * CNT_N, h->stream));
  return launch_push(h, in_buf);
}

// The device step counter (the Philox counter's first word) set to the host's
// value, passed as a kernel argument: ordered on the stream like a copy, but
// with no pageable host buffer to stage (staging may make the host wait for the
// stream, which would idle the device between calls of pic_step).
__global__ void k_set_step(uint32_t *d_step, uint32_t v) { *d_step = v; }

// If the learned solve ended on a non-finite value, restart from the warm start.
__global__ void k_restore_warm(int nn, const int8_t *kind, const double *stats, const double *warm, double *phi) {
  if (stats[2] != -7.0) return;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nn; a += gridDim.x * blockDim.x)
    if (kind[a] == 0) phi[a] = warm[a];
}

int enqueue_solve(pic_handle *h, int mode) {
  if (h->keep_warm || mode == PIC_SOLVER_LEARNED)
    CK(cudaMemcpyAsync(h->d_phi_warm, field_target(h), sizeof(double) * h->nn, cudaMemcpyDeviceToDevice, h->stream));
  if (mode == PIC_SOLVER_LEARNED) {
    // flexible CG with the network; the plain PCG below then confirms the
    // residual in FP64 (zero iterations when it holds) or finishes the solve
    if (!h->fcg_exec) return PIC_EINVAL;
    CK(cudaGraphLaunch(h->fcg_exec, h->stream));
    k_restore_warm<<<h->fcg_nblk, 256, 0, h->stream>>>(h->nn, h->d_node_kind, h->d_lstats, h->d_phi_warm, h->d_phi);
    CK(cudaGetLastError());
  }
  CK(cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream));
  PcgParams P = pcg_params(h, h->d_Gr, h->d_Gz, h->d_dinv, h->d_qrhs, field_target(h), h->cfg.pcg_tol, h->d_pcg_out);
  const int finisher = mode == PIC_SOLVER_LEARNED ? h->learned_finish : mode;
  if (finisher == PIC_SOLVER_MIXED) CK(launch_pcg_mixed(P, h->pcg_grid, h->stream));
  else if (finisher == PIC_SOLVER_MG) CK(launch_pcg_mg(P, h->mg, h->pcg_grid, h->stream));
  else CK(launch_pcg(P, h->pcg_grid, h->stream));
  return PIC_OK;
}

// Parameters of the learned solve / training pairs (network grid nz x nr).
learned::FcgParams fcg_params(pic_handle *h) {
  learned::FcgParams F;
  memset(&F, 0, sizeof(F));
  F.nr = h->nr; F.nz = h->nz; F.nn = h->nn;
  F.H = h->nz; F.W = h->nr;
  int n = 0;
  for (int j = 0; j < h->nz; ++j)
    for (int i = 0; i < h->nr; ++i) n += h->node_kind[nidx(h, i, j)] == 0;
  F.n_cov = n;
  F.node_kind = h->d_node_kind;
  F.Gr = h->d_Gr; F.Gz = h->d_Gz; F.dinv = h->d_dinv; F.qrhs = h->d_qrhs; F.chi = h->d_chi;
  F.phi = h->d_phi;
  F.tol = h->cfg.pcg_tol;
  return F;
}

// Step before the field solve: layout, particle phase, circuit, assembly.
int enqueue_step_pre(pic_handle *h, int in_buf, cudaEvent_t *ev) {
  int st;
  if (ev) CK(cudaEventRecord(ev[0], h->stream));
  CK(launch_layout(layout_params(h, in_buf), h->stream));
  CK(cudaMemsetAsync(h->d_dep[0], 0, sizeof(unsigned long long) * h->nn, h->stream));
  CK(cudaMemsetAsync(h->d_dep[1], 0, sizeof(unsigned long long) * h->nn, h->stream));
  CK(cudaMemsetAsync(h->d_counters, 0, sizeof(unsigned long long) * CNT_N, h->stream));
  if (ev) CK(cudaEventRecord(ev[1], h->stream));
  if ((st = launch_push(h, in_buf))) return st;
  if (ev) CK(cudaEventRecord(ev[2], h->stream));
  CK(launch_circuit(circuit_params(h, 1, nullptr, nullptr), h->stream));
  if (ev) CK(cudaEventRecord(ev[3], h->stream));
  CK(launch_assemble(field_params(h, h->d_chi, h->d_Gr, h->d_Gz, h->d_dinv), h->stream));
  if (ev) CK(cudaEventRecord(ev[4], h->stream));
  return PIC_OK;
}

// Step after the field solve: node E field and diagnostics (advances the device step).
int enqueue_step_post(pic_handle *h, cudaEvent_t *ev) {
  if (h->vahedi) CK(launch_vahedi_combine(vahedi_params(h), h->stream));
  CK(launch_efield(efield_params(h), h->stream));
  if (ev) CK(cudaEventRecord(ev[6], h->stream));
  CK(launch_diag(diag_params(h), h->stream));
  if (ev) CK(cudaEventRecord(ev[7], h->stream));
  return PIC_OK;
}

int enqueue_step(pic_handle *h, int in_buf, cudaEvent_t *ev) {
  int st;
  if ((st = enqueue_step_pre(h, in_buf, ev))) return st;
  if ((st = enqueue_solve(h, h->cfg.solver))) return st;
  if (ev) CK(cudaEventRecord(ev[5], h->stream));
  return enqueue_step_post(h, ev);
}

// C_eq from the field energy of the unit-voltage solution (Eqs. 6-7), with
// or without chi; result in d_ceq_out[0] (energy route) and [1] (Gauss route).
int enqueue_ceq(pic_handle *h, bool with_chi) {
  FieldParams F = field_params(h, with_chi ? h->d_chi : h->d_zero, h->d_Grc, h->d_Gzc, h->d_dinvc);
  F.phi = h->d_phiL;
  // edges only (the node pass would overwrite rho~ and chi)
  CK(launch_assemble_edges_only(F, h->stream));
  CK(launch_set_dirichlet(h->nn, h->d_node_kind, h->d_phiL, 1.0, h->stream));
  CK(cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream));
  double tol = h->cfg.pcg_tol < 1e-12 ? h->cfg.pcg_tol : 1e-12;
  PcgParams P = pcg_params(h, h->d_Grc, h->d_Gzc, h->d_dinvc, h->d_zero, h->d_phiL, tol, h->d_pcg_out + 4);
  CK(launch_pcg(P, h->pcg_grid, h->stream));
  CK(launch_energy(h->nr, h->nz, h->d_node_kind, h->d_Grc, h->d_Gzc, h->d_phiL, h->d_ceq_out, h->stream));
  return PIC_OK;
}

// Unit Laplace solutions of the driven electrodes (Eq. 4) on the operator the
// last enqueue_ceq built (vacuum or with chi), each from its previous solution,
// to the C_eq solve's tolerance.  The powered electrode's is that C_eq solve's.
int enqueue_laplace(pic_handle *h) {
  double tol = h->cfg.pcg_tol < 1e-12 ? h->cfg.pcg_tol : 1e-12;
  for (int k = 0; k < h->cfg.n_drive; ++k) {
    CK(launch_set_dirichlet_unit(h->nn, h->d_node_kind, h->d_phiLd[k], PIC_NODE_DRIVEN + k, h->stream));
    CK(cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream));
    PcgParams P = pcg_params(h, h->d_Grc, h->d_Gzc, h->d_dinvc, h->d_zero, h->d_phiLd[k], tol, h->d_pcg_out + 4);
    CK(launch_pcg(P, h->pcg_grid, h->stream));
  }
  return PIC_OK;
}

int sync(pic_handle *h) {
  CK(cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

void free_learned(pic_handle *h) {
  if (h->fcg_exec) cudaGraphExecDestroy(h->fcg_exec);
  h->fcg_exec = nullptr;
  for (void *p : h->lallocs) cudaFree(p);
  h->lallocs.clear();
  h->net = nullptr;
}

void free_all(pic_handle *h) {
  free_learned(h);
  if (h->side) cudaStreamDestroy(h->side);
  h->side = nullptr;
  for (int k = 0; k < 2; ++k)
    if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
  for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
  h->tev.clear();
  for (void *p : h->allocs) cudaFree(p);
  h->allocs.clear();
}

int capture_graph(pic_handle *h, int buf) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return PIC_ECUDA;
  }
  int st = enqueue_step(h, buf, nullptr);
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (st || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return PIC_ECUDA;
  }
  e = cudaGraphInstantiate(&h->graph[buf], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->graph[buf] = nullptr;
    return PIC_ECUDA;
  }
  return PIC_OK;
}

int window_end(pic_handle *h) {
  CK(launch_diag_window(diag_params(h), h->stream));
  if (h->cfg.ceq_refresh) {
    int st = enqueue_ceq(h, true);
    if (st) return st;
    CK(cudaMemcpyAsync(h->d_scalars + SC_CEQ, h->d_ceq_out, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(h->d_scalars + SC_CEQ_GAUSS, h->d_ceq_out + 1, sizeof(double), cudaMemcpyDeviceToDevice,
                       h->stream));
    CK(launch_circuit_prepare(circuit_params(h, 1, nullptr, nullptr), h->stream));
    if (h->vahedi && (st = enqueue_laplace(h))) return st;
  }
  return PIC_OK;
}

bool check_config(const pic_config *c) {
  if (!c || c->nr < 2 || c->nz < 2 || !(c->dr > 0) || !(c->dz > 0) || !(c->dt > 0)) return false;
  if (!c->node_kind || !c->cell_kind || !c->cell_eps || !c->xs_energy || !c->xs_sigma || c->n_xs < 2) return false;
  if (c->circuit < 0 || c->circuit > 2 || c->n_sub < 1 || c->steps_per_rf < 1 || c->pcg_maxit < 1) return false;
  if (c->precision != PIC_FP32 && c->precision != PIC_FP64) return false;
  if (c->solver != PIC_SOLVER_PLAIN && c->solver != PIC_SOLVER_MIXED && c->solver != PIC_SOLVER_LEARNED &&
      c->solver != PIC_SOLVER_MG)
    return false;
  if (c->capacity[0] < 1 || c->capacity[1] < 1 || c->capacity[0] > 2000000000ll || c->capacity[1] > 2000000000ll)
    return false;
  if (c->spin_limit < 0) return false;
  if (c->weighted != 0 && c->weighted != 1) return false;
  if (c->split_cells < 0 || c->split_cells > c->nr || (c->split_cells > 0 && !c->weighted)) return false;
  if (c->n_drive < 0 || c->n_drive > 3) return false;
  for (int k = 0; k < c->n_drive; ++k)
    if (!std::isfinite(c->drive_V[k]) || !std::isfinite(c->drive_f[k]) || !std::isfinite(c->drive_phase[k]))
      return false;
  if (c->field_mode != PIC_FIELD_DIRECT && c->field_mode != PIC_FIELD_VAHEDI) return false;
  if (c->field_mode == PIC_FIELD_VAHEDI && c->solver == PIC_SOLVER_LEARNED) return false;
  if (!(c->m[0] > 0) || !(c->m[1] > 0) || !(c->m_gas > 0)) return false;
  for (int k = 0; k + 1 < c->n_xs; ++k)
    if (!(c->xs_energy[k + 1] > c->xs_energy[k]) || !(c->xs_energy[k] > 0)) return false;
  int tr = c->tile_r > 0 ? c->tile_r : 4, tz = c->tile_z > 0 ? c->tile_z : 4;
  if (!tile_supported(tr, tz)) return false;
  if (c->circuit == PIC_CIRCUIT_RLC && !(c->circ[0] >= 0 && c->circ[1] > 0 && c->circ[2] > 0)) return false;
  if (c->circuit == PIC_CIRCUIT_IMN)
    for (int k = 0; k < 8; ++k)
      if (!(c->circ[k] > 0)) return false;
  return true;
}

// Upload of one species: the raw FP64 columns go to the device as they are,
// and the device bins them (cell, rank within the bin, scatter into the
// store); the host only scans the bins' counts.
template <typename T>
int upload_species(pic_handle *h, int s, int64_t n, const pic_particles *p) {
  const pic_config &c = h->cfg;
  Store &S = h->st[h->cur][s];
  const int nb = h->nbins;
  std::vector<int> start(nb, 0), fill(nb, 0);
  if (n > 0) {
    struct DevTmp {  // freed on every return
      void *p = nullptr;
      ~DevTmp() { if (p) cudaFree(p); }
    } raw, work, bins;
    const size_t m = (size_t)n;
    const bool has_w = h->weighted && p->w;
    CK(cudaMalloc(&raw.p, (has_w ? 10 : 9) * sizeof(double) * m));
    CK(cudaMalloc(&work.p, (sizeof(int2) + 2 * sizeof(T)) * m));
    CK(cudaMalloc(&bins.p, sizeof(int) * (2 * (size_t)nb + 1)));
    double *d_raw = static_cast<double *>(raw.p);
    const double *cols[8] = {p->r, p->z, p->vr, p->vt, p->vz, p->ar, p->at, p->az};
    for (int k = 0; k < 8; ++k)
      CK(cudaMemcpyAsync(d_raw + k * m, cols[k], sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
    auto *d_id = reinterpret_cast<unsigned long long *>(d_raw + 8 * m);
    CK(cudaMemcpyAsync(d_id, p->id, sizeof(unsigned long long) * m, cudaMemcpyHostToDevice, h->stream));
    if (has_w) CK(cudaMemcpyAsync(d_raw + 9 * m, p->w, sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
    int *d_count = static_cast<int *>(bins.p), *d_start = d_count + nb;
    unsigned *d_err = reinterpret_cast<unsigned *>(d_start + nb);
    CK(cudaMemsetAsync(d_count, 0, sizeof(int) * ((size_t)nb + 0), h->stream));
    CK(cudaMemsetAsync(d_err, 0, sizeof(unsigned), h->stream));
    UploadParams<T> U;
    U.n = n;
    U.r = d_raw; U.z = d_raw + m; U.vr = d_raw + 2 * m; U.vt = d_raw + 3 * m; U.vz = d_raw + 4 * m;
    U.ar = d_raw + 5 * m; U.at = d_raw + 6 * m; U.az = d_raw + 7 * m;
    U.id = d_id;
    U.w = has_w ? d_raw + 9 * m : nullptr;
    U.dr = c.dr; U.dz = c.dz;
    U.map = h->map;
    U.cell_kind = h->d_cell_kind;
    U.count = d_count;
    U.start = d_start;
    U.bin_rank = static_cast<int2 *>(work.p);
    U.fr_tmp = reinterpret_cast<T *>(U.bin_rank + m);
    U.fz_tmp = U.fr_tmp + m;
    U.err = d_err;
    U.out = view<T>(h, h->cur, s);
    CK(launch_upload_bin<T>(U, h->stream));
    unsigned err = 0;
    CK(cudaMemcpyAsync(fill.data(), d_count, sizeof(int) * nb, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&err, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    if (sync(h)) return PIC_ECUDA;
    if (err) return PIC_EINVAL;  // a particle outside the plasma or a bad ratio: the store is untouched
    int run = 0;
    for (int b = 0; b < nb; ++b) { start[b] = run; run += fill[b]; }
    CK(cudaMemcpyAsync(d_start, start.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, h->stream));
    CK(launch_upload_scatter<T>(U, h->stream));
    if (sync(h)) return PIC_ECUDA;
  }
  CK(cudaMemcpy(S.start, start.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(S.cap, fill.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(S.fill, fill.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
  BinMeta meta{(int)n, 0, (long long)n};
  CK(cudaMemcpy(S.meta, &meta, sizeof(BinMeta), cudaMemcpyHostToDevice));
  return PIC_OK;
}

template <typename T>
int download_species(pic_handle *h, int s, pic_particles *out, int64_t capn, int64_t *nout) {
  Store &S = h->st[h->cur][s];
  std::vector<int> start(h->nbins), cap(h->nbins), fill(h->nbins);
  BinMeta m;
  CK(cudaMemcpy(start.data(), S.start, sizeof(int) * h->nbins, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(cap.data(), S.cap, sizeof(int) * h->nbins, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(fill.data(), S.fill, sizeof(int) * h->nbins, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&m, S.meta, sizeof(BinMeta), cudaMemcpyDeviceToHost));
  int64_t total = 0;
  for (int b = 0; b < h->nbins; ++b) total += fill[b] < cap[b] ? fill[b] : cap[b];
  int novf = m.ovf_n;
  if (novf > h->capacity[s] - m.ovf_base) novf = (int)(h->capacity[s] - m.ovf_base);
  if (novf < 0) novf = 0;
  total += novf;
  *nout = total;
  if (!out) return PIC_OK;
  if (total > capn) return PIC_EINVAL;
  size_t used = (size_t)m.ovf_base + novf;
  if (used == 0) return PIC_OK;
  std::vector<Vec4<T>> va(used), vb(used);
  std::vector<unsigned long long> id(used);
  std::vector<int> cell(used);
  std::vector<T> wr(h->weighted ? used : 0);
  if (h->weighted) CK(cudaMemcpy(wr.data(), S.w, sizeof(T) * used, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(va.data(), S.pa, sizeof(Vec4<T>) * used, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(vb.data(), S.pb, sizeof(Vec4<T>) * used, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(id.data(), S.id, sizeof(unsigned long long) * used, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(cell.data(), S.cell, sizeof(int) * used, cudaMemcpyDeviceToHost));
  const double dr = h->cfg.dr, dz = h->cfg.dz;
  int64_t k = 0;
  auto put = [&](size_t slot, int i, int j) {
    const Vec4<T> &a = va[slot], &b = vb[slot];
    out->r[k] = ((double)i + (double)a.x) * dr;
    out->z[k] = ((double)j + (double)a.y) * dz;
    out->vr[k] = a.z; out->vt[k] = a.w; out->vz[k] = b.x;
    out->ar[k] = b.y; out->at[k] = b.z; out->az[k] = b.w;
    out->id[k] = id[slot];
    if (out->cell) out->cell[k] = j * h->nr + i;
    if (out->w) out->w[k] = h->weighted ? (double)wr[slot] : 1.0;
    ++k;
  };
  for (int b = 0; b < h->nbins; ++b) {
    int nb = fill[b] < cap[b] ? fill[b] : cap[b];
    if (!nb) continue;
    int i, j;
    h->map.cell(b, i, j);
    for (int q = 0; q < nb; ++q) put((size_t)start[b] + q, i, j);
  }
  for (int q = 0; q < novf; ++q) {
    size_t slot = (size_t)m.ovf_base + q;
    int c = cell[slot];
    put(slot, c % h->nr, c / h->nr);
  }
  return PIC_OK;
}

// ---- batched sweep -----------------------------------------------------------------
void batch_free(pic_batch *b) {
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
  if (b->done) cudaEventDestroy(b->done);
  if (b->stream) cudaStreamDestroy(b->stream);
}

// Captures what `enqueue` puts on handle h's stream into a child graph node of G.
template <class F>
cudaError_t add_child(cudaGraph_t G, pic_handle *h, cudaStream_t cap, const cudaGraphNode_t *deps, size_t nd,
                             cudaGraphNode_t *node, F enqueue) {
  cudaStream_t keep = h->stream;
  h->stream = cap;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { h->stream = keep; return e; }
  const int st = enqueue(h);
  e = cudaStreamEndCapture(cap, &g);
  h->stream = keep;
  if (st != PIC_OK && e == cudaSuccess) e = cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(node, G, deps, nd, g);
  if (g) cudaGraphDestroy(g);
  return e;
}

// One step of every discharge: per discharge the chain [layout, particles,
// circuit, assembly] -> [multigrid field solve on one thread-block cluster] ->
// [E field, diagnostics]; the chains are independent branches of one graph, so
// one discharge's solve overlaps another's particle phase.
cudaError_t batch_build(pic_batch *b, int parity) {
  cudaGraph_t G = nullptr;
  cudaError_t e = cudaGraphCreate(&G, 0);
  if (e != cudaSuccess) return e;
  const size_t n = b->hs.size();
  std::vector<cudaGraphNode_t> pre(n), solve(n), post(n);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    e = add_child(G, b->hs[i], b->stream, nullptr, 0, &pre[i],
                  [&](pic_handle *h) { return enqueue_step_pre(h, parity, nullptr); });
    if (e != cudaSuccess) break;
    e = add_child(G, b->hs[i], b->stream, &pre[i], 1, &solve[i], [&](pic_handle *h) {
      const PcgParams P =
          pcg_params(h, h->d_Gr, h->d_Gz, h->d_dinv, h->d_qrhs, field_target(h), h->cfg.pcg_tol, h->d_pcg_out);
      return launch_pcg_mg_cluster(P, h->mg, mg_cluster_size(h->nn), h->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
    });
    if (e != cudaSuccess) break;
    e = add_child(G, b->hs[i], b->stream, &solve[i], 1, &post[i],
                  [&](pic_handle *h) { return enqueue_step_post(h, nullptr); });
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[parity], G, 0);
  cudaGraphDestroy(G);
  if (e != cudaSuccess) {
    b->graph[parity] = nullptr;
    cudaGetLastError();
  }
  return e;
}

// The PIC_NSCALARS scalars of pic_diag(PIC_DIAG_SCALARS), assembled by one
// thread from the device scalars, the last solve's result and the step's
// counters, with the host-side values (step, nu_max, collision probabilities,
// q w per species) passed in.  Both the synchronous and the enqueued read use
// it, so their values agree bit for bit.
struct ScalarPack {
  const double *sc, *pcg;
  const unsigned long long *cnt;
  double step, t, numax[2], pcoll[2], qw[2];
  int weighted;
  double *out;
};

__global__ void k_pack_scalars(const ScalarPack K) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double *sc = K.sc;
  const unsigned long long *cnt = K.cnt;
  double *o = K.out;
  o[0] = K.step; o[1] = K.t; o[2] = sc[SC_UE]; o[3] = sc[SC_QE]; o[4] = sc[SC_CEQ];
  o[5] = sc[SC_ICONV]; o[6] = sc[SC_ICCP];
  for (int k = 0; k < 6; ++k) o[7 + k] = sc[SC_Y0 + k];
  o[13] = K.pcg[0]; o[14] = K.pcg[1];
  o[15] = K.numax[0]; o[16] = K.numax[1]; o[17] = K.pcoll[0]; o[18] = K.pcoll[1];
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 3; ++k) {
      o[19 + 3 * s + k] = K.qw[s] * (K.weighted ? (double)cnt[CNT_ABSW + 3 * s + k] / kCreditOne
                                                : (double)cnt[CNT_ABS + 3 * s + k]);
      o[25 + 3 * s + k] = (double)cnt[CNT_ABS + 3 * s + k];
      o[31 + 3 * s + k] = (double)cnt[CNT_COLL + 3 * s + k];
    }
  o[36] = 0.0;
  o[37] = (double)cnt[CNT_BORN + 0]; o[38] = (double)cnt[CNT_BORN + 1];
  for (int k = 0; k < 3; ++k) o[39 + k] = sc[SC_IONCUR + k];
  o[42] = sc[SC_I1_RE]; o[43] = sc[SC_I1_IM]; o[44] = sc[SC_WINDOWS]; o[45] = sc[SC_CEQ_GAUSS];
  o[46] = K.pcg[2];
  o[47] = (double)cnt[CNT_SPLIT + 0]; o[48] = (double)cnt[CNT_SPLIT + 1];
}

// Enqueue the scalars' assembly and (host_buf not NULL) their copy into host_buf on
// the handle's stream.
int enqueue_scalars(pic_handle *h, double *host_buf) {
  const pic_config &c = h->cfg;
  ScalarPack K;
  K.sc = h->d_scalars;
  K.pcg = h->d_pcg_out;
  K.cnt = h->d_counters;
  K.step = h->step;
  K.t = h->step * c.dt;
  for (int s = 0; s < 2; ++s) {
    K.numax[s] = h->numax[s];
    K.pcoll[s] = h->pcoll[s];
    K.qw[s] = c.q[s] * c.w[s];
  }
  K.weighted = h->weighted ? 1 : 0;
  K.out = h->d_scal_pack;
  k_pack_scalars<<<1, 32, 0, h->stream>>>(K);
  CK(cudaGetLastError());
  if (host_buf)
    CK(cudaMemcpyAsync(host_buf, h->d_scal_pack, sizeof(double) * PIC_NSCALARS, cudaMemcpyDeviceToHost, h->stream));
  return PIC_OK;
}

// Fixed-point node counts to doubles on the device, with the host path's
// arithmetic and rounding: out = sa * (double)a (deposits), or
// qa * (a * us) + qb * (b * us) (surface charge of both species).  No fused
// multiply-add, so the values equal pic_diag's host conversion bit for bit.
__global__ void k_counts_to_f64(int n, const unsigned long long *a, const unsigned long long *b, double sa,
                                double qa, double qb, double us, double *out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    if (b == nullptr) {
      out[k] = __dmul_rn((double)a[k], sa);
    } else {
      out[k] = __dadd_rn(__dmul_rn(qa, __dmul_rn((double)a[k], us)), __dmul_rn(qb, __dmul_rn((double)b[k], us)));
    }
  }
}

// Enqueue the conversion of PIC_DIAG_DEP_E, _DEP_I or _SIGMA into dst (device).
int enqueue_counts(pic_handle *h, int what, double *dst) {
  if (what == PIC_DIAG_SIGMA) {
    const pic_config &c = h->cfg;
    k_counts_to_f64<<<256, 256, 0, h->stream>>>(h->nn, h->d_surf[0], h->d_surf[1], 0.0, c.q[0] * c.w[0],
                                               c.q[1] * c.w[1], h->weighted ? 1.0 / kCreditOne : 1.0, dst);
  } else {
    k_counts_to_f64<<<256, 256, 0, h->stream>>>(h->nn, h->d_dep[what - PIC_DIAG_DEP_E], nullptr, dep_inv_scale(h),
                                               0.0, 0.0, 0.0, dst);
  }
  CK(cudaGetLastError());
  return PIC_OK;
}

// pic_diag into a device buffer: enqueued on the handle's stream, no host wait.
int diag_to_device(pic_handle *h, int what, double *dst, size_t bytes) {
  const size_t nb = sizeof(double) * h->nn;
  if (what == PIC_DIAG_SCALARS) {
    if (bytes < sizeof(double) * PIC_NSCALARS) return PIC_EINVAL;
    int st = enqueue_scalars(h, nullptr);
    if (st) return st;
    CK(cudaMemcpyAsync(dst, h->d_scal_pack, sizeof(double) * PIC_NSCALARS, cudaMemcpyDeviceToDevice, h->stream));
    return PIC_OK;
  }
  if (bytes < nb) return PIC_EINVAL;
  const double *src = nullptr;
  switch (what) {
    case PIC_DIAG_PHI: src = h->d_phi; break;
    case PIC_DIAG_ER: src = h->d_Er; break;
    case PIC_DIAG_EZ: src = h->d_Ez; break;
    case PIC_DIAG_CHI: src = h->d_chi; break;
    case PIC_DIAG_VNODE: src = h->d_vnode; break;
    case PIC_DIAG_RHO: src = h->d_qrhs; break;
    case PIC_DIAG_NE_AVG: src = h->d_dens_avg[0]; break;
    case PIC_DIAG_NI_AVG: src = h->d_dens_avg[1]; break;
    case PIC_DIAG_PHI_WARM: src = h->d_phi_warm; break;
    case PIC_DIAG_PHI_P: src = h->vahedi ? h->d_phiP : nullptr; break;
    case PIC_DIAG_PHI_L0: src = h->vahedi ? h->d_phiL : nullptr; break;
    case PIC_DIAG_PHI_L0 + 1:
    case PIC_DIAG_PHI_L0 + 2:
    case PIC_DIAG_PHI_L0 + 3: {
      const int k = what - PIC_DIAG_PHI_L0 - 1;
      src = (h->vahedi && k < h->cfg.n_drive) ? h->d_phiLd[k] : nullptr;
      break;
    }
    case PIC_DIAG_DEP_E:
    case PIC_DIAG_DEP_I:
    case PIC_DIAG_SIGMA: return enqueue_counts(h, what, dst);
    default: return PIC_EINVAL;
  }
  if (src == nullptr) return PIC_EINVAL;
  CK(cudaMemcpyAsync(dst, src, nb, cudaMemcpyDeviceToDevice, h->stream));
  return PIC_OK;
}

}  // namespace

// =============================================================================
extern "C" {

const char *pic_strerror(int code) {
  switch (code) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument or configuration";
    case PIC_ENOMEM: return "out of memory";
    case PIC_ECUDA: return "CUDA runtime error";
    case PIC_ENOCONV: return "field solve did not converge within its iteration cap";
    case PIC_ETIMEOUT: return "a bounded device-side wait timed out";
    case PIC_EOVERFLOW: return "particle store overflow";
    case PIC_ENAN: return "non-finite value in the field solve";
    case PIC_EIO: return "restart file could not be written or read, or is not a restart file";
    default: return "unknown error";
  }
}

void pic_destroy(pic_handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

int pic_init(const pic_config *cfg, void *cuda_stream, pic_handle **out) {
  if (!out || !check_config(cfg)) return PIC_EINVAL;
  *out = nullptr;
  pic_handle *h = new (std::nothrow) pic_handle();
  if (!h) return PIC_ENOMEM;
  h->cfg = *cfg;
  h->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return PIC_ECUDA; }
  h->nr = cfg->nr; h->nz = cfg->nz;
  h->nn = (h->nr + 1) * (h->nz + 1);
  h->nc = h->nr * h->nz;
  h->prec = cfg->precision;
  h->esz = h->prec == PIC_FP32 ? 4 : 8;
  h->node_kind.assign(cfg->node_kind, cfg->node_kind + h->nn);
  h->cell_kind.assign(cfg->cell_kind, cfg->cell_kind + h->nc);
  h->cell_eps.assign(cfg->cell_eps, cfg->cell_eps + h->nc);
  h->xs_E.assign(cfg->xs_energy, cfg->xs_energy + cfg->n_xs);
  h->xs_S.assign(cfg->xs_sigma, cfg->xs_sigma + 5 * (size_t)cfg->n_xs);
  for (int a = 0; a < h->nn; ++a)
    if (h->node_kind[a] < 0 || h->node_kind[a] > 2 + cfg->n_drive) { delete h; return PIC_EINVAL; }
  for (int c = 0; c < h->nc; ++c)
    if (h->cell_kind[c] < 0 || h->cell_kind[c] > 3 || !(h->cell_eps[c] > 0)) { delete h; return PIC_EINVAL; }
  h->cfg.node_kind = h->node_kind.data();
  h->cfg.cell_kind = h->cell_kind.data();
  h->cfg.cell_eps = h->cell_eps.data();
  h->cfg.xs_energy = h->xs_E.data();
  h->cfg.xs_sigma = h->xs_S.data();
  h->slack = cfg->bin_slack > 0 ? (float)cfg->bin_slack : 0.25f;
  h->capacity[0] = cfg->capacity[0];
  h->capacity[1] = cfg->capacity[1];
  h->weighted = cfg->weighted != 0;
  h->vahedi = cfg->field_mode == PIC_FIELD_VAHEDI;
  int TX = cfg->tile_r > 0 ? cfg->tile_r : 4, TY = cfg->tile_z > 0 ? cfg->tile_z : 4;
  h->map.nr = h->nr; h->map.nz = h->nz; h->map.TX = TX; h->map.TY = TY;
  h->map.ntx = (h->nr + TX - 1) / TX; h->map.nty = (h->nz + TY - 1) / TY;
  h->nbins = h->map.nbins();
  h->ntiles = h->map.ntiles();
  null_bounds(h);
  int st = [&]() -> int {
    const size_t nn = h->nn;
    DA(h->d_node_kind, nn);
    DA(h->d_cell_kind, h->nc);
    DA(h->d_bin_plasma, h->nbins);
    DA(h->d_Gvac_r, sizeof(double) * (h->nz + 1) * h->nr);
    DA(h->d_Gpl_r, sizeof(double) * (h->nz + 1) * h->nr);
    DA(h->d_Gvac_z, sizeof(double) * h->nz * (h->nr + 1));
    DA(h->d_Gpl_z, sizeof(double) * h->nz * (h->nr + 1));
    DA(h->d_Gr, sizeof(double) * (h->nz + 1) * h->nr);
    DA(h->d_Gz, sizeof(double) * h->nz * (h->nr + 1));
    DA(h->d_Grc, sizeof(double) * (h->nz + 1) * h->nr);
    DA(h->d_Gzc, sizeof(double) * h->nz * (h->nr + 1));
    DA(h->d_vnode, sizeof(double) * nn);
    DA(h->d_chi, sizeof(double) * nn);
    DA(h->d_zero, sizeof(double) * nn);
    DA(h->d_qrhs, sizeof(double) * nn);
    DA(h->d_phi, sizeof(double) * nn);
    DA(h->d_phiL, sizeof(double) * nn);
    DA(h->d_dinv, sizeof(double) * nn);
    DA(h->d_dinvc, sizeof(double) * nn);
    DA(h->d_Er, sizeof(double) * nn);
    DA(h->d_Ez, sizeof(double) * nn);
    DA(h->d_E, 2 * h->esz * nn);
    DA(h->d_work, sizeof(double) * 8 * nn);
    DA(h->d_work32, sizeof(float) * 12 * nn);
    {
      const long long mgf = mg_plan(h->nr, h->nz, &h->mg);
      DA(h->mg.ws, sizeof(float) * (size_t)mgf);
      const long long lv = mgf - 5LL * (long long)nn;
      h->mg.p = h->mg.ws + lv;
      h->mg.p2 = h->mg.p + nn;
      h->mg.q = h->mg.p2 + nn;
      h->mg.x = h->mg.q + nn;
      h->mg.r2 = h->mg.x + nn;
      DA(h->mg.persist, sizeof(float) * (size_t)(h->mg.smem_floats > 0 ? h->mg.smem_floats : 1));
      DA(h->mg.solves, sizeof(int));
    }
    h->pcg_grid = pcg_grid_size(h->device);
    DA(h->d_partial, sizeof(double) * 16 * (h->pcg_grid + 32));
    DA(h->d_bar, 4 * sizeof(unsigned));
    DA(h->d_pcg_out, sizeof(double) * 8);
    DA(h->d_phi_warm, sizeof(double) * nn);
    if (h->vahedi) {
      DA(h->d_phiP, sizeof(double) * nn);
      for (int k = 0; k < cfg->n_drive; ++k) DA(h->d_phiLd[k], sizeof(double) * nn);
    }
    DA(h->d_lstats, sizeof(double) * 4);
    DA(h->d_pair_s2, sizeof(double) * 2);
    DA(h->d_energy, sizeof(double) * 2);
    DA(h->d_ceq_out, sizeof(double) * 2);
    DA(h->d_counters, sizeof(unsigned long long) * CNT_N);
    DA(h->d_scalars, sizeof(double) * SC_N);
    DA(h->d_scal_pack, sizeof(double) * PIC_NSCALARS);
    DA(h->d_prop, sizeof(double) * 64);
    {
      int nblk = (h->nbins + 1023) / 1024;
      if (nblk > 1024) return PIC_EINVAL;
      DA(h->d_lay_part, sizeof(long long) * 2 * 4 * nblk);
      DA(h->d_lay_boff, sizeof(long long) * 2 * nblk);
      DA(h->d_lay_use, sizeof(int) * 2);
    }
    DA(h->d_step, sizeof(uint32_t) * 2);
    DA(h->d_flags, sizeof(uint32_t) * 2);
    DA(h->d_xsE, h->esz * cfg->n_xs);
    DA(h->d_xsS, h->esz * 5 * cfg->n_xs);
    DA(h->d_xsG, sizeof(float4) * 3 * (cfg->n_xs - 1));
    for (int s = 0; s < 2; ++s) {
      DA(h->d_dep[s], sizeof(unsigned long long) * nn);
      DA(h->d_surf[s], sizeof(unsigned long long) * nn);
      DA(h->d_dens_sum[s], sizeof(double) * nn);
      DA(h->d_dens_avg[s], sizeof(double) * nn);
      for (int b = 0; b < 2; ++b) {
        Store &S = h->st[b][s];
        size_t cap = (size_t)h->capacity[s];
        DA(S.pa, 4 * h->esz * cap);
        DA(S.pb, 4 * h->esz * cap);
        DA(S.id, sizeof(unsigned long long) * cap);
        if (h->weighted) DA(S.w, h->esz * cap);
        DA(S.cell, sizeof(int) * cap);
        DA(S.start, sizeof(int) * h->nbins);
        DA(S.cap, sizeof(int) * h->nbins);
        DA(S.fill, sizeof(int) * h->nbins);
        DA(S.meta, sizeof(BinMeta));
      }
    }
    // geometry
    std::vector<double> Gvr, Gpr, Gvz, Gpz, vnode;
    build_geometry(h, Gvr, Gpr, Gvz, Gpz, vnode);
    CK(cudaMemcpy(h->d_node_kind, h->node_kind.data(), nn, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_cell_kind, h->cell_kind.data(), h->nc, cudaMemcpyHostToDevice));
    std::vector<int8_t> bp(h->nbins, 0);
    for (int b = 0; b < h->nbins; ++b) {
      int i, j;
      h->map.cell(b, i, j);
      if (i < h->nr && j < h->nz) bp[b] = h->cell_kind[(size_t)j * h->nr + i] == PIC_CELL_PLASMA;
    }
    CK(cudaMemcpy(h->d_bin_plasma, bp.data(), h->nbins, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_Gvac_r, Gvr.data(), sizeof(double) * Gvr.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_Gpl_r, Gpr.data(), sizeof(double) * Gpr.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_Gvac_z, Gvz.data(), sizeof(double) * Gvz.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_Gpl_z, Gpz.data(), sizeof(double) * Gpz.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_vnode, vnode.data(), sizeof(double) * nn, cudaMemcpyHostToDevice));
    if (h->prec == PIC_FP32) {
      std::vector<float> e(h->xs_E.begin(), h->xs_E.end()), s(h->xs_S.begin(), h->xs_S.end());
      CK(cudaMemcpy(h->d_xsE, e.data(), 4 * e.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_xsS, s.data(), 4 * s.size(), cudaMemcpyHostToDevice));
      // lookup groups: on interval k the linear interpolation of Sec. 2's tables is
      // sigma(E) = sigma_k + (E - E_k) (sigma_{k+1} - sigma_k) / (E_{k+1} - E_k)
      const int n = cfg->n_xs;
      std::vector<float4> g(3 * (size_t)(n - 1));
      auto sg = [&](int p, int k) { return h->xs_S[(size_t)p * n + k]; };
      for (int k = 0; k + 1 < n; ++k) {
        const double w = h->xs_E[k + 1] - h->xs_E[k];
        auto sl = [&](int p) { return (float)((sg(p, k + 1) - sg(p, k)) / w); };
        g[3 * k + 0] = make_float4((float)sg(0, k), (float)sg(1, k), (float)sg(2, k), 0.0f);
        g[3 * k + 1] = make_float4(sl(0), sl(1), sl(2), 0.0f);
        g[3 * k + 2] = make_float4((float)sg(3, k), (float)sg(4, k), sl(3), sl(4));
      }
      CK(cudaMemcpy(h->d_xsG, g.data(), sizeof(float4) * g.size(), cudaMemcpyHostToDevice));
    } else {
      CK(cudaMemcpy(h->d_xsE, h->xs_E.data(), 8 * h->xs_E.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_xsS, h->xs_S.data(), 8 * h->xs_S.size(), cudaMemcpyHostToDevice));
    }
    double sc[SC_N] = {0};
    sc[SC_CEQ] = 1.0;
    CK(cudaMemcpy(h->d_scalars, sc, sizeof(sc), cudaMemcpyHostToDevice));
    CK(cudaStreamSynchronize(h->stream));
    return PIC_OK;
  }();
  if (st) {
    free_all(h);
    delete h;
    return st;
  }
  *out = h;
  return PIC_OK;
}

int pic_set_particles(pic_handle *h, int species, int64_t n, const pic_particles *p) {
  if (!h || species < 0 || species > 1 || n < 0 || (n > 0 && (!p || !p->r || !p->z || !p->vr || !p->vt || !p->vz ||
                                                                !p->ar || !p->at || !p->az || !p->id)))
    return PIC_EINVAL;
  if (n > 0 && p->w && !h->weighted) return PIC_EINVAL;  // ratios need a weighted handle
  if (n > h->capacity[species]) return PIC_EOVERFLOW;
  if (sync(h)) return PIC_ECUDA;
  return h->prec == PIC_FP32 ? upload_species<float>(h, species, n, p) : upload_species<double>(h, species, n, p);
}

int pic_count(pic_handle *h, int species, int64_t *n) {
  if (!h || !n || species < 0 || species > 1) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  return h->prec == PIC_FP32 ? download_species<float>(h, species, nullptr, 0, n)
                             : download_species<double>(h, species, nullptr, 0, n);
}

int pic_get_particles(pic_handle *h, int species, pic_particles *out, int64_t cap, int64_t *n) {
  if (!h || !out || !n || species < 0 || species > 1) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  return h->prec == PIC_FP32 ? download_species<float>(h, species, out, cap, n)
                             : download_species<double>(h, species, out, cap, n);
}

int pic_start(pic_handle *h) {
  if (!h) return PIC_EINVAL;
  // deposit x~_0
  CK(cudaMemsetAsync(h->d_dep[0], 0, sizeof(unsigned long long) * h->nn, h->stream));
  CK(cudaMemsetAsync(h->d_dep[1], 0, sizeof(unsigned long long) * h->nn, h->stream));
  cudaError_t e = h->prec == PIC_FP32 ? launch_deposit_only<float>(push_params<float>(h, h->cur), h->stream)
                                      : launch_deposit_only<double>(push_params<double>(h, h->cur), h->stream);
  if (e != cudaSuccess) return PIC_ECUDA;
  // vacuum C_eq
  int st = enqueue_ceq(h, false);
  if (st) return st;
  double ce[2];
  CK(cudaMemcpyAsync(ce, h->d_ceq_out, sizeof(ce), cudaMemcpyDeviceToHost, h->stream));
  double sc[SC_N];
  CK(cudaMemcpyAsync(sc, h->d_scalars, sizeof(sc), cudaMemcpyDeviceToHost, h->stream));
  if (sync(h)) return PIC_ECUDA;
  const pic_config &c = h->cfg;
  sc[SC_CEQ] = ce[0];
  sc[SC_CEQ_GAUSS] = ce[1];
  uint32_t step = h->step;
  double t = step * c.dt;
  if (c.circuit == PIC_CIRCUIT_DIRECT) {
    sc[SC_UE] = c.V_src * std::sin(2.0 * kPi * c.f_src * t + c.phase_src);
    sc[SC_QE] = sc[SC_CEQ] * sc[SC_UE];
  } else {
    int n = c.circuit == PIC_CIRCUIT_RLC ? 3 : 6;
    sc[SC_QE] = sc[SC_Y0 + n - 1];
    sc[SC_UE] = sc[SC_QE] / sc[SC_CEQ];
  }
  sc[SC_T] = t;
  CK(cudaMemcpyAsync(h->d_scalars, sc, sizeof(sc), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_step, &step, sizeof(step), cudaMemcpyHostToDevice, h->stream));
  CK(launch_circuit_prepare(circuit_params(h, 1, nullptr, nullptr), h->stream));
  if (h->vahedi && (st = enqueue_laplace(h))) return st;  // vacuum, like C_eq
  CK(launch_assemble(field_params(h, h->d_chi, h->d_Gr, h->d_Gz, h->d_dinv), h->stream));
  if ((st = enqueue_solve(h, h->cfg.solver))) return st;
  if (h->vahedi) CK(launch_vahedi_combine(vahedi_params(h), h->stream));
  CK(launch_efield(efield_params(h), h->stream));
  if (sync(h)) return PIC_ECUDA;
  h->started = true;
  return PIC_OK;
}

int pic_particle_phase(pic_handle *h) {
  if (!h) return PIC_EINVAL;
  k_set_step<<<1, 1, 0, h->stream>>>(h->d_step, h->step);
  CK(cudaGetLastError());
  int st = enqueue_particle_phase(h, h->cur);
  if (st) return st;
  h->cur ^= 1;
  return sync(h);
}

int pic_step(pic_handle *h, int nsteps) {
  if (!h || nsteps < 0) return PIC_EINVAL;
  if (!h->started) {
    int st = pic_start(h);
    if (st) return st;
  }
  k_set_step<<<1, 1, 0, h->stream>>>(h->d_step, h->step);
  CK(cudaGetLastError());
  for (int k = 0; k < nsteps; ++k) {
    int buf = h->cur;
    if (h->timing) {
      cudaEvent_t ev[8];
      for (int q = 0; q < 8; ++q) {
        CK(cudaEventCreate(&ev[q]));
        h->tev.push_back(ev[q]);
      }
      int st = enqueue_step(h, buf, ev);
      if (st) return st;
    } else {
      if (h->cfg.solver == PIC_SOLVER_LEARNED && !h->fcg_exec) return PIC_EINVAL;
      if (!h->graph[buf] && !h->graph_failed && h->cfg.solver != PIC_SOLVER_LEARNED) {
        if (capture_graph(h, buf)) h->graph_failed = true;
      }
      if (h->graph[buf]) {
        CK(cudaGraphLaunch(h->graph[buf], h->stream));
      } else {
        int st = enqueue_step(h, buf, nullptr);
        if (st) return st;
      }
    }
    h->cur ^= 1;
    h->step++;
    if (h->step % (uint32_t)h->cfg.steps_per_rf == 0) {
      int st = window_end(h);
      if (st) return st;
    }
  }
  return PIC_OK;
}

int pic_enable_timing(pic_handle *h, int on) {
  if (!h) return PIC_EINVAL;
  h->timing = on != 0;
  return PIC_OK;
}

int pic_step_timing(pic_handle *h, double *out7) {
  if (!h || !out7) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (size_t b = 0; b + 8 <= h->tev.size(); b += 8)
    for (int q = 0; q < 7; ++q) {
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, h->tev[b + q], h->tev[b + q + 1]));
      acc[q] += ms;
    }
  for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
  h->tev.clear();
  for (int q = 0; q < 7; ++q) out7[q] = acc[q];
  return PIC_OK;
}

int pic_field_solve(pic_handle *h, int mode, int *iters, double *rel_resid) {
  if (!h || (mode != PIC_SOLVER_PLAIN && mode != PIC_SOLVER_MIXED && mode != PIC_SOLVER_LEARNED && mode != PIC_SOLVER_MG))
    return PIC_EINVAL;
  if (mode == PIC_SOLVER_LEARNED && !h->fcg_exec) return PIC_EINVAL;
  CK(launch_assemble(field_params(h, h->d_chi, h->d_Gr, h->d_Gz, h->d_dinv), h->stream));
  int st = enqueue_solve(h, mode);
  if (st) return st;
  if (h->vahedi) CK(launch_vahedi_combine(vahedi_params(h), h->stream));
  CK(launch_efield(efield_params(h), h->stream));
  double out[3];
  CK(cudaMemcpyAsync(out, h->d_pcg_out, sizeof(out), cudaMemcpyDeviceToHost, h->stream));
  if (sync(h)) return PIC_ECUDA;
  if (iters) *iters = (int)out[0];
  if (rel_resid) *rel_resid = out[1];
  int s = (int)out[2];
  return s == 0 ? PIC_OK : (s == -5 ? PIC_ETIMEOUT : (s == -7 ? PIC_ENAN : PIC_ENOCONV));
}

int pic_batch_create(pic_handle *const *hs, int n, pic_batch **out) {
  if (!hs || n < 1 || !out) return PIC_EINVAL;
  *out = nullptr;
  pic_batch *b = new (std::nothrow) pic_batch();
  if (!b) return PIC_ENOMEM;
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || hs[i]->device != hs[0]->device || hs[i]->cur != hs[0]->cur) { delete b; return PIC_EINVAL; }
    for (int k = 0; k < i; ++k)
      if (hs[k] == hs[i]) { delete b; return PIC_EINVAL; }
    b->hs.push_back(hs[i]);
  }
  for (pic_handle *h : b->hs) {
    if (!h->started) {
      int st = pic_start(h);
      if (st) { delete b; return st; }
    }
    if (sync(h)) { delete b; return PIC_ECUDA; }
  }
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    delete b;
    return PIC_ECUDA;
  }
  *out = b;
  return PIC_OK;
}

int pic_batch_step(pic_batch *b, int nsteps) {
  if (!b || nsteps < 0) return PIC_EINVAL;
  for (pic_handle *h : b->hs) {
    if (h->cur != b->hs[0]->cur) return PIC_EINVAL;
    if (sync(h)) return PIC_ECUDA;
    uint32_t step = h->step;
    CK(cudaMemcpy(h->d_step, &step, sizeof(step), cudaMemcpyHostToDevice));
  }
  for (int k = 0; k < nsteps; ++k) {
    const int parity = b->hs[0]->cur;
    if (!b->graph[parity]) {
      cudaError_t e = batch_build(b, parity);
      if (e != cudaSuccess) {
        fprintf(stderr, "pic: batch graph: %s\n", cudaGetErrorString(e));
        return PIC_ECUDA;
      }
    }
    CK(cudaGraphLaunch(b->graph[parity], b->stream));
    bool window = false;
    for (pic_handle *h : b->hs) {
      h->cur ^= 1;
      h->step++;
      window |= h->step % (uint32_t)h->cfg.steps_per_rf == 0;
    }
    if (window) {
      CK(cudaStreamSynchronize(b->stream));
      for (pic_handle *h : b->hs)
        if (h->step % (uint32_t)h->cfg.steps_per_rf == 0) {
          int st = window_end(h);
          if (st) return st;
        }
      // the window ends run on the handles' own streams (concurrently): the next
      // step waits for them, since they rewrite C_eq, the circuit propagator and
      // the solver scratch that the step's own solve uses
      for (pic_handle *h : b->hs)
        if (h->step % (uint32_t)h->cfg.steps_per_rf == 0) {
          CK(cudaEventRecord(b->done, h->stream));
          CK(cudaStreamWaitEvent(b->stream, b->done, 0));
        }
    }
  }
  // whatever is enqueued on a handle's own stream next (a read, a step) runs
  // after the batch's steps
  CK(cudaEventRecord(b->done, b->stream));
  for (pic_handle *h : b->hs) CK(cudaStreamWaitEvent(h->stream, b->done, 0));
  return PIC_OK;
}

int pic_batch_sync(pic_batch *b) {
  if (!b) return PIC_EINVAL;
  CK(cudaStreamSynchronize(b->stream));
  return PIC_OK;
}

void pic_batch_destroy(pic_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
}

int pic_attach_unet(pic_handle *h, pic_unet *u, int maxit, int smooth, int finish) {
  if (!h || maxit < 1 || smooth < 0 || smooth > 8) return PIC_EINVAL;
  if (finish != PIC_SOLVER_PLAIN && finish != PIC_SOLVER_MIXED && finish != PIC_SOLVER_MG) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  free_learned(h);
  if (!u) return PIC_OK;
  int H = 0, W = 0;
  unet::net_dims(u, &H, &W);
  if (H != h->nz || W != h->nr) return PIC_EINVAL;
  if (!h->side) CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  learned::FcgParams F = fcg_params(h);
  if (F.n_cov == 0) return PIC_EINVAL;
  const int nblk = learned::node_blocks(h->device);
  const size_t nn = h->nn;
  auto la = [&](void **p, size_t bytes) -> int {
    if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); return PIC_ENOMEM; }
    h->lallocs.push_back(*p);
    return cudaMemsetAsync(*p, 0, bytes, h->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
  };
  int st = 0;
  void *v = nullptr;
  st |= la(&v, sizeof(double) * 7 * nn);
  if (st) { free_learned(h); return PIC_ENOMEM; }
  double *d = (double *)v;
  F.r = d; F.z = d + nn; F.p[0] = d + 2 * nn; F.p[1] = d + 3 * nn; F.q[0] = d + 4 * nn; F.q[1] = d + 5 * nn;
  F.z2 = d + 6 * nn;
  F.smooth = smooth;
  F.omega = 2.0 / 3.0;
  st |= la(&v, sizeof(double) * 4 * 4 * nblk); F.part = (double *)v;
  st |= la(&v, sizeof(double) * 8); F.sc = (double *)v;
  st |= la(&v, sizeof(double) * nn); F.snap = (double *)v;
  st |= la(&v, sizeof(float) * 3 * (size_t)H * W); F.in3 = (float *)v;
  st |= la(&v, sizeof(float) * (size_t)H * W); F.out_net = (float *)v;
  if (st) { free_learned(h); return PIC_ENOMEM; }
  F.maxit = maxit;
  F.stats = h->d_lstats;
  if (sync(h)) { free_learned(h); return PIC_ECUDA; }
  cudaError_t e = learned::build_fcg_graph(F, nblk, u, h->side, &h->fcg_exec);
  if (e != cudaSuccess) {
    fprintf(stderr, "pic: learned solver graph: %s\n", cudaGetErrorString(e));
    h->fcg_exec = nullptr;
    free_learned(h);
    return PIC_ECUDA;
  }
  h->fcg = F;
  h->fcg_nblk = nblk;
  h->net = u;
  h->learned_finish = finish;
  return PIC_OK;
}

int pic_set_solver(pic_handle *h, int solver) {
  if (!h || (solver != PIC_SOLVER_PLAIN && solver != PIC_SOLVER_MIXED && solver != PIC_SOLVER_LEARNED &&
             solver != PIC_SOLVER_MG))
    return PIC_EINVAL;
  if (solver == PIC_SOLVER_LEARNED && h->vahedi) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  if (h->cfg.solver != solver) {
    for (int k = 0; k < 2; ++k)
      if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    h->graph[0] = h->graph[1] = nullptr;
    h->graph_failed = false;
  }
  h->cfg.solver = solver;
  return PIC_OK;
}

int pic_keep_warm(pic_handle *h, int on) {
  if (!h) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  if (h->keep_warm != (on != 0)) {
    // the step graphs hold the solve sequence: capture them again
    for (int k = 0; k < 2; ++k)
      if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    h->graph[0] = h->graph[1] = nullptr;
    h->graph_failed = false;
  }
  h->keep_warm = on != 0;
  return PIC_OK;
}

int pic_learned_snapshot(pic_handle *h, int k) {
  if (!h || k < 0 || !h->fcg_exec) return PIC_EINVAL;
  double v = (double)k;
  CK(cudaMemcpyAsync(h->fcg.sc + 6, &v, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  return sync(h);
}

int pic_learned_pair(pic_handle *h, int source, float *in3, float *target, double *scale) {
  if (!h || !in3 || !target || source < 0 || source > 1) return PIC_EINVAL;
  if (source == 0 && !h->keep_warm && !h->fcg_exec) return PIC_EINVAL;
  if (source == 1 && !h->fcg_exec) return PIC_EINVAL;
  learned::FcgParams F = fcg_params(h);
  if (F.n_cov == 0) return PIC_EINVAL;
  F.in3 = in3;
  const double *from = source == 0 ? h->d_phi_warm : h->fcg.snap;
  CK(learned::launch_pair(F, learned::node_blocks(h->device), from, target, h->d_pair_s2, h->stream));
  double s2 = 0.0;
  CK(cudaMemcpyAsync(&s2, h->d_pair_s2, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (sync(h)) return PIC_ECUDA;
  if (scale) *scale = std::sqrt(s2 / (double)F.n_cov);
  return PIC_OK;
}

int pic_learned_stats(pic_handle *h, double *out4) {
  if (!h || !out4) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  double ls[4], ps[3];
  CK(cudaMemcpy(ls, h->d_lstats, sizeof(ls), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(ps, h->d_pcg_out, sizeof(ps), cudaMemcpyDeviceToHost));
  out4[0] = ls[0];
  out4[1] = ls[1];
  out4[2] = ls[2];
  out4[3] = ps[0];
  return PIC_OK;
}

int pic_ceq(pic_handle *h, int with_chi, double *ceq, double *gauss) {
  if (!h) return PIC_EINVAL;
  int st = enqueue_ceq(h, with_chi != 0);
  if (st) return st;
  double ce[2];
  CK(cudaMemcpyAsync(ce, h->d_ceq_out, sizeof(ce), cudaMemcpyDeviceToHost, h->stream));
  if (sync(h)) return PIC_ECUDA;
  if (ceq) *ceq = ce[0];
  if (gauss) *gauss = ce[1];
  return PIC_OK;
}

int pic_diag_async(pic_handle *h, int what, void *host_buf, size_t bytes) {
  if (!h || !host_buf || what != PIC_DIAG_SCALARS || bytes < sizeof(double) * PIC_NSCALARS) return PIC_EINVAL;
  return enqueue_scalars(h, static_cast<double *>(host_buf));
}

int pic_sync(pic_handle *h) {
  if (!h) return PIC_EINVAL;
  return sync(h);
}

int pic_diag(pic_handle *h, int what, void *host_buf, size_t bytes) {
  if (!h || !host_buf) return PIC_EINVAL;
  if (what & PIC_DIAG_DEVICE) return diag_to_device(h, what & ~PIC_DIAG_DEVICE, static_cast<double *>(host_buf), bytes);
  const size_t nb = sizeof(double) * h->nn;
  if (sync(h)) return PIC_ECUDA;
  double *o = (double *)host_buf;
  if (what == PIC_DIAG_SCALARS) {
    if (bytes < sizeof(double) * PIC_NSCALARS) return PIC_EINVAL;
    int st = enqueue_scalars(h, o);
    if (st) return st;
    return sync(h);
  }
  if (what == PIC_DIAG_CIRCUIT) {
    if (bytes < sizeof(double) * 18) return PIC_EINVAL;
    CK(cudaMemcpy(o, h->d_scalars + SC_COUT, sizeof(double) * 18, cudaMemcpyDeviceToHost));
    return PIC_OK;
  }
  if (what == PIC_DIAG_SOLVER) {
    if (bytes < sizeof(double) * 5) return PIC_EINVAL;
    int solves = 0;
    double pcg[4];
    CK(cudaMemcpy(&solves, h->mg.solves, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(pcg, h->d_pcg_out, sizeof(pcg), cudaMemcpyDeviceToHost));
    o[0] = solves;
    o[1] = h->mg.rebuild_every;
    o[2] = pcg[0];
    o[3] = pcg[3];
    o[4] = pcg[2];
    return PIC_OK;
  }
  if (what == PIC_DIAG_STORE) {
    if (bytes < sizeof(double) * 8) return PIC_EINVAL;
    std::vector<int> cap(h->nbins), fill(h->nbins);
    for (int s = 0; s < 2; ++s) {
      const Store &S = h->st[h->cur][s];
      BinMeta m;
      CK(cudaMemcpy(cap.data(), S.cap, sizeof(int) * h->nbins, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(fill.data(), S.fill, sizeof(int) * h->nbins, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(&m, S.meta, sizeof(BinMeta), cudaMemcpyDeviceToHost));
      int64_t in_bins = 0;
      for (int b = 0; b < h->nbins; ++b) in_bins += fill[b] < cap[b] ? fill[b] : cap[b];
      int64_t novf = m.ovf_n;
      if (novf > h->capacity[s] - m.ovf_base) novf = h->capacity[s] - m.ovf_base;
      if (novf < 0) novf = 0;
      o[4 * s + 0] = (double)in_bins;
      o[4 * s + 1] = (double)novf;
      o[4 * s + 2] = (double)h->capacity[s];
      o[4 * s + 3] = (double)m.ovf_base;
    }
    return PIC_OK;
  }
  if (bytes < nb) return PIC_EINVAL;
  switch (what) {
    case PIC_DIAG_PHI: CK(cudaMemcpy(o, h->d_phi, nb, cudaMemcpyDeviceToHost)); return PIC_OK;
    case PIC_DIAG_ER: CK(cudaMemcpy(o, h->d_Er, nb, cudaMemcpyDeviceToHost)); return PIC_OK;
    case PIC_DIAG_EZ: CK(cudaMemcpy(o, h->d_Ez, nb, cudaMemcpyDeviceToHost)); return PIC_OK;
    case PIC_DIAG_CHI: CK(cudaMemcpy(o, h->d_chi, nb, cudaMemcpyDeviceToHost)); return PIC_OK;
    case PIC_DIAG_VNODE: CK(cudaMemcpy(o, h->d_vnode, nb, cudaMemcpyDeviceToHost)); return PIC_OK;
    case PIC_DIAG_RHO: CK(cudaMemcpy(o, h->d_qrhs, nb, cudaMemcpyDeviceToHost)); return PIC_OK;
    case PIC_DIAG_NE_AVG: CK(cudaMemcpy(o, h->d_dens_avg[0], nb, cudaMemcpyDeviceToHost)); return PIC_OK;
    case PIC_DIAG_NI_AVG: CK(cudaMemcpy(o, h->d_dens_avg[1], nb, cudaMemcpyDeviceToHost)); return PIC_OK;
    case PIC_DIAG_PHI_WARM: CK(cudaMemcpy(o, h->d_phi_warm, nb, cudaMemcpyDeviceToHost)); return PIC_OK;
    case PIC_DIAG_PHI_P:
      if (!h->vahedi) return PIC_EINVAL;
      CK(cudaMemcpy(o, h->d_phiP, nb, cudaMemcpyDeviceToHost));
      return PIC_OK;
    case PIC_DIAG_PHI_L0:
      if (!h->vahedi) return PIC_EINVAL;
      CK(cudaMemcpy(o, h->d_phiL, nb, cudaMemcpyDeviceToHost));
      return PIC_OK;
    case PIC_DIAG_PHI_L0 + 1:
    case PIC_DIAG_PHI_L0 + 2:
    case PIC_DIAG_PHI_L0 + 3: {
      const int k = what - PIC_DIAG_PHI_L0 - 1;
      if (!h->vahedi || k >= h->cfg.n_drive) return PIC_EINVAL;
      CK(cudaMemcpy(o, h->d_phiLd[k], nb, cudaMemcpyDeviceToHost));
      return PIC_OK;
    }
    case PIC_DIAG_DEP_E:
    case PIC_DIAG_DEP_I:
    case PIC_DIAG_SIGMA: {
      // converted on the device (the solver's scratch vector holds them), as in
      // the device form, then copied
      int st = enqueue_counts(h, what, h->d_work);
      if (st) return st;
      CK(cudaMemcpyAsync(o, h->d_work, nb, cudaMemcpyDeviceToHost, h->stream));
      return sync(h);
    }
    default: return PIC_EINVAL;
  }
}

int pic_set_field(pic_handle *h, int what, const double *host_buf, size_t n) {
  if (!h || !host_buf || n != (size_t)h->nn) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  const size_t nb = sizeof(double) * h->nn;
  switch (what) {
    case PIC_DIAG_PHI: CK(cudaMemcpy(h->d_phi, host_buf, nb, cudaMemcpyHostToDevice)); return PIC_OK;
    case PIC_DIAG_RHO: CK(cudaMemcpy(h->d_qrhs, host_buf, nb, cudaMemcpyHostToDevice)); return PIC_OK;
    case PIC_DIAG_ER:
    case PIC_DIAG_EZ: {
      CK(cudaMemcpy(what == PIC_DIAG_ER ? h->d_Er : h->d_Ez, host_buf, nb, cudaMemcpyHostToDevice));
      std::vector<double> er(h->nn), ez(h->nn);
      CK(cudaMemcpy(er.data(), h->d_Er, nb, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(ez.data(), h->d_Ez, nb, cudaMemcpyDeviceToHost));
      if (h->prec == PIC_FP32) {
        std::vector<float2> e(h->nn);
        for (int a = 0; a < h->nn; ++a) e[a] = make_float2((float)er[a], (float)ez[a]);
        CK(cudaMemcpy(h->d_E, e.data(), sizeof(float2) * h->nn, cudaMemcpyHostToDevice));
      } else {
        std::vector<double2> e(h->nn);
        for (int a = 0; a < h->nn; ++a) e[a] = make_double2(er[a], ez[a]);
        CK(cudaMemcpy(h->d_E, e.data(), sizeof(double2) * h->nn, cudaMemcpyHostToDevice));
      }
      return PIC_OK;
    }
    case PIC_DIAG_DEP_E:
    case PIC_DIAG_DEP_I: {
      std::vector<unsigned long long> u(h->nn);
      double sc = 1.0 / dep_inv_scale(h);
      for (int a = 0; a < h->nn; ++a) u[a] = (unsigned long long)std::llround(host_buf[a] * sc);
      CK(cudaMemcpy(h->d_dep[what - PIC_DIAG_DEP_E], u.data(), sizeof(unsigned long long) * h->nn,
                    cudaMemcpyHostToDevice));
      return PIC_OK;
    }
    default: return PIC_EINVAL;
  }
}

int pic_set_step(pic_handle *h, uint32_t step) {
  if (!h) return PIC_EINVAL;
  h->step = step;
  CK(cudaMemcpyAsync(h->d_step, &h->step, sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream));
  return sync(h);
}

int pic_set_ceq(pic_handle *h, double ceq) {
  if (!h || !(ceq > 0)) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  CK(cudaMemcpy(h->d_scalars + SC_CEQ, &ceq, sizeof(double), cudaMemcpyHostToDevice));
  CK(launch_circuit_prepare(circuit_params(h, 1, nullptr, nullptr), h->stream));
  return sync(h);
}

int pic_set_circuit_state(pic_handle *h, const double *y6) {
  if (!h || !y6) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  double sc[SC_N];
  CK(cudaMemcpy(sc, h->d_scalars, sizeof(sc), cudaMemcpyDeviceToHost));
  for (int k = 0; k < 6; ++k) sc[SC_Y0 + k] = y6[k];
  int n = h->cfg.circuit == PIC_CIRCUIT_RLC ? 3 : (h->cfg.circuit == PIC_CIRCUIT_IMN ? 6 : 0);
  if (n) sc[SC_QE] = sc[SC_Y0 + n - 1];
  sc[SC_UE] = sc[SC_QE] / sc[SC_CEQ];
  CK(cudaMemcpy(h->d_scalars, sc, sizeof(sc), cudaMemcpyHostToDevice));
  return PIC_OK;
}

int pic_set_conv_current(pic_handle *h, double I_conv) {
  // The circuit kernel derives I_conv from the absorbed-particle counters;
  // express the requested current as an electron count at the powered node.
  if (!h) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  unsigned long long cnt[CNT_N] = {0};
  const pic_config &c = h->cfg;
  double per = c.q[0] * c.w[0] / c.dt;
  if (I_conv != 0.0) {
    double k = I_conv / per;
    if (h->weighted) {  // weighted tallies hold macro weights to 2^-32
      if (!(k >= 0) || !(k < 1e9)) return PIC_EINVAL;
      cnt[CNT_ABSW + 0] = (unsigned long long)std::llround(k * kCreditOne);
    } else {
      if (!(k >= 0) || std::fabs(k - std::llround(k)) > 1e-9 * (1 + std::fabs(k))) return PIC_EINVAL;
      cnt[CNT_ABS + 0] = (unsigned long long)std::llround(k);
    }
  }
  CK(cudaMemcpy(h->d_counters, cnt, sizeof(cnt), cudaMemcpyHostToDevice));
  return PIC_OK;
}

int pic_circuit_run(pic_handle *h, int n, double *U_out) {
  if (!h || n < 0) return PIC_EINVAL;
  double *d_hist = nullptr;
  if (U_out && n > 0) {
    if (cudaMalloc(&d_hist, sizeof(double) * n) != cudaSuccess) return PIC_ENOMEM;
  }
  uint32_t step = h->step;
  CK(cudaMemcpyAsync(h->d_step, &step, sizeof(step), cudaMemcpyHostToDevice, h->stream));
  cudaError_t e = launch_circuit(circuit_params(h, n, d_hist, h->d_step), h->stream);
  if (e == cudaSuccess && d_hist) e = cudaMemcpyAsync(U_out, d_hist, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (d_hist) cudaFree(d_hist);
  if (e != cudaSuccess) return PIC_ECUDA;
  h->step += n;
  return PIC_OK;
}

int pic_status(pic_handle *h, uint32_t *flags) {
  if (!h || !flags) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  uint32_t f = 0;
  CK(cudaMemcpy(&f, h->d_flags, sizeof(f), cudaMemcpyDeviceToHost));
  uint32_t z = 0;
  CK(cudaMemcpy(h->d_flags, &z, sizeof(z), cudaMemcpyHostToDevice));
  *flags = f;
  return PIC_OK;
}

int pic_check(pic_handle *h) {
  if (!h) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  uint32_t f = 0;
  CK(cudaMemcpy(&f, h->d_flags, sizeof(f), cudaMemcpyDeviceToHost));
  if (f & PIC_FLAG_OVERFLOW) return PIC_EOVERFLOW;
  if (f & PIC_FLAG_TIMEOUT) return PIC_ETIMEOUT;
  if (f & PIC_FLAG_NAN) return PIC_ENAN;
  if (f & PIC_FLAG_NOCONV) return PIC_ENOCONV;
  return PIC_OK;
}

int pic_set_spin_limit(pic_handle *h, int64_t cycles) {
  if (!h || cycles < 0) return PIC_EINVAL;
  if (sync(h)) return PIC_ECUDA;
  if (h->cfg.spin_limit != cycles) {
    // the step graphs hold the solve's parameters: capture them again
    for (int k = 0; k < 2; ++k)
      if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    h->graph[0] = h->graph[1] = nullptr;
    h->graph_failed = false;
  }
  h->cfg.spin_limit = cycles;
  return PIC_OK;
}

int pic_philox(pic_handle *h, int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  if (!h || n < 0 || (n > 0 && (!ctr || !key || !out))) return PIC_EINVAL;
  if (n == 0) return PIC_OK;
  uint32_t *d = nullptr;
  size_t bytes = sizeof(uint32_t) * (size_t)n * 10;
  if (cudaMalloc(&d, bytes) != cudaSuccess) return PIC_ENOMEM;
  cudaError_t e = cudaMemcpy(d, ctr, sizeof(uint32_t) * 4 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d + 4 * n, key, sizeof(uint32_t) * 2 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_philox(n, d, d + 4 * n, d + 6 * n, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(out, d + 6 * n, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

}  // extern "C"
