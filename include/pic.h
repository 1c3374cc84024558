/*
 * pic.h -- C ABI of the GB300 implicit r-z PIC/MCC library (libpic_gb300.so).
 *
 * The library advances a 2D axisymmetric electrostatic direct-implicit
 * particle-in-cell / Monte Carlo collision model of a capacitively coupled
 * argon discharge driven through an external circuit (arXiv:2310.04957,
 * Sec. 2).  One handle is one discharge on the current CUDA device.
 *
 * Conventions
 *   - Every function returns PIC_OK (0) or a negative PIC_E* code; nothing
 *     traps and no C++ exception crosses this boundary.
 *   - Pointers marked "host" are read or written synchronously and stay owned
 *     by the caller; the library copies what it keeps.  Device memory the
 *     library allocates belongs to the handle and is freed by pic_destroy.
 *   - Work is enqueued on the CUDA stream given to pic_init; functions that
 *     return host data synchronise that stream first.
 *   - Node arrays are [(nz+1) x (nr+1)] row-major, index j*(nr+1)+i with
 *     r_i = i*dr, z_j = j*dz; cell arrays are [nz x nr], index j*nr+i.
 *   - Species 0 = electrons, 1 = Ar+.
 */
#ifndef PIC_GB300_H
#define PIC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PIC_OK 0
#define PIC_EINVAL -1    /* bad argument or configuration */
#define PIC_ENOMEM -2    /* device or host allocation failed */
#define PIC_ECUDA -3     /* a CUDA runtime call failed */
#define PIC_ENOCONV -4   /* field solve hit its iteration cap */
#define PIC_ETIMEOUT -5  /* a bounded device-side wait ran out */
#define PIC_EOVERFLOW -6 /* particle store or overflow region full */
#define PIC_ENAN -7      /* non-finite value in the field solve */
#define PIC_EIO -8       /* restart file could not be written or read, or is not one */

/* status-word bits (pic_status) */
#define PIC_FLAG_OVERFLOW 0x1u
#define PIC_FLAG_TIMEOUT 0x2u
#define PIC_FLAG_NOCONV 0x4u
#define PIC_FLAG_NAN 0x8u
#define PIC_FLAG_OUTSIDE 0x10u /* a stored particle was found outside the plasma */

/* ---- enumerations ------------------------------------------------------ */
#define PIC_NODE_FREE 0
#define PIC_NODE_POWERED 1
#define PIC_NODE_GROUNDED 2
#define PIC_NODE_DRIVEN 3   /* first voltage-driven electrode: kinds 3, 4, 5 are
                               electrodes 1..3 of pic_config.drive_* (a particle
                               absorbed there counts as a grounded-type exit) */

#define PIC_CELL_PLASMA 0
#define PIC_CELL_POWERED 1
#define PIC_CELL_GROUNDED 2
#define PIC_CELL_DIELECTRIC 3

#define PIC_CIRCUIT_DIRECT 0 /* U_E = V sin(2 pi f t + phase) imposed           */
#define PIC_CIRCUIT_RLC 1    /* circuit I, Eq. 9: source + series Rb, Lb, Cb    */
#define PIC_CIRCUIT_IMN 2    /* circuit II, Eq. 10: source Rs, L-type matching
                                network (shunt Cm1, series Rm Lm Cm2) and stray
                                branch (Rstray, Lstray, Cstray)                  */

#define PIC_FP32 0 /* particle state and push in FP32; FP64 reductions, field, circuit */
#define PIC_FP64 1 /* everything in FP64 (the plain method)                          */

/* Field composition (Sec. 2, Eqs. 2-4). */
#define PIC_FIELD_DIRECT 0 /* one solve of Eq. 1 with every electrode at its voltage */
#define PIC_FIELD_VAHEDI 1 /* phi = phi_P + U_E phi_L0 + sum_k U_k phi_Lk (Eq. 2):
                              phi_P solves Eq. 1 with every electrode at 0 (Eq. 3)
                              each step; phi_L0 / phi_Lk are the unit-voltage
                              solutions of the powered / driven electrodes (Eq. 4,
                              the implicit operator with the chi of their last
                              refresh), re-solved together with C_eq: in vacuum
                              at start and with chi at every RF-window end when
                              ceq_refresh is set                                 */

#define PIC_SOLVER_PLAIN 0 /* FP64 Jacobi-preconditioned CG                        */
#define PIC_SOLVER_MIXED 1 /* FP32 Jacobi-preconditioned inner CG, FP64
                              residual and iterative refinement                    */
#define PIC_SOLVER_MG 3      /* FP32 CG preconditioned by a multigrid V-cycle
                              (2x2 aggregation, smoothed prolongation at the
                              finest level, damped Jacobi smoothing), FP64
                              residual and iterative refinement                */
#define PIC_SOLVER_LEARNED 2 /* flexible CG preconditioned by the attached U-Net
                              (pic_attach_unet), FP64 recurrences; the plain or
                              mixed PCG then confirms the residual and finishes
                              the solve if the learned loop stopped short     */

/* ---- configuration ------------------------------------------------------
 * Everything that defines one discharge (Sec. 2: reactor geometry on a
 * regular r-z grid, argon gas and species, cross sections, external circuit,
 * time step).  Arrays are host pointers, copied by pic_init. */
typedef struct pic_config {
  int32_t nr, nz;              /* cells in r and z (nodes (nr+1) x (nz+1))        */
  double dr, dz;               /* cell sizes, m                                    */
  const int8_t *node_kind;     /* host [(nz+1)*(nr+1)] PIC_NODE_*: metal nodes are
                                  Dirichlet (powered at U_E, grounded at 0)      */
  const int8_t *cell_kind;     /* host [nz*nr] PIC_CELL_*: particles live in plasma
                                  cells and are absorbed elsewhere               */
  const double *cell_eps;      /* host [nz*nr] relative permittivity per cell     */
  double dt;                   /* time step, s                                     */
  double n_gas, T_gas, m_gas;  /* neutral density m^-3, temperature K, mass kg     */
  double q[2], m[2], w[2];     /* per species charge C, mass kg, macro weight      */
  int32_t n_xs;                /* cross-section table length (>= 2)                */
  const double *xs_energy;     /* host [n_xs] eV, logarithmically spaced           */
  const double *xs_sigma;      /* host [5*n_xs] m^2: e elastic, e excitation,
                                  e ionization, Ar+ isotropic, Ar+ charge exchange */
  double thr_ex, thr_iz;       /* excitation / ionization thresholds, eV           */
  double B_ej;                 /* ejected-electron energy-sharing parameter, eV    */
  int32_t circuit;             /* PIC_CIRCUIT_*                                    */
  double circ[8];              /* RLC: Rb, Lb, Cb.  IMN: Rs, Cm1, Lm, Cm2, Rm,
                                  Cstray, Rstray, Lstray (SI units)              */
  double V_src, f_src, phase_src; /* source amplitude V, frequency Hz, phase rad   */
  int32_t n_sub;               /* trapezoidal circuit substeps per dt              */
  int32_t steps_per_rf;        /* diagnostic window (one RF period), steps         */
  double pcg_tol;              /* relative residual target of the field solve      */
  int32_t pcg_maxit;           /* iteration cap (PIC_ENOCONV beyond)               */
  int32_t ceq_refresh;         /* recompute C_eq with chi after every window       */
  uint32_t seed;               /* fourth word of every Philox counter              */
  int64_t capacity[2];         /* particle capacity per species                    */
  int32_t precision;           /* PIC_FP32 or PIC_FP64                             */
  int32_t solver;              /* PIC_SOLVER_*                                     */
  int32_t tile_r, tile_z;      /* cells per CTA tile (0 = library default)         */
  double bin_slack;            /* extra bin room as a fraction of last count (0 = default) */
  int64_t spin_limit;          /* clock cycles a field-solve grid barrier may wait
                                  for the other blocks before the solve gives up
                                  with PIC_ETIMEOUT (0 = default, 4e9: ~2 s)     */
  int32_t weighted;            /* 1: unequal macroparticle weights (Sec. 2) -- each
                                  particle carries a weight ratio w in (0, 1]
                                  (macro weight w * w[species]) that scales its
                                  deposit and absorbed charge; newborn particles
                                  take their parent's ratio.  0: all ratios 1  */
  int32_t split_cells;         /* particle splitting near the axis (Sec. 2;
                                  requires weighted = 1; 0 = off, at most nr):
                                  radial cell i < split_cells has the target
                                  ratio (2i+1)/(2 split_cells + 1), 1 beyond; a
                                  particle that enters a cell with a ratio above
                                  twice its target is split into two halves of
                                  the same state, the second with the id
                                  Philox4x32-10(key = parent id, counter = (step,
                                  0x5B17, 0, seed)) with bit 63 set; both halves
                                  count as deposited by the parent's deposit   */
  int32_t n_drive;             /* voltage-driven electrodes (0..3): node kinds 3 ..
                                  2 + n_drive, electrode k at
                                  drive_V[k] sin(2 pi drive_f[k] t + drive_phase[k])
                                  (V, Hz, rad) -- an ideal source, no circuit  */
  double drive_V[3], drive_f[3], drive_phase[3];
  int32_t field_mode;          /* PIC_FIELD_DIRECT or PIC_FIELD_VAHEDI (not with
                                  PIC_SOLVER_LEARNED)                            */
} pic_config;

/* Particle arrays of one species in FP64 host memory (caller-owned).  Position
 * (r, z) is x~, the predicted position; (vr, vt, vz) the velocity v_{n-3/2}
 * in the local (r, theta, z) frame; (ar, at, az) the D1 time-filtered
 * acceleration a-bar_{n-2}; id the 64-bit identifier that keys its random
 * numbers.  `cell` (output only, may be NULL) is j*nr+i of x~. */
typedef struct pic_particles {
  double *r, *z, *vr, *vt, *vz, *ar, *at, *az;
  uint64_t *id;
  int32_t *cell;
  double *w;  /* weight ratios in (0, 1]: input of weighted handles (NULL = all 1;
                 must be NULL for unweighted ones), output if not NULL (all 1
                 for unweighted handles) */
} pic_particles;

typedef struct pic_handle pic_handle;

/* pic_init -- create a discharge.  Validates `cfg`, copies the geometry,
 * cross sections and circuit, builds the vacuum part of the finite-volume
 * operator of Eq. 1 and the null-collision bounds, allocates the particle
 * stores (two buffers of cfg->capacity per species) on the current device.
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 * Errors: PIC_EINVAL (bad sizes, kinds, table), PIC_ENOMEM, PIC_ECUDA. */
int pic_init(const pic_config *cfg, void *cuda_stream, pic_handle **out);

/* pic_set_particles -- replace species `species` with `n` particles from host
 * FP64 arrays (converted to the handle's precision, cell-relative position).
 * Errors: PIC_EINVAL (a particle outside the plasma region or bad species),
 * PIC_EOVERFLOW (n > capacity). */
int pic_set_particles(pic_handle *h, int species, int64_t n, const pic_particles *p);

/* pic_count -- number of stored particles of a species (synchronises). */
int pic_count(pic_handle *h, int species, int64_t *n);

/* pic_get_particles -- copy a species to host FP64 arrays of length >= cap;
 * *n receives the count.  Order is by cell (bins), unspecified within a cell. */
int pic_get_particles(pic_handle *h, int species, pic_particles *out, int64_t cap, int64_t *n);

/* pic_start -- start-up of the implicit scheme: deposit x~_0, C_eq of the
 * vacuum (Eqs. 6-7), U_E(t_0), assemble and solve Eq. 1, node E field. */
int pic_start(pic_handle *h);

/* pic_step -- advance `nsteps` full time steps (particle phase, circuit with
 * Eqs. 5 and 8-10, assembly and solve of Eq. 1, E field, diagnostics), as one
 * captured CUDA graph per step.  Asynchronous; errors surface in pic_status. */
int pic_step(pic_handle *h, int nsteps);

/* pic_particle_phase -- only the particle phase of one step (gather, D1
 * correction, absorption, null-collision MCC, predictor with cylindrical
 * rotation, re-bin by cell, deposit of counts).  Does not advance the step
 * counter.  Asynchronous. */
int pic_particle_phase(pic_handle *h);

/* pic_field_solve -- assemble rho~ and chi from the current deposits and
 * solve Eq. 1 with solver `mode` (PIC_SOLVER_*), then the node E field.
 * Synchronises; returns iterations and the final relative residual.
 * Errors: PIC_ENOCONV, PIC_ETIMEOUT, PIC_ENAN. */
int pic_field_solve(pic_handle *h, int mode, int *iters, double *rel_resid);

/* pic_ceq -- equivalent capacitance from the field energy of the unit-voltage
 * solution (Eqs. 6-7), with (with_chi=1) or without the current chi; also the
 * Gauss-law electrode charge.  Does not change the handle's C_eq. */
int pic_ceq(pic_handle *h, int with_chi, double *ceq, double *gauss);

/* Diagnostic selectors for pic_diag (host buffer of doubles). */
#define PIC_DIAG_PHI 0     /* potential, V                     [nodes] */
#define PIC_DIAG_ER 1      /* E_r, V/m                         [nodes] */
#define PIC_DIAG_EZ 2      /* E_z, V/m                         [nodes] */
#define PIC_DIAG_CHI 3     /* implicit susceptibility          [nodes] */
#define PIC_DIAG_DEP_E 4   /* deposited electron counts        [nodes] */
#define PIC_DIAG_DEP_I 5   /* deposited ion counts             [nodes] */
#define PIC_DIAG_SIGMA 6   /* surface charge on free nodes, C  [nodes] */
#define PIC_DIAG_VNODE 7   /* plasma node volume, m^3          [nodes] */
#define PIC_DIAG_RHO 8     /* node charge rho~ (incl. surface) [nodes] */
#define PIC_DIAG_NE_AVG 9  /* last window's mean n_e, m^-3     [nodes] */
#define PIC_DIAG_NI_AVG 10 /* last window's mean n_i, m^-3     [nodes] */
#define PIC_DIAG_PHI_WARM 11 /* warm start of the last solve, V (kept by
                                pic_keep_warm or the learned solver) [nodes] */
#define PIC_DIAG_PHI_P 12    /* PIC_FIELD_VAHEDI: zero-boundary part phi_P, V [nodes] */
#define PIC_DIAG_PHI_L0 13   /* PIC_FIELD_VAHEDI: unit Laplace solution of the powered
                                electrode; 14..16 those of driven electrodes 1..3
                                (dimensionless) [nodes] */
#define PIC_DIAG_SCALARS 100 /* PIC_NSCALARS doubles, see below  */
#define PIC_DIAG_STORE 101   /* 8 doubles: per species (electrons, then ions)
                                particles in their cell bins, particles in the
                                overflow region (those that did not fit their
                                bin at the last re-bin), capacity, first slot
                                of the overflow region */
#define PIC_DIAG_CIRCUIT 103 /* 18 doubles, circuit post-processing of the last
                                RF window (Sec. 3): [0..1] Z_ccp = U_E,1 / I_ccp,1
                                and [2..3] Z_load = U_in,1 / I_1,1 (ohm, Re, Im;
                                first harmonics by DFT over the window, Eq. 11;
                                U_in is the voltage after the source resistance,
                                I_1 the source current), [4..5] Gamma =
                                (Z_load - R_s)/(Z_load + R_s) (Eq. 12; circuit II
                                only), [6] |Gamma|, window-averaged powers
                                (Eq. 13, W): [7] source U_s I_1, [8] R_s, [9] the
                                series element (R_m of the matching network; R_b
                                in circuit I), [10] stray branch, [11] plasma load
                                U_E I_ccp, [12] forward (U_in I_1), [13] reflected
                                P_forward |Gamma|^2 (Eq. 14); [14..15] first
                                harmonic of U_E (V); [16] mean U_E over the
                                window, the DC self-bias of Sec. 3's circuit I
                                (V); [17] mean I_ccp (A).  Direct drive: U_s =
                                U_in = U_E and I_1 = I_ccp. */
#define PIC_DIAG_SOLVER 102  /* 5 doubles: multigrid solves counter (the next
                                PIC_SOLVER_MG solve rebuilds the coarse
                                hierarchy when it is a multiple of [1], else
                                reuses it; a failed solve resets it to 0),
                                rebuild period, last solve's iterations,
                                outer refinement steps, status */
#define PIC_NSCALARS 49
/* Scalars: [0] step, [1] t, [2] U_E, [3] Q_E, [4] C_eq, [5] I_conv, [6] I_ccp,
 * [7..12] circuit state (RLC: Qb, Ib, QE; IMN: Q1, Q2, I2, Qccp, Istray, QE),
 * [13] field-solve iterations, [14] relative residual, [15..16] nu_max e/i,
 * [17..18] collision probability e/i, [19..24] absorbed charge of the last
 * step (e: powered, grounded, surface; i: same), [25..30] absorbed counts,
 * [31..36] collisions of the last step (e: elastic, excitation, ionization;
 * i: isotropic, charge exchange, 0), [37..38] births e/i, [39..41] ion
 * current of the last window (powered, grounded, surface), [42..43] first
 * harmonic of I_ccp over the last window (Re, Im), [44] windows completed,
 * [45] C_eq by the Gauss route, [46] field-solve status, [47..48] particles
 * split near the axis in the last step e/i.  The absorbed charge of weighted
 * handles sums the particles' weight ratios (to 2^-32 of a macro weight). */

/* pic_diag -- copy one diagnostic to a host buffer of `bytes` bytes
 * (synchronises).  With PIC_DIAG_DEVICE or'ed into `what`, the buffer is device
 * memory on the handle's device (a CUDA tensor, say) and the copy is enqueued on
 * the handle's stream without waiting; work on another stream that reads the
 * buffer must wait for that stream.  The device form serves the node arrays and
 * PIC_DIAG_SCALARS, with the values of the host form bit for bit; the other
 * selectors are host-only.  Errors: PIC_EINVAL for an unknown selector, a
 * host-only selector with PIC_DIAG_DEVICE, or a short buffer. */
#define PIC_DIAG_DEVICE 0x10000
int pic_diag(pic_handle *h, int what, void *host_buf, size_t bytes);

/* pic_diag_async -- enqueue, on the handle's stream, the read of the scalars
 * (what = PIC_DIAG_SCALARS only; PIC_NSCALARS doubles, the values pic_diag
 * gives at the same point of the stream) into host_buf, and return without
 * waiting.  host_buf is the caller's and must stay valid until the copy has
 * run: after pic_sync, or any call that synchronises, it holds the scalars of
 * the step the read followed.  In page-locked memory (cudaHostAlloc, a pinned
 * tensor) the copy is asynchronous; from pageable memory the CUDA runtime may
 * make it wait.  A run can so log every step's scalars while the host keeps
 * enqueuing steps ahead of the device.  Errors: PIC_EINVAL for another
 * selector, a NULL buffer or fewer than PIC_NSCALARS doubles. */
int pic_diag_async(pic_handle *h, int what, void *host_buf, size_t bytes);

/* pic_sync -- wait until everything enqueued on the handle's stream has run.
 * Errors: PIC_ECUDA if a launch or copy failed. */
int pic_sync(pic_handle *h);

/* pic_set_field -- overwrite a node array (PIC_DIAG_PHI, _ER, _EZ, _DEP_E,
 * _DEP_I, _SIGMA or _RHO) from a host buffer: test and restart hook.
 * Setting _ER/_EZ updates the copy the particle gather reads. */
int pic_set_field(pic_handle *h, int what, const double *host_buf, size_t n);

/* State hooks (restart and component tests). */
int pic_set_step(pic_handle *h, uint32_t step);
int pic_set_ceq(pic_handle *h, double ceq);
int pic_set_circuit_state(pic_handle *h, const double *y6);
int pic_set_conv_current(pic_handle *h, double I_conv);
/* Advance only the circuit (and the step counter) for n steps on the device,
 * writing U_E after each step to host `U_out` (may be NULL). */
int pic_circuit_run(pic_handle *h, int n, double *U_out);

/* pic_status -- synchronise and return the accumulated device status bits
 * (PIC_FLAG_*), then clear them. */
int pic_status(pic_handle *h, uint32_t *flags);

/* pic_check -- synchronise and turn the accumulated status bits into a code:
 * PIC_OK when none is set, else the most severe one's -- PIC_EOVERFLOW (a
 * particle was dropped: store or overflow region full), PIC_ETIMEOUT (a
 * bounded device-side wait ran out), PIC_ENAN (non-finite residual),
 * PIC_ENOCONV (iteration cap).  The bits stay set until pic_status reads them.
 * Errors: PIC_ECUDA if the stream reports a CUDA error. */
int pic_check(pic_handle *h);

/* pic_set_spin_limit -- change cfg.spin_limit (clock cycles per grid-barrier
 * wait, 0 = default) for later solves and steps. */
int pic_set_spin_limit(pic_handle *h, int64_t cycles);

/* pic_philox -- fill host `out[4*n]` with Philox4x32-10 outputs computed on
 * the device for counters ctr[4*n] and keys key[2*n] (host arrays); used to
 * check that device and host generators agree bit for bit. */
int pic_philox(pic_handle *h, int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out);

/* pic_enable_timing / pic_step_timing -- while timing is on, pic_step launches
 * the step's kernels directly (no graph) with CUDA events on the handle's
 * stream between phases.  pic_step_timing synchronises and returns the summed
 * device time (ms) of every step since the last call: out[0] bin layout and
 * zeroing, [1] particle kernel, [2] circuit, [3] assembly, [4] field solve,
 * [5] E field, [6] diagnostics. */
int pic_enable_timing(pic_handle *h, int on);
int pic_step_timing(pic_handle *h, double *out7);

/* pic_save -- write the discharge's complete state to the restart file
 * `path`.  The paper's runs (Sec. 2) write their state out and continue over
 * thousands of RF cycles; here that state is one binary file holding the
 * configuration and its arrays, the step counter, the circuit and electrode
 * state with C_eq (Eqs. 5, 8-10), the particle stores exactly as stored
 * (cell-relative positions in the handle's precision, bins and overflow
 * region), phi, the gather field, the deposits, the surface charge, the
 * RF-window sums and the multigrid hierarchy.  A handle restored by pic_load
 * continues bit for bit as this one would: the random numbers are keyed on
 * particle id and step, so no generator state exists.  Not saved: an
 * attached U-Net (attach it again before a PIC_SOLVER_LEARNED step), the
 * timing and keep-warm switches.  The file is in the host's byte order, for
 * the same library build on the same kind of host.  Synchronises.
 * Errors: PIC_EINVAL (NULL argument), PIC_EIO, PIC_ENOMEM, PIC_ECUDA. */
int pic_save(pic_handle *h, const char *path);

/* pic_load -- create a handle on the current device, enqueueing on
 * `cuda_stream`, from a file written by pic_save; *out receives it (the
 * caller destroys it with pic_destroy).  Errors: PIC_EIO (missing, truncated
 * or foreign file, or sizes that do not match its configuration),
 * PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA. */
int pic_load(const char *path, void *cuda_stream, pic_handle **out);

/* pic_pcg_solve_static -- the paper has no counterpart to this entry point;
 * it exists for callers that cannot allocate GPU memory when they need a
 * field solve (an application that owns all device memory through its own
 * pool, a plugin called from a loop that must not wait on the allocator).
 * It solves the same system as the plain solver of pic_field_solve --
 * Jacobi-preconditioned CG in FP64 on the free nodes of
 * sum_b G_ab (phi_a - phi_b) = qrhs_a, warm start from phi, stop at
 * ||r|| <= tol ||b|| -- on arrays the caller owns, and allocates nothing: its
 * work vectors live in one fixed array inside the library, sized for
 * PIC_STATIC_MAX_NODES nodes (about 10 MB), which every GPU that loads the
 * library keeps until the process exits.
 *   nr, nz     grid cells (nodes (nr+1)*(nz+1) <= PIC_STATIC_MAX_NODES, else
 *              PIC_EINVAL)
 *   node_kind  device [(nz+1)*(nr+1)] PIC_NODE_* (Dirichlet where non-zero)
 *   Gr, Gz     device edge conductances, [(nz+1)*nr] radial, [nz*(nr+1)] axial
 *   qrhs       device node charge [(nz+1)*(nr+1)]
 *   phi        device [(nz+1)*(nr+1)], in: Dirichlet values + initial guess,
 *              out: solution
 *   iters, rel_resid  host, may both be NULL: then the call returns once the
 *              work is enqueued on cuda_stream and reports no failure itself
 *              (pic_pcg_static_result reads the outcome later); otherwise it
 *              synchronises the stream and returns PIC_ENOCONV / PIC_ETIMEOUT /
 *              PIC_ENAN on failure.
 * The first call on each device looks up the work array's device address;
 * make that first call before any stream capture.  All calls share the work
 * array and it keeps the last call's contents: calls that can overlap on the
 * GPU (other streams, other host threads on the same device) race on it and
 * must be serialised by the caller. */
#define PIC_STATIC_MAX_NODES 139264
int pic_pcg_solve_static(int32_t nr, int32_t nz, const int8_t *node_kind, const double *Gr, const double *Gz,
                         const double *qrhs, double *phi, double tol, int32_t maxit, void *cuda_stream,
                         int32_t *iters, double *rel_resid);
/* pic_pcg_static_result -- outcome of the last pic_pcg_solve_static call on
 * the current device (a later call overwrites it): synchronises cuda_stream,
 * fills iters and rel_resid (each may be NULL) and returns PIC_OK,
 * PIC_ENOCONV, PIC_ETIMEOUT or PIC_ENAN as that call would have. */
int pic_pcg_static_result(void *cuda_stream, int32_t *iters, double *rel_resid);

/* ---- learned field-solve preconditioner (U-Net) -------------------------
 * A 4-level U-Net (32 base channels, BF16 weights and activations, FP32
 * accumulation on the tensor cores) mapping (rho~, chi, boundary-voltage
 * mask) on an H x W node grid to phi; used as the initial guess and the
 * preconditioner of the field solve.  H, W multiples of 8, H*W <= 2^24.
 * Tensors passed in are device FP32 arrays in the caller's memory; the
 * network owns its weights, activations and gradient buffers. */
typedef struct pic_unet pic_unet;
int pic_unet_create(int H, int W, void *cuda_stream, pic_unet **out);
void pic_unet_destroy(pic_unet *u);
/* number of parameters; order: per conv (14) W[cout][9][cin] then bias[cout],
 * then the 1x1 output conv's 32 weights and its bias */
int pic_unet_param_count(const pic_unet *u, int64_t *n);
int pic_unet_set_params(pic_unet *u, const float *host, int64_t n);
int pic_unet_get_params(pic_unet *u, float *host, int64_t n);
/* accumulated parameter gradients, same order as the parameters */
int pic_unet_get_grads(pic_unet *u, float *host, int64_t n);
int pic_unet_zero_grads(pic_unet *u);
/* in: device [3][H*W] (rho~, chi, mask, channel-major); out: device [H*W] */
int pic_unet_forward(pic_unet *u, const float *in, float *out);
/* backward of the last forward for dLoss/dout (device [H*W]); adds to the gradients */
int pic_unet_backward(pic_unet *u, const float *gout);
/* Relative L2 loss of the last forward's output o against target t (device
 * FP32 [H*W]) over the pixels where in3's channel 2 (the Dirichlet mask) is 0:
 * L = sum (o - t)^2 / sum t^2.  Adds dL/do's backward to the gradients and L
 * to *loss (device FP32, may be NULL).  Asynchronous. */
int pic_unet_loss_backward(pic_unet *u, const float *in3, const float *target, float *loss);
/* one Adam step (t = step number from 1) on the accumulated gradients */
int pic_unet_adam(pic_unet *u, float lr, float beta1, float beta2, float eps, int t);
/* synchronise; *err = 1 if a bounded tensor-core wait timed out since the last call */
int pic_unet_status(pic_unet *u, int *err);
/* One tensor-core convolution on caller-owned device tensors (dense NHWC BF16,
 * H x W pixels, Cin and Cout multiples of 16), for kernel tests:
 *   op 0: out = FP32 [H*W][Cout] conv3x3(in, w), w = BF16 [Cout][9][Cin]
 *   op 1: out = BF16 [H*W][Cout] ReLU(conv3x3(in, w) + bias)
 *   op 2: out = FP32 [9*Cin][Cout] weight gradient: sum_p in[p + off(tap)][cin] w[p][cout]
 *         (here `w` is the output gradient, BF16 [H*W][Cout]; Cout <= 256)
 * Ops 0 and 1 run the TMA-fed kernel when W is a multiple of 8 and some tiling
 * fits, else the cp.async gather kernel (Cout <= 256).
 * Synchronises the stream.  Errors: PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ETIMEOUT. */
int pic_conv3x3_op(int op, int H, int W, const void *in, int Cin, const void *w, const float *bias, void *out,
                   int Cout, void *cuda_stream);
/* As pic_conv3x3_op with a chosen tiling for ops 0 and 1: tile_n = output
 * channels per CTA (32, 64, 128, 256; must divide Cout), tile_mma = 128-pixel
 * accumulators per CTA (1, 2, 4, 8); 0 = automatic; tile_n = -1 forces the
 * gather kernel.  PIC_EINVAL if the forced tiling does not fit. */
int pic_conv3x3_op_ex(int op, int H, int W, const void *in, int Cin, const void *w, const float *bias, void *out,
                      int Cout, int tile_n, int tile_mma, void *cuda_stream);

/* ---- learned field solve -------------------------------------------------
 * pic_attach_unet -- use network u (created with H = nz, W = nr; it covers
 * nodes i < nr, j < nz) as the preconditioner of PIC_SOLVER_LEARNED solves:
 * z = s U(D^-1 r / s, chi, Dirichlet mask) with D the operator diagonal and s
 * the rms of D^-1 r over the covered free nodes, followed by `smooth` (0..8)
 * damped Jacobi steps z += (2/3) D^-1 (r - A z); flexible CG with one stored
 * direction, at most `maxit` network applications per solve, then the solver
 * `finish` (PIC_SOLVER_PLAIN, _MIXED or _MG) confirms the FP64 residual
 * and finishes the solve from the learned iterate when needed.  The first
 * application on the warm start's residual is the learned initial-guess
 * correction.  u = NULL detaches.  The handle does not own u; keep it alive
 * while attached.  Builds one CUDA graph with a device-side loop.
 * Errors: PIC_EINVAL (grid mismatch), PIC_ENOMEM, PIC_ECUDA. */
int pic_attach_unet(pic_handle *h, pic_unet *u, int maxit, int smooth, int finish);
/* pic_set_solver -- change the solver of later steps (PIC_SOLVER_*; LEARNED
 * needs an attached network when the step runs). */
int pic_set_solver(pic_handle *h, int solver);
/* pic_keep_warm -- keep a copy of each solve's warm start (needed by
 * pic_learned_pair with the plain and mixed solvers). */
int pic_keep_warm(pic_handle *h, int on);
/* pic_learned_snapshot -- in later learned solves, keep the iterate after k
 * network applications (k = 0: off) for pic_learned_pair(source 1). */
int pic_learned_snapshot(pic_handle *h, int k);
/* pic_learned_pair -- a training pair of the last solve, from a start
 * phi_w (source 0: the solve's warm start; source 1: the learned iterate kept by
 * pic_learned_snapshot, valid when that solve made at least k applications) and
 * the solution phi: r0 = b - A phi_w, delta = phi - phi_w = A^-1 r0, and with
 * s = rms of D^-1 r0 over the covered free nodes:
 *   in3    (device FP32 [3][nz*nr]) = D^-1 r0 / s, chi, Dirichlet mask,
 *   target (device FP32 [nz*nr])    = delta / s  (0 at Dirichlet nodes);
 * *scale = s.  Synchronises. */
int pic_learned_pair(pic_handle *h, int source, float *in3, float *target, double *scale);
/* pic_learned_stats -- last learned solve: [0] network applications,
 * [1] its final relative residual, [2] its status (0 converged, -4 hit maxit,
 * -7 non-finite: restarted from the warm start), [3] iterations the plain PCG
 * added afterwards (0 when the learned solve met the tolerance). */
int pic_learned_stats(pic_handle *h, double *out4);

/* ---- batched sweep ----------------------------------------------------------
 * pic_batch_create -- step n independent discharges (a parameter sweep with
 * uneven grids and particle counts) together.  Each step is one CUDA graph
 * launch holding one independent chain per discharge: particle phase, circuit
 * and assembly, then its field solve on one thread-block cluster of 1-8 CTAs
 * by grid size (the PIC_SOLVER_MG method -- multigrid-preconditioned FP32 CG
 * inside FP64 residual refinement to the discharge's pcg_tol -- whatever its
 * cfg.solver, with hardware cluster barriers instead of a grid barrier, so the
 * chains never wait on one another), then its E field and diagnostics.  The
 * handles must share a device and be at the same buffer
 * parity (stepped the same number of times); they stay owned by the caller and
 * must outlive the batch.  Unstarted handles are started.
 * pic_batch_step advances all of them by nsteps (asynchronous, except at RF
 * window ends, which run per handle as in pic_step); pic_batch_sync waits.
 * Each handle's own stream waits for the batch's steps, so a later call on a
 * handle (pic_diag, pic_diag_async, pic_step) sees their result.
 * Errors: PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA. */
typedef struct pic_batch pic_batch;
int pic_batch_create(pic_handle *const *hs, int n, pic_batch **out);
int pic_batch_step(pic_batch *b, int nsteps);
int pic_batch_sync(pic_batch *b);
void pic_batch_destroy(pic_batch *b);

const char *pic_strerror(int code);
void pic_destroy(pic_handle *h);

#ifdef __cplusplus
}
#endif
#endif
