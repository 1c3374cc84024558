/*
 * pic_oracle.h -- private header of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA path; only
 * tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm
 * may build, load or call it.  It shares no code, header, table or constant
 * with the CUDA library: this header is included by oracle/pic_oracle.c alone.
 *
 * Method: 2D axisymmetric (r-z) electrostatic direct-implicit PIC/MCC of a
 * capacitively coupled argon discharge, coupled to an external circuit through
 * the electrode's equivalent capacitance (arXiv:2310.04957, Sec. 2,
 * Eqs. 1 and 5-10).  Every detail the paper leaves open follows the readings
 * listed in the repository's design notes; each function cites what it follows.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#define ORC_FREE 0
#define ORC_POWERED 1
#define ORC_GROUNDED 2
#define ORC_DRIVEN 3   /* first of up to three voltage-driven electrodes: 3, 4, 5 */
#define ORC_MAX_DRIVE 3

#define ORC_FIELD_DIRECT 0  /* one solve with every electrode at its voltage   */
#define ORC_FIELD_VAHEDI 1  /* phi = phi_P + sum_i U_Ei phi_Li (Eqs. 2-4)      */

#define ORC_CELL_PLASMA 0
#define ORC_CELL_POWERED 1
#define ORC_CELL_GROUNDED 2
#define ORC_CELL_DIELECTRIC 3

#define ORC_CIRCUIT_DIRECT 0
#define ORC_CIRCUIT_RLC 1
#define ORC_CIRCUIT_IMN 2

/* Everything the oracle needs to define one discharge.  Arrays are copied. */
typedef struct orc_setup {
  int32_t nr, nz;            /* cells in r and z; nodes are (nr+1)*(nz+1)       */
  double dr, dz;             /* cell sizes (m)                                   */
  const int8_t *node_kind;   /* [(nz+1)*(nr+1)], index j*(nr+1)+i: ORC_FREE/... */
  const int8_t *cell_kind;   /* [nz*nr], index j*nr+i: ORC_CELL_*                */
  const double *cell_eps;    /* [nz*nr] relative permittivity per cell           */
  double dt;                 /* time step (s)                                    */
  double n_gas, T_gas, m_gas;/* neutral density (m^-3), temperature (K), mass  */
  double q[2], m[2], w[2];   /* species 0 = electrons, 1 = ions: charge, mass, weight */
  int32_t n_xs;              /* cross-section table length                       */
  const double *xs_energy;   /* [n_xs] eV, log-spaced                            */
  const double *xs_sigma;    /* [5*n_xs] m^2: e-elastic, e-excitation, e-ionization, i-isotropic, i-charge-exchange */
  double thr_ex, thr_iz;     /* inelastic thresholds (eV)                        */
  double B_ej;               /* ejected-electron energy parameter (eV)           */
  int32_t circuit;           /* ORC_CIRCUIT_*                                    */
  double circ[8];            /* RLC: Rb, Lb, Cb.  IMN: Rs, Cm1, Lm, Cm2, Rm, Cstray, Rstray, Lstray */
  double V_src, f_src, phase_src; /* source amplitude (V), frequency (Hz), phase (rad) */
  int32_t n_sub;             /* trapezoidal substeps per dt for the circuit      */
  int32_t steps_per_rf;      /* diagnostic window length (steps)                 */
  double pcg_tol;            /* relative residual target                         */
  int32_t pcg_maxit;
  int32_t ceq_refresh;       /* recompute C_eq with chi once per window           */
  uint32_t seed;             /* fourth Philox counter word                       */
  int64_t capacity[2];       /* particle capacity per species                    */
  int32_t split_cells;       /* particle splitting in the first split_cells radial
                                cells (0: off); see split_target() */
  int32_t n_drive;           /* voltage-driven electrodes (node kinds 3 .. 2+n_drive) */
  double drive_V[ORC_MAX_DRIVE], drive_f[ORC_MAX_DRIVE], drive_phase[ORC_MAX_DRIVE];
                             /* U_k(t) = V sin(2 pi f t + phase)                  */
  int32_t field_mode;        /* ORC_FIELD_DIRECT or ORC_FIELD_VAHEDI              */
} orc_setup;

typedef struct orc_sim orc_sim;

/* Status codes (negative on failure). */
#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ENOCONV -4
#define ORC_EOVERFLOW -6

#endif
