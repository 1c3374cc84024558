/*
 * pic_oracle.c -- plain FP64 CPU oracle of the implicit r-z PIC/MCC step.
 *
 * TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm are the only callers.  The product path never
 * loads this file.  It shares no code with the CUDA library.
 *
 * What it computes (arXiv:2310.04957, Sec. 2):
 *   - the implicit Poisson equation of Eq. 1, div[(1+chi) eps grad phi] = -rho~,
 *     on a node-centred axisymmetric finite-volume grid, metals as Dirichlet
 *     nodes, dielectrics through a per-cell relative permittivity;
 *   - the electrode potential U_E = Q_E / C_eq (Eq. 5), C_eq from the
 *     electrostatic energy of the unit-voltage solution (Eqs. 6-7), and the
 *     electrode charge balance dQ_E/dt = I_ccp + I_conv (Eq. 8) integrated
 *     together with circuit I (Eq. 9) or circuit II (Eq. 10);
 *   - the particle step: direct-implicit (D1) push in r-z with the cylindrical
 *     rotation of (v_r, v_theta), null-collision Monte Carlo collisions of
 *     electrons and Ar+ with argon (Sec. 2, Vahedi's null-collision method),
 *     deposition of charge and of the implicit susceptibility chi.
 * The paper is silent on the push, weighting, discretisation, kinematics and
 * random numbers; each such step below follows one stated reading.
 *
 * Floating point: every quantity is FP64, IEEE, no contraction (the build
 * passes -ffp-contract=off) so that x86 and Arm hosts agree.
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* Physical constants (SI, CODATA 2018 exact / recommended values). */
static const double QE_C = 1.602176634e-19;     /* elementary charge, C */
static const double EPS0 = 8.8541878128e-12;    /* vacuum permittivity, F/m */
static const double KB = 1.380649e-23;          /* Boltzmann constant, J/K */
static const double PI = 3.141592653589793238462643383279;
static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3): ten rounds of  */
/* two 32x32->64 multiplications whose halves are mixed with the other two   */
/* words and the round key; the key is bumped by two Weyl constants between  */
/* rounds.                                                                   */
/* ------------------------------------------------------------------------ */
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u; /* golden ratio */
      k1 += 0xBB67AE85u; /* sqrt(3) - 1 */
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in [0,1) from the top 24 bits: exactly representable in FP32 and FP64. */
static double unif(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* Random numbers of one particle in one step: key = particle id, counter =
 * (step, call, species, seed). */
static void draw(uint64_t id, uint32_t step, uint32_t call, uint32_t species, uint32_t seed, double u[4]) {
  uint32_t ctr[4] = {step, call, species, seed};
  uint32_t key[2] = {(uint32_t)id, (uint32_t)(id >> 32)};
  uint32_t x[4];
  philox4x32_10(ctr, key, x);
  for (int k = 0; k < 4; ++k) u[k] = unif(x[k]);
}

/* Box-Muller: two standard normals from two uniforms; the logarithm takes 1-u in (0,1]. */
static void box_muller(double ua, double ub, double *na, double *nb) {
  double rad = sqrt(-2.0 * log(1.0 - ua));
  *na = rad * cos(TWO_PI * ub);
  *nb = rad * sin(TWO_PI * ub);
}

/* ------------------------------------------------------------------------ */
/* State                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t n, cap;
  double *r, *z, *vr, *vt, *vz, *ar, *at, *az; /* x~, v, a-bar */
  double *w;                                   /* weight ratio: macro weight w_p = w * cfg.w[species] */
  uint64_t *id;
  int32_t *cell;
} orc_species;

typedef struct {
  double r, z, vr, vt, vz, ar, at, az;
  double w;
  uint64_t id;
} orc_particle;

struct orc_sim {
  orc_setup cfg;
  int nn;            /* nodes */
  int nc;            /* cells */
  int8_t *node_kind, *cell_kind;
  double *cell_eps;
  double *xs_energy, *xs_sigma;
  double *vnode;     /* plasma-restricted node volume */
  double *Gr, *Gz;   /* edge conductances of the current operator */
  double *dep[2];    /* deposited counts per species */
  double *sigma;     /* surface charge on free boundary nodes */
  double *chi, *qrhs, *phi, *Er, *Ez;
  /* Vahedi decomposition (Eqs. 2-4): phi_P of the last solve (its warm start)
   * and the unit-voltage Laplace solutions of the powered electrode (0) and of
   * the driven electrodes (1..n_drive) */
  double *phiP, *phiL[1 + ORC_MAX_DRIVE];
  double t_field;    /* time of the field being assembled and solved */
  double numax[2], pcoll[2];
  orc_species sp[2];
  /* births created during one particle phase */
  orc_particle *born[2];
  int64_t n_born[2], cap_born[2];
  /* second halves of particles split during one particle phase */
  orc_particle *split[2];
  int64_t n_split[2], cap_split[2];
  /* per-step tallies: [species][0 powered,1 grounded,2 surface] */
  double abs_q[2][3];
  int64_t abs_n[2][3];
  int64_t coll[2][3];    /* collisions per species per process */
  /* circuit */
  double y[6];
  double ceq, U_E, Q_E, I_conv, I_ccp;
  uint32_t step;
  int pcg_iters; double pcg_relres; int pcg_status;
  double ceq_gauss;
  /* diagnostics */
  double *dens_sum[2], *dens_avg[2];
  double ion_q_sum[3], ion_cur_avg[3];
  double dft_re, dft_im, i1_re, i1_im;
  int win_count, windows_done;
  /* circuit post-processing over the window (Sec. 3, Eqs. 11-14): first-harmonic
   * DFT sums of five waveforms (U_s, source-loop current I_1, matching-network
   * input voltage U_in, U_E = U_ccp, I_ccp) and sums of the five powers U_s I_1,
   * R_s I_1^2, series-element loss, stray-branch loss, U_ccp I_ccp, U_in I_1 */
  double cw_re[5], cw_im[5], cp_sum[6], cdc[2];
  double circ_out[18];
  /* decision margins (test instrumentation, see orc_trace): [0] random-number
   * and energy thresholds, relative; [1] position tests, cell units; [2]
   * conditioning of the predictor's rotation angle */
  int trace;
  double margin[3];
};

static int nidx(const orc_sim *s, int i, int j) { return j * (s->cfg.nr + 1) + i; }

/* ------------------------------------------------------------------------ */
/* Decision margins.  Every branch of a particle's step is decided by        */
/* comparing a computed quantity with a threshold: a uniform with P_null, a  */
/* scaled uniform with the cumulative collision frequencies, an energy with  */
/* an inelastic threshold, a position with a cell face across which the      */
/* particle leaves the plasma, a radius with the axis.  A second             */
/* implementation that rounds differently (FP32) can take the other branch   */
/* only where the quantity lies within its own rounding of the threshold.    */
/* When tracing is on the step records the smallest such distance; it never  */
/* changes what the step computes.                                           */
/* ------------------------------------------------------------------------ */
static void note_margin(orc_sim *s, int kind, double v) {
  if (s->trace && v < s->margin[kind]) s->margin[kind] = v;
}

/* Plasma membership of cell (i,j); outside the domain nothing is plasma,
 * except across the axis, which is a symmetry line, not a boundary. */
static int member(const orc_sim *s, int i, int j) {
  if (i < 0) i = 0;
  if (i >= s->cfg.nr || j < 0 || j >= s->cfg.nz) return 0;
  return s->cell_kind[j * s->cfg.nr + i] == ORC_CELL_PLASMA;
}

/* Distance, in cell units, from (r,z) to the nearest cell face (or corner)
 * across which plasma membership changes. */
static double face_margin(const orc_sim *s, double r, double z) {
  double x = r / s->cfg.dr, y = z / s->cfg.dz;
  int i = (int)floor(x), j = (int)floor(y);
  int in = member(s, i, j);
  double lo_x = x - i, hi_x = i + 1 - x, lo_y = y - j, hi_y = j + 1 - y;
  double m = 1e300;
  if (member(s, i - 1, j) != in && lo_x < m) m = lo_x;
  if (member(s, i + 1, j) != in && hi_x < m) m = hi_x;
  if (member(s, i, j - 1) != in && lo_y < m) m = lo_y;
  if (member(s, i, j + 1) != in && hi_y < m) m = hi_y;
  for (int di = -1; di <= 1; di += 2)
    for (int dj = -1; dj <= 1; dj += 2)
      if (member(s, i + di, j + dj) != in) {
        double dx = di < 0 ? lo_x : hi_x, dy = dj < 0 ? lo_y : hi_y;
        double d = dx > dy ? dx : dy;
        if (d < m) m = d;
      }
  return m;
}

/* Relative distance of x from threshold t (t > 0). */
static double rel_gap(double x, double t) { return fabs(x - t) / t; }

/* ------------------------------------------------------------------------ */
/* Cross sections: linear interpolation in E between bracketing table nodes  */
/* found by bisection; values clamped outside the table; inelastic processes */
/* vanish below threshold (Sec. 2, null-collision MCC; table reading).       */
/* ------------------------------------------------------------------------ */
static double xs_lookup(const orc_sim *s, int proc, double E) {
  int n = s->cfg.n_xs;
  const double *Et = s->xs_energy;
  const double *sg = s->xs_sigma + (size_t)proc * n;
  if (proc == 1 && E < s->cfg.thr_ex) return 0.0;
  if (proc == 2 && E < s->cfg.thr_iz) return 0.0;
  if (E <= Et[0]) return sg[0];
  if (E >= Et[n - 1]) return sg[n - 1];
  int lo = 0, hi = n - 1; /* Et[lo] <= E < Et[hi] */
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (Et[mid] <= E) lo = mid; else hi = mid;
  }
  double f = (E - Et[lo]) / (Et[lo + 1] - Et[lo]);
  return sg[lo] + f * (sg[lo + 1] - sg[lo]);
}

/* nu_max = n_g * max over table intervals of (larger node sigma_T) x (speed at
 * the interval's upper energy): an upper bound of n_g sigma_T(E) v(E) for
 * every E in the table (the null-collision bound, Sec. 2). */
static void compute_numax(orc_sim *s) {
  int n = s->cfg.n_xs;
  for (int spc = 0; spc < 2; ++spc) {
    double mass = spc == 0 ? s->cfg.m[0] : s->cfg.m_gas;
    int p0 = spc == 0 ? 0 : 3, p1 = spc == 0 ? 3 : 5;
    double best = 0.0;
    for (int k = 0; k + 1 < n; ++k) {
      double sa = 0.0, sb = 0.0;
      for (int p = p0; p < p1; ++p) {
        sa += s->xs_sigma[(size_t)p * n + k];
        sb += s->xs_sigma[(size_t)p * n + k + 1];
      }
      double smax = sa > sb ? sa : sb;
      double v = sqrt(2.0 * s->xs_energy[k + 1] * QE_C / mass);
      double nu = s->cfg.n_gas * smax * v;
      if (nu > best) best = nu;
    }
    s->numax[spc] = best;
    s->pcoll[spc] = 1.0 - exp(-best * s->cfg.dt);
  }
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */
/* Cell of a point and whether it lies in the plasma region. */
static int inside_plasma(const orc_sim *s, double r, double z, int *ci, int *cj) {
  double R = s->cfg.nr * s->cfg.dr, Z = s->cfg.nz * s->cfg.dz;
  if (!(r < R) || !(z >= 0.0) || !(z < Z) || !(r >= 0.0)) return 0;
  int i = (int)floor(r / s->cfg.dr);
  int j = (int)floor(z / s->cfg.dz);
  if (i > s->cfg.nr - 1) i = s->cfg.nr - 1;
  if (j > s->cfg.nz - 1) j = s->cfg.nz - 1;
  *ci = i; *cj = j;
  return s->cell_kind[j * s->cfg.nr + i] == ORC_CELL_PLASMA;
}

/* Weights of the four nodes of cell (i,j) for a point (r,z): linear in z,
 * by annulus area in r, w_{i+1} = (r^2 - r_i^2)/(r_{i+1}^2 - r_i^2)
 * ("volume weighting"; the same weights gather and deposit). */
static void node_weights(const orc_sim *s, double r, double z, int i, int j, double w[4]) {
  double ri = i * s->cfg.dr, ri1 = (i + 1) * s->cfg.dr;
  double wr1 = (r * r - ri * ri) / (ri1 * ri1 - ri * ri);
  double wr0 = 1.0 - wr1;
  double wz1 = (z - j * s->cfg.dz) / s->cfg.dz;
  double wz0 = 1.0 - wz1;
  w[0] = wr0 * wz0; /* (i,   j)   */
  w[1] = wr1 * wz0; /* (i+1, j)   */
  w[2] = wr0 * wz1; /* (i,   j+1) */
  w[3] = wr1 * wz1; /* (i+1, j+1) */
}

/* An absorbed particle's charge goes to the node nearest to where it left
 * the plasma (position clamped into the domain): a powered node adds to the
 * electrode's convective charge (Eq. 8), a grounded node is only counted, a
 * free node (dielectric surface) keeps it as surface charge. */
static void credit(orc_sim *s, int spc, double r, double z, double w) {
  double R = s->cfg.nr * s->cfg.dr, Z = s->cfg.nz * s->cfg.dz;
  double rc = r < 0 ? 0 : (r > R ? R : r);
  double zc = z < 0 ? 0 : (z > Z ? Z : z);
  int i = (int)floor(rc / s->cfg.dr + 0.5);
  int j = (int)floor(zc / s->cfg.dz + 0.5);
  if (i > s->cfg.nr) i = s->cfg.nr;
  if (j > s->cfg.nz) j = s->cfg.nz;
  int node = nidx(s, i, j);
  double qw = s->cfg.q[spc] * s->cfg.w[spc] * w;
  int kind = s->node_kind[node];
  if (kind == ORC_POWERED) { s->abs_q[spc][0] += qw; s->abs_n[spc][0] += 1; }
  else if (kind != ORC_FREE) { s->abs_q[spc][1] += qw; s->abs_n[spc][1] += 1; } /* grounded or driven metal */
  else { s->sigma[node] += qw; s->abs_q[spc][2] += qw; s->abs_n[spc][2] += 1; }
}

/* Node counts of a particle of weight ratio pw: its four node weights times pw. */
static void deposit(orc_sim *s, int spc, double r, double z, int i, int j, double pw) {
  double w[4];
  node_weights(s, r, z, i, j, w);
  double *d = s->dep[spc];
  d[nidx(s, i, j)] += pw * w[0];
  d[nidx(s, i + 1, j)] += pw * w[1];
  d[nidx(s, i, j + 1)] += pw * w[2];
  d[nidx(s, i + 1, j + 1)] += pw * w[3];
}

/* ------------------------------------------------------------------------ */
/* Collision kinematics (Vahedi & Surendra 1995, the method cited in Sec. 2) */
/* ------------------------------------------------------------------------ */
/* Scattering-angle cosine for an electron of energy E (eV):
 * cos chi = (2 + E - 2 (1+E)^R) / E, whose E -> 0 limit is 1 - 2R. */
static double scatter_cos(double E, double R) {
  double c;
  if (E < 1e-12) c = 1.0 - 2.0 * R;
  else c = (2.0 + E - 2.0 * pow(1.0 + E, R)) / E;
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  return c;
}

/* Turn unit vector (cx,cy,cz) by polar angle chi (cosine cc) and azimuth phi
 * about itself, in the orthonormal frame {c, c x z / |c x z|, c x (c x z)...}. */
static void turn(double c[3], double cc, double phi) {
  double sc = sqrt(1.0 - cc * cc > 0 ? 1.0 - cc * cc : 0.0);
  double cp = cos(phi), sp = sin(phi);
  double st = sqrt(c[0] * c[0] + c[1] * c[1]);
  double o[3];
  if (st > 1e-12) {
    o[0] = c[0] * cc + sc / st * (c[0] * c[2] * cp + c[1] * sp);
    o[1] = c[1] * cc + sc / st * (c[1] * c[2] * cp - c[0] * sp);
    o[2] = c[2] * cc - sc * st * cp;
  } else {
    double sg = c[2] >= 0 ? 1.0 : -1.0;
    o[0] = sc * cp * sg;
    o[1] = -sc * sp;
    o[2] = cc * sg;
  }
  c[0] = o[0]; c[1] = o[1]; c[2] = o[2];
}

static void push_birth(orc_sim *s, int spc, const orc_particle *p) {
  if (s->n_born[spc] == s->cap_born[spc]) {
    int64_t nc = s->cap_born[spc] ? 2 * s->cap_born[spc] : 1024;
    orc_particle *nb = (orc_particle *)realloc(s->born[spc], (size_t)nc * sizeof(orc_particle));
    if (!nb) { fprintf(stderr, "oracle: out of memory for births\n"); abort(); }
    s->born[spc] = nb; s->cap_born[spc] = nc;
  }
  s->born[spc][s->n_born[spc]++] = *p;
}

/* Identifier of the k-th particle born from parent `id` in `step`: 64 Philox
 * bits with the top bit set (initial particles have ids below 2^63). */
static uint64_t child_id(uint64_t id, uint32_t step, uint32_t k, uint32_t seed) {
  uint32_t ctr[4] = {step, 0xB1B1u, k, seed};
  uint32_t key[2] = {(uint32_t)id, (uint32_t)(id >> 32)};
  uint32_t x[4];
  philox4x32_10(ctr, key, x);
  return ((uint64_t)x[0] | ((uint64_t)x[1] << 32)) | (1ull << 63);
}

/* Electron null-collision test and collision (elastic, 11.5 eV excitation,
 * 15.76 eV ionization).  Random draws: call 0 = (candidate, process, angle,
 * azimuth); ionization adds call 1 (angles of both electrons) and call 2 (the
 * new ion's Maxwellian velocity). */
static void mcc_electron(orc_sim *s, orc_particle *p, double r, double z) {
  const orc_setup *c = &s->cfg;
  double u[4];
  draw(p->id, s->step, 0, 0, c->seed, u);
  note_margin(s, 0, rel_gap(u[0], s->pcoll[0]));
  if (!(u[0] < s->pcoll[0])) return;
  double v2 = p->vr * p->vr + p->vt * p->vt + p->vz * p->vz;
  double speed = sqrt(v2);
  double E = 0.5 * c->m[0] * v2 / QE_C;
  double nu_el = c->n_gas * xs_lookup(s, 0, E) * speed;
  double nu_ex = c->n_gas * xs_lookup(s, 1, E) * speed;
  double nu_iz = c->n_gas * xs_lookup(s, 2, E) * speed;
  double x = u[1] * s->numax[0];
  if (s->trace) {
    note_margin(s, 0, rel_gap(E, c->thr_ex));
    note_margin(s, 0, rel_gap(E, c->thr_iz));
    double cum[3] = {nu_el, nu_el + nu_ex, nu_el + nu_ex + nu_iz};
    for (int k = 0; k < 3; ++k)
      if (cum[k] > 0.0) note_margin(s, 0, rel_gap(x, cum[k]));
  }
  if (speed <= 0.0) return;
  double dir[3] = {p->vr / speed, p->vt / speed, p->vz / speed};
  if (x < nu_el) {
    double cc = scatter_cos(E, u[2]);
    double En = E * (1.0 - 2.0 * c->m[0] / c->m_gas * (1.0 - cc));
    turn(dir, cc, TWO_PI * u[3]);
    double sp = sqrt(2.0 * En * QE_C / c->m[0]);
    p->vr = sp * dir[0]; p->vt = sp * dir[1]; p->vz = sp * dir[2];
    s->coll[0][0]++;
  } else if (x < nu_el + nu_ex) {
    double En = E - c->thr_ex;
    double cc = scatter_cos(En, u[2]);
    turn(dir, cc, TWO_PI * u[3]);
    double sp = sqrt(2.0 * En * QE_C / c->m[0]);
    p->vr = sp * dir[0]; p->vt = sp * dir[1]; p->vz = sp * dir[2];
    s->coll[0][1]++;
  } else if (x < nu_el + nu_ex + nu_iz) {
    double Eex = E - c->thr_iz;
    double Eej = c->B_ej * tan(u[2] * atan(Eex / (2.0 * c->B_ej)));
    double Esc = Eex - Eej;
    if (Esc < 0.0) Esc = 0.0;
    double u1[4], u2[4];
    draw(p->id, s->step, 1, 0, c->seed, u1);
    draw(p->id, s->step, 2, 0, c->seed, u2);
    double dsc[3] = {dir[0], dir[1], dir[2]};
    double dej[3] = {dir[0], dir[1], dir[2]};
    turn(dsc, scatter_cos(Esc, u1[0]), TWO_PI * u1[1]);
    turn(dej, scatter_cos(Eej, u1[2]), TWO_PI * u1[3]);
    double ssc = sqrt(2.0 * Esc * QE_C / c->m[0]);
    double sej = sqrt(2.0 * Eej * QE_C / c->m[0]);
    p->vr = ssc * dsc[0]; p->vt = ssc * dsc[1]; p->vz = ssc * dsc[2];
    orc_particle e = {r, z, sej * dej[0], sej * dej[1], sej * dej[2], 0, 0, 0, p->w,
                      child_id(p->id, s->step, 0, c->seed)};
    double n0, n1, n2, n3;
    box_muller(u2[0], u2[1], &n0, &n1);
    box_muller(u2[2], u2[3], &n2, &n3);
    double vth = sqrt(KB * c->T_gas / c->m_gas);
    orc_particle ion = {r, z, vth * n0, vth * n1, vth * n2, 0, 0, 0, p->w,
                        child_id(p->id, s->step, 1, c->seed)};
    push_birth(s, 0, &e);
    push_birth(s, 1, &ion);
    s->coll[0][2]++;
  }
}

/* Ion null-collision test against a neutral drawn from the 300 K Maxwellian
 * (Sec. 2): relative velocity g, table energy 1/2 M g^2; isotropic scattering
 * in the centre-of-mass frame or charge exchange (ion takes the neutral's
 * velocity).  Draws: call 0 = (candidate, process, cos theta, azimuth),
 * call 1 = neutral velocity normals. */
static void mcc_ion(orc_sim *s, orc_particle *p) {
  const orc_setup *c = &s->cfg;
  double u[4], u1[4];
  draw(p->id, s->step, 0, 1, c->seed, u);
  note_margin(s, 0, rel_gap(u[0], s->pcoll[1]));
  if (!(u[0] < s->pcoll[1])) return;
  draw(p->id, s->step, 1, 1, c->seed, u1);
  double n0, n1, n2, n3;
  box_muller(u1[0], u1[1], &n0, &n1);
  box_muller(u1[2], u1[3], &n2, &n3);
  double vth = sqrt(KB * c->T_gas / c->m_gas);
  double vn[3] = {vth * n0, vth * n1, vth * n2};
  double g[3] = {p->vr - vn[0], p->vt - vn[1], p->vz - vn[2]};
  double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  double gm = sqrt(g2);
  double eps = 0.5 * c->m_gas * g2 / QE_C;
  double nu_iso = c->n_gas * xs_lookup(s, 3, eps) * gm;
  double nu_cx = c->n_gas * xs_lookup(s, 4, eps) * gm;
  double x = u[1] * s->numax[1];
  if (s->trace) {
    if (nu_iso > 0.0) note_margin(s, 0, rel_gap(x, nu_iso));
    if (nu_iso + nu_cx > 0.0) note_margin(s, 0, rel_gap(x, nu_iso + nu_cx));
  }
  if (x < nu_iso) {
    double mi = c->m[1], M = c->m_gas;
    double ct = 1.0 - 2.0 * u[2];
    double st = sqrt(1.0 - ct * ct > 0 ? 1.0 - ct * ct : 0.0);
    double ph = TWO_PI * u[3];
    double gp[3] = {gm * st * cos(ph), gm * st * sin(ph), gm * ct};
    double vcm[3];
    for (int k = 0; k < 3; ++k) vcm[k] = (mi * (k == 0 ? p->vr : k == 1 ? p->vt : p->vz) + M * vn[k]) / (mi + M);
    p->vr = vcm[0] + M / (mi + M) * gp[0];
    p->vt = vcm[1] + M / (mi + M) * gp[1];
    p->vz = vcm[2] + M / (mi + M) * gp[2];
    s->coll[1][0]++;
  } else if (x < nu_iso + nu_cx) {
    p->vr = vn[0]; p->vt = vn[1]; p->vz = vn[2];
    s->coll[1][1]++;
  }
}

/* Predictor of the D1 scheme and cylindrical rotation: u = v + dt/2 a-bar;
 * the particle moves by dt*u in its local Cartesian frame (x along r, y along
 * theta); the new radius is |(r + dt u_r, dt u_theta)| and (v_r, v_theta),
 * (a_r, a_theta) are turned by the swept angle alpha. */
static void predict(orc_sim *s, orc_particle *p, double r, double z) {
  double dt = s->cfg.dt;
  double ur = p->vr + 0.5 * dt * p->ar;
  double ut = p->vt + 0.5 * dt * p->at;
  double uz = p->vz + 0.5 * dt * p->az;
  double X = r + dt * ur, Y = dt * ut;
  double rn = sqrt(X * X + Y * Y);
  /* the swept angle's sensitivity to a position error grows as 1/rn */
  note_margin(s, 2, rn / (s->cfg.dr + dt * sqrt(ur * ur + ut * ut)));
  double ca = 1.0, sa = 0.0;
  if (rn > 0.0) { ca = X / rn; sa = Y / rn; }
  double vr = ca * p->vr + sa * p->vt, vt = -sa * p->vr + ca * p->vt;
  double ar = ca * p->ar + sa * p->at, at = -sa * p->ar + ca * p->at;
  p->vr = vr; p->vt = vt; p->ar = ar; p->at = at;
  p->r = rn;
  p->z = z + dt * uz;
}

/* Particle splitting near the axis (Sec. 2: unequal weights make the few
 * particles of the small axial cells heavy and noisy; splitting restores their
 * number).  Radial cell i has the target weight ratio (2i+1)/(2 i_s + 1),
 * proportional to its volume, within the first i_s = split_cells cells and 1
 * beyond; a particle heavier than twice the target of the cell it enters splits
 * into two halves.  The second half has the id split_id(parent, step). */
static double split_target(const orc_sim *s, int i) {
  int is = s->cfg.split_cells;
  if (is <= 0 || i >= is) return 1.0;
  return (2.0 * i + 1.0) / (2.0 * is + 1.0);
}

static uint64_t split_id(uint64_t id, uint32_t step, uint32_t seed) {
  uint32_t ctr[4] = {step, 0x5B17u, 0u, seed};
  uint32_t key[2] = {(uint32_t)id, (uint32_t)(id >> 32)};
  uint32_t x[4];
  philox4x32_10(ctr, key, x);
  return ((uint64_t)x[0] | ((uint64_t)x[1] << 32)) | (1ull << 63);
}

static void push_split(orc_sim *s, int spc, const orc_particle *p) {
  if (s->n_split[spc] == s->cap_split[spc]) {
    int64_t nc = s->cap_split[spc] ? 2 * s->cap_split[spc] : 1024;
    orc_particle *nb = (orc_particle *)realloc(s->split[spc], (size_t)nc * sizeof(orc_particle));
    if (!nb) { fprintf(stderr, "oracle: out of memory for splits\n"); abort(); }
    s->split[spc] = nb; s->cap_split[spc] = nc;
  }
  s->split[spc][s->n_split[spc]++] = *p;
}

/* Finish a particle at x_n (after correction and MCC): predictor, absorption
 * test at x~_{n+1}, deposit, split.  Returns 1 if it stays. */
static int finish_particle(orc_sim *s, int spc, orc_particle *p, double r, double z, int32_t *cell) {
  predict(s, p, r, z);
  note_margin(s, 1, face_margin(s, p->r, p->z));
  int i, j;
  if (!inside_plasma(s, p->r, p->z, &i, &j)) {
    credit(s, spc, p->r, p->z, p->w);
    return 0;
  }
  deposit(s, spc, p->r, p->z, i, j, p->w);
  *cell = j * s->cfg.nr + i;
  if (s->cfg.split_cells > 0 && p->w > 2.0 * split_target(s, i)) {
    p->w *= 0.5;
    orc_particle half = *p;
    half.id = split_id(p->id, s->step, s->cfg.seed);
    push_split(s, spc, &half);
  }
  return 1;
}

static void sp_store(orc_species *S, int64_t k, const orc_particle *p, int32_t cell) {
  S->r[k] = p->r; S->z[k] = p->z; S->vr[k] = p->vr; S->vt[k] = p->vt; S->vz[k] = p->vz;
  S->ar[k] = p->ar; S->at[k] = p->at; S->az[k] = p->az; S->w[k] = p->w; S->id[k] = p->id; S->cell[k] = cell;
}

static orc_particle sp_load(const orc_species *S, int64_t k) {
  orc_particle p = {S->r[k], S->z[k], S->vr[k], S->vt[k], S->vz[k], S->ar[k], S->at[k], S->az[k], S->w[k], S->id[k]};
  return p;
}

/* Stable re-bin of one species by cell index (counting sort). */
static int rebin(orc_sim *s, int spc) {
  orc_species *S = &s->sp[spc];
  int64_t n = S->n;
  int nc = s->nc;
  int64_t *start = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  orc_particle *tmp = (orc_particle *)malloc((size_t)(n ? n : 1) * sizeof(orc_particle));
  int32_t *tcell = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
  if (!start || !tmp || !tcell) { free(start); free(tmp); free(tcell); return ORC_ENOMEM; }
  for (int64_t k = 0; k < n; ++k) start[S->cell[k] + 1]++;
  for (int c = 0; c < nc; ++c) start[c + 1] += start[c];
  for (int64_t k = 0; k < n; ++k) {
    int64_t d = start[S->cell[k]]++;
    tmp[d] = sp_load(S, k);
    tcell[d] = S->cell[k];
  }
  for (int64_t k = 0; k < n; ++k) sp_store(S, k, &tmp[k], tcell[k]);
  free(start); free(tmp); free(tcell);
  return ORC_OK;
}

/* One particle phase: for every particle, gather E at x~_n, correct to x_n,
 * D1 time filter and velocity update, axis reflection, absorption test, MCC,
 * predictor + rotation, absorption test, deposit of counts at x~_{n+1};
 * births take a-bar = 0 and the same predictor and deposit; then re-bin. */
static int particle_phase(orc_sim *s) {
  const orc_setup *c = &s->cfg;
  double dt = c->dt;
  for (int spc = 0; spc < 2; ++spc) {
    memset(s->dep[spc], 0, sizeof(double) * s->nn);
    s->n_born[spc] = 0;
    s->n_split[spc] = 0;
    for (int k = 0; k < 3; ++k) { s->abs_q[spc][k] = 0; s->abs_n[spc][k] = 0; s->coll[spc][k] = 0; }
  }
  for (int spc = 0; spc < 2; ++spc) {
    orc_species *S = &s->sp[spc];
    double qm = c->q[spc] / c->m[spc];
    int64_t kept = 0;
    for (int64_t k = 0; k < S->n; ++k) {
      orc_particle p = sp_load(S, k);
      int i, j;
      if (!inside_plasma(s, p.r, p.z, &i, &j)) { credit(s, spc, p.r, p.z, p.w); continue; }
      double w[4];
      node_weights(s, p.r, p.z, i, j, w);
      int nd[4] = {nidx(s, i, j), nidx(s, i + 1, j), nidx(s, i, j + 1), nidx(s, i + 1, j + 1)};
      double Er = 0, Ez = 0;
      for (int m = 0; m < 4; ++m) { Er += w[m] * s->Er[nd[m]]; Ez += w[m] * s->Ez[nd[m]]; }
      double an_r = qm * Er, an_z = qm * Ez;
      double r = p.r + 0.5 * dt * dt * an_r;
      double z = p.z + 0.5 * dt * dt * an_z;
      p.ar = 0.5 * (an_r + p.ar);
      p.at = 0.5 * (0.0 + p.at);
      p.az = 0.5 * (an_z + p.az);
      p.vr += dt * p.ar; p.vt += dt * p.at; p.vz += dt * p.az;
      note_margin(s, 1, fabs(r) / s->cfg.dr);
      if (r < 0.0) { r = -r; p.vr = -p.vr; p.vt = -p.vt; p.ar = -p.ar; p.at = -p.at; }
      note_margin(s, 1, face_margin(s, r, z));
      if (!inside_plasma(s, r, z, &i, &j)) { credit(s, spc, r, z, p.w); continue; }
      if (spc == 0) mcc_electron(s, &p, r, z); else mcc_ion(s, &p);
      int32_t cell;
      if (finish_particle(s, spc, &p, r, z, &cell)) sp_store(S, kept++, &p, cell);
    }
    S->n = kept;
  }
  for (int spc = 0; spc < 2; ++spc) {
    orc_species *S = &s->sp[spc];
    for (int64_t b = 0; b < s->n_born[spc]; ++b) {
      orc_particle p = s->born[spc][b];
      int32_t cell;
      double r = p.r, z = p.z;
      if (finish_particle(s, spc, &p, r, z, &cell)) {
        if (S->n >= S->cap) return ORC_EOVERFLOW;
        sp_store(S, S->n++, &p, cell);
      }
    }
    /* second halves of this phase's splits (already pushed and deposited) */
    for (int64_t b = 0; b < s->n_split[spc]; ++b) {
      orc_particle p = s->split[spc][b];
      int i, j;
      inside_plasma(s, p.r, p.z, &i, &j);
      if (S->n >= S->cap) return ORC_EOVERFLOW;
      sp_store(S, S->n++, &p, j * s->cfg.nr + i);
    }
    int st = rebin(s, spc);
    if (st) return st;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Field: operator, assembly, PCG, E at nodes, C_eq                          */
/* ------------------------------------------------------------------------ */
/* Plasma-restricted node volume: each plasma cell gives a quarter of its
 * volume pi (r_{i+1}^2 - r_i^2) dz to each of its four nodes (the volume the
 * area weighting assigns to a node for a uniform density). */
static void compute_vnode(orc_sim *s) {
  int nr = s->cfg.nr, nz = s->cfg.nz;
  double dr = s->cfg.dr, dz = s->cfg.dz;
  memset(s->vnode, 0, sizeof(double) * s->nn);
  for (int j = 0; j < nz; ++j)
    for (int i = 0; i < nr; ++i) {
      if (s->cell_kind[j * nr + i] != ORC_CELL_PLASMA) continue;
      double ri = i * dr, ri1 = (i + 1) * dr;
      double vq = 0.25 * PI * (ri1 * ri1 - ri * ri) * dz;
      s->vnode[nidx(s, i, j)] += vq;
      s->vnode[nidx(s, i + 1, j)] += vq;
      s->vnode[nidx(s, i, j + 1)] += vq;
      s->vnode[nidx(s, i + 1, j + 1)] += vq;
    }
}

/* chi at nodes: (dt^2 / 2 eps0) sum_s q_s^2 n_s / m_s (the D1 susceptibility
 * that turns Eq. 1 implicit). */
static void compute_chi(orc_sim *s) {
  const orc_setup *c = &s->cfg;
  double pre = c->dt * c->dt / (2.0 * EPS0);
  for (int a = 0; a < s->nn; ++a) {
    double v = s->vnode[a];
    double x = 0.0;
    if (v > 0.0)
      for (int spc = 0; spc < 2; ++spc)
        x += c->q[spc] * c->q[spc] / c->m[spc] * (c->w[spc] * s->dep[spc][a] / v);
    s->chi[a] = pre * x;
  }
}

/* Edge conductances of the finite-volume form of Eq. 1: each cell adjacent to
 * an edge contributes eps0 (eps_r,cell + chi_edge [cell is plasma]) times its
 * part of the control-volume face, divided by the edge length; chi_edge is
 * the mean of the edge's two nodes. */
static void build_operator(orc_sim *s, double *Gr, double *Gz, const double *chi) {
  int nr = s->cfg.nr, nz = s->cfg.nz;
  double dr = s->cfg.dr, dz = s->cfg.dz;
  /* radial edges (i,j)-(i+1,j) */
  for (int j = 0; j <= nz; ++j)
    for (int i = 0; i < nr; ++i) {
      double rh = (i + 0.5) * dr;
      double half = 2.0 * PI * rh * 0.5 * dz; /* face part inside one adjacent cell */
      double xe = chi ? 0.5 * (chi[nidx(s, i, j)] + chi[nidx(s, i + 1, j)]) : 0.0;
      double g = 0.0;
      for (int cj = j - 1; cj <= j; ++cj) {
        if (cj < 0 || cj >= nz) continue;
        int cell = cj * nr + i;
        double k = s->cell_eps[cell] + (s->cell_kind[cell] == ORC_CELL_PLASMA ? xe : 0.0);
        g += k * half;
      }
      Gr[j * nr + i] = EPS0 * g / dr;
    }
  /* axial edges (i,j)-(i,j+1) */
  for (int j = 0; j < nz; ++j)
    for (int i = 0; i <= nr; ++i) {
      double ri = i * dr;
      double xe = chi ? 0.5 * (chi[nidx(s, i, j)] + chi[nidx(s, i, j + 1)]) : 0.0;
      double g = 0.0;
      if (i > 0) { /* cell (i-1,j): annulus r in [r_{i-1/2}, r_i] */
        double rl = (i - 0.5) * dr;
        int cell = j * nr + (i - 1);
        double k = s->cell_eps[cell] + (s->cell_kind[cell] == ORC_CELL_PLASMA ? xe : 0.0);
        g += k * PI * (ri * ri - rl * rl);
      }
      if (i < nr) { /* cell (i,j): annulus r in [r_i, r_{i+1/2}] */
        double rh = (i + 0.5) * dr;
        int cell = j * nr + i;
        double k = s->cell_eps[cell] + (s->cell_kind[cell] == ORC_CELL_PLASMA ? xe : 0.0);
        g += k * PI * (rh * rh - ri * ri);
      }
      Gz[j * (nr + 1) + i] = EPS0 * g / dz;
    }
}

/* Visit the (up to four) neighbours of node (i,j) with their conductances. */
#define FOR_NEIGHBOURS(s, Gr, Gz, i, j, NB, G, BODY)                                   \
  do {                                                                                 \
    int nr_ = (s)->cfg.nr, nz_ = (s)->cfg.nz;                                          \
    if ((i) > 0) { int NB = nidx((s), (i) - 1, (j)); double G = (Gr)[(j) * nr_ + (i) - 1]; BODY } \
    if ((i) < nr_) { int NB = nidx((s), (i) + 1, (j)); double G = (Gr)[(j) * nr_ + (i)]; BODY } \
    if ((j) > 0) { int NB = nidx((s), (i), (j) - 1); double G = (Gz)[((j) - 1) * (nr_ + 1) + (i)]; BODY } \
    if ((j) < nz_) { int NB = nidx((s), (i), (j) + 1); double G = (Gz)[(j) * (nr_ + 1) + (i)]; BODY } \
  } while (0)

/* Voltage of driven electrode k (0-based) at time t. */
static double drive_voltage(const orc_setup *c, int k, double t) {
  return c->drive_V[k] * sin(TWO_PI * c->drive_f[k] * t + c->drive_phase[k]);
}

/* Set Dirichlet values: powered metal at U, grounded metal at 0, driven
 * electrode k at Ud[k] (Ud = NULL: all driven electrodes at 0). */
static void apply_dirichlet_all(orc_sim *s, double *phi, double U, const double *Ud) {
  for (int a = 0; a < s->nn; ++a) {
    int k = s->node_kind[a];
    if (k == ORC_POWERED) phi[a] = U;
    else if (k == ORC_GROUNDED) phi[a] = 0.0;
    else if (k >= ORC_DRIVEN) phi[a] = Ud ? Ud[k - ORC_DRIVEN] : 0.0;
  }
}

/* The C_eq problem's boundary: the powered electrode at U, every other metal at 0. */
static void apply_dirichlet(orc_sim *s, double *phi, double U) { apply_dirichlet_all(s, phi, U, NULL); }

/* Unit-voltage boundary of electrode `e` (a node kind): 1 on it, 0 on all other metal. */
static void apply_dirichlet_unit(orc_sim *s, double *phi, int e) {
  for (int a = 0; a < s->nn; ++a)
    if (s->node_kind[a] != ORC_FREE) phi[a] = s->node_kind[a] == e ? 1.0 : 0.0;
}

/* Jacobi-preconditioned conjugate gradients on the free nodes of
 * sum_b G_ab (phi_a - phi_b) = qrhs_a, Dirichlet values held in phi.
 * Stops when ||b - A phi||_2 <= tol ||b||_2 (b includes the Dirichlet lift),
 * confirmed on the recomputed residual. */
static int pcg_solve(orc_sim *s, const double *Gr, const double *Gz, double *phi, const double *qrhs,
                     double tol, int maxit, int *iters_out, double *relres_out) {
  int nn = s->nn, nr = s->cfg.nr, nz = s->cfg.nz;
  double *r = (double *)calloc(nn, sizeof(double));
  double *zv = (double *)calloc(nn, sizeof(double));
  double *p = (double *)calloc(nn, sizeof(double));
  double *Ap = (double *)calloc(nn, sizeof(double));
  double *dinv = (double *)calloc(nn, sizeof(double));
  if (!r || !zv || !p || !Ap || !dinv) { free(r); free(zv); free(p); free(Ap); free(dinv); return ORC_ENOMEM; }
  double bnorm2 = 0.0;
  for (int j = 0; j <= nz; ++j)
    for (int i = 0; i <= nr; ++i) {
      int a = nidx(s, i, j);
      if (s->node_kind[a] != ORC_FREE) continue;
      double d = 0.0, b = qrhs[a];
      FOR_NEIGHBOURS(s, Gr, Gz, i, j, nb, G, { d += G; if (s->node_kind[nb] != ORC_FREE) b += G * phi[nb]; });
      dinv[a] = d > 0 ? 1.0 / d : 0.0;
      bnorm2 += b * b;
    }
  double bnorm = sqrt(bnorm2);
  double target = tol * bnorm;
  if (bnorm == 0.0) target = 1e-30;
  int it = 0, status = ORC_ENOCONV;
  double rnorm = 0.0;
  while (it < maxit) {
    /* true residual */
    double rr = 0.0;
    for (int j = 0; j <= nz; ++j)
      for (int i = 0; i <= nr; ++i) {
        int a = nidx(s, i, j);
        if (s->node_kind[a] != ORC_FREE) { r[a] = 0.0; continue; }
        double acc = qrhs[a];
        FOR_NEIGHBOURS(s, Gr, Gz, i, j, nb, G, { acc -= G * (phi[a] - phi[nb]); });
        r[a] = acc;
        rr += acc * acc;
      }
    rnorm = sqrt(rr);
    if (rnorm <= target) { status = ORC_OK; break; }
    double rz = 0.0;
    for (int a = 0; a < nn; ++a) { zv[a] = dinv[a] * r[a]; p[a] = zv[a]; rz += r[a] * zv[a]; }
    while (it < maxit) {
      double pAp = 0.0;
      for (int j = 0; j <= nz; ++j)
        for (int i = 0; i <= nr; ++i) {
          int a = nidx(s, i, j);
          if (s->node_kind[a] != ORC_FREE) { Ap[a] = 0.0; continue; }
          double acc = 0.0;
          FOR_NEIGHBOURS(s, Gr, Gz, i, j, nb, G, { acc += G * (p[a] - p[nb]); });
          Ap[a] = acc;
          pAp += p[a] * acc;
        }
      double alpha = rz / pAp;
      double rr2 = 0.0;
      for (int a = 0; a < nn; ++a) {
        if (s->node_kind[a] != ORC_FREE) continue;
        phi[a] += alpha * p[a];
        r[a] -= alpha * Ap[a];
        rr2 += r[a] * r[a];
      }
      ++it;
      if (sqrt(rr2) <= target) break;
      double rz2 = 0.0;
      for (int a = 0; a < nn; ++a) { zv[a] = dinv[a] * r[a]; rz2 += r[a] * zv[a]; }
      double beta = rz2 / rz;
      rz = rz2;
      for (int a = 0; a < nn; ++a) p[a] = zv[a] + beta * p[a];
    }
  }
  if (status != ORC_OK) {
    /* final check after the last iteration */
    double rr = 0.0;
    for (int j = 0; j <= nz; ++j)
      for (int i = 0; i <= nr; ++i) {
        int a = nidx(s, i, j);
        if (s->node_kind[a] != ORC_FREE) continue;
        double acc = qrhs[a];
        FOR_NEIGHBOURS(s, Gr, Gz, i, j, nb, G, { acc -= G * (phi[a] - phi[nb]); });
        rr += acc * acc;
      }
    rnorm = sqrt(rr);
    if (rnorm <= target) status = ORC_OK;
  }
  *iters_out = it;
  *relres_out = bnorm > 0 ? rnorm / bnorm : rnorm;
  free(r); free(zv); free(p); free(Ap); free(dinv);
  return status;
}

/* E = -grad phi at nodes: central differences; E_r = 0 on the axis; one-sided
 * at the domain edge; at a Dirichlet node with exactly one free neighbour in a
 * direction, one-sided toward that neighbour. */
static void compute_efield(orc_sim *s) {
  int nr = s->cfg.nr, nz = s->cfg.nz;
  double dr = s->cfg.dr, dz = s->cfg.dz;
  const double *phi = s->phi;
  for (int j = 0; j <= nz; ++j)
    for (int i = 0; i <= nr; ++i) {
      int a = nidx(s, i, j);
      int dir = s->node_kind[a] != ORC_FREE;
      double er, ez;
      if (i == 0) er = 0.0;
      else if (i == nr) er = -(phi[a] - phi[nidx(s, i - 1, j)]) / dr;
      else {
        int fl = s->node_kind[nidx(s, i - 1, j)] == ORC_FREE, fh = s->node_kind[nidx(s, i + 1, j)] == ORC_FREE;
        if (dir && fl && !fh) er = -(phi[a] - phi[nidx(s, i - 1, j)]) / dr;
        else if (dir && fh && !fl) er = -(phi[nidx(s, i + 1, j)] - phi[a]) / dr;
        else er = -(phi[nidx(s, i + 1, j)] - phi[nidx(s, i - 1, j)]) / (2.0 * dr);
      }
      if (j == 0) ez = -(phi[nidx(s, i, 1)] - phi[a]) / dz;
      else if (j == nz) ez = -(phi[a] - phi[nidx(s, i, j - 1)]) / dz;
      else {
        int fl = s->node_kind[nidx(s, i, j - 1)] == ORC_FREE, fh = s->node_kind[nidx(s, i, j + 1)] == ORC_FREE;
        if (dir && fl && !fh) ez = -(phi[a] - phi[nidx(s, i, j - 1)]) / dz;
        else if (dir && fh && !fl) ez = -(phi[nidx(s, i, j + 1)] - phi[a]) / dz;
        else ez = -(phi[nidx(s, i, j + 1)] - phi[nidx(s, i, j - 1)]) / (2.0 * dz);
      }
      s->Er[a] = er;
      s->Ez[a] = ez;
    }
}

/* Equivalent capacitance from the field energy (Eqs. 6-7): solve with the
 * powered electrode at 1 V and the rest grounded, then 1/2 C U^2 = sum over
 * edges of 1/2 G (phi_a - phi_b)^2.  Also returns the Gauss-law charge on the
 * electrode (net flux out of the powered nodes), which must agree. */
static int compute_ceq(orc_sim *s, int with_chi, double *ceq, double *gauss) {
  int nn = s->nn, nr = s->cfg.nr, nz = s->cfg.nz;
  double *Gr = (double *)malloc(sizeof(double) * (size_t)(nz + 1) * nr);
  double *Gz = (double *)malloc(sizeof(double) * (size_t)nz * (nr + 1));
  double *phiL = (double *)calloc(nn, sizeof(double));
  double *q0 = (double *)calloc(nn, sizeof(double));
  if (!Gr || !Gz || !phiL || !q0) { free(Gr); free(Gz); free(phiL); free(q0); return ORC_ENOMEM; }
  build_operator(s, Gr, Gz, with_chi ? s->chi : NULL);
  apply_dirichlet(s, phiL, 1.0);
  int it; double rel;
  double tol = s->cfg.pcg_tol < 1e-12 ? s->cfg.pcg_tol : 1e-12;
  int st = pcg_solve(s, Gr, Gz, phiL, q0, tol, s->cfg.pcg_maxit, &it, &rel);
  double energy2 = 0.0, q = 0.0;
  for (int j = 0; j <= nz; ++j)
    for (int i = 0; i < nr; ++i) {
      int a = nidx(s, i, j), b = nidx(s, i + 1, j);
      double d = phiL[a] - phiL[b], g = Gr[j * nr + i];
      energy2 += g * d * d;
      if (s->node_kind[a] == ORC_POWERED && s->node_kind[b] != ORC_POWERED) q += g * d;
      if (s->node_kind[b] == ORC_POWERED && s->node_kind[a] != ORC_POWERED) q -= g * d;
    }
  for (int j = 0; j < nz; ++j)
    for (int i = 0; i <= nr; ++i) {
      int a = nidx(s, i, j), b = nidx(s, i, j + 1);
      double d = phiL[a] - phiL[b], g = Gz[j * (nr + 1) + i];
      energy2 += g * d * d;
      if (s->node_kind[a] == ORC_POWERED && s->node_kind[b] != ORC_POWERED) q += g * d;
      if (s->node_kind[b] == ORC_POWERED && s->node_kind[a] != ORC_POWERED) q -= g * d;
    }
  *ceq = energy2; /* 2 * (1/2 sum G dphi^2) / U^2 with U = 1 */
  *gauss = q;
  /* the same solution is the powered electrode's unit Laplace solution phi_L0 */
  if (s->cfg.field_mode == ORC_FIELD_VAHEDI && st == ORC_OK) memcpy(s->phiL[0], phiL, sizeof(double) * nn);
  free(Gr); free(Gz); free(phiL); free(q0);
  return st;
}

/* Unit-voltage Laplace solutions of the driven electrodes (Eq. 4 with the
 * implicit operator of Eq. 1: phi_Lk = 1 on electrode k, 0 on all other
 * metal, no charge), with the current chi or in vacuum.  Solved to the C_eq
 * solve's tolerance, each from its previous solution. */
static int refresh_laplace(orc_sim *s, int with_chi) {
  int nn = s->nn, nr = s->cfg.nr, nz = s->cfg.nz;
  double *Gr = (double *)malloc(sizeof(double) * (size_t)(nz + 1) * nr);
  double *Gz = (double *)malloc(sizeof(double) * (size_t)nz * (nr + 1));
  double *q0 = (double *)calloc(nn, sizeof(double));
  if (!Gr || !Gz || !q0) { free(Gr); free(Gz); free(q0); return ORC_ENOMEM; }
  build_operator(s, Gr, Gz, with_chi ? s->chi : NULL);
  double tol = s->cfg.pcg_tol < 1e-12 ? s->cfg.pcg_tol : 1e-12;
  int st = ORC_OK;
  for (int k = 0; k < s->cfg.n_drive && st == ORC_OK; ++k) {
    int it; double rel;
    apply_dirichlet_unit(s, s->phiL[k + 1], ORC_DRIVEN + k);
    st = pcg_solve(s, Gr, Gz, s->phiL[k + 1], q0, tol, s->cfg.pcg_maxit, &it, &rel);
  }
  free(Gr); free(Gz); free(q0);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Circuit (Eqs. 5, 8, 9, 10)                                                */
/* ------------------------------------------------------------------------ */
static double source_voltage(const orc_setup *c, double t) { return c->V_src * sin(TWO_PI * c->f_src * t + c->phase_src); }

static int circuit_dim(const orc_setup *c) { return c->circuit == ORC_CIRCUIT_RLC ? 3 : c->circuit == ORC_CIRCUIT_IMN ? 6 : 0; }

/* Right-hand side of the circuit ODEs together with the electrode charge
 * balance, written as printed.  Circuit I state (Q_b, I_b, Q_E), Eq. 9;
 * circuit II state (Q_1, Q_2, I_2, Q_ccp, I_stray, Q_E), Eq. 10; in both
 * dQ_E/dt = I_ccp + I_conv (Eq. 8) and U_E = U_ccp = Q_E / C_eq (Eq. 5).
 * `with_source` = 0 drops U_s and I_conv, leaving the linear part. */
static void circuit_rhs(const orc_sim *s, double t, const double *y, int with_source, double *f) {
  const orc_setup *c = &s->cfg;
  double Us = with_source ? source_voltage(c, t) : 0.0;
  double Ic = with_source ? s->I_conv : 0.0;
  if (c->circuit == ORC_CIRCUIT_RLC) {
    double Rb = c->circ[0], Lb = c->circ[1], Cb = c->circ[2];
    double Qb = y[0], Ib = y[1], QE = y[2];
    double UE = QE / s->ceq;
    f[0] = Ib;
    f[1] = (Us - UE - Qb / Cb - Ib * Rb) / Lb;
    f[2] = Ib + Ic;
  } else {
    double Rs = c->circ[0], Cm1 = c->circ[1], Lm = c->circ[2], Cm2 = c->circ[3], Rm = c->circ[4];
    double Cst = c->circ[5], Rst = c->circ[6], Lst = c->circ[7];
    double Q1 = y[0], Q2 = y[1], I2 = y[2], Qccp = y[3], Ist = y[4], QE = y[5];
    double Uccp = QE / s->ceq;
    f[0] = (Us - (Q1 - Q2) / Cm1) / Rs;
    f[1] = I2;
    f[2] = ((Q1 - Q2) / Cm1 - Uccp - Q2 / Cm2 - I2 * Rm) / Lm;
    f[3] = I2 - Ist;
    f[4] = (Uccp - (Q2 - Qccp) / Cst - Ist * Rst) / Lst;
    f[5] = (I2 - Ist) + Ic;
  }
}

/* Gaussian elimination with partial pivoting, n <= 6. */
static void solve_dense(int n, double A[6][6], double *b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int r = k + 1; r < n; ++r) if (fabs(A[r][k]) > fabs(A[piv][k])) piv = r;
    if (piv != k) {
      for (int cc = 0; cc < n; ++cc) { double t = A[k][cc]; A[k][cc] = A[piv][cc]; A[piv][cc] = t; }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int r = k + 1; r < n; ++r) {
      double m = A[r][k] / A[k][k];
      for (int cc = k; cc < n; ++cc) A[r][cc] -= m * A[k][cc];
      b[r] -= m * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double acc = b[k];
    for (int cc = k + 1; cc < n; ++cc) acc -= A[k][cc] * b[cc];
    b[k] = acc / A[k][k];
  }
}

/* Advance the circuit from t_n to t_{n+1} with n_sub trapezoidal substeps,
 * I_conv held at this step's tally; then U_E = Q_E / C_eq.  Direct drive
 * imposes U_E = U_s(t_{n+1}) and Q_E = C_eq U_E. */
static void circuit_advance(orc_sim *s) {
  const orc_setup *c = &s->cfg;
  double tn = (double)s->step * c->dt;
  double t1 = tn + c->dt;
  if (c->circuit == ORC_CIRCUIT_DIRECT) {
    double U_old = source_voltage(c, tn);
    s->U_E = source_voltage(c, t1);
    s->Q_E = s->ceq * s->U_E;
    s->I_ccp = s->ceq * (s->U_E - U_old) / c->dt - s->I_conv;
    return;
  }
  int n = circuit_dim(c);
  double Mx[6][6];
  for (int k = 0; k < n; ++k) {
    double e[6] = {0, 0, 0, 0, 0, 0}, f[6];
    e[k] = 1.0;
    circuit_rhs(s, 0.0, e, 0, f);
    for (int r = 0; r < n; ++r) Mx[r][k] = f[r];
  }
  double h = c->dt / c->n_sub;
  double zero[6] = {0, 0, 0, 0, 0, 0};
  for (int sub = 0; sub < c->n_sub; ++sub) {
    double ta = tn + sub * h, tb = tn + (sub + 1) * h;
    double fa[6], sb[6], A[6][6], rhs[6];
    circuit_rhs(s, ta, s->y, 1, fa);
    circuit_rhs(s, tb, zero, 1, sb);
    for (int r = 0; r < n; ++r) {
      rhs[r] = s->y[r] + 0.5 * h * fa[r] + 0.5 * h * sb[r];
      for (int k = 0; k < n; ++k) A[r][k] = (r == k ? 1.0 : 0.0) - 0.5 * h * Mx[r][k];
    }
    solve_dense(n, A, rhs);
    for (int r = 0; r < n; ++r) s->y[r] = rhs[r];
  }
  if (c->circuit == ORC_CIRCUIT_RLC) { s->Q_E = s->y[2]; s->I_ccp = s->y[1]; }
  else { s->Q_E = s->y[5]; s->I_ccp = s->y[2] - s->y[4]; }
  s->U_E = s->Q_E / s->ceq;
}

/* ------------------------------------------------------------------------ */
/* Assembly, field solve, diagnostics, step                                  */
/* ------------------------------------------------------------------------ */
/* rho~ per node (charge, Gauss form of Eq. 1) and chi, then the operator. */
static void assemble(orc_sim *s) {
  const orc_setup *c = &s->cfg;
  compute_chi(s);
  for (int a = 0; a < s->nn; ++a) {
    double q = s->sigma[a];
    for (int spc = 0; spc < 2; ++spc) q += c->q[spc] * c->w[spc] * s->dep[spc][a];
    s->qrhs[a] = q;
  }
  build_operator(s, s->Gr, s->Gz, s->chi);
  if (c->field_mode == ORC_FIELD_VAHEDI) {
    apply_dirichlet_all(s, s->phiP, 0.0, NULL);  /* Eq. 3: zero on every electrode */
  } else {
    double Ud[ORC_MAX_DRIVE];
    for (int k = 0; k < c->n_drive; ++k) Ud[k] = drive_voltage(c, k, s->t_field);
    apply_dirichlet_all(s, s->phi, s->U_E, Ud);
  }
}

/* Direct mode: one solve of Eq. 1 with every electrode at its voltage.
 * Vahedi mode: the zero-boundary solve phi_P (Eq. 3), then Eq. 2,
 * phi = phi_P + U_E phi_L0 + sum_k U_k phi_Lk, with the Laplace solutions of
 * the last refresh. */
static int field_solve(orc_sim *s) {
  const orc_setup *c = &s->cfg;
  double *target = c->field_mode == ORC_FIELD_VAHEDI ? s->phiP : s->phi;
  int st = pcg_solve(s, s->Gr, s->Gz, target, s->qrhs, c->pcg_tol, c->pcg_maxit, &s->pcg_iters, &s->pcg_relres);
  s->pcg_status = st;
  if (c->field_mode == ORC_FIELD_VAHEDI) {
    double Ud[ORC_MAX_DRIVE];
    for (int k = 0; k < c->n_drive; ++k) Ud[k] = drive_voltage(c, k, s->t_field);
    for (int a = 0; a < s->nn; ++a) {
      double v = s->phiP[a] + s->U_E * s->phiL[0][a];
      for (int k = 0; k < c->n_drive; ++k) v += Ud[k] * s->phiL[k + 1][a];
      s->phi[a] = v;
    }
  }
  compute_efield(s);
  return st;
}

/* The waveforms and element powers of the circuit at t_{n+1} (Sec. 3): the
 * source voltage U_s, the current I_1 leaving the source, the voltage U_in at
 * the matching network's input (after R_s), U_E = U_ccp and I_ccp; powers
 * U_s I_1, R_s I_1^2, the series element's loss (R_m I_2^2 in circuit II,
 * R_b I_b^2 in circuit I), the stray branch's loss R_stray I_stray^2,
 * U_ccp I_ccp and U_in I_1. */
static void circuit_waveforms(const orc_sim *s, double t1, double w[5], double p[6]) {
  const orc_setup *c = &s->cfg;
  double Us = source_voltage(c, t1);
  for (int k = 0; k < 6; ++k) p[k] = 0.0;
  if (c->circuit == ORC_CIRCUIT_IMN) {
    double Rs = c->circ[0], Cm1 = c->circ[1], Rm = c->circ[4], Rst = c->circ[6];
    double Uin = (s->y[0] - s->y[1]) / Cm1;
    double I1 = (Us - Uin) / Rs;
    double I2 = s->y[2], Ist = s->y[4];
    w[0] = Us; w[1] = I1; w[2] = Uin;
    p[1] = Rs * I1 * I1;
    p[2] = Rm * I2 * I2;
    p[3] = Rst * Ist * Ist;
    p[5] = Uin * I1;
    p[0] = Us * I1;
  } else if (c->circuit == ORC_CIRCUIT_RLC) {
    double Ib = s->y[1];
    w[0] = Us; w[1] = Ib; w[2] = Us;
    p[0] = Us * Ib;
    p[2] = c->circ[0] * Ib * Ib;
    p[5] = Us * Ib;
  } else {
    w[0] = s->U_E; w[1] = s->I_ccp; w[2] = s->U_E;
    p[0] = p[5] = s->U_E * s->I_ccp;
  }
  w[3] = s->U_E;
  w[4] = s->I_ccp;
  p[4] = s->U_E * s->I_ccp;
}

/* Close the circuit window (Sec. 3): Z = U_1 / I_1 of the fundamental
 * (Eq. 11: modulus ratio and phase difference of the two first harmonics),
 * Gamma = (Z_load - R_s) / (Z_load + R_s) (Eq. 12), period-averaged powers
 * (Eq. 13) and P_ref = P_forward |Gamma|^2 (Eq. 14) with P_forward the power
 * into the matching network's input. */
static void circuit_window(orc_sim *s, int N) {
  double Ur = s->cw_re[3], Ui = s->cw_im[3], Ir = s->cw_re[4], Ii = s->cw_im[4];
  double den = Ir * Ir + Ii * Ii;
  double zc_re = den > 0 ? (Ur * Ir + Ui * Ii) / den : 0.0, zc_im = den > 0 ? (Ui * Ir - Ur * Ii) / den : 0.0;
  Ur = s->cw_re[2]; Ui = s->cw_im[2]; Ir = s->cw_re[1]; Ii = s->cw_im[1];
  den = Ir * Ir + Ii * Ii;
  double zl_re = den > 0 ? (Ur * Ir + Ui * Ii) / den : 0.0, zl_im = den > 0 ? (Ui * Ir - Ur * Ii) / den : 0.0;
  double g_re = 0.0, g_im = 0.0;
  if (s->cfg.circuit == ORC_CIRCUIT_IMN) {
    double Rs = s->cfg.circ[0];
    double nr = zl_re - Rs, ni = zl_im, dr = zl_re + Rs, di = zl_im;
    double dd = dr * dr + di * di;
    g_re = (nr * dr + ni * di) / dd;
    g_im = (ni * dr - nr * di) / dd;
  }
  double g2 = g_re * g_re + g_im * g_im;
  double *o = s->circ_out;
  o[0] = zc_re; o[1] = zc_im; o[2] = zl_re; o[3] = zl_im; o[4] = g_re; o[5] = g_im; o[6] = sqrt(g2);
  for (int k = 0; k < 6; ++k) o[7 + k] = s->cp_sum[k] / N;
  o[13] = o[12] * g2;
  o[14] = 2.0 * s->cw_re[3] / N; /* first harmonic of U_E */
  o[15] = 2.0 * s->cw_im[3] / N;
  o[16] = s->cdc[0] / N;          /* mean U_E: the DC self-bias (Sec. 3, circuit I) */
  o[17] = s->cdc[1] / N;          /* mean I_ccp */
  for (int k = 0; k < 5; ++k) s->cw_re[k] = s->cw_im[k] = 0.0;
  for (int k = 0; k < 6; ++k) s->cp_sum[k] = 0.0;
  s->cdc[0] = s->cdc[1] = 0.0;
}

static void diag_accumulate(orc_sim *s) {
  const orc_setup *c = &s->cfg;
  for (int spc = 0; spc < 2; ++spc)
    for (int a = 0; a < s->nn; ++a)
      if (s->vnode[a] > 0) s->dens_sum[spc][a] += c->w[spc] * s->dep[spc][a] / s->vnode[a];
  for (int k = 0; k < 3; ++k) s->ion_q_sum[k] += s->abs_q[1][k];
  double t1 = (double)(s->step + 1) * c->dt;
  double ph = TWO_PI * c->f_src * t1;
  s->dft_re += s->I_ccp * cos(ph);
  s->dft_im -= s->I_ccp * sin(ph);
  double w[5], p[6];
  circuit_waveforms(s, t1, w, p);
  for (int k = 0; k < 5; ++k) {
    s->cw_re[k] += w[k] * cos(ph);
    s->cw_im[k] -= w[k] * sin(ph);
  }
  for (int k = 0; k < 6; ++k) s->cp_sum[k] += p[k];
  s->cdc[0] += w[3];
  s->cdc[1] += w[4];
  s->win_count++;
  if (s->win_count == c->steps_per_rf) {
    int N = s->win_count;
    for (int spc = 0; spc < 2; ++spc)
      for (int a = 0; a < s->nn; ++a) { s->dens_avg[spc][a] = s->dens_sum[spc][a] / N; s->dens_sum[spc][a] = 0.0; }
    for (int k = 0; k < 3; ++k) { s->ion_cur_avg[k] = s->ion_q_sum[k] / (N * c->dt); s->ion_q_sum[k] = 0.0; }
    s->i1_re = 2.0 * s->dft_re / N;
    s->i1_im = 2.0 * s->dft_im / N;
    s->dft_re = s->dft_im = 0.0;
    circuit_window(s, N);
    s->win_count = 0;
    s->windows_done++;
  }
}

static int one_step(orc_sim *s) {
  int st = particle_phase(s);
  if (st) return st;
  s->I_conv = (s->abs_q[0][0] + s->abs_q[1][0]) / s->cfg.dt;
  circuit_advance(s);
  s->t_field = (double)(s->step + 1) * s->cfg.dt;
  assemble(s);
  st = field_solve(s);
  diag_accumulate(s);
  s->step++;
  if (s->cfg.ceq_refresh && s->win_count == 0) {
    double cq, g;
    int st2 = compute_ceq(s, 1, &cq, &g);
    if (st2 == ORC_OK) { s->ceq = cq; s->ceq_gauss = g; }
    if (st2 == ORC_OK && s->cfg.field_mode == ORC_FIELD_VAHEDI) st2 = refresh_laplace(s, 1);
    if (st2 != ORC_OK && st == ORC_OK) st = st2;
    if (s->cfg.circuit != ORC_CIRCUIT_DIRECT) s->U_E = s->Q_E / s->ceq;
  }
  return st;
}

/* ------------------------------------------------------------------------ */
/* Exported API (ctypes)                                                     */
/* ------------------------------------------------------------------------ */
static void free_species(orc_species *S) {
  free(S->r); free(S->z); free(S->vr); free(S->vt); free(S->vz);
  free(S->ar); free(S->at); free(S->az); free(S->w); free(S->id); free(S->cell);
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  free(s->node_kind); free(s->cell_kind); free(s->cell_eps); free(s->xs_energy); free(s->xs_sigma);
  free(s->vnode); free(s->Gr); free(s->Gz); free(s->sigma); free(s->chi); free(s->qrhs);
  free(s->phi); free(s->Er); free(s->Ez); free(s->phiP);
  for (int k = 0; k <= ORC_MAX_DRIVE; ++k) free(s->phiL[k]);
  for (int k = 0; k < 2; ++k) {
    free(s->dep[k]); free_species(&s->sp[k]); free(s->born[k]); free(s->split[k]); free(s->dens_sum[k]);
    free(s->dens_avg[k]);
  }
  free(s);
}

int orc_create(const orc_setup *cfg, orc_sim **out) {
  if (!cfg || !out || cfg->nr < 1 || cfg->nz < 1 || cfg->n_xs < 2 || cfg->dt <= 0) return ORC_EINVAL;
  if (cfg->circuit < 0 || cfg->circuit > 2 || cfg->steps_per_rf < 1 || cfg->n_sub < 1) return ORC_EINVAL;
  if (cfg->n_drive < 0 || cfg->n_drive > ORC_MAX_DRIVE) return ORC_EINVAL;
  if (cfg->field_mode != ORC_FIELD_DIRECT && cfg->field_mode != ORC_FIELD_VAHEDI) return ORC_EINVAL;
  for (int a = 0; a < (cfg->nr + 1) * (cfg->nz + 1); ++a)
    if (cfg->node_kind[a] < 0 || cfg->node_kind[a] > ORC_GROUNDED + cfg->n_drive) return ORC_EINVAL;
  orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
  if (!s) return ORC_ENOMEM;
  s->cfg = *cfg;
  int nr = cfg->nr, nz = cfg->nz;
  s->nn = (nr + 1) * (nz + 1);
  s->nc = nr * nz;
  s->node_kind = (int8_t *)malloc(s->nn);
  s->cell_kind = (int8_t *)malloc(s->nc);
  s->cell_eps = (double *)malloc(sizeof(double) * s->nc);
  s->xs_energy = (double *)malloc(sizeof(double) * cfg->n_xs);
  s->xs_sigma = (double *)malloc(sizeof(double) * 5 * cfg->n_xs);
  s->vnode = (double *)calloc(s->nn, sizeof(double));
  s->Gr = (double *)calloc((size_t)(nz + 1) * nr, sizeof(double));
  s->Gz = (double *)calloc((size_t)nz * (nr + 1), sizeof(double));
  s->sigma = (double *)calloc(s->nn, sizeof(double));
  s->chi = (double *)calloc(s->nn, sizeof(double));
  s->qrhs = (double *)calloc(s->nn, sizeof(double));
  s->phi = (double *)calloc(s->nn, sizeof(double));
  s->Er = (double *)calloc(s->nn, sizeof(double));
  s->Ez = (double *)calloc(s->nn, sizeof(double));
  s->phiP = (double *)calloc(s->nn, sizeof(double));
  int ok = s->node_kind && s->cell_kind && s->cell_eps && s->xs_energy && s->xs_sigma && s->vnode && s->Gr &&
           s->Gz && s->sigma && s->chi && s->qrhs && s->phi && s->Er && s->Ez && s->phiP;
  for (int k = 0; k <= cfg->n_drive && ok; ++k) {
    s->phiL[k] = (double *)calloc(s->nn, sizeof(double));
    ok = s->phiL[k] != NULL;
  }
  for (int k = 0; k < 2 && ok; ++k) {
    s->dep[k] = (double *)calloc(s->nn, sizeof(double));
    s->dens_sum[k] = (double *)calloc(s->nn, sizeof(double));
    s->dens_avg[k] = (double *)calloc(s->nn, sizeof(double));
    orc_species *S = &s->sp[k];
    int64_t cap = cfg->capacity[k] > 0 ? cfg->capacity[k] : 1;
    S->cap = cap;
    S->r = (double *)malloc(sizeof(double) * cap); S->z = (double *)malloc(sizeof(double) * cap);
    S->vr = (double *)malloc(sizeof(double) * cap); S->vt = (double *)malloc(sizeof(double) * cap);
    S->vz = (double *)malloc(sizeof(double) * cap); S->ar = (double *)malloc(sizeof(double) * cap);
    S->at = (double *)malloc(sizeof(double) * cap); S->az = (double *)malloc(sizeof(double) * cap);
    S->w = (double *)malloc(sizeof(double) * cap);
    S->id = (uint64_t *)malloc(sizeof(uint64_t) * cap); S->cell = (int32_t *)malloc(sizeof(int32_t) * cap);
    ok = s->dep[k] && s->dens_sum[k] && s->dens_avg[k] && S->r && S->z && S->vr && S->vt && S->vz && S->ar &&
         S->at && S->az && S->w && S->id && S->cell;
  }
  if (!ok) { orc_destroy(s); return ORC_ENOMEM; }
  memcpy(s->node_kind, cfg->node_kind, s->nn);
  memcpy(s->cell_kind, cfg->cell_kind, s->nc);
  memcpy(s->cell_eps, cfg->cell_eps, sizeof(double) * s->nc);
  memcpy(s->xs_energy, cfg->xs_energy, sizeof(double) * cfg->n_xs);
  memcpy(s->xs_sigma, cfg->xs_sigma, sizeof(double) * 5 * cfg->n_xs);
  s->cfg.node_kind = s->node_kind; s->cfg.cell_kind = s->cell_kind; s->cfg.cell_eps = s->cell_eps;
  s->cfg.xs_energy = s->xs_energy; s->cfg.xs_sigma = s->xs_sigma;
  compute_vnode(s);
  compute_numax(s);
  s->ceq = 1.0;
  *out = s;
  return ORC_OK;
}

/* w: weight ratios in (0, 1] (NULL: all 1). */
int orc_set_particles(orc_sim *s, int spc, int64_t n, const double *r, const double *z, const double *vr,
                      const double *vt, const double *vz, const double *ar, const double *at, const double *az,
                      const uint64_t *id, const double *w) {
  if (!s || spc < 0 || spc > 1 || n < 0) return ORC_EINVAL;
  orc_species *S = &s->sp[spc];
  if (n > S->cap) return ORC_EOVERFLOW;
  for (int64_t k = 0; k < n; ++k) {
    int i, j;
    if (!inside_plasma(s, r[k], z[k], &i, &j)) return ORC_EINVAL;
    if (w && !(w[k] > 0.0 && w[k] <= 1.0)) return ORC_EINVAL;
    S->r[k] = r[k]; S->z[k] = z[k]; S->vr[k] = vr[k]; S->vt[k] = vt[k]; S->vz[k] = vz[k];
    S->ar[k] = ar[k]; S->at[k] = at[k]; S->az[k] = az[k]; S->id[k] = id[k];
    S->w[k] = w ? w[k] : 1.0;
    S->cell[k] = j * s->cfg.nr + i;
  }
  S->n = n;
  return ORC_OK;
}

int64_t orc_count(const orc_sim *s, int spc) { return s->sp[spc].n; }

int orc_get_particles(const orc_sim *s, int spc, double *r, double *z, double *vr, double *vt, double *vz,
                      double *ar, double *at, double *az, uint64_t *id, int32_t *cell, double *w) {
  const orc_species *S = &s->sp[spc];
  for (int64_t k = 0; k < S->n; ++k) {
    r[k] = S->r[k]; z[k] = S->z[k]; vr[k] = S->vr[k]; vt[k] = S->vt[k]; vz[k] = S->vz[k];
    ar[k] = S->ar[k]; at[k] = S->at[k]; az[k] = S->az[k]; id[k] = S->id[k]; cell[k] = S->cell[k];
    if (w) w[k] = S->w[k];
  }
  return ORC_OK;
}

/* Node-field access: 0 phi, 1 E_r, 2 E_z, 3 chi, 4 electron counts,
 * 5 ion counts, 6 surface charge, 7 node volume, 8 rho~ (charge per node),
 * 9 average n_e of the last window, 10 average n_i of the last window. */
static double *field_ptr(orc_sim *s, int which) {
  switch (which) {
    case 0: return s->phi; case 1: return s->Er; case 2: return s->Ez; case 3: return s->chi;
    case 4: return s->dep[0]; case 5: return s->dep[1]; case 6: return s->sigma; case 7: return s->vnode;
    case 8: return s->qrhs; case 9: return s->dens_avg[0]; case 10: return s->dens_avg[1];
    case 11: return s->phiP;
    case 12: case 13: case 14: case 15: return s->phiL[which - 12];  /* NULL beyond n_drive */
    default: return NULL;
  }
}

int orc_get_field(orc_sim *s, int which, double *out) {
  double *p = field_ptr(s, which);
  if (!p) return ORC_EINVAL;
  memcpy(out, p, sizeof(double) * s->nn);
  return ORC_OK;
}

int orc_set_field(orc_sim *s, int which, const double *in) {
  double *p = field_ptr(s, which);
  if (!p) return ORC_EINVAL;
  memcpy(p, in, sizeof(double) * s->nn);
  return ORC_OK;
}

/* Edge conductances: which 0 = radial [(nz+1)*nr], 1 = axial [nz*(nr+1)]. */
int orc_get_operator(orc_sim *s, int which, double *out) {
  if (which == 0) memcpy(out, s->Gr, sizeof(double) * (size_t)(s->cfg.nz + 1) * s->cfg.nr);
  else if (which == 1) memcpy(out, s->Gz, sizeof(double) * (size_t)s->cfg.nz * (s->cfg.nr + 1));
  else return ORC_EINVAL;
  return ORC_OK;
}

void orc_set_step(orc_sim *s, uint32_t step) { s->step = step; }

int orc_particle_phase(orc_sim *s) { return particle_phase(s); }

/* Deposit the current x~ without moving anything (start-up). */
int orc_deposit_only(orc_sim *s) {
  for (int spc = 0; spc < 2; ++spc) {
    memset(s->dep[spc], 0, sizeof(double) * s->nn);
    orc_species *S = &s->sp[spc];
    for (int64_t k = 0; k < S->n; ++k) {
      int i, j;
      if (!inside_plasma(s, S->r[k], S->z[k], &i, &j)) return ORC_EINVAL;
      deposit(s, spc, S->r[k], S->z[k], i, j, S->w[k]);
    }
  }
  return ORC_OK;
}

int orc_assemble(orc_sim *s) { assemble(s); return ORC_OK; }

int orc_field_solve(orc_sim *s, int *iters, double *relres) {
  int st = field_solve(s);
  if (iters) *iters = s->pcg_iters;
  if (relres) *relres = s->pcg_relres;
  return st;
}

int orc_solve_tol(orc_sim *s, double tol, int *iters, double *relres) {
  int st = pcg_solve(s, s->Gr, s->Gz, s->phi, s->qrhs, tol, s->cfg.pcg_maxit, &s->pcg_iters, &s->pcg_relres);
  compute_efield(s);
  if (iters) *iters = s->pcg_iters;
  if (relres) *relres = s->pcg_relres;
  return st;
}

int orc_efield(orc_sim *s) { compute_efield(s); return ORC_OK; }

int orc_ceq(orc_sim *s, int with_chi, double *ceq, double *gauss) { return compute_ceq(s, with_chi, ceq, gauss); }

void orc_set_ceq(orc_sim *s, double ceq) { s->ceq = ceq; }

void orc_set_conv_current(orc_sim *s, double I) { s->I_conv = I; }

int orc_circuit_advance(orc_sim *s) { circuit_advance(s); return ORC_OK; }

void orc_set_circuit_state(orc_sim *s, const double *y) {
  for (int k = 0; k < 6; ++k) s->y[k] = y[k];
  int n = circuit_dim(&s->cfg);
  if (n) s->Q_E = s->y[n - 1];
  s->U_E = s->Q_E / s->ceq;
}

/* Start-up: deposit x~_0, vacuum C_eq, U_E(0), assemble, solve. */
int orc_init_fields(orc_sim *s) {
  int st = orc_deposit_only(s);
  if (st) return st;
  double cq, g;
  st = compute_ceq(s, 0, &cq, &g);
  if (st) return st;
  s->ceq = cq; s->ceq_gauss = g;
  if (s->cfg.field_mode == ORC_FIELD_VAHEDI && (st = refresh_laplace(s, 0))) return st;
  if (s->cfg.circuit == ORC_CIRCUIT_DIRECT) {
    s->U_E = source_voltage(&s->cfg, (double)s->step * s->cfg.dt);
    s->Q_E = s->ceq * s->U_E;
  } else {
    int n = circuit_dim(&s->cfg);
    s->Q_E = s->y[n - 1];
    s->U_E = s->Q_E / s->ceq;
  }
  s->t_field = (double)s->step * s->cfg.dt;
  assemble(s);
  return field_solve(s);
}

int orc_step(orc_sim *s, int nsteps) {
  for (int k = 0; k < nsteps; ++k) {
    int st = one_step(s);
    if (st) return st;
  }
  return ORC_OK;
}

/* Scalars: [0] step, [1] t, [2] U_E, [3] Q_E, [4] C_eq, [5] I_conv, [6] I_ccp,
 * [7..12] circuit state, [13] pcg iterations, [14] pcg relative residual,
 * [15] nu_max e, [16] nu_max i, [17] P_coll e, [18] P_coll i,
 * [19..24] absorbed charge (e: powered, grounded, surface; i: same),
 * [25..30] absorbed counts (same order), [31..36] collisions
 * (e: elastic, excitation, ionization; i: isotropic, charge exchange, -),
 * [37] births e, [38] births i, [39..41] ion current of the last window
 * (powered, grounded, surface), [42] Re I1, [43] Im I1, [44] windows done,
 * [45] C_eq Gauss route, [46] pcg status, [47..48] splits of the last
 * particle phase (e, i). */
int orc_scalars(const orc_sim *s, double *o, int n) {
  double v[49];
  v[0] = s->step; v[1] = s->step * s->cfg.dt; v[2] = s->U_E; v[3] = s->Q_E; v[4] = s->ceq;
  v[5] = s->I_conv; v[6] = s->I_ccp;
  for (int k = 0; k < 6; ++k) v[7 + k] = s->y[k];
  v[13] = s->pcg_iters; v[14] = s->pcg_relres;
  v[15] = s->numax[0]; v[16] = s->numax[1]; v[17] = s->pcoll[0]; v[18] = s->pcoll[1];
  for (int spc = 0; spc < 2; ++spc)
    for (int k = 0; k < 3; ++k) {
      v[19 + 3 * spc + k] = s->abs_q[spc][k];
      v[25 + 3 * spc + k] = (double)s->abs_n[spc][k];
      v[31 + 3 * spc + k] = (double)s->coll[spc][k];
    }
  v[37] = (double)s->n_born[0]; v[38] = (double)s->n_born[1];
  for (int k = 0; k < 3; ++k) v[39 + k] = s->ion_cur_avg[k];
  v[42] = s->i1_re; v[43] = s->i1_im; v[44] = s->windows_done; v[45] = s->ceq_gauss; v[46] = s->pcg_status;
  v[47] = (double)s->n_split[0]; v[48] = (double)s->n_split[1];
  for (int k = 0; k < n && k < 49; ++k) o[k] = v[k];
  return ORC_OK;
}

/* Decision-margin tracing (test instrumentation): enable = 1 resets the
 * three margins to +inf and starts recording them in later particle phases,
 * 0 stops; out3 (may be NULL) receives the margins recorded so far:
 * [0] smallest relative gap between a uniform or an energy and its threshold,
 * [1] smallest distance (cell units) from a tested position to a face across
 * which the particle would change plasma membership, or to the axis,
 * [2] smallest |(X, Y)| / (dr + dt |u_perp|) of a predictor rotation. */
int orc_trace(orc_sim *s, int enable, double *out3) {
  if (out3)
    for (int k = 0; k < 3; ++k) out3[k] = s->margin[k];
  if (enable == 1) {
    s->trace = 1;
    for (int k = 0; k < 3; ++k) s->margin[k] = 1e300;
  } else if (enable == 0) {
    s->trace = 0;
  }
  return ORC_OK;
}

/* Ids of the electron (out[2k]) and ion (out[2k+1]) that an ionization of
 * parents[k] would create in `step` (test hook). */
void orc_child_ids(uint32_t step, uint32_t seed, int64_t n, const uint64_t *parents, uint64_t *out) {
  for (int64_t k = 0; k < n; ++k) {
    out[2 * k] = child_id(parents[k], step, 0, seed);
    out[2 * k + 1] = child_id(parents[k], step, 1, seed);
  }
}

/* Id of the second half of parents[k] if it splits in `step` (test hook). */
void orc_split_ids(uint32_t step, uint32_t seed, int64_t n, const uint64_t *parents, uint64_t *out) {
  for (int64_t k = 0; k < n; ++k) out[k] = split_id(parents[k], step, seed);
}

/* Circuit post-processing of the last closed window (Sec. 3, Eqs. 11-14):
 * [0..1] Z_ccp, [2..3] Z_load (ohm, Re/Im), [4..5] Gamma, [6] |Gamma|,
 * [7] P_source, [8] P_Rs, [9] series-element loss (P_IMN; R_b in circuit I),
 * [10] P_stray, [11] P_ccp, [12] P_forward, [13] P_ref (W), [14..15] first
 * harmonic of U_E (V, Re/Im), [16] mean U_E (the DC self-bias), [17] mean
 * I_ccp. */
int orc_circuit_diag(const orc_sim *s, double *out18) {
  for (int k = 0; k < 18; ++k) out18[k] = s->circ_out[k];
  return ORC_OK;
}

/* Test hooks. */
void orc_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out) { philox4x32_10(ctr, key, out); }
double orc_xs(const orc_sim *s, int proc, double E) { return xs_lookup(s, proc, E); }
double orc_scatter_cos(double E, double R) { return scatter_cos(E, R); }
void orc_turn(double *c, double cc, double phi) { turn(c, cc, phi); }

/* Advance only the circuit for n steps from the current step counter,
 * recording U_E after each step (circuit tests). */
int orc_circuit_run(orc_sim *s, int n, double *U_out) {
  for (int k = 0; k < n; ++k) {
    circuit_advance(s);
    diag_accumulate(s);
    s->step++;
    if (U_out) U_out[k] = s->U_E;
  }
  return ORC_OK;
}
