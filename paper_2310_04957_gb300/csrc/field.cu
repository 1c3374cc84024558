// field.cu -- assembly of the implicit field equation, plain FP64 PCG, node E
// field, field-energy integral for C_eq, circuit integrator and diagnostics.
//
// Eq. 1 of arXiv:2310.04957, div[(1+chi) eps grad phi] = -rho~, is discretised
// by finite volumes on the node-centred r-z grid: node a's control volume
// exchanges flux with each neighbour b through an edge conductance G_ab, and
// sum_b G_ab (phi_a - phi_b) = Q_a, the charge in the control volume.  G is the
// vacuum part (eps0 eps_r face area / length, from the geometry) plus the
// plasma part times the mean chi of the edge's two nodes.  Metal nodes are
// Dirichlet (powered at U_E, grounded at 0).
#include <cstdint>

#include "pic_device.cuh"
#include "pic_kernels.h"

namespace pic {

// Macro particles absorbed in the last step in tally slot k (species*3 + kind):
// the count, or for weighted particles the sum of their weight ratios.
__device__ __forceinline__ double absorbed(const unsigned long long *counters, int weighted, int k) {
  return weighted ? (double)counters[CNT_ABSW + k] * (1.0 / kCreditOne) : (double)counters[CNT_ABS + k];
}

// ---- assembly ---------------------------------------------------------------
// Node pass: chi (D1 susceptibility dt^2/(2 eps0) sum_s q_s^2 n_s/m_s), node
// charge (particles + surface), Dirichlet values.
__global__ void k_assemble_nodes(const FieldParams F) {
  const double UE = F.scalars[SC_UE];
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < F.nn; a += gridDim.x * blockDim.x) {
    double Qe = (double)F.dep[0][a] * F.dep_inv_scale;
    double Qi = (double)F.dep[1][a] * F.dep_inv_scale;
    double v = F.vnode[a];
    F.chi[a] = v > 0.0 ? (F.chi_coef[0] * Qe + F.chi_coef[1] * Qi) / v : 0.0;
    F.qrhs[a] = F.qw[0] * (Qe + (double)F.surf[0][a] * F.surf_scale) +
                F.qw[1] * (Qi + (double)F.surf[1][a] * F.surf_scale);
    int k = F.node_kind[a];
    if (F.vahedi) {
      if (k != 0) F.phi[a] = 0.0;  // phi_P: every electrode at 0 (Eq. 3)
    } else if (k == 1) {
      F.phi[a] = UE;
    } else if (k == 2) {
      F.phi[a] = 0.0;
    } else if (k >= 3) {
      F.phi[a] = F.drive.voltage(k - 3, F.scalars[SC_T]);
    }
  }
}

// Edge pass: each node writes its right and upper edge and the inverse of its
// diagonal (sum of its up to four edges).
__global__ void k_assemble_edges(const FieldParams F) {
  const int nr = F.nr, nz = F.nz, W = nr + 1;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < F.nn; a += gridDim.x * blockDim.x) {
    int j = a / W, i = a - j * W;
    double ca = F.chi[a];
    double d = 0.0;
    if (i < nr) {
      int e = j * nr + i;
      double g = F.Gvac_r[e] + 0.5 * (ca + F.chi[a + 1]) * F.Gpl_r[e];
      F.Gr[e] = g;
      d += g;
    }
    if (i > 0) {
      int e = j * nr + i - 1;
      d += F.Gvac_r[e] + 0.5 * (ca + F.chi[a - 1]) * F.Gpl_r[e];
    }
    if (j < nz) {
      int e = j * W + i;
      double g = F.Gvac_z[e] + 0.5 * (ca + F.chi[a + W]) * F.Gpl_z[e];
      F.Gz[e] = g;
      d += g;
    }
    if (j > 0) {
      int e = (j - 1) * W + i;
      d += F.Gvac_z[e] + 0.5 * (ca + F.chi[a - W]) * F.Gpl_z[e];
    }
    F.dinv[a] = (F.node_kind[a] == 0 && d > 0.0) ? 1.0 / d : 0.0;
  }
}

cudaError_t launch_assemble_edges_only(const FieldParams &F, cudaStream_t st) {
  int blocks = (F.nn + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_assemble_edges<<<blocks, 256, 0, st>>>(F);
  return cudaGetLastError();
}

__global__ void k_set_dirichlet(int nn, const int8_t *kind, double *phi, double U) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nn; a += gridDim.x * blockDim.x) {
    if (kind[a] == 1) phi[a] = U;
    else if (kind[a] >= 2) phi[a] = 0.0;  // grounded and driven metal
  }
}

cudaError_t launch_set_dirichlet(int nn, const int8_t *kind, double *phi, double U, cudaStream_t st) {
  int blocks = (nn + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_set_dirichlet<<<blocks, 256, 0, st>>>(nn, kind, phi, U);
  return cudaGetLastError();
}

__global__ void k_set_dirichlet_unit(int nn, const int8_t *kind, double *phi, int e) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nn; a += gridDim.x * blockDim.x)
    if (kind[a] != 0) phi[a] = kind[a] == e ? 1.0 : 0.0;
}

cudaError_t launch_set_dirichlet_unit(int nn, const int8_t *kind, double *phi, int e, cudaStream_t st) {
  int blocks = (nn + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_set_dirichlet_unit<<<blocks, 256, 0, st>>>(nn, kind, phi, e);
  return cudaGetLastError();
}

// Eq. 2 at the time of the field (scalars[SC_T]); at metal nodes it gives each
// electrode's voltage exactly (phi_P = 0 there, phi_L one-hot).
__global__ void k_vahedi_combine(const VahediParams V) {
  const double t = V.scalars[SC_T], UE = V.scalars[SC_UE];
  double U[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < V.drive.n; ++k) U[k] = V.drive.voltage(k, t);
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < V.nn; a += gridDim.x * blockDim.x) {
    double v = V.phiP[a] + UE * V.phiL[0][a];
    for (int k = 0; k < V.drive.n; ++k) v += U[k] * V.phiL[k + 1][a];
    V.phi[a] = v;
  }
}

cudaError_t launch_vahedi_combine(const VahediParams &V, cudaStream_t st) {
  int blocks = (V.nn + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_vahedi_combine<<<blocks, 256, 0, st>>>(V);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const FieldParams &F, cudaStream_t st) {
  int blocks = (F.nn + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_assemble_nodes<<<blocks, 256, 0, st>>>(F);
  k_assemble_edges<<<blocks, 256, 0, st>>>(F);
  return cudaGetLastError();
}

// ---- E field at nodes -----------------------------------------------------------
// E = -grad phi: central differences; E_r = 0 on the axis; one-sided at the
// domain edge; at a Dirichlet node with exactly one free neighbour along a
// direction, one-sided toward that neighbour.
__global__ void k_efield(const EfieldParams E) {
  const int nr = E.nr, nz = E.nz, W = nr + 1, nn = W * (nz + 1);
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nn; a += gridDim.x * blockDim.x) {
    int j = a / W, i = a - j * W;
    const double *phi = E.phi;
    bool dir = E.node_kind[a] != 0;
    double er, ez;
    if (i == 0) er = 0.0;
    else if (i == nr) er = -(phi[a] - phi[a - 1]) / E.dr;
    else {
      bool fl = E.node_kind[a - 1] == 0, fh = E.node_kind[a + 1] == 0;
      if (dir && fl && !fh) er = -(phi[a] - phi[a - 1]) / E.dr;
      else if (dir && fh && !fl) er = -(phi[a + 1] - phi[a]) / E.dr;
      else er = -(phi[a + 1] - phi[a - 1]) / (2.0 * E.dr);
    }
    if (j == 0) ez = -(phi[a + W] - phi[a]) / E.dz;
    else if (j == nz) ez = -(phi[a] - phi[a - W]) / E.dz;
    else {
      bool fl = E.node_kind[a - W] == 0, fh = E.node_kind[a + W] == 0;
      if (dir && fl && !fh) ez = -(phi[a] - phi[a - W]) / E.dz;
      else if (dir && fh && !fl) ez = -(phi[a + W] - phi[a]) / E.dz;
      else ez = -(phi[a + W] - phi[a - W]) / (2.0 * E.dz);
    }
    E.Er[a] = er;
    E.Ez[a] = ez;
    if (E.E32) E.E32[a] = make_float2((float)er, (float)ez);
    if (E.E64) E.E64[a] = make_double2(er, ez);
  }
}

cudaError_t launch_efield(const EfieldParams &E, cudaStream_t st) {
  int nn = (E.nr + 1) * (E.nz + 1);
  int blocks = (nn + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_efield<<<blocks, 256, 0, st>>>(E);
  return cudaGetLastError();
}

// ---- field energy (Eqs. 6-7) ------------------------------------------------------
// out[0] = sum over edges G (phi_a - phi_b)^2 (= 2 x energy = C_eq U^2),
// out[1] = Gauss-law charge on the powered nodes.  One CTA, fixed order.
__global__ void __launch_bounds__(1024) k_energy(int nr, int nz, const int8_t *node_kind, const double *Gr,
                                                 const double *Gz, const double *phi, double *out) {
  const int W = nr + 1, nn = W * (nz + 1);
  double e = 0.0, q = 0.0;
  for (int a = threadIdx.x; a < nn; a += blockDim.x) {
    int j = a / W, i = a - j * W;
    bool pa = node_kind[a] == 1;
    if (i < nr) {
      double d = phi[a] - phi[a + 1], g = Gr[j * nr + i];
      e += g * d * d;
      bool pb = node_kind[a + 1] == 1;
      if (pa && !pb) q += g * d;
      if (pb && !pa) q -= g * d;
    }
    if (j < nz) {
      double d = phi[a] - phi[a + W], g = Gz[j * W + i];
      e += g * d * d;
      bool pb = node_kind[a + W] == 1;
      if (pa && !pb) q += g * d;
      if (pb && !pa) q -= g * d;
    }
  }
  __shared__ double se[32], sq[32];
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  if ((threadIdx.x & 31) == 0) { se[threadIdx.x >> 5] = e; sq[threadIdx.x >> 5] = q; }
  __syncthreads();
  if (threadIdx.x < 32) {
    int nw = blockDim.x >> 5;
    e = threadIdx.x < nw ? se[threadIdx.x] : 0.0;
    q = threadIdx.x < nw ? sq[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if (threadIdx.x == 0) { out[0] = e; out[1] = q; }
  }
}

cudaError_t launch_energy(int nr, int nz, const int8_t *node_kind, const double *Gr, const double *Gz, const double *phi,
                          double *out2, cudaStream_t st) {
  k_energy<<<1, 1024, 0, st>>>(nr, nz, node_kind, Gr, Gz, phi, out2);
  return cudaGetLastError();
}

// ---- circuit (Eqs. 5, 8, 9, 10) ------------------------------------------------------
// Linear ODE y' = M y + s(t) of the circuit states with the electrode charge
// Q_E, U_E = Q_E / C_eq.  Trapezoidal rule with nsub substeps per dt:
// y_{k+1} = (I - h/2 M)^{-1} [(I + h/2 M) y_k + h/2 (s_k + s_{k+1})].
__device__ void circuit_matrix(const CircuitParams &C, double ceq, double M[6][6], double e_src[6], double e_conv[6],
                               int &n) {
  for (int r = 0; r < 6; ++r) {
    e_src[r] = e_conv[r] = 0.0;
    for (int k = 0; k < 6; ++k) M[r][k] = 0.0;
  }
  if (C.kind == 1) {  // Qb, Ib, QE
    double Rb = C.c[0], Lb = C.c[1], Cb = C.c[2];
    n = 3;
    M[0][1] = 1.0;
    M[1][0] = -1.0 / (Lb * Cb);
    M[1][1] = -Rb / Lb;
    M[1][2] = -1.0 / (Lb * ceq);
    M[2][1] = 1.0;
    e_src[1] = 1.0 / Lb;
    e_conv[2] = 1.0;
  } else {  // Q1, Q2, I2, Qccp, Istray, QE
    double Rs = C.c[0], Cm1 = C.c[1], Lm = C.c[2], Cm2 = C.c[3], Rm = C.c[4], Cs = C.c[5], Rst = C.c[6], Ls = C.c[7];
    n = 6;
    M[0][0] = -1.0 / (Rs * Cm1);
    M[0][1] = 1.0 / (Rs * Cm1);
    M[1][2] = 1.0;
    M[2][0] = 1.0 / (Lm * Cm1);
    M[2][1] = -1.0 / (Lm * Cm1) - 1.0 / (Lm * Cm2);
    M[2][2] = -Rm / Lm;
    M[2][5] = -1.0 / (Lm * ceq);
    M[3][2] = 1.0;
    M[3][4] = -1.0;
    M[4][1] = -1.0 / (Ls * Cs);
    M[4][3] = 1.0 / (Ls * Cs);
    M[4][4] = -Rst / Ls;
    M[4][5] = 1.0 / (Ls * ceq);
    M[5][2] = 1.0;
    M[5][4] = -1.0;
    e_src[0] = 1.0 / Rs;
    e_conv[5] = 1.0;
  }
}

// In-place Gauss-Jordan inverse with partial pivoting (n <= 6).
__device__ void invert6(int n, double A[6][6], double Inv[6][6]) {
  for (int r = 0; r < n; ++r)
    for (int k = 0; k < n; ++k) Inv[r][k] = r == k ? 1.0 : 0.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t;
        t = Inv[c][k]; Inv[c][k] = Inv[piv][k]; Inv[piv][k] = t;
      }
    double d = 1.0 / A[c][c];
    for (int k = 0; k < n; ++k) { A[c][k] *= d; Inv[c][k] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r][c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) { A[r][k] -= f * A[c][k]; Inv[r][k] -= f * Inv[c][k]; }
    }
  }
}

// Propagator of one time step: the n_sub trapezoidal substeps compose, for a
// fixed C_eq, into y_{n+1} = Phi y_n + Im(exp(i(w t_n + phase)) c) + g I_conv,
// with B = (I - h/2 M)^-1 (I + h/2 M), Phi = B^n_sub, and c, g the sums of
// the propagated source terms (the source is V sin(w t + phase)).  Rebuilt
// whenever C_eq changes.  prop layout: Phi[36], c_re[6], c_im[6], g[6], n.
__global__ void k_circuit_prepare(const CircuitParams C) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || C.kind == 0) return;
  double *S = C.scalars;
  const double two_pi = 6.283185307179586476925286766559;
  double ceq = S[SC_CEQ];
  double M[6][6], es[6], ec[6], A[6][6], Inv[6][6], B[6][6], Phi[6][6], T[6][6];
  int n;
  circuit_matrix(C, ceq, M, es, ec, n);
  double h = C.dt / C.nsub;
  for (int r = 0; r < n; ++r)
    for (int k = 0; k < n; ++k) A[r][k] = (r == k ? 1.0 : 0.0) - 0.5 * h * M[r][k];
  invert6(n, A, Inv);
  for (int r = 0; r < n; ++r)
    for (int k = 0; k < n; ++k) {
      double acc = 0.0;
      for (int m = 0; m < n; ++m) acc += Inv[r][m] * ((m == k ? 1.0 : 0.0) + 0.5 * h * M[m][k]);
      B[r][k] = acc;
      Phi[r][k] = r == k ? 1.0 : 0.0;
    }
  double cre[6] = {0, 0, 0, 0, 0, 0}, cim[6] = {0, 0, 0, 0, 0, 0}, g[6] = {0, 0, 0, 0, 0, 0};
  double srcv[6], srcg[6];
  for (int r = 0; r < n; ++r) {
    double a = 0.0, b = 0.0;
    for (int m = 0; m < n; ++m) { a += Inv[r][m] * es[m]; b += Inv[r][m] * ec[m]; }
    srcv[r] = 0.5 * h * C.V * a;  // Inv (h/2) e_src V
    srcg[r] = h * b;              // Inv h e_conv
  }
  for (int k = 0; k < C.nsub; ++k) {
    // acc <- B acc + term_k
    double nre[6], nim[6], ng[6];
    double ph0 = two_pi * C.f * k * h, ph1 = two_pi * C.f * (k + 1) * h;
    double er = cos(ph0) + cos(ph1), ei = sin(ph0) + sin(ph1);
    for (int r = 0; r < n; ++r) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int m = 0; m < n; ++m) { a += B[r][m] * cre[m]; b += B[r][m] * cim[m]; c += B[r][m] * g[m]; }
      nre[r] = a + srcv[r] * er;
      nim[r] = b + srcv[r] * ei;
      ng[r] = c + srcg[r];
    }
    for (int r = 0; r < n; ++r) { cre[r] = nre[r]; cim[r] = nim[r]; g[r] = ng[r]; }
    for (int r = 0; r < n; ++r)
      for (int q = 0; q < n; ++q) {
        double acc = 0.0;
        for (int m = 0; m < n; ++m) acc += B[r][m] * Phi[m][q];
        T[r][q] = acc;
      }
    for (int r = 0; r < n; ++r)
      for (int q = 0; q < n; ++q) Phi[r][q] = T[r][q];
  }
  double *o = C.prop;
  for (int r = 0; r < 6; ++r)
    for (int q = 0; q < 6; ++q) o[r * 6 + q] = (r < n && q < n) ? Phi[r][q] : 0.0;
  for (int r = 0; r < 6; ++r) {
    o[36 + r] = r < n ? cre[r] : 0.0;
    o[42 + r] = r < n ? cim[r] : 0.0;
    o[48 + r] = r < n ? g[r] : 0.0;
  }
  o[54] = n;
  // U_E = Q_E / C_eq (Eq. 5) with the C_eq this propagator was built for
  S[SC_UE] = S[SC_QE] / ceq;
}

__global__ void k_circuit(const CircuitParams C) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double *S = C.scalars;
  const double two_pi = 6.283185307179586476925286766559;
  double ceq = S[SC_CEQ];
  double Iconv = (C.qw[0] * absorbed(C.counters, C.weighted, 0) + C.qw[1] * absorbed(C.counters, C.weighted, 3)) / C.dt;
  S[SC_ICONV] = Iconv;
  uint32_t step = *C.step_ptr;
  if (C.kind == 0) {
    for (int k = 0; k < C.n_run; ++k) {
      double tn = (double)(step + k) * C.dt, t1 = tn + C.dt;
      double U0 = C.V * sin(two_pi * C.f * tn + C.phase);
      double U1 = C.V * sin(two_pi * C.f * t1 + C.phase);
      S[SC_UE] = U1;
      S[SC_QE] = ceq * U1;
      S[SC_ICCP] = ceq * (U1 - U0) / C.dt - Iconv;
      if (C.U_hist) C.U_hist[k] = U1;
    }
  } else {
    const double *pr = C.prop;
    const int n = (int)pr[54];
    double y[6];
    for (int r = 0; r < 6; ++r) y[r] = S[SC_Y0 + r];
    for (int k = 0; k < C.n_run; ++k) {
      double tn = (double)(step + k) * C.dt;
      double sn, cs;
      sincos(two_pi * C.f * tn + C.phase, &sn, &cs);
      double yn[6];
      for (int r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int m = 0; m < n; ++m) acc += pr[r * 6 + m] * y[m];
        // Im((cs + i sn)(c_re + i c_im)) = sn c_re + cs c_im
        yn[r] = acc + sn * pr[36 + r] + cs * pr[42 + r] + pr[48 + r] * Iconv;
      }
      for (int r = 0; r < n; ++r) y[r] = yn[r];
      double QE = y[n - 1];
      S[SC_QE] = QE;
      S[SC_UE] = QE / ceq;
      S[SC_ICCP] = C.kind == 1 ? y[1] : y[2] - y[4];
      if (C.U_hist) C.U_hist[k] = QE / ceq;
    }
    for (int r = 0; r < 6; ++r) S[SC_Y0 + r] = y[r];
  }
  S[SC_T] = (double)(step + C.n_run) * C.dt;
  if (C.step_inc) *C.step_inc = step + C.n_run;
}

cudaError_t launch_circuit_prepare(const CircuitParams &C, cudaStream_t st) {
  k_circuit_prepare<<<1, 32, 0, st>>>(C);
  return cudaGetLastError();
}

cudaError_t launch_circuit(const CircuitParams &C, cudaStream_t st) {
  k_circuit<<<1, 32, 0, st>>>(C);
  return cudaGetLastError();
}

// ---- diagnostics -----------------------------------------------------------------
// Circuit waveforms at t_{n+1} for the window's post-processing (Sec. 3): source
// voltage U_s, the current I_1 leaving the source, the matching network's
// input voltage U_in, U_E (= U_ccp) and I_ccp; and the element powers U_s I_1,
// R_s I_1^2, the series element's loss (R_m I_2^2; R_b I_b^2 in circuit I),
// the stray branch's loss R_stray I_stray^2, U_ccp I_ccp and U_in I_1.
__device__ void circuit_waveforms(const DiagParams &D, const double *S, double t1, double w[5], double p[6]) {
  const double two_pi = 6.283185307179586476925286766559;
  const double Us = D.V * sin(two_pi * D.f * t1 + D.phase);
  for (int k = 0; k < 6; ++k) p[k] = 0.0;
  const double UE = S[SC_UE], Iccp = S[SC_ICCP];
  if (D.kind == 2) {
    const double Uin = (S[SC_Y0 + 0] - S[SC_Y0 + 1]) / D.c[1];
    const double I1 = (Us - Uin) / D.c[0];
    const double I2 = S[SC_Y0 + 2], Ist = S[SC_Y0 + 4];
    w[0] = Us; w[1] = I1; w[2] = Uin;
    p[0] = Us * I1;
    p[1] = D.c[0] * I1 * I1;
    p[2] = D.c[4] * I2 * I2;
    p[3] = D.c[6] * Ist * Ist;
    p[5] = Uin * I1;
  } else if (D.kind == 1) {
    const double Ib = S[SC_Y0 + 1];
    w[0] = Us; w[1] = Ib; w[2] = Us;
    p[0] = Us * Ib;
    p[2] = D.c[0] * Ib * Ib;
    p[5] = Us * Ib;
  } else {
    w[0] = UE; w[1] = Iccp; w[2] = UE;
    p[0] = p[5] = UE * Iccp;
  }
  w[3] = UE;
  w[4] = Iccp;
  p[4] = UE * Iccp;
}

// Complex ratio (ar + i ai) / (br + i bi); 0 when the divisor vanishes.
__device__ void cdiv(double ar, double ai, double br, double bi, double &r, double &i) {
  const double d = br * br + bi * bi;
  r = d > 0.0 ? (ar * br + ai * bi) / d : 0.0;
  i = d > 0.0 ? (ai * br - ar * bi) / d : 0.0;
}

// Per step: running sums of node densities, ion charge to each surface kind,
// first-harmonic DFT of I_ccp and of the circuit waveforms at t_{n+1}, element
// power sums; then the step counter advances.
__global__ void k_diag(const DiagParams D) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < D.nn; a += gridDim.x * blockDim.x) {
    double v = D.vnode[a];
    if (v > 0.0) {
      D.dens_sum[0][a] += D.w[0] * (double)D.dep[0][a] * D.dep_inv_scale / v;
      D.dens_sum[1][a] += D.w[1] * (double)D.dep[1][a] * D.dep_inv_scale / v;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double *S = D.scalars;
    uint32_t step = *D.step_ptr;
    const double two_pi = 6.283185307179586476925286766559;
    double t1 = (double)(step + 1) * D.dt;
    double ph = two_pi * D.f * t1;
    const double cph = cos(ph), sph = sin(ph);
    S[SC_DFT_RE] += S[SC_ICCP] * cph;
    S[SC_DFT_IM] -= S[SC_ICCP] * sph;
    double w[5], p[6];
    circuit_waveforms(D, S, t1, w, p);
    for (int k = 0; k < 5; ++k) {
      S[SC_CW_RE + k] += w[k] * cph;
      S[SC_CW_IM + k] -= w[k] * sph;
    }
    for (int k = 0; k < 6; ++k) S[SC_CP + k] += p[k];
    S[SC_CDC + 0] += w[3];
    S[SC_CDC + 1] += w[4];
    for (int k = 0; k < 3; ++k) S[SC_IONQ + k] += D.qw_ion * absorbed(D.counters, D.weighted, 3 + k);
    S[SC_WINCOUNT] += 1.0;
    *D.step_mut = step + 1;
  }
}

// Close a diagnostic window: averages over the window's steps, reset sums.
__global__ void k_diag_window(const DiagParams D) {
  double N = D.scalars[SC_WINCOUNT];
  if (N <= 0.0) return;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < D.nn; a += gridDim.x * blockDim.x) {
    for (int s = 0; s < 2; ++s) {
      D.dens_avg[s][a] = D.dens_sum[s][a] / N;
      D.dens_sum[s][a] = 0.0;
    }
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double *S = D.scalars;
    for (int k = 0; k < 3; ++k) { S[SC_IONCUR + k] = S[SC_IONQ + k] / (N * D.dt); S[SC_IONQ + k] = 0.0; }
    S[SC_I1_RE] = 2.0 * S[SC_DFT_RE] / N;
    S[SC_I1_IM] = 2.0 * S[SC_DFT_IM] / N;
    S[SC_DFT_RE] = S[SC_DFT_IM] = 0.0;
    // circuit post-processing (Sec. 3): Z = U_1 / I_1 of the fundamental (Eq. 11),
    // Gamma = (Z_load - R_s) / (Z_load + R_s) (Eq. 12), period-averaged powers
    // (Eq. 13), P_ref = P_forward |Gamma|^2 (Eq. 14)
    double *o = S + SC_COUT;
    cdiv(S[SC_CW_RE + 3], S[SC_CW_IM + 3], S[SC_CW_RE + 4], S[SC_CW_IM + 4], o[0], o[1]);
    cdiv(S[SC_CW_RE + 2], S[SC_CW_IM + 2], S[SC_CW_RE + 1], S[SC_CW_IM + 1], o[2], o[3]);
    o[4] = o[5] = 0.0;
    if (D.kind == 2) cdiv(o[2] - D.c[0], o[3], o[2] + D.c[0], o[3], o[4], o[5]);
    const double g2 = o[4] * o[4] + o[5] * o[5];
    o[6] = sqrt(g2);
    for (int k = 0; k < 6; ++k) o[7 + k] = S[SC_CP + k] / N;
    o[13] = o[12] * g2;
    o[14] = 2.0 * S[SC_CW_RE + 3] / N;
    o[15] = 2.0 * S[SC_CW_IM + 3] / N;
    o[16] = S[SC_CDC + 0] / N;  // mean U_E: the DC self-bias (Sec. 3, circuit I)
    o[17] = S[SC_CDC + 1] / N;
    for (int k = 0; k < 5; ++k) S[SC_CW_RE + k] = S[SC_CW_IM + k] = 0.0;
    for (int k = 0; k < 6; ++k) S[SC_CP + k] = 0.0;
    S[SC_CDC + 0] = S[SC_CDC + 1] = 0.0;
    S[SC_WINCOUNT] = 0.0;
    S[SC_WINDOWS] += 1.0;
  }
}

cudaError_t launch_diag(const DiagParams &D, cudaStream_t st) {
  int blocks = (D.nn + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_diag<<<blocks, 256, 0, st>>>(D);
  return cudaGetLastError();
}

cudaError_t launch_diag_window(const DiagParams &D, cudaStream_t st) {
  int blocks = (D.nn + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_diag_window<<<blocks, 256, 0, st>>>(D);
  return cudaGetLastError();
}

}  // namespace pic
