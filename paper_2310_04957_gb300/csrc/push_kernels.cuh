// push_kernels.cuh -- the particle phase of one time step (gather, D1 correction,
// absorption, null-collision MCC, predictor with cylindrical rotation,
// re-bin into the next store, deposit of counts), fused in one kernel.
//
// Method (arXiv:2310.04957, Sec. 2): direct-implicit (D1) push -- the particle
// is first moved with the field it has not yet seen (predictor), the field
// solve at t_{n+1} then corrects it by dt^2/2 a_{n+1} -- null-collision MCC of
// electrons and Ar+ in argon, deposition of charge and of the implicit
// susceptibility (both from the same per-species node counts).
//
// One CTA = one tile of TX x TY cells of one species (plus a few CTAs for the
// overflow region).  It reads the tile's bins (contiguous slots); in FP32 each
// warp takes whole 32-particle chunks of one bin, staged by cp.async, and
// gathers E from a shared-memory copy of the tile's nodes.  Every
// particle is pushed in registers and claims a slot in its new bin of the write
// store: one ballot and one atomic for the lanes that stay in the warp's home
// cell, match_any groups for the others.  The four node weights are 2^-26
// fixed-point integers (2^-40 in FP64): home-cell weights are summed in
// registers and reduced once per bin, the others added to a shared-memory node
// tile (tile + halo), which is flushed with one 64-bit global add per node.
// Integer sums are exact and order-independent.  Weighted particles (ratios,
// splitting) are a separate template instance (WT).
#pragma once
#include <cstdint>

#include "pic_device.cuh"
#include "pic_kernels.h"

namespace pic {

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

// ---- math wrappers (library functions, not re-implemented) -----------------
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_log2(float x) { return log2f(x); }
__device__ __forceinline__ double m_log2(double x) { return log2(x); }
__device__ __forceinline__ float m_tan(float x) { return tanf(x); }
__device__ __forceinline__ double m_tan(double x) { return tan(x); }
__device__ __forceinline__ float m_atan(float x) { return atanf(x); }
__device__ __forceinline__ double m_atan(double x) { return atan(x); }
__device__ __forceinline__ void m_sincospi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void m_sincospi(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }
// Reciprocal and reciprocal square root: FP32 uses the hardware reciprocal
// approximation (__fdividef, at most 2 ulp; the arguments here are normal
// numbers of order 1..1e3) and one Newton step on the hardware rsqrt estimate
// (~1 ulp, unbiased); FP64 keeps IEEE division and square root.  The FP32
// path's tolerances (1e-5 per particle, FLIP_MARGIN in the parity proofs) are
// far above these errors.
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rsq(float q) {
  float y = rsqrtf(q);
  return y * (1.5f - 0.5f * q * y * y);
}
__device__ __forceinline__ double rsq(double q) { return 1.0 / sqrt(q); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bin of cell (i, j) for compile-time tile sizes (powers of two).
template <int TX, int TY>
__device__ __forceinline__ int bin_key(int i, int j, int ntx) {
  int tx = i / TX, ty = j / TY;
  return ((ty * ntx + tx) * TY + (j & (TY - 1))) * TX + (i & (TX - 1));
}

template <typename T>
struct Part {
  int ci, cj;
  T fr, fz, vr, vt, vz, ar, at, az;
  T w;  // weight ratio (1 for unweighted particles)
  unsigned long long id;
};

// Bring (c, f) back to f in [0,1).
template <typename T>
__device__ __forceinline__ void renorm(int &c, T &f) {
  T d = m_floor(f);
  c += (int)d;
  f -= d;
  if (f >= (T)1) { f -= (T)1; c += 1; }
  if (f < (T)0) f = (T)0;
}

template <typename T>
__device__ __forceinline__ bool in_plasma(const PushParams<T> &P, int ci, int cj) {
  if (ci < 0 || ci >= P.nr || cj < 0 || cj >= P.nz) return false;
  return __ldg(P.cell_kind + cj * P.nr + ci) == 0;
}

// Tally slot of an exit through a node of kind k: 0 the powered electrode,
// 2 a free node (dielectric surface charge), 1 any other metal (grounded or
// voltage-driven).
__device__ __forceinline__ int tally_kind(int k) { return k == 1 ? 0 : (k == 0 ? 2 : 1); }

// Node nearest to an exit point given in cell units (position clamped into the domain).
template <typename T>
__device__ __forceinline__ int exit_node(const PushParams<T> &P, int ci, T fr, int cj, T fz) {
  int ni = ci >= P.nr ? P.nr : ci + (fr >= (T)0.5 ? 1 : 0);
  int nj = cj < 0 ? 0 : (cj >= P.nz ? P.nz : cj + (fz >= (T)0.5 ? 1 : 0));
  if (ni < 0) ni = 0;
  return nj * (P.nr + 1) + ni;
}

// Cross sections at energy E (eV): linear interpolation between the bracketing
// log-spaced table nodes, clamped outside the table.  xs_interval returns the
// interval k with E_k <= E < E_{k+1} (-1 below the table, n-1 above it): a guess
// from log2 E, corrected by one node either way.
template <typename T>
__device__ __forceinline__ int xs_interval(const PushParams<T> &P, T E) {
  const T *Et = P.xs_E;
  const int n = P.n_xs;
  if (E <= __ldg(Et)) return -1;
  if (E >= __ldg(Et + n - 1)) return n - 1;
  int k;
  if constexpr (sizeof(T) == 4) k = (int)((__log2f(E) - P.log2E0) * P.inv_dlog2);
  else k = (int)((m_log2(E) - P.log2E0) * P.inv_dlog2);
  k = k < 0 ? 0 : (k > n - 2 ? n - 2 : k);
  if (E < __ldg(Et + k) && k > 0) --k;
  else if (E >= __ldg(Et + k + 1) && k < n - 2) ++k;
  return k;
}

// sigma of process `proc` on interval k (FP64: the table's own arithmetic).
template <typename T>
__device__ __forceinline__ T xs_at(const PushParams<T> &P, int proc, int k, T E) {
  const T *S = P.xs_S + proc * P.n_xs;
  if (k < 0) return __ldg(S);
  if (k >= P.n_xs - 1) return __ldg(S + P.n_xs - 1);
  T e0 = __ldg(P.xs_E + k), e1 = __ldg(P.xs_E + k + 1);
  T s0 = __ldg(S + k), s1 = __ldg(S + k + 1);
  return s0 + (E - e0) / (e1 - e0) * (s1 - s0);
}

// The three electron cross sections (elastic, excitation, ionization) at E.
__device__ __forceinline__ void xs_electron(const PushParams<float> &P, float E, float s[3]) {
  const int k = xs_interval(P, E);
  if (k < 0 || k >= P.n_xs - 1) {
#pragma unroll
    for (int p = 0; p < 3; ++p) s[p] = __ldg(P.xs_S + p * P.n_xs + (k < 0 ? 0 : P.n_xs - 1));
    return;
  }
  const float4 a = __ldg(P.xs_g + 3 * k), b = __ldg(P.xs_g + 3 * k + 1);
  const float dE = E - __ldg(P.xs_E + k);
  s[0] = a.x + dE * b.x;
  s[1] = a.y + dE * b.y;
  s[2] = a.z + dE * b.z;
}
__device__ __forceinline__ void xs_electron(const PushParams<double> &P, double E, double s[3]) {
  const int k = xs_interval(P, E);
#pragma unroll
  for (int p = 0; p < 3; ++p) s[p] = xs_at(P, p, k, E);
}

// The two ion cross sections (isotropic, charge exchange) at table energy E.
__device__ __forceinline__ void xs_ion(const PushParams<float> &P, float E, float s[2]) {
  const int k = xs_interval(P, E);
  if (k < 0 || k >= P.n_xs - 1) {
#pragma unroll
    for (int p = 0; p < 2; ++p) s[p] = __ldg(P.xs_S + (3 + p) * P.n_xs + (k < 0 ? 0 : P.n_xs - 1));
    return;
  }
  const float4 c = __ldg(P.xs_g + 3 * k + 2);
  const float dE = E - __ldg(P.xs_E + k);
  s[0] = c.x + dE * c.z;
  s[1] = c.y + dE * c.w;
}
__device__ __forceinline__ void xs_ion(const PushParams<double> &P, double E, double s[2]) {
  const int k = xs_interval(P, E);
  s[0] = xs_at(P, 3, k, E);
  s[1] = xs_at(P, 4, k, E);
}

// Electron scattering angle (Vahedi & Surendra): cos chi = (2 + E - 2 (1+E)^R)/E,
// returned as (cos chi, sin chi).  FP64 keeps the plain form, sin chi =
// sqrt(1 - cos^2 chi).  In FP32 that square root loses accuracy as chi -> 0
// or pi, so with x = ((1+E)^R - 1)/E the angle is cos chi = 1 - 2x and
// sin chi = 2 sqrt(x (1-x)), where x and 1 - x = (1+E)(1 - (1+E)^(R-1))/E are
// both formed by expm1/log1p without cancellation (R and 1 - R are exact).
__device__ __forceinline__ void scatter_cs(float E, float R, float &cc, float &sc) {
  float x, y;
  if (E < 1e-6f) {
    x = R;
    y = 1.0f - R;
  } else {
    const float L = log1pf(E), inv = 1.0f / E;
    x = expm1f(R * L) * inv;
    y = -(1.0f + E) * expm1f(-(1.0f - R) * L) * inv;
  }
  x = fminf(fmaxf(x, 0.0f), 1.0f);
  y = fminf(fmaxf(y, 0.0f), 1.0f);
  cc = x < 0.5f ? 1.0f - 2.0f * x : 2.0f * y - 1.0f;
  sc = 2.0f * sqrtf(x * y);
}
__device__ __forceinline__ void scatter_cs(double E, double R, double &cc, double &sc) {
  double c = E < 1e-6 ? 1.0 - 2.0 * R : 1.0 - 2.0 * expm1(R * log1p(E)) / E;
  cc = c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
  sc = sqrt(1.0 - cc * cc > 0.0 ? 1.0 - cc * cc : 0.0);
}

// Turn unit vector d by the polar angle (cos cc, sin sc) and azimuth 2 pi u.
template <typename T>
__device__ __forceinline__ void turn(T d[3], T cc, T sc, T u) {
  T sp, cp;
  m_sincospi((T)2 * u, &sp, &cp);
  T st = m_sqrt(d[0] * d[0] + d[1] * d[1]);
  T o0, o1, o2;
  if (st > (T)1e-12) {
    T k = sc / st;
    o0 = d[0] * cc + k * (d[0] * d[2] * cp + d[1] * sp);
    o1 = d[1] * cc + k * (d[1] * d[2] * cp - d[0] * sp);
    o2 = d[2] * cc - sc * st * cp;
  } else {
    T sg = d[2] >= (T)0 ? (T)1 : (T)-1;
    o0 = sc * cp * sg;
    o1 = -sc * sp;
    o2 = cc * sg;
  }
  d[0] = o0; d[1] = o1; d[2] = o2;
}

// Isotropic polar angle from uniform u: cos theta = 1 - 2u, sin theta =
// 2 sqrt(u (1-u)) (exact in FP32; the FP64 path keeps sqrt(1 - cos^2)).
__device__ __forceinline__ void iso_cs(float u, float &ct, float &st) {
  ct = 1.0f - 2.0f * u;
  st = 2.0f * sqrtf(u * (1.0f - u));
}
__device__ __forceinline__ void iso_cs(double u, double &ct, double &st) {
  ct = 1.0 - 2.0 * u;
  st = sqrt(1.0 - ct * ct > 0.0 ? 1.0 - ct * ct : 0.0);
}

template <typename T>
__device__ __forceinline__ void draw4(const PushParams<T> &P, unsigned long long id, uint32_t call, uint32_t spc, T u[4]) {
  uint32_t x[4];
  philox10(__ldg(P.step_ptr), call, spc, P.seed, (uint32_t)id, (uint32_t)(id >> 32), x);
#pragma unroll
  for (int k = 0; k < 4; ++k) u[k] = unif24<T>(x[k]);
}

template <typename T>
__device__ __forceinline__ void box_muller(T ua, T ub, T &na, T &nb) {
  T rad = m_sqrt((T)-2 * m_log((T)1 - ua));
  T s, c;
  m_sincospi((T)2 * ub, &s, &c);
  na = rad * c;
  nb = rad * s;
}

template <typename T>
__device__ __forceinline__ unsigned long long child_id(const PushParams<T> &P, unsigned long long id, uint32_t k) {
  uint32_t x[4];
  philox10(__ldg(P.step_ptr), 0xB1B1u, k, P.seed, (uint32_t)id, (uint32_t)(id >> 32), x);
  return ((unsigned long long)x[0] | ((unsigned long long)x[1] << 32)) | (1ull << 63);
}

// Id of the second half of a particle split in this step: Philox4x32-10 of the
// counter (step, 0x5B17, 0, seed) under the parent's id, top bit set.
template <typename T>
__device__ __forceinline__ unsigned long long split_id(const PushParams<T> &P, unsigned long long id) {
  uint32_t x[4];
  philox10(__ldg(P.step_ptr), 0x5B17u, 0u, P.seed, (uint32_t)id, (uint32_t)(id >> 32), x);
  return ((unsigned long long)x[0] | ((unsigned long long)x[1] << 32)) | (1ull << 63);
}

// Splitting near the axis (Sec. 2): radial cell i < i_s has the target weight
// ratio (2i+1)/(2 i_s + 1), proportional to its volume (1 beyond); a particle
// entering it with more than twice that ratio is split into two halves.
template <typename T>
__device__ __forceinline__ bool splits(const PushParams<T> &P, int ci, T w) {
  if (ci >= P.split_cells) return false;
  return w > (T)2 * ((T)(2 * ci + 1) / (T)(2 * P.split_cells + 1));
}

// Fixed-point credit of an absorbed weighted particle (units of 2^-32).
__device__ __forceinline__ unsigned long long credit_units(float w) { return __float2ull_rn(w * 4294967296.0f); }
__device__ __forceinline__ unsigned long long credit_units(double w) { return __double2ull_rn(w * 4294967296.0); }

// Predictor of the D1 scheme with the cylindrical rotation, in cell units:
// u = v + dt/2 a-bar; X = r + dt u_r, Y = dt u_theta; the radial displacement
// |(X,Y)| - r is formed as (dx (2r + dx) + Y^2) / (|(X,Y)| + r) so FP32 keeps
// the particle's offset inside its cell; (v_r, v_theta) and (a_r, a_theta)
// turn by the swept angle.
template <typename T>
__device__ __forceinline__ void predict(const PushParams<T> &P, Part<T> &p) {
  T ur = p.vr + P.hdt * p.ar, ut = p.vt + P.hdt * p.at, uz = p.vz + P.hdt * p.az;
  T r = ((T)p.ci + p.fr) * P.dr;
  T dx = P.dt * ur, Y = P.dt * ut;
  T X = r + dx;
  T q = X * X + Y * Y;
  T ca = (T)1, sa = (T)0, rn = (T)0;
  if (q > (T)0) {
    T inv = rsq(q);
    rn = q * inv;
    ca = X * inv;
    sa = Y * inv;
  }
  T den = rn + r;
  T disp = den > (T)0 ? (dx * ((T)2 * r + dx) + Y * Y) * rcp(den) : (T)0;
  T vr = ca * p.vr + sa * p.vt, vt = -sa * p.vr + ca * p.vt;
  T ar = ca * p.ar + sa * p.at, at = -sa * p.ar + ca * p.at;
  p.vr = vr; p.vt = vt; p.ar = ar; p.at = at;
  p.fr += disp * P.inv_dr;
  p.fz += P.dt * uz * P.inv_dz;
  renorm(p.ci, p.fr);
  renorm(p.cj, p.fz);
}

// Outcome of one particle's step.
struct Outcome {
  int alive;      // 1 -> write to its new bin and deposit
  int abs_kind;   // -1 none, 0 powered, 1 grounded, 2 surface
  int abs_node;
  int coll;       // -1 none, else process index
  int birth;      // 1 -> electron + ion born at x_n (electrons only)
};

// Electron null-collision method (Sec. 2, Vahedi's method).  The test: the
// step's four uniforms u of the particle, a candidate if u0 < P_null.
template <typename T>
__device__ __forceinline__ bool electron_candidate(const PushParams<T> &P, const Part<T> &p, T u[4]) {
  draw4(P, p.id, 0u, 0u, u);
  return u[0] < P.pcoll[0];
}

// The process of a candidate, from u1 against the cumulative collision
// frequencies at its energy E (eV, returned): -1 null, else 0 elastic,
// 1 excitation, 2 ionization.  Its kinematics use u2 and u3.
template <typename T>
__device__ __forceinline__ int mcc_electron_select(const PushParams<T> &P, const Part<T> &p, const T u[4], T &E) {
  T v2 = p.vr * p.vr + p.vt * p.vt + p.vz * p.vz;
  T speed = m_sqrt(v2);
  if (!(speed > (T)0)) return -1;
  E = P.e_per_v2[0] * v2;
  T ng_v = P.n_gas * speed;
  T sg[3];
  xs_electron(P, E, sg);
  T nu_el = ng_v * sg[0];
  T nu_ex = E < P.thr_ex ? (T)0 : ng_v * sg[1];
  T nu_iz = E < P.thr_iz ? (T)0 : ng_v * sg[2];
  T x = u[1] * P.numax[0];
  if (x < nu_el) return 0;
  if (x < nu_el + nu_ex) return 1;
  if (x < nu_el + nu_ex + nu_iz) return 2;
  return -1;
}

// Kinematics of electron process `coll` at energy E (Vahedi & Surendra): the
// scattered velocity, and for an ionization the ejected electron `be` and the
// new ion `bi` (Maxwellian at the gas temperature) at the parent's x_n.
template <typename T>
__device__ __forceinline__ void mcc_electron_apply(const PushParams<T> &P, Part<T> &p, int coll, T E, T u2, T u3,
                                                   Part<T> &be, Part<T> &bi) {
  T speed = m_sqrt(p.vr * p.vr + p.vt * p.vt + p.vz * p.vz);
  T d[3] = {p.vr / speed, p.vt / speed, p.vz / speed};
  if (coll == 0) {
    T cc, sc;
    scatter_cs(E, u2, cc, sc);
    T frac = (T)1 - P.two_me_over_M * ((T)1 - cc);
    turn(d, cc, sc, u3);
    T sp = speed * m_sqrt(frac);
    p.vr = sp * d[0]; p.vt = sp * d[1]; p.vz = sp * d[2];
    return;
  }
  if (coll == 1) {
    T En = E - P.thr_ex;
    T cc, sc;
    scatter_cs(En, u2, cc, sc);
    turn(d, cc, sc, u3);
    T sp = m_sqrt(En * P.v2_per_e[0]);
    p.vr = sp * d[0]; p.vt = sp * d[1]; p.vz = sp * d[2];
    return;
  }
  T Eex = E - P.thr_iz;
  T Eej = P.B_ej * m_tan(u2 * m_atan(Eex / ((T)2 * P.B_ej)));
  T Esc = Eex - Eej;
  if (Esc < (T)0) Esc = (T)0;
  T w1[4], w2[4];
  draw4(P, p.id, 1u, 0u, w1);
  draw4(P, p.id, 2u, 0u, w2);
  T ds[3] = {d[0], d[1], d[2]}, de[3] = {d[0], d[1], d[2]};
  T cc, sc;
  scatter_cs(Esc, w1[0], cc, sc);
  turn(ds, cc, sc, w1[1]);
  scatter_cs(Eej, w1[2], cc, sc);
  turn(de, cc, sc, w1[3]);
  T ssc = m_sqrt(Esc * P.v2_per_e[0]), sej = m_sqrt(Eej * P.v2_per_e[0]);
  p.vr = ssc * ds[0]; p.vt = ssc * ds[1]; p.vz = ssc * ds[2];
  be = p;
  be.vr = sej * de[0]; be.vt = sej * de[1]; be.vz = sej * de[2];
  be.ar = be.at = be.az = (T)0;
  be.id = child_id(P, p.id, 0u);
  T n0, n1, n2, n3;
  box_muller(w2[0], w2[1], n0, n1);
  box_muller(w2[2], w2[3], n2, n3);
  bi = be;
  bi.vr = P.vth_gas * n0; bi.vt = P.vth_gas * n1; bi.vz = P.vth_gas * n2;
  bi.id = child_id(P, p.id, 1u);
}

// Electron collision: test, then kinematics when one occurs.
template <typename T>
__device__ __forceinline__ int mcc_electron(const PushParams<T> &P, Part<T> &p, Part<T> &be, Part<T> &bi) {
  T u[4];
  if (!electron_candidate(P, p, u)) return -1;
  T E = (T)0;
  const int c = mcc_electron_select(P, p, u, E);
  if (c >= 0) mcc_electron_apply(P, p, c, E, u[2], u[3], be, bi);
  return c;
}

// Ion collision against a neutral drawn from the gas Maxwellian (Sec. 2):
// isotropic scattering in the centre-of-mass frame, or charge exchange.
template <typename T>
__device__ __forceinline__ int mcc_ion(const PushParams<T> &P, Part<T> &p) {
  T u[4];
  draw4(P, p.id, 0u, 1u, u);
  if (!(u[0] < P.pcoll[1])) return -1;
  T u1[4];
  draw4(P, p.id, 1u, 1u, u1);
  T n0, n1, n2, n3;
  box_muller(u1[0], u1[1], n0, n1);
  box_muller(u1[2], u1[3], n2, n3);
  T vn0 = P.vth_gas * n0, vn1 = P.vth_gas * n1, vn2 = P.vth_gas * n2;
  T g0 = p.vr - vn0, g1 = p.vt - vn1, g2 = p.vz - vn2;
  T gg = g0 * g0 + g1 * g1 + g2 * g2;
  T gm = m_sqrt(gg);
  T eps = P.e_per_v2[1] * gg;
  T ng_g = P.n_gas * gm;
  T sg[2];
  xs_ion(P, eps, sg);
  T nu_iso = ng_g * sg[0];
  T nu_cx = ng_g * sg[1];
  T x = u[1] * P.numax[1];
  if (x < nu_iso) {
    T ct, st;
    iso_cs(u[2], ct, st);
    T sp, cp;
    m_sincospi((T)2 * u[3], &sp, &cp);
    T wi = P.mi_frac, wn = (T)1 - P.mi_frac;  // m_i/(m_i+M), M/(m_i+M)
    T c0 = wi * p.vr + wn * vn0, c1 = wi * p.vt + wn * vn1, c2 = wi * p.vz + wn * vn2;
    p.vr = c0 + wn * gm * st * cp;
    p.vt = c1 + wn * gm * st * sp;
    p.vz = c2 + wn * gm * ct;
    return 0;
  }
  if (x < nu_iso + nu_cx) {
    p.vr = vn0; p.vt = vn1; p.vz = vn2;
    return 1;
  }
  return -1;
}

// Gather, correction, D1 filter, axis, absorption, MCC, predictor, absorption.
// E at the four nodes of cell (ci, cj): 00, 10, 01, 11.
template <typename T>
__device__ __forceinline__ void gather_nodes(const PushParams<T> &P, int ci, int cj, typename V2<T>::type e[4]) {
  using E2 = typename V2<T>::type;
  const E2 *E = reinterpret_cast<const E2 *>(P.E);
  int n00 = cj * (P.nr + 1) + ci;
  e[0] = E[n00];
  e[1] = E[n00 + 1];
  e[2] = E[n00 + P.nr + 1];
  e[3] = E[n00 + P.nr + 2];
}

// Cell (i, j) is in the plasma: (kci, kcj) is a cell known to be (the warp's
// home cell: particles are only stored in plasma cells), else the cell map decides.
template <typename T>
__device__ __forceinline__ bool in_plasma_k(const PushParams<T> &P, int ci, int cj, int kci, int kcj) {
  return (ci == kci && cj == kcj) || in_plasma(P, ci, cj);
}

// Gather, correction, D1 filter and velocity update, axis, absorption test at
// x_n.  Returns false (with the absorption in o) if the particle left the plasma.
// (kci, kcj): a cell known to be plasma (-1: none).
template <typename T>
__device__ __forceinline__ bool to_xn(const PushParams<T> &P, int s, Part<T> &p, const typename V2<T>::type en[4],
                                      Outcome &o, int kci = -1, int kcj = -1) {
  // gather E at x~_n with the deposit weights: linear in z, by annulus area in r
  T ir = (T)p.ci;
  T a = p.fr * ((T)2 * ir + p.fr) * rcp((T)2 * ir + (T)1);
  T b = p.fz;
  using E2 = typename V2<T>::type;
  const E2 e00 = en[0], e10 = en[1], e01 = en[2], e11 = en[3];
  T w00 = ((T)1 - a) * ((T)1 - b), w10 = a * ((T)1 - b), w01 = ((T)1 - a) * b, w11 = a * b;
  T Er = w00 * e00.x + w10 * e10.x + w01 * e01.x + w11 * e11.x;
  T Ez = w00 * e00.y + w10 * e10.y + w01 * e01.y + w11 * e11.y;
  T anr = P.qm[s] * Er, anz = P.qm[s] * Ez;
  // correction x_n = x~_n + dt^2/2 a_n
  p.fr += P.hdt2 * anr * P.inv_dr;
  p.fz += P.hdt2 * anz * P.inv_dz;
  // D1 time filter and velocity update
  p.ar = (T)0.5 * (anr + p.ar);
  p.at = (T)0.5 * p.at;
  p.az = (T)0.5 * (anz + p.az);
  p.vr += P.dt * p.ar; p.vt += P.dt * p.at; p.vz += P.dt * p.az;
  // axis: a radial move through r = 0 continues on the far side
  T rho = (T)p.ci + p.fr;
  if (rho < (T)0) {
    rho = -rho;
    p.ci = 0;
    p.fr = rho;
    p.vr = -p.vr; p.vt = -p.vt; p.ar = -p.ar; p.at = -p.at;
  }
  renorm(p.ci, p.fr);
  renorm(p.cj, p.fz);
  if (!in_plasma_k(P, p.ci, p.cj, kci, kcj)) {
    o.abs_node = exit_node(P, p.ci, p.fr, p.cj, p.fz);
    o.abs_kind = (int)__ldg(P.node_kind + o.abs_node);
    o.abs_kind = tally_kind(o.abs_kind);
    return false;
  }
  return true;
}

// Predictor to x~_{n+1} and the absorption test there.
template <typename T>
__device__ __forceinline__ void finish_push(const PushParams<T> &P, Part<T> &p, Outcome &o, int kci = -1,
                                            int kcj = -1) {
  predict(P, p);
  if (!in_plasma_k(P, p.ci, p.cj, kci, kcj)) {
    o.abs_node = exit_node(P, p.ci, p.fr, p.cj, p.fz);
    o.abs_kind = (int)__ldg(P.node_kind + o.abs_node);
    o.abs_kind = tally_kind(o.abs_kind);
    return;
  }
  o.alive = 1;
}

// The whole push of one particle with its collision in line.
template <typename T>
__device__ __forceinline__ Outcome advance(const PushParams<T> &P, int s, Part<T> &p, Part<T> &be, Part<T> &bi,
                                           const typename V2<T>::type en[4], int kci = -1, int kcj = -1) {
  Outcome o{0, -1, 0, -1, 0};
  if (!to_xn(P, s, p, en, o, kci, kcj)) return o;
  // MCC at x_n on v_{n-1/2}
  if (s == 0) {
    o.coll = mcc_electron(P, p, be, bi);
    o.birth = o.coll == 2;
  } else {
    o.coll = mcc_ion(P, p);
  }
  finish_push(P, p, o, kci, kcj);
  return o;
}

// Store a particle with id `id` and (weighted stores) weight ratio `w`; its
// cell is implied by the bin except in the overflow region (ovf = true), where
// it is stored explicitly.
template <bool WT, typename T>
__device__ __forceinline__ void store_particle(const StoreView<T> &S, int slot, const Part<T> &p, int cell_rowmajor,
                                               bool ovf, unsigned long long id, T w) {
  S.pa[slot] = Vec4<T>{p.fr, p.fz, p.vr, p.vt};
  S.pb[slot] = Vec4<T>{p.vz, p.ar, p.at, p.az};
  S.id[slot] = id;
  if constexpr (WT) S.w[slot] = w;
  if (ovf) S.cell[slot] = cell_rowmajor;
}

// Slot in the write store for a particle of bin `key`; -1 if dropped.
template <typename T>
__device__ __forceinline__ int overflow_slot(const PushParams<T> &P, const StoreView<T> &S) {
  int k = atomicAdd(&S.meta->ovf_n, 1);
  int slot = S.meta->ovf_base + k;
  if (slot >= S.capacity) {
    atomicAdd(P.counters + CNT_OVERFLOW, 1ull);
    atomicOr(P.flags, 1u);
    return -1;
  }
  return slot;
}

// Quantised deposit weights (sum exactly `one`): a = radial weight of node i+1,
// b = axial weight of node j+1.
template <typename T>
__device__ __forceinline__ void qweights(T a, T b, T scale, unsigned long long one, unsigned long long W[4]) {
  unsigned long long A = (unsigned long long)(a * scale + (T)0.5);
  unsigned long long B = (unsigned long long)(b * scale + (T)0.5);
  if (A > one) A = one;
  if (B > one) B = one;
  int sh = 63 - __clzll((long long)one);
  unsigned long long W11;
  if (sh <= 32) {
    W11 = (A * B + (one >> 1)) >> sh;
  } else {  // 128-bit product for the FP64 scale
    unsigned long long lo = A * B, hi = __umul64hi(A, B);
    unsigned long long add = lo + (one >> 1);
    hi += add < lo;
    W11 = (add >> sh) | (hi << (64 - sh));
  }
  W[3] = W11;
  W[1] = A - W11;
  W[2] = B - W11;
  W[0] = one - A - B + W11;
}

// FP32 path: 2^26 fixed point with 32-bit conversions and one 32x32->64
// product (the four weights still sum to exactly 2^26).
__device__ __forceinline__ void qweights32(float a, float b, unsigned long long W[4]) {
  const unsigned one = 1u << 26;
  unsigned A = __float2uint_rn(a * 67108864.0f), B = __float2uint_rn(b * 67108864.0f);
  A = A > one ? one : A;
  B = B > one ? one : B;
  unsigned W11 = (unsigned)(((unsigned long long)A * B + (1ull << 25)) >> 26);
  W[3] = W11;
  W[1] = A - W11;
  W[2] = B - W11;
  W[0] = one - A - B + W11;
}

// Weighted particle of ratio w: its total O = round(w one), the weights of
// nodes i+1 and j+1, A = round(w a one) and B = round(w b one), and of node
// (i+1, j+1), round(w a b one) kept inside [max(0, A+B-O), min(A, B)], so the
// four are non-negative and sum exactly to O.
template <typename T>
__device__ __forceinline__ void qweights_w(T a, T b, T w, T one, unsigned long long W[4]) {
  unsigned long long O, A, B, W11;
  if constexpr (sizeof(T) == 4) {
    O = __float2ull_rn(w * one);
    A = __float2ull_rn(a * w * one);
    B = __float2ull_rn(b * w * one);
    W11 = __float2ull_rn(a * b * w * one);
  } else {
    O = __double2ull_rn(w * one);
    A = __double2ull_rn(a * w * one);
    B = __double2ull_rn(b * w * one);
    W11 = __double2ull_rn(a * b * w * one);
  }
  A = A > O ? O : A;
  B = B > O ? O : B;
  const unsigned long long hi = A < B ? A : B, lo = A + B > O ? A + B - O : 0ull;
  W11 = W11 > hi ? hi : (W11 < lo ? lo : W11);
  W[3] = W11;
  W[1] = A - W11;
  W[2] = B - W11;
  W[0] = O - A - B + W11;
}

template <bool WT>
__device__ __forceinline__ void node_weights_q(const PushParams<float> &P, const Part<float> &p, unsigned long long W[4]) {
  float ir = (float)p.ci;
  float a = p.fr * (2.0f * ir + p.fr) * rcp(2.0f * ir + 1.0f);
  if constexpr (WT) qweights_w(a, p.fz, p.w, 67108864.0f, W);
  else qweights32(a, p.fz, W);
}

template <bool WT>
__device__ __forceinline__ void node_weights_q(const PushParams<double> &P, const Part<double> &p,
                                               unsigned long long W[4]) {
  double ir = (double)p.ci;
  double a = p.fr * (2.0 * ir + p.fr) * rcp(2.0 * ir + 1.0);
  if constexpr (WT) qweights_w(a, p.fz, p.w, P.dep_scale, W);
  else qweights(a, p.fz, P.dep_scale, P.dep_one, W);
}

// Deposit of one particle's 4 node weights straight to global memory.
template <bool WT, typename T>
__device__ __forceinline__ void deposit_global(const PushParams<T> &P, int s, const Part<T> &p) {
  unsigned long long W[4];
  node_weights_q<WT>(P, p, W);
  int n00 = p.cj * (P.nr + 1) + p.ci;
  unsigned long long *d = P.dep[s];
  atomicAdd(d + n00, W[0]);
  atomicAdd(d + n00 + 1, W[1]);
  atomicAdd(d + n00 + P.nr + 1, W[2]);
  atomicAdd(d + n00 + P.nr + 2, W[3]);
}

struct TileCtx {
  unsigned long long *tile;  // shared node tile, (TX+1+2H) x (TY+1+2H), or nullptr
  int ci0, cj0;
  unsigned *cnt;             // the CTA's tallies in shared memory (Counter slots), flushed at its end
  unsigned long long *cntw;  // weighted absorption tallies (CNT_ABSW slots), likewise
};

// Charge of an absorbed particle of species s at `node`: the weighted tally
// (the count is tallied warp-wide by the caller) and, on a free node, the
// surface charge -- one count per particle, or its fixed-point weight.
template <bool WT, typename T>
__device__ __forceinline__ void credit(const PushParams<T> &P, const TileCtx &tc, int s, int kind, int node, T w) {
  if constexpr (WT) {
    const unsigned long long cu = credit_units(w);
    atomicAdd(tc.cntw + 3 * s + kind, cu);
    if (kind == 2) atomicAdd(P.surf[s] + node, cu);
  } else {
    if (kind == 2) atomicAdd(P.surf[s] + node, 1ull);
  }
}

// 64-bit shared accumulator updated with 32-bit atomics (faster than 64-bit
// shared atomics): add to the low word, carry into the high word on wrap.
__device__ __forceinline__ void add_shared64(unsigned long long *t, unsigned v) {
  unsigned *w = reinterpret_cast<unsigned *>(t);
  unsigned old = atomicAdd(w, v);
  if (old + v < old) atomicAdd(w + 1, 1u);
}

// Warp-aggregated increment of a CTA tally in shared memory.
__device__ __forceinline__ void count_warp(unsigned *c, bool pred) {
  unsigned m = __ballot_sync(0xffffffffu, pred);
  if (m && (threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(c, (unsigned)__popc(m));
}

// Add the CTA's tallies to the global counters: one atomic per non-zero slot
// (hundreds of warps on every SM bump the same few counters, so they meet in
// shared memory first).  Call after a block barrier.
template <bool WT>
__device__ __forceinline__ void flush_counts(unsigned long long *counters, const unsigned *cnt,
                                             const unsigned long long *cntw) {
  if (threadIdx.x < CNT_N && cnt[threadIdx.x]) atomicAdd(counters + threadIdx.x, (unsigned long long)cnt[threadIdx.x]);
  if (WT && threadIdx.x < 6 && cntw[threadIdx.x]) atomicAdd(counters + CNT_ABSW + threadIdx.x, cntw[threadIdx.x]);
}

// Warp-collective slot claim: the lanes with key >= 0 take consecutive slots of
// bin `key` of write store S (one atomic per group of lanes with the same key)
// and store particle p there with id `id` and weight ratio w.  Returns the
// lane's group (its match_any mask).
template <bool WT, typename T>
__device__ __forceinline__ unsigned claim_store(const PushParams<T> &P, const StoreView<T> &S, int key,
                                                const Part<T> &p, unsigned long long id, T w) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(FULL, key);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (key >= 0 && lane == leader) base = atomicAdd(S.fill + key, __popc(peers));
  base = __shfl_sync(FULL, base, leader);
  if (key >= 0) {
    const int pos = base + __popc(peers & ((1u << lane) - 1u));
    const bool ovf = !(pos < __ldg(S.cap + key));
    const int slot = ovf ? overflow_slot(P, S) : __ldg(S.start + key) + pos;
    if (slot >= 0) store_particle<WT>(S, slot, p, p.cj * P.nr + p.ci, ovf, id, w);
  }
  return peers;
}

// Second halves of the weighted particles that split on entering their new
// cell (lanes with `split`): the same state with half the ratio and the split
// id, stored in the same bin.  The caller stores the first half with half the
// ratio; the deposit takes the whole ratio once.  Warp-collective.
template <bool WT, typename T, int TX, int TY>
__device__ __forceinline__ void emit_split(const PushParams<T> &P, int s, bool split, const Part<T> &p,
                                           const TileCtx &tc) {
  if constexpr (WT) {
    if (!__any_sync(0xffffffffu, split)) return;
    count_warp(tc.cnt + CNT_SPLIT + s, split);
    claim_store<WT>(P, P.out[s], split ? bin_key<TX, TY>(p.ci, p.cj, P.map.ntx) : -1, p,
                    split ? split_id(P, p.id) : 0ull, p.w * (T)0.5);
  }
}

// Warp-collective: write the alive lanes' particles into their new bins of the
// species' write store and deposit them.  All 32 lanes must call it.
template <typename T, int TX, int TY, bool WT>
__device__ __forceinline__ void emit(const PushParams<T> &P, int s, bool alive, const Part<T> &p, const TileCtx &tc) {
  constexpr int TW = TX + 1 + 2 * kHalo;
  const int lane = threadIdx.x & 31;
  bool split = false;
  if constexpr (WT) split = alive && splits(P, p.ci, p.w);
  const int key = alive ? bin_key<TX, TY>(p.ci, p.cj, P.map.ntx) : -1;
  const unsigned peers = claim_store<WT>(P, P.out[s], key, p, p.id, split ? p.w * (T)0.5 : p.w);
  emit_split<WT, T, TX, TY>(P, s, split, p, tc);
  // deposit
  unsigned long long W[4] = {0, 0, 0, 0};
  if (alive) node_weights_q<WT>(P, p, W);
  int li = p.ci - tc.ci0 + kHalo, lj = p.cj - tc.cj0 + kHalo;
  bool in_tile = tc.tile != nullptr && li >= 0 && lj >= 0 && li < TX + 2 * kHalo && lj < TY + 2 * kHalo;
  if (sizeof(T) == 4) {
    // 32-bit fixed point: each group of lanes with the same new cell (disjoint
    // masks from match_any) reduces its four node weights with one redux.sync
    // per node; the group's lanes then share the four atomic adds by rank.
    unsigned s4[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) s4[k] = __reduce_add_sync(peers, (unsigned)W[k]);
    if (key >= 0) {
      const int rank = __popc(peers & ((1u << lane) - 1u)), size = __popc(peers);
      const int n00 = p.cj * (P.nr + 1) + p.ci;
      for (int n = rank; n < 4; n += size) {
        unsigned v = n == 0 ? s4[0] : (n == 1 ? s4[1] : (n == 2 ? s4[2] : s4[3]));
        if (!v) continue;
        int dx = n & 1, dy = n >> 1;
        if (in_tile) add_shared64(tc.tile + (lj + dy) * TW + li + dx, v);
        else atomicAdd(P.dep[s] + n00 + dy * (P.nr + 1) + dx, (unsigned long long)v);
      }
    }
  } else if (alive) {
    if (in_tile) {
      unsigned long long *t = tc.tile + lj * TW + li;
      atomicAdd(t, W[0]);
      atomicAdd(t + 1, W[1]);
      atomicAdd(t + TW, W[2]);
      atomicAdd(t + TW + 1, W[3]);
    } else {
      int n00 = p.cj * (P.nr + 1) + p.ci;
      unsigned long long *d = P.dep[s];
      atomicAdd(d + n00, W[0]);
      atomicAdd(d + n00 + 1, W[1]);
      atomicAdd(d + n00 + P.nr + 1, W[2]);
      atomicAdd(d + n00 + P.nr + 2, W[3]);
    }
  }
}

// ---- FP32: warps process whole chunks of one bin -------------------------------------
// A warp's 32 particles come from one cell (its "home"), and in a step most of
// them stay there.  Those claim their slots in the home bin with one ballot and
// one atomic, and add their four node weights to per-lane registers; the warp
// reduces the registers into the shared node tile once per bin (flush_home).
// Particles that leave the home cell claim by match_any groups and deposit
// directly.  Both claim atomics are issued before the deposit and their results
// read after it, so the deposit arithmetic covers the atomics' latency.
// Warp-collective.
template <int TX, int TY, bool WT>
__device__ __forceinline__ void emit_home(const PushParams<float> &P, int s, bool alive, const Part<float> &p,
                                          const TileCtx &tc, int hci, int hcj, int hkey, unsigned acc[4]) {
  constexpr int TW = TX + 1 + 2 * kHalo;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const StoreView<float> &S = P.out[s];
  const bool home = alive && p.ci == hci && p.cj == hcj;
  bool split = false;
  if constexpr (WT) split = alive && splits(P, p.ci, p.w);
  const unsigned hm = __ballot_sync(FULL, home);
  const bool other = alive && !home;
  const unsigned om = __ballot_sync(FULL, other);
  int hbase = 0, hl = 0;
  if (hm) {
    hl = __ffs(hm) - 1;
    if (lane == hl) hbase = atomicAdd(S.fill + hkey, __popc(hm));
  }
  int okey = -1, base = 0, leader = 0;
  unsigned peers = 0u;
  if (om) {
    okey = other ? bin_key<TX, TY>(p.ci, p.cj, P.map.ntx) : -1;
    peers = __match_any_sync(FULL, okey);
    leader = __ffs(peers) - 1;
    if (okey >= 0 && lane == leader) base = atomicAdd(S.fill + okey, __popc(peers));
  }
  // the claimed bin's capacity and start, loaded ahead of the deposit as well
  const int k0 = home ? hkey : okey;
  int cap0 = 0, start0 = 0;
  if (k0 >= 0) {
    cap0 = __ldg(S.cap + k0);
    start0 = __ldg(S.start + k0);
  }
  if (alive) {
    unsigned long long W[4];
    node_weights_q<WT>(P, p, W);
    if (home) {
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += (unsigned)W[k];
    } else {
      const int li = p.ci - tc.ci0 + kHalo, lj = p.cj - tc.cj0 + kHalo;
      const bool in_tile = tc.tile != nullptr && li >= 0 && lj >= 0 && li < TX + 2 * kHalo && lj < TY + 2 * kHalo;
      const int n00 = p.cj * (P.nr + 1) + p.ci;
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        const int dx = n & 1, dy = n >> 1;
        if (!W[n]) continue;
        if (in_tile) add_shared64(tc.tile + (lj + dy) * TW + li + dx, (unsigned)W[n]);
        else atomicAdd(P.dep[s] + n00 + dy * (P.nr + 1) + dx, W[n]);
      }
    }
  }
  int key = -1, pos = 0;
  if (hm) {
    hbase = __shfl_sync(FULL, hbase, hl);
    if (home) {
      key = hkey;
      pos = hbase + __popc(hm & lt);
    }
  }
  if (om) {
    base = __shfl_sync(FULL, base, leader);
    if (other) {
      key = okey;
      pos = base + __popc(peers & lt);
    }
  }
  if (key >= 0) {
    const bool ovf = !(pos < cap0);
    const int slot = ovf ? overflow_slot(P, S) : start0 + pos;
    if (slot >= 0) store_particle<WT>(S, slot, p, p.cj * P.nr + p.ci, ovf, p.id, split ? p.w * 0.5f : p.w);
  }
  emit_split<WT, float, TX, TY>(P, s, split, p, tc);
}

// Add the warp's home-cell node weights (per-lane sums below 2^32) to the
// shared node tile: each sum split into 16-bit halves, so the warp totals of
// the halves fit 32 bits and one redux.sync each forms them.  Warp-collective.
template <int TX, int TY>
__device__ __forceinline__ void flush_home(const TileCtx &tc, int hci, int hcj, unsigned acc[4]) {
  constexpr int TW = TX + 1 + 2 * kHalo;
  const unsigned FULL = 0xffffffffu;
  unsigned long long t[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned lo = __reduce_add_sync(FULL, acc[k] & 0xffffu), hi = __reduce_add_sync(FULL, acc[k] >> 16);
    t[k] = ((unsigned long long)hi << 16) + lo;
    acc[k] = 0u;
  }
  const int lane = threadIdx.x & 31;
  if (lane < 4) {
    const unsigned long long v = lane == 0 ? t[0] : (lane == 1 ? t[1] : (lane == 2 ? t[2] : t[3]));
    const int li = hci - tc.ci0 + kHalo + (lane & 1), lj = hcj - tc.cj0 + kHalo + (lane >> 1);
    if (v) atomicAdd(tc.tile + lj * TW + li, v);
  }
}

// Absorption of a particle at an exit point: the tally slot kind (0 powered,
// 1 grounded, 2 free node) and the node.
template <typename T>
__device__ __forceinline__ int exit_kind(const PushParams<T> &P, const Part<T> &p, int &node) {
  node = exit_node(P, p.ci, p.fr, p.cj, p.fz);
  const int k = (int)__ldg(P.node_kind + node);
  return tally_kind(k);
}

// A newborn ion from an electron CTA: predictor, absorption, write (and split),
// deposit (per lane: births are rare).
template <typename T, int TX, int TY, bool WT>
__device__ __forceinline__ void emit_ion_birth(const PushParams<T> &P, Part<T> &bi, const TileCtx &tc) {
  predict(P, bi);
  if (!in_plasma(P, bi.ci, bi.cj)) {
    int node;
    const int k = exit_kind(P, bi, node);
    atomicAdd(tc.cnt + CNT_ABS + 3 + k, 1u);
    credit<WT>(P, tc, 1, k, node, bi.w);
    return;
  }
  bool split = false;
  if constexpr (WT) split = splits(P, bi.ci, bi.w);
  const StoreView<T> &S = P.out[1];
  const int key = bin_key<TX, TY>(bi.ci, bi.cj, P.map.ntx);
  const int halves = split ? 2 : 1;
  const int pos = atomicAdd(S.fill + key, halves);
  for (int h = 0; h < halves; ++h) {
    const bool ovf = !(pos + h < __ldg(S.cap + key));
    const int slot = ovf ? overflow_slot(P, S) : __ldg(S.start + key) + pos + h;
    if (slot >= 0)
      store_particle<WT>(S, slot, bi, bi.cj * P.nr + bi.ci, ovf, h ? split_id(P, bi.id) : bi.id,
                         split ? bi.w * (T)0.5 : bi.w);
  }
  if (split) atomicAdd(tc.cnt + CNT_SPLIT + 1, 1u);
  deposit_global<WT>(P, 1, bi);
}

template <typename T, bool WT>
__device__ __forceinline__ void tally(const PushParams<T> &P, int s, const Outcome &o, bool active, const Part<T> &p,
                                      const TileCtx &tc) {
  if (!__any_sync(0xffffffffu, active && (o.abs_kind >= 0 || o.coll >= 0))) return;
  // each lane sets bit 10k of its absorption word for kind k and of its collision word
  // for process k; one redux.sync per word sums the warp's counts into three 10-bit
  // fields (at most 32 each), which lanes 0..5 add to the CTA's tallies
  const unsigned pa = (active && o.abs_kind >= 0) ? 1u << (10 * o.abs_kind) : 0u;
  const unsigned pc = (active && o.coll >= 0) ? 1u << (10 * o.coll) : 0u;
  const unsigned sa = __reduce_add_sync(0xffffffffu, pa), scl = __reduce_add_sync(0xffffffffu, pc);
  const int lane = threadIdx.x & 31;
  if (lane < 6) {
    const int k = lane < 3 ? lane : lane - 3;
    const unsigned v = ((lane < 3 ? sa : scl) >> (10 * k)) & 1023u;
    if (v) atomicAdd(tc.cnt + (lane < 3 ? CNT_ABS : CNT_COLL) + 3 * s + k, v);
  }
  if (active && o.abs_kind >= 0) credit<WT>(P, tc, s, o.abs_kind, o.abs_node, p.w);
}

template <bool WT, typename T>
__device__ __forceinline__ void load_particle(const StoreView<T> &S, int slot, Part<T> &p) {
  const Vec4<T> a = S.pa[slot], b = S.pb[slot];
  p.fr = a.x; p.fz = a.y; p.vr = a.z; p.vt = a.w;
  p.vz = b.x; p.ar = b.y; p.at = b.z; p.az = b.w;
  p.id = S.id[slot];
  p.w = WT ? S.w[slot] : (T)1;
}

// The pair an ionization created (lanes with `birth`, both with the parent's
// weight ratio): predictor and absorption test of the newborn electron,
// warp-wide emit, then the newborn ion.  Warp-collective.  Out of line: few
// warps have a birth in a step, and the inlined body costs the common path
// registers and instruction-cache room (measured 2.6 % of the kernel).
template <typename T, int TX, int TY, bool WT>
__device__ __noinline__ void emit_births_body(const PushParams<T> &P, bool birth, Part<T> &be, Part<T> &bi,
                                              const TileCtx &tc);

template <typename T, int TX, int TY, bool WT>
__device__ __forceinline__ void emit_births(const PushParams<T> &P, bool birth, Part<T> &be, Part<T> &bi,
                                            const TileCtx &tc) {
  if (!__any_sync(0xffffffffu, birth)) return;
  emit_births_body<T, TX, TY, WT>(P, birth, be, bi, tc);
}

template <typename T, int TX, int TY, bool WT>
__device__ __noinline__ void emit_births_body(const PushParams<T> &P, bool birth, Part<T> &be, Part<T> &bi,
                                              const TileCtx &tc) {
  count_warp(tc.cnt + CNT_BORN + 0, birth);
  count_warp(tc.cnt + CNT_BORN + 1, birth);
  bool e_alive = false;
  if (!birth) {  // lanes without a birth take part in the warp-wide emit as dead lanes
    be.ci = 0;
    be.cj = 0;
  }
  if (birth) {
    predict(P, be);
    e_alive = in_plasma(P, be.ci, be.cj);
    if (!e_alive) {
      int node;
      const int k = exit_kind(P, be, node);
      atomicAdd(tc.cnt + CNT_ABS + k, 1u);
      credit<WT>(P, tc, 0, k, node, be.w);
    }
  }
  emit<T, TX, TY, WT>(P, 0, e_alive, be, tc);
  if (birth) emit_ion_birth<T, TX, TY, WT>(P, bi, tc);
}

// Process one particle (already loaded) of species s: step, tallies, emit,
// births.  Warp-collective.
template <typename T, int TX, int TY, bool WT>
__device__ __forceinline__ void process(const PushParams<T> &P, int s, bool active, Part<T> &p, const TileCtx &tc,
                                        const typename V2<T>::type en[4]) {
  // the newborn electron and ion are written in full by an ionizing collision
  // (and read only after one), so nothing of them is live during the push
  Part<T> be, bi;
  Outcome o{0, -1, 0, -1, 0};
  if (active) o = advance(P, s, p, be, bi, en);
  tally<T, WT>(P, s, o, active, p, tc);
  emit<T, TX, TY, WT>(P, s, active && o.alive, p, tc);
  emit_births<T, TX, TY, WT>(P, active && o.birth, be, bi, tc);
}

// process() for an FP32 warp whose particles all start in its home cell.
template <int TX, int TY, bool WT>
__device__ __forceinline__ void process_home(const PushParams<float> &P, int s, bool active, Part<float> &p,
                                             const TileCtx &tc, const float2 en[4], int hci, int hcj, int hkey,
                                             unsigned acc[4]) {
  Part<float> be, bi;
  Outcome o{0, -1, 0, -1, 0};
  if (active) o = advance(P, s, p, be, bi, en, hci, hcj);
  tally<float, WT>(P, s, o, active, p, tc);
  emit_home<TX, TY, WT>(P, s, active && o.alive, p, tc, hci, hcj, hkey, acc);
  emit_births<float, TX, TY, WT>(P, active && o.birth, be, bi, tc);
}

// Shared memory of a particle CTA (declared once in the kernel, shared by both
// species' code): the node tile of the deposit, the tile's bin prefix and
// offsets, and (FP32) the double-buffered next-chunk particle state.
template <typename T, int TX, int TY, bool WT>
struct ParticleSmem {
  static constexpr int kW = sizeof(T) == 4 ? kThreads / 32 : 1;
  unsigned long long tile[(TX + 1 + 2 * kHalo) * (TY + 1 + 2 * kHalo)];
  int pre[TX * TY + 1];
  int cpre[TX * TY + 1];  // prefix of the bins' 32-particle chunk counts
  int off[TX * TY];
  Vec4<float> wa[kW][2][32], wb[kW][2][32];  // per-warp staging of the next chunk
  unsigned long long wid[kW][2][32];
  float ww[WT ? kW : 1][2][32];  // weight ratios (weighted particles)
  float2 et[(TX + 1) * (TY + 1)];  // E at the tile's nodes (FP32 tile CTAs)
  unsigned cnt[CNT_N];   // the CTA's tallies
  unsigned long long cntw[6];  // and its weighted absorption tallies
};

// One species' CTA (species known at compile time: its store views, charge
// to mass ratio and deposit array are fixed kernel-parameter operands, and only
// its own collision code is compiled in).  A tile CTA takes the particles of
// its tile's bins; an overflow CTA (blockIdx.x >= tiles) a share of the read
// store's overflow region, whose particles carry their cells.  Both run the
// same loop with one call of the push, so a particle's arithmetic is the same
// code whichever region it was stored in (which region that is depends on the
// order of the slot claims of the previous step).
template <typename T, int TX, int TY, int s, bool WT>
__device__ __forceinline__ void particles_cta(const PushParams<T> &P, ParticleSmem<T, TX, TY, WT> &sh) {
  constexpr int per = TX * TY;
  constexpr int TW = TX + 1 + 2 * kHalo, TH = TY + 1 + 2 * kHalo;
  const StoreView<T> &A = P.in[s];
  unsigned long long *smem = sh.tile;
  int *s_pre = sh.pre;
  int *s_off = sh.off;
  const int ntiles = P.map.ntiles();
  const bool ovf_cta = (int)blockIdx.x >= ntiles;
  const int tile = blockIdx.x;
  const int b0 = tile * per;
  TileCtx tc{nullptr, 0, 0, sh.cnt, sh.cntw};
  if (threadIdx.x < CNT_N) sh.cnt[threadIdx.x] = 0u;
  if (WT && threadIdx.x < 6) sh.cntw[threadIdx.x] = 0ull;
  if (!ovf_cta) {
    const int tyi = tile / P.map.ntx, txi = tile - tyi * P.map.ntx;
    tc.tile = smem;
    tc.ci0 = txi * TX;
    tc.cj0 = tyi * TY;
    for (int k = threadIdx.x; k < TW * TH; k += blockDim.x) smem[k] = 0ull;
    if constexpr (sizeof(T) == 4) {
      for (int k = threadIdx.x; k < (TX + 1) * (TY + 1); k += blockDim.x) {
        const int ni = tc.ci0 + k % (TX + 1), nj = tc.cj0 + k / (TX + 1);
        float2 v = make_float2(0.f, 0.f);
        if (ni <= P.nr && nj <= P.nz) v = reinterpret_cast<const float2 *>(P.E)[nj * (P.nr + 1) + ni];
        sh.et[k] = v;
      }
    }
    if (threadIdx.x < 32) {
      // prefix of the tile's in-bin counts and chunk counts
      int carry = 0, ccarry = 0;
#pragma unroll
      for (int c0 = 0; c0 < per; c0 += 32) {
        int b = c0 + threadIdx.x;
        int n = 0, off = 0;
        if (b < per) {
          int f = A.fill[b0 + b], cp = A.cap[b0 + b];
          n = f < cp ? f : cp;
          off = A.start[b0 + b];
        }
        const int nc = (n + 31) >> 5;
        int incl = n, cincl = nc;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          int y = __shfl_up_sync(0xffffffffu, incl, d), yc = __shfl_up_sync(0xffffffffu, cincl, d);
          if ((int)threadIdx.x >= d) { incl += y; cincl += yc; }
        }
        if (b < per) { s_pre[b] = carry + incl - n; s_off[b] = off; sh.cpre[b] = ccarry + cincl - nc; }
        carry += __shfl_sync(0xffffffffu, incl, 31);
        ccarry += __shfl_sync(0xffffffffu, cincl, 31);
      }
      if (threadIdx.x == 0) { s_pre[per] = carry; sh.cpre[per] = ccarry; }
    }
  }
  __syncthreads();
  // overflow region of the read store: unsorted particles with explicit cells
  const int novf = ovf_cta ? min(A.meta->ovf_n, A.capacity - A.meta->ovf_base) : 0;
  const int first = ovf_cta ? A.meta->ovf_base : 0;
  const int nocta = (int)gridDim.x - ntiles;
  if constexpr (sizeof(T) == 4) {
    // Chunks of 32 particles.  A tile CTA's chunks are its bins' particles in
    // bin order, 32 of one bin each; warp w takes the w-th of eight equal runs
    // of them, so a warp stays in one bin (its "home") for a run of chunks.  An
    // overflow CTA's warps take every (overflow warps)-th chunk of the region.
    // While a chunk is processed the next one streams from HBM into the warp's
    // shared staging with cp.async (two 16-byte copies and the id per lane, and
    // the ratio of weighted particles; each lane reads back only its own copy).
    constexpr int kW = ParticleSmem<T, TX, TY, WT>::kW;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int *s_cpre = sh.cpre;
    int c0, c1, cstep;
    if (!ovf_cta) {
      const int nch = s_cpre[per];
      c0 = (int)((long long)nch * w / kW);
      c1 = (int)((long long)nch * (w + 1) / kW);
      cstep = 1;
    } else {
      c0 = ((int)blockIdx.x - ntiles) * kW + w;
      c1 = (novf + 31) >> 5;
      cstep = nocta * kW;
    }
    auto bin_of = [&](int c) {  // largest bin with s_cpre[bin] <= c
      int lo = 0;
#pragma unroll
      for (int step = per / 2; step >= 1; step >>= 1)
        if (lo + step < per && s_cpre[lo + step] <= c) lo += step;
      return lo;
    };
    // slot of this lane's particle in chunk c; false if the chunk has none for it
    auto locate = [&](int c, int bb, int &slot) {
      if (ovf_cta) {
        const int k = c * 32 + lane;
        slot = first + k;
        return k < novf;
      }
      const int k = (c - s_cpre[bb]) * 32 + lane;
      slot = s_off[bb] + k;
      return k < s_pre[bb + 1] - s_pre[bb];
    };
    auto issue = [&](int c, int buf) {
      if (c < c1) {
        int slot;
        if (locate(c, ovf_cta ? 0 : bin_of(c), slot)) {
          cp_async16(&sh.wa[w][buf][lane], A.pa + slot);
          cp_async16(&sh.wb[w][buf][lane], A.pb + slot);
          cp_async8(&sh.wid[w][buf][lane], A.id + slot);
          if (WT) cp_async4(&sh.ww[w][buf][lane], A.w + slot);
        }
      }
      cp_async_commit_group();
    };
    int home = -1, hci = -1, hcj = -1, nin = 0;
    unsigned acc[4] = {0u, 0u, 0u, 0u};
    issue(c0, 0);
    for (int c = c0, it = 0; c < c1; c += cstep, ++it) {
      const int buf = it & 1;
      issue(c + cstep, buf ^ 1);
      cp_async_wait_group<1>();
      int bb = 0;
      if (!ovf_cta) {
        bb = bin_of(c);
        if (bb != home || nin == 63) {  // a lane's sum holds at most 63 quantised weights
          if (home >= 0) flush_home<TX, TY>(tc, hci, hcj, acc);
          home = bb;
          hci = tc.ci0 + (bb & (TX - 1));
          hcj = tc.cj0 + bb / TX;
          nin = 0;
        }
        ++nin;
      }
      int slot;
      const bool active = locate(c, bb, slot);
      Part<T> p;
      p.ci = 0;
      p.cj = 0;
      float2 en[4];
      if (active) {
        const Vec4<float> va = sh.wa[w][buf][lane], vb = sh.wb[w][buf][lane];
        p.fr = va.x; p.fz = va.y; p.vr = va.z; p.vt = va.w;
        p.vz = vb.x; p.ar = vb.y; p.at = vb.z; p.az = vb.w;
        p.id = sh.wid[w][buf][lane];
        p.w = WT ? sh.ww[w][buf][lane] : 1.0f;
        if (ovf_cta) {
          const int cl = __ldg(A.cell + slot);
          p.cj = cl / P.nr;
          p.ci = cl - p.cj * P.nr;
        } else {
          p.ci = hci;
          p.cj = hcj;
        }
        if (ovf_cta) {
          gather_nodes(P, p.ci, p.cj, en);
        } else {  // the home cell's nodes, from the tile's copy of E
          const int e00 = (p.cj - tc.cj0) * (TX + 1) + p.ci - tc.ci0;
          en[0] = sh.et[e00];
          en[1] = sh.et[e00 + 1];
          en[2] = sh.et[e00 + TX + 1];
          en[3] = sh.et[e00 + TX + 2];
        }
      }
      // overflow chunks have no home (hci = -1): their lanes claim and deposit by groups
      process_home<TX, TY, WT>(P, s, active, p, tc, en, hci, hcj, b0 + bb, acc);
    }
    cp_async_wait_group<0>();
    if (home >= 0) flush_home<TX, TY>(tc, hci, hcj, acc);
  } else {
    const int nitems = ovf_cta ? novf : s_pre[per];
    const int bstart = ovf_cta ? ((int)blockIdx.x - ntiles) * (int)blockDim.x : 0;
    const int bstep = ovf_cta ? nocta * (int)blockDim.x : (int)blockDim.x;
    for (int base = bstart; base < nitems; base += bstep) {
      const int k = base + threadIdx.x;
      const bool active = k < nitems;
      Part<T> p;
      p.ci = 0; p.cj = 0;
      typename V2<T>::type en[4];
      if (active) {
        int slot;
        if (ovf_cta) {
          slot = first + k;
          const int cl = A.cell[slot];
          p.cj = cl / P.nr;
          p.ci = cl - p.cj * P.nr;
        } else {
          int lo = 0;  // largest bin with s_pre[lo] <= k
#pragma unroll
          for (int step = per / 2; step >= 1; step >>= 1)
            if (lo + step < per && s_pre[lo + step] <= k) lo += step;
          slot = s_off[lo] + (k - s_pre[lo]);
          p.ci = tc.ci0 + (lo & (TX - 1));
          p.cj = tc.cj0 + (lo / TX);
        }
        load_particle<WT>(A, slot, p);
        gather_nodes(P, p.ci, p.cj, en);
      }
      process<T, TX, TY, WT>(P, s, active, p, tc, en);
    }
  }
  __syncthreads();
  flush_counts<WT>(P.counters, sh.cnt, sh.cntw);
  if (!ovf_cta) {
    unsigned long long *d = P.dep[s];
    for (int k = threadIdx.x; k < TW * TH; k += blockDim.x) {
      unsigned long long v = smem[k];
      if (v) {
        int ni = tc.ci0 - kHalo + k % TW, nj = tc.cj0 - kHalo + k / TW;
        atomicAdd(d + nj * (P.nr + 1) + ni, v);
      }
    }
  }
}

template <typename T, int TX, int TY, bool WT>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 4 : 2) k_particles(const PushParams<T> P) {
  __shared__ ParticleSmem<T, TX, TY, WT> sh;
  if (blockIdx.y == 0) particles_cta<T, TX, TY, 0, WT>(P, sh);
  else particles_cta<T, TX, TY, 1, WT>(P, sh);
}

// ---- launch over the tile shapes compiled in ---------------------------------
template <typename T, int TX, int TY, bool W>
cudaError_t launch_tiles(const PushParams<T> &P, cudaStream_t st) {
  dim3 grid(P.map.ntiles() + kOvfCtas, 2);
  k_particles<T, TX, TY, W><<<grid, kThreads, 0, st>>>(P);
  return cudaGetLastError();
}

template <typename T, bool W>
cudaError_t launch_particles_tiles(const PushParams<T> &P, cudaStream_t st) {
  const int tx = P.map.TX, ty = P.map.TY;
  if (tx == 2 && ty == 2) return launch_tiles<T, 2, 2, W>(P, st);
  if (tx == 4 && ty == 2) return launch_tiles<T, 4, 2, W>(P, st);
  if (tx == 2 && ty == 4) return launch_tiles<T, 2, 4, W>(P, st);
  if (tx == 8 && ty == 2) return launch_tiles<T, 8, 2, W>(P, st);
  if (tx == 4 && ty == 4) return launch_tiles<T, 4, 4, W>(P, st);
  if (tx == 8 && ty == 4) return launch_tiles<T, 8, 4, W>(P, st);
  if (tx == 8 && ty == 8) return launch_tiles<T, 8, 8, W>(P, st);
  if (tx == 16 && ty == 4) return launch_tiles<T, 16, 4, W>(P, st);
  if (tx == 16 && ty == 8) return launch_tiles<T, 16, 8, W>(P, st);
  if (tx == 32 && ty == 4) return launch_tiles<T, 32, 4, W>(P, st);
  if (tx == 4 && ty == 8) return launch_tiles<T, 4, 8, W>(P, st);
  return cudaErrorInvalidValue;
}

}  // namespace pic
