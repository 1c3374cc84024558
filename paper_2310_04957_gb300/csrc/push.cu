// push.cu -- the particle phase of one time step (gather, D1 correction,
// absorption, null-collision MCC, predictor with cylindrical rotation,
// re-bin into the next store, deposit of counts), fused in one kernel.
//
// Method (arXiv:2310.04957, Sec. 2): direct-implicit (D1) push -- the particle
// is first moved with the field it has not yet seen (predictor), the field
// solve at t_{n+1} then corrects it by dt^2/2 a_{n+1} -- null-collision MCC of
// electrons and Ar+ in argon, deposition of charge and of the implicit
// susceptibility (both from the same per-species node counts).
//
// One CTA = one tile of TX x TY cells of one species.  It reads the tile's bins
// (contiguous slots), pushes every particle in registers, claims a slot in the
// particle's new bin of the write store (warp-aggregated: lanes with the same
// new bin share one atomicAdd on the bin's fill counter), and deposits the
// four node weights as 2^-26 fixed-point integers: summed over lanes of the
// same new cell with redux.sync, added to a shared-memory node tile (tile +
// halo), and flushed with one 64-bit global add per tile node.  Integer sums
// are exact and order-independent.
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
// Reciprocal and reciprocal square root: FP32 uses the correctly rounded
// reciprocal and one Newton step on the hardware rsqrt estimate (error ~1 ulp,
// unbiased); FP64 keeps IEEE division and square root.
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
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

// Electron null-collision test (Sec. 2, Vahedi's method): -1 for a null
// collision, else the process (0 elastic, 1 excitation, 2 ionization).  Returns
// the energy E (eV) and the uniforms u2, u3 its kinematics use.
template <typename T>
__device__ __forceinline__ int mcc_electron_choose(const PushParams<T> &P, const Part<T> &p, T &E, T &u2, T &u3) {
  T u[4];
  draw4(P, p.id, 0u, 0u, u);
  if (!(u[0] < P.pcoll[0])) return -1;
  T v2 = p.vr * p.vr + p.vt * p.vt + p.vz * p.vz;
  T speed = m_sqrt(v2);
  if (!(speed > (T)0)) return -1;
  E = P.e_per_v2[0] * v2;
  u2 = u[2];
  u3 = u[3];
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
  T E = (T)0, u2 = (T)0, u3 = (T)0;
  const int c = mcc_electron_choose(P, p, E, u2, u3);
  if (c >= 0) mcc_electron_apply(P, p, c, E, u2, u3, be, bi);
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

template <typename T>
__device__ __forceinline__ Outcome advance(const PushParams<T> &P, int s, Part<T> &p, Part<T> &be, Part<T> &bi,
                                           const typename V2<T>::type en[4]) {
  Outcome o{0, -1, 0, -1, 0};
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
  if (!in_plasma(P, p.ci, p.cj)) {
    o.abs_node = exit_node(P, p.ci, p.fr, p.cj, p.fz);
    o.abs_kind = (int)__ldg(P.node_kind + o.abs_node);
    o.abs_kind = o.abs_kind == 1 ? 0 : (o.abs_kind == 2 ? 1 : 2);
    return o;
  }
  // MCC at x_n on v_{n-1/2}
  if (s == 0) {
    o.coll = mcc_electron(P, p, be, bi);
    o.birth = o.coll == 2;
  } else {
    o.coll = mcc_ion(P, p);
  }
  predict(P, p);
  if (!in_plasma(P, p.ci, p.cj)) {
    o.abs_node = exit_node(P, p.ci, p.fr, p.cj, p.fz);
    o.abs_kind = (int)__ldg(P.node_kind + o.abs_node);
    o.abs_kind = o.abs_kind == 1 ? 0 : (o.abs_kind == 2 ? 1 : 2);
    return o;
  }
  o.alive = 1;
  return o;
}

// Store a particle; its cell is implied by the bin except in the overflow
// region (ovf = true), where it is stored explicitly.
template <typename T>
__device__ __forceinline__ void store_particle(const StoreView<T> &S, int slot, const Part<T> &p, int cell_rowmajor,
                                               bool ovf) {
  S.pa[slot] = Vec4<T>{p.fr, p.fz, p.vr, p.vt};
  S.pb[slot] = Vec4<T>{p.vz, p.ar, p.at, p.az};
  S.id[slot] = p.id;
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

__device__ __forceinline__ void node_weights_q(const PushParams<float> &P, const Part<float> &p, unsigned long long W[4]) {
  float ir = (float)p.ci;
  float a = p.fr * (2.0f * ir + p.fr) * rcp(2.0f * ir + 1.0f);
  qweights32(a, p.fz, W);
}

__device__ __forceinline__ void node_weights_q(const PushParams<double> &P, const Part<double> &p,
                                               unsigned long long W[4]) {
  double ir = (double)p.ci;
  double a = p.fr * (2.0 * ir + p.fr) * rcp(2.0 * ir + 1.0);
  qweights(a, p.fz, P.dep_scale, P.dep_one, W);
}

// Deposit of one particle's 4 node weights straight to global memory.
template <typename T>
__device__ __forceinline__ void deposit_global(const PushParams<T> &P, int s, const Part<T> &p) {
  unsigned long long W[4];
  node_weights_q(P, p, W);
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
};

// 64-bit shared accumulator updated with 32-bit atomics (faster than 64-bit
// shared atomics): add to the low word, carry into the high word on wrap.
__device__ __forceinline__ void add_shared64(unsigned long long *t, unsigned v) {
  unsigned *w = reinterpret_cast<unsigned *>(t);
  unsigned old = atomicAdd(w, v);
  if (old + v < old) atomicAdd(w + 1, 1u);
}

// Warp-collective: write the alive lanes' particles into their new bins of the
// species' write store and deposit them.  All 32 lanes must call it.
template <typename T, int TX, int TY>
__device__ __forceinline__ void emit(const PushParams<T> &P, int s, bool alive, const Part<T> &p, const TileCtx &tc) {
  constexpr int TW = TX + 1 + 2 * kHalo;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const StoreView<T> &S = P.out[s];
  int key = alive ? bin_key<TX, TY>(p.ci, p.cj, P.map.ntx) : -1;
  unsigned peers = __match_any_sync(FULL, key);
  int leader = __ffs(peers) - 1;
  int base = 0;
  if (key >= 0 && lane == leader) base = atomicAdd(S.fill + key, __popc(peers));
  base = __shfl_sync(FULL, base, leader);
  if (key >= 0) {
    int pos = base + __popc(peers & ((1u << lane) - 1u));
    bool ovf = !(pos < __ldg(S.cap + key));
    int slot = ovf ? overflow_slot(P, S) : __ldg(S.start + key) + pos;
    if (slot >= 0) store_particle(S, slot, p, p.cj * P.nr + p.ci, ovf);
  }
  // deposit
  unsigned long long W[4] = {0, 0, 0, 0};
  if (alive) node_weights_q(P, p, W);
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
// directly.  Warp-collective.
template <int TX, int TY>
__device__ __forceinline__ void emit_home(const PushParams<float> &P, int s, bool alive, const Part<float> &p,
                                          const TileCtx &tc, int hci, int hcj, int hkey, unsigned acc[4]) {
  constexpr int TW = TX + 1 + 2 * kHalo;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const StoreView<float> &S = P.out[s];
  const bool home = alive && p.ci == hci && p.cj == hcj;
  const unsigned hm = __ballot_sync(FULL, home);
  int key = -1, pos = 0;
  if (hm) {
    const int hl = __ffs(hm) - 1;
    int hbase = 0;
    if (lane == hl) hbase = atomicAdd(S.fill + hkey, __popc(hm));
    hbase = __shfl_sync(FULL, hbase, hl);
    if (home) {
      key = hkey;
      pos = hbase + __popc(hm & lt);
    }
  }
  const bool other = alive && !home;
  if (__any_sync(FULL, other)) {
    const int okey = other ? bin_key<TX, TY>(p.ci, p.cj, P.map.ntx) : -1;
    const unsigned peers = __match_any_sync(FULL, okey);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (okey >= 0 && lane == leader) base = atomicAdd(S.fill + okey, __popc(peers));
    base = __shfl_sync(FULL, base, leader);
    if (other) {
      key = okey;
      pos = base + __popc(peers & lt);
    }
  }
  if (key >= 0) {
    const bool ovf = !(pos < __ldg(S.cap + key));
    const int slot = ovf ? overflow_slot(P, S) : __ldg(S.start + key) + pos;
    if (slot >= 0) store_particle(S, slot, p, p.cj * P.nr + p.ci, ovf);
  }
  if (!alive) return;
  unsigned long long W[4];
  node_weights_q(P, p, W);
  if (home) {
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] += (unsigned)W[k];
    return;
  }
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

// A newborn ion from an electron CTA: predictor, absorption, write, deposit
// (per lane: births are rare).
template <typename T, int TX, int TY>
__device__ __forceinline__ void emit_ion_birth(const PushParams<T> &P, Part<T> &bi) {
  predict(P, bi);
  if (!in_plasma(P, bi.ci, bi.cj)) {
    int node = exit_node(P, bi.ci, bi.fr, bi.cj, bi.fz);
    int k = (int)__ldg(P.node_kind + node);
    k = k == 1 ? 0 : (k == 2 ? 1 : 2);
    atomicAdd(P.counters + CNT_ABS + 3 + k, 1ull);
    if (k == 2) atomicAdd(P.surf[1] + node, 1ull);
    return;
  }
  const StoreView<T> &S = P.out[1];
  int key = bin_key<TX, TY>(bi.ci, bi.cj, P.map.ntx);
  int pos = atomicAdd(S.fill + key, 1);
  bool ovf = !(pos < __ldg(S.cap + key));
  int slot = ovf ? overflow_slot(P, S) : __ldg(S.start + key) + pos;
  if (slot >= 0) store_particle(S, slot, bi, bi.cj * P.nr + bi.ci, ovf);
  deposit_global(P, 1, bi);
}

// Warp-aggregated counter increment.
__device__ __forceinline__ void count_warp(unsigned long long *c, bool pred) {
  unsigned m = __ballot_sync(0xffffffffu, pred);
  if (m && (threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(c, (unsigned long long)__popc(m));
}

template <typename T>
__device__ __forceinline__ void tally(const PushParams<T> &P, int s, const Outcome &o, bool active) {
  if (!__any_sync(0xffffffffu, active && (o.abs_kind >= 0 || o.coll >= 0))) return;
  count_warp(P.counters + CNT_ABS + 3 * s + 0, active && o.abs_kind == 0);
  count_warp(P.counters + CNT_ABS + 3 * s + 1, active && o.abs_kind == 1);
  count_warp(P.counters + CNT_ABS + 3 * s + 2, active && o.abs_kind == 2);
  if (active && o.abs_kind == 2) atomicAdd(P.surf[s] + o.abs_node, 1ull);
  count_warp(P.counters + CNT_COLL + 3 * s + 0, active && o.coll == 0);
  count_warp(P.counters + CNT_COLL + 3 * s + 1, active && o.coll == 1);
  count_warp(P.counters + CNT_COLL + 3 * s + 2, active && o.coll == 2);
}

template <typename T>
__device__ __forceinline__ void load_particle(const StoreView<T> &S, int slot, Part<T> &p) {
  const Vec4<T> a = S.pa[slot], b = S.pb[slot];
  p.fr = a.x; p.fz = a.y; p.vr = a.z; p.vt = a.w;
  p.vz = b.x; p.ar = b.y; p.at = b.z; p.az = b.w;
  p.id = S.id[slot];
}

// The pair an ionization created (lanes with `birth`): predictor and absorption
// test of the newborn electron, warp-wide emit, then the newborn ion.
// Warp-collective.
template <typename T, int TX, int TY>
__device__ __forceinline__ void emit_births(const PushParams<T> &P, bool birth, Part<T> &be, Part<T> &bi,
                                            const TileCtx &tc) {
  if (!__any_sync(0xffffffffu, birth)) return;
  count_warp(P.counters + CNT_BORN + 0, birth);
  count_warp(P.counters + CNT_BORN + 1, birth);
  bool e_alive = false;
  if (!birth) {  // lanes without a birth take part in the warp-wide emit as dead lanes
    be.ci = 0;
    be.cj = 0;
  }
  if (birth) {
    predict(P, be);
    e_alive = in_plasma(P, be.ci, be.cj);
    if (!e_alive) {
      int node = exit_node(P, be.ci, be.fr, be.cj, be.fz);
      int k = (int)__ldg(P.node_kind + node);
      k = k == 1 ? 0 : (k == 2 ? 1 : 2);
      atomicAdd(P.counters + CNT_ABS + k, 1ull);
      if (k == 2) atomicAdd(P.surf[0] + node, 1ull);
    }
  }
  emit<T, TX, TY>(P, 0, e_alive, be, tc);
  if (birth) emit_ion_birth<T, TX, TY>(P, bi);
}

// Process one particle (already loaded) of species s: step, tallies, emit,
// births.  Warp-collective.
template <typename T, int TX, int TY>
__device__ __forceinline__ void process(const PushParams<T> &P, int s, bool active, Part<T> &p, const TileCtx &tc,
                                        const typename V2<T>::type en[4]) {
  // the newborn electron and ion are written in full by an ionizing collision
  // (and read only after one), so nothing of them is live during the push
  Part<T> be, bi;
  Outcome o{0, -1, 0, -1, 0};
  if (active) o = advance(P, s, p, be, bi, en);
  tally(P, s, o, active);
  emit<T, TX, TY>(P, s, active && o.alive, p, tc);
  emit_births<T, TX, TY>(P, active && o.birth, be, bi, tc);
}

// process() for an FP32 warp whose particles all start in its home cell.
template <int TX, int TY>
__device__ __forceinline__ void process_home(const PushParams<float> &P, int s, bool active, Part<float> &p,
                                             const TileCtx &tc, const float2 en[4], int hci, int hcj, int hkey,
                                             unsigned acc[4]) {
  Part<float> be, bi;
  Outcome o{0, -1, 0, -1, 0};
  if (active) o = advance(P, s, p, be, bi, en);
  tally(P, s, o, active);
  emit_home<TX, TY>(P, s, active && o.alive, p, tc, hci, hcj, hkey, acc);
  emit_births<float, TX, TY>(P, active && o.birth, be, bi, tc);
}

// One species' CTA (species known at compile time: its store views, charge
// to mass ratio and deposit array are fixed kernel-parameter operands, and only
// its own collision code is compiled in).
// Shared memory of a particle CTA (declared once in the kernel, shared by both
// species' code): the node tile of the deposit, the tile's bin prefix and
// offsets, and (FP32) the double-buffered next-round particle state.
template <typename T, int TX, int TY>
struct ParticleSmem {
  static constexpr int kW = sizeof(T) == 4 ? kThreads / 32 : 1;
  unsigned long long tile[(TX + 1 + 2 * kHalo) * (TY + 1 + 2 * kHalo)];
  int pre[TX * TY + 1];
  int cpre[TX * TY + 1];  // prefix of the bins' 32-particle chunk counts
  int off[TX * TY];
  Vec4<float> wa[kW][2][32], wb[kW][2][32];  // per-warp staging of the next chunk
  unsigned long long wid[kW][2][32];
};

template <typename T, int TX, int TY, int s>
__device__ __forceinline__ void particles_cta(const PushParams<T> &P, ParticleSmem<T, TX, TY> &sh) {
  constexpr int per = TX * TY;
  constexpr int TW = TX + 1 + 2 * kHalo, TH = TY + 1 + 2 * kHalo;
  const StoreView<T> &A = P.in[s];
  unsigned long long *smem = sh.tile;
  int *s_pre = sh.pre;
  int *s_off = sh.off;
  const int ntiles = P.map.ntiles();
  if ((int)blockIdx.x < ntiles) {
    const int tile = blockIdx.x;
    const int b0 = tile * per;
    const int tyi = tile / P.map.ntx, txi = tile - tyi * P.map.ntx;
    TileCtx tc;
    tc.tile = smem;
    tc.ci0 = txi * TX;
    tc.cj0 = tyi * TY;
    for (int k = threadIdx.x; k < TW * TH; k += blockDim.x) smem[k] = 0ull;
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
    __syncthreads();
    const int ntot = s_pre[per];
    if constexpr (sizeof(T) == 4) {
      // Warp w takes the w-th of eight equal runs of the tile's chunks (32
      // particles of one bin each, in bin order), so a warp stays in one bin
      // for a run of chunks.  While a chunk is processed the next one streams
      // from HBM into the warp's shared staging with cp.async (two 16-byte
      // copies and the id per lane; each lane reads back only its own copy).
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
      const int *s_cpre = sh.cpre;
      const int nch = s_cpre[per];
      const int c0 = (int)((long long)nch * w / ParticleSmem<T, TX, TY>::kW);
      const int c1 = (int)((long long)nch * (w + 1) / ParticleSmem<T, TX, TY>::kW);
      auto bin_of = [&](int c) {  // largest bin with s_cpre[bin] <= c
        int lo = 0;
#pragma unroll
        for (int step = per / 2; step >= 1; step >>= 1)
          if (lo + step < per && s_cpre[lo + step] <= c) lo += step;
        return lo;
      };
      auto issue = [&](int c, int buf) {
        if (c < c1) {
          const int bb = bin_of(c);
          const int k = (c - s_cpre[bb]) * 32 + lane;
          if (k < s_pre[bb + 1] - s_pre[bb]) {
            const int slot = s_off[bb] + k;
            cp_async16(&sh.wa[w][buf][lane], A.pa + slot);
            cp_async16(&sh.wb[w][buf][lane], A.pb + slot);
            cp_async8(&sh.wid[w][buf][lane], A.id + slot);
          }
        }
        cp_async_commit_group();
      };
      int home = -1, hci = 0, hcj = 0, nin = 0;
      unsigned acc[4] = {0u, 0u, 0u, 0u};
      issue(c0, 0);
      for (int c = c0, it = 0; c < c1; ++c, ++it) {
        const int buf = it & 1;
        issue(c + 1, buf ^ 1);
        cp_async_wait_group<1>();
        const int bb = bin_of(c);
        if (bb != home || nin == 63) {  // a lane's sum holds at most 63 quantised weights
          if (home >= 0) flush_home<TX, TY>(tc, hci, hcj, acc);
          home = bb;
          hci = tc.ci0 + (bb & (TX - 1));
          hcj = tc.cj0 + bb / TX;
          nin = 0;
        }
        ++nin;
        const int k = (c - s_cpre[bb]) * 32 + lane;
        const bool active = k < s_pre[bb + 1] - s_pre[bb];
        Part<T> p;
        p.ci = hci;
        p.cj = hcj;
        float2 en[4];
        if (active) {
          const Vec4<float> va = sh.wa[w][buf][lane], vb = sh.wb[w][buf][lane];
          p.fr = va.x; p.fz = va.y; p.vr = va.z; p.vt = va.w;
          p.vz = vb.x; p.ar = vb.y; p.at = vb.z; p.az = vb.w;
          p.id = sh.wid[w][buf][lane];
          gather_nodes(P, hci, hcj, en);  // E is small and L1/L2-resident
        }
        process_home<TX, TY>(P, s, active, p, tc, en, hci, hcj, b0 + bb, acc);
      }
      cp_async_wait_group<0>();
      if (home >= 0) flush_home<TX, TY>(tc, hci, hcj, acc);
    } else {
      for (int base = 0; base < ntot; base += blockDim.x) {
        int k = base + threadIdx.x;
        bool active = k < ntot;
        Part<T> p;
        p.ci = 0; p.cj = 0;
        typename V2<T>::type en[4];
        if (active) {
          int lo = 0;  // largest bin with s_pre[lo] <= k
#pragma unroll
          for (int step = per / 2; step >= 1; step >>= 1)
            if (lo + step < per && s_pre[lo + step] <= k) lo += step;
          int slot = s_off[lo] + (k - s_pre[lo]);
          load_particle(A, slot, p);
          p.ci = tc.ci0 + (lo & (TX - 1));
          p.cj = tc.cj0 + (lo / TX);
          gather_nodes(P, p.ci, p.cj, en);
        }
        process<T, TX, TY>(P, s, active, p, tc, en);
      }
    }
    __syncthreads();
    unsigned long long *d = P.dep[s];
    for (int k = threadIdx.x; k < TW * TH; k += blockDim.x) {
      unsigned long long v = smem[k];
      if (v) {
        int ni = tc.ci0 - kHalo + k % TW, nj = tc.cj0 - kHalo + k / TW;
        atomicAdd(d + nj * (P.nr + 1) + ni, v);
      }
    }
  } else {
    // overflow region of the read store: unsorted particles with explicit cells
    TileCtx tc{nullptr, 0, 0};
    const int novf = min(A.meta->ovf_n, A.capacity - A.meta->ovf_base);
    const int first = A.meta->ovf_base;
    const int stride = (gridDim.x - ntiles) * blockDim.x;
    for (int base = (blockIdx.x - ntiles) * blockDim.x; base < novf; base += stride) {
      int k = base + threadIdx.x;
      bool active = k < novf;
      Part<T> p;
      p.ci = 0; p.cj = 0;
      typename V2<T>::type en[4];
      if (active) {
        int slot = first + k;
        load_particle(A, slot, p);
        int c = A.cell[slot];
        p.cj = c / P.nr;
        p.ci = c - p.cj * P.nr;
        gather_nodes(P, p.ci, p.cj, en);
      }
      process<T, TX, TY>(P, s, active, p, tc, en);
    }
  }
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 5 : 2) k_particles(const PushParams<T> P) {
  __shared__ ParticleSmem<T, TX, TY> sh;
  if (blockIdx.y == 0) particles_cta<T, TX, TY, 0>(P, sh);
  else particles_cta<T, TX, TY, 1>(P, sh);
}

// ---------------------------------------------------------------------------
// Bin layout of the next write store, both species at once: room of a bin =
// fill + slack*fill + 8 for bins of plasma cells (0 elsewhere), or exactly the
// fill if that does not fit in 90 % of the capacity; start = exclusive scan of
// the rooms (clamped to the capacity); fill counters of the write store zeroed.
// Three launches: block sums, one scan of the block sums, block scans + writes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long room_of(int f, int plasma, int use_slack, float slack) {
  if (!plasma) return 0;
  return use_slack ? (long long)f + (long long)(slack * (float)f) + 8 : (long long)f;
}

template <int K>
__device__ __forceinline__ void block_sum_ll(long long v[K], long long *sh /* [K][32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    long long x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k * 32 + wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      long long x = lane < (int)(blockDim.x >> 5) ? sh[k * 32 + lane] : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) sh[k * 32] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sh[k * 32];
}

// Exclusive scan over the block (blockDim.x = 1024); returns the block total.
__device__ __forceinline__ long long block_exscan_ll(long long v, long long &excl, long long *sh /* [32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= d) t += y;
    }
    sh[lane] = t;  // inclusive warp totals
  }
  __syncthreads();
  long long before = wid > 0 ? sh[wid - 1] : 0;
  excl = before + x - v;
  long long total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(1024) k_layout_sums(const LayoutParams L) {
  __shared__ long long sh[3 * 32];
  const int s = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  long long v[3] = {0, 0, 0};
  if (b < L.nbins) {
    int f = L.fill_in[s][b], pl = L.bin_plasma[b];
    v[0] = room_of(f, pl, 1, L.slack);
    v[1] = room_of(f, pl, 0, L.slack);
    v[2] = f;
  }
  block_sum_ll<3>(v, sh);
  if (threadIdx.x < 3) L.part[((size_t)s * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = v[threadIdx.x];
}

__global__ void __launch_bounds__(1024) k_layout_scan(const LayoutParams L, int nblk) {
  __shared__ long long sh[3 * 32];
  __shared__ int s_use;
  const int s = blockIdx.x;
  const long long *part = L.part + (size_t)s * nblk * 4;
  long long v[3] = {0, 0, 0};
  if ((int)threadIdx.x < nblk) {
    v[0] = part[threadIdx.x * 4 + 0];
    v[1] = part[threadIdx.x * 4 + 1];
    v[2] = part[threadIdx.x * 4 + 2];
  }
  long long tot[3] = {v[0], v[1], v[2]};
  block_sum_ll<3>(tot, sh);
  if (threadIdx.x == 0) s_use = tot[0] <= (long long)(0.9 * (double)L.capacity[s]) ? 1 : 0;
  __syncthreads();
  int use = s_use;
  long long mine = use ? v[0] : v[1];
  long long excl;
  long long total = block_exscan_ll(mine, excl, sh);
  if ((int)threadIdx.x < nblk) L.boff[(size_t)s * nblk + threadIdx.x] = excl;
  if (threadIdx.x == 0) {
    L.use_slack[s] = use;
    L.meta_out[s]->ovf_base = (int)(total < L.capacity[s] ? total : L.capacity[s]);
    L.meta_out[s]->ovf_n = 0;
    L.meta_out[s]->total = 0;
    L.meta_in[s]->total = tot[2];
  }
}

__global__ void __launch_bounds__(1024) k_layout_write(const LayoutParams L) {
  __shared__ long long sh[32];
  const int s = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int use = L.use_slack[s];
  long long c = 0;
  if (b < L.nbins) c = room_of(L.fill_in[s][b], L.bin_plasma[b], use, L.slack);
  long long excl;
  block_exscan_ll(c, excl, sh);
  if (b < L.nbins) {
    long long run = L.boff[(size_t)s * gridDim.x + blockIdx.x] + excl;
    long long cap = L.capacity[s];
    if (run + c > cap) c = run < cap ? cap - run : 0;  // never hand out room past the buffer
    L.start[s][b] = (int)(run < cap ? run : cap);
    L.cap[s][b] = (int)c;
    L.fill_out[s][b] = 0;
  }
}

// Deposit of the read store's particles at their current x~ (start-up).
template <typename T>
__global__ void k_deposit_only(const PushParams<T> P) {
  const int s = blockIdx.y;
  const StoreView<T> &A = P.in[s];
  const int nb = P.map.nbins();
  // one warp per bin, then the overflow region
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int b = warp; b < nb; b += nwarps) {
    int f = A.fill[b], c = A.cap[b];
    int n = f < c ? f : c;
    int ci, cj;
    P.map.cell(b, ci, cj);
    for (int k = lane; k < n; k += 32) {
      Part<T> p;
      load_particle(A, A.start[b] + k, p);
      p.ci = ci; p.cj = cj;
      deposit_global(P, s, p);
    }
  }
  int novf = min(A.meta->ovf_n, A.capacity - A.meta->ovf_base);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < novf; k += gridDim.x * blockDim.x) {
    int slot = A.meta->ovf_base + k;
    Part<T> p;
    load_particle(A, slot, p);
    int c = A.cell[slot];
    p.cj = c / P.nr;
    p.ci = c - p.cj * P.nr;
    deposit_global(P, s, p);
  }
}

__global__ void k_philox(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x[4];
    philox10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], key[2 * i], key[2 * i + 1], x);
    out[4 * i] = x[0]; out[4 * i + 1] = x[1]; out[4 * i + 2] = x[2]; out[4 * i + 3] = x[3];
  }
}

// ---- host launchers ---------------------------------------------------------
template <typename T, int TX, int TY>
static cudaError_t launch_tiles(const PushParams<T> &P, cudaStream_t st) {
  dim3 grid(P.map.ntiles() + kOvfCtas, 2);
  k_particles<T, TX, TY><<<grid, kThreads, 0, st>>>(P);
  return cudaGetLastError();
}

// Tile shapes compiled in (cells in r x z); others are rejected at pic_init.
bool tile_supported(int tx, int ty) {
  return (tx == 2 && ty == 2) || (tx == 4 && ty == 2) || (tx == 2 && ty == 4) || (tx == 4 && ty == 4) ||
         (tx == 8 && ty == 4) || (tx == 8 && ty == 8) || (tx == 16 && ty == 4) || (tx == 16 && ty == 8) ||
         (tx == 32 && ty == 4) || (tx == 4 && ty == 8) || (tx == 8 && ty == 2);
}

template <typename T>
cudaError_t launch_particles(const PushParams<T> &P, cudaStream_t st) {
  const int tx = P.map.TX, ty = P.map.TY;
  if (tx == 2 && ty == 2) return launch_tiles<T, 2, 2>(P, st);
  if (tx == 4 && ty == 2) return launch_tiles<T, 4, 2>(P, st);
  if (tx == 2 && ty == 4) return launch_tiles<T, 2, 4>(P, st);
  if (tx == 8 && ty == 2) return launch_tiles<T, 8, 2>(P, st);
  if (tx == 4 && ty == 4) return launch_tiles<T, 4, 4>(P, st);
  if (tx == 8 && ty == 4) return launch_tiles<T, 8, 4>(P, st);
  if (tx == 8 && ty == 8) return launch_tiles<T, 8, 8>(P, st);
  if (tx == 16 && ty == 4) return launch_tiles<T, 16, 4>(P, st);
  if (tx == 16 && ty == 8) return launch_tiles<T, 16, 8>(P, st);
  if (tx == 32 && ty == 4) return launch_tiles<T, 32, 4>(P, st);
  if (tx == 4 && ty == 8) return launch_tiles<T, 4, 8>(P, st);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_deposit_only(const PushParams<T> &P, cudaStream_t st) {
  dim3 grid(1024, 2);
  k_deposit_only<T><<<grid, 256, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_layout(const LayoutParams &L, cudaStream_t st) {
  int nblk = (L.nbins + 1023) / 1024;
  if (nblk > 1024) return cudaErrorInvalidValue;
  k_layout_sums<<<dim3(nblk, 2), 1024, 0, st>>>(L);
  k_layout_scan<<<2, 1024, 0, st>>>(L, nblk);
  k_layout_write<<<dim3(nblk, 2), 1024, 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_philox(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_philox<<<blocks, 256, 0, st>>>(n, ctr, key, out);
  return cudaGetLastError();
}

template cudaError_t launch_particles<float>(const PushParams<float> &, cudaStream_t);

template cudaError_t launch_particles<double>(const PushParams<double> &, cudaStream_t);
template cudaError_t launch_deposit_only<float>(const PushParams<float> &, cudaStream_t);
template cudaError_t launch_deposit_only<double>(const PushParams<double> &, cudaStream_t);

}  // namespace pic
