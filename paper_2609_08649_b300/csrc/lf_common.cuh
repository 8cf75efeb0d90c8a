// Device math shared by the lens-equation kernels: scalar overloads (float / double),
// float-float (FP32 pair) accumulation, and the closed forms of each component.
//
// Closed forms (Sec. 2.1 quantities; profile forms of Keeton 2001 for the softened
// isothermal ellipsoid and its dPIE difference, Bartelmann 1996 for the spherical NFW):
//   SIE, frame (u, v) rotated by the position angle, psi~ = sqrt(q^2 (s^2 + u^2) + v^2),
//   e = sqrt(1 - q^2):  alpha_u = (b q / e) atan(e u / (psi~ + s)),
//                       alpha_v = (b q / e) atanh(e v / (psi~ + q^2 s)),
//   psi_uu = f (q^2 s^2 + v^2 + s psi~), psi_vv = f (s^2 + u^2 + s psi~), psi_uv = -f u v,
//   f = b q / (psi~ D), D = (1 + q^2) s^2 + 2 psi~ s + u^2 + v^2.
//   Round cored isothermal: alpha = b x / (S + s), S = sqrt(s^2 + r^2), and
//   psi_ij = kbar delta_ij + t x_i x_j with t = 2 (kappa - kbar) / r^2 = -b / (S (S + s)^2),
//   a form with no 0/0 at the centre.  dPIE = cored(core) - cored(cut).
//   NFW (unit kappa_s): kbar = 4 h(x) / x^2 and kappa = 2 (F - 1) / (1 - x^2), x = r / rs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include <type_traits>

#include "lf_cse_table.h"

#define LF_INLINE __device__ __forceinline__
#ifndef LF_NOINLINE
#define LF_NOINLINE __device__ __noinline__
#endif

// ------------------------------------------------------------------ scalar math ----
LF_INLINE float lf_rsqrt(float x) { return rsqrtf(x); }
LF_INLINE double lf_rsqrt(double x) { return rsqrt(x); }
LF_INLINE float lf_rcp(float x) { return __fdividef(1.0f, x); }
LF_INLINE double lf_rcp(double x) { return 1.0 / x; }
LF_INLINE float lf_sqrt(float x) { return sqrtf(x); }
LF_INLINE double lf_sqrt(double x) { return sqrt(x); }
LF_INLINE float lf_atan(float x) { return atanf(x); }
LF_INLINE double lf_atan(double x) { return atan(x); }
LF_INLINE float lf_atanh(float x) { return atanhf(x); }
LF_INLINE double lf_atanh(double x) { return atanh(x); }
LF_INLINE float lf_log(float x) { return logf(x); }
LF_INLINE double lf_log(double x) { return log(x); }
LF_INLINE float lf_log1p(float x) { return log1pf(x); }
LF_INLINE double lf_log1p(double x) { return log1p(x); }
LF_INLINE float lf_acos(float x) { return acosf(x); }
LF_INLINE double lf_acos(double x) { return acos(x); }
LF_INLINE float lf_fma(float a, float b, float c) { return fmaf(a, b, c); }
LF_INLINE double lf_fma(double a, double b, double c) { return fma(a, b, c); }
LF_INLINE float lf_cos(float x) { return cosf(x); }
LF_INLINE double lf_cos(double x) { return cos(x); }
LF_INLINE float lf_sin(float x) { return sinf(x); }
LF_INLINE double lf_sin(double x) { return sin(x); }

template <class T> struct Out5 { T ax, ay, pxx, pyy, pxy; };

// ------------------------------------------------------ float-float accumulation ----
// Error-free transformations (Knuth's TwoSum; Dekker's Fast2Sum) keep a running sum as an
// unevaluated pair hi + lo of FP32 numbers, about 48 significant bits.
struct ff { float hi, lo; };

LF_INLINE ff ff_zero() { ff r; r.hi = 0.f; r.lo = 0.f; return r; }

LF_INLINE void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// acc += x (x a plain float); the low word collects the rounding error of the high word.
LF_INLINE void ff_acc(ff& acc, float x) {
  float s, e;
  two_sum(acc.hi, x, s, e);
  acc.hi = s;
  acc.lo += e;
}

LF_INLINE double ff_to_double(const ff& a) { return (double)a.hi + (double)a.lo; }

// A float-float value from the lane `off` positions away (butterfly exchange; all lanes take part).
LF_INLINE ff ff_shfl_xor(const ff& v, int off) {
  ff r;
  r.hi = __shfl_xor_sync(0xffffffffu, v.hi, off);
  r.lo = __shfl_xor_sync(0xffffffffu, v.lo, off);
  return r;
}

// Float-float arithmetic (Dekker 1971; Knuth TAOCP 4.2.2): each value is an unevaluated sum
// hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits, built from FP32 operations and
// the exact product error fmaf(a, b, -a b).
LF_INLINE ff ff_make(float hi, float lo) { ff r; r.hi = hi; r.lo = lo; return r; }
LF_INLINE ff fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  return ff_make(s, b - (s - a));
}
LF_INLINE ff ff_add(const ff& a, const ff& b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return fast_two_sum(s, e);
}
LF_INLINE ff ff_neg(const ff& a) { return ff_make(-a.hi, -a.lo); }
LF_INLINE ff ff_sub(const ff& a, const ff& b) { return ff_add(a, ff_neg(b)); }
LF_INLINE ff ff_add_f(const ff& a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e += a.lo;
  return fast_two_sum(s, e);
}
LF_INLINE ff ff_mul(const ff& a, const ff& b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
LF_INLINE ff ff_mul_f(const ff& a, float b) {
  float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return fast_two_sum(p, e);
}
LF_INLINE ff ff_sqr(const ff& a) {
  float p = a.hi * a.hi;
  float e = fmaf(a.hi, a.hi, -p);
  e = fmaf(2.0f * a.hi, a.lo, e);
  return fast_two_sum(p, e);
}
// 1 / a: FP32 reciprocal and one Newton step r + r (1 - a r) with the residual in float-float.
LF_INLINE ff ff_rcp(const ff& a) {
  float r = __fdividef(1.0f, a.hi);
  float e = -fmaf(a.hi, r, -1.0f);
  e = fmaf(-a.lo, r, e);
  return fast_two_sum(r, r * e);
}
// a / b: the FP32 quotient refined twice with the exact remainder.
LF_INLINE ff ff_div(const ff& a, const ff& b) {
  float r = __fdividef(1.0f, b.hi);
  float q1 = a.hi * r;
  ff rem = ff_sub(a, ff_mul_f(b, q1));
  float q2 = rem.hi * r;
  ff q = fast_two_sum(q1, q2);
  rem = ff_sub(a, ff_mul(b, q));
  return ff_add_f(q, rem.hi * r);
}
// sqrt(a) for a > 0: FP32 root plus one Newton correction with the exact square error.
LF_INLINE ff ff_sqrt(const ff& a) {
  float ir = rsqrtf(a.hi);
  float s = a.hi * ir;
  float p = s * s;
  float e = fmaf(s, s, -p);
  float r = ((a.hi - p) - e) + a.lo;
  return fast_two_sum(s, r * 0.5f * ir);
}
LF_INLINE ff ff_from_double(double v) {
  float h = (float)v;
  return ff_make(h, (float)(v - (double)h));
}

// atan and atanh in float-float by the addition formulas
//   atan(z)  = atan(c)  + atan((z - c) / (1 + z c)),
//   atanh(z) = atanh(c) + atanh((z - c) / (1 - z c)),
// with c = k/64 the nearest table point (tables of atan(k/64), atanh(k/64) held in shared
// memory as float-float, k = 0..64), and the reduced argument t handled by its odd Taylor
// series t -+ t^3/3 + t^5/5 -+ ... : t exactly in float-float, the higher terms (relatively
// below t^2/3) in FP32.  |z| > 1 for atan uses atan(z) = pi/2 - atan(1/z).
#define LF_TAB_N 65
LF_INLINE float series_corr(float t2, float sgn) {
  // t^2 (-+1/3 + t^2 (1/5 -+ t^2 (1/7 + ...)))  (sgn = -1 atan, +1 atanh), through t^13
  float p = sgn * (1.0f / 13.0f);
  p = fmaf(p, t2, 1.0f / 11.0f);
  p = fmaf(p, t2 * sgn, 1.0f / 9.0f);
  p = fmaf(p, t2 * sgn, 1.0f / 7.0f);
  p = fmaf(p, t2 * sgn, 1.0f / 5.0f);
  p = fmaf(p, t2 * sgn, 1.0f / 3.0f);
  return p * t2 * sgn;
}
LF_INLINE ff ff_atan(const ff& z, const float2* tab) {
  const bool neg = z.hi < 0.f;
  ff a = neg ? ff_neg(z) : z;
  const bool inv = a.hi > 1.f;
  if (inv) a = ff_div(ff_make(1.f, 0.f), a);
  const int k = __float2int_rn(a.hi * 64.f);
  const float c = (float)k * (1.0f / 64.0f);
  ff num = ff_add_f(a, -c);
  ff den = ff_add_f(ff_mul_f(a, c), 1.0f);
  ff t = ff_div(num, den);
  ff r = ff_add_f(t, t.hi * series_corr(t.hi * t.hi, -1.f));
  r = ff_add(r, ff_make(tab[k].x, tab[k].y));
  if (inv) r = ff_sub(ff_make(1.5707963705062866f, -4.371138828673793e-08f), r);
  return neg ? ff_neg(r) : r;
}
LF_INLINE ff ff_atanh(const ff& z, const float2* tab) {
  const bool neg = z.hi < 0.f;
  ff a = neg ? ff_neg(z) : z;
  int k = __float2int_rn(a.hi * 64.f);
  k = k > 63 ? 63 : k;
  const float c = (float)k * (1.0f / 64.0f);
  ff num = ff_add_f(a, -c);
  ff den = ff_add_f(ff_mul_f(a, -c), 1.0f);
  ff t = ff_div(num, den);
  ff r = ff_add_f(t, t.hi * series_corr(t.hi * t.hi, 1.f));
  r = ff_add(r, ff_make(tab[LF_TAB_N + k].x, tab[LF_TAB_N + k].y));
  return neg ? ff_neg(r) : r;
}
// Fills the two tables (2 * LF_TAB_N float2) from FP64 atan / atanh; whole block.
__device__ inline void init_ff_tables(float2* tab) {
  for (int i = threadIdx.x; i < 2 * LF_TAB_N; i += blockDim.x) {
    const int k = i % LF_TAB_N;
    const double c = k / 64.0;
    const double v = (i < LF_TAB_N) ? atan(c) : (k < 64 ? atanh(c) : 0.0);
    const float h = (float)v;
    tab[i] = make_float2(h, (float)(v - (double)h));
  }
}

// Splits a double into hi + lo floats (hi = nearest float, lo = nearest float of the rest).
__host__ __device__ inline void split_ff(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// ----------------------------------------------------------- profile closed forms ----
// Softened isothermal ellipsoid of unit strength in its own (u, v) frame.
// qe = q / e; round != 0 evaluates at q = 1 (e and qe unused): alpha from the expansions
// (q/e) atan(e X) = q X (1 - e^2 X^2 / 3 + O(e^4)) and (q/e) atanh(e Y) = q Y (1 + e^2 Y^2 / 3
// + O(e^4)), X = u / (psi~ + s), Y = v / (psi~ + q^2 s), whose dropped terms have a vanishing
// first derivative in q there, so that dual numbers over q (or eps) get the exact derivative.
template <class T>
LF_INLINE void sie_uv(T u, T v, T q, T q2, T e, T qe, T s, T s2, T q2s, T D0, bool round,
                      T& au, T& av, T& puu, T& pvv, T& puv) {
  T uu = u * u, vv = v * v;
  T p2 = lf_fma(q2, s2 + uu, vv);
  T ip = lf_rsqrt(p2);
  T psi = p2 * ip;
  if (round) {
    const T third = (T)(1.0 / 3.0);
    T e2 = ((T)1 - q) * ((T)1 + q);
    T X = u * lf_rcp(psi + s), Y = v * lf_rcp(psi + q2s);
    au = q * X * ((T)1 - e2 * X * X * third);
    av = q * Y * ((T)1 + e2 * Y * Y * third);
  } else {
    au = qe * lf_atan(e * u * lf_rcp(psi + s));
    av = qe * lf_atanh(e * v * lf_rcp(psi + q2s));
  }
  T D = D0 + (T)2 * psi * s + uu + vv;
  T f = q * ip * lf_rcp(D);
  T sp = s * psi;
  puu = f * (q2 * s2 + vv + sp);
  pvv = f * (s2 + uu + sp);
  puv = -f * u * v;
}

// alpha = M^T alpha_uv, Psi = M^T Psi_uv M, M = [[c, sn], [-sn, c]].
template <class T>
LF_INLINE void rotate_back(T c, T sn, T au, T av, T puu, T pvv, T puv, Out5<T>& o) {
  o.ax = c * au - sn * av;
  o.ay = sn * au + c * av;
  T cc = c * c, ss = sn * sn, cs = c * sn;
  o.pxx = cc * puu - (T)2 * cs * puv + ss * pvv;
  o.pyy = ss * puu + (T)2 * cs * puv + cc * pvv;
  o.pxy = cs * (puu - pvv) + (cc - ss) * puv;
}

// Round cored isothermal of unit strength and core s: kbar = 1/(S + s),
// t = -1/(S (S + s)^2).  Returns kbar and t.
template <class T>
LF_INLINE void cored_round(T r2, T s, T s2, T& kbar, T& t) {
  T S2 = s2 + r2;
  T iS = lf_rsqrt(S2);
  T S = S2 * iS;
  T P = lf_rcp(S + s);
  kbar = P;
  t = -P * P * iS;
}

// Round dPIE / pseudo-Jaffe of strength b, core s and cut a.  With S = sqrt(s^2 + r^2),
// R = sqrt(a^2 + r^2), P = 1/(S + s), Q = 1/(R + a), the mean convergence b (P - Q) is
// written without the far-field cancellation (which loses log2(r / (a - s)) bits):
//   kbar = b (a - s) [(a + s)/(R + S) + 1] P Q,
// using R - S = (a^2 - s^2)/(R + S).  PQ takes one reciprocal of (S + s)(R + a), and
// P = PQ (R + a), Q = PQ (S + s).  The tensor term t = 2 (kappa - kbar)/r^2 =
// b (Q^2/R - P^2/S) cancels only where it is small (|t r^2| ~ 2 b (a - s)/r^2).
// alpha = kbar x, psi_ij = kbar delta_ij + t x_i x_j.
// In FP64 the plain difference b (P - Q) keeps ~48 bits in the far field, so the FP64
// path (the plain comparator) uses it and saves a reciprocal.
template <class T>
LF_INLINE void pje_round(T dx, T dy, T b, T s, T s2, T a, T a2, Out5<T>& o) {
  T r2 = lf_fma(dx, dx, dy * dy);
  T S2 = s2 + r2, R2 = a2 + r2;
  T iS = lf_rsqrt(S2), iR = lf_rsqrt(R2);
  T S = S2 * iS, R = R2 * iR;
  T Ss = S + s, Ra = R + a;
  T PQ = lf_rcp(Ss * Ra);
  T P = PQ * Ra, Q = PQ * Ss;
  T kbar;
  if constexpr (std::is_same<T, double>::value) kbar = b * (P - Q);
  else kbar = b * (a - s) * PQ * lf_fma(a + s, lf_rcp(R + S), (T)1);
  T t = b * (Q * Q * iR - P * P * iS);
  o.ax = kbar * dx;
  o.ay = kbar * dy;
  o.pxx = lf_fma(t * dx, dx, kbar);
  o.pyy = lf_fma(t * dy, dy, kbar);
  o.pxy = t * dx * dy;
}

// Scalar type of an evaluation type (float, double, or dual numbers over one of them).
template <class T> struct scalar_of { typedef T type; };

// Near x = 1 (w = 1 - x^2 small) the NFW functions as series in w, free of the cancellation
// of their closed forms there:
//   g = (F - 1)/(1 - x^2) = sum_{n>=1} w^(n-1) / (2n + 1),
//   h = (1 - ln 2) - (1/2) sum_{n>=1} w^n / (n (2n + 1))   (from dh/dx = x g, h(1) = 1 - ln 2).
// FP32 uses them for |w| < 0.5 (26 and 24 terms), FP64 for |w| < 0.1 (17 and 16 terms).
template <class T, int N> LF_INLINE T nfw_series_g(T w) {
  T r = (T)(1.0 / (2.0 * N + 1.0));
#pragma unroll
  for (int n = N - 1; n >= 1; --n) r = lf_fma(r, w, (T)(1.0 / (2.0 * n + 1.0)));
  return r;
}
template <class T, int N> LF_INLINE T nfw_series_h(T w) {
  T r = (T)(1.0 / (N * (2.0 * N + 1.0)));
#pragma unroll
  for (int n = N - 1; n >= 1; --n) r = lf_fma(r, w, (T)(1.0 / (n * (2.0 * n + 1.0))));
  return r * w;
}

// Spherical NFW of strength ks and scale radius rs (irs = 1/rs).
//  g = (F - 1)/(1 - x^2) so that kappa = 2 ks g;
//  h(x) for x < 1 in the cancellation-free arrangement
//     h = [d (ln 2 - ln x) + log1p(-d/2)] / w,  w = sqrt(1 - x^2), d = x^2 / (1 + w),
//  for x > 1: h = ln(x/2) + acos(1/x) / sqrt(x^2 - 1); near x = 1 the series above.
template <class T>
LF_INLINE void nfw_sph(T dx, T dy, T ks, T irs, Out5<T>& o) {
  T r2 = lf_fma(dx, dx, dy * dy);
  T x2 = r2 * irs * irs;
  T x = lf_sqrt(x2);
  T w2 = ((T)1 - x) * ((T)1 + x);  // 1 - x^2
  T g, h;
  const T ln2 = (T)0.69314718055994530942;
  constexpr bool f32 = std::is_same<typename scalar_of<T>::type, float>::value;
  const T band = (T)(f32 ? 0.5 : 0.1);
  if (w2 < band && w2 > -band) {
    if constexpr (f32) {
      g = nfw_series_g<T, 26>(w2);
      h = (T)0.30685281944005469058 - (T)0.5 * nfw_series_h<T, 24>(w2);
    } else {
      g = nfw_series_g<T, 17>(w2);
      h = (T)0.30685281944005469058 - (T)0.5 * nfw_series_h<T, 16>(w2);
    }
  } else if (w2 > (T)0) {
    T w = lf_sqrt(w2);
    T F = lf_log(((T)1 + w) * lf_rcp(x)) * lf_rcp(w);   // atanh(w) = ln((1 + w)/x)
    g = (F - (T)1) * lf_rcp(w2);
    T d = x2 * lf_rcp((T)1 + w);
    h = (d * (ln2 - lf_log(x)) + lf_log1p(-(T)0.5 * d)) * lf_rcp(w);
  } else {
    T w = lf_sqrt(-w2);
    T F = lf_atan(w) * lf_rcp(w);
    g = (F - (T)1) * lf_rcp(w2);
    h = lf_log(x * (T)0.5) + lf_acos(lf_rcp(x)) * lf_rcp(w);
  }
  T kappa = (T)2 * ks * g;
  T kbar = (T)4 * ks * h * lf_rcp(x2);
  T t = (r2 > (T)0) ? (T)2 * (kappa - kbar) * lf_rcp(r2) : (T)0;
  o.ax = kbar * dx;
  o.ay = kbar * dy;
  o.pxx = lf_fma(t * dx, dx, kbar);
  o.pyy = lf_fma(t * dy, dy, kbar);
  o.pxy = t * dx * dy;
}

// ------------------------------------------------------------ digested tables ------
// Component kinds as stored in the digested tables.
enum { K_SIE = 1, K_DPIE = 2, K_NFW = 3, K_SHEAR = 4, K_MPOLE3 = 5, K_ENFW = 6 };

// An explicit component prepared for evaluation in precision T.  Centre as
// float-float for T = float (offsets are taken in two FP32 subtractions), double else.
template <class T> struct CompT {
  int kind, round;
  T xh, xl, yh, yl;     // centre (xl = yl = 0 for double)
  T c, sn;              // cos / sin of the position angle (shear: 2 pa, multipole: 3 pa)
  T b;                  // strength (NFW: kappa_s, shear: gamma)
  T q, q2, e, qe;
  T s1, s1sq, q2s1, D01;  // core terms
  T s2, s2sq, q2s2, D02;  // cut terms (dPIE)
  T irs;                  // NFW 1/rs
  // low words of the float-float constants used by the extended-precision deflection of
  // elliptical components and the shear (zero for double)
  T lc, lsn, lb, lq2, le, lqe, ls1, ls1sq, lq2s1, ls2, ls2sq, lq2s2;
};

// A cluster member (round pseudo-Jaffe) prepared for evaluation in precision T.
// The first three 16-byte groups are what the evaluation reads; the fourth is read only by
// the adjoint.
template <class T> struct MemT {
  T xh, xl, yh, yl;
  T bd, s, a, apc;        // bd = b (a - s), apc = a + s
  T s2, a2, b, fb;        // fb = (L/L*)^(2 lam) = b / b*
  T fs, loglr, pad0, pad1;  // fs = (L/L*)^beta = s / core*, loglr = ln(L/L*)
};

// A member's change from the plan's base fields to the sample's, for the anchored member sum
// of the gradient's forward pass: ds = s - s0, da = a - a0, db = b - b0 (each from the sampled
// factors' small perturbations, so that FP32 rounds the change, not the field), and the base
// core and cut with their squares.
struct MemA {
  float ds, da, db, s0;
  float a0, s02, a02, pad;
};

// Builds the evaluation constants of one explicit component from its fields.
template <class T>
__host__ __device__ inline void digest_comp(int kind, double x, double y, double b, double eps,
                                            double pa, double core, double cut, CompT<T>& c) {
  c.kind = kind;
  c.round = (eps == 0.0);
  if (sizeof(T) == 4) {
    float h, l;
    split_ff(x, h, l); c.xh = (T)h; c.xl = (T)l;
    split_ff(y, h, l); c.yh = (T)h; c.yl = (T)l;
  } else {
    c.xh = (T)x; c.xl = (T)0; c.yh = (T)y; c.yl = (T)0;
  }
  double q = (1.0 - eps) / (1.0 + eps);
  double e = sqrt((1.0 - q) * (1.0 + q));
  double cc, ss;
  sincos(kind == K_SHEAR ? 2.0 * pa : kind == K_MPOLE3 ? 3.0 * pa : pa, &ss, &cc);
  c.c = (T)cc;
  c.sn = (T)ss;
  c.b = (T)b;
  c.q = (T)q; c.q2 = (T)(q * q); c.e = (T)e; c.qe = (T)(e > 0 ? q / e : 0.0);
  c.s1 = (T)core; c.s1sq = (T)(core * core); c.q2s1 = (T)(q * q * core);
  c.D01 = (T)((1.0 + q * q) * core * core);
  c.s2 = (T)cut; c.s2sq = (T)(cut * cut); c.q2s2 = (T)(q * q * cut);
  c.D02 = (T)((1.0 + q * q) * cut * cut);
  c.irs = (T)((kind == K_NFW || kind == K_ENFW) && core > 0 ? 1.0 / core : 0.0);
  // low words: v - (T)v (zero when T is double)
  const double q2 = q * q, qe = e > 0 ? q / e : 0.0;
  c.lc = (T)(cc - (double)c.c); c.lsn = (T)(ss - (double)c.sn); c.lb = (T)(b - (double)c.b);
  c.lq2 = (T)(q2 - (double)c.q2); c.le = (T)(e - (double)c.e); c.lqe = (T)(qe - (double)c.qe);
  c.ls1 = (T)(core - (double)c.s1); c.ls1sq = (T)(core * core - (double)c.s1sq);
  c.lq2s1 = (T)(q2 * core - (double)c.q2s1);
  c.ls2 = (T)(cut - (double)c.s2); c.ls2sq = (T)(cut * cut - (double)c.s2sq);
  c.lq2s2 = (T)(q2 * cut - (double)c.q2s2);
}

template <class T>
__host__ __device__ inline void digest_member(double x, double y, double b, double s, double a,
                                              double loglr, MemT<T>& m, double fb = 0.0,
                                              double fs = 0.0) {
  if (sizeof(T) == 4) {
    float h, l;
    split_ff(x, h, l); m.xh = (T)h; m.xl = (T)l;
    split_ff(y, h, l); m.yh = (T)h; m.yl = (T)l;
  } else {
    m.xh = (T)x; m.xl = (T)0; m.yh = (T)y; m.yl = (T)0;
  }
  m.bd = (T)(b * (a - s)); m.s = (T)s; m.a = (T)a; m.apc = (T)(a + s);
  m.s2 = (T)(s * s); m.a2 = (T)(a * a); m.b = (T)b; m.fb = (T)fb;
  m.fs = (T)fs; m.loglr = (T)loglr; m.pad0 = (T)0; m.pad1 = (T)0;
}

// Offset from a centre: float-float difference for FP32, plain for FP64.
LF_INLINE float offset_of(float ph, float pl, float ch, float cl) { return (ph - ch) + (pl - cl); }
LF_INLINE double offset_of(double ph, double pl, double ch, double cl) { return ph - ch; }

// Third-order multipole psi = r^2 cos 3(phi - phi_3) (unit amplitude; c3, s3 = cos, sin of
// 3 phi_3).  With the unit vector n = (dx, dy) / r and G = cos 3(phi - phi_3)
// = c3 (nx^3 - 3 nx ny^2) + s3 (3 nx^2 ny - ny^3):
//   alpha = r (3 (c3 (nx^2 - ny^2) + 2 s3 nx ny) - G nx, 3 (s3 (nx^2 - ny^2) - 2 c3 nx ny) - G ny),
//   and psi_ij, homogeneous of degree 0, a function of n alone:
//   psi_xx =  6 (c3 nx + s3 ny) - 2 nx Hx - G + 3 G nx^2,
//   psi_yy = -6 (c3 nx + s3 ny) - 2 ny Hy - G + 3 G ny^2,
//   psi_xy =  6 (s3 nx - c3 ny) - ny Hx - nx Hy + 3 G nx ny,
// with (Hx, Hy) = 3 (c3 (nx^2 - ny^2) + 2 s3 nx ny, s3 (nx^2 - ny^2) - 2 c3 nx ny); this is
// the Cartesian derivative chain of the cubic harmonic F = r^3 G, free of overflow at small
// r.  Zero at r = 0 exactly.  Also evaluated on dual numbers for the adjoint.
template <class T>
LF_INLINE void multipole3(T dx, T dy, T c3, T s3, Out5<T>& o) {
  const T r2 = dx * dx + dy * dy;
  if (!(r2 > (T)0)) {
    o.ax = (T)0; o.ay = (T)0; o.pxx = (T)0; o.pyy = (T)0; o.pxy = (T)0;
    return;
  }
  const T ir = lf_rsqrt(r2);
  const T r = r2 * ir, nx = dx * ir, ny = dy * ir;
  const T xx = nx * nx, yy = ny * ny, xy = nx * ny, d = xx - yy;
  const T G = c3 * nx * (xx - (T)3 * yy) + s3 * ny * ((T)3 * xx - yy);
  const T Hx = (T)3 * (c3 * d + (T)2 * s3 * xy);
  const T Hy = (T)3 * (s3 * d - (T)2 * c3 * xy);
  const T L = (T)6 * (c3 * nx + s3 * ny);
  o.ax = r * (Hx - G * nx);
  o.ay = r * (Hy - G * ny);
  o.pxx = L - (T)2 * nx * Hx - G + (T)3 * G * xx;
  o.pyy = -L - (T)2 * ny * Hy - G + (T)3 * G * yy;
  o.pxy = (T)6 * (s3 * nx - c3 * ny) - ny * Hx - nx * Hy + (T)3 * G * xy;
}

// ------------------------------------------------------- elliptical NFW (CSE sum) ---
// The spherical NFW convergence 2 kappa_s g(x), x = r / r_s, as a sum of cored steep
// ellipsoids g(x) = sum_i a_i / (2 (s_i^2 + x^2)^(3/2)) (the method of Oguri 2021; table from
// gen_cse_table.py), made elliptical by x^2 -> xi^2 = u^2 + v^2/q^2 in r_s units.
__constant__ double c_cse_sd[LF_CSE_N] = {LF_CSE_S_LIST};
__constant__ double c_cse_ad[LF_CSE_N] = {LF_CSE_A_LIST};
__constant__ float c_cse_sf[LF_CSE_N] = {LF_CSE_S_LIST};
__constant__ float c_cse_af[LF_CSE_N] = {LF_CSE_A_LIST};
template <class T> __device__ __forceinline__ T cse_s(int i);
template <class T> __device__ __forceinline__ T cse_a(int i);
template <> __device__ __forceinline__ float cse_s<float>(int i) { return c_cse_sf[i]; }
template <> __device__ __forceinline__ float cse_a<float>(int i) { return c_cse_af[i]; }
template <> __device__ __forceinline__ double cse_s<double>(int i) { return c_cse_sd[i]; }
template <> __device__ __forceinline__ double cse_a<double>(int i) { return c_cse_ad[i]; }

// Sum over the table of unit CSEs in the (u, v) frame, offsets in r_s units.  A CSE of core s
// is -(1/s) d/ds of the unit cored isothermal ellipsoid, which removes its atan / atanh: with
// P = sqrt(q^2 (s^2 + u^2) + v^2), D = (1 + q^2) s^2 + 2 P s + u^2 + v^2, A = P + q^2 s,
// B = P + s and f = q / (s P D):
//   alpha_u = f u A, alpha_v = f v B,
//   psi_uu = f [A - q^4 s u^2 / P^2 - 2 u^2 A^2 / (P D)],
//   psi_vv = f [B - s v^2 / P^2 - 2 v^2 B^2 / (P D)],
//   psi_uv = -f u v [q^2 s / P^2 + 2 A B / (P D)].
// T: the table's precision; U: T or dual numbers over it.
template <class T, class U>
LF_INLINE void enfw_uv(U u, U v, U q, U q2, U& au, U& av, U& puu, U& pvv, U& puv) {
  const U uu = u * u, vv = v * v, r2 = uu + vv, q4 = q2 * q2, opq2 = U(1.0) + q2;
  au = U(0.0); av = U(0.0); puu = U(0.0); pvv = U(0.0); puv = U(0.0);
#pragma unroll 2
  for (int i = 0; i < LF_CSE_N; ++i) {
    const T si = cse_s<T>(i);
    const U s = U(si), s2 = U(si * si);
    const U P2 = lf_fma(q2, s2 + uu, vv);
    const U iP = lf_rsqrt(P2);
    const U P = P2 * iP;
    const U D = lf_fma(opq2, s2, lf_fma(U(2.0) * P, s, r2));
    const U iD = lf_rcp(D);
    const U A = lf_fma(q2, s, P), B = P + s;
    const U f = U(cse_a<T>(i) / si) * q * iP * iD;
    const U iP2 = iP * iP, g = U(2.0) * iP * iD;
    au = lf_fma(f * u, A, au);
    av = lf_fma(f * v, B, av);
    puu = lf_fma(f, A - q4 * s * uu * iP2 - g * uu * A * A, puu);
    pvv = lf_fma(f, B - s * vv * iP2 - g * vv * B * B, pvv);
    puv = puv - f * u * v * (q2 * s * iP2 + g * A * B);
  }
}

// The unit CSE sum's potential (offsets in r_s units): per term, -(1/s) d/ds of the cored
// isothermal potential less its value at the centre,
//   u alpha_u + v alpha_v + (q / (2 s)) ln(D / ((1 + q)^2 s^2))
//     - q [s (q^2 u^2 + v^2) / P + u^2 + v^2] / (s D).
template <class U, class T = typename scalar_of<U>::type>   // U: the arithmetic (T or dual numbers)
LF_INLINE U enfw_potential_uv(U u, U v, U q, U q2) {
  typedef U T_;
  const U uu = u * u, vv = v * v, r2 = uu + vv, opq2 = (U)1 + q2, opq = (U)1 + q;
  const U w = lf_fma(q2, uu, vv);
  U p = (U)0;
  for (int i = 0; i < LF_CSE_N; ++i) {
    const U s = U(cse_s<T>(i)), s2 = s * s;
    const T_ P2 = lf_fma(q2, s2 + uu, vv);
    const T_ iP = lf_rsqrt(P2);
    const T_ P = P2 * iP;
    const T_ D = lf_fma(opq2, s2, lf_fma((T_)2 * P, s, r2));
    const T_ iD = lf_rcp(D);
    const T_ qs = q * lf_rcp(s);
    const T_ lin = qs * iP * iD * (u * u * lf_fma(q2, s, P) + vv * (P + s));   // u alpha_u + v alpha_v
    const T_ lg = (T_)0.5 * qs * lf_log(D * lf_rcp(opq * opq * s2));
    const T_ cst = qs * iD * lf_fma(s * w, iP, r2);
    p = lf_fma(U(cse_a<T>(i)), lin + lg - cst, p);
  }
  return p;
}

// alpha and psi_ij of one explicit component at offset (dx, dy), evaluated in U (T itself, or
// dual numbers over the offset for third derivatives) with the component's constants in T.
template <class T, class U>
LF_INLINE void eval_comp_g(const CompT<T>& c, U dx, U dy, Out5<U>& o) {
  const U b = U(c.b), cc = U(c.c), sn = U(c.sn);
  if (c.kind == K_ENFW) {
    // offsets in r_s units; alpha = 2 kappa_s r_s alpha_cse, Psi = 2 kappa_s Psi_cse
    const U irs = U(c.irs);
    const U u = (cc * dx + sn * dy) * irs, v = (cc * dy - sn * dx) * irs;
    U au, av, puu, pvv, puv;
    enfw_uv<T, U>(u, v, U(c.q), U(c.q2), au, av, puu, pvv, puv);
    const U k2 = U(2.0) * b, k2r = k2 * U(c.s1);
    rotate_back(cc, sn, k2r * au, k2r * av, k2 * puu, k2 * pvv, k2 * puv, o);
    return;
  }
  if (c.kind == K_MPOLE3) {
    multipole3(dx, dy, cc, sn, o);
    o.ax = b * o.ax; o.ay = b * o.ay; o.pxx = b * o.pxx; o.pyy = b * o.pyy; o.pxy = b * o.pxy;
    return;
  }
  if (c.kind == K_SHEAR) {
    U g1 = b * cc, g2 = b * sn;
    o.ax = g1 * dx + g2 * dy;
    o.ay = g2 * dx - g1 * dy;
    o.pxx = g1; o.pyy = -g1; o.pxy = g2;
    return;
  }
  if (c.kind == K_NFW) {
    nfw_sph(dx, dy, b, U(c.irs), o);
    return;
  }
  if (c.round) {
    if (c.kind == K_DPIE) {
      pje_round(dx, dy, b, U(c.s1), U(c.s1sq), U(c.s2), U(c.s2sq), o);
    } else {
      U r2 = lf_fma(dx, dx, dy * dy);
      U kbar, t;
      cored_round(r2, U(c.s1), U(c.s1sq), kbar, t);
      kbar = b * kbar; t = b * t;
      o.ax = kbar * dx; o.ay = kbar * dy;
      o.pxx = lf_fma(t * dx, dx, kbar);
      o.pyy = lf_fma(t * dy, dy, kbar);
      o.pxy = t * dx * dy;
    }
    return;
  }
  U u = cc * dx + sn * dy;
  U v = cc * dy - sn * dx;
  U au, av, puu, pvv, puv;
  sie_uv(u, v, U(c.q), U(c.q2), U(c.e), U(c.qe), U(c.s1), U(c.s1sq), U(c.q2s1), U(c.D01), false, au, av,
         puu, pvv, puv);
  if (c.kind == K_DPIE) {
    U bu, bv, quu, qvv, quv;
    sie_uv(u, v, U(c.q), U(c.q2), U(c.e), U(c.qe), U(c.s2), U(c.s2sq), U(c.q2s2), U(c.D02), false, bu, bv,
           quu, qvv, quv);
    au -= bu; av -= bv; puu -= quu; pvv -= qvv; puv -= quv;
  }
  au *= b; av *= b; puu *= b; pvv *= b; puv *= b;
  rotate_back(cc, sn, au, av, puu, pvv, puv, o);
}

template <class T>
LF_INLINE void eval_comp(const CompT<T>& c, T dx, T dy, Out5<T>& o) {
  eval_comp_g<T, T>(c, dx, dy, o);
}

// One member with its precomputed b (a - s) and a + s (same forms as pje_round).
template <class T>
LF_INLINE void eval_member(const MemT<T>& m, T dx, T dy, Out5<T>& o) {
  T r2 = lf_fma(dx, dx, dy * dy);
  T S2 = m.s2 + r2, R2 = m.a2 + r2;
  T iS = lf_rsqrt(S2), iR = lf_rsqrt(R2);
  T S = S2 * iS, R = R2 * iR;
  T Ss = S + m.s, Ra = R + m.a;
  T PQ = lf_rcp(Ss * Ra);
  T P = PQ * Ra, Q = PQ * Ss;
  T kbar;
  if constexpr (std::is_same<T, double>::value) kbar = m.b * (P - Q);
  else kbar = m.bd * PQ * lf_fma(m.apc, lf_rcp(R + S), (T)1);
  T t = m.b * (Q * Q * iR - P * P * iS);
  o.ax = kbar * dx;
  o.ay = kbar * dy;
  o.pxx = lf_fma(t * dx, dx, kbar);
  o.pyy = lf_fma(t * dy, dy, kbar);
  o.pxy = t * dx * dy;
}

// The change of a pseudo-Jaffe member's deflection from its base fields (b0, s0, a0) to the
// sample's (b, s, a) at a fixed offset, and the sample's psi_ij.  With P = 1/(S + s),
// Q = 1/(R + a), S = sqrt(s^2 + r^2), R = sqrt(a^2 + r^2) and kbar = P - Q:
//   P - P0 = -ds (P + P0) / (S + S0),   Q - Q0 = -da (Q + Q0) / (R + R0),
//   b kbar - b0 kbar0 = db kbar + b0 (kbar - kbar0),
// with kbar in its cancellation-free form (a - s) P Q (1 + (a + s) / (R + S)).  Every FP32
// rounding falls on a term proportional to (ds, da, db), so the change carries a relative
// error of a few u of itself instead of u of the member's whole deflection.  o.ax, o.ay: the
// change; o.pxx, o.pyy, o.pxy: the sample's psi_ij.  Three reciprocals share two MUFU rcp.
LF_INLINE void eval_member_anchored(const MemT<float>& m, const MemA& d, float dx, float dy,
                                    Out5<float>& o) {
  const float r2 = fmaf(dx, dx, dy * dy);
  const float S2 = m.s2 + r2, R2 = m.a2 + r2, S02 = d.s02 + r2, R02 = d.a02 + r2;
  const float iS = lf_rsqrt(S2), iR = lf_rsqrt(R2), iS0 = lf_rsqrt(S02), iR0 = lf_rsqrt(R02);
  const float S = S2 * iS, R = R2 * iR, S0 = S02 * iS0, R0 = R02 * iR0;
  const float Ss = S + m.s, Ra = R + m.a, Ss0 = S0 + d.s0, Ra0 = R0 + d.a0;
  const float X = Ss * Ra, X0 = Ss0 * Ra0;
  const float inv = lf_rcp(X * X0);
  const float PQ = inv * X0, P0Q0 = inv * X;
  const float P = PQ * Ra, Q = PQ * Ss, P0 = P0Q0 * Ra0, Q0 = P0Q0 * Ss0;
  const float Y1 = S + S0, Y2 = R + R0, Y3 = R + S;
  const float Y12 = Y1 * Y2;
  const float inv2 = lf_rcp(Y12 * Y3);
  const float iY3 = inv2 * Y12, iY12 = inv2 * Y3;
  const float dP = -d.ds * (P + P0) * (iY12 * Y2);
  const float dQ = -d.da * (Q + Q0) * (iY12 * Y1);
  const float kk = (m.a - m.s) * PQ * fmaf(m.apc, iY3, 1.0f);   // kbar of the sample
  const float dK = fmaf(d.db, kk, (m.b - d.db) * (dP - dQ));
  const float K = m.b * kk;
  const float t = m.b * (Q * Q * iR - P * P * iS);
  o.ax = dK * dx;
  o.ay = dK * dy;
  o.pxx = fmaf(t * dx, dx, K);
  o.pyy = fmaf(t * dy, dy, K);
  o.pxy = t * dx * dy;
}

// ----------------------------------------------- potential and third derivatives ---
// The lens potential psi (up to a constant per component), for the arrival time of the
// time-delay term (Eq. time_delay), and the third derivatives psi_xxx, psi_xxy, psi_xyy, psi_yyy,
// for grad mu of the flux term (Sec. 3.2).
//   softened isothermal ellipsoid (Keeton 2001), in its (u, v) frame:
//     psi = u alpha_u + v alpha_v - b q s ln sqrt((psi~ + s)^2 + (1 - q^2) u^2)   (round: q = 1)
//   round pseudo-Jaffe member: psi = b [(S - s ln(S + s)) - (R - a ln(R + a))], with
//     S - R = (s^2 - a^2) / (S + R);
//   NFW: psi = 2 ks rs^2 g(x), g = ln(x^2 / (2 (1 + w))) ln((1 + w) / 2), w = sqrt(1 - x^2) (x < 1),
//     g = ln^2(x/2) + atan^2 sqrt(x^2 - 1) (x >= 1);
//   shear: psi = (g1 (x^2 - y^2) + 2 g2 x y) / 2;  multipole: psi = A r^2 cos 3(phi - phi_3).
template <class T>
LF_INLINE T sie_potential_uv(T u, T v, T q, T q2, T e, T qe, T s, T s2, T q2s, T D0, bool round) {
  // alpha from sie_uv (its round branch keeps the exact first derivative in q at q = 1, for
  // dual numbers over eps) and psi~ in the elliptical form, equal to sqrt(s^2 + r^2) at q = 1
  T au, av, puu, pvv, puv;
  sie_uv(u, v, q, q2, e, qe, s, s2, q2s, D0, round, au, av, puu, pvv, puv);
  const T w = lf_sqrt(lf_fma(q2, s2 + u * u, v * v)) + s;
  return u * au + v * av - (T)0.5 * q * s * lf_log(lf_fma(w, w, ((T)1 - q2) * u * u));
}

template <class T>
LF_INLINE T nfw_potential(T dx, T dy, T ks, T irs) {
  const T x = lf_sqrt(lf_fma(dx, dx, dy * dy)) * irs;
  if (!(x > (T)0)) return (T)0;
  const T rs = lf_rcp(irs);
  T g;
  if (x < (T)1) {
    const T w = lf_sqrt(((T)1 - x) * ((T)1 + x));
    g = lf_log(x * x / ((T)2 * ((T)1 + w))) * lf_log(((T)1 + w) * (T)0.5);
  } else {
    const T l = lf_log(x * (T)0.5), t = lf_atan(lf_sqrt((x - (T)1) * (x + (T)1)));
    g = l * l + t * t;
  }
  return (T)2 * ks * rs * rs * g;
}

template <class T>
LF_INLINE T pje_potential(T r2, T b, T s, T a) {
  const T S = lf_sqrt(s * s + r2), R = lf_sqrt(a * a + r2);
  return b * ((s - a) * (s + a) * lf_rcp(S + R) - s * lf_log(S + s) + a * lf_log(R + a));
}

template <class T>
LF_INLINE T comp_potential(const CompT<T>& c, T dx, T dy) {
  if (c.kind == K_MPOLE3) {
    const T r2 = lf_fma(dx, dx, dy * dy);
    if (!(r2 > (T)0)) return (T)0;
    const T ir = lf_rsqrt(r2), nx = dx * ir, ny = dy * ir;
    const T G = c.c * nx * (nx * nx - (T)3 * ny * ny) + c.sn * ny * ((T)3 * nx * nx - ny * ny);
    return c.b * r2 * G;
  }
  if (c.kind == K_SHEAR)
    return c.b * ((T)0.5 * c.c * (dx * dx - dy * dy) + c.sn * dx * dy);
  if (c.kind == K_NFW) return nfw_potential(dx, dy, c.b, c.irs);
  if (c.kind == K_ENFW) {   // psi = 2 kappa_s r_s^2 psi_cse(u / r_s, v / r_s)
    const T u = (c.c * dx + c.sn * dy) * c.irs, v = (c.c * dy - c.sn * dx) * c.irs;
    return (T)2 * c.b * c.s1sq * enfw_potential_uv(u, v, c.q, c.q2);
  }
  const T u = c.round ? dx : c.c * dx + c.sn * dy;
  const T v = c.round ? dy : c.c * dy - c.sn * dx;
  T p = sie_potential_uv(u, v, c.q, c.q2, c.e, c.qe, c.s1, c.s1sq, c.q2s1, c.D01, (bool)c.round);
  if (c.kind == K_DPIE)
    p -= sie_potential_uv(u, v, c.q, c.q2, c.e, c.qe, c.s2, c.s2sq, c.q2s2, c.D02, (bool)c.round);
  return c.b * p;
}

// ------------------------------------------------------- packed member pairs ---
// Two members per record (lane x = member 2j, lane y = member 2j + 1) so that the packed
// FP32 instructions of sm_100 and later (add / mul / fma .rn.f32x2) evaluate both at one
// position: every packed instruction does two members' work in one issue slot.  Centres
// are stored negated so that each offset is a pair of adds, rounded exactly as
// (x_h - c_h) + (x_l - c_l).  A lane past the last member holds a zero-strength member
// (b = 0), whose every contribution is exactly zero.
struct __align__(16) MemPair {
  float2 nxh, nxl, nyh, nyl;  // -(float-float centre)
  float2 s2, a2, s, a;        // core^2, cut^2, core, cut
  float2 apc, bd, b, pad;     // a + s, b (a - s), b
};

LF_INLINE void set_lane(float2& v, int lane, float x) {
  if (lane) v.y = x; else v.x = x;
}

__device__ inline void digest_member_lane(double x, double y, double b, double s, double a,
                                          MemPair& p, int lane) {
  float h, l;
  split_ff(x, h, l); set_lane(p.nxh, lane, -h); set_lane(p.nxl, lane, -l);
  split_ff(y, h, l); set_lane(p.nyh, lane, -h); set_lane(p.nyl, lane, -l);
  set_lane(p.s2, lane, (float)(s * s)); set_lane(p.a2, lane, (float)(a * a));
  set_lane(p.s, lane, (float)s); set_lane(p.a, lane, (float)a);
  set_lane(p.apc, lane, (float)(a + s)); set_lane(p.bd, lane, (float)(b * (a - s)));
  set_lane(p.b, lane, (float)b); set_lane(p.pad, lane, 0.f);
}
__device__ inline void digest_pad_lane(MemPair& p, int lane) {
  digest_member_lane(0.0, 0.0, 0.0, 1.0, 2.0, p, lane);
}

LF_INLINE float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
LF_INLINE float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
LF_INLINE float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// The round-PJE closed form (pje_round) for the two members of a record at one position,
// added into packed chunk sums laid out so that psi needs no per-member diagonal terms:
//   c[0] += kbar dx, c[1] += kbar dy, c[2] += kbar, c[3] += t dx^2, c[4] += t dx dy,
//   c[5] += t r^2;  then psi_xx = c2 + c3, psi_yy = c2 + c5 - c3, psi_xy = c4
// (psi_ij = kbar delta_ij + t x_i x_j, so psi_yy = kbar + t (r^2 - dx^2)).
// 31 FP32 lane-operations and 4 MUFU per member.
// The position's low word is left out of the offsets here (dx = (x_h - c_h) - c_l): the caller
// adds the first-order term Psi x_l of the members' sums instead (accumulate_packed).
LF_INLINE void member_pair_acc(const MemPair& m, float2 pxh, float2 pyh, float2 (&c)[6]) {
  const float2 dx = add2(add2(pxh, m.nxh), m.nxl);
  const float2 dy = add2(add2(pyh, m.nyh), m.nyl);
  const float2 r2 = fma2(dx, dx, mul2(dy, dy));
  const float2 S2 = add2(m.s2, r2), R2 = add2(m.a2, r2);
  // Every consumer of a MUFU result is a scalar FP32 operation on one lane, writing its half
  // of the pair directly (packing MUFU results first costs extra FP32-pipe cycles).
  float2 iS, iR, S, R;
  iS.x = rsqrtf(S2.x); iS.y = rsqrtf(S2.y);
  iR.x = rsqrtf(R2.x); iR.y = rsqrtf(R2.y);
  S.x = S2.x * iS.x; S.y = S2.y * iS.y;
  R.x = R2.x * iR.x; R.y = R2.y * iR.y;
  const float2 Ss = add2(S, m.s), Ra = add2(R, m.a);
  const float2 X = mul2(Ss, Ra);
  const float2 RS = add2(R, S);
  float2 PQ, iRS, P, Q, bq, w;
  PQ.x = __fdividef(1.f, X.x); PQ.y = __fdividef(1.f, X.y);
  iRS.x = __fdividef(1.f, RS.x); iRS.y = __fdividef(1.f, RS.y);
  P.x = PQ.x * Ra.x; P.y = PQ.y * Ra.y;
  Q.x = PQ.x * Ss.x; Q.y = PQ.y * Ss.y;
  bq.x = m.bd.x * PQ.x; bq.y = m.bd.y * PQ.y;
  w.x = fmaf(m.apc.x, iRS.x, 1.f); w.y = fmaf(m.apc.y, iRS.y, 1.f);
  const float2 kb = mul2(bq, w);
  const float2 Q2 = mul2(Q, Q), P2 = mul2(P, P);
  float2 tt;
  tt.x = fmaf(-P2.x, iS.x, Q2.x * iR.x); tt.y = fmaf(-P2.y, iS.y, Q2.y * iR.y);
  const float2 t = mul2(m.b, tt);
  c[0] = fma2(kb, dx, c[0]);
  c[1] = fma2(kb, dy, c[1]);
  c[2] = add2(c[2], kb);
  const float2 tdx = mul2(t, dx);
  c[3] = fma2(tdx, dx, c[3]);
  c[4] = fma2(tdx, dy, c[4]);
  c[5] = fma2(t, r2, c[5]);
}

// ------------------------------------- extended-precision deflection (mixed path) ---
// Offset from a centre as float-float: (x_h - c_h) with its exact rounding error, plus the
// difference of the low words.
LF_INLINE ff offset_ff(float ph, float pl, float ch, float cl) {
  float s, e;
  two_sum(ph, -ch, s, e);
  e += pl - cl;
  return fast_two_sum(s, e);
}

// psi_ij of a unit-strength softened isothermal ellipsoid in its (u, v) frame, FP32.
LF_INLINE void sie_psi(float u, float v, float q, float q2, float s, float s2, float D0,
                       float& puu, float& pvv, float& puv) {
  float uu = u * u, vv = v * v;
  float p2 = fmaf(q2, s2 + uu, vv);
  float ip = rsqrtf(p2);
  float psi = p2 * ip;
  float D = D0 + 2.f * psi * s + uu + vv;
  float f = q * ip * __fdividef(1.0f, D);
  float sp = s * psi;
  puu = f * (q2 * s2 + vv + sp);
  pvv = f * (s2 + uu + sp);
  puv = -f * u * v;
}

// alpha of a unit-strength softened isothermal ellipsoid in its (u, v) frame, float-float.
LF_INLINE void sie_alpha_ff(const ff& u, const ff& v, const ff& uu, const ff& vv, const ff& q2,
                            const ff& e, const ff& qe, const ff& s, const ff& ssq, const ff& q2s,
                            const float2* tab, ff& au, ff& av) {
  ff p2 = ff_add(ff_mul(q2, ff_add(ssq, uu)), vv);
  ff psi = ff_sqrt(p2);
  ff z1 = ff_div(ff_mul(e, u), ff_add(psi, s));
  ff z2 = ff_div(ff_mul(e, v), ff_add(psi, q2s));
  au = ff_mul(qe, ff_atan(z1, tab));
  av = ff_mul(qe, ff_atanh(z2, tab));
}

// alpha of a unit-strength dPIE (core s, cut a) in its (u, v) frame, float-float: the
// difference of the two isothermal ellipsoids folded into one atan and one atanh by
//   atan(z_s) - atan(z_a) = atan((z_s - z_a) / (1 + z_s z_a)),
//   atanh(z_s) - atanh(z_a) = atanh((z_s - z_a) / (1 - z_s z_a)),
// with z = e u / (psi~ + s) (resp. e v / (psi~ + q^2 s)) for each radius.  Writing X = psi_s + s,
// Y = psi_a + a (X2, Y2 with q^2 s, q^2 a) and w = (a + s) / (psi_a + psi_s), the differences are
// cancellation-free: Y - X = (a - s)(1 + q^2 w) and Y2 - X2 = q^2 (a - s)(1 + w), because
// psi_a - psi_s = q^2 (a^2 - s^2) / (psi_a + psi_s).  So
//   alpha_u = (q/e) atan(e u (Y - X) / (X Y + e^2 u^2)),
//   alpha_v = (q/e) atanh(e v (Y2 - X2) / (X2 Y2 - e^2 v^2)).
LF_INLINE void dpie_alpha_ff(const ff& u, const ff& v, const ff& uu, const ff& vv, const ff& q2,
                             const ff& e, const ff& qe, const ff& s, const ff& ssq, const ff& q2s,
                             const ff& a, const ff& asq, const ff& q2a, const float2* tab, ff& au,
                             ff& av) {
  const ff ps = ff_sqrt(ff_add(ff_mul(q2, ff_add(ssq, uu)), vv));
  const ff pa = ff_sqrt(ff_add(ff_mul(q2, ff_add(asq, uu)), vv));
  const ff amin = ff_sub(a, s);
  const ff w = ff_div(ff_add(a, s), ff_add(pa, ps));
  const ff eu = ff_mul(e, u), ev = ff_mul(e, v);
  const ff num1 = ff_mul(ff_mul(eu, amin), ff_add_f(ff_mul(q2, w), 1.f));
  const ff den1 = ff_add(ff_mul(ff_add(ps, s), ff_add(pa, a)), ff_sqr(eu));
  const ff num2 = ff_mul(ff_mul(ff_mul(ev, q2), amin), ff_add_f(w, 1.f));
  const ff den2 = ff_sub(ff_mul(ff_add(ps, q2s), ff_add(pa, q2a)), ff_sqr(ev));
  au = ff_mul(qe, ff_atan(ff_div(num1, den1), tab));
  av = ff_mul(qe, ff_atanh(ff_div(num2, den2), tab));
}

// alpha of the elliptical NFW's CSE sum (enfw_uv) with every operation in float-float: offsets
// (u, v) in r_s units; returns the unit-kappa_s, r_s = 1 deflection in the (u, v) frame.
__constant__ float2 c_cse_sff[LF_CSE_N] = {LF_CSE_S_FF_LIST};
__constant__ float2 c_cse_cff[LF_CSE_N] = {LF_CSE_C_FF_LIST};   // a_i / s_i
LF_INLINE void enfw_alpha_ff(const ff& u, const ff& v, const ff& q, const ff& q2, ff& au, ff& av) {
  const ff uu = ff_sqr(u), vv = ff_sqr(v), r2 = ff_add(uu, vv), opq2 = ff_add_f(q2, 1.f);
  au = ff_zero();
  av = ff_zero();
  for (int i = 0; i < LF_CSE_N; ++i) {
    const float2 sv = c_cse_sff[i], cv = c_cse_cff[i];
    const ff s = ff_make(sv.x, sv.y), s2 = ff_sqr(s);
    const ff P = ff_sqrt(ff_add(ff_mul(q2, ff_add(s2, uu)), vv));
    const ff D = ff_add(ff_add(ff_mul(opq2, s2), ff_mul_f(ff_mul(P, s), 2.f)), r2);
    const ff f = ff_div(ff_mul(ff_make(cv.x, cv.y), q), ff_mul(P, D));
    au = ff_add(au, ff_mul(ff_mul(f, u), ff_add(P, ff_mul(q2, s))));
    av = ff_add(av, ff_mul(ff_mul(f, v), ff_add(P, s)));
  }
}

// Reduced-precision float-float atan / atanh of a ratio N / D (D > 0) for the chi^2 kernel's
// mixed tier, ~1e-9 relative instead of ~1e-14: with c = k/64 the table point nearest |N|/D,
//   atan(N/D) = atan(c) + atan(t),   t = (|N| - c D) / (D + c |N|),
//   atanh(N/D) = atanh(c) + atanh(t), t = (|N| - c D) / (D - c |N|),
// (|N| / D > 1 for atan: pi/2 - atan(D / |N|)).  The numerator of t is formed in float-float
// (it cancels) and rounded once; t itself (|t| <= 1/128 for atan, < 0.05 for the atanh
// arguments of ellipticities below 0.9) and its odd series are FP32, so t's rounding moves the
// result by ~u |t|.  No float-float division is taken.
LF_INLINE float series_t(float t, float sgn) {       // t -+ t^3/3 + t^5/5 -+ t^7/7 + t^9/9
  const float t2 = t * t;
  float p = fmaf(sgn * (1.0f / 9.0f), t2, 1.0f / 7.0f);
  p = fmaf(p, t2 * sgn, 1.0f / 5.0f);
  p = fmaf(p, t2 * sgn, 1.0f / 3.0f);
  return fmaf(p * t2 * sgn, t, t);
}
LF_INLINE ff ff_atan_ratio_mx(const ff& N, const ff& D, const float2* tab) {
  const bool neg = N.hi < 0.f;
  const ff aN = neg ? ff_neg(N) : N;
  const bool inv = aN.hi > D.hi;
  const ff& U = inv ? D : aN;          // atan(U / V), U <= V
  const ff& V = inv ? aN : D;
  const int k = __float2int_rn(U.hi * __fdividef(64.f, V.hi));
  const float c = (float)k * (1.0f / 64.0f);
  const float num = ff_sub(U, ff_mul_f(V, c)).hi;
  const float den = fmaf(c, U.hi, V.hi);
  ff r = ff_add_f(ff_make(tab[k].x, tab[k].y), series_t(num * __fdividef(1.f, den), -1.f));
  if (inv) r = ff_sub(ff_make(1.5707963705062866f, -4.371138828673793e-08f), r);
  return neg ? ff_neg(r) : r;
}
LF_INLINE ff ff_atanh_ratio_mx(const ff& N, const ff& D, const float2* tab) {
  const bool neg = N.hi < 0.f;
  const ff aN = neg ? ff_neg(N) : N;
  int k = __float2int_rn(aN.hi * __fdividef(64.f, D.hi));
  k = k > 63 ? 63 : k;
  const float c = (float)k * (1.0f / 64.0f);
  const float num = ff_sub(aN, ff_mul_f(D, c)).hi;
  const float den = ff_sub(D, ff_mul_f(aN, c)).hi;
  const ff r = ff_add_f(ff_make(tab[LF_TAB_N + k].x, tab[LF_TAB_N + k].y), series_t(num * __fdividef(1.f, den), 1.f));
  return neg ? ff_neg(r) : r;
}
// a / b with one correction of the FP32 quotient by the exact remainder (~44 bits).
LF_INLINE ff ff_div1(const ff& a, const ff& b) {
  const float r = __fdividef(1.0f, b.hi);
  const float q1 = a.hi * r;
  const ff rem = ff_sub(a, ff_mul_f(b, q1));
  return fast_two_sum(q1, rem.hi * r);
}
// dpie_alpha_ff / sie_alpha_ff with the reduced-precision ratio forms above (chi^2 kernel,
// LF_MIXED): the same cancellation-free arguments, one correction step for w.
LF_INLINE void dpie_alpha_mx(const ff& u, const ff& v, const ff& uu, const ff& vv, const ff& q2,
                             const ff& e, const ff& qe, const ff& s, const ff& ssq, const ff& q2s,
                             const ff& a, const ff& asq, const ff& q2a, const float2* tab, ff& au,
                             ff& av) {
  const ff ps = ff_sqrt(ff_add(ff_mul(q2, ff_add(ssq, uu)), vv));
  const ff pa = ff_sqrt(ff_add(ff_mul(q2, ff_add(asq, uu)), vv));
  const ff amin = ff_sub(a, s);
  const ff w = ff_div1(ff_add(a, s), ff_add(pa, ps));
  const ff eu = ff_mul(e, u), ev = ff_mul(e, v);
  const ff num1 = ff_mul(ff_mul(eu, amin), ff_add_f(ff_mul(q2, w), 1.f));
  const ff den1 = ff_add(ff_mul(ff_add(ps, s), ff_add(pa, a)), ff_sqr(eu));
  const ff num2 = ff_mul(ff_mul(ff_mul(ev, q2), amin), ff_add_f(w, 1.f));
  const ff den2 = ff_sub(ff_mul(ff_add(ps, q2s), ff_add(pa, q2a)), ff_sqr(ev));
  au = ff_mul(qe, ff_atan_ratio_mx(num1, den1, tab));
  av = ff_mul(qe, ff_atanh_ratio_mx(num2, den2, tab));
}
LF_INLINE void sie_alpha_mx(const ff& u, const ff& v, const ff& uu, const ff& vv, const ff& q2,
                            const ff& e, const ff& qe, const ff& s, const ff& ssq, const ff& q2s,
                            const float2* tab, ff& au, ff& av) {
  const ff psi = ff_sqrt(ff_add(ff_mul(q2, ff_add(ssq, uu)), vv));
  au = ff_mul(qe, ff_atan_ratio_mx(ff_mul(e, u), ff_add(psi, s), tab));
  av = ff_mul(qe, ff_atanh_ratio_mx(ff_mul(e, v), ff_add(psi, q2s), tab));
}

// One explicit component for the mixed path: alpha in float-float for elliptical
// isothermal components (SIE, dPIE), the elliptical NFW and the shear, FP32 otherwise;
// psi_ij in FP32.
template <bool FAST>
LF_NOINLINE void eval_comp_mixed_t(const CompT<float>& c, float ph_x, float pl_x, float ph_y,
                               float pl_y, const float2* tab, ff& ax, ff& ay, Out5<float>& o) {
  const bool ell = (c.kind == K_SIE || c.kind == K_DPIE) && !c.round;
  if (c.kind == K_MPOLE3) {
    // psi_ij in FP32; alpha = b r (Hx - G nx, Hy - G ny) in float-float (see multipole3)
    ff dx = offset_ff(ph_x, pl_x, c.xh, c.xl);
    ff dy = offset_ff(ph_y, pl_y, c.yh, c.yl);
    eval_comp(c, dx.hi, dy.hi, o);
    const ff r2 = ff_add(ff_sqr(dx), ff_sqr(dy));
    if (!(r2.hi > 0.f)) { ax = ff_zero(); ay = ff_zero(); return; }
    const ff cc = ff_make(c.c, c.lc), sn = ff_make(c.sn, c.lsn), b = ff_make(c.b, c.lb);
    const ff r = ff_sqrt(r2);
    const ff nx = ff_div(dx, r), ny = ff_div(dy, r);
    const ff xx = ff_sqr(nx), yy = ff_sqr(ny), xy = ff_mul(nx, ny), d = ff_sub(xx, yy);
    const ff G = ff_add(ff_mul(cc, ff_mul(nx, ff_sub(xx, ff_mul_f(yy, 3.f)))),
                        ff_mul(sn, ff_mul(ny, ff_sub(ff_mul_f(xx, 3.f), yy))));
    const ff Hx = ff_mul_f(ff_add(ff_mul(cc, d), ff_mul_f(ff_mul(sn, xy), 2.f)), 3.f);
    const ff Hy = ff_mul_f(ff_sub(ff_mul(sn, d), ff_mul_f(ff_mul(cc, xy), 2.f)), 3.f);
    const ff br = ff_mul(b, r);
    ax = ff_mul(br, ff_sub(Hx, ff_mul(G, nx)));
    ay = ff_mul(br, ff_sub(Hy, ff_mul(G, ny)));
    return;
  }
  if (c.kind == K_ENFW) {
    // psi_ij from the FP32 CSE sum; alpha recomputed in float-float
    ff dx = offset_ff(ph_x, pl_x, c.xh, c.xl);
    ff dy = offset_ff(ph_y, pl_y, c.yh, c.yl);
    eval_comp(c, dx.hi, dy.hi, o);
    const ff cc = ff_make(c.c, c.lc), sn = ff_make(c.sn, c.lsn), b = ff_make(c.b, c.lb);
    const ff rs = ff_make(c.s1, c.ls1), q2 = ff_make(c.q2, c.lq2), q = ff_sqrt(q2);
    const ff u = ff_div(ff_add(ff_mul(cc, dx), ff_mul(sn, dy)), rs);
    const ff v = ff_div(ff_sub(ff_mul(cc, dy), ff_mul(sn, dx)), rs);
    ff au, av;
    enfw_alpha_ff(u, v, q, q2, au, av);
    const ff k = ff_mul_f(ff_mul(b, rs), 2.f);
    au = ff_mul(k, au);
    av = ff_mul(k, av);
    ax = ff_sub(ff_mul(cc, au), ff_mul(sn, av));
    ay = ff_add(ff_mul(sn, au), ff_mul(cc, av));
    return;
  }
  if (!ell && c.kind != K_SHEAR) {
    float dx = offset_of(ph_x, pl_x, c.xh, c.xl);
    float dy = offset_of(ph_y, pl_y, c.yh, c.yl);
    eval_comp(c, dx, dy, o);
    ax = ff_make(o.ax, 0.f);
    ay = ff_make(o.ay, 0.f);
    return;
  }
  ff dx = offset_ff(ph_x, pl_x, c.xh, c.xl);
  ff dy = offset_ff(ph_y, pl_y, c.yh, c.yl);
  const ff cc = ff_make(c.c, c.lc), sn = ff_make(c.sn, c.lsn), b = ff_make(c.b, c.lb);
  if (c.kind == K_SHEAR) {
    ff g1 = ff_mul(b, cc), g2 = ff_mul(b, sn);
    ax = ff_add(ff_mul(g1, dx), ff_mul(g2, dy));
    ay = ff_sub(ff_mul(g2, dx), ff_mul(g1, dy));
    o.pxx = g1.hi; o.pyy = -g1.hi; o.pxy = g2.hi;
    return;
  }
  ff u = ff_add(ff_mul(cc, dx), ff_mul(sn, dy));
  ff v = ff_sub(ff_mul(cc, dy), ff_mul(sn, dx));
  ff uu = ff_mul(u, u), vv = ff_mul(v, v);
  const ff q2 = ff_make(c.q2, c.lq2), e = ff_make(c.e, c.le), qe = ff_make(c.qe, c.lqe);
  ff au, av;
  if (c.kind == K_DPIE) {
    if constexpr (FAST)
      dpie_alpha_mx(u, v, uu, vv, q2, e, qe, ff_make(c.s1, c.ls1), ff_make(c.s1sq, c.ls1sq),
                    ff_make(c.q2s1, c.lq2s1), ff_make(c.s2, c.ls2), ff_make(c.s2sq, c.ls2sq),
                    ff_make(c.q2s2, c.lq2s2), tab, au, av);
    else
      dpie_alpha_ff(u, v, uu, vv, q2, e, qe, ff_make(c.s1, c.ls1), ff_make(c.s1sq, c.ls1sq),
                    ff_make(c.q2s1, c.lq2s1), ff_make(c.s2, c.ls2), ff_make(c.s2sq, c.ls2sq),
                    ff_make(c.q2s2, c.lq2s2), tab, au, av);
  } else {
    if constexpr (FAST)
      sie_alpha_mx(u, v, uu, vv, q2, e, qe, ff_make(c.s1, c.ls1), ff_make(c.s1sq, c.ls1sq),
                   ff_make(c.q2s1, c.lq2s1), tab, au, av);
    else
      sie_alpha_ff(u, v, uu, vv, q2, e, qe, ff_make(c.s1, c.ls1), ff_make(c.s1sq, c.ls1sq),
                   ff_make(c.q2s1, c.lq2s1), tab, au, av);
  }
  float puu, pvv, puv;
  sie_psi(u.hi, v.hi, c.q, c.q2, c.s1, c.s1sq, c.D01, puu, pvv, puv);
  if (c.kind == K_DPIE) {
    float quu, qvv, quv;
    sie_psi(u.hi, v.hi, c.q, c.q2, c.s2, c.s2sq, c.D02, quu, qvv, quv);
    puu -= quu; pvv -= qvv; puv -= quv;
  }
  au = ff_mul(b, au);
  av = ff_mul(b, av);
  ax = ff_sub(ff_mul(cc, au), ff_mul(sn, av));
  ay = ff_add(ff_mul(sn, au), ff_mul(cc, av));
  Out5<float> t;
  rotate_back(c.c, c.sn, 0.f, 0.f, c.b * puu, c.b * pvv, c.b * puv, t);
  o.pxx = t.pxx; o.pyy = t.pyy; o.pxy = t.pxy;
}

LF_INLINE void eval_comp_mixed(const CompT<float>& c, float ph_x, float pl_x, float ph_y, float pl_y,
                               const float2* tab, ff& ax, ff& ay, Out5<float>& o) {
  eval_comp_mixed_t<false>(c, ph_x, pl_x, ph_y, pl_y, tab, ax, ay, o);
}

// ln(y), y > 0, in float-float: y = m 2^e with m in [1/sqrt 2, sqrt 2) (exact scaling by a
// power of two), ln y = e ln 2 + 2 atanh((m - 1)/(m + 1)), |(m - 1)/(m + 1)| <= 0.172.
LF_INLINE ff ff_log(const ff& y, const float2* tab) {
  int e;
  float m = frexpf(y.hi, &e);                 // y.hi = m 2^e, m in [0.5, 1)
  if (m < 0.70710678f) e -= 1;
  const float sc = ldexpf(1.f, -e);
  const ff mm = ff_make(y.hi * sc, y.lo * sc);
  const ff z = ff_div(ff_add_f(mm, -1.f), ff_add_f(mm, 1.f));
  const ff ln2 = ff_make(0.693147182464599609375f, -1.904654323148236e-09f);
  return ff_add(ff_mul_f(ff_atanh(z, tab), 2.f), ff_mul_f(ln2, (float)e));
}

// The float-float tier's evaluation of one explicit component: as eval_comp_mixed, plus
// float-float deflections for the round isothermal and pseudo-Jaffe components and the
// spherical NFW (psi_ij stays FP32):
//   round cored isothermal: kbar = b / (S + s), S = sqrt(s^2 + r^2);
//   round pseudo-Jaffe: kbar = b (a - s) P Q [1 + (a + s)/(R + S)], P = 1/(S + s), Q = 1/(R + a);
//   NFW: kbar = 4 ks h(x) / x^2, x = r / r_s, with
//     1 - x^2 >= 0.02:  h = [d ln(2/x) + ln(1 - d/2)] / w, w = sqrt(1 - x^2), d = x^2/(1 + w);
//     |1 - x^2| < 0.02: h = (1 - ln 2) - (1/2) sum_n w^n / (n (2n + 1)), w = 1 - x^2;
//     x^2 - 1 >= 0.02:  h = ln(x/2) + atan(w) / w, w = sqrt(x^2 - 1).
LF_NOINLINE void eval_comp_ext(const CompT<float>& c, float ph_x, float pl_x, float ph_y, float pl_y,
                               const float2* tab, ff& ax, ff& ay, Out5<float>& o) {
  const bool rnd = (c.kind == K_SIE || c.kind == K_DPIE) && c.round;
  if (!rnd && c.kind != K_NFW) {
    eval_comp_mixed(c, ph_x, pl_x, ph_y, pl_y, tab, ax, ay, o);
    return;
  }
  const ff dx = offset_ff(ph_x, pl_x, c.xh, c.xl), dy = offset_ff(ph_y, pl_y, c.yh, c.yl);
  eval_comp(c, dx.hi, dy.hi, o);              // psi_ij (and an FP32 alpha, replaced below)
  const ff r2 = ff_add(ff_sqr(dx), ff_sqr(dy));
  const ff b = ff_make(c.b, c.lb);
  ff kb;
  if (!(r2.hi > 0.f)) {
    ax = ff_zero();
    ay = ff_zero();
    return;
  }
  if (rnd) {
    const ff s = ff_make(c.s1, c.ls1);
    const ff S = ff_sqrt(ff_add(ff_make(c.s1sq, c.ls1sq), r2));
    const ff P = ff_div(ff_make(1.f, 0.f), ff_add(S, s));
    if (c.kind == K_SIE) {
      kb = ff_mul(b, P);
    } else {
      const ff a = ff_make(c.s2, c.ls2);
      const ff R = ff_sqrt(ff_add(ff_make(c.s2sq, c.ls2sq), r2));
      const ff Q = ff_div(ff_make(1.f, 0.f), ff_add(R, a));
      const ff w = ff_add_f(ff_div(ff_add(a, s), ff_add(R, S)), 1.f);
      kb = ff_mul(ff_mul(b, ff_sub(a, s)), ff_mul(ff_mul(P, Q), w));
    }
  } else {
    const ff rs2 = ff_make(c.s1sq, c.ls1sq);
    const ff x2 = ff_div(r2, rs2);
    const ff x = ff_sqrt(x2);
    const ff w2 = ff_sub(ff_make(1.f, 0.f), x2);
    ff h;
    if (w2.hi >= 0.02f) {
      const ff w = ff_sqrt(w2);
      const ff d = ff_div(x2, ff_add_f(w, 1.f));
      const ff l2x = ff_log(ff_div(ff_make(2.f, 0.f), x), tab);
      const ff l1 = ff_log(ff_add_f(ff_mul_f(d, -0.5f), 1.f), tab);
      h = ff_div(ff_add(ff_mul(d, l2x), l1), w);
    } else if (w2.hi > -0.02f) {
      // h = (1 - ln 2) - (1/2) sum_n w^n / (n (2n + 1)): the n = 1, 2 terms in float-float, the
      // rest (below |w|^3 / 21 <= 4e-7) in FP32
      float t = 1.f / 136.f;
      for (int n = 7; n >= 3; --n) t = fmaf(t, w2.hi, 1.f / (float)(n * (2 * n + 1)));
      const ff third = ff_make(3.333333433e-01f, -9.934107759e-09f);
      const ff tenth = ff_make(1.000000015e-01f, -1.490116142e-09f);
      const ff sum = ff_add(ff_add(ff_mul(w2, third), ff_mul(ff_sqr(w2), tenth)),
                            ff_make(t * w2.hi * w2.hi * w2.hi, 0.f));
      h = ff_sub(ff_make(3.068528175e-01f, 1.904654212e-09f), ff_mul_f(sum, 0.5f));
    } else {
      const ff w = ff_sqrt(ff_neg(w2));
      h = ff_add(ff_log(ff_mul_f(x, 0.5f), tab), ff_div(ff_atan(w, tab), w));
    }
    kb = ff_div(ff_mul_f(ff_mul(b, h), 4.f), x2);
  }
  ax = ff_mul(kb, dx);
  ay = ff_mul(kb, dy);
}

// Member record of the float-float tier: float-float centre and constants of the
// cancellation-free mean convergence, FP32 values for psi_ij, and the scaling factors.
struct MemX {
  float xh, xl, yh, yl;
  float s2h, s2l, a2h, a2l;      // core^2, cut^2
  float sh, sl, ah, al;          // core, cut
  float bdh, bdl, apch, apcl;    // b (cut - core), cut + core
  float b, fb, fs, loglr;        // FP32 strength, (L/L*)^(2 lam), (L/L*)^beta, ln(L/L*)
};

__host__ __device__ inline void digest_member_x(double x, double y, double b, double s, double a,
                                                double loglr, MemX& m, double fb = 0.0,
                                                double fs = 0.0) {
  split_ff(x, m.xh, m.xl);
  split_ff(y, m.yh, m.yl);
  split_ff(s * s, m.s2h, m.s2l);
  split_ff(a * a, m.a2h, m.a2l);
  split_ff(s, m.sh, m.sl);
  split_ff(a, m.ah, m.al);
  split_ff(b * (a - s), m.bdh, m.bdl);
  split_ff(a + s, m.apch, m.apcl);
  m.b = (float)b; m.fb = (float)fb; m.fs = (float)fs; m.loglr = (float)loglr;
}

// alpha of one member at the float-float offset (dx, dy), in float-float (the form below).
LF_INLINE void member_alpha_ff(const MemX& m, const ff& dx, const ff& dy, ff& ax, ff& ay) {
  const ff r2 = ff_add(ff_sqr(dx), ff_sqr(dy));
  const ff S = ff_sqrt(ff_add(ff_make(m.s2h, m.s2l), r2));
  const ff R = ff_sqrt(ff_add(ff_make(m.a2h, m.a2l), r2));
  const ff PQ = ff_rcp(ff_mul(ff_add(S, ff_make(m.sh, m.sl)), ff_add(R, ff_make(m.ah, m.al))));
  const ff br = ff_add_f(ff_mul(ff_make(m.apch, m.apcl), ff_rcp(ff_add(R, S))), 1.0f);
  const ff kbar = ff_mul(ff_mul(ff_make(m.bdh, m.bdl), PQ), br);
  ax = ff_mul(kbar, dx);
  ay = ff_mul(kbar, dy);
}

// alpha of one member in float-float: kbar = b (a - s) [(a + s)/(R + S) + 1] / ((S + s)(R + a)),
// alpha = kbar x; psi_ij in FP32 from the same form (pje_round).
LF_INLINE void eval_member_x(const MemX& m, float ph_x, float pl_x, float ph_y, float pl_y, ff& ax,
                             ff& ay, Out5<float>& o) {
  ff dx = offset_ff(ph_x, pl_x, m.xh, m.xl);
  ff dy = offset_ff(ph_y, pl_y, m.yh, m.yl);
  ff r2 = ff_add(ff_sqr(dx), ff_sqr(dy));
  ff S = ff_sqrt(ff_add(ff_make(m.s2h, m.s2l), r2));
  ff R = ff_sqrt(ff_add(ff_make(m.a2h, m.a2l), r2));
  ff Ss = ff_add(S, ff_make(m.sh, m.sl));
  ff Ra = ff_add(R, ff_make(m.ah, m.al));
  ff PQ = ff_rcp(ff_mul(Ss, Ra));
  ff br = ff_add_f(ff_mul(ff_make(m.apch, m.apcl), ff_rcp(ff_add(R, S))), 1.0f);
  ff kbar = ff_mul(ff_mul(ff_make(m.bdh, m.bdl), PQ), br);
  ax = ff_mul(kbar, dx);
  ay = ff_mul(kbar, dy);
  // psi_ij in FP32
  float r2f = r2.hi;
  float iS = rsqrtf(m.s2h + r2f), iR = rsqrtf(m.a2h + r2f);
  float P = __fdividef(1.0f, Ss.hi), Q = __fdividef(1.0f, Ra.hi);
  float t = m.b * (Q * Q * iR - P * P * iS);
  float kb = kbar.hi;
  o.pxx = fmaf(t * dx.hi, dx.hi, kb);
  o.pyy = fmaf(t * dy.hi, dy.hi, kb);
  o.pxy = t * dx.hi * dy.hi;
}

// ---------------------------------------------------------------- error word ------
// Set by a kernel whose bounded wait ran out; read and cleared by lf_device_error().
__device__ unsigned int g_lf_err;

LF_INLINE void lf_flag_error(unsigned int code) { atomicOr(&g_lf_err, code); }

// ------------------------------------------------ bulk-copy staging (TMA engine) -----
// Global -> shared copies by the bulk-copy engine, completion tracked by an mbarrier
// transaction count.  Waits are bounded: after LF_WAIT_LIMIT polls the block records
// LF_DEVERR_TIMEOUT in the error word and gives up.
#define LF_DEVERR_TIMEOUT 1u
#define LF_DEVERR_BADCOMP 2u
#define LF_DEVERR_BADARG 4u    // an invalid per-item argument (e.g. a_dis outside (0, 1]) was skipped
#define LF_DEVERR_BOUNDS 8u    // an index check of an LF_CHECK_BOUNDS build failed (the access was skipped)

// Index checks of the LF_CHECK_BOUNDS build (off by default): LF_CHECK(cond) is true when the
// condition holds; otherwise it records LF_DEVERR_BOUNDS and is false, so that the caller skips
// the access.  In the default build it is the constant true and costs nothing.
#ifndef LF_CHECK_BOUNDS
#define LF_CHECK_BOUNDS 0
#endif
#if LF_CHECK_BOUNDS
LF_INLINE bool lf_check(bool ok) {
  if (!ok) lf_flag_error(LF_DEVERR_BOUNDS);
  return ok;
}
#define LF_CHECK(...) lf_check((__VA_ARGS__))
#else
#define LF_CHECK(...) true
#endif
// Bytes of dynamic shared memory the running block was launched with.
LF_INLINE uint32_t lf_dyn_smem() {
  uint32_t v;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}
#define LF_WAIT_LIMIT (1u << 24)

LF_INLINE uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

LF_INLINE void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

LF_INLINE void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 16-byte aligned src/dst, bytes a multiple of 16.
LF_INLINE void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Returns true when the phase with the given parity has completed, false once `limit` polls
// have found it still pending.
LF_INLINE bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = LF_WAIT_LIMIT) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < limit; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Stages `bytes` (multiple of 16, both pointers 16-byte aligned) from global into shared
// memory with one elected thread issuing bulk copies of at most 32 KiB each; every thread
// of the block returns once the data has landed (or the bounded wait ran out, in which
// case the function returns false for all threads).
LF_INLINE bool stage_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                             uint32_t parity) {
  if (bytes == 0) return true;
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, bytes);
    const uint32_t CH = 32768u;
    for (uint32_t off = 0; off < bytes; off += CH) {
      uint32_t n = bytes - off < CH ? bytes - off : CH;
      bulk_g2s((char*)dst + off, (const char*)src + off, n, bar);
    }
  }
  bool ok = mbar_wait(bar, parity);
  if (!ok && threadIdx.x == 0) {
    lf_flag_error(LF_DEVERR_TIMEOUT);
    mbar_wait(bar, parity);  // bounded second wait for the copies still in flight
  }
  return __syncthreads_and(ok ? 1 : 0) != 0;
}
