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

#define LF_INLINE __device__ __forceinline__

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
LF_INLINE void ff_add(ff& acc, float x) {
  float s, e;
  two_sum(acc.hi, x, s, e);
  acc.hi = s;
  acc.lo += e;
}

LF_INLINE double ff_to_double(const ff& a) { return (double)a.hi + (double)a.lo; }

// Splits a double into hi + lo floats (hi = nearest float, lo = nearest float of the rest).
__host__ __device__ inline void split_ff(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// ----------------------------------------------------------- profile closed forms ----
// Softened isothermal ellipsoid of unit strength in its own (u, v) frame.
// qe = q / e; round != 0 uses the q = 1 limit.
template <class T>
LF_INLINE void sie_uv(T u, T v, T q, T q2, T e, T qe, T s, T s2, T q2s, T D0, bool round,
                      T& au, T& av, T& puu, T& pvv, T& puv) {
  T uu = u * u, vv = v * v;
  T p2 = lf_fma(q2, s2 + uu, vv);
  T ip = lf_rsqrt(p2);
  T psi = p2 * ip;
  if (round) {
    T r = lf_rcp(psi + s);
    au = u * r;
    av = v * r;
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

// Round dPIE / pseudo-Jaffe of strength b: kbar = b (P - Q), t = b (Q^2/R - P^2/S).
template <class T>
LF_INLINE void pje_round(T dx, T dy, T b, T s, T s2, T a, T a2, Out5<T>& o) {
  T r2 = lf_fma(dx, dx, dy * dy);
  T k1, t1, k2, t2;
  cored_round(r2, s, s2, k1, t1);
  cored_round(r2, a, a2, k2, t2);
  T kbar = b * (k1 - k2);
  T t = b * (t1 - t2);
  o.ax = kbar * dx;
  o.ay = kbar * dy;
  o.pxx = lf_fma(t * dx, dx, kbar);
  o.pyy = lf_fma(t * dy, dy, kbar);
  o.pxy = t * dx * dy;
}

// sum_{n>=0} w^n / (2n + 1) truncated (for |w| < 0.1, 9 terms reach 1e-10 relative).
template <class T> LF_INLINE T series_odd(T w) {
  T r = (T)(1.0 / 19.0);
  r = lf_fma(r, w, (T)(1.0 / 17.0));
  r = lf_fma(r, w, (T)(1.0 / 15.0));
  r = lf_fma(r, w, (T)(1.0 / 13.0));
  r = lf_fma(r, w, (T)(1.0 / 11.0));
  r = lf_fma(r, w, (T)(1.0 / 9.0));
  r = lf_fma(r, w, (T)(1.0 / 7.0));
  r = lf_fma(r, w, (T)(1.0 / 5.0));
  r = lf_fma(r, w, (T)(1.0 / 3.0));
  r = lf_fma(r, w, (T)1);
  return r;
}
// sum_{n>=1} w^(n-1) / (2n + 1)
template <class T> LF_INLINE T series_tail(T w) {
  T r = (T)(1.0 / 21.0);
  r = lf_fma(r, w, (T)(1.0 / 19.0));
  r = lf_fma(r, w, (T)(1.0 / 17.0));
  r = lf_fma(r, w, (T)(1.0 / 15.0));
  r = lf_fma(r, w, (T)(1.0 / 13.0));
  r = lf_fma(r, w, (T)(1.0 / 11.0));
  r = lf_fma(r, w, (T)(1.0 / 9.0));
  r = lf_fma(r, w, (T)(1.0 / 7.0));
  r = lf_fma(r, w, (T)(1.0 / 5.0));
  r = lf_fma(r, w, (T)(1.0 / 3.0));
  return r;
}

// Spherical NFW of strength ks and scale radius rs (irs = 1/rs).
//  g = (F - 1)/(1 - x^2) so that kappa = 2 ks g;
//  h(x) for x < 1 in the cancellation-free arrangement
//     h = [d (ln 2 - ln x) + log1p(-d/2)] / w,  w = sqrt(1 - x^2), d = x^2 / (1 + w),
//  for x > 1: h = ln(x/2) + acos(1/x) / sqrt(x^2 - 1); near x = 1 the power series
//     h = ln(x/2) + (2/(1+x)) sum_n u^n/(2n+1), u = (1-x)/(1+x).
template <class T>
LF_INLINE void nfw_sph(T dx, T dy, T ks, T irs, Out5<T>& o) {
  T r2 = lf_fma(dx, dx, dy * dy);
  T x2 = r2 * irs * irs;
  T x = lf_sqrt(x2);
  T w2 = ((T)1 - x) * ((T)1 + x);  // 1 - x^2
  T g, h;
  const T ln2 = (T)0.69314718055994530942;
  if (w2 < (T)0.1 && w2 > (T)-0.1) {
    g = series_tail(w2);
    T u = ((T)1 - x) * lf_rcp((T)1 + x);
    h = lf_log(x * (T)0.5) + (T)2 * lf_rcp((T)1 + x) * series_odd(u);
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
enum { K_SIE = 1, K_DPIE = 2, K_NFW = 3, K_SHEAR = 4 };

// An explicit component prepared for evaluation in precision T.  Centre as
// float-float for T = float (offsets are taken in two FP32 subtractions), double else.
template <class T> struct CompT {
  int kind, round;
  T xh, xl, yh, yl;     // centre (xl = yl = 0 for double)
  T c, sn;              // cos / sin of the position angle (shear: cos 2pa, sin 2pa)
  T b;                  // strength (NFW: kappa_s, shear: gamma)
  T q, q2, e, qe;
  T s1, s1sq, q2s1, D01;  // core terms
  T s2, s2sq, q2s2, D02;  // cut terms (dPIE)
  T irs;                  // NFW 1/rs
};

// A cluster member (round pseudo-Jaffe) prepared for evaluation in precision T.
template <class T> struct MemT {
  T xh, xl, yh, yl;
  T b, s, a, fb;          // fb = (L/L*)^(2 lam) = b / b*
  T s2, a2, loglr, fs;    // loglr = ln(L/L*), fs = (L/L*)^beta = s / core*
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
  if (kind == K_SHEAR) {
    c.c = (T)cos(2.0 * pa);
    c.sn = (T)sin(2.0 * pa);
  } else {
    c.c = (T)cos(pa);
    c.sn = (T)sin(pa);
  }
  c.b = (T)b;
  c.q = (T)q; c.q2 = (T)(q * q); c.e = (T)e; c.qe = (T)(e > 0 ? q / e : 0.0);
  c.s1 = (T)core; c.s1sq = (T)(core * core); c.q2s1 = (T)(q * q * core);
  c.D01 = (T)((1.0 + q * q) * core * core);
  c.s2 = (T)cut; c.s2sq = (T)(cut * cut); c.q2s2 = (T)(q * q * cut);
  c.D02 = (T)((1.0 + q * q) * cut * cut);
  c.irs = (T)(kind == K_NFW && core > 0 ? 1.0 / core : 0.0);
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
  m.b = (T)b; m.s = (T)s; m.a = (T)a; m.fb = (T)fb;
  m.s2 = (T)(s * s); m.a2 = (T)(a * a); m.loglr = (T)loglr; m.fs = (T)fs;
}

// Offset from a centre: float-float difference for FP32, plain for FP64.
LF_INLINE float offset_of(float ph, float pl, float ch, float cl) { return (ph - ch) + (pl - cl); }
LF_INLINE double offset_of(double ph, double pl, double ch, double cl) { return ph - ch; }

// alpha and psi_ij of one explicit component at offset (dx, dy).
template <class T>
LF_INLINE void eval_comp(const CompT<T>& c, T dx, T dy, Out5<T>& o) {
  if (c.kind == K_SHEAR) {
    T g1 = c.b * c.c, g2 = c.b * c.sn;
    o.ax = g1 * dx + g2 * dy;
    o.ay = g2 * dx - g1 * dy;
    o.pxx = g1; o.pyy = -g1; o.pxy = g2;
    return;
  }
  if (c.kind == K_NFW) {
    nfw_sph(dx, dy, c.b, c.irs, o);
    return;
  }
  if (c.round) {
    if (c.kind == K_DPIE) {
      pje_round(dx, dy, c.b, c.s1, c.s1sq, c.s2, c.s2sq, o);
    } else {
      T r2 = lf_fma(dx, dx, dy * dy);
      T kbar, t;
      cored_round(r2, c.s1, c.s1sq, kbar, t);
      kbar = c.b * kbar; t = c.b * t;
      o.ax = kbar * dx; o.ay = kbar * dy;
      o.pxx = lf_fma(t * dx, dx, kbar);
      o.pyy = lf_fma(t * dy, dy, kbar);
      o.pxy = t * dx * dy;
    }
    return;
  }
  T u = c.c * dx + c.sn * dy;
  T v = c.c * dy - c.sn * dx;
  T au, av, puu, pvv, puv;
  sie_uv(u, v, c.q, c.q2, c.e, c.qe, c.s1, c.s1sq, c.q2s1, c.D01, false, au, av, puu, pvv, puv);
  if (c.kind == K_DPIE) {
    T bu, bv, quu, qvv, quv;
    sie_uv(u, v, c.q, c.q2, c.e, c.qe, c.s2, c.s2sq, c.q2s2, c.D02, false, bu, bv, quu, qvv, quv);
    au -= bu; av -= bv; puu -= quu; pvv -= qvv; puv -= quv;
  }
  au *= c.b; av *= c.b; puu *= c.b; pvv *= c.b; puv *= c.b;
  rotate_back(c.c, c.sn, au, av, puu, pvv, puv, o);
}

template <class T>
LF_INLINE void eval_member(const MemT<T>& m, T dx, T dy, Out5<T>& o) {
  pje_round(dx, dy, m.b, m.s, m.s2, m.a, m.a2, o);
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

// Returns true when the phase with the given parity has completed.
LF_INLINE bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < LF_WAIT_LIMIT; ++it) {
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
