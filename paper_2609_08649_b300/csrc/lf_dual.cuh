// Forward-mode dual numbers: value plus N tangents, carried through the same closed forms
// as the forward kernels.  The chi^2 adjoint uses them to obtain the exact derivative of one
// component's (alpha, psi_ij) with respect to that component's own fields, which it then
// contracts with the cotangents of the source-plane chi^2.
#pragma once
#include "lf_common.cuh"

namespace lf {

// The scalar overloads, visible beside the dual ones below, so that the dual rules can call
// the elementary functions of their value type whether it is a scalar or itself dual (dual
// numbers nest: Dual<Dual<T, 2>, 6> carries mixed second derivatives).
using ::lf_rcp;
using ::lf_rsqrt;
using ::lf_sqrt;
using ::lf_atan;
using ::lf_atanh;
using ::lf_log;
using ::lf_log1p;
using ::lf_acos;
using ::lf_cos;
using ::lf_sin;

template <class T, int N> struct Dual {
  T v;
  T d[N];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(double c) : v((T)c) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = (T)0;
  }
  __device__ __forceinline__ static Dual var(T x, int slot) {
    Dual r(0.0);
    r.v = x;
    if (slot >= 0) r.d[slot] = (T)1;
    return r;
  }
  __device__ __forceinline__ static Dual cst(T x) {
    Dual r(0.0);
    r.v = x;
    return r;
  }
};

#define DUAL_T template <class T, int N>
#define D Dual<T, N>

DUAL_T __device__ __forceinline__ D chain(const D& a, T f, T df) {
  D r;
  r.v = f;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = df * a.d[i];
  return r;
}
DUAL_T __device__ __forceinline__ D operator+(const D& a, const D& b) {
  D r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
DUAL_T __device__ __forceinline__ D operator-(const D& a, const D& b) {
  D r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
DUAL_T __device__ __forceinline__ D operator-(const D& a) {
  D r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
DUAL_T __device__ __forceinline__ D operator*(const D& a, const D& b) {
  D r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
DUAL_T __device__ __forceinline__ D& operator+=(D& a, const D& b) { a = a + b; return a; }
DUAL_T __device__ __forceinline__ D& operator-=(D& a, const D& b) { a = a - b; return a; }
DUAL_T __device__ __forceinline__ D& operator*=(D& a, const D& b) { a = a * b; return a; }
DUAL_T __device__ __forceinline__ bool operator<(const D& a, const D& b) { return a.v < b.v; }
DUAL_T __device__ __forceinline__ bool operator>(const D& a, const D& b) { return a.v > b.v; }

// Elementary functions: value from the scalar routine, derivative from the calculus rule.
DUAL_T __device__ __forceinline__ D lf_rcp(const D& a) {
  T r = lf_rcp(a.v);
  return chain(a, r, -r * r);
}
DUAL_T __device__ __forceinline__ D operator/(const D& a, const D& b) { return a * lf_rcp(b); }
DUAL_T __device__ __forceinline__ D lf_rsqrt(const D& a) {
  T r = lf_rsqrt(a.v);
  return chain(a, r, (T)-0.5 * r * r * r);
}
DUAL_T __device__ __forceinline__ D lf_sqrt(const D& a) {
  T s = lf_sqrt(a.v);
  return chain(a, s, (T)0.5 * lf_rcp(s));
}
DUAL_T __device__ __forceinline__ D lf_atan(const D& a) {
  return chain(a, lf_atan(a.v), lf_rcp((T)1 + a.v * a.v));
}
DUAL_T __device__ __forceinline__ D lf_atanh(const D& a) {
  return chain(a, lf_atanh(a.v), lf_rcp(((T)1 - a.v) * ((T)1 + a.v)));
}
DUAL_T __device__ __forceinline__ D lf_log(const D& a) { return chain(a, lf_log(a.v), lf_rcp(a.v)); }
DUAL_T __device__ __forceinline__ D lf_log1p(const D& a) {
  return chain(a, lf_log1p(a.v), lf_rcp((T)1 + a.v));
}
DUAL_T __device__ __forceinline__ D lf_acos(const D& a) {
  return chain(a, lf_acos(a.v), -lf_rsqrt(((T)1 - a.v) * ((T)1 + a.v)));
}
DUAL_T __device__ __forceinline__ D lf_fma(const D& a, const D& b, const D& c) { return a * b + c; }
DUAL_T __device__ __forceinline__ D lf_cos(const D& a) { return chain(a, lf_cos(a.v), -lf_sin(a.v)); }
DUAL_T __device__ __forceinline__ D lf_sin(const D& a) { return chain(a, lf_sin(a.v), lf_cos(a.v)); }

#undef D
#undef DUAL_T

// Third derivatives (psi_xxx, psi_xxy, psi_xyy, psi_yyy) of one explicit component: psi_ij of
// the closed form on dual numbers over the offset.
template <class T>
LF_INLINE void comp_d3(const CompT<T>& c, T dx, T dy, T (&d3)[4]) {
  typedef Dual<T, 2> D;
  Out5<D> o;
  eval_comp_g<T, D>(c, D::var(dx, 0), D::var(dy, 1), o);
  d3[0] = o.pxx.d[0]; d3[1] = o.pxx.d[1]; d3[2] = o.pyy.d[0]; d3[3] = o.pyy.d[1];
}

// The same for one round pseudo-Jaffe member of strength b, core s, cut a.
template <class T>
LF_INLINE void member_d3(T dx, T dy, T b, T s, T a, T (&d3)[4]) {
  typedef Dual<T, 2> D;
  Out5<D> o;
  pje_round(D::var(dx, 0), D::var(dy, 1), D(b), D(s), D(s * s), D(a), D(a * a), o);
  d3[0] = o.pxx.d[0]; d3[1] = o.pxx.d[1]; d3[2] = o.pyy.d[0]; d3[3] = o.pyy.d[1];
}


}  // namespace lf

template <class T, int N> struct scalar_of<lf::Dual<T, N>> { typedef typename scalar_of<T>::type type; };

