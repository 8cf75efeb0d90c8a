// Batched source-plane chi^2 (Eq. chi2_src with the analytic source of Sec. 3.1) and its
// parameter gradient, for thousands of parameter samples and many clusters per launch.
//
// One persistent launch: every block takes work items (one parameter sample of one
// cluster) from an atomic counter.  Items are ordered cluster by cluster, most expensive
// cluster first, so a block re-stages a cluster's tables (bulk copy into shared memory)
// only when the cluster changes.  Per item the block
//   A1  writes the sample's parameters into the component table (transforms km/s -> b,
//       degrees -> radians, kpc -> arcsec) and re-derives the members from the scaling
//       relations of Eq. scaling when those are sampled;
//   A3-A4 sums alpha and psi_ij at every observed image: tasks (image, component slice)
//       with KS slices per image reduced by warp shuffles;
//   A5-A7 forms beta_i = theta_i - a_f alpha_i, A_i = I - a_f Psi_i (or the multi-plane
//       recursion of Sec. 2.2), mu_i = A_i^-1 and M_i = mu_i^T S_i^-1 mu_i in FP64;
//   A8  per family G = sum M_i, g = sum M_i beta_i, beta_model = G^-1 g and
//       chi^2_f = sum (beta_i - beta_model)^T M_i (beta_i - beta_model), then a block
//       reduction to chi^2 of the sample.
// The gradient (A9) holds beta_model at its optimum (d chi^2 / d beta_model = 0), so with
// d_i = beta_i - beta_model, w = M_i d_i and z = mu_i d_i,
//   d chi^2 = sum_i 2 a_f [ -w^T d alpha_i + w^T d Psi_i z ],
// i.e. cotangents alpha_bar = -2 a w and Psi_bar = 2 a sym(w z^T).  A second pass over the
// same (image, slice) tasks contracts them with the derivative of each component's
// (alpha, Psi) with respect to its own fields, obtained by forward-mode dual numbers, and
// with the member scaling-relation chain rule.
#include "lf_internal.h"
#include "lf_eval.cuh"
#include "lf_dual.cuh"

namespace lf {

constexpr int LF_MAX_P = 64;
constexpr int LF_MAX_FREE = 16;
constexpr int LF_MAX_IMG = 2048;
constexpr int LF_TAB_OFF = 512;      // shared header: barrier, item index, reduction scratch
constexpr int LF_HDR = LF_TAB_OFF + 2 * LF_TAB_N * 8;   // then the float-float function tables
constexpr double LF_C_KMS = 299792.458;
constexpr double LF_ARCSEC_PER_RAD = 206264.80624709636;
constexpr double LF_PI = 3.14159265358979323846;

// Per-cluster member tables built by the plan: (L/L*)^(2 lam0), ^beta0, ^alpha0 at the base
// exponents (float-float for the mixed tier) and ln(L/L*).  A sampled exponent e changes a
// factor to f0 exp((e - e0) k ln L), evaluated as f0 (1 + expm1(.)) so that the FP32 rounding
// applies to the small perturbation only.
struct MemPreF { float xh, xl, yh, yl, fb, fs, fa, lnl, fbl, fsl, fal, pad; };
struct MemPreD { double x, y, fb, fs, fa, lnl, pad0, pad1; };

struct PlaneDesc {
  const lf_comp* comp;
  const void* mpre;
  int nc, nm;
  lf_scaling sc;
  double apk;
  uint32_t off_rawc, off_mpre, off_dc;
  uint32_t off_dm;                 // scalar member records (adjoint, flux / time-delay pass)
  uint32_t off_dmp;                // the mixed tier's packed pairs (forward passes); = off_dm else
  uint32_t off_mfac;               // the mixed tier's members' base factors (fb, fs, fa), FP32
  uint32_t off_dma;                // the mixed tier's gradient: each member's change (MemA)
};

struct ClusterDesc {
  int np;
  PlaneDesc pl[LF_MAX_PLANES];
  double r[LF_MAX_PLANES][LF_MAX_PLANES];
  int n_img, n_fam;
  const double* theta;
  const double* sinv;
  const int* fam_off;
  const int* img_fam;
  const double* fam_ratio;
  int P;
  int n_free;
  int free_plane[LF_MAX_FREE], free_comp[LF_MAX_FREE];
  int free_p[LF_MAX_FREE][7];
  int scal_plane;
  int scal_free;
  int scal_p[6];
  int aux;                         // flux (1) and time-delay (2) terms present (one plane)
  const double *aux_mag, *aux_wmag, *aux_td, *aux_wtd;   // per image; weight 0: no measurement
  double td_scale;                 // (1 + z_d) D_d theta_0^2 / c, days
  int n_afree;                     // families whose a_dis is a sampled parameter (one plane)
  int afree_fam[LF_MAX_P], afree_p[LF_MAX_P];
  int p_xform[LF_MAX_P];
  int p_plane[LF_MAX_P];
  int ks;
  int img_stride;                  // FP64 records: doubles per image (LF_FP64 tier)
  int img_stride_f;                // mixed tiers: floats per image
  int img_stride_d;                // mixed tiers: doubles per image (multi-plane state)
  // mixed tiers: positions, distance ratios and S^-1 split for float-float / FP32 use
  const float4* theta_ff;          // [n_img] (x_hi, x_lo, y_hi, y_lo)
  const float2* ratio_ff;          // [n_fam * np]
  const float4* sinv_f;            // [n_img] (xx, xy, yy, 0)
  // the mixed tier's gradient (one plane): every image's member deflection sum at the plan's
  // base fields, FP64 rounded to float-float (x_hi, x_lo, y_hi, y_lo); null: not anchored
  const float4* mbase;
  int mpg_stride;                  // multi-plane adjoint: doubles per image record
  uint32_t off_img, off_imgd, off_fam, off_par, off_free, off_newton, off_fama, off_aux, off_mpg;
  uint32_t off_auxg;               // adjoint of the flux / time-delay terms: per image records
  // shared memory of each launch kind: the common regions, then only the member records and
  // scratch that kind reads (source-plane chi^2; image-plane chi^2; flux / time delay; adjoint)
  uint32_t smem, smem_img, smem_aux, smem_grad;
};

// ------------------------------------------------------------------ transforms -----
// b = 4 pi (v / c)^2 in arcsec, as one constant times v^2 (no FP64 division per sample)
constexpr double LF_VDISP_K = 4.0 * LF_PI * LF_ARCSEC_PER_RAD / (LF_C_KMS * LF_C_KMS);
__host__ __device__ inline double apply_xform(int xf, double v, double apk) {
  switch (xf) {
    case LF_XF_VDISP: return LF_VDISP_K * v * v;
    case LF_XF_DEG: return v * (LF_PI / 180.0);
    case LF_XF_KPC: return v * apk;
    default: return v;
  }
}
__host__ __device__ inline double xform_deriv(int xf, double v, double apk) {
  switch (xf) {
    case LF_XF_VDISP: return 2.0 * LF_VDISP_K * v;
    case LF_XF_DEG: return LF_PI / 180.0;
    case LF_XF_KPC: return apk;
    default: return 1.0;
  }
}


// The scaling relation of the sample: base values with the sampled slots overwritten.
__device__ __forceinline__ void sample_scaling(const ClusterDesc& C, const double* th, lf_scaling& sc) {
  const double apk = C.pl[C.scal_plane].apk;
  for (int k = 0; k < 6; ++k) {
    const int p = C.scal_p[k];
    if (p < 0) continue;
    const double v = apply_xform(C.p_xform[p], th[p], apk);
    if (k == LF_S_BSTAR) sc.b_star = v;
    else if (k == LF_S_CORESTAR) sc.core_star = v;
    else if (k == LF_S_CUTSTAR) sc.cut_star = v;
    else if (k == LF_S_LAM) sc.lam = v;
    else if (k == LF_S_BETA) sc.beta = v;
    else sc.alpha = v;
  }
}

__device__ __forceinline__ void set_field(lf_comp& c, int f, double v) {
  switch (f) {
    case LF_F_X: c.x = v; break;
    case LF_F_Y: c.y = v; break;
    case LF_F_B: c.b = v; break;
    case LF_F_EPS: c.eps = v; break;
    case LF_F_PA: c.pa = v; break;
    case LF_F_CORE: c.core = v; break;
    default: c.cut = v; break;
  }
}

// Sum over the 32 lanes of a warp (every lane takes part and gets the sum).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; the total is returned on thread 0 (0 elsewhere).
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) r += scratch[i];
  }
  return r;
}

// ------------------------------------------------------- dual component evaluation -
// Unit-strength (alpha, Psi) of one explicit component and its derivatives with respect to
// (x, y, eps, pa, core, cut) in tangent slots 0..5, at the offset (dx0, dy0) from its centre.
// S is the offset's scalar: T, or dual numbers over the offset itself (Dual<T, 2>), which
// carry in addition the derivatives of Psi in position (the third derivatives of psi) and,
// through the outer tangents, their derivatives in the fields.
template <class T, class S>
__device__ void comp_dual_g(const lf_comp& rc, S dx0, S dy0, Out5<Dual<S, 6>>& o) {
  typedef Dual<S, 6> DT;
  // d(dx)/dx_c = -1, d(dy)/dy_c = -1
  DT dx = DT::cst(dx0), dy = DT::cst(dy0);
  dx.d[0] = S(-1.0);
  dy.d[1] = S(-1.0);
  DT pa = DT::var(S(rc.pa), 3);
  if (rc.kind == LF_MULTIPOLE3) {
    DT three(3.0);
    multipole3(dx, dy, lf_cos(three * pa), lf_sin(three * pa), o);
    return;
  }
  if (rc.kind == LF_SHEAR) {
    DT two(2.0);
    DT c2 = lf_cos(two * pa), s2 = lf_sin(two * pa);
    o.ax = c2 * dx + s2 * dy;
    o.ay = s2 * dx - c2 * dy;
    o.pxx = c2; o.pyy = -c2; o.pxy = s2;
    return;
  }
  DT core = DT::var(S(rc.core), 4);
  if (rc.kind == LF_NFW) {
    nfw_sph(dx, dy, DT(1.0), lf_rcp(core), o);
    return;
  }
  if (rc.kind == LF_ENFW) {   // unit kappa_s; tangents x, y, eps, pa and core (= r_s)
    DT eps = DT::var(S(rc.eps), 2);
    DT one(1.0), two(2.0);
    DT q = (one - eps) / (one + eps);
    DT c = lf_cos(pa), sn = lf_sin(pa);
    DT irs = lf_rcp(core);
    DT u = (c * dx + sn * dy) * irs, v = (c * dy - sn * dx) * irs;
    DT au, av, puu, pvv, puv;
    enfw_uv<T, DT>(u, v, q, q * q, au, av, puu, pvv, puv);
    DT k2r = two * core;
    rotate_back(c, sn, k2r * au, k2r * av, two * puu, two * pvv, two * puv, o);
    return;
  }
  // eps = 0 is the round profile, as in the forward pass (sie_uv's q = 1 branch keeps the
  // exact first derivative in eps); else the elliptical closed form
  const bool round = rc.eps == 0.0;
  DT eps = DT::var(S(rc.eps), 2);
  DT one(1.0);
  DT q = (one - eps) / (one + eps);
  DT q2 = q * q;
  DT e = round ? DT(0.0) : lf_sqrt((one - q) * (one + q));
  DT qe = round ? DT(0.0) : q / e;
  DT c = lf_cos(pa), sn = lf_sin(pa);
  DT u = c * dx + sn * dy;
  DT v = c * dy - sn * dx;
  DT au, av, puu, pvv, puv;
  DT s2 = core * core;
  sie_uv(u, v, q, q2, e, qe, core, s2, q2 * core, (one + q2) * s2, round, au, av, puu, pvv, puv);
  if (rc.kind == LF_DPIE) {
    DT cut = DT::var(S(rc.cut), 5);
    DT c2 = cut * cut;
    DT bu, bv, quu, qvv, quv;
    sie_uv(u, v, q, q2, e, qe, cut, c2, q2 * cut, (one + q2) * c2, round, bu, bv, quu, qvv, quv);
    au = au - bu; av = av - bv; puu = puu - quu; pvv = pvv - qvv; puv = puv - quv;
  }
  rotate_back(c, sn, au, av, puu, pvv, puv, o);
}

// The same at the position (px, py), offsets taken in FP64.
template <class T>
__device__ void comp_dual(const lf_comp& rc, double px, double py, Out5<Dual<T, 6>>& o) {
  comp_dual_g<T, T>(rc, (T)(px - rc.x), (T)(py - rc.y), o);
}

// The unit-strength lens potential of one explicit component (the closed forms of the forward
// flux / time-delay pass, on raw fields) with its derivatives in the same six tangent slots.
template <class T>
__device__ Dual<T, 6> comp_potential_dual(const lf_comp& rc, T dx0, T dy0) {
  typedef Dual<T, 6> DT;
  DT dx = DT::cst(dx0), dy = DT::cst(dy0);
  dx.d[0] = (T)-1;
  dy.d[1] = (T)-1;
  DT pa = DT::var((T)rc.pa, 3);
  if (rc.kind == LF_MULTIPOLE3) {   // r^2 cos 3(phi - pa)
    const DT r2 = dx * dx + dy * dy;
    if (!(r2.v > (T)0)) return DT(0.0);
    const DT ir = lf_rsqrt(r2), nx = dx * ir, ny = dy * ir;
    const DT three(3.0);
    const DT c3 = lf_cos(three * pa), s3 = lf_sin(three * pa);
    return r2 * (c3 * nx * (nx * nx - three * ny * ny) + s3 * ny * (three * nx * nx - ny * ny));
  }
  if (rc.kind == LF_SHEAR) {
    const DT two(2.0);
    return DT(0.5) * lf_cos(two * pa) * (dx * dx - dy * dy) + lf_sin(two * pa) * dx * dy;
  }
  DT core = DT::var((T)rc.core, 4);
  if (rc.kind == LF_NFW) return nfw_potential(dx, dy, DT(1.0), lf_rcp(core));
  DT eps = DT::var((T)rc.eps, 2);
  DT one(1.0);
  DT q = (one - eps) / (one + eps);
  DT c = lf_cos(pa), sn = lf_sin(pa);
  if (rc.kind == LF_ENFW) {   // 2 r_s^2 psi_cse(u / r_s, v / r_s)
    DT irs = lf_rcp(core);
    DT u = (c * dx + sn * dy) * irs, v = (c * dy - sn * dx) * irs;
    return DT(2.0) * core * core * enfw_potential_uv(u, v, q, q * q);
  }
  const bool round = rc.eps == 0.0;
  DT q2 = q * q;
  DT e = round ? DT(0.0) : lf_sqrt((one - q) * (one + q));
  DT qe = round ? DT(0.0) : q / e;
  DT u = c * dx + sn * dy;
  DT v = c * dy - sn * dx;
  DT s2 = core * core;
  DT p = sie_potential_uv(u, v, q, q2, e, qe, core, s2, q2 * core, (one + q2) * s2, round);
  if (rc.kind == LF_DPIE) {
    DT cut = DT::var((T)rc.cut, 5);
    DT c2 = cut * cut;
    p = p - sie_potential_uv(u, v, q, q2, e, qe, cut, c2, q2 * cut, (one + q2) * c2, round);
  }
  return p;
}

template <class T, int N>
__device__ __forceinline__ T contract(const Out5<Dual<T, N>>& o, const T* cot, int slot) {
  if (slot < 0)
    return cot[0] * o.ax.v + cot[1] * o.ay.v + cot[2] * o.pxx.v + cot[3] * o.pyy.v + cot[4] * o.pxy.v;
  return cot[0] * o.ax.d[slot] + cot[1] * o.ay.d[slot] + cot[2] * o.pxx.d[slot] +
         cot[3] * o.pyy.d[slot] + cot[4] * o.pxy.d[slot];
}

// ------------------------------------------------------------------ the kernel -----
// Member accessors shared by the two member records.
template <class T> __device__ __forceinline__ T mem_s(const MemT<T>& m) { return m.s; }
template <class T> __device__ __forceinline__ T mem_a(const MemT<T>& m) { return m.a; }
__device__ __forceinline__ float mem_s(const MemX& m) { return m.sh; }
__device__ __forceinline__ float mem_a(const MemX& m) { return m.ah; }

// Sampled components of every sample, digested in one pass over (sample, component) before the
// chi^2 kernel (their FP64 set-up is then off the per-sample critical path).
template <int MODE>
__global__ void k_chi2_prep(const ClusterDesc* __restrict__ cds, int spc, int S, int nfree_max,
                            const double* __restrict__ theta, void* dig, lf_comp* raw) {
  typedef typename std::conditional<MODE != LF_FP64, float, double>::type T;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;    // dense over (sample, component)
  const int s = t / nfree_max, f = t - s * nfree_max;
  if (s >= S) return;
  const ClusterDesc& C = cds[s / spc];
  if (f >= C.n_free) return;
  const int idx = s * LF_MAX_FREE + f;
  const PlaneDesc& P = C.pl[C.free_plane[f]];
  lf_comp rc = P.comp[C.free_comp[f]];
  for (int fld = 0; fld < 7; ++fld) {
    const int p = C.free_p[f][fld];
    if (p >= 0) set_field(rc, fld, apply_xform(C.p_xform[p], theta[(size_t)s * C.P + p], P.apk));
  }
  raw[idx] = rc;
  digest_one_comp<T>(rc, reinterpret_cast<CompT<T>*>(dig)[idx]);
}

// Flux / time-delay records (doubles): per image psi, psi_xxx, psi_xxy, psi_xyy, psi_yyy, y_i,
// d_i; per family m_src, Delta t_0 and lambda = G^-1 beta_model_bar (2); the adjoint's per-image
// record psi_bar, T_bar (4), beta_bar (2), A_bar (00, 11, 01 + 10), (beta_model - beta)_bar (2),
// M (00, 01, 11), one spare.
constexpr uint32_t LF_AUXI = 7, LF_AUXF = 4, LF_AUXG = 16;

// Record of one image in the mixed tiers (floats): [0..9] alpha, psi sums as float-float pairs
// (then the five cotangents in [0..4]); [10..13] beta (x_hi, x_lo, y_hi, y_lo); [14..16] M;
// [17..20] mu (00, 01, 10, 11).
constexpr int IMGF = 22;

// Member pairs per FP32 partial sum of the mixed tier's packed loop (64 members; each partial is
// then folded into float-float).
constexpr int LF_PAIR_CHUNK = 32;

#ifndef LF_CHI2_THREADS
#define LF_CHI2_THREADS 512
#endif
#ifndef LF_CHI2_MINB
#define LF_CHI2_MINB 1
#endif
#ifndef LF_CHI2_BLOCK
#define LF_CHI2_BLOCK 256
#endif
// The mixed tier's forward passes (packed members) run under a register cap that lets
// LF_CHI2_FWD_MINB blocks of up to LF_CHI2_FWD_THREADS threads share an SM: each block works
// on one sample, whose ~100 image pairs fill only a few warps, so warps come from more
// resident samples.
#ifndef LF_CHI2_IPT
#define LF_CHI2_IPT 2     // images per task in the mixed tiers' evaluation
#endif
#ifndef LF_CHI2_FWD_THREADS
#define LF_CHI2_FWD_THREADS 128
#endif
#ifndef LF_CHI2_FWD_MINB
#define LF_CHI2_FWD_MINB 5
#endif
#define LF_CHI2_CAPPED(MODE, GRAD, PASS) ((MODE) == LF_MIXED && !(GRAD) && (PASS) != 2)
// largest block a plan of this tier may use
// Threads per block of the mixed tier's gradient launch: at its 128 registers per thread and
// ~50 KB of shared memory per block, 4 blocks of 128 fill the SM's registers (16 warps)
#ifndef LF_CHI2_GRAD_BLOCK
#define LF_CHI2_GRAD_BLOCK 128
#endif
static inline int chi2_max_block(int precision) {
  return precision == LF_MIXED ? std::min(LF_CHI2_THREADS, LF_CHI2_FWD_THREADS) : LF_CHI2_THREADS;
}
// PASS 0: source-plane chi^2 (and its gradient when GRAD).  PASS 1: image-plane chi^2 of
// Eq. chi2_img with model images found by `iters` Newton steps from the observed images
// towards the family's analytic source (written to chi2), and the image-plane rms (to rms).
// ----------------------------------------------------- flux / time-delay helpers ---
__device__ __forceinline__ void mem_geom(const MemT<float>& m, float& xh, float& xl, float& yh,
                                         float& yl, float& b, float& s, float& a) {
  xh = m.xh; xl = m.xl; yh = m.yh; yl = m.yl; b = m.b; s = m.s; a = m.a;
}
__device__ __forceinline__ void mem_geom(const MemT<double>& m, double& xh, double& xl, double& yh,
                                         double& yl, double& b, double& s, double& a) {
  xh = m.xh; xl = 0.0; yh = m.yh; yl = 0.0; b = m.b; s = m.s; a = m.a;
}
__device__ __forceinline__ void mem_geom(const MemX& m, float& xh, float& xl, float& yh, float& yl,
                                         float& b, float& s, float& a) {
  xh = m.xh; xl = m.xl; yh = m.yh; yl = m.yl; b = m.b; s = m.sh; a = m.ah;
}

// psi and its third derivatives summed over the components [k0, k1) of one plane at one
// position: out = (psi, psi_xxx, psi_xxy, psi_xyy, psi_yyy); psi in float-float (mixed tiers)
// or FP64, the third derivatives in T.
template <class T, class Mem>
__device__ void aux_sum(const CompT<T>* dc, int nc, const Mem* dm, int nm, int k0, int k1, T pxh,
                        T pxl, T pyh, T pyl, double (&out)[5]) {
  ff pf = ff_zero();
  double pd = 0.0;
  T s3[4] = {(T)0, (T)0, (T)0, (T)0};
  const int c1 = min(k1, nc);
  for (int c = k0; c < c1; ++c) {
    const CompT<T>& C = dc[c];
    if (C.kind == 0) continue;
    const T dx = offset_of(pxh, pxl, C.xh, C.xl), dy = offset_of(pyh, pyl, C.yh, C.yl);
    const T p = comp_potential(C, dx, dy);
    T d3[4];
    comp_d3(C, dx, dy, d3);
    if constexpr (std::is_same<T, float>::value) ff_acc(pf, p); else pd += p;
    for (int q = 0; q < 4; ++q) s3[q] += d3[q];
  }
  const int m_beg = max(k0, nc) - nc, m_end = min(k1, nc + nm) - nc;
  for (int m = m_beg; m < m_end; ++m) {
    T xh, xl, yh, yl, b, sc, ac;
    mem_geom(dm[m], xh, xl, yh, yl, b, sc, ac);
    const T dx = offset_of(pxh, pxl, xh, xl), dy = offset_of(pyh, pyl, yh, yl);
    const T p = pje_potential(::lf_fma(dx, dx, dy * dy), b, sc, ac);
    T d3[4];
    member_d3(dx, dy, b, sc, ac, d3);
    if constexpr (std::is_same<T, float>::value) ff_acc(pf, p); else pd += p;
    for (int q = 0; q < 4; ++q) s3[q] += d3[q];
  }
  if constexpr (std::is_same<T, float>::value) out[0] = ff_to_double(pf); else out[0] = pd;
  for (int q = 0; q < 4; ++q) out[q + 1] = (double)s3[q];
}

// The third derivatives of psi alone, summed over [k0, k1) at one position (multi-plane adjoint).
template <class T, class Mem>
__device__ void d3_sum(const CompT<T>* dc, int nc, const Mem* dm, int nm, int k0, int k1, T pxh,
                       T pxl, T pyh, T pyl, double (&out)[4]) {
  T s3[4] = {(T)0, (T)0, (T)0, (T)0};
  const int c1 = min(k1, nc);
  for (int c = k0; c < c1; ++c) {
    const CompT<T>& C = dc[c];
    if (C.kind == 0) continue;
    T d3[4];
    comp_d3(C, offset_of(pxh, pxl, C.xh, C.xl), offset_of(pyh, pyl, C.yh, C.yl), d3);
    for (int q = 0; q < 4; ++q) s3[q] += d3[q];
  }
  const int m_beg = max(k0, nc) - nc, m_end = min(k1, nc + nm) - nc;
  for (int m = m_beg; m < m_end; ++m) {
    T xh, xl, yh, yl, b, sc, ac;
    mem_geom(dm[m], xh, xl, yh, yl, b, sc, ac);
    T d3[4];
    member_d3(offset_of(pxh, pxl, xh, xl), offset_of(pyh, pyl, yh, yl), b, sc, ac, d3);
    for (int q = 0; q < 4; ++q) s3[q] += d3[q];
  }
  for (int q = 0; q < 4; ++q) out[q] = (double)s3[q];
}

// M of a mixed-tier image record: FP32 words 14..16, or float-float words 14..19 when word 21
// is set (the forward source-plane chi^2).
__device__ __forceinline__ void image_M(const float* r, ff& M00, ff& M01, ff& M11) {
  if (r[21] != 0.0f) {
    M00 = ff_make(r[14], r[15]); M01 = ff_make(r[16], r[17]); M11 = ff_make(r[18], r[19]);
  } else {
    M00 = ff_make(r[14], 0.f); M01 = ff_make(r[15], 0.f); M11 = ff_make(r[16], 0.f);
  }
}

// Float-float sum over the block (every thread takes part); the total is returned on thread 0.
__device__ __forceinline__ ff block_sum_ff(ff v, ff* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_xor(v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  ff r = ff_zero();
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = ff_add(r, scratch[w]);
  return r;
}

template <int MODE, bool GRAD, int PASS = 0>   // MODE: LF_FP64, LF_MIXED or LF_FF
__global__ void __launch_bounds__(LF_CHI2_CAPPED(MODE, GRAD, PASS) ? LF_CHI2_FWD_THREADS : LF_CHI2_THREADS,
                                  LF_CHI2_CAPPED(MODE, GRAD, PASS) ? LF_CHI2_FWD_MINB : LF_CHI2_MINB) k_chi2(const ClusterDesc* __restrict__ cds,
                                              const int* __restrict__ corder, int spc, int S,
                                              const double* __restrict__ theta, double* chi2,
                                              double* grad, int* counter, int chunk,
                                              const void* __restrict__ free_dig,
                                              const lf_comp* __restrict__ free_raw,
                                              int iters = 0, double* rms = nullptr) {
  constexpr bool MIXED = MODE != LF_FP64;
  typedef typename std::conditional<MIXED, float, double>::type T;
  typedef typename std::conditional<MODE == LF_MIXED, MemPreF, MemPreD>::type MemPre;
  typedef typename std::conditional<MODE == LF_FF, MemX, MemT<T>>::type Mem;
  // the mixed tier's forward passes evaluate members two at a time (packed pair records, f32x2);
  // the adjoint and the flux / time-delay pass read the scalar records
  constexpr bool PACKM = (MODE == LF_MIXED) && !GRAD && PASS != 2;
  // PASS 2: the flux / time-delay terms (the forward pass, or with GRAD their adjoint too); the
  // other instantiations carry none of that code
  constexpr bool AUX = PASS == 2;
  // the source-plane chi^2 of the mixed tiers (and its adjoint) keeps every image's M in
  // float-float words
  constexpr bool FFM = MIXED && PASS == 0;
  constexpr bool FFSUM = PACKM && PASS == 0;
  // images per evaluation task (independent chains per thread; with packed members, two
  // member evaluations per instruction and chain); the FP64 tier takes two
  constexpr int IPT = MIXED ? LF_CHI2_IPT : 2;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  int* s_item = reinterpret_cast<int*>(smem + 8);
  int* wctr = reinterpret_cast<int*>(smem + 288);           // warp-task counter (packed members)
  double* scratch = reinterpret_cast<double*>(smem + 16);   // 32 doubles
  const int tid = threadIdx.x;
  float2* tab = reinterpret_cast<float2*>(smem + LF_TAB_OFF);
  if (tid == 0) {
    mbar_init(bar, 1);
    *wctr = 0;
  }
  init_ff_tables(tab);
  if (tid == 0) *s_item = atomicAdd(counter, 1);     // the first work item
  __syncthreads();
  uint32_t phase = 0;
  int cur = -1;

  for (;;) {
    // the item was taken during the previous item (its atomic's latency hidden behind that
    // item's work) and published by the barriers since
    const int w = *s_item;
    if (w >= S) break;
    const int c = corder[w / spc];
    const int s = c * spc + (w % spc);
    const ClusterDesc& C = cds[c];
#if LF_CHECK_BOUNDS
    {
      // the host's layout of this launch kind fits the block's window, and the image and
      // family index arrays stay in range (a failed check skips the sample)
      const uint32_t need = GRAD ? C.smem_grad : PASS == 1 ? C.smem_img : PASS == 2 ? C.smem_aux : C.smem;
      bool okb = need <= lf_dyn_smem() && C.fam_off[0] == 0 && C.fam_off[C.n_fam] == C.n_img;
      for (int f = tid; f < C.n_fam; f += blockDim.x) okb = okb && C.fam_off[f] < C.fam_off[f + 1];
      for (int i = tid; i < C.n_img; i += blockDim.x) okb = okb && C.img_fam[i] >= 0 && C.img_fam[i] < C.n_fam;
      if (!__syncthreads_and(LF_CHECK(okb) ? 1 : 0)) {
        if (tid == 0) {
          chi2[s] = NAN;
          *s_item = atomicAdd(counter, 1);
        }
        __syncthreads();
        continue;
      }
    }
#endif
    double* th = reinterpret_cast<double*>(smem + C.off_par);
    double* gacc = th + C.P;
    lf_comp* fraw = reinterpret_cast<lf_comp*>(smem + C.off_free);
    double* img = reinterpret_cast<double*>(smem + C.off_img);      // LF_FP64 records
    float* imgf = reinterpret_cast<float*>(smem + C.off_img);       // mixed-tier records
    double* imgd = reinterpret_cast<double*>(smem + C.off_imgd);    // mixed-tier multi-plane state
    double* fam = reinterpret_cast<double*>(smem + C.off_fam);
    // single plane: this sample's a_dis per family (fixed, or a sampled parameter)
    double* fa = reinterpret_cast<double*>(smem + C.off_fama);
    float2* faf = reinterpret_cast<float2*>(fa + C.n_fam);
    int* fap = reinterpret_cast<int*>(faf + C.n_fam);
    for (int p = tid; p < C.P; p += blockDim.x) {
      th[p] = theta[(size_t)s * C.P + p];
      if (GRAD) gacc[p] = 0.0;
    }
    const bool fresh = (c != cur);
    if (fresh) {
      bool ok = true;
      for (int j = 0; j < C.np && ok; ++j) {
        const PlaneDesc& P = C.pl[j];
        if (P.nc > 0) {
          ok = stage_to_smem(smem + P.off_rawc, P.comp, (uint32_t)P.nc * 64u, bar, phase & 1u);
          ++phase;
        }
      }
      if (!ok) return;
      for (int j = 0; j < C.np; ++j) {
        const PlaneDesc& P = C.pl[j];
        const lf_comp* rawc = reinterpret_cast<const lf_comp*>(smem + P.off_rawc);
        CompT<T>* dc = reinterpret_cast<CompT<T>*>(smem + P.off_dc);
        for (int i = tid; i < P.nc; i += blockDim.x) digest_one_comp<T>(rawc[i], dc[i]);
      }
      cur = c;
    }
    __syncthreads();
    if (tid == 0) *s_item = atomicAdd(counter, 1);    // every thread has read this item

    // ---- A1: this sample's parameters into the tables
    for (int f = tid; f < C.n_free; f += blockDim.x) {
      const PlaneDesc& P = C.pl[C.free_plane[f]];
      CompT<T>* slot = reinterpret_cast<CompT<T>*>(smem + P.off_dc) + C.free_comp[f];
      if (free_dig) {            // digested by k_chi2_prep
        *slot = reinterpret_cast<const CompT<T>*>(free_dig)[(size_t)s * LF_MAX_FREE + f];
        if (GRAD) fraw[f] = free_raw[(size_t)s * LF_MAX_FREE + f];
      } else {
        const lf_comp* rawc = reinterpret_cast<const lf_comp*>(smem + P.off_rawc);
        lf_comp rc = rawc[C.free_comp[f]];
        for (int fld = 0; fld < 7; ++fld) {
          int p = C.free_p[f][fld];
          if (p >= 0) set_field(rc, fld, apply_xform(C.p_xform[p], th[p], P.apk));
        }
        fraw[f] = rc;
        digest_one_comp<T>(rc, *slot);
      }
    }
    if (C.np == 1) {
      // a sampled a_dis outside (0, 1] makes the family's chi^2 non-finite, i.e. +inf
      for (int f = tid; f < C.n_fam; f += blockDim.x) {
        int p = -1;
        for (int q = 0; q < C.n_afree; ++q)
          if (C.afree_fam[q] == f) p = C.afree_p[q];
        double a = C.fam_ratio[f];
        float2 a2 = C.ratio_ff[f];
        if (p >= 0) {
          a = th[p];
          if (!(a > 0.0 && a <= 1.0)) a = NAN;
          split_ff(a, a2.x, a2.y);
        }
        fa[f] = a;
        faf[f] = a2;
        fap[f] = p;
      }
    }
    for (int j = 0; j < C.np; ++j) {
      const PlaneDesc& P = C.pl[j];
      const bool sampled = (j == C.scal_plane) && C.scal_free;
      if (P.nm == 0 || !(fresh || sampled)) continue;
      lf_scaling sc = P.sc;
      if (sampled) sample_scaling(C, th, sc);
      const bool lam_free = sampled && C.scal_p[LF_S_LAM] >= 0;
      const bool beta_free = sampled && C.scal_p[LF_S_BETA] >= 0;
      const bool alpha_free = sampled && C.scal_p[LF_S_ALPHA] >= 0;
      const MemPre* mp = reinterpret_cast<const MemPre*>(P.mpre);   // plan table, L2-resident
      Mem* dm = reinterpret_cast<Mem*>(smem + P.off_dm);
      const T bstar = (T)sc.b_star, cstar = (T)sc.core_star, astar = (T)sc.cut_star;
      // the gradient's anchored member sum: the plan's base scaling and the sample's change
      const float bstar0 = (float)P.sc.b_star, cstar0 = (float)P.sc.core_star, astar0 = (float)P.sc.cut_star;
      const float dbstar = (float)(sc.b_star - P.sc.b_star), dcstar = (float)(sc.core_star - P.sc.core_star),
                  dastar = (float)(sc.cut_star - P.sc.cut_star);
      const int n_lanes = PACKM ? 2 * (int)mem_records<MemPair>(P.nm) : P.nm;
      for (int i = tid; i < n_lanes; i += blockDim.x) {
        if constexpr (PACKM) {
          MemPair* dp = reinterpret_cast<MemPair*>(smem + P.off_dmp);
          if (i >= P.nm) {      // zero-strength pad of an odd member count
            pair_lane(dp[i >> 1], i & 1, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f, 2.f);
            continue;
          }
          if (!fresh && !lam_free && !beta_free && !alpha_free) {
            // only the scaling relation's amplitudes are sampled: the centres stay, and the base
            // factors are in shared memory (no reload of the plan's table)
            const float3 f3 = reinterpret_cast<const float3*>(smem + P.off_mfac)[i];
            pair_lane_scale(dp[i >> 1], i & 1, bstar * f3.x, cstar * f3.y, astar * f3.z);
            continue;
          }
          if (fresh) {
            const MemPreF& mb = reinterpret_cast<const MemPreF*>(P.mpre)[i];
            reinterpret_cast<float3*>(smem + P.off_mfac)[i] = make_float3(mb.fb, mb.fs, mb.fa);
          }
        }
        const MemPre& m = mp[i];
        if constexpr (MODE == LF_FF) {
          const double fb = lam_free ? exp(2.0 * sc.lam * m.lnl) : m.fb;
          const double fs = beta_free ? exp(sc.beta * m.lnl) : m.fs;
          const double fa = alpha_free ? exp(sc.alpha * m.lnl) : m.fa;
          digest_member_x(m.x, m.y, sc.b_star * fb, sc.core_star * fs, sc.cut_star * fa, m.lnl,
                          dm[i], fb, fs);
        } else {
          T fb, fs, fa;
          MemT<T> d;
          if constexpr (MODE == LF_MIXED) {
            const float eb = lam_free ? expm1f((float)(2.0 * (sc.lam - P.sc.lam)) * m.lnl) : 0.f;
            const float es = beta_free ? expm1f((float)(sc.beta - P.sc.beta) * m.lnl) : 0.f;
            const float ea = alpha_free ? expm1f((float)(sc.alpha - P.sc.alpha) * m.lnl) : 0.f;
            fb = lam_free ? m.fb + fmaf(m.fb, eb, m.fbl) : m.fb;
            fs = beta_free ? m.fs + fmaf(m.fs, es, m.fsl) : m.fs;
            fa = alpha_free ? m.fa + fmaf(m.fa, ea, m.fal) : m.fa;
            d.xh = m.xh; d.xl = m.xl; d.yh = m.yh; d.yl = m.yl;
            if (GRAD && C.mbase && j == 0) {
              // b - b0 = (b* - b0*) f_b + b0* f_b0 expm1(2 dlam ln L), and alike for the core and
              // the cut: FP32 rounds the change, not the field
              MemA& q = reinterpret_cast<MemA*>(smem + P.off_dma)[i];
              const float s0 = cstar0 * m.fs, a0 = astar0 * m.fa;
              q.db = fmaf(dbstar, fb, bstar0 * m.fb * eb);
              q.ds = fmaf(dcstar, fs, s0 * es);
              q.da = fmaf(dastar, fa, a0 * ea);
              q.s0 = s0;
              q.a0 = a0;
              q.s02 = s0 * s0;
              q.a02 = a0 * a0;
              q.pad = 0.f;
            }
          } else {
            fb = lam_free ? exp(2.0 * sc.lam * m.lnl) : m.fb;
            fs = beta_free ? exp(sc.beta * m.lnl) : m.fs;
            fa = alpha_free ? exp(sc.alpha * m.lnl) : m.fa;
            d.xh = m.x; d.xl = 0; d.yh = m.y; d.yl = 0;
          }
          d.b = bstar * fb;
          d.s = cstar * fs;
          d.a = astar * fa;
          d.bd = d.b * (d.a - d.s);
          d.apc = d.a + d.s;
          d.fb = fb;
          d.fs = fs;
          d.s2 = d.s * d.s;
          d.a2 = d.a * d.a;
          d.loglr = (T)m.lnl;
          d.pad0 = (T)0;
          d.pad1 = (T)0;
          if constexpr (PACKM)
            pair_lane(reinterpret_cast<MemPair*>(smem + P.off_dmp)[i >> 1], i & 1, d.xh, d.xl, d.yh, d.yl,
                      d.b, d.s, d.a);
          else
            dm[i] = d;
        }
      }
    }
    __syncthreads();

    // ---- A3-A6: alpha and Psi at every image, plane by plane.  A task is (image pair,
    // component slice): two images per thread give two independent evaluation chains.
    const int n_img = C.n_img, KS = C.ks, IS = C.img_stride, ISF = C.img_stride_f,
              ISD = C.img_stride_d;
    const int n_unit = (n_img + IPT - 1) / IPT;
    // The units that do not fill whole warps (the tail) share one warp with more component
    // slices each (KST), so that no warp runs the whole component loop with a few active
    // lanes.  Main tasks end on a warp boundary, so each warp has one slice count.
    const int n_main = (n_unit * KS / 32) * (32 / KS);
    const int n_tail = n_unit - n_main;
    int KST = KS;
    while (n_tail > 0 && n_tail * KST * 2 <= 32) KST *= 2;
    const int t_main = n_main * KS;
    const int ntask = t_main + n_tail * KST;
    // pos: null = the observed images; else positions (x, y) at pos[4 i], pos[4 i + 1]
    auto eval_planes = [&](const double* pos) {
    for (int j = 0; j < C.np; ++j) {
      const PlaneDesc& P = C.pl[j];
      const CompT<T>* dc = reinterpret_cast<const CompT<T>*>(smem + P.off_dc);
      const Mem* dm = reinterpret_cast<const Mem*>(smem + P.off_dm);
      const int K = P.nc + (PACKM ? (int)mem_records<MemPair>(P.nm) : P.nm);   // slices of these units
      // position of image i on plane j as float-float (observed, given, or the recursion's theta_j)
      auto image_pos = [&](int i, float& xh, float& xl, float& yh, float& yl) {
        if (j == 0 && !pos) {
          const float4 tf = C.theta_ff[i];
          xh = tf.x; xl = tf.y; yh = tf.z; yl = tf.w;
        } else if (j == 0) {
          split_ff(pos[4 * i], xh, xl);
          split_ff(pos[4 * i + 1], yh, yl);
        } else {
          split_ff(imgd[i * ISD + 0], xh, xl);
          split_ff(imgd[i * ISD + 1], yh, yl);
        }
      };
      if constexpr (PACKM) {
        // Warp tasks taken from a block counter, most expensive first: groups of 32 member tasks
        // (the main (image pair, slice) tasks, then the tail group), then groups of 32 images
        // whose explicit components (float-float halos, shear, ...) one lane each evaluates.  The
        // member warps do no explicit work, so the warps that finish their member groups early
        // (the tail group's) take the explicit groups instead of waiting at the barrier.
        const MemPair* dp = reinterpret_cast<const MemPair*>(smem + P.off_dmp);
        const int K2 = (int)mem_records<MemPair>(P.nm);
        const int lane = tid & 31;
        const int n_mw = (ntask + 31) / 32;
        const int n_wt = n_mw + (P.nc > 0 ? (n_img + 31) / 32 : 0);
        for (;;) {
          int wt = 0;
          if (lane == 0) wt = atomicAdd(wctr, 1);
          wt = __shfl_sync(0xffffffffu, wt, 0);
          if (wt >= n_wt) break;
          if (wt < n_mw) {
            const int t = 32 * wt + lane;
            const bool act = t < ntask;
            const bool tail = t >= t_main;
            const int ks = tail ? KST : KS;             // uniform over each group
            const int tt = tail ? t - t_main : t;
            const int pr = act ? (tail ? n_main + tt / KST : tt / KS) : 0;
            const int k = act ? (tail ? tt - (pr - n_main) * KST : tt - pr * KS) : 0;
            const int k0 = (int)((long long)K2 * k / ks), k1 = (int)((long long)K2 * (k + 1) / ks);
            float xh[IPT], xl[IPT], yh[IPT], yl[IPT];
            int ii[IPT];
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
              ii[q] = min(IPT * pr + q, n_img - 1);
              image_pos(ii[q], xh[q], xl[q], yh[q], yl[q]);
            }
            ff acc[5][IPT];
#pragma unroll
            for (int c5 = 0; c5 < 5; ++c5)
#pragma unroll
              for (int q = 0; q < IPT; ++q) acc[c5][q] = ff_zero();
            if (act) accumulate_packed<IPT>(dp, P.nm, k0, k1, LF_PAIR_CHUNK, xh, xl, yh, yl, acc);
            for (int off = 1; off < ks; off <<= 1)
#pragma unroll
              for (int c5 = 0; c5 < 5; ++c5)
#pragma unroll
                for (int q = 0; q < IPT; ++q) acc[c5][q] = ff_add(acc[c5][q], ff_shfl_xor(acc[c5][q], off));
            if (act && k == 0) {
#pragma unroll
              for (int q = 0; q < IPT; ++q) {
                if (q > 0 && ii[q] == ii[q - 1]) break;     // the clamped repeats of the last unit
                for (int c5 = 0; c5 < 5; ++c5) {
                  imgf[ii[q] * ISF + 2 * c5] = acc[c5][q].hi;
                  imgf[ii[q] * ISF + 2 * c5 + 1] = acc[c5][q].lo;
                }
              }
            }
          } else {
            const int i = 32 * (wt - n_mw) + lane;
            if (i < n_img) {
              float xh, xl, yh, yl;
              image_pos(i, xh, xl, yh, yl);
              ff e5[5];
              for (int c5 = 0; c5 < 5; ++c5) e5[c5] = ff_zero();
              for (int c = 0; c < P.nc; ++c) {
                const CompT<float>& Cc = dc[c];
                if (Cc.kind == 0) continue;
                ff ax, ay;
                Out5<float> o;
                eval_comp_mixed_t<true>(Cc, xh, xl, yh, yl, tab, ax, ay, o);
                e5[0] = ff_add(e5[0], ax);
                e5[1] = ff_add(e5[1], ay);
                ff_acc(e5[2], o.pxx); ff_acc(e5[3], o.pyy); ff_acc(e5[4], o.pxy);
              }
              for (int c5 = 0; c5 < 5; ++c5) {
                imgf[i * ISF + 10 + 2 * c5] = e5[c5].hi;
                imgf[i * ISF + 11 + 2 * c5] = e5[c5].lo;
              }
            }
          }
        }
        __syncthreads();
        if (P.nc > 0) {
          // explicit components' sums into the members' (record words 10..19 are free until the
          // per-image algebra writes them)
          for (int i = tid; i < n_img; i += blockDim.x) {
            float* r = imgf + i * ISF;
            for (int c5 = 0; c5 < 5; ++c5) {
              const ff v = ff_add(ff_make(r[2 * c5], r[2 * c5 + 1]), ff_make(r[10 + 2 * c5], r[11 + 2 * c5]));
              r[2 * c5] = v.hi;
              r[2 * c5 + 1] = v.lo;
            }
          }
        }
        if (tid == 0) *wctr = 0;      // for the next plane (the barrier below orders it)
      } else
      for (int base = 0; base < ntask; base += blockDim.x) {
        const int t = base + tid;
        const bool act = t < ntask;
        const bool tail = t >= t_main;
        const int ks = tail ? KST : KS;             // uniform over each warp
        const int tt = tail ? t - t_main : t;
        const int pr = act ? (tail ? n_main + tt / KST : tt / KS) : 0;
        const int k = act ? (tail ? tt - (pr - n_main) * KST : tt - pr * KS) : 0;
        const int ia = 2 * pr, ib = min(2 * pr + 1, n_img - 1);
        const int k0 = (int)((long long)K * k / ks), k1 = (int)((long long)K * (k + 1) / ks);
        if constexpr (MIXED) {
          float xh[IPT], xl[IPT], yh[IPT], yl[IPT];
          int ii[IPT];
#pragma unroll
          for (int q = 0; q < IPT; ++q) ii[q] = min(IPT * pr + q, n_img - 1);
#pragma unroll
          for (int q = 0; q < IPT; ++q) {
            if (j == 0 && !pos) {
              const float4 tf = C.theta_ff[ii[q]];
              xh[q] = tf.x; xl[q] = tf.y; yh[q] = tf.z; yl[q] = tf.w;
            } else if (j == 0) {
              split_ff(pos[4 * ii[q]], xh[q], xl[q]);
              split_ff(pos[4 * ii[q] + 1], yh[q], yl[q]);
            } else {
              split_ff(imgd[ii[q] * ISD + 0], xh[q], xl[q]);
              split_ff(imgd[ii[q] * ISD + 1], yh[q], yl[q]);
            }
          }
          ff acc[5][IPT];
#pragma unroll
          for (int c5 = 0; c5 < 5; ++c5)
#pragma unroll
            for (int q = 0; q < IPT; ++q) acc[c5][q] = ff_zero();
          if (act) {
            if constexpr (MODE == LF_FF)
              accumulate_ext<IPT>(dc, P.nc, dm, P.nm, k0, k1, xh, xl, yh, yl, tab, acc);
            else if (GRAD && C.mbase)   // anchored plans: one plane
              accumulate_anchored<IPT>(dc, P.nc, dm, reinterpret_cast<const MemA*>(smem + P.off_dma), P.nm,
                                       k0, k1, chunk, xh, xl, yh, yl, tab, acc);
            else
              accumulate_mixed<IPT>(dc, P.nc, dm, P.nm, k0, k1, chunk, xh, xl, yh, yl, tab, acc);
          }
          for (int off = 1; off < ks; off <<= 1)
#pragma unroll
            for (int c5 = 0; c5 < 5; ++c5)
#pragma unroll
              for (int q = 0; q < IPT; ++q) {
                ff o;
                o.hi = __shfl_xor_sync(0xffffffffu, acc[c5][q].hi, off);
                o.lo = __shfl_xor_sync(0xffffffffu, acc[c5][q].lo, off);
                acc[c5][q] = ff_add(acc[c5][q], o);
              }
          if (act && k == 0) {
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
              if (q > 0 && ii[q] == ii[q - 1]) break;     // the clamped repeats of the last unit
              if (MODE == LF_MIXED && GRAD && C.mbase && j == 0) {  // the members' base sum
                const float4 b4 = C.mbase[ii[q]];
                acc[0][q] = ff_add(acc[0][q], ff_make(b4.x, b4.y));
                acc[1][q] = ff_add(acc[1][q], ff_make(b4.z, b4.w));
              }
              for (int c5 = 0; c5 < 5; ++c5) {
                imgf[ii[q] * ISF + 2 * c5] = acc[c5][q].hi;
                imgf[ii[q] * ISF + 2 * c5 + 1] = acc[c5][q].lo;
              }
            }
          }
        } else {
          double v[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
          if (act) {
            const int ii[2] = {ia, ib};
            for (int q = 0; q < 2; ++q) {
              const double x = j > 0 ? img[ii[q] * IS + 14] : pos ? pos[4 * ii[q]] : C.theta[2 * ii[q]];
              const double y = j > 0 ? img[ii[q] * IS + 15] : pos ? pos[4 * ii[q] + 1] : C.theta[2 * ii[q] + 1];
              accumulate_fp64(dc, P.nc, dm, P.nm, k0, k1, x, y, v[q]);
            }
          }
          for (int off = 1; off < ks; off <<= 1)
#pragma unroll
            for (int c5 = 0; c5 < 5; ++c5) {
              v[0][c5] += __shfl_xor_sync(0xffffffffu, v[0][c5], off);
              v[1][c5] += __shfl_xor_sync(0xffffffffu, v[1][c5], off);
            }
          if (act && k == 0) {
            for (int c5 = 0; c5 < 5; ++c5) img[ia * IS + c5] = v[0][c5];
            if (ib != ia)
              for (int c5 = 0; c5 < 5; ++c5) img[ib * IS + c5] = v[1][c5];
          }
        }
      }
      __syncthreads();
      if (C.np > 1) {
        // recursion state (FP64): theta_{j+1}, then per plane alpha (2) and Psi_j A_j (4)
        for (int i = tid; i < n_img; i += blockDim.x) {
          double sm[5];
          double* st;
          if constexpr (MIXED) {
            for (int c5 = 0; c5 < 5; ++c5)
              sm[c5] = (double)imgf[i * ISF + 2 * c5] + (double)imgf[i * ISF + 2 * c5 + 1];
            st = imgd + i * ISD;
          } else {
            for (int c5 = 0; c5 < 5; ++c5) sm[c5] = img[i * IS + c5];
            st = img + i * IS + 14;
          }
          double a00 = 1, a01 = 0, a10 = 0, a11 = 1;
          for (int l = 0; l < j; ++l) {
            const double* pl = st + 2 + 6 * l;
            double rr = C.r[l][j];
            a00 -= rr * pl[2]; a01 -= rr * pl[3]; a10 -= rr * pl[4]; a11 -= rr * pl[5];
          }
          if constexpr (GRAD) {       // theta_j and Psi_j for the reverse sweep
            double* rec = reinterpret_cast<double*>(smem + C.off_mpg) + i * C.mpg_stride + 10 * j;
            if (j == 0) { rec[0] = C.theta[2 * i]; rec[1] = C.theta[2 * i + 1]; }
            else { rec[0] = st[0]; rec[1] = st[1]; }
            rec[2] = sm[2]; rec[3] = sm[3]; rec[4] = sm[4];
          }
          double* pj = st + 2 + 6 * j;
          pj[0] = sm[0]; pj[1] = sm[1];
          pj[2] = sm[2] * a00 + sm[4] * a10;
          pj[3] = sm[2] * a01 + sm[4] * a11;
          pj[4] = sm[4] * a00 + sm[3] * a10;
          pj[5] = sm[4] * a01 + sm[3] * a11;
          if (j + 1 < C.np) {
            double tx = pos ? pos[4 * i] : C.theta[2 * i], ty = pos ? pos[4 * i + 1] : C.theta[2 * i + 1];
            for (int l = 0; l <= j; ++l) {
              tx -= C.r[l][j + 1] * st[2 + 6 * l];
              ty -= C.r[l][j + 1] * st[2 + 6 * l + 1];
            }
            st[0] = tx;
            st[1] = ty;
          }
        }
        __syncthreads();
      }
    }
    };
    eval_planes(nullptr);

    double my = 0.0;
    // the mixed tier's source-plane chi^2: the block's sum in float-float (FP32 pipe), with
    // any non-finite family flagged apart
    ff myf = ff_zero();
    bool mybad = false;
    if constexpr (MIXED) {
      // ---- A5, A7 (mixed tiers): beta in float-float, det A in float-float, then
      // mu = A^-1 and M = mu^T S^-1 mu in FP32
      for (int i = tid; i < n_img; i += blockDim.x) {
        float* r = imgf + i * ISF;
        const int f = C.img_fam[i];
        ff bx, by;
        float a00, a01, a10, a11, det;
        ff fA00 = ff_zero(), fA11 = ff_zero(), fA01 = ff_zero();
        double dM[3] = {0.0, 0.0, 0.0};     // several planes: M from the FP64 A (forward chi^2)
        if (C.np == 1) {
          const float2 af = faf[f];
          const ff a = ff_make(af.x, af.y);
          const float4 tf = C.theta_ff[i];
          bx = ff_sub(ff_make(tf.x, tf.y), ff_mul(a, ff_make(r[0], r[1])));
          by = ff_sub(ff_make(tf.z, tf.w), ff_mul(a, ff_make(r[2], r[3])));
          const ff A00 = ff_add_f(ff_neg(ff_mul(a, ff_make(r[4], r[5]))), 1.0f);
          const ff A11 = ff_add_f(ff_neg(ff_mul(a, ff_make(r[6], r[7]))), 1.0f);
          const ff A01 = ff_neg(ff_mul(a, ff_make(r[8], r[9])));
          det = ff_sub(ff_mul(A00, A11), ff_sqr(A01)).hi;
          a00 = A00.hi; a11 = A11.hi; a01 = a10 = A01.hi;
          fA00 = A00; fA11 = A11; fA01 = A01;
        } else {
          const double* st = imgd + i * ISD;
          double dbx = C.theta[2 * i], dby = C.theta[2 * i + 1];
          double A00 = 1, A01 = 0, A10 = 0, A11 = 1;
          for (int l = 0; l < C.np; ++l) {
            const double rs = C.fam_ratio[f * C.np + l];
            const double* pl = st + 2 + 6 * l;
            dbx -= rs * pl[0]; dby -= rs * pl[1];
            A00 -= rs * pl[2]; A01 -= rs * pl[3]; A10 -= rs * pl[4]; A11 -= rs * pl[5];
          }
          bx = ff_from_double(dbx);
          by = ff_from_double(dby);
          det = (float)(A00 * A11 - A01 * A10);
          a00 = (float)A00; a01 = (float)A01; a10 = (float)A10; a11 = (float)A11;
          if constexpr (FFM) {
            // M = mu^T S^-1 mu with mu = A^-1 (A not symmetric), from the FP64 A
            const double id = 1.0 / (A00 * A11 - A01 * A10);
            const double u00 = A11 * id, u01 = -A01 * id, u10 = -A10 * id, u11 = A00 * id;
            const double s0 = C.sinv[3 * i], s1 = C.sinv[3 * i + 1], s2 = C.sinv[3 * i + 2];
            const double X00 = s0 * u00 + s1 * u10, X01 = s0 * u01 + s1 * u11;
            const double X10 = s1 * u00 + s2 * u10, X11 = s1 * u01 + s2 * u11;
            dM[0] = u00 * X00 + u10 * X10;
            dM[1] = u00 * X01 + u10 * X11;
            dM[2] = u01 * X01 + u11 * X11;
          }
        }
        const float id = 1.0f / det;
        const float m00 = a11 * id, m01 = -a01 * id, m10 = -a10 * id, m11 = a00 * id;
        const float4 sv = C.sinv_f[i];
        const float X00 = fmaf(sv.x, m00, sv.y * m10), X01 = fmaf(sv.x, m01, sv.y * m11);
        const float X10 = fmaf(sv.y, m00, sv.z * m10), X11 = fmaf(sv.y, m01, sv.z * m11);
        r[10] = bx.hi; r[11] = bx.lo; r[12] = by.hi; r[13] = by.lo;
        r[14] = fmaf(m00, X00, m10 * X10);
        r[15] = fmaf(m00, X01, m10 * X11);
        r[16] = fmaf(m01, X01, m11 * X11);
        r[17] = m00; r[18] = m01; r[19] = m10; r[20] = m11;
        r[21] = 0.0f;                 // M in FP32 words 14..16
        if constexpr (FFM) {
          // M in float-float words (14..19; the forward pass reads no mu).  Near a critical curve
          // M ~ mu^2 / sigma^2 is nearly of rank one, and its weak direction, which carries the
          // family's chi^2, is lost in FP32 words of M already at moderate magnification
          // (|det A| ~ 0.02): several planes from the FP64 A, one plane as
          // M = adj(A) S^-1 adj(A) / det A^2 from the float-float A
          if (C.np > 1) {
            split_ff(dM[0], r[14], r[15]);
            split_ff(dM[1], r[16], r[17]);
            split_ff(dM[2], r[18], r[19]);
            r[21] = 1.0f;
          } else {
            const ff inv2 = ff_rcp(ff_sqr(ff_sub(ff_mul(fA00, fA11), ff_sqr(fA01))));
            const ff T00 = ff_sub(ff_mul_f(fA11, sv.x), ff_mul_f(fA01, sv.y));
            const ff T10 = ff_sub(ff_mul_f(fA11, sv.y), ff_mul_f(fA01, sv.z));
            const ff T01 = ff_sub(ff_mul_f(fA00, sv.y), ff_mul_f(fA01, sv.x));
            const ff T11 = ff_sub(ff_mul_f(fA00, sv.z), ff_mul_f(fA01, sv.y));
            const ff M00 = ff_mul(ff_sub(ff_mul(fA11, T00), ff_mul(fA01, T10)), inv2);
            const ff M01 = ff_mul(ff_sub(ff_mul(fA11, T01), ff_mul(fA01, T11)), inv2);
            const ff M11 = ff_mul(ff_sub(ff_mul(fA00, T11), ff_mul(fA01, T01)), inv2);
            r[14] = M00.hi; r[15] = M00.lo; r[16] = M01.hi; r[17] = M01.lo; r[18] = M11.hi; r[19] = M11.lo;
            r[21] = 1.0f;
          }
        }
      }
      __syncthreads();
      // ---- A8 (mixed tiers): per family, offsets e_i = beta_i - beta_ref from the family's
      // first image, G = sum M_i, g = sum M_i e_i, the 2x2 solve and chi^2_f, all in
      // float-float on the FP32 pipe (the FP64 pipe is the slow one on this part).  The
      // 48-bit float-float result carries beta_model to the accuracy the adjoint needs (an
      // error in it enters the gradient at first order); it is stored as FP64.
      for (int f = tid; f < C.n_fam; f += blockDim.x) {
        const int i0 = C.fam_off[f], i1 = C.fam_off[f + 1];
        const float* r0 = imgf + i0 * ISF;
        const ff br0 = ff_make(r0[10], r0[11]), br1 = ff_make(r0[12], r0[13]);
        ff G00 = ff_zero(), G01 = ff_zero(), G11 = ff_zero(), g0 = ff_zero(), g1 = ff_zero();
        for (int i = i0; i < i1; ++i) {
          const float* r = imgf + i * ISF;
          const ff e0 = ff_sub(ff_make(r[10], r[11]), br0), e1 = ff_sub(ff_make(r[12], r[13]), br1);
          ff M00, M01, M11;
          image_M(r, M00, M01, M11);
          G00 = ff_add(G00, M00); G01 = ff_add(G01, M01); G11 = ff_add(G11, M11);
          g0 = ff_add(g0, ff_add(ff_mul(e0, M00), ff_mul(e1, M01)));
          g1 = ff_add(g1, ff_add(ff_mul(e0, M01), ff_mul(e1, M11)));
        }
        double cf = 0.0, c0 = 0.0, c1 = 0.0;
        if (i1 - i0 == 1) {
          if (!(isfinite(G00.hi) && isfinite(G01.hi) && isfinite(G11.hi) && isfinite(br0.hi) && isfinite(br1.hi)))
            cf = INFINITY;
        } else {
          const ff dG = ff_sub(ff_mul(G00, G11), ff_sqr(G01));
          const ff cx = ff_div(ff_sub(ff_mul(G11, g0), ff_mul(G01, g1)), dG);
          const ff cy = ff_div(ff_sub(ff_mul(G00, g1), ff_mul(G01, g0)), dG);
          ff acc = ff_zero();
          for (int i = i0; i < i1; ++i) {
            const float* r = imgf + i * ISF;
            const ff d0 = ff_sub(ff_sub(ff_make(r[10], r[11]), br0), cx);
            const ff d1 = ff_sub(ff_sub(ff_make(r[12], r[13]), br1), cy);
            ff M00, M01, M11;
            image_M(r, M00, M01, M11);
            acc = ff_add(acc, ff_add(ff_mul(ff_sqr(d0), M00),
                                     ff_add(ff_mul_f(ff_mul(ff_mul(d0, d1), M01), 2.f), ff_mul(ff_sqr(d1), M11))));
          }
          cf = ff_to_double(acc);
          c0 = ff_to_double(cx);
          c1 = ff_to_double(cy);
          if (!isfinite(cf) || !(dG.hi > 0.f)) cf = INFINITY;
          if constexpr (FFSUM) myf = ff_add(myf, acc);
        }
        fam[3 * f] = cf;
        fam[3 * f + 1] = c0;
        fam[3 * f + 2] = c1;
        if constexpr (FFSUM) mybad = mybad || !isfinite(cf);
        else my += cf;
      }
    } else {
      // ---- A5, A7 (FP64 tier): beta_i, A_i, mu_i, M_i
      for (int i = tid; i < n_img; i += blockDim.x) {
        double* r = img + i * IS;
        const int f = C.img_fam[i];
        const double tx = C.theta[2 * i], ty = C.theta[2 * i + 1];
        double bx, by, A00, A01, A10, A11;
        if (C.np == 1) {
          const double a = fa[f];
          bx = tx - a * r[0];
          by = ty - a * r[1];
          A00 = 1.0 - a * r[2]; A11 = 1.0 - a * r[3]; A01 = A10 = -a * r[4];
        } else {
          bx = tx; by = ty; A00 = 1; A01 = 0; A10 = 0; A11 = 1;
          for (int l = 0; l < C.np; ++l) {
            const double rs = C.fam_ratio[f * C.np + l];
            const double* pl = r + 16 + 6 * l;
            bx -= rs * pl[0]; by -= rs * pl[1];
            A00 -= rs * pl[2]; A01 -= rs * pl[3]; A10 -= rs * pl[4]; A11 -= rs * pl[5];
          }
        }
        const double id = 1.0 / (A00 * A11 - A01 * A10);
        const double m00 = A11 * id, m01 = -A01 * id, m10 = -A10 * id, m11 = A00 * id;
        const double s0 = C.sinv[3 * i], s1 = C.sinv[3 * i + 1], s2 = C.sinv[3 * i + 2];
        const double X00 = s0 * m00 + s1 * m10, X01 = s0 * m01 + s1 * m11;
        const double X10 = s1 * m00 + s2 * m10, X11 = s1 * m01 + s2 * m11;
        r[5] = m00 * X00 + m10 * X10;
        r[6] = m00 * X01 + m10 * X11;
        r[7] = m01 * X01 + m11 * X11;
        r[10] = m00; r[11] = m01; r[12] = m10; r[13] = m11;
        r[8] = bx; r[9] = by;
      }
      __syncthreads();
      // ---- A8 (FP64 tier): analytic source and chi^2 per family
      for (int f = tid; f < C.n_fam; f += blockDim.x) {
        const int i0 = C.fam_off[f], i1 = C.fam_off[f + 1];
        // beta_model = beta_ref + G^-1 sum M_i (beta_i - beta_ref), beta_ref the first image
        const double br0 = img[i0 * IS + 8], br1 = img[i0 * IS + 9];
        double G00 = 0, G01 = 0, G11 = 0, g0 = 0, g1 = 0;
        for (int i = i0; i < i1; ++i) {
          const double* r = img + i * IS;
          const double e0 = r[8] - br0, e1 = r[9] - br1;
          G00 += r[5]; G01 += r[6]; G11 += r[7];
          g0 += r[5] * e0 + r[6] * e1;
          g1 += r[6] * e0 + r[7] * e1;
        }
        double c0 = 0.0, c1 = 0.0, cf = 0.0;
        if (i1 - i0 == 1) {
          if (!(isfinite(G00) && isfinite(G01) && isfinite(G11) && isfinite(br0) && isfinite(br1)))
            cf = INFINITY;
        } else {
          const double dG = G00 * G11 - G01 * G01;
          const double idG = 1.0 / dG;
          c0 = (G11 * g0 - G01 * g1) * idG;
          c1 = (G00 * g1 - G01 * g0) * idG;
          for (int i = i0; i < i1; ++i) {
            const double* r = img + i * IS;
            const double d0 = (r[8] - br0) - c0, d1 = (r[9] - br1) - c1;
            cf += r[5] * d0 * d0 + 2.0 * r[6] * d0 * d1 + r[7] * d1 * d1;
          }
          if (!isfinite(cf) || !(dG > 0.0)) cf = INFINITY;
        }
        fam[3 * f] = cf;
        fam[3 * f + 1] = c0;      // beta_model - beta_ref
        fam[3 * f + 2] = c1;
        my += cf;
      }
    }
    // Per-image state of the flux / time-delay terms (one plane, FP64 from the sums): a_dis,
    // theta, beta, beta_model, A, det A, mu, grad det A (from the third derivatives of psi at
    // aux[LF_AUXI i + 1 ..]), beta_model - beta and A^-1 (beta_model - beta).
    struct AuxImg {
      double a, tx, ty, bx, by, A00, A11, A01, det, mu, gx, gy, db0, db1, dt0, dt1;
    };
    auto aux_image = [&](int i, const double* aux, AuxImg& q) {
      const int f = C.img_fam[i], i0 = C.fam_off[f];
      const double a = fa[f];
      double sm[5], bmx, bmy;
      if constexpr (MIXED) {
        const float* r = imgf + i * ISF;
        const float* r0 = imgf + i0 * ISF;
        for (int k = 0; k < 5; ++k) sm[k] = (double)r[2 * k] + (double)r[2 * k + 1];
        q.bx = ff_to_double(ff_make(r[10], r[11]));
        q.by = ff_to_double(ff_make(r[12], r[13]));
        bmx = ff_to_double(ff_make(r0[10], r0[11])) + fam[3 * f + 1];
        bmy = ff_to_double(ff_make(r0[12], r0[13])) + fam[3 * f + 2];
      } else {
        const double* r = img + i * IS;
        for (int k = 0; k < 5; ++k) sm[k] = r[k];
        q.bx = r[8]; q.by = r[9];
        bmx = img[i0 * IS + 8] + fam[3 * f + 1];
        bmy = img[i0 * IS + 9] + fam[3 * f + 2];
      }
      q.a = a;
      q.tx = C.theta[2 * i]; q.ty = C.theta[2 * i + 1];
      q.A00 = 1.0 - a * sm[2]; q.A11 = 1.0 - a * sm[3]; q.A01 = -a * sm[4];
      q.det = q.A00 * q.A11 - q.A01 * q.A01;
      q.mu = 1.0 / q.det;
      const double* d3 = aux + LF_AUXI * i + 1;
      // grad det A from psi_xxx, psi_xxy, psi_xyy, psi_yyy; grad mu = -mu^2 grad det A
      q.gx = -a * (d3[0] * q.A11 + d3[2] * q.A00) + 2.0 * a * q.A01 * d3[1];
      q.gy = -a * (d3[1] * q.A11 + d3[3] * q.A00) + 2.0 * a * q.A01 * d3[2];
      q.db0 = bmx - q.bx; q.db1 = bmy - q.by;
      q.dt0 = (q.A11 * q.db0 - q.A01 * q.db1) / q.det;
      q.dt1 = (q.A00 * q.db1 - q.A01 * q.db0) / q.det;
    };
    if constexpr (AUX) {
      if (C.aux) {
        // ---- flux and time-delay terms in their source-plane forms (Sec. 3.2-3.3): psi and its
        // third derivatives at every observed image, the linearised magnification
        // mu + [A^-1 (beta_model - beta_i)] . grad mu and arrival time
        // K [(theta - beta_i)^2 / 2 - a psi] + K (beta_model - beta_i) . (beta_i - theta),
        // K = td_scale / a, then per family the nuisances m_src and Delta t_0
        double* aux = reinterpret_cast<double*>(smem + C.off_aux);
        double* auxf = aux + LF_AUXI * n_img;
        __syncthreads();
        const PlaneDesc& P = C.pl[0];
        const CompT<T>* dc = reinterpret_cast<const CompT<T>*>(smem + P.off_dc);
        const Mem* dm = reinterpret_cast<const Mem*>(smem + P.off_dm);
        const int K = P.nc + P.nm;
        const int ntask_img = n_img * KS;
        for (int base = 0; base < ntask_img; base += blockDim.x) {
          const int t = base + tid;
          const bool act = t < ntask_img;
          const int i = act ? t / KS : 0, k = act ? t - i * KS : 0;
          const int k0 = (int)((long long)K * k / KS), k1 = (int)((long long)K * (k + 1) / KS);
          double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
          if (act) {
            T xh, xl, yh, yl;
            if constexpr (MIXED) {
              const float4 tf = C.theta_ff[i];
              xh = tf.x; xl = tf.y; yh = tf.z; yl = tf.w;
            } else {
              xh = C.theta[2 * i]; xl = (T)0; yh = C.theta[2 * i + 1]; yl = (T)0;
            }
            aux_sum<T, Mem>(dc, P.nc, dm, P.nm, k0, k1, xh, xl, yh, yl, v);
          }
          for (int off = 1; off < KS; off <<= 1)
#pragma unroll
            for (int q = 0; q < 5; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
          if (act && k == 0)
            for (int q = 0; q < 5; ++q) aux[LF_AUXI * i + q] = v[q];
        }
        __syncthreads();
        for (int i = tid; i < n_img; i += blockDim.x) {
          AuxImg q;
          aux_image(i, aux, q);
          double y = 0.0, dd = 0.0;
          if (C.aux_wmag[i] > 0.0) {
            const double mu_m = q.mu - q.mu * q.mu * (q.dt0 * q.gx + q.dt1 * q.gy);
            y = C.aux_mag[i] + 2.5 * log10(fabs(mu_m));
          }
          if (C.aux_wtd[i] > 0.0) {
            const double Kf = C.td_scale / q.a;
            const double ex = q.tx - q.bx, ey = q.ty - q.by;
            const double geo = 0.5 * (ex * ex + ey * ey);
            const double Ti = Kf * (geo - q.a * aux[LF_AUXI * i]) - Kf * (q.db0 * ex + q.db1 * ey);
            dd = C.aux_td[i] - Ti;
          }
          aux[LF_AUXI * i + 5] = y;
          aux[LF_AUXI * i + 6] = dd;
        }
        __syncthreads();
        for (int f = tid; f < C.n_fam; f += blockDim.x) {
          const int i0 = C.fam_off[f], i1 = C.fam_off[f + 1];
          double wm = 0.0, ym = 0.0, wt = 0.0, yt = 0.0;
          for (int i = i0; i < i1; ++i) {
            wm += C.aux_wmag[i]; ym += C.aux_wmag[i] * aux[LF_AUXI * i + 5];
            wt += C.aux_wtd[i]; yt += C.aux_wtd[i] * aux[LF_AUXI * i + 6];
          }
          double add = 0.0, m_src = 0.0, t0 = 0.0;
          if (wm > 0.0) {
            m_src = ym / wm;
            for (int i = i0; i < i1; ++i) {
              const double e = aux[LF_AUXI * i + 5] - m_src;
              add += C.aux_wmag[i] * e * e;
            }
          }
          if (wt > 0.0) {
            t0 = yt / wt;
            for (int i = i0; i < i1; ++i) {
              const double e = aux[LF_AUXI * i + 6] - t0;
              add += C.aux_wtd[i] * e * e;
            }
          }
          auxf[LF_AUXF * f] = m_src;
          auxf[LF_AUXF * f + 1] = t0;
          my += isfinite(add) ? add : INFINITY;
        }
      }
    }
    if constexpr (PASS == 1) {
      // ---- image-plane chi^2: Newton steps theta <- theta - A^-1 (beta(theta) - beta_model)
      // from the observed images, then chi^2_img = sum (theta_obs - theta)^T S^-1 (...)
      double* nst = reinterpret_cast<double*>(smem + C.off_newton);   // [4 i]: theta, beta_model
      __syncthreads();
      for (int i = tid; i < n_img; i += blockDim.x) {
        const int f = C.img_fam[i], i0 = C.fam_off[f];
        double bm0, bm1;
        if constexpr (MIXED) {
          const float* r0 = imgf + i0 * ISF;
          bm0 = ff_to_double(ff_make(r0[10], r0[11])) + fam[3 * f + 1];
          bm1 = ff_to_double(ff_make(r0[12], r0[13])) + fam[3 * f + 2];
        } else {
          bm0 = img[i0 * IS + 8] + fam[3 * f + 1];
          bm1 = img[i0 * IS + 9] + fam[3 * f + 2];
        }
        nst[4 * i] = C.theta[2 * i];
        nst[4 * i + 1] = C.theta[2 * i + 1];
        nst[4 * i + 2] = bm0;
        nst[4 * i + 3] = bm1;
      }
      __syncthreads();
      for (int it = 0; it < iters; ++it) {
        eval_planes(nst);
        for (int i = tid; i < n_img; i += blockDim.x) {
          double sm[5];
          if constexpr (MIXED) {
            for (int c5 = 0; c5 < 5; ++c5)
              sm[c5] = (double)imgf[i * ISF + 2 * c5] + (double)imgf[i * ISF + 2 * c5 + 1];
          } else {
            for (int c5 = 0; c5 < 5; ++c5) sm[c5] = img[i * IS + c5];
          }
          const double tx = nst[4 * i], ty = nst[4 * i + 1];
          if (C.np > 1) {
            // beta and the (non-symmetric) A of the recursion to the family's source plane
            const int f = C.img_fam[i];
            const double* st = MIXED ? imgd + i * ISD : img + i * IS + 14;
            double bx = tx, by = ty, A00 = 1, A01 = 0, A10 = 0, A11 = 1;
            for (int l = 0; l < C.np; ++l) {
              const double rs = C.fam_ratio[f * C.np + l];
              const double* pl = st + 2 + 6 * l;
              bx -= rs * pl[0]; by -= rs * pl[1];
              A00 -= rs * pl[2]; A01 -= rs * pl[3]; A10 -= rs * pl[4]; A11 -= rs * pl[5];
            }
            const double rx = bx - nst[4 * i + 2], ry = by - nst[4 * i + 3];
            const double id = 1.0 / (A00 * A11 - A01 * A10);
            nst[4 * i] = tx - (A11 * rx - A01 * ry) * id;
            nst[4 * i + 1] = ty - (A00 * ry - A10 * rx) * id;
            continue;
          }
          const double a = fa[C.img_fam[i]];
          const double rx = tx - a * sm[0] - nst[4 * i + 2];
          const double ry = ty - a * sm[1] - nst[4 * i + 3];
          const double A00 = 1.0 - a * sm[2], A11 = 1.0 - a * sm[3], A01 = -a * sm[4];
          const double id = 1.0 / (A00 * A11 - A01 * A01);
          nst[4 * i] = tx - (A11 * rx - A01 * ry) * id;
          nst[4 * i + 1] = ty - (A00 * ry - A01 * rx) * id;
        }
        __syncthreads();
      }
      double c2 = 0.0, d2 = 0.0;
      for (int i = tid; i < n_img; i += blockDim.x) {
        const double d0 = C.theta[2 * i] - nst[4 * i], d1 = C.theta[2 * i + 1] - nst[4 * i + 1];
        c2 += C.sinv[3 * i] * d0 * d0 + 2.0 * C.sinv[3 * i + 1] * d0 * d1 + C.sinv[3 * i + 2] * d1 * d1;
        d2 += d0 * d0 + d1 * d1;
      }
      const double tc = block_sum(c2, scratch);
      const double td = block_sum(d2, scratch);
      if (tid == 0) {
        chi2[s] = isfinite(tc) ? tc : INFINITY;
        if (rms) rms[s] = sqrt(td / n_img);
      }
      __syncthreads();
      continue;
    }
    double total;
    if constexpr (FFSUM) {
      const bool bad = __syncthreads_or(mybad ? 1 : 0) != 0;
      const ff t = block_sum_ff(myf, reinterpret_cast<ff*>(scratch));
      total = bad ? INFINITY : ff_to_double(t);
    } else {
      total = block_sum(my, scratch);
    }
    if (tid == 0) chi2[s] = total;

    if constexpr (GRAD) {
      double* mpg = reinterpret_cast<double*>(smem + C.off_mpg);
      const int MPS = C.mpg_stride;
      if (C.np > 1) {
        // third derivatives of psi at theta_j of every plane after the first (the positions
        // theta_j depend on the parameters through the earlier planes' deflections)
        for (int j = 1; j < C.np; ++j) {
          const PlaneDesc& P = C.pl[j];
          const CompT<T>* dc = reinterpret_cast<const CompT<T>*>(smem + P.off_dc);
          const Mem* dm = reinterpret_cast<const Mem*>(smem + P.off_dm);
          const int K = P.nc + P.nm, nt = n_img * KS;
          for (int base = 0; base < nt; base += blockDim.x) {
            const int t = base + tid;
            const bool act = t < nt;
            const int i = act ? t / KS : 0, k = act ? t - i * KS : 0;
            const int k0 = (int)((long long)K * k / KS), k1 = (int)((long long)K * (k + 1) / KS);
            double d3[4] = {0, 0, 0, 0};
            if (act) {
              const double* rec = mpg + i * MPS + 10 * j;
              T xh, xl, yh, yl;
              if constexpr (MIXED) { split_ff(rec[0], xh, xl); split_ff(rec[1], yh, yl); }
              else { xh = rec[0]; xl = 0.0; yh = rec[1]; yl = 0.0; }
              d3_sum(dc, P.nc, dm, P.nm, k0, k1, xh, xl, yh, yl, d3);
            }
            for (int off = 1; off < KS; off <<= 1)
#pragma unroll
              for (int q = 0; q < 4; ++q) d3[q] += __shfl_xor_sync(0xffffffffu, d3[q], off);
            if (act && k == 0)
              for (int q = 0; q < 4; ++q) mpg[i * MPS + 10 * C.np + 4 * (j - 1) + q] = d3[q];
          }
        }
        __syncthreads();
      }
      // Adjoint of the flux / time-delay terms (one plane, FP64 from the sums).  With
      // y_i = m_i + 2.5 log10|mu_model,i| and d_i = dt_i - T_model,i, the family nuisances are
      // the weighted means, so y_bar = 2 w_m (y - m_src) and T_bar = -2 w_t (d - Delta t_0).
      // Reverse sweep of mu_model = mu - mu^2 dtheta . grad det A, dtheta = A^-1 (beta_model -
      // beta), T_model above: cotangents of psi, of its third derivatives, of beta_i, of A_i, and
      // of beta_model, summed per family into lambda = G^-1 beta_model_bar (beta_model =
      // G^-1 sum_j M_j beta_j, G = sum_j M_j).
      double* auxg = reinterpret_cast<double*>(smem + C.off_auxg);
      double* auxp = reinterpret_cast<double*>(smem + C.off_aux);
      double* auxf = auxp + LF_AUXI * n_img;
      if (AUX && C.np == 1 && C.aux) {
        constexpr double LOG10E_25 = 2.5 * 0.43429448190325182765;   // 2.5 / ln 10
        for (int i = tid; i < n_img; i += blockDim.x) {
          const int f = C.img_fam[i];
          AuxImg q;
          aux_image(i, auxp, q);
          const double* d3 = auxp + LF_AUXI * i + 1;
          const double a = q.a;
          const double ex = q.bx - q.tx, ey = q.by - q.ty;       // beta - theta
          const double h = q.dt0 * q.gx + q.dt1 * q.gy;
          const double mu_m = q.mu - q.mu * q.mu * h;
          const double ybar = C.aux_wmag[i] > 0.0 ? 2.0 * C.aux_wmag[i] * (auxp[LF_AUXI * i + 5] - auxf[LF_AUXF * f]) : 0.0;
          const double tbar = C.aux_wtd[i] > 0.0 ? -2.0 * C.aux_wtd[i] * (auxp[LF_AUXI * i + 6] - auxf[LF_AUXF * f + 1]) : 0.0;
          const double mbar = ybar != 0.0 ? ybar * LOG10E_25 / mu_m : 0.0;
          const double mubar = mbar * (1.0 - 2.0 * q.mu * h);
          const double k = -mbar * q.mu * q.mu;
          const double thb0 = k * q.gx, thb1 = k * q.gy;        // dtheta_bar
          const double hb0 = k * q.dt0, hb1 = k * q.dt1;        // (grad det A)_bar
          double* g = auxg + LF_AUXG * i;
          // grad det A = -a (T0 A11 + T2 A00) + 2 a A01 T1, -a (T1 A11 + T3 A00) + 2 a A01 T2
          double A00b = -a * (hb0 * d3[2] + hb1 * d3[3]);
          double A11b = -a * (hb0 * d3[0] + hb1 * d3[1]);
          double A01b = 2.0 * a * (hb0 * d3[1] + hb1 * d3[2]);
          g[1] = -a * q.A11 * hb0;
          g[2] = 2.0 * a * q.A01 * hb0 - a * q.A11 * hb1;
          g[3] = -a * q.A00 * hb0 + 2.0 * a * q.A01 * hb1;
          g[4] = -a * q.A00 * hb1;
          // mu = 1 / det A
          const double detb = -q.mu * q.mu * mubar;
          A00b += detb * q.A11; A11b += detb * q.A00; A01b -= 2.0 * q.A01 * detb;
          // dtheta = A^-1 db: db_bar = A^-1 dtheta_bar, A_bar -= (A^-1 dtheta_bar) dtheta^T
          const double u00 = q.A11 * q.mu, u11 = q.A00 * q.mu, u01 = -q.A01 * q.mu;
          const double l0 = u00 * thb0 + u01 * thb1, l1 = u01 * thb0 + u11 * thb1;
          A00b -= l0 * q.dt0; A11b -= l1 * q.dt1; A01b -= l0 * q.dt1 + l1 * q.dt0;
          // T_model = K [(theta - beta)^2 / 2 - a psi] + K db . (beta - theta), K = td_scale / a
          const double K = C.td_scale / a;
          const double dbb0 = l0 + tbar * K * ex, dbb1 = l1 + tbar * K * ey;
          g[0] = -tbar * K * a;
          g[5] = tbar * K * (ex + q.db0) - dbb0;                // beta_bar (db = beta_model - beta)
          g[6] = tbar * K * (ey + q.db1) - dbb1;
          g[7] = A00b; g[8] = A11b; g[9] = A01b;
          g[10] = dbb0; g[11] = dbb1;
          // M = A^-T S^-1 A^-1 in FP64
          const double s0 = C.sinv[3 * i], s1 = C.sinv[3 * i + 1], s2 = C.sinv[3 * i + 2];
          const double X00 = s0 * u00 + s1 * u01, X01 = s0 * u01 + s1 * u11;
          const double X10 = s1 * u00 + s2 * u01, X11 = s1 * u01 + s2 * u11;
          g[12] = u00 * X00 + u01 * X10;
          g[13] = u00 * X01 + u01 * X11;
          g[14] = u01 * X01 + u11 * X11;
          g[15] = 0.0;
        }
        __syncthreads();
        for (int f = tid; f < C.n_fam; f += blockDim.x) {
          const int i0 = C.fam_off[f], i1 = C.fam_off[f + 1];
          double b0 = 0.0, b1 = 0.0, G00 = 0.0, G01 = 0.0, G11 = 0.0;
          for (int i = i0; i < i1; ++i) {
            const double* g = auxg + LF_AUXG * i;
            b0 += g[10]; b1 += g[11];
            G00 += g[12]; G01 += g[13]; G11 += g[14];
          }
          if (i1 - i0 > 1) {      // lambda = G^-1 beta_model_bar; one image: beta_model = beta
            const double idG = 1.0 / (G00 * G11 - G01 * G01);
            auxf[LF_AUXF * f + 2] = (G11 * b0 - G01 * b1) * idG;
            auxf[LF_AUXF * f + 3] = (G00 * b1 - G01 * b0) * idG;
          } else {
            auxf[LF_AUXF * f + 2] = b0;
            auxf[LF_AUXF * f + 3] = b1;
          }
        }
        __syncthreads();
      }
      // cotangents of alpha and Psi at each image: with d = beta_i - beta_model, w = M d,
      // z = mu d: beta_bar = 2 w, A_bar = -2 w z^T; one plane: alpha_bar = -2 a w,
      // Psi_bar = 2 a sym(w z^T)
      for (int i = tid; i < n_img; i += blockDim.x) {
        const int f = C.img_fam[i];
        const int n_f = C.fam_off[f + 1] - C.fam_off[f];
        const int i0 = C.fam_off[f];
        double d0, d1, M00, M01, M11, u00, u01, u10, u11;
        if constexpr (MIXED) {
          const float* r = imgf + i * ISF;
          const float* r0 = imgf + i0 * ISF;
          d0 = ff_to_double(ff_sub(ff_make(r[10], r[11]), ff_make(r0[10], r0[11]))) - fam[3 * f + 1];
          d1 = ff_to_double(ff_sub(ff_make(r[12], r[13]), ff_make(r0[12], r0[13]))) - fam[3 * f + 2];
          ff m00, m01, m11;
          image_M(r, m00, m01, m11);
          M00 = ff_to_double(m00); M01 = ff_to_double(m01); M11 = ff_to_double(m11);
          // mu = A^-1 again in FP64 (words 17..20 hold M's low words): one plane from the
          // float-float psi sums, several from the recursion's FP64 A
          double A00 = 1.0, A01 = 0.0, A10 = 0.0, A11 = 1.0;
          if (C.np == 1) {
            const double a = fa[f];
            A00 -= a * ((double)r[4] + (double)r[5]);
            A11 -= a * ((double)r[6] + (double)r[7]);
            A01 = A10 = -a * ((double)r[8] + (double)r[9]);
          } else {
            const double* st = imgd + i * ISD;
            for (int l = 0; l < C.np; ++l) {
              const double rs = C.fam_ratio[f * C.np + l];
              const double* pl = st + 2 + 6 * l;
              A00 -= rs * pl[2]; A01 -= rs * pl[3]; A10 -= rs * pl[4]; A11 -= rs * pl[5];
            }
          }
          const double id = 1.0 / (A00 * A11 - A01 * A10);
          u00 = A11 * id; u01 = -A01 * id; u10 = -A10 * id; u11 = A00 * id;
        } else {
          const double* r = img + i * IS;
          d0 = (r[8] - img[i0 * IS + 8]) - fam[3 * f + 1];
          d1 = (r[9] - img[i0 * IS + 9]) - fam[3 * f + 2];
          M00 = r[5]; M01 = r[6]; M11 = r[7];
          u00 = r[10]; u01 = r[11]; u10 = r[12]; u11 = r[13];
        }
        const double w0 = M00 * d0 + M01 * d1, w1 = M01 * d0 + M11 * d1;
        const double z0 = u00 * d0 + u01 * d1, z1 = u10 * d0 + u11 * d1;
        if (C.np > 1) {
          // reverse sweep of the recursion theta_{j} = theta - sum_{l<j} r_lj alpha_l,
          // A_j = I - sum_{l<j} r_lj Psi_l A_l, beta = theta - sum_l r_ls alpha_l,
          // A = I - sum_l r_ls Psi_l A_l, with P_l = Psi_l A_l:
          //   P_bar -> Psi_bar_j = P_bar A_j^T, A_bar_j = Psi_j P_bar;
          //   theta_bar_j = Psi_j alpha_bar_j + Psi_bar_j : d Psi / d theta (at theta_j)
          double* rec = mpg + i * MPS;
          const double* stp = MIXED ? imgd + i * ISD + 2 : img + i * IS + 16;   // alpha_l, P_l
          const double k2 = n_f > 1 ? 2.0 : 0.0;
          double ab[LF_MAX_PLANES][2], pb[LF_MAX_PLANES][4];
          for (int l = 0; l < C.np; ++l) {
            const double rs = k2 * C.fam_ratio[f * C.np + l];
            ab[l][0] = -rs * w0; ab[l][1] = -rs * w1;
            pb[l][0] = rs * w0 * z0; pb[l][1] = rs * w0 * z1; pb[l][2] = rs * w1 * z0; pb[l][3] = rs * w1 * z1;
          }
          for (int j = C.np - 1; j >= 0; --j) {
            double a00 = 1, a01 = 0, a10 = 0, a11 = 1;
            for (int l = 0; l < j; ++l) {
              const double rr = C.r[l][j];
              const double* pl = stp + 6 * l;
              a00 -= rr * pl[2]; a01 -= rr * pl[3]; a10 -= rr * pl[4]; a11 -= rr * pl[5];
            }
            double* rj = rec + 10 * j;
            const double pxx = rj[2], pyy = rj[3], pxy = rj[4];
            const double* b = pb[j];
            const double G00 = b[0] * a00 + b[1] * a01, G01 = b[0] * a10 + b[1] * a11;
            const double G10 = b[2] * a00 + b[3] * a01, G11 = b[2] * a10 + b[3] * a11;
            const double Gs = G01 + G10;
            rj[5] = ab[j][0]; rj[6] = ab[j][1]; rj[7] = G00; rj[8] = G11; rj[9] = Gs;
            if (j == 0) break;
            const double* d3 = rec + 10 * C.np + 4 * (j - 1);   // xxx, xxy, xyy, yyy
            const double tbx = pxx * ab[j][0] + pxy * ab[j][1] + G00 * d3[0] + Gs * d3[1] + G11 * d3[2];
            const double tby = pxy * ab[j][0] + pyy * ab[j][1] + G00 * d3[1] + Gs * d3[2] + G11 * d3[3];
            const double A00 = pxx * b[0] + pxy * b[2], A01 = pxx * b[1] + pxy * b[3];
            const double A10 = pxy * b[0] + pyy * b[2], A11 = pxy * b[1] + pyy * b[3];
            for (int l = 0; l < j; ++l) {
              const double rr = C.r[l][j];
              ab[l][0] -= rr * tbx; ab[l][1] -= rr * tby;
              pb[l][0] -= rr * A00; pb[l][1] -= rr * A01; pb[l][2] -= rr * A10; pb[l][3] -= rr * A11;
            }
          }
          continue;
        }
        const double a = fa[f];
        const double k2a = n_f > 1 ? 2.0 * a : 0.0;
        double cot[5] = {-k2a * w0, -k2a * w1, k2a * w0 * z0, k2a * w1 * z1, k2a * (w0 * z1 + w1 * z0)};
        if (AUX && C.aux) {
          // flux / time delay: beta_j_bar += M_j lambda and, through M_j = A_j^-T S^-1 A_j^-1,
          // A_j_bar -= (M_j e_j)(A_j^-1 lambda)^T + (M_j lambda)(A_j^-1 e_j)^T, e_j = beta_j -
          // beta_model; then alpha_bar = -a beta_bar, Psi_bar = -a A_bar
          AuxImg q;
          aux_image(i, auxp, q);
          const double* g = auxg + LF_AUXG * i;
          const double l0 = auxf[LF_AUXF * f + 2], l1 = auxf[LF_AUXF * f + 3];
          double bb0 = g[5], bb1 = g[6], A00b = g[7], A11b = g[8], A01b = g[9];
          if (n_f == 1) {
            bb0 += l0; bb1 += l1;
          } else {
            const double M00_ = g[12], M01_ = g[13], M11_ = g[14];
            const double u00 = q.A11 * q.mu, u11 = q.A00 * q.mu, u01 = -q.A01 * q.mu;
            const double e0 = -q.db0, e1 = -q.db1;
            const double Ml0 = M00_ * l0 + M01_ * l1, Ml1 = M01_ * l0 + M11_ * l1;
            const double Me0 = M00_ * e0 + M01_ * e1, Me1 = M01_ * e0 + M11_ * e1;
            const double ul0 = u00 * l0 + u01 * l1, ul1 = u01 * l0 + u11 * l1;
            const double ue0 = u00 * e0 + u01 * e1, ue1 = u01 * e0 + u11 * e1;
            bb0 += Ml0; bb1 += Ml1;
            A00b -= Me0 * ul0 + Ml0 * ue0;
            A11b -= Me1 * ul1 + Ml1 * ue1;
            A01b -= Me0 * ul1 + Me1 * ul0 + Ml0 * ue1 + Ml1 * ue0;
          }
          cot[0] -= a * bb0; cot[1] -= a * bb1;
          cot[2] -= a * A00b; cot[3] -= a * A11b; cot[4] -= a * A01b;
        }
        if (fap[f] >= 0 && n_f > 1) {
          // a sampled a_dis: beta = theta - a alpha and A = I - a Psi give
          // d chi^2 / d a = (1/a) sum_i (alpha_bar . alpha_i + Psi_bar : Psi_i)
          double sm[5];
          if constexpr (MIXED) {
            const float* r = imgf + i * ISF;
            for (int q = 0; q < 5; ++q) sm[q] = (double)r[2 * q] + (double)r[2 * q + 1];
          } else {
            const double* r = img + i * IS;
            for (int q = 0; q < 5; ++q) sm[q] = r[q];
          }
          double g = 0.0;
          for (int q = 0; q < 5; ++q) g += cot[q] * sm[q];
          atomicAdd(&gacc[fap[f]], g / a);
        }
        if constexpr (MIXED) {
          float* r = imgf + i * ISF;
          for (int q = 0; q < 5; ++q) r[q] = (float)cot[q];
        } else {
          double* r = img + i * IS;
          for (int q = 0; q < 5; ++q) r[q] = cot[q];
        }
      }
      __syncthreads();
      // contraction with each plane's components at theta_j
      for (int j = 0; j < C.np; ++j) {
      const PlaneDesc& P = C.pl[j];
      const Mem* dm = reinterpret_cast<const Mem*>(smem + P.off_dm);
      const int K = P.nc + P.nm;
      const bool mem_grad = (C.scal_plane == j) && C.scal_free;
      lf_scaling ssc = P.sc;
      if (mem_grad) sample_scaling(C, th, ssc);
      const T inv_cut_star = (T)(1.0 / ssc.cut_star);
      const int ntask_img = n_img * KS;   // one image per task in the adjoint pass
      // Every lane of a warp runs each round (inactive ones with zero terms), so that each
      // parameter's terms are summed over the warp by shuffles and added to the block's
      // accumulator by one lane: one shared-memory atomic per warp, not one per lane.
      if constexpr (!AUX) {
        // The sampled explicit components: one task per (component, image), the images padded
        // to whole warps so that a warp's lanes share the component and its terms are summed
        // by shuffles (a cluster with few images still fills the block).
        const int n_imgp = (n_img + 31) & ~31;
        const int ntask_e = C.n_free * n_imgp;
        for (int base = 0; base < ntask_e; base += blockDim.x) {
          const int t = base + tid;
          const int f = min(t / n_imgp, C.n_free - 1);
          const int i = t - (t / n_imgp) * n_imgp;
          const lf_comp& rc = fraw[f];
          if (t >= ntask_e || C.free_plane[f] != j || rc.kind < 1 || rc.kind > 6) continue;   // whole warps
          T g[7] = {(T)0, (T)0, (T)0, (T)0, (T)0, (T)0, (T)0};
          if (i < n_img) {
            T cot[5];
            double px, py;
            if (C.np > 1) {
              const double* rj = mpg + i * MPS + 10 * j;
              for (int q = 0; q < 5; ++q) cot[q] = (T)rj[5 + q];
              px = rj[0]; py = rj[1];
            } else {
              if constexpr (MIXED) {
                for (int q = 0; q < 5; ++q) cot[q] = imgf[i * ISF + q];
              } else {
                for (int q = 0; q < 5; ++q) cot[q] = img[i * IS + q];
              }
              px = C.theta[2 * i]; py = C.theta[2 * i + 1];
            }
            Out5<Dual<T, 6>> o;
            comp_dual<T>(rc, px, py, o);
            // field order x, y, b, eps, pa, core, cut; tangent slots x0 y1 eps2 pa3 core4 cut5
            const int slot[7] = {0, 1, -1, 2, 3, 4, 5};
            const T b = (T)rc.b;
            for (int q = 0; q < 7; ++q) g[q] = q == LF_F_B ? contract(o, cot, -1) : b * contract(o, cot, slot[q]);
          }
          for (int q = 0; q < 7; ++q) {
            const int p = C.free_p[f][q];
            if (p < 0) continue;
            const double gw = warp_sum((double)g[q]);
            if ((tid & 31) == 0) atomicAdd(&gacc[p], gw * xform_deriv(C.p_xform[p], th[p], P.apk));
          }
        }
      }
      if constexpr (!AUX) {
        if (mem_grad) {
          // The members: one task per (image pair, component slice), two independent chains
          // per lane and one shared-memory read of each member record for both images.  Each
          // member's (alpha, Psi) per unit strength is kbar (dx, dy) and Psi_ij = kbar delta_ij +
          // t x_i x_j; its derivative in a parameter contracts with the cotangents as
          // kbar' U + t' V, with U and V below.  Closed forms, P = 1/(S + s), Q = 1/(R + a):
          // dkbar/ds = -P/S, dkbar/da = Q/R, dt/ds = (P^2/S^2)(2 + s/S), dt/da =
          // -(Q^2/R^2)(2 + a/R); kbar = P - Q is taken in its cancellation-free form.
          const int ntask_m = ((n_img + 1) / 2) * KS;
          for (int base = 0; base < ntask_m; base += blockDim.x) {
            const int t = base + tid;
            const bool act = t < ntask_m;
            const int pr = act ? t / KS : 0, k = act ? t - pr * KS : 0;
            const int k0 = act ? (int)((long long)K * k / KS) : 0;
            const int k1 = act ? (int)((long long)K * (k + 1) / KS) : 0;
            const int m0 = act ? max(k0, P.nc) - P.nc : 0, m1 = act ? min(k1, K) - P.nc : 0;
            T cot[2][5], qxh[2], qxl[2], qyh[2], qyl[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int i = min(2 * pr + h, n_img - 1);
              double px, py;
              if (C.np > 1) {
                const double* rj = mpg + i * MPS + 10 * j;
                for (int q = 0; q < 5; ++q) cot[h][q] = (T)rj[5 + q];
                px = rj[0]; py = rj[1];
              } else {
                if constexpr (MIXED) {
                  for (int q = 0; q < 5; ++q) cot[h][q] = imgf[i * ISF + q];
                } else {
                  for (int q = 0; q < 5; ++q) cot[h][q] = img[i * IS + q];
                }
                px = C.theta[2 * i]; py = C.theta[2 * i + 1];
              }
              if (2 * pr + h >= n_img)      // the odd image count's empty slot
                for (int q = 0; q < 5; ++q) cot[h][q] = (T)0;
              if constexpr (MIXED) {
                float a_, b_, c_, d_;
                split_ff(px, a_, b_);
                split_ff(py, c_, d_);
                qxh[h] = a_; qxl[h] = b_; qyh[h] = c_; qyl[h] = d_;
              } else {
                qxh[h] = (T)px; qxl[h] = (T)0; qyh[h] = (T)py; qyl[h] = (T)0;
              }
            }
            T gs[6] = {0, 0, 0, 0, 0, 0};
            // FP32 tiers: the two images are the two lanes of packed f32x2 instructions (the
            // MUFU results are consumed by scalar operations, as in member_pair_acc)
            float2 px2, pxl2, py2, pyl2, c0, c1, c23, c2, c3, c4;
            if constexpr (MIXED) {
              px2 = make_float2(qxh[0], qxh[1]); pxl2 = make_float2(qxl[0], qxl[1]);
              py2 = make_float2(qyh[0], qyh[1]); pyl2 = make_float2(qyl[0], qyl[1]);
              c0 = make_float2(cot[0][0], cot[1][0]); c1 = make_float2(cot[0][1], cot[1][1]);
              c2 = make_float2(cot[0][2], cot[1][2]); c3 = make_float2(cot[0][3], cot[1][3]);
              c4 = make_float2(cot[0][4], cot[1][4]);
              c23 = add2(c2, c3);
            }
            for (int m = m0; m < m1; ++m) {
              const Mem& M = dm[m];
              const T Ms = mem_s(M), Ma = mem_a(M);
              T Gb = (T)0, Gs = (T)0, Ga = (T)0;
              if constexpr (MIXED) {
                const float2 dx = add2(add2(px2, make_float2(-M.xh, -M.xh)), add2(pxl2, make_float2(-M.xl, -M.xl)));
                const float2 dy = add2(add2(py2, make_float2(-M.yh, -M.yh)), add2(pyl2, make_float2(-M.yl, -M.yl)));
                const float2 Ms2 = make_float2(Ms, Ms), Ma2 = make_float2(Ma, Ma);
                const float2 dxx = mul2(dx, dx), dyy = mul2(dy, dy), r2 = add2(dxx, dyy);
                const float2 S2 = fma2(Ms2, Ms2, r2), R2 = fma2(Ma2, Ma2, r2);
                float2 iS, iR, S, R, Pq, Qq, iRS, w, pq, nP2iS, Q2iR, gsU, gsV, gaU, gaV;
                iS.x = rsqrtf(S2.x); iS.y = rsqrtf(S2.y);
                iR.x = rsqrtf(R2.x); iR.y = rsqrtf(R2.y);
                S.x = S2.x * iS.x; S.y = S2.y * iS.y;
                R.x = R2.x * iR.x; R.y = R2.y * iR.y;
                const float2 Ss = add2(S, Ms2), Ra = add2(R, Ma2), RS = add2(R, S);
                Pq.x = __fdividef(1.f, Ss.x); Pq.y = __fdividef(1.f, Ss.y);
                Qq.x = __fdividef(1.f, Ra.x); Qq.y = __fdividef(1.f, Ra.y);
                iRS.x = __fdividef(1.f, RS.x); iRS.y = __fdividef(1.f, RS.y);
                const float amp = Ma + Ms, ams = Ma - Ms;
                w.x = fmaf(amp, iRS.x, 1.f); w.y = fmaf(amp, iRS.y, 1.f);
                pq.x = Pq.x * Qq.x; pq.y = Pq.y * Qq.y;
                nP2iS.x = -(Pq.x * Pq.x) * iS.x; nP2iS.y = -(Pq.y * Pq.y) * iS.y;
                Q2iR.x = Qq.x * Qq.x * iR.x; Q2iR.y = Qq.y * Qq.y * iR.y;
                gsU.x = -Pq.x * iS.x; gsU.y = -Pq.y * iS.y;
                gsV.x = -nP2iS.x * iS.x * fmaf(Ms, iS.x, 2.f); gsV.y = -nP2iS.y * iS.y * fmaf(Ms, iS.y, 2.f);
                gaU.x = Qq.x * iR.x; gaU.y = Qq.y * iR.y;
                gaV.x = -Q2iR.x * iR.x * fmaf(Ma, iR.x, 2.f); gaV.y = -Q2iR.y * iR.y * fmaf(Ma, iR.y, 2.f);
                const float2 kb = mul2(mul2(make_float2(ams, ams), pq), w);
                const float2 U = fma2(c0, dx, fma2(c1, dy, c23));
                const float2 V = fma2(c2, dxx, fma2(c3, dyy, mul2(c4, mul2(dx, dy))));
                const float2 gb = fma2(kb, U, mul2(add2(Q2iR, nP2iS), V));
                const float2 gss = fma2(gsU, U, mul2(gsV, V));
                const float2 gaa = fma2(gaU, U, mul2(gaV, V));
                Gb = gb.x + gb.y;
                Gs = gss.x + gss.y;
                Ga = gaa.x + gaa.y;
              } else {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                T dx, dy;
                if constexpr (MIXED) {
                  dx = offset_of(qxh[h], qxl[h], M.xh, M.xl);
                  dy = offset_of(qyh[h], qyl[h], M.yh, M.yl);
                } else {
                  dx = qxh[h] - M.xh;
                  dy = qyh[h] - M.yh;
                }
                const T* c = cot[h];
                const T dxx = dx * dx, dyy = dy * dy, r2 = dxx + dyy;
                const T iS = ::lf_rsqrt(::lf_fma(Ms, Ms, r2)), iR = ::lf_rsqrt(::lf_fma(Ma, Ma, r2));
                const T S = ::lf_fma(Ms, Ms, r2) * iS, R = ::lf_fma(Ma, Ma, r2) * iR;
                const T Pq = ::lf_rcp(S + Ms), Qq = ::lf_rcp(R + Ma);
                const T kb = (Ma - Ms) * Pq * Qq * ::lf_fma(Ma + Ms, ::lf_rcp(R + S), (T)1);
                const T P2iS = Pq * Pq * iS, Q2iR = Qq * Qq * iR;
                const T U = ::lf_fma(c[0], dx, ::lf_fma(c[1], dy, c[2] + c[3]));
                const T V = ::lf_fma(c[2], dxx, ::lf_fma(c[3], dyy, c[4] * dx * dy));
                Gb += ::lf_fma(kb, U, (Q2iR - P2iS) * V);
                Gs += ::lf_fma(-Pq * iS, U, P2iS * iS * ::lf_fma(Ms, iS, (T)2) * V);
                Ga += ::lf_fma(Qq * iR, U, -Q2iR * iR * ::lf_fma(Ma, iR, (T)2) * V);
              }
              }
              Gs *= M.b;
              Ga *= M.b;
              const T fa = Ma * inv_cut_star;
              gs[LF_S_BSTAR] += Gb * M.fb;
              gs[LF_S_LAM] += Gb * M.b * (T)2 * M.loglr;
              gs[LF_S_CORESTAR] += Gs * M.fs;
              gs[LF_S_BETA] += Gs * Ms * M.loglr;
              gs[LF_S_CUTSTAR] += Ga * fa;
              gs[LF_S_ALPHA] += Ga * Ma * M.loglr;
            }
            for (int q = 0; q < 6; ++q) {
              const int p = C.scal_p[q];
              if (p < 0) continue;
              const double gw = warp_sum((double)gs[q]);
              if ((tid & 31) == 0) atomicAdd(&gacc[p], gw * xform_deriv(C.p_xform[p], th[p], P.apk));
            }
          }
        }
      } else
      for (int base = 0; base < ntask_img; base += blockDim.x) {
        const int t = base + tid;
        const bool act = t < ntask_img;
        const int i = act ? t / KS : 0, k = act ? t - i * KS : 0;
        const int k0 = act ? (int)((long long)K * k / KS) : 0;
        const int k1 = act ? (int)((long long)K * (k + 1) / KS) : 0;
        const bool lead = (tid & 31) == 0;
        T cot[5];
        T pb = (T)0, tb[4] = {(T)0, (T)0, (T)0, (T)0};   // flux / time delay: psi_bar, T_bar
        double px, py;
        if (AUX && C.np == 1 && C.aux) {
          const double* g = auxg + LF_AUXG * i;
          pb = (T)g[0];
          for (int q = 0; q < 4; ++q) tb[q] = (T)g[1 + q];
        }
        if (C.np > 1) {
          const double* rj = mpg + i * MPS + 10 * j;
          for (int q = 0; q < 5; ++q) cot[q] = (T)rj[5 + q];
          px = rj[0]; py = rj[1];
        } else {
          if constexpr (MIXED) {
            for (int q = 0; q < 5; ++q) cot[q] = imgf[i * ISF + q];
          } else {
            for (int q = 0; q < 5; ++q) cot[q] = img[i * IS + q];
          }
          px = C.theta[2 * i]; py = C.theta[2 * i + 1];
        }
        if constexpr (AUX)
        for (int f = 0; f < C.n_free; ++f) {
          const int kc = C.free_comp[f];
          if (C.free_plane[f] != j) continue;
          const lf_comp& rc = fraw[f];
          if (rc.kind < 1 || rc.kind > 6) continue;
          const bool mine = kc >= k0 && kc < k1;      // false for inactive lanes (k0 = k1)
          // field order x, y, b, eps, pa, core, cut; tangent slots x0 y1 eps2 pa3 core4 cut5
          const int slot[7] = {0, 1, -1, 2, 3, 4, 5};
          T g[7] = {0, 0, 0, 0, 0, 0, 0};
          if (AUX && mine && C.aux) {
            // with the flux / time-delay terms: also psi (its field derivatives) and the third
            // derivatives of psi (dual numbers over the offset inside those over the fields)
            typedef Dual<T, 2> S2;
            const T ox = (T)(px - rc.x), oy = (T)(py - rc.y);
            Out5<Dual<S2, 6>> o;
            comp_dual_g<T, S2>(rc, S2::var(ox, 0), S2::var(oy, 1), o);
            const Dual<T, 6> ps = comp_potential_dual<T>(rc, ox, oy);
            const T b = (T)rc.b;
            for (int fld = 0; fld < 7; ++fld) {
              if (C.free_p[f][fld] < 0) continue;
              const int sl = slot[fld];
              const S2 ax = sl < 0 ? o.ax.v : o.ax.d[sl], ay = sl < 0 ? o.ay.v : o.ay.d[sl];
              const S2 xx = sl < 0 ? o.pxx.v : o.pxx.d[sl], yy = sl < 0 ? o.pyy.v : o.pyy.d[sl];
              const S2 xy = sl < 0 ? o.pxy.v : o.pxy.d[sl];
              T v = cot[0] * ax.v + cot[1] * ay.v + cot[2] * xx.v + cot[3] * yy.v + cot[4] * xy.v;
              v += pb * (sl < 0 ? ps.v : ps.d[sl]);
              v += tb[0] * xx.d[0] + tb[1] * xx.d[1] + tb[2] * yy.d[0] + tb[3] * yy.d[1];
              g[fld] = sl < 0 ? v : b * v;
            }
          } else if (mine) {
            Out5<Dual<T, 6>> o;
            comp_dual<T>(rc, px, py, o);
            const T b = (T)rc.b;
            for (int fld = 0; fld < 7; ++fld)
              if (C.free_p[f][fld] >= 0)
                g[fld] = (fld == LF_F_B) ? contract(o, cot, -1) : b * contract(o, cot, slot[fld]);
          }
          for (int fld = 0; fld < 7; ++fld) {
            const int p = C.free_p[f][fld];
            if (p < 0) continue;
            const double gw = warp_sum((double)g[fld]);
            if (lead) atomicAdd(&gacc[p], gw * xform_deriv(C.p_xform[p], th[p], P.apk));
          }
        }
        if (mem_grad) {
          const int m0 = act ? max(k0, P.nc) - P.nc : 0, m1 = act ? min(k1, K) - P.nc : 0;
          T gs[6] = {0, 0, 0, 0, 0, 0};
          T qxh, qxl, qyh, qyl;
          if constexpr (MIXED) {
            float a_, b_, c_, d_;
            split_ff(px, a_, b_);
            split_ff(py, c_, d_);
            qxh = a_; qxl = b_; qyh = c_; qyl = d_;
          } else {
            qxh = (T)px; qxl = (T)0; qyh = (T)py; qyl = (T)0;
          }
          // Each member's (alpha, Psi) per unit strength is kbar (dx, dy) and
          // Psi_ij = kbar delta_ij + t x_i x_j; its derivative in a parameter contracts with the
          // cotangents as kbar' U + t' V, with U and V below.  Closed forms, P = 1/(S + s),
          // Q = 1/(R + a): dkbar/ds = -P/S, dkbar/da = Q/R, dt/ds = (P^2/S^2)(2 + s/S),
          // dt/da = -(Q^2/R^2)(2 + a/R); kbar = P - Q is taken in its cancellation-free form.
          for (int m = m0; m < m1; ++m) {
            const Mem& M = dm[m];
            const T Ms = mem_s(M), Ma = mem_a(M);
            T dx, dy;
            if constexpr (MIXED) {
              dx = offset_of(qxh, qxl, M.xh, M.xl);
              dy = offset_of(qyh, qyl, M.yh, M.yl);
            } else {
              dx = qxh - M.xh;
              dy = qyh - M.yh;
            }
            const T dxx = dx * dx, dyy = dy * dy, r2 = dxx + dyy;
            const T iS = ::lf_rsqrt(::lf_fma(Ms, Ms, r2)), iR = ::lf_rsqrt(::lf_fma(Ma, Ma, r2));
            const T S = ::lf_fma(Ms, Ms, r2) * iS, R = ::lf_fma(Ma, Ma, r2) * iR;
            const T Pq = ::lf_rcp(S + Ms), Qq = ::lf_rcp(R + Ma);
            const T kb = (Ma - Ms) * Pq * Qq * ::lf_fma(Ma + Ms, ::lf_rcp(R + S), (T)1);
            const T P2iS = Pq * Pq * iS, Q2iR = Qq * Qq * iR;
            const T U = ::lf_fma(cot[0], dx, ::lf_fma(cot[1], dy, cot[2] + cot[3]));
            const T V = ::lf_fma(cot[2], dxx, ::lf_fma(cot[3], dyy, cot[4] * dx * dy));
            T Gb = ::lf_fma(kb, U, (Q2iR - P2iS) * V);
            T Gs = M.b * ::lf_fma(-Pq * iS, U, P2iS * iS * ::lf_fma(Ms, iS, (T)2) * V);
            T Ga = M.b * ::lf_fma(Qq * iR, U, -Q2iR * iR * ::lf_fma(Ma, iR, (T)2) * V);
            if (AUX && C.aux) {
              // flux / time delay.  psi per unit b is (S - R) - s ln(S + s) + a ln(R + a), with
              // d/ds = -ln(S + s) and d/da = ln(R + a).  A round profile has d kbar / d(r^2) = t / 2,
              // so psi_ijk = t (x_k delta_ij + x_j delta_ik + x_i delta_jk) + 2 t' x_i x_j x_k,
              // t' = dt / d(r^2) = (P^2 / S^2)(P + 1 / (2S)) - (Q^2 / R^2)(Q + 1 / (2R)), and the
              // contraction with T_bar is t W1 + 2 t' W3; t and t' on dual numbers over (s, a).
              typedef Dual<T, 2> D2;
              const D2 s_ = D2::var(Ms, 0), a_ = D2::var(Ma, 1);
              const D2 Sd = lf_sqrt(s_ * s_ + D2::cst(r2));
              const D2 Rd = lf_sqrt(a_ * a_ + D2::cst(r2));
              const D2 iSd = lf_rcp(Sd), iRd = lf_rcp(Rd);
              const D2 Pd = lf_rcp(Sd + s_), Qd = lf_rcp(Rd + a_);
              const D2 P2d = Pd * Pd * iSd, Q2d = Qd * Qd * iRd;
              const D2 td = Q2d - P2d;
              const D2 tp = P2d * iSd * (Pd + D2(0.5) * iSd) - Q2d * iRd * (Qd + D2(0.5) * iRd);
              const T W1 = (T)3 * (tb[0] * dx + tb[3] * dy) + tb[1] * dy + tb[2] * dx;
              const T W3 = dxx * (tb[0] * dx + tb[1] * dy) + dyy * (tb[2] * dx + tb[3] * dy);
              const T psi_u = (Ms - Ma) * (Ms + Ma) * ::lf_rcp(S + R) - Ms * ::lf_log(S + Ms) + Ma * ::lf_log(R + Ma);
              Gb += pb * psi_u + td.v * W1 + (T)2 * tp.v * W3;
              Gs += M.b * (-pb * ::lf_log(S + Ms) + td.d[0] * W1 + (T)2 * tp.d[0] * W3);
              Ga += M.b * (pb * ::lf_log(R + Ma) + td.d[1] * W1 + (T)2 * tp.d[1] * W3);
            }
            const T fa = Ma * inv_cut_star;
            gs[LF_S_BSTAR] += Gb * M.fb;
            gs[LF_S_LAM] += Gb * M.b * (T)2 * M.loglr;
            gs[LF_S_CORESTAR] += Gs * M.fs;
            gs[LF_S_BETA] += Gs * Ms * M.loglr;
            gs[LF_S_CUTSTAR] += Ga * fa;
            gs[LF_S_ALPHA] += Ga * Ma * M.loglr;
          }
          for (int q = 0; q < 6; ++q) {
            const int p = C.scal_p[q];
            if (p < 0) continue;
            const double gw = warp_sum((double)gs[q]);
            if (lead) atomicAdd(&gacc[p], gw * xform_deriv(C.p_xform[p], th[p], P.apk));
          }
        }
      }
      }
      __syncthreads();
      for (int p = tid; p < C.P; p += blockDim.x) grad[(size_t)s * C.P + p] = gacc[p];
    }
    __syncthreads();
  }
}

// The anchor of the mixed tier's gradient: every image's member deflection sum at the plan's
// base fields (Eq. scaling, from the plan's float-float factor table), in FP64, rounded to
// float-float words.  One thread per image; run once per plan.
__global__ void k_member_base(const double* __restrict__ theta, int n_img, const MemPreF* __restrict__ mp,
                              int nm, lf_scaling sc, float4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_img) return;
  const double x = theta[2 * i], y = theta[2 * i + 1];
  double ax = 0.0, ay = 0.0;
  for (int k = 0; k < nm; ++k) {
    const MemPreF m = mp[k];
    const double dx = x - ((double)m.xh + (double)m.xl), dy = y - ((double)m.yh + (double)m.yl);
    const double b = sc.b_star * ((double)m.fb + (double)m.fbl);
    const double s = sc.core_star * ((double)m.fs + (double)m.fsl);
    const double a = sc.cut_star * ((double)m.fa + (double)m.fal);
    const double r2 = dx * dx + dy * dy;
    const double S = sqrt(s * s + r2), R = sqrt(a * a + r2);
    // b (1/(S + s) - 1/(R + a)) without its far-field cancellation
    const double kb = b * (a - s) / ((S + s) * (R + a)) * (1.0 + (a + s) / (R + S));
    ax += kb * dx;
    ay += kb * dy;
  }
  float xh, xl, yh, yl;
  split_ff(ax, xh, xl);
  split_ff(ay, yh, yl);
  out[i] = make_float4(xh, xl, yh, yl);
}

}  // namespace lf

// ======================================================================= host =======
using namespace lf;

// Nelder-Mead workspace (allocated on the first lf_nm_run, for max_samples runs).
struct NmWork {
  double *tmp = nullptr, *xb = nullptr, *xr = nullptr, *fr = nullptr, *x2 = nullptr,
         *f2 = nullptr, *shrink = nullptr, *fs = nullptr;
  int *step = nullptr, *flag = nullptr, *flag_host = nullptr;   // flag_host: pinned
};

struct lf_plan {
  int n_clusters = 0, P = 0, precision = LF_MIXED, flags = 0, max_samples = 0;
  NmWork nm;
  bool single_plane = true;
  bool has_aux = false;            // some cluster carries flux / time-delay measurements
  bool aux_afree = false;          // ... and samples a family's a_dis (no gradient then)
  std::vector<ClusterDesc> desc;
  std::vector<double> cost;
  ClusterDesc* d_desc = nullptr;
  int* d_counter = nullptr;
  int* d_order = nullptr;
  int nfree_max = 0;               // largest number of sampled components of a cluster
  // sampler workspace (allocated on the first lf_aies_run): proposals of one half, their z,
  // prior flags and chi^2
  double* d_prop = nullptr;
  double* d_z = nullptr;
  int* d_inside = nullptr;
  double* d_chi2_prop = nullptr;
  void* d_free_dig = nullptr;      // [max_samples * LF_MAX_FREE] digested sampled components
  lf_comp* d_free_raw = nullptr;   // [max_samples * LF_MAX_FREE] their fields (adjoint)
  std::vector<void*> allocs;
  int block = LF_CHI2_BLOCK;
  int block_grad = LF_CHI2_BLOCK;  // threads per block of the gradient launch
  int ks_cap = 32;
  bool tuned = false;
  uint32_t smem = 0, smem_img = 0, smem_aux = 0;
  uint32_t smem_grad = 0;          // gradient launches (0: the plan has no gradient kernel)
  int grid_chi2 = 0, grid_grad = 0, grid_aux = 0, grid_img = 0;   // grid_grad: of the plan's gradient kernel
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // CUDA graphs of the chi^2 launch (slot 0) and the gradient launch (slot 1), each with the
  // buffers and S it was captured for
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  const void* g_theta[2] = {nullptr, nullptr};
  void* g_out[2] = {nullptr, nullptr};
  int g_S[2] = {-1, -1};
  // The cotangents of the adjoint are weighted by the offsets d_i = beta_i - beta_model, which
  // are only ~sigma_pos: FP32 member deflections (a few 1e-6 arcsec) would put ~1e-4 relative
  // errors on them.  A single-plane LF_MIXED plan without flux / time-delay terms therefore
  // anchors its gradient's member sums at the plan's base fields (grad_anchor: the base sums
  // per image in FP64, the sample's change in FP32); any other LF_MIXED plan runs its gradient
  // on grad_ff, the LF_FF plan over the same clusters.
  bool grad_anchor = false;
  lf_plan* grad_ff = nullptr;
};

namespace lf {

static lf_status plan_alloc(lf_plan* pl, void** out, size_t bytes) {
  *out = nullptr;
  if (bytes == 0) return LF_OK;
  cudaError_t e = cudaMalloc(out, bytes);
  if (e != cudaSuccess) return fail(LF_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  pl->allocs.push_back(*out);
  return LF_OK;
}

template <class X>
static lf_status plan_upload(lf_plan* pl, const X* host, size_t n, X** dev) {
  void* p = nullptr;
  LF_TRY(plan_alloc(pl, &p, n * sizeof(X)));
  if (n) LF_CUDA(cudaMemcpy(p, host, n * sizeof(X), cudaMemcpyHostToDevice));
  *dev = reinterpret_cast<X*>(p);
  return LF_OK;
}

static bool comp_ok(const lf_comp& r) {
  bool ok = r.kind >= 1 && r.kind <= 6 && std::isfinite(r.x) && std::isfinite(r.y) &&
            std::isfinite(r.b) && std::isfinite(r.pa);
  if (r.kind == LF_SIE || r.kind == LF_DPIE)
    ok = ok && r.eps >= 0.0 && r.eps < 1.0 && r.core >= 0.0 && std::isfinite(r.core);
  if (r.kind == LF_DPIE) ok = ok && std::isfinite(r.cut) && r.cut > r.core;
  if (r.kind == LF_NFW) ok = ok && r.core > 0.0 && std::isfinite(r.core);
  if (r.kind == LF_ENFW)
    ok = ok && r.core > 0.0 && std::isfinite(r.core) && r.eps >= 0.0 && r.eps < 1.0;
  return ok;
}

static int pow2_floor(int v) {
  int r = 1;
  while (r * 2 <= v) r *= 2;
  return r;
}

// Component slices per image: the power of two minimising a simple cost model of one work
// item, rounds x (components per slice + per-task overhead), capped by the tuner's choice.
static int choose_ks(int n_img, int K, int block, int cap, int ipt) {
  const double overhead = 24.0;   // task set-up and shuffle reduction, in component evaluations
  int best = 1;
  double best_cost = 1e300;
  for (int ks = 1; ks <= 32 && ks <= cap; ks *= 2) {
    if (ks > 1 && K / ks < 8) break;
    long long tasks = (long long)((n_img + ipt - 1) / ipt) * ks;   // image groups x slices
    long long rounds = (tasks + block - 1) / block;
    double cost = (double)rounds * ((double)K / ks + overhead);
    if (cost < best_cost * 0.97) { best_cost = cost; best = ks; }
  }
  return best;
}

// Parameter map of one cluster into its descriptor (C.np, C.pl[].nm and C.n_fam set):
// p_comp >= 0 a component field, -1 a scaling-relation slot of the first plane that has
// members, -2 the a_dis of family p_field (single-plane clusters, sampled directly).
static lf_status parse_params(const lf_cluster& cl, const int* comp_base, ClusterDesc& C) {
  if (cl.P < 1 || cl.P > LF_MAX_P || !cl.p_comp || !cl.p_field || !cl.p_xform)
    return fail(LF_EINVAL, "need 1..%d parameters with a complete map", LF_MAX_P);
  C.P = cl.P;
  C.scal_plane = -1;
  for (int j = 0; j < C.np; ++j)
    if (C.pl[j].nm > 0) { C.scal_plane = j; break; }
  for (int k = 0; k < 6; ++k) C.scal_p[k] = -1;
  C.scal_free = 0;
  C.n_free = 0;
  C.n_afree = 0;
  for (int p = 0; p < cl.P; ++p) {
    const int gc = cl.p_comp[p], fld = cl.p_field[p], xf = cl.p_xform[p];
    if (xf < 0 || xf > 3) return fail(LF_EINVAL, "parameter %d: unknown transform", p);
    C.p_xform[p] = xf;
    if (gc == -2) {
      if (C.np != 1) return fail(LF_EUNSUPPORTED, "parameter %d: a sampled a_dis needs a single-plane cluster", p);
      if (fld < 0 || fld >= C.n_fam) return fail(LF_EINVAL, "parameter %d: family %d out of range", p, fld);
      if (xf != LF_XF_IDENT) return fail(LF_EINVAL, "parameter %d: a_dis is sampled directly (transform 0)", p);
      for (int q = 0; q < C.n_afree; ++q)
        if (C.afree_fam[q] == fld) return fail(LF_EINVAL, "a_dis of family %d targeted twice", fld);
      C.afree_fam[C.n_afree] = fld;
      C.afree_p[C.n_afree] = p;
      ++C.n_afree;
      C.p_plane[p] = 0;
      continue;
    }
    if (gc == -1) {
      if (C.scal_plane < 0) return fail(LF_EINVAL, "parameter %d targets a scaling relation but no plane has members", p);
      if (fld < 0 || fld > 5) return fail(LF_EINVAL, "parameter %d: unknown scaling slot", p);
      if (C.scal_p[fld] >= 0) return fail(LF_EINVAL, "scaling slot %d targeted twice", fld);
      C.scal_p[fld] = p;
      C.scal_free = 1;
      C.p_plane[p] = C.scal_plane;
      continue;
    }
    if (gc < 0) return fail(LF_EINVAL, "parameter %d: unknown target %d", p, gc);
    if (fld < 0 || fld > 6) return fail(LF_EINVAL, "parameter %d: unknown field", p);
    if (gc >= comp_base[C.np]) return fail(LF_EINVAL, "parameter %d: component %d out of range", p, gc);
    int j = 0;
    while (gc >= comp_base[j + 1]) ++j;
    const int k = gc - comp_base[j];
    C.p_plane[p] = j;
    int f = 0;
    while (f < C.n_free && !(C.free_plane[f] == j && C.free_comp[f] == k)) ++f;
    if (f == C.n_free) {
      if (C.n_free == LF_MAX_FREE) return fail(LF_EUNSUPPORTED, "more than %d sampled components", LF_MAX_FREE);
      C.free_plane[f] = j;
      C.free_comp[f] = k;
      for (int q = 0; q < 7; ++q) C.free_p[f][q] = -1;
      ++C.n_free;
    }
    if (C.free_p[f][fld] >= 0) return fail(LF_EINVAL, "field targeted twice");
    C.free_p[f][fld] = p;
  }
  return LF_OK;
}

static void layout_cluster(ClusterDesc& C, int precision, int block, int ks_cap) {
  const bool mixed = precision != LF_FP64;
  const uint32_t mem_sz = precision == LF_FF ? sizeof(MemX) : precision == LF_MIXED ? sizeof(MemT<float>)
                                                                                   : sizeof(MemT<double>);
  auto al = [](uint32_t v) { return (v + 15u) & ~15u; };
  // regions every launch reads
  uint32_t o = LF_HDR;
  for (int j = 0; j < C.np; ++j) {
    PlaneDesc& P = C.pl[j];
    o = al(o); P.off_rawc = o; o += (uint32_t)P.nc * 64u;
    P.off_mpre = 0;   // the member pre-table is read from global memory, not staged
    o = al(o); P.off_dc = o; o += (uint32_t)P.nc * (mixed ? sizeof(CompT<float>) : sizeof(CompT<double>));
  }
  C.img_stride = C.np > 1 ? 16 + 6 * C.np : 14;
  C.img_stride_f = IMGF;
  C.img_stride_d = C.np > 1 ? 2 + 6 * C.np : 0;
  o = al(o); C.off_img = o;
  o += mixed ? (uint32_t)C.n_img * IMGF * 4u : (uint32_t)C.n_img * C.img_stride * 8u;
  o = al(o); C.off_imgd = o;
  if (mixed) o += (uint32_t)C.n_img * C.img_stride_d * 8u;
  C.off_fam = o; o += (uint32_t)C.n_fam * 3u * 8u;
  C.off_par = o; o += (uint32_t)C.P * 2u * 8u;
  o = al(o); C.off_free = o; o += (uint32_t)C.n_free * 64u;
  // per sample: a_dis of each family (double, float-float) and the parameter setting it
  o = al(o); C.off_fama = o; o += (uint32_t)C.n_fam * (8u + 8u + 4u);
  const uint32_t var = al(o);
  // forward passes: the members as packed pairs (mixed tier) or scalar records
  uint32_t of = var, os = var;
  for (int j = 0; j < C.np; ++j) {
    PlaneDesc& P = C.pl[j];
    P.off_dmp = al(of);
    of = P.off_dmp + (precision == LF_MIXED ? mem_records<MemPair>(P.nm) * (uint32_t)sizeof(MemPair)
                                            : (uint32_t)P.nm * mem_sz);
    P.off_mfac = al(of);
    if (precision == LF_MIXED) of = P.off_mfac + (uint32_t)P.nm * 12u;
    P.off_dm = al(os);
    os = P.off_dm + (uint32_t)P.nm * mem_sz;
    P.off_dma = al(os);
    if (precision == LF_MIXED && C.mbase) os = P.off_dma + (uint32_t)P.nm * (uint32_t)sizeof(MemA);
  }
  if (precision != LF_MIXED)
    for (int j = 0; j < C.np; ++j) C.pl[j].off_dmp = C.pl[j].off_dm;
  C.smem = al(of);
  // image-plane chi^2: + Newton state per image
  C.off_newton = al(of);
  C.smem_img = al(C.off_newton + (uint32_t)C.n_img * 4u * 8u);
  // flux / time-delay pass: scalar members + per image psi, the third derivatives, y_i and d_i
  // (LF_AUXI doubles), then per family m_src, Delta t_0 and the adjoint's lambda (LF_AUXF)
  C.off_aux = al(os);
  const uint32_t aux_b = C.aux ? ((uint32_t)C.n_img * LF_AUXI + (uint32_t)C.n_fam * LF_AUXF) * 8u : 0u;
  C.smem_aux = al(C.off_aux + aux_b);
  // adjoint: scalar members + (several planes) per image and plane the position theta_j (2),
  // Psi_j (3) and the cotangents of (alpha_j, Psi_j) (5); then the third derivatives of psi
  // (4) at every plane after the first.  One plane with flux / time-delay terms: the forward
  // pass's records above, then the adjoint's per-image records (LF_AUXG doubles).
  C.off_mpg = al(os);
  C.mpg_stride = C.np > 1 ? 10 * C.np + 4 * (C.np - 1) : 0;
  C.smem_grad = al(C.off_mpg + (uint32_t)C.n_img * (uint32_t)C.mpg_stride * 8u);
  C.off_auxg = C.smem_aux;
  if (C.aux) C.smem_grad = std::max(C.smem_grad, al(C.off_auxg + (uint32_t)C.n_img * LF_AUXG * 8u));
  int K = 0;
  for (int j = 0; j < C.np; ++j) K = std::max(K, C.pl[j].nc + C.pl[j].nm);
  C.ks = choose_ks(C.n_img, K, block, ks_cap, 2);
}

static lf_status relayout(lf_plan* pl) {
  pl->smem = pl->smem_img = pl->smem_aux = pl->smem_grad = 0;
  for (auto& C : pl->desc) {
    layout_cluster(C, pl->precision, pl->block, pl->ks_cap);
    pl->smem = std::max(pl->smem, C.smem);
    pl->smem_img = std::max(pl->smem_img, C.smem_img);
    pl->smem_aux = std::max(pl->smem_aux, C.smem_aux);
    pl->smem_grad = std::max(pl->smem_grad, C.smem_grad);
  }
  if (pl->smem > LF_SMEM_MAX || pl->smem_aux > LF_SMEM_MAX)
    return fail(LF_EUNSUPPORTED, "cluster too large for shared memory (%u B)", std::max(pl->smem, pl->smem_aux));
  if (pl->smem_img > LF_SMEM_MAX) pl->smem_img = 0;     // the image-plane chi^2 is refused at call time
  if (pl->smem_grad > LF_SMEM_MAX) pl->smem_grad = 0;   // the gradient is refused at call time
  LF_CUDA(cudaMemcpy(pl->d_desc, pl->desc.data(), pl->desc.size() * sizeof(ClusterDesc),
                     cudaMemcpyHostToDevice));
  int dev = 0, nsm = 0, occ = 0;
  LF_CUDA(cudaGetDevice(&dev));
  LF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  auto kset = [&](const void* k, uint32_t bytes) -> lf_status {
    LF_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    LF_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    return LF_OK;
  };
  const void* kc = pl->precision == LF_MIXED ? (const void*)k_chi2<LF_MIXED, false>
                   : pl->precision == LF_FF  ? (const void*)k_chi2<LF_FF, false>
                                             : (const void*)k_chi2<LF_FP64, false>;
  // the gradient (with the flux / time-delay adjoint when the plan has measurements); a mixed
  // plan's gradient is anchored (one plane, no flux / time-delay terms) or runs on its LF_FF
  // companion
  const void* kg = pl->precision == LF_MIXED ? (pl->grad_anchor ? (const void*)k_chi2<LF_MIXED, true> : nullptr)
                   : pl->precision == LF_FF  ? (pl->has_aux ? (const void*)k_chi2<LF_FF, true, 2>
                                                            : (const void*)k_chi2<LF_FF, true>)
                                             : (pl->has_aux ? (const void*)k_chi2<LF_FP64, true, 2>
                                                            : (const void*)k_chi2<LF_FP64, true>);
  const void* ki = pl->precision == LF_MIXED ? (const void*)k_chi2<LF_MIXED, false, 1>
                   : pl->precision == LF_FF  ? (const void*)k_chi2<LF_FF, false, 1>
                                             : (const void*)k_chi2<LF_FP64, false, 1>;
  const void* ka = pl->precision == LF_MIXED ? (const void*)k_chi2<LF_MIXED, false, 2>
                   : pl->precision == LF_FF  ? (const void*)k_chi2<LF_FF, false, 2>
                                             : (const void*)k_chi2<LF_FP64, false, 2>;
  LF_TRY(kset(kc, pl->smem));
  pl->grid_img = 0;
  if (pl->smem_img > 0) {
    LF_TRY(kset(ki, pl->smem_img));
    LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ki, pl->block, pl->smem_img));
    pl->grid_img = nsm * std::max(occ, 1);
  }
  if (pl->has_aux) {
    LF_TRY(kset(ka, pl->smem_aux));
    LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ka, pl->block, pl->smem_aux));
    pl->grid_aux = nsm * std::max(occ, 1);
  }
  LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kc, pl->block, pl->smem));
  pl->grid_chi2 = nsm * std::max(occ, 1);
  pl->grid_grad = 0;
  pl->block_grad = pl->grad_anchor ? LF_CHI2_GRAD_BLOCK : pl->block;
  if (pl->smem_grad > 0 && kg) {
    LF_TRY(kset(kg, pl->smem_grad));
    LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kg, pl->block_grad, pl->smem_grad));
    pl->grid_grad = nsm * std::max(occ, 1);
  }
  for (int g = 0; g < 2; ++g)
    if (pl->gexec[g]) {
      cudaGraphExecDestroy(pl->gexec[g]);
      pl->gexec[g] = nullptr;
    }
  return LF_OK;
}

static lf_status build_cluster(lf_plan* pl, const lf_cluster& cl, ClusterDesc& C, double& cost) {
  memset(&C, 0, sizeof C);
  if (cl.n_planes < 1 || cl.n_planes > LF_MAX_PLANES || !cl.planes)
    return fail(LF_EINVAL, "cluster needs 1..8 planes");
  if (cl.n_planes > 1 && !cl.ratios) return fail(LF_EINVAL, "multi-plane cluster needs ratios");
  if (!cl.arcsec_per_kpc) return fail(LF_EINVAL, "arcsec_per_kpc is NULL");
  C.np = cl.n_planes;
  const bool mixed = pl->precision == LF_MIXED;   // FP32 member pre-table (LF_FF keeps FP64)
  std::vector<int> comp_base(C.np + 1, 0);
  std::vector<std::vector<lf_comp>> comps(C.np);
  cost = 0.0;
  for (int j = 0; j < C.np; ++j) {
    const lf_plane& src = cl.planes[j];
    LF_TRY(check_plane(&src));
    PlaneDesc& P = C.pl[j];
    P.nc = src.n_comp;
    P.nm = src.n_mem;
    P.sc = src.scaling;
    P.apk = cl.arcsec_per_kpc[j];
    if (!(std::isfinite(P.apk) && P.apk > 0)) return fail(LF_EINVAL, "invalid arcsec_per_kpc");
    comps[j].resize(P.nc);
    if (P.nc) LF_CUDA(cudaMemcpy(comps[j].data(), src.comp, P.nc * sizeof(lf_comp), cudaMemcpyDeviceToHost));
    for (int i = 0; i < P.nc; ++i)
      if (!comp_ok(comps[j][i])) return fail(LF_EINVAL, "plane %d component %d is invalid", j, i);
    lf_comp* dcomp = nullptr;
    LF_TRY(plan_upload(pl, comps[j].data(), P.nc, &dcomp));
    P.comp = dcomp;
    std::vector<lf_member> mem(P.nm);
    if (P.nm) LF_CUDA(cudaMemcpy(mem.data(), src.mem, P.nm * sizeof(lf_member), cudaMemcpyDeviceToHost));
    const double LN10 = 2.302585092994045684;
    if (mixed) {
      std::vector<MemPreF> pre(P.nm);
      for (int i = 0; i < P.nm; ++i) {
        double lnl = mem[i].log_l * LN10;
        split_ff(mem[i].x, pre[i].xh, pre[i].xl);
        split_ff(mem[i].y, pre[i].yh, pre[i].yl);
        split_ff(std::exp(2.0 * P.sc.lam * lnl), pre[i].fb, pre[i].fbl);
        split_ff(std::exp(P.sc.beta * lnl), pre[i].fs, pre[i].fsl);
        split_ff(std::exp(P.sc.alpha * lnl), pre[i].fa, pre[i].fal);
        pre[i].lnl = (float)lnl;
        pre[i].pad = 0.f;
        if (!std::isfinite(mem[i].x) || !std::isfinite(mem[i].y) || !std::isfinite(lnl))
          return fail(LF_EINVAL, "plane %d member %d is not finite", j, i);
      }
      MemPreF* d = nullptr;
      LF_TRY(plan_upload(pl, pre.data(), pre.size(), &d));
      P.mpre = d;
    } else {
      std::vector<MemPreD> pre(P.nm);
      for (int i = 0; i < P.nm; ++i) {
        double lnl = mem[i].log_l * LN10;
        pre[i] = MemPreD{mem[i].x, mem[i].y, std::exp(2.0 * P.sc.lam * lnl), std::exp(P.sc.beta * lnl),
                         std::exp(P.sc.alpha * lnl), lnl, 0.0, 0.0};
        if (!std::isfinite(mem[i].x) || !std::isfinite(mem[i].y) || !std::isfinite(lnl))
          return fail(LF_EINVAL, "plane %d member %d is not finite", j, i);
      }
      MemPreD* d = nullptr;
      LF_TRY(plan_upload(pl, pre.data(), pre.size(), &d));
      P.mpre = d;
    }
    comp_base[j + 1] = comp_base[j] + P.nc;
    if (C.np > 1)
      for (int l = 0; l < C.np; ++l) C.r[j][l] = (l > j) ? cl.ratios[j * C.np + l] : 0.0;
  }
  // images
  const lf_images& im = cl.images;
  if (im.n_img < 1 || im.n_img > LF_MAX_IMG) return fail(LF_EINVAL, "need 1..%d images", LF_MAX_IMG);
  if (im.n_fam < 1 || !im.theta_obs || !im.sinv || !im.fam_off || !im.fam_ratio)
    return fail(LF_EINVAL, "incomplete image set");
  if (im.fam_off[0] != 0 || im.fam_off[im.n_fam] != im.n_img)
    return fail(LF_EINVAL, "fam_off must run from 0 to n_img");
  std::vector<int> img_fam(im.n_img);
  for (int f = 0; f < im.n_fam; ++f) {
    if (im.fam_off[f + 1] <= im.fam_off[f]) return fail(LF_EINVAL, "family %d is empty", f);
    for (int i = im.fam_off[f]; i < im.fam_off[f + 1]; ++i) img_fam[i] = f;
    for (int l = 0; l < C.np; ++l) {
      double v = im.fam_ratio[f * C.np + l];
      bool ok = std::isfinite(v) && (C.np == 1 ? (v > 0.0 && v <= 1.0) : (v >= 0.0 && v <= 1.0));
      if (!ok) return fail(LF_EINVAL, "family %d has an invalid distance ratio", f);
    }
  }
  for (int i = 0; i < im.n_img; ++i) {
    double a = im.sinv[3 * i], b = im.sinv[3 * i + 1], c = im.sinv[3 * i + 2];
    if (!(std::isfinite(im.theta_obs[2 * i]) && std::isfinite(im.theta_obs[2 * i + 1]) &&
          std::isfinite(a) && std::isfinite(b) && std::isfinite(c) && a > 0 && c > 0 && a * c - b * b > 0))
      return fail(LF_EINVAL, "image %d: non-finite position or S^-1 not positive definite", i);
  }
  C.n_img = im.n_img;
  C.n_fam = im.n_fam;
  double* dtheta = nullptr; double* dsinv = nullptr; double* dratio = nullptr;
  int* doff = nullptr; int* dif = nullptr;
  LF_TRY(plan_upload(pl, im.theta_obs, 2 * (size_t)im.n_img, &dtheta));
  LF_TRY(plan_upload(pl, im.sinv, 3 * (size_t)im.n_img, &dsinv));
  LF_TRY(plan_upload(pl, im.fam_ratio, (size_t)im.n_fam * C.np, &dratio));
  LF_TRY(plan_upload(pl, im.fam_off, (size_t)im.n_fam + 1, &doff));
  LF_TRY(plan_upload(pl, img_fam.data(), img_fam.size(), &dif));
  C.theta = dtheta; C.sinv = dsinv; C.fam_ratio = dratio; C.fam_off = doff; C.img_fam = dif;
  {
    std::vector<float4> tf(im.n_img), sf(im.n_img);
    std::vector<float2> rf((size_t)im.n_fam * C.np);
    for (int i = 0; i < im.n_img; ++i) {
      split_ff(im.theta_obs[2 * i], tf[i].x, tf[i].y);
      split_ff(im.theta_obs[2 * i + 1], tf[i].z, tf[i].w);
      sf[i] = make_float4((float)im.sinv[3 * i], (float)im.sinv[3 * i + 1], (float)im.sinv[3 * i + 2], 0.f);
    }
    for (size_t q = 0; q < rf.size(); ++q) split_ff(im.fam_ratio[q], rf[q].x, rf[q].y);
    float4* dtf = nullptr; float4* dsf = nullptr; float2* drf = nullptr;
    LF_TRY(plan_upload(pl, tf.data(), tf.size(), &dtf));
    LF_TRY(plan_upload(pl, sf.data(), sf.size(), &dsf));
    LF_TRY(plan_upload(pl, rf.data(), rf.size(), &drf));
    C.theta_ff = dtf; C.sinv_f = dsf; C.ratio_ff = drf;
  }
  // flux and time-delay measurements (optional)
  C.aux = 0;
  if (im.mag || im.td) {
    if (C.np != 1) return fail(LF_EUNSUPPORTED, "flux and time-delay terms need a single-plane cluster");
    if (im.mag && !im.mag_err) return fail(LF_EINVAL, "mag given without mag_err");
    if (im.td && !im.td_err) return fail(LF_EINVAL, "td given without td_err");
    if (im.td && !(std::isfinite(im.td_scale) && im.td_scale > 0))
      return fail(LF_EINVAL, "td_scale must be finite and > 0");
    std::vector<double> v(4 * (size_t)im.n_img, 0.0);
    for (int i = 0; i < im.n_img; ++i) {
      if (im.mag && std::isfinite(im.mag[i]) && std::isfinite(im.mag_err[i]) && im.mag_err[i] > 0) {
        v[i] = im.mag[i];
        v[im.n_img + i] = 1.0 / (im.mag_err[i] * im.mag_err[i]);
      }
      if (im.td && std::isfinite(im.td[i]) && std::isfinite(im.td_err[i]) && im.td_err[i] > 0) {
        v[2 * im.n_img + i] = im.td[i];
        v[3 * im.n_img + i] = 1.0 / (im.td_err[i] * im.td_err[i]);
      }
    }
    double* dv = nullptr;
    LF_TRY(plan_upload(pl, v.data(), v.size(), &dv));
    C.aux_mag = dv; C.aux_wmag = dv + im.n_img; C.aux_td = dv + 2 * im.n_img; C.aux_wtd = dv + 3 * im.n_img;
    C.td_scale = im.td ? im.td_scale : 0.0;
    C.aux = (im.mag ? 1 : 0) | (im.td ? 2 : 0);
  }
  // parameter map
  LF_TRY(parse_params(cl, comp_base.data(), C));
  int K = 0;
  for (int j = 0; j < C.np; ++j) K += C.pl[j].nc + C.pl[j].nm;
  cost = (double)C.n_img * K;
  return LF_OK;
}

template <int MODE>
static void launch_mode(lf_plan* pl, const double* theta, int S, double* chi2, double* grad,
                        cudaStream_t st, int spc) {
  const int nprep = S * pl->nfree_max;
  if (nprep > 0)
    k_chi2_prep<MODE><<<(nprep + 63) / 64, 64, 0, st>>>(pl->d_desc, spc, S, pl->nfree_max, theta,
                                                        pl->d_free_dig, pl->d_free_raw);
  if (grad) {
    int g = std::min(pl->grid_grad, S);
    if constexpr (MODE == LF_MIXED) {   // anchored plans only (the others use their LF_FF plan)
      k_chi2<MODE, true><<<g, pl->block_grad, pl->smem_grad, st>>>(pl->d_desc, pl->d_order, spc, S, theta,
                                                              chi2, grad, pl->d_counter, g_member_chunk,
                                                              pl->d_free_dig, pl->d_free_raw);
    } else {
      if (pl->has_aux)
        k_chi2<MODE, true, 2><<<g, pl->block, pl->smem_grad, st>>>(pl->d_desc, pl->d_order, spc, S, theta,
                                                              chi2, grad, pl->d_counter, g_member_chunk,
                                                              pl->d_free_dig, pl->d_free_raw);
      else
        k_chi2<MODE, true><<<g, pl->block, pl->smem_grad, st>>>(pl->d_desc, pl->d_order, spc, S, theta, chi2,
                                                           grad, pl->d_counter, g_member_chunk,
                                                           pl->d_free_dig, pl->d_free_raw);
    }
  } else if (pl->has_aux) {
    int g = std::min(pl->grid_aux, S);
    k_chi2<MODE, false, 2><<<g, pl->block, pl->smem_aux, st>>>(pl->d_desc, pl->d_order, spc, S, theta, chi2,
                                                           nullptr, pl->d_counter, g_member_chunk,
                                                           pl->d_free_dig, nullptr);
  } else {
    int g = std::min(pl->grid_chi2, S);
    k_chi2<MODE, false><<<g, pl->block, pl->smem, st>>>(pl->d_desc, pl->d_order, spc, S, theta, chi2,
                                                        nullptr, pl->d_counter, g_member_chunk,
                                                        pl->d_free_dig, pl->d_free_raw);
  }
}

template <int MODE>
static void launch_img(lf_plan* pl, const double* theta, int S, int iters, double* chi2, double* rms,
                       cudaStream_t st, int spc) {
  const int nprep = S * pl->nfree_max;
  if (nprep > 0)
    k_chi2_prep<MODE><<<(nprep + 63) / 64, 64, 0, st>>>(pl->d_desc, spc, S, pl->nfree_max, theta,
                                                        pl->d_free_dig, pl->d_free_raw);
  int g = std::min(pl->grid_img, S);
  k_chi2<MODE, false, 1><<<g, pl->block, pl->smem_img, st>>>(pl->d_desc, pl->d_order, spc, S, theta, chi2,
                                                         nullptr, pl->d_counter, g_member_chunk,
                                                         pl->d_free_dig, nullptr, iters, rms);
}

static lf_status ensure_nm_workspace(lf_plan* pl, int M) {
  if (pl->nm.xb) return LF_OK;
  const size_t m = (size_t)pl->max_samples, P = (size_t)pl->P;
  void* p = nullptr;
  NmWork& w = pl->nm;
  LF_TRY(plan_alloc(pl, &p, m * (P + 1) * P * sizeof(double))); w.tmp = (double*)p;
  LF_TRY(plan_alloc(pl, &p, m * P * sizeof(double))); w.xb = (double*)p;
  LF_TRY(plan_alloc(pl, &p, m * P * sizeof(double))); w.xr = (double*)p;
  LF_TRY(plan_alloc(pl, &p, m * P * sizeof(double))); w.x2 = (double*)p;
  LF_TRY(plan_alloc(pl, &p, m * sizeof(double))); w.fr = (double*)p;
  LF_TRY(plan_alloc(pl, &p, m * sizeof(double))); w.f2 = (double*)p;
  LF_TRY(plan_alloc(pl, &p, m * P * P * sizeof(double))); w.shrink = (double*)p;
  LF_TRY(plan_alloc(pl, &p, m * P * sizeof(double))); w.fs = (double*)p;
  LF_TRY(plan_alloc(pl, &p, m * sizeof(int))); w.step = (int*)p;
  LF_TRY(plan_alloc(pl, &p, sizeof(int))); w.flag = (int*)p;
  LF_CUDA(cudaMallocHost(&p, sizeof(int)));
  w.flag_host = (int*)p;
  (void)M;
  return LF_OK;
}

static lf_status ensure_sampler_workspace(lf_plan* pl) {
  if (pl->d_prop) return LF_OK;
  const size_t h = (size_t)pl->max_samples;
  void* p = nullptr;
  LF_TRY(plan_alloc(pl, &p, h * pl->P * sizeof(double)));
  pl->d_prop = (double*)p;
  LF_TRY(plan_alloc(pl, &p, h * sizeof(double)));
  pl->d_z = (double*)p;
  LF_TRY(plan_alloc(pl, &p, h * sizeof(int)));
  pl->d_inside = (int*)p;
  LF_TRY(plan_alloc(pl, &p, h * sizeof(double)));
  pl->d_chi2_prop = (double*)p;
  return LF_OK;
}

static lf_status launch_chi2(lf_plan* pl, const double* theta, int S, double* chi2, double* grad,
                             cudaStream_t st) {
  const int spc = S / pl->n_clusters;
  LF_CUDA(cudaMemsetAsync(pl->d_counter, 0, sizeof(int), st));
  if (pl->precision == LF_MIXED) launch_mode<LF_MIXED>(pl, theta, S, chi2, grad, st, spc);
  else if (pl->precision == LF_FF) launch_mode<LF_FF>(pl, theta, S, chi2, grad, st, spc);
  else launch_mode<LF_FP64>(pl, theta, S, chi2, grad, st, spc);
  LF_CUDA(cudaGetLastError());
  return LF_OK;
}

// Times candidate (block, slice cap) shapes on the caller's inputs and keeps the fastest.
static lf_status autotune(lf_plan* pl, const double* theta, int S, double* chi2, cudaStream_t st) {
  // any multiple of a warp lets (image pair x slice) tasks fill the block
  const int blocks[15] = {64, 96, 128, 160, 192, 224, 256, 288, 320, 352, 384, 416, 448, 480, 512};
  const int caps[4] = {1, 2, 4, 8};
  cudaEvent_t e0, e1;
  LF_CUDA(cudaEventCreate(&e0));
  LF_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bb = pl->block, bc = pl->ks_cap;
  for (int b : blocks)
    for (int cap : caps) {
      if (b > chi2_max_block(pl->precision)) continue;   // beyond the kernels' launch bounds
      pl->block = b;
      pl->ks_cap = cap;
      if (relayout(pl) != LF_OK) continue;
      LF_TRY(launch_chi2(pl, theta, S, chi2, nullptr, st));
      LF_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < 2; ++r) LF_TRY(launch_chi2(pl, theta, S, chi2, nullptr, st));
      LF_CUDA(cudaEventRecord(e1, st));
      LF_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      LF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; bb = b; bc = cap; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pl->block = bb;
  pl->ks_cap = bc;
  LF_TRY(relayout(pl));
  pl->tuned = true;
  return LF_OK;
}

static lf_status run(lf_plan* pl, const double* theta, int S, double* chi2, double* grad, void* stream) {
  if (!pl) return fail(LF_EINVAL, "plan is NULL");
  if (!theta || !chi2) return fail(LF_EINVAL, "theta and chi2 are required");
  if (S < 1 || S > pl->max_samples) return fail(LF_EINVAL, "S must be in 1..%d", pl->max_samples);
  if (S % pl->n_clusters) return fail(LF_EINVAL, "S must be a multiple of the number of clusters");
  cudaStream_t st = (cudaStream_t)stream;
  if ((pl->flags & 2) && !pl->tuned) LF_TRY(autotune(pl, theta, S, chi2, st));
  if (!(pl->flags & 1)) return launch_chi2(pl, theta, S, chi2, grad, st);
  // CUDA graph: the counter reset and the persistent launch, replayed while the buffers and
  // S are unchanged, on the plan's stream ordered after / before the caller's stream.
  void* out_key = grad ? (void*)grad : (void*)chi2;
  const int gs = grad ? 1 : 0;
  if (!pl->gexec[gs] || pl->g_theta[gs] != theta || pl->g_out[gs] != out_key || pl->g_S[gs] != S) {
    if (pl->gexec[gs]) { cudaGraphExecDestroy(pl->gexec[gs]); pl->gexec[gs] = nullptr; }
    cudaGraph_t g = nullptr;
    LF_CUDA(cudaStreamBeginCapture(pl->gstream, cudaStreamCaptureModeThreadLocal));
    lf_status ls = launch_chi2(pl, theta, S, chi2, grad, pl->gstream);
    cudaError_t ce = cudaStreamEndCapture(pl->gstream, &g);
    if (ls != LF_OK) { if (g) cudaGraphDestroy(g); return ls; }
    if (ce != cudaSuccess) return fail(LF_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&pl->gexec[gs], g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fail(LF_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
    pl->g_theta[gs] = theta; pl->g_out[gs] = out_key; pl->g_S[gs] = S;
  }
  LF_CUDA(cudaEventRecord(pl->ev_in, st));
  LF_CUDA(cudaStreamWaitEvent(pl->gstream, pl->ev_in, 0));
  LF_CUDA(cudaGraphLaunch(pl->gexec[gs], pl->gstream));
  LF_CUDA(cudaEventRecord(pl->ev_out, pl->gstream));
  LF_CUDA(cudaStreamWaitEvent(st, pl->ev_out, 0));
  return LF_OK;
}

}  // namespace lf

extern "C" lf_status lf_plan_destroy(lf_plan* pl) {
  if (!pl) return LF_OK;
  if (pl->grad_ff) lf_plan_destroy(pl->grad_ff);
  for (int g = 0; g < 2; ++g)
    if (pl->gexec[g]) cudaGraphExecDestroy(pl->gexec[g]);
  if (pl->ev_in) cudaEventDestroy(pl->ev_in);
  if (pl->ev_out) cudaEventDestroy(pl->ev_out);
  if (pl->gstream) cudaStreamDestroy(pl->gstream);
  for (void* p : pl->allocs) cudaFree(p);
  if (pl->nm.flag_host) cudaFreeHost(pl->nm.flag_host);
  delete pl;
  return LF_OK;
}

extern "C" lf_status lf_plan_create(lf_plan** out, const lf_cluster* clusters, int32_t n_clusters,
                                    int32_t max_samples, int32_t precision, int32_t flags) {
  if (!out) return fail(LF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!clusters || n_clusters < 1) return fail(LF_EINVAL, "need at least one cluster");
  if (max_samples < n_clusters) return fail(LF_EINVAL, "max_samples must be >= n_clusters");
  if (precision < LF_FP64 || precision > LF_FF) return fail(LF_EINVAL, "unknown precision");
  if (flags & ~3) return fail(LF_EINVAL, "unknown flags");
  lf_plan* pl = new lf_plan();
  pl->n_clusters = n_clusters;
  pl->precision = precision;
  pl->block = std::min(pl->block, chi2_max_block(precision));
  pl->flags = flags;
  pl->max_samples = max_samples;
  pl->P = clusters[0].P;
  pl->desc.resize(n_clusters);
  pl->cost.resize(n_clusters);
  lf_status st = LF_OK;
  for (int c = 0; c < n_clusters && st == LF_OK; ++c) {
    if (clusters[c].P != pl->P) st = fail(LF_EINVAL, "every cluster must have the same P");
    else st = build_cluster(pl, clusters[c], pl->desc[c], pl->cost[c]);
    if (st == LF_OK && pl->desc[c].np > 1) pl->single_plane = false;
    if (st == LF_OK && pl->desc[c].aux) pl->has_aux = true;
    if (st == LF_OK && pl->desc[c].aux && pl->desc[c].n_afree > 0) pl->aux_afree = true;
    if (st == LF_OK) pl->nfree_max = std::max(pl->nfree_max, pl->desc[c].n_free);
  }
  if (st == LF_OK) {
    std::vector<int> order(n_clusters);
    for (int c = 0; c < n_clusters; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pl->cost[a] > pl->cost[b]; });
    void* p = nullptr;
    st = plan_alloc(pl, &p, n_clusters * sizeof(int));
    if (st == LF_OK) {
      pl->d_order = (int*)p;
      if (cudaMemcpy(pl->d_order, order.data(), n_clusters * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        st = fail(LF_ECUDA, "upload of the cluster order failed");
    }
    if (st == LF_OK) st = plan_alloc(pl, &p, sizeof(int));
    if (st == LF_OK) pl->d_counter = (int*)p;
    const size_t nfree = (size_t)max_samples * LF_MAX_FREE;
    const size_t dsz = precision == LF_FP64 ? sizeof(CompT<double>) : sizeof(CompT<float>);
    if (st == LF_OK) st = plan_alloc(pl, &p, nfree * dsz);
    if (st == LF_OK) pl->d_free_dig = p;
    if (st == LF_OK) st = plan_alloc(pl, &p, nfree * sizeof(lf_comp));
    if (st == LF_OK) pl->d_free_raw = (lf_comp*)p;
    if (st == LF_OK) st = plan_alloc(pl, &p, n_clusters * sizeof(ClusterDesc));
    if (st == LF_OK) pl->d_desc = (ClusterDesc*)p;
    // the anchored gradient: one plane, whose member positions and images are fixed.  (With
    // members on the first of several planes only, the later planes' explicit components in
    // float-float set the time: 3.00 ms against 2.92 ms for the float-float companion on the
    // three-plane workload, so such plans keep the companion.)
    if (st == LF_OK && precision == LF_MIXED && pl->single_plane && !pl->has_aux) {
      // the anchored gradient: the members' base sums at every image
      for (int c = 0; c < n_clusters && st == LF_OK; ++c) {
        ClusterDesc& C = pl->desc[c];
        st = plan_alloc(pl, &p, (size_t)std::max(C.n_img, 1) * sizeof(float4));
        if (st != LF_OK) break;
        const PlaneDesc& P0 = C.pl[0];
        if (C.n_img > 0)
          k_member_base<<<(C.n_img + 127) / 128, 128>>>(C.theta, C.n_img, (const MemPreF*)P0.mpre, P0.nm,
                                                        P0.sc, (float4*)p);
        C.mbase = (const float4*)p;
      }
      if (st == LF_OK && (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess))
        st = fail(LF_ECUDA, "the members' base sums failed");
      pl->grad_anchor = st == LF_OK;
    }
    if (st == LF_OK) st = relayout(pl);
    if (st == LF_OK && (flags & 1)) {
      if (cudaStreamCreateWithFlags(&pl->gstream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&pl->ev_in, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&pl->ev_out, cudaEventDisableTiming) != cudaSuccess)
        st = fail(LF_ECUDA, "stream / event creation failed");
    }
  }
  if (st == LF_OK && precision == LF_MIXED && !pl->grad_anchor)
    st = lf_plan_create(&pl->grad_ff, clusters, n_clusters, max_samples, LF_FF, flags);
  if (st != LF_OK) {
    lf_plan_destroy(pl);
    return st;
  }
  *out = pl;
  return LF_OK;
}

extern "C" lf_status lf_chi2_batch(lf_plan* plan, const double* theta, int32_t S, double* chi2,
                                   void* stream) {
  return run(plan, theta, S, chi2, nullptr, stream);
}

extern "C" lf_status lf_chi2_grad_batch(lf_plan* plan, const double* theta, int32_t S, double* chi2,
                                        double* grad, void* stream) {
  if (!plan) return fail(LF_EINVAL, "plan is NULL");
  if (!grad) return fail(LF_EINVAL, "grad is NULL");
  if (plan->grad_ff) plan = plan->grad_ff;
  if (plan->precision == LF_MIXED && !plan->grad_anchor)
    return fail(LF_EUNSUPPORTED, "no gradient plan");
  if (plan->smem_grad == 0)
    return fail(LF_EUNSUPPORTED, "the multi-plane adjoint's per-image records do not fit in shared memory");
  if (plan->aux_afree)
    return fail(LF_EUNSUPPORTED, "no gradient of the flux and time-delay terms with a sampled a_dis");
  return run(plan, theta, S, chi2, grad, stream);
}

extern "C" lf_status lf_chi2_img_batch(lf_plan* plan, const double* theta, int32_t S, int32_t iters,
                                       double* chi2_img, double* rms, void* stream) {
  if (!plan) return fail(LF_EINVAL, "plan is NULL");
  if (!theta || !chi2_img) return fail(LF_EINVAL, "theta and chi2_img are required");
  if (S < 1 || S > plan->max_samples) return fail(LF_EINVAL, "S must be in 1..%d", plan->max_samples);
  if (S % plan->n_clusters) return fail(LF_EINVAL, "S must be a multiple of the number of clusters");
  if (iters < 1 || iters > 64) return fail(LF_EINVAL, "iters must be in 1..64");
  if (plan->smem_img == 0) return fail(LF_EUNSUPPORTED, "the image-plane Newton state does not fit in shared memory");
  cudaStream_t st = (cudaStream_t)stream;
  const int spc = S / plan->n_clusters;
  LF_CUDA(cudaMemsetAsync(plan->d_counter, 0, sizeof(int), st));
  if (plan->precision == LF_MIXED) launch_img<LF_MIXED>(plan, theta, S, iters, chi2_img, rms, st, spc);
  else if (plan->precision == LF_FF) launch_img<LF_FF>(plan, theta, S, iters, chi2_img, rms, st, spc);
  else launch_img<LF_FP64>(plan, theta, S, iters, chi2_img, rms, st, spc);
  LF_CUDA(cudaGetLastError());
  return LF_OK;
}

extern "C" lf_status lf_plan_info(const lf_plan* plan, int32_t* kslices, int32_t* block, int32_t* graph) {
  if (!plan) return fail(LF_EINVAL, "plan is NULL");
  if (kslices) *kslices = plan->desc.empty() ? 0 : plan->desc[0].ks;
  if (block) *block = plan->block;
  if (graph) *graph = (plan->flags & 1) ? 1 : 0;
  return LF_OK;
}
