// Plane evaluation loops shared by the map, trace and chi^2 kernels.
//
// A plane's components are indexed 0..nc-1 (explicit components) then nc..nc+nm-1
// (members).  accumulate_mixed sums the index range [k0, k1) for PPT positions: explicit
// components go straight into float-float accumulators, members are summed in FP32
// over `chunk` consecutive members and each chunk sum is folded into the float-float
// accumulators (FP32 accumulation per component block, extended precision across blocks).
#pragma once
#include "lf_common.cuh"

namespace lf {

// Shared memory of the map and trace kernels: mbarrier (16 B), the float-float atan / atanh
// tables (2 x LF_TAB_N float2), then the staged planes.
constexpr uint32_t LF_MAP_BASE = 16u + 2u * LF_TAB_N * 8u;

// Shared-memory layout of a staged plane (host and device agree on it).
struct PlaneLayout {
  uint32_t rawc, rawm, dc, dm, total;
};

// Number of digested member records: one per member, or one per pair of members.
template <class M> __host__ __device__ inline uint32_t mem_records(int nm) { return (uint32_t)nm; }
template <> __host__ __device__ inline uint32_t mem_records<MemPair>(int nm) {
  return (uint32_t)(nm + 1) / 2u;
}

template <class T, class M = MemT<T>>
__host__ __device__ inline PlaneLayout plane_layout(int nc, int nm, uint32_t base) {
  PlaneLayout L;
  uint32_t o = (base + 15u) & ~15u;
  L.rawc = o; o += (uint32_t)nc * 64u;
  L.rawm = o; o += (uint32_t)nm * 32u;
  o = (o + 15u) & ~15u;
  L.dc = o; o += (uint32_t)nc * (uint32_t)sizeof(CompT<T>);
  o = (o + 15u) & ~15u;
  L.dm = o; o += mem_records<M>(nm) * (uint32_t)sizeof(M);
  L.total = (o + 15u) & ~15u;
  return L;
}

// Validates and digests one raw component (device side; invalid -> kind 0 + error bit).
template <class T>
__device__ inline void digest_one_comp(const lf_comp& r, CompT<T>& out) {
  bool ok = r.kind >= 1 && r.kind <= 6 && isfinite(r.x) && isfinite(r.y) && isfinite(r.b) &&
            isfinite(r.pa);
  if (r.kind == LF_SIE || r.kind == LF_DPIE)
    ok = ok && r.eps >= 0.0 && r.eps < 1.0 && r.core >= 0.0 && isfinite(r.core);
  if (r.kind == LF_DPIE) ok = ok && isfinite(r.cut) && r.cut > r.core;
  if (r.kind == LF_NFW) ok = ok && r.core > 0.0 && isfinite(r.core);
  if (r.kind == LF_ENFW)
    ok = ok && r.core > 0.0 && isfinite(r.core) && r.eps >= 0.0 && r.eps < 1.0;
  digest_comp<T>(ok ? r.kind : 0, r.x, r.y, r.b, r.eps, r.pa, r.core, r.cut, out);
  if (!ok) lf_flag_error(LF_DEVERR_BADCOMP);
}

// Member strength, core and cut from the scaling relations (Eq. scaling), FP64.
__device__ inline void member_fields(const lf_scaling& sc, double log_l, double& b, double& s,
                                     double& a, double& ll) {
  ll = log_l * 2.302585092994045684;
  b = sc.b_star * exp(2.0 * sc.lam * ll);
  s = sc.core_star * exp(sc.beta * ll);
  a = sc.cut_star * exp(sc.alpha * ll);
}

// Digests a staged plane (raw tables already in shared memory), whole block.
template <class T>
__device__ void digest_plane(const lf_comp* rawc, int nc, const lf_member* rawm, int nm,
                             const lf_scaling& sc, CompT<T>* dc, MemT<T>* dm) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) digest_one_comp<T>(rawc[i], dc[i]);
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    double b, s, a, ll;
    member_fields(sc, rawm[i].log_l, b, s, a, ll);
    digest_member<T>(rawm[i].x, rawm[i].y, b, s, a, ll, dm[i]);
  }
}

__device__ inline void digest_plane_x(const lf_comp* rawc, int nc, const lf_member* rawm, int nm,
                                      const lf_scaling& sc, CompT<float>* dc, MemX* dm) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) digest_one_comp<float>(rawc[i], dc[i]);
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    double b, s, a, ll;
    member_fields(sc, rawm[i].log_l, b, s, a, ll);
    digest_member_x(rawm[i].x, rawm[i].y, b, s, a, ll, dm[i]);
  }
}

// Digests a staged plane into explicit components and packed member pairs, whole block.
__device__ inline void digest_plane_pairs(const lf_comp* rawc, int nc, const lf_member* rawm,
                                          int nm, const lf_scaling& sc, CompT<float>* dc,
                                          MemPair* dp) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) digest_one_comp<float>(rawc[i], dc[i]);
  const int n2 = 2 * (int)mem_records<MemPair>(nm);
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    if (i < nm) {
      double b, s, a, ll;
      member_fields(sc, rawm[i].log_l, b, s, a, ll);
      digest_member_lane(rawm[i].x, rawm[i].y, b, s, a, dp[i >> 1], i & 1);
    } else {
      digest_pad_lane(dp[i >> 1], i & 1);
    }
  }
}

// LF_MIXED members in packed pairs (f32x2), two members per instruction: [k0, k1) counts member
// pairs, `chunk` pairs per FP32 partial sum, each folded into the float-float accumulators.  The
// offsets leave out the position's low word x_l (member_pair_acc); its first-order effect on the
// members' deflection, Psi x_l, is added at the end from the members' own psi sums (the second
// order, x_l^2 / 2 times the derivative of psi, stays below 1e-11 arcsec at |x_l| <= 5e-6").
template <int PPT>
__device__ __forceinline__ void accumulate_packed(const MemPair* dp, int nm, int k0, int k1, int chunk,
                                                  const float* pxh, const float* pxl,
                                                  const float* pyh, const float* pyl,
                                                  ff (&acc)[5][PPT]) {
  float2 qxh[PPT], qyh[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    qxh[k] = make_float2(pxh[k], pxh[k]);
    qyh[k] = make_float2(pyh[k], pyh[k]);
  }
  ff m5[5][PPT];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int k = 0; k < PPT; ++k) m5[v][k] = ff_zero();
  const int np = (int)mem_records<MemPair>(nm);
  const int j_beg = k0, j_end = min(k1, np);
  for (int j0 = j_beg; j0 < j_end; j0 += chunk) {
    const int j1 = min(j0 + chunk, j_end);
    float2 cs[PPT][6];
#pragma unroll
    for (int k = 0; k < PPT; ++k)
#pragma unroll
      for (int v = 0; v < 6; ++v) cs[k][v] = make_float2(0.f, 0.f);
#if LF_MAP_UNROLL == 2
#pragma unroll 2
#endif
    for (int j = j0; j < j1; ++j) {
      const MemPair M = dp[j];
#pragma unroll
      for (int k = 0; k < PPT; ++k) member_pair_acc(M, qxh[k], qyh[k], cs[k]);
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const float kb = cs[k][2].x + cs[k][2].y, txx = cs[k][3].x + cs[k][3].y;
      const float trr = cs[k][5].x + cs[k][5].y;
      ff_acc(m5[0][k], cs[k][0].x + cs[k][0].y);
      ff_acc(m5[1][k], cs[k][1].x + cs[k][1].y);
      ff_acc(m5[2][k], kb + txx);
      ff_acc(m5[3][k], kb + (trr - txx));
      ff_acc(m5[4][k], cs[k][4].x + cs[k][4].y);
    }
  }
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    ff_acc(m5[0][k], fmaf(m5[2][k].hi, pxl[k], m5[4][k].hi * pyl[k]));
    ff_acc(m5[1][k], fmaf(m5[4][k].hi, pxl[k], m5[3][k].hi * pyl[k]));
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v][k] = ff_add(acc[v][k], m5[v][k]);
  }
}

// Writes one member (FP32 fields: float-float centre, strength b, core s, cut a) into lane
// `lane` of a packed pair record, with the same derived constants as the scalar record.
__device__ __forceinline__ void pair_lane(MemPair& p, int lane, float xh, float xl, float yh, float yl,
                                          float b, float s, float a) {
  float* f = reinterpret_cast<float*>(&p) + lane;     // field k of the lane at f[2 k]
  f[0] = -xh; f[2] = -xl; f[4] = -yh; f[6] = -yl;
  f[8] = s * s; f[10] = a * a; f[12] = s; f[14] = a;
  f[16] = a + s; f[18] = b * (a - s); f[20] = b; f[22] = 0.f;
}

// Rewrites lane `lane`'s strength, core and cut fields (with the derived constants) of a packed
// pair record, keeping its centre.
__device__ __forceinline__ void pair_lane_scale(MemPair& p, int lane, float b, float s, float a) {
  float* f = reinterpret_cast<float*>(&p) + lane;
  f[8] = s * s; f[10] = a * a; f[12] = s; f[14] = a;
  f[16] = a + s; f[18] = b * (a - s); f[20] = b;
}

// Float-float tier: every deflection in float-float, accumulated in float-float.
template <int PPT>
__device__ __forceinline__ void accumulate_ext(const CompT<float>* dc, int nc, const MemX* dm,
                                               int nm, int k0, int k1, const float* pxh,
                                               const float* pxl, const float* pyh,
                                               const float* pyl, const float2* tab,
                                               ff (&acc)[5][PPT]) {
  const int c1 = min(k1, nc);
  for (int c = k0; c < c1; ++c) {
    const CompT<float>& C = dc[c];
    if (C.kind == 0) continue;
    for (int k = 0; k < PPT; ++k) {
      ff ax, ay;
      Out5<float> o;
      eval_comp_ext(C, pxh[k], pxl[k], pyh[k], pyl[k], tab, ax, ay, o);
      acc[0][k] = ff_add(acc[0][k], ax);
      acc[1][k] = ff_add(acc[1][k], ay);
      ff_acc(acc[2][k], o.pxx); ff_acc(acc[3][k], o.pyy); ff_acc(acc[4][k], o.pxy);
    }
  }
  const int m_beg = max(k0, nc) - nc, m_end = min(k1, nc + nm) - nc;
  for (int m = m_beg; m < m_end; ++m) {
    const MemX M = dm[m];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      ff ax, ay;
      Out5<float> o;
      eval_member_x(M, pxh[k], pxl[k], pyh[k], pyl[k], ax, ay, o);
      acc[0][k] = ff_add(acc[0][k], ax);
      acc[1][k] = ff_add(acc[1][k], ay);
      ff_acc(acc[2][k], o.pxx); ff_acc(acc[3][k], o.pyy); ff_acc(acc[4][k], o.pxy);
    }
  }
}

template <int PPT>
__device__ __forceinline__ void accumulate_mixed(const CompT<float>* dc, int nc,
                                                 const MemT<float>* dm, int nm, int k0, int k1,
                                                 int chunk, const float* pxh, const float* pxl,
                                                 const float* pyh, const float* pyl,
                                                 const float2* tab, ff (&acc)[5][PPT]) {
  const int c1 = min(k1, nc);
  for (int c = k0; c < c1; ++c) {
    const CompT<float>& C = dc[c];
    if (C.kind == 0) continue;
    for (int k = 0; k < PPT; ++k) {
      if (C.kind == K_NFW) {
        // the spherical NFW is all FP32 (the same operations as eval_comp_mixed's): inline,
        // so that planes with many of them make no out-of-line call per component
        Out5<float> o;
        nfw_sph(offset_of(pxh[k], pxl[k], C.xh, C.xl), offset_of(pyh[k], pyl[k], C.yh, C.yl), C.b,
                C.irs, o);
        acc[0][k] = ff_add(acc[0][k], ff_make(o.ax, 0.f));
        acc[1][k] = ff_add(acc[1][k], ff_make(o.ay, 0.f));
        ff_acc(acc[2][k], o.pxx); ff_acc(acc[3][k], o.pyy); ff_acc(acc[4][k], o.pxy);
        continue;
      }
      ff ax, ay;
      Out5<float> o;
      eval_comp_mixed(C, pxh[k], pxl[k], pyh[k], pyl[k], tab, ax, ay, o);
      acc[0][k] = ff_add(acc[0][k], ax);
      acc[1][k] = ff_add(acc[1][k], ay);
      ff_acc(acc[2][k], o.pxx); ff_acc(acc[3][k], o.pyy); ff_acc(acc[4][k], o.pxy);
    }
  }
  const int m_beg = max(k0, nc) - nc, m_end = min(k1, nc + nm) - nc;
  // all PPT positions on one row (the usual case on grids): one y offset per member
  bool same_y = true;
#pragma unroll
  for (int k = 1; k < PPT; ++k) same_y = same_y && pyh[k] == pyh[0] && pyl[k] == pyl[0];
  for (int m0 = m_beg; m0 < m_end; m0 += chunk) {
    const int m1 = min(m0 + chunk, m_end);
    float cs[5][PPT];
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int k = 0; k < PPT; ++k) cs[v][k] = 0.f;
    if (same_y) {
      for (int m = m0; m < m1; ++m) {
        const MemT<float> M = dm[m];
        const float dy = offset_of(pyh[0], pyl[0], M.yh, M.yl);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          float dx = offset_of(pxh[k], pxl[k], M.xh, M.xl);
          Out5<float> o;
          eval_member(M, dx, dy, o);
          cs[0][k] += o.ax; cs[1][k] += o.ay;
          cs[2][k] += o.pxx; cs[3][k] += o.pyy; cs[4][k] += o.pxy;
        }
      }
    } else {
      for (int m = m0; m < m1; ++m) {
        const MemT<float> M = dm[m];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          float dx = offset_of(pxh[k], pxl[k], M.xh, M.xl);
          float dy = offset_of(pyh[k], pyl[k], M.yh, M.yl);
          Out5<float> o;
          eval_member(M, dx, dy, o);
          cs[0][k] += o.ax; cs[1][k] += o.ay;
          cs[2][k] += o.pxx; cs[3][k] += o.pyy; cs[4][k] += o.pxy;
        }
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int k = 0; k < PPT; ++k) ff_acc(acc[v][k], cs[v][k]);
  }
}

// The gradient's forward sums of the mixed tier: each member adds its change from the plan's
// base fields (eval_member_anchored) to alpha, and the caller adds the base sum of every
// image's members, taken once per plan in FP64; psi_ij is the sample's.  The explicit
// components take the float-float tier's forms (eval_comp_ext: float-float deflections for
// the round profiles and the spherical NFW as well), since the adjoint's cotangents need
// every deflection beyond FP32.
template <int PPT>
__device__ __forceinline__ void accumulate_anchored(const CompT<float>* dc, int nc,
                                                    const MemT<float>* dm, const MemA* da, int nm,
                                                    int k0, int k1, int chunk, const float* pxh,
                                                    const float* pxl, const float* pyh,
                                                    const float* pyl, const float2* tab,
                                                    ff (&acc)[5][PPT]) {
  const int c1 = min(k1, nc);
  for (int c = k0; c < c1; ++c) {
    const CompT<float>& C = dc[c];
    if (C.kind == 0) continue;
    for (int k = 0; k < PPT; ++k) {
      ff ax, ay;
      Out5<float> o;
      eval_comp_ext(C, pxh[k], pxl[k], pyh[k], pyl[k], tab, ax, ay, o);
      acc[0][k] = ff_add(acc[0][k], ax);
      acc[1][k] = ff_add(acc[1][k], ay);
      ff_acc(acc[2][k], o.pxx); ff_acc(acc[3][k], o.pyy); ff_acc(acc[4][k], o.pxy);
    }
  }
  const int m_beg = max(k0, nc) - nc, m_end = min(k1, nc + nm) - nc;
  for (int m0 = m_beg; m0 < m_end; m0 += chunk) {
    const int m1 = min(m0 + chunk, m_end);
    float cs[5][PPT];
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int k = 0; k < PPT; ++k) cs[v][k] = 0.f;
    for (int m = m0; m < m1; ++m) {
      const MemT<float> M = dm[m];
      const MemA D = da[m];
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const float dx = offset_of(pxh[k], pxl[k], M.xh, M.xl);
        const float dy = offset_of(pyh[k], pyl[k], M.yh, M.yl);
        Out5<float> o;
        eval_member_anchored(M, D, dx, dy, o);
        cs[0][k] += o.ax; cs[1][k] += o.ay;
        cs[2][k] += o.pxx; cs[3][k] += o.pyy; cs[4][k] += o.pxy;
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int k = 0; k < PPT; ++k) ff_acc(acc[v][k], cs[v][k]);
  }
}

// FP64 version for one position: plain sum.
__device__ __forceinline__ void accumulate_fp64(const CompT<double>* dc, int nc,
                                                const MemT<double>* dm, int nm, int k0, int k1,
                                                double x, double y, double (&acc)[5]) {
  const int c1 = min(k1, nc);
  for (int c = k0; c < c1; ++c) {
    const CompT<double>& C = dc[c];
    if (C.kind == 0) continue;
    Out5<double> o;
    eval_comp(C, x - C.xh, y - C.yh, o);
    acc[0] += o.ax; acc[1] += o.ay; acc[2] += o.pxx; acc[3] += o.pyy; acc[4] += o.pxy;
  }
  const int m_beg = max(k0, nc) - nc, m_end = min(k1, nc + nm) - nc;
  for (int m = m_beg; m < m_end; ++m) {
    const MemT<double>& M = dm[m];
    Out5<double> o;
    eval_member(M, x - M.xh, y - M.yh, o);
    acc[0] += o.ax; acc[1] += o.ay; acc[2] += o.pxx; acc[3] += o.pyy; acc[4] += o.pxy;
  }
}

}  // namespace lf
