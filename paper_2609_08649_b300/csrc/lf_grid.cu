// Grid / point maps of alpha, kappa, gamma and mu (Sec. 2.1; Eq. lens_eq, Eq. jac).
//
// Persistent kernels: one block per SM slot stages the component and member tables
// into shared memory once with the bulk-copy engine, digests them (member scaling
// relations of Eq. scaling, trigonometry, float-float centres), then walks tiles of
// positions with a grid stride.
//
//  LF_MIXED: tiles of 16 x 16 pixels (or 256 points) anchored at their centre: each member's
//            deflection there in float-float and its change across the tile in FP32 (below);
//            FP64 det A and mu.
//  LF_FF:    every deflection in float-float at every position, psi_ij in FP32.
//  LF_FP64:  the same closed forms in FP64 throughout, one position per thread.
#include "lf_internal.h"
#include "lf_eval.cuh"

namespace lf {

struct PosArgs {
  const double* pts;  // n x 2, or null for a grid
  double x0, y0, dx, dy;
  int nx;
  long long n;
};

struct OutArgs {
  double *ax, *ay, *mu;
  float *kappa, *g1, *g2;
  double a_dis;
};

__device__ __forceinline__ void position_of(const PosArgs& P, long long p, double& x, double& y) {
  if (P.pts) {
    x = P.pts[2 * p];
    y = P.pts[2 * p + 1];
  } else {
    long long j = p / P.nx;
    long long i = p - j * P.nx;
    x = P.x0 + (double)i * P.dx;
    y = P.y0 + (double)j * P.dy;
  }
}

// write_out from float-float sums, with kappa, gamma, det A and mu = 1/det A in float-float on
// the FP32 pipe (det A to ~1e-14 absolute) and only the FP64 stores' conversions on the FP64
// pipe, which runs FP64 arithmetic at 1/64 of the FP32 rate on this part.
__device__ __forceinline__ void write_out_ff(const OutArgs& O, const ff& a_dis, long long p, const ff& ax,
                                            const ff& ay, const ff& pxx, const ff& pyy, const ff& pxy) {
  if (O.ax) O.ax[p] = ff_to_double(ax);
  if (O.ay) O.ay[p] = ff_to_double(ay);
  // (the accumulators' low words may exceed half an ulp of the high ones: renormalise)
  const ff kappa = ff_mul_f(ff_add(pxx, pyy), 0.5f), g1 = ff_mul_f(ff_sub(pxx, pyy), 0.5f);
  const ff g2 = fast_two_sum(pxy.hi, pxy.lo);
  if (O.kappa) O.kappa[p] = kappa.hi;
  if (O.g1) O.g1[p] = g1.hi;
  if (O.g2) O.g2[p] = g2.hi;
  if (O.mu) {
    const ff t = ff_add_f(ff_neg(ff_mul(a_dis, kappa)), 1.0f);
    const ff det = ff_sub(ff_sqr(t), ff_mul(ff_sqr(a_dis), ff_add(ff_sqr(g1), ff_sqr(g2))));
    O.mu[p] = ff_to_double(ff_div(ff_make(1.f, 0.f), det));
  }
}

__device__ __forceinline__ void write_out(const OutArgs& O, long long p, double ax, double ay,
                                          double pxx, double pyy, double pxy) {
  if (O.ax) O.ax[p] = ax;
  if (O.ay) O.ay[p] = ay;
  double kappa = 0.5 * (pxx + pyy), g1 = 0.5 * (pxx - pyy), g2 = pxy;
  if (O.kappa) O.kappa[p] = (float)kappa;
  if (O.g1) O.g1[p] = (float)g1;
  if (O.g2) O.g2[p] = (float)g2;
  if (O.mu) {
    double a = O.a_dis;
    double t = 1.0 - a * kappa;
    double det = t * t - a * a * (g1 * g1 + g2 * g2);
    O.mu[p] = 1.0 / det;
  }
}

// --------------------------------------------------------------------- LF_FF -------
#ifndef LF_MAP_MINB
#define LF_MAP_MINB 3   // at most 85 registers, 3 blocks of 256
#endif
#ifndef LF_MAP_CHUNK
#define LF_MAP_CHUNK 16   // anchored maps: member pairs per FP32 partial sum (16 terms per lane)
#endif

// The float-float tier's maps: every component's deflection in float-float at every position.
__global__ void __launch_bounds__(256, LF_MAP_MINB) k_map_ff(const lf_comp* __restrict__ comp, int nc,
                                                             const lf_member* __restrict__ mem, int nm,
                                                             lf_scaling sc, PosArgs P, OutArgs O) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  const PlaneLayout L = plane_layout<float, MemX>(nc, nm, LF_MAP_BASE);
  lf_comp* rawc = reinterpret_cast<lf_comp*>(smem + L.rawc);
  lf_member* rawm = reinterpret_cast<lf_member*>(smem + L.rawm);
  CompT<float>* dc = reinterpret_cast<CompT<float>*>(smem + L.dc);
  MemX* dm = reinterpret_cast<MemX*>(smem + L.dm);
  float2* tab = reinterpret_cast<float2*>(smem + 16);
  if (!LF_CHECK(L.total <= lf_dyn_smem())) return;
  if (threadIdx.x == 0) mbar_init(bar, 1);
  init_ff_tables(tab);
  __syncthreads();
  bool ok = stage_to_smem(rawc, comp, (uint32_t)nc * 64u, bar, 0);
  if (ok) ok = stage_to_smem(rawm, mem, (uint32_t)nm * 32u, bar, nc > 0 ? 1 : 0);
  if (!ok) return;
  digest_plane_x(rawc, nc, rawm, nm, sc, dc, dm);
  __syncthreads();

  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P.n;
       p += (long long)gridDim.x * blockDim.x) {
    float pxh[1], pxl[1], pyh[1], pyl[1];
    double x, y;
    position_of(P, p, x, y);
    split_ff(x, pxh[0], pxl[0]);
    split_ff(y, pyh[0], pyl[0]);
    ff acc[5][1];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v][0] = ff_zero();
    accumulate_ext<1>(dc, nc, dm, nm, 0, nc + nm, pxh, pxl, pyh, pyl, tab, acc);
    write_out(O, p, ff_to_double(acc[0][0]), ff_to_double(acc[1][0]), ff_to_double(acc[2][0]),
              ff_to_double(acc[3][0]), ff_to_double(acc[4][0]));
  }
}

// ---------------------------------------------------- LF_MIXED: anchored tiles ------
// The LF_MIXED maps.  A block owns a tile of positions (16 x 16 pixels of a grid, or 256
// consecutive points of a list) and an anchor theta0 at the tile's centre.  Each member's
// deflection at theta0 is evaluated once per tile in float-float; at each position only the
// change alpha_k(theta) - alpha_k(theta0) is evaluated in FP32, from exact differences:
// with d0 = theta0 - c, e = theta - theta0 and u = |d0 + e|^2,
//   du = u - u0 = 2 d0.e + |e|^2,   S - S0 = du / (S + S0)   (S = sqrt(s^2 + u)),
//   1/(S + s) - 1/(S0 + s) = -du / ((S + S0)(S + s)(S0 + s)),  likewise for R = sqrt(a^2 + u),
//   kbar = b [1/(S + s) - 1/(R + a)],  alpha_k(theta) - alpha_k(theta0) = dkbar d0 + kbar e.
// No term cancels, so the FP32 rounding scales with the change (about 3 kbar(theta0) h over a
// tile of half-diagonal h) instead of with |alpha_k|: on the cluster field at 0.04" pixels this
// cuts the deflection error from ~1e-6" rms to ~2e-8".  Members whose change across the tile
// is not small (3 kbar(theta0) h > T, or closer to theta0 than 2 h) are evaluated per position
// in float-float instead.  The elliptical isothermal components (SIE, dPIE) are anchored the
// same way (sie_anchor_delta: their deflection at theta0 in float-float, its change by exact
// differences of the atan / atanh arguments in FP32); every other explicit component is
// evaluated in float-float at each position.  psi_ij is FP32 as in the other mixed kernels.
// T = LF_ANCHOR_T min(1, LF_ANCHOR_H0 / h): coarse tiles send more members to the float-float
// path, so the precision does not depend on the pixel scale.
// Each thread evaluates LF_AMAP_PPT positions of its tile (256 / LF_AMAP_PPT threads per
// block): the positions share every member record load and run as independent chains.
#ifndef LF_AMAP_PPT
#define LF_AMAP_PPT 2
#endif
constexpr int LF_AMAP_THREADS = 256 / LF_AMAP_PPT;
// Two positions: 128 registers, 4 blocks of 128 per SM (8.87 ms per 4096^2 cluster map with the
// per-position tail unrolled; 9.34 ms at 5 blocks, 9.65 ms at 6, and 9.09 ms for one position per
// thread at 3 blocks of 256).
#ifndef LF_ANCHOR_MINB
#define LF_ANCHOR_MINB (LF_AMAP_PPT == 1 ? 3 : 4)
#endif
#ifndef LF_ANCHOR_T
#define LF_ANCHOR_T 0.3f
#endif
#ifndef LF_ANCHOR_H0
#define LF_ANCHOR_H0 0.5f
#endif
#ifndef LF_ANCHOR_HALO
#define LF_ANCHOR_HALO 2.0f   // arcsec: bound on an anchored isothermal component's change across a tile
#endif
constexpr int LF_ATILE = 16;   // anchored grid tile: 16 x 16 pixels (one per thread of a 256-thread block)

// Two members per record at one tile's anchor (lane x: member 2j, lane y: member 2j + 1).
struct __align__(16) AnchorPair {
  float2 dx0, dy0;   // theta0 - c, rounded to FP32
  float2 S20, R20;   // s^2 + u0, a^2 + u0, u0 = |d0|^2
  float2 S0s, R0a;   // S0 s, R0 a
  float2 cs, ca;     // S0 + s, R0 + a
  float2 P0, Q0;     // 1 / (S0 + s), 1 / (R0 + a)
  float2 b, kb0;     // strength (0 for a member evaluated per position), kbar(theta0)
};

__device__ __forceinline__ void anchor_pad_lane(AnchorPair& p, int lane) {
  float* f = reinterpret_cast<float*>(&p) + lane;   // field k of the lane at f[2 k]
  f[0] = 0.f; f[2] = 0.f; f[4] = 1.f; f[6] = 1.f; f[8] = 0.f; f[10] = 0.f;
  f[12] = 1.f; f[14] = 1.f; f[16] = 0.f; f[18] = 0.f; f[20] = 0.f; f[22] = 0.f;
}

// The change of both members' alpha and their psi_ij at one position (offset e from the
// anchor; e2 = 2 e, ee = |e|^2, all duplicated into both halves), added into packed chunk
// sums: c[0], c[1] += change of alpha_x, alpha_y; c[2] += kbar; c[3] += t dx^2;
// c[4] += t dx dy; c[5] += t dy^2 (psi_ij = kbar delta_ij + t x_i x_j, t = b (Q^2/R - P^2/S)).
// 36 FP32 lane-operations and 4 MUFU per member.
__device__ __forceinline__ void anchor_pair_acc(const AnchorPair& m, float2 e2x, float2 e2y, float2 ee,
                                                float2 ex, float2 ey, float2 (&c)[6]) {
  const float2 du = fma2(m.dx0, e2x, fma2(m.dy0, e2y, ee));
  const float2 S2 = add2(m.S20, du), R2 = add2(m.R20, du);
  float2 iS, iR, S, R;
  iS.x = rsqrtf(S2.x); iS.y = rsqrtf(S2.y);
  iR.x = rsqrtf(R2.x); iR.y = rsqrtf(R2.y);
  S.x = S2.x * iS.x; S.y = S2.y * iS.y;
  R.x = R2.x * iR.x; R.y = R2.y * iR.y;
  // (S + S0)(S + s)(S0 + s) = (S^2 + S0 s + S (S0 + s)) (S0 + s), likewise for R
  const float2 As = mul2(fma2(S, m.cs, add2(S2, m.S0s)), m.cs);
  const float2 Aa = mul2(fma2(R, m.ca, add2(R2, m.R0a)), m.ca);
  float2 gS, gA;     // the decrease of 1/(S + s) and of 1/(R + a) from the anchor
  gS.x = du.x * __fdividef(1.f, As.x); gS.y = du.y * __fdividef(1.f, As.y);
  gA.x = du.x * __fdividef(1.f, Aa.x); gA.y = du.y * __fdividef(1.f, Aa.y);
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 P = fma2(gS, m1, m.P0), Q = fma2(gA, m1, m.Q0);
  const float2 dk = mul2(m.b, fma2(gS, m1, gA));
  const float2 kb = add2(m.kb0, dk);
  c[0] = fma2(kb, ex, fma2(dk, m.dx0, c[0]));
  c[1] = fma2(kb, ey, fma2(dk, m.dy0, c[1]));
  const float2 P2 = mul2(P, P), Q2 = mul2(Q, Q);
  float2 tt;
  tt.x = fmaf(-P2.x, iS.x, Q2.x * iR.x); tt.y = fmaf(-P2.y, iS.y, Q2.y * iR.y);
  const float2 t = mul2(m.b, tt);
  const float2 dx = add2(m.dx0, ex), dy = add2(m.dy0, ey);
  c[2] = add2(c[2], kb);
  const float2 tdx = mul2(t, dx), tdy = mul2(t, dy);
  c[3] = fma2(tdx, dx, c[3]);
  c[4] = fma2(tdx, dy, c[4]);
  c[5] = fma2(tdy, dy, c[5]);
}

// An elliptical isothermal component (SIE or dPIE) at one tile's anchor: its frame offsets
// u0, v0 and psi~ = sqrt(q^2 (r^2 + u^2) + v^2) there for the core and the cut radius, FP32;
// anchored = 0 for the kinds evaluated in float-float at every position instead.
struct __align__(16) AnchorComp {
  float u0, v0, ps0, pa0;
  int anchored, pad0, pad1, pad2;
};

// One isothermal ellipsoid of unit strength and radius r at (u, v) = (u0 + du, v0 + dv) in
// its frame: the change of its deflection from the anchor (u0, v0), and its psi_ij, in FP32.
// With dp2 = psi~^2 - psi0~^2 = q^2 du (2 u0 + du) + dv (2 v0 + dv) (cancellation-free) and
// psi~ - psi0~ = dp2 / (psi~ + psi0~), the changes of z1 = e u / (psi~ + r) and
// z2 = e v / (psi~ + q^2 r) enter through
//   atan(z1) - atan(z10) = atan(e (du (psi0~ + r) - u0 (psi~ - psi0~)) / ((psi~ + r)(psi0~ + r) + e^2 u u0)),
//   atanh(z2) - atanh(z20) = atanh(e (dv (psi0~ + q^2 r) - v0 (psi~ - psi0~))
//                                   / ((psi~ + q^2 r)(psi0~ + q^2 r) - e^2 v v0)),
// so the FP32 rounding scales with the change, not with the deflection.
__device__ __forceinline__ void sie_anchor_delta(float u0, float v0, float du, float dv, float dp2, float ps0,
                                                 float q, float q2, float e, float qe, float r, float r2,
                                                 float q2r, float D0, float& dau, float& dav, float& puu,
                                                 float& pvv, float& puv) {
  const float ps2 = fmaf(ps0, ps0, dp2);
  const float ips = rsqrtf(ps2), ps = ps2 * ips;
  const float dps = dp2 * __fdividef(1.f, ps + ps0);
  const float u = u0 + du, v = v0 + dv;
  const float A = ps0 + r, B = ps0 + q2r, ee = e * e;
  const float n1 = e * fmaf(du, A, -u0 * dps), d1 = fmaf(ps + r, A, ee * u * u0);
  const float t2 = e * fmaf(dv, B, -v0 * dps) * __fdividef(1.f, fmaf(ps + q2r, B, -ee * v * v0));
  // 1 + z1 z10 < 0 (|z1| > 1 on both sides of u = 0, possible for q^2 < 1/2): atan's branch
  // moves by pi, with the sign of z1 - z10 (that of n1)
  dau = qe * (atanf(n1 * __fdividef(1.f, d1)) + (d1 < 0.f ? copysignf(3.14159265358979f, n1) : 0.f));
  dav = qe * atanhf(t2);     // |z2|, |z20| < 1: 1 - z2 z20 > 0
  const float uu = u * u, vv = v * v;
  const float f = q * ips * __fdividef(1.f, D0 + 2.f * ps * r + uu + vv);
  const float sp = r * ps;
  puu = f * (fmaf(q2, r2, vv) + sp);
  pvv = f * (r2 + uu + sp);
  puv = -f * u * v;
}

// Shared memory of the anchored kernel (host and device agree on it).
struct AnchorLayout {
  uint32_t rawc, rawm, dc, dm, ap, ac, bits, red, total;
};
__host__ __device__ inline AnchorLayout anchor_layout(int nc, int nm) {
  AnchorLayout L;
  uint32_t o = (LF_MAP_BASE + 15u) & ~15u;
  L.rawc = o; o += (uint32_t)nc * 64u;
  L.rawm = o; o += (uint32_t)nm * 32u;
  o = (o + 15u) & ~15u;
  L.dc = o; o += (uint32_t)nc * (uint32_t)sizeof(CompT<float>);
  o = (o + 15u) & ~15u;
  L.dm = o; o += (uint32_t)nm * (uint32_t)sizeof(MemX);
  o = (o + 15u) & ~15u;
  L.ap = o; o += (uint32_t)((nm + 1) / 2) * (uint32_t)sizeof(AnchorPair);
  o = (o + 15u) & ~15u;
  L.ac = o; o += (uint32_t)nc * (uint32_t)sizeof(AnchorComp);
  o = (o + 15u) & ~15u;
  L.bits = o; o += (uint32_t)((nm + 31) / 32) * 4u;
  o = (o + 15u) & ~15u;
  L.red = o; o += 8u * 4u * 8u;      // 8 warps x 4 doubles
  L.total = (o + 15u) & ~15u;
  return L;
}

template <bool GRID>
__global__ void __launch_bounds__(LF_AMAP_THREADS, LF_ANCHOR_MINB) k_map_anchor(const lf_comp* __restrict__ comp, int nc,
                                                                  const lf_member* __restrict__ mem, int nm,
                                                                  lf_scaling sc, PosArgs P, OutArgs O, int chunk) {
  constexpr int NT = LF_AMAP_THREADS, PPT = LF_AMAP_PPT, NWARP = NT / 32;
  const ff a_ff = ff_from_double(O.a_dis);
  const ff dxf = ff_from_double(P.dx), dyf = ff_from_double(P.dy);
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  const AnchorLayout L = anchor_layout(nc, nm);
  lf_comp* rawc = reinterpret_cast<lf_comp*>(smem + L.rawc);
  lf_member* rawm = reinterpret_cast<lf_member*>(smem + L.rawm);
  CompT<float>* dc = reinterpret_cast<CompT<float>*>(smem + L.dc);
  MemX* dm = reinterpret_cast<MemX*>(smem + L.dm);
  AnchorPair* ap = reinterpret_cast<AnchorPair*>(smem + L.ap);
  AnchorComp* acp = reinterpret_cast<AnchorComp*>(smem + L.ac);
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem + L.bits);
  double* red = reinterpret_cast<double*>(smem + L.red);
  float2* tab = reinterpret_cast<float2*>(smem + 16);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (!LF_CHECK(L.total <= lf_dyn_smem() && blockDim.x == NT)) return;   // the host's layout
  if (tid == 0) mbar_init(bar, 1);
  init_ff_tables(tab);
  __syncthreads();
  bool ok = stage_to_smem(rawc, comp, (uint32_t)nc * 64u, bar, 0);
  if (ok) ok = stage_to_smem(rawm, mem, (uint32_t)nm * 32u, bar, nc > 0 ? 1 : 0);
  if (!ok) return;
  digest_plane_x(rawc, nc, rawm, nm, sc, dc, dm);
  __syncthreads();

  const int np = (nm + 1) / 2, nw = (nm + 31) / 32;
  const long long tiles_x = GRID ? (P.nx + LF_ATILE - 1) / LF_ATILE : 1;
  const long long ny = GRID ? P.n / P.nx : 0;
  const long long n_tiles = GRID ? tiles_x * ((ny + LF_ATILE - 1) / LF_ATILE) : (P.n + 255) / 256;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    // this thread's PPT positions (rows tid / 16 + 16 q / PPT of the tile, or points
    // tile * 256 + tid + NT q) and the tile's anchor (FP64)
    double x[PPT], y[PPT], cx, cy;
    float hf;     // the tile's half-diagonal: thresholds only, so FP32 (the FP64 pipe is slow)
    long long pid[PPT];
    bool valid[PPT];
    if constexpr (GRID) {
      const long long tx = tile % tiles_x, ty = tile / tiles_x;
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int t = tid + NT * q;
        const long long i = tx * LF_ATILE + (t & (LF_ATILE - 1)), j = ty * LF_ATILE + t / LF_ATILE;
        valid[q] = i < P.nx && j < ny;
        pid[q] = j * P.nx + i;
        x[q] = P.x0 + (double)i * P.dx;
        y[q] = P.y0 + (double)j * P.dy;
      }
      cx = P.x0 + ((double)(tx * LF_ATILE) + 0.5 * (LF_ATILE - 1)) * P.dx;
      cy = P.y0 + ((double)(ty * LF_ATILE) + 0.5 * (LF_ATILE - 1)) * P.dy;
      hf = 0.5f * (LF_ATILE - 1) * sqrtf((float)(P.dx * P.dx + P.dy * P.dy));
    } else {
      // the tile's bounding box (non-finite positions ignored)
      double b4[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        pid[q] = tile * 256 + tid + NT * q;
        valid[q] = pid[q] < P.n;
        x[q] = valid[q] ? P.pts[2 * pid[q]] : 0.0;
        y[q] = valid[q] ? P.pts[2 * pid[q] + 1] : 0.0;
        const bool fin = valid[q] && isfinite(x[q]) && isfinite(y[q]);
        if (fin) {
          b4[0] = fmin(b4[0], x[q]); b4[1] = fmin(b4[1], -x[q]);
          b4[2] = fmin(b4[2], y[q]); b4[3] = fmin(b4[3], -y[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        for (int off = 16; off > 0; off >>= 1) b4[q] = fmin(b4[q], __shfl_xor_sync(0xffffffffu, b4[q], off));
      if (lane == 0)
        for (int q = 0; q < 4; ++q) red[warp * 4 + q] = b4[q];
      __syncthreads();
      for (int q = 0; q < 4; ++q) {
        b4[q] = red[q];
        for (int w = 1; w < NWARP; ++w) b4[q] = fmin(b4[q], red[w * 4 + q]);
      }
      __syncthreads();
      if (!(b4[0] <= -b4[1])) { b4[0] = 0.0; b4[1] = 0.0; }     // no finite position in the tile
      if (!(b4[2] <= -b4[3])) { b4[2] = 0.0; b4[3] = 0.0; }
      cx = 0.5 * (b4[0] - b4[1]);
      cy = 0.5 * (b4[2] - b4[3]);
      hf = 0.5f * sqrtf((float)((b4[0] + b4[1]) * (b4[0] + b4[1]) + (b4[2] + b4[3]) * (b4[2] + b4[3])));
#pragma unroll
      for (int q = 0; q < PPT; ++q)
        if (!valid[q]) { x[q] = cx; y[q] = cy; }
    }
    float ahx, alx, ahy, aly;
    split_ff(cx, ahx, alx);
    split_ff(cy, ahy, aly);
    const float thr = LF_ANCHOR_T * fminf(1.f, LF_ANCHOR_H0 * __frcp_rn(fmaxf(hf, 1e-30f)));

    // ---- anchor pass: each member's record, its float-float deflection at theta0 (summed
    // over the block), and the members left to the per-position float-float path
    ff sax = ff_zero(), say = ff_zero();
    for (int k0 = 0; k0 < 2 * np; k0 += NT) {
      const int k = k0 + tid;
      bool near = false;
      if (k < 2 * np && LF_CHECK((uint32_t)(k >> 1) < (uint32_t)np)) {
        AnchorPair& rec = ap[k >> 1];
        float* f = reinterpret_cast<float*>(&rec) + (k & 1);
        if (k < nm) {
          const MemX& m = dm[k];
          const ff d0x = offset_ff(ahx, alx, m.xh, m.xl), d0y = offset_ff(ahy, aly, m.yh, m.yl);
          const float dx0 = d0x.hi, dy0 = d0y.hi;
          const float u0 = fmaf(dx0, dx0, dy0 * dy0);
          const float S20 = m.s2h + u0, R20 = m.a2h + u0;
          const float S0 = S20 * rsqrtf(S20), R0 = R20 * rsqrtf(R20);
          const float cs = S0 + m.sh, ca = R0 + m.ah;
          const float P0 = __fdividef(1.f, cs), Q0 = __fdividef(1.f, ca);
          const float kb0 = m.bdh * P0 * Q0 * fmaf(m.apch, __fdividef(1.f, R0 + S0), 1.f);
          near = (3.f * kb0 * hf > thr) || (u0 < 4.f * hf * hf);
          if (!near) {
            ff ax, ay;
            member_alpha_ff(m, d0x, d0y, ax, ay);
            sax = ff_add(sax, ax);
            say = ff_add(say, ay);
            f[0] = dx0; f[2] = dy0; f[4] = S20; f[6] = R20; f[8] = S0 * m.sh; f[10] = R0 * m.ah;
            f[12] = cs; f[14] = ca; f[16] = P0; f[18] = Q0; f[20] = m.b; f[22] = kb0;
          } else {
            anchor_pad_lane(rec, k & 1);
          }
        } else {
          anchor_pad_lane(rec, k & 1);   // the zero-strength partner of an odd member count
        }
      }
      const uint32_t word = __ballot_sync(0xffffffffu, near);
      const int wi = (k0 >> 5) + warp;
      if (lane == 0 && wi < nw && LF_CHECK(wi >= 0)) bits[wi] = word;
    }
    // elliptical isothermal components: frame offsets and psi~ at the anchor, and their
    // float-float deflection there (on the threads with the fewest member records)
    for (int c = NT - 1 - tid; c >= 0 && c < nc; c += NT) {
      const CompT<float>& C = dc[c];
      AnchorComp rec;
      const bool ell = (C.kind == K_SIE || C.kind == K_DPIE) && !C.round;
      rec.pad0 = rec.pad1 = rec.pad2 = 0;
      rec.u0 = rec.v0 = rec.ps0 = rec.pa0 = 0.f;
      if (ell) {
        const float dx0 = offset_ff(ahx, alx, C.xh, C.xl).hi, dy0 = offset_ff(ahy, aly, C.yh, C.yl).hi;
        rec.u0 = fmaf(C.c, dx0, C.sn * dy0);
        rec.v0 = fmaf(C.c, dy0, -C.sn * dx0);
        const float uu = rec.u0 * rec.u0, vv = rec.v0 * rec.v0;
        rec.ps0 = sqrtf(fmaf(C.q2, C.s1sq + uu, vv));
        rec.pa0 = C.kind == K_DPIE ? sqrtf(fmaf(C.q2, C.s2sq + uu, vv)) : 0.f;
      }
      // anchored when its deflection changes little across the tile: |psi_ij| <~ b / psi~ with
      // psi~ >= max(psi0~ - h, q s) over the tile, so the change is below b h / that
      rec.anchored = ell && hf <= LF_ANCHOR_H0 &&
                     C.b * hf <= LF_ANCHOR_HALO * fmaxf(rec.ps0 - hf, C.q * C.s1);
      if (rec.anchored) {
        ff ax, ay;
        Out5<float> o;
        eval_comp_mixed(C, ahx, alx, ahy, aly, tab, ax, ay, o);
        sax = ff_add(sax, ax);
        say = ff_add(say, ay);
      }
      acp[c] = rec;
    }
    for (int off = 16; off > 0; off >>= 1) {
      sax = ff_add(sax, ff_shfl_xor(sax, off));
      say = ff_add(say, ff_shfl_xor(say, off));
    }
    float* redf = reinterpret_cast<float*>(red);
    if (lane == 0) {
      redf[warp * 4 + 0] = sax.hi; redf[warp * 4 + 1] = sax.lo;
      redf[warp * 4 + 2] = say.hi; redf[warp * 4 + 3] = say.lo;
    }
    __syncthreads();
    sax = ff_make(redf[0], redf[1]);
    say = ff_make(redf[2], redf[3]);
    for (int w = 1; w < NWARP; ++w) {
      sax = ff_add(sax, ff_make(redf[w * 4 + 0], redf[w * 4 + 1]));
      say = ff_add(say, ff_make(redf[w * 4 + 2], redf[w * 4 + 3]));
    }

    // ---- per position: the anchored members' changes (the PPT positions share each record
    // load and run as independent chains), then the float-float terms
    float exl[PPT], eyl[PPT], exf[PPT], eyf[PPT];
    float2 e2x[PPT], e2y[PPT], ee[PPT], ex2[PPT], ey2[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      float ex, ey;
      if constexpr (GRID) {
        // the offset from the anchor is (l - 7.5) times the pixel size for the l-th pixel of the
        // tile's row (column): one float-float product on the FP32 pipe
        const int t = tid + NT * q;
        const ff gx = ff_mul_f(dxf, (float)(t & (LF_ATILE - 1)) - 0.5f * (LF_ATILE - 1));
        const ff gy = ff_mul_f(dyf, (float)(t / LF_ATILE) - 0.5f * (LF_ATILE - 1));
        ex = gx.hi; ey = gy.hi;
        exl[q] = gx.lo; eyl[q] = gy.lo;
      } else {
        const double exd = x[q] - cx, eyd = y[q] - cy;
        ex = (float)exd; ey = (float)eyd;
        exl[q] = (float)(exd - (double)ex); eyl[q] = (float)(eyd - (double)ey);
      }
      exf[q] = ex; eyf[q] = ey;
      e2x[q] = make_float2(2.f * ex, 2.f * ex); e2y[q] = make_float2(2.f * ey, 2.f * ey);
      ee[q] = make_float2(fmaf(ex, ex, ey * ey), fmaf(ex, ex, ey * ey));
      ex2[q] = make_float2(ex, ex); ey2[q] = make_float2(ey, ey);
    }
    ff acc[PPT][5];
#pragma unroll
    for (int q = 0; q < PPT; ++q)
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[q][v] = ff_zero();
    for (int j0 = 0; j0 < np; j0 += chunk) {
      const int j1 = min(j0 + chunk, np);
      float2 c6[PPT][6];
#pragma unroll
      for (int q = 0; q < PPT; ++q)
#pragma unroll
        for (int v = 0; v < 6; ++v) c6[q][v] = make_float2(0.f, 0.f);
#if LF_AMAP_PPT == 1
#pragma unroll 2
#endif
      for (int j = j0; j < j1; ++j) {
        const AnchorPair M = ap[j];
#pragma unroll
        for (int q = 0; q < PPT; ++q) anchor_pair_acc(M, e2x[q], e2y[q], ee[q], ex2[q], ey2[q], c6[q]);
      }
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const float kb = c6[q][2].x + c6[q][2].y;
        ff_acc(acc[q][0], c6[q][0].x + c6[q][0].y);
        ff_acc(acc[q][1], c6[q][1].x + c6[q][1].y);
        ff_acc(acc[q][2], kb + (c6[q][3].x + c6[q][3].y));
        ff_acc(acc[q][3], kb + (c6[q][5].x + c6[q][5].y));
        ff_acc(acc[q][4], c6[q][4].x + c6[q][4].y);
      }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const float ex = exf[q], ey = eyf[q];
      ff* a5 = acc[q];
      // the anchored explicit components: their change from the anchor and their psi_ij
      for (int c = 0; c < nc; ++c) {
        const AnchorComp R = acp[c];
        if (!R.anchored) continue;
        const CompT<float>& C = dc[c];
        const float du = fmaf(C.c, ex, C.sn * ey), dv = fmaf(C.c, ey, -C.sn * ex);
        const float dp2 = fmaf(C.q2 * du, fmaf(2.f, R.u0, du), dv * fmaf(2.f, R.v0, dv));
        float dau, dav, puu, pvv, puv;
        sie_anchor_delta(R.u0, R.v0, du, dv, dp2, R.ps0, C.q, C.q2, C.e, C.qe, C.s1, C.s1sq, C.q2s1, C.D01,
                         dau, dav, puu, pvv, puv);
        if (C.kind == K_DPIE) {
          float bau, bav, quu, qvv, quv;
          sie_anchor_delta(R.u0, R.v0, du, dv, dp2, R.pa0, C.q, C.q2, C.e, C.qe, C.s2, C.s2sq, C.q2s2, C.D02,
                           bau, bav, quu, qvv, quv);
          dau -= bau; dav -= bav; puu -= quu; pvv -= qvv; puv -= quv;
        }
        Out5<float> o;
        rotate_back(C.c, C.sn, C.b * dau, C.b * dav, C.b * puu, C.b * pvv, C.b * puv, o);
        ff_acc(a5[0], o.ax); ff_acc(a5[1], o.ay);
        ff_acc(a5[2], o.pxx); ff_acc(a5[3], o.pyy); ff_acc(a5[4], o.pxy);
      }
      // the offset e was rounded to FP32: first-order correction with the anchored terms' psi
      ff_acc(a5[0], fmaf(a5[2].hi, exl[q], a5[4].hi * eyl[q]));
      ff_acc(a5[1], fmaf(a5[4].hi, exl[q], a5[3].hi * eyl[q]));
      a5[0] = ff_add(a5[0], sax);
      a5[1] = ff_add(a5[1], say);
      float pxh, pxl, pyh, pyl;
      split_ff(x[q], pxh, pxl);
      split_ff(y[q], pyh, pyl);
      for (int c = 0; c < nc; ++c) {
        const CompT<float>& C = dc[c];
        if (C.kind == 0 || acp[c].anchored) continue;
        ff ax, ay;
        Out5<float> o;
        eval_comp_ext(C, pxh, pxl, pyh, pyl, tab, ax, ay, o);
        a5[0] = ff_add(a5[0], ax);
        a5[1] = ff_add(a5[1], ay);
        ff_acc(a5[2], o.pxx); ff_acc(a5[3], o.pyy); ff_acc(a5[4], o.pxy);
      }
      for (int w = 0; w < nw; ++w) {
        uint32_t word = bits[w];
        while (word) {
          const int k = w * 32 + __ffs(word) - 1;
          word &= word - 1u;
          if (!LF_CHECK(k < nm)) continue;
          ff ax, ay;
          Out5<float> o;
          eval_member_x(dm[k], pxh, pxl, pyh, pyl, ax, ay, o);
          a5[0] = ff_add(a5[0], ax);
          a5[1] = ff_add(a5[1], ay);
          ff_acc(a5[2], o.pxx); ff_acc(a5[3], o.pyy); ff_acc(a5[4], o.pxy);
        }
      }
      if (valid[q]) {
        write_out_ff(O, a_ff, pid[q], a5[0], a5[1], a5[2], a5[3], a5[4]);
      }
    }
    __syncthreads();     // the next tile rewrites the records, the bits and the sums
  }
}

// -------------------------------------------------------------------- LF_FP64 ------
__global__ void __launch_bounds__(256) k_map_fp64(const lf_comp* __restrict__ comp, int nc,
                                                  const lf_member* __restrict__ mem, int nm,
                                                  lf_scaling sc, PosArgs P, OutArgs O) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  const PlaneLayout L = plane_layout<double>(nc, nm, 16);
  lf_comp* rawc = reinterpret_cast<lf_comp*>(smem + L.rawc);
  lf_member* rawm = reinterpret_cast<lf_member*>(smem + L.rawm);
  CompT<double>* dc = reinterpret_cast<CompT<double>*>(smem + L.dc);
  MemT<double>* dm = reinterpret_cast<MemT<double>*>(smem + L.dm);
  if (!LF_CHECK(L.total <= lf_dyn_smem())) return;
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  bool ok = stage_to_smem(rawc, comp, (uint32_t)nc * 64u, bar, 0);
  if (ok) ok = stage_to_smem(rawm, mem, (uint32_t)nm * 32u, bar, nc > 0 ? 1 : 0);
  if (!ok) return;
  digest_plane<double>(rawc, nc, rawm, nm, sc, dc, dm);
  __syncthreads();

  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P.n;
       p += (long long)gridDim.x * blockDim.x) {
    double x, y;
    position_of(P, p, x, y);
    double acc[5] = {0, 0, 0, 0, 0};
    accumulate_fp64(dc, nc, dm, nm, 0, nc + nm, x, y, acc);
    write_out(O, p, acc[0], acc[1], acc[2], acc[3], acc[4]);
  }
}

// ---------------------------------------------------------------------- host -------
lf_status check_plane(const lf_plane* pl) {
  if (!pl) return fail(LF_EINVAL, "plane is NULL");
  if (pl->n_comp < 0 || pl->n_mem < 0) return fail(LF_EINVAL, "negative component count");
  if (pl->n_comp > 0 && !pl->comp) return fail(LF_EINVAL, "n_comp > 0 but comp is NULL");
  if (pl->n_mem > 0 && !pl->mem) return fail(LF_EINVAL, "n_mem > 0 but mem is NULL");
  if (((uintptr_t)pl->comp & 15u) || ((uintptr_t)pl->mem & 15u))
    return fail(LF_EINVAL, "component / member arrays must be 16-byte aligned");
  if (pl->n_mem > 0) {
    const lf_scaling& s = pl->scaling;
    if (!(std::isfinite(s.b_star) && s.b_star >= 0 && std::isfinite(s.core_star) &&
          s.core_star >= 0 && std::isfinite(s.cut_star) && s.cut_star > 0 &&
          std::isfinite(s.lam) && std::isfinite(s.beta) && std::isfinite(s.alpha)))
      return fail(LF_EINVAL, "invalid member scaling relation");
  }
  return LF_OK;
}

static lf_status launch_ff(const lf_plane* pl, const PosArgs& P, const OutArgs& O, int nsm, cudaStream_t s) {
  PlaneLayout L = plane_layout<float, MemX>(pl->n_comp, pl->n_mem, LF_MAP_BASE);
  if (L.total > LF_SMEM_MAX) return fail(LF_EUNSUPPORTED, "plane too large for shared memory");
  LF_CUDA(cudaFuncSetAttribute(k_map_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  int occ = 0;
  LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_map_ff, 256, L.total));
  const long long tiles = (P.n + 255) / 256;
  const long long grid = std::min<long long>(tiles, (long long)nsm * std::max(occ, 1));
  k_map_ff<<<(unsigned)grid, 256, L.total, s>>>(pl->comp, pl->n_comp, pl->mem, pl->n_mem, pl->scaling, P, O);
  return LF_OK;
}

template <bool GRID>
static lf_status launch_anchor(const lf_plane* pl, const PosArgs& P, const OutArgs& O, int nsm,
                               cudaStream_t s) {
  const AnchorLayout L = anchor_layout(pl->n_comp, pl->n_mem);
  if (L.total > LF_SMEM_MAX) return fail(LF_EUNSUPPORTED, "plane too large for shared memory");
  auto k = k_map_anchor<GRID>;
  LF_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  int occ = 0;
  LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, LF_AMAP_THREADS, L.total));
  long long tiles;
  if (GRID) {
    const long long ny = P.n / P.nx;
    tiles = ((P.nx + LF_ATILE - 1) / LF_ATILE) * ((ny + LF_ATILE - 1) / LF_ATILE);
  } else {
    tiles = (P.n + 255) / 256;
  }
  const long long grid = std::min<long long>(tiles, (long long)nsm * std::max(occ, 1));
  k<<<(unsigned)grid, LF_AMAP_THREADS, L.total, s>>>(pl->comp, pl->n_comp, pl->mem, pl->n_mem, pl->scaling,
                                                     P, O, LF_MAP_CHUNK);
  return LF_OK;
}

static lf_status launch_map(const lf_plane* pl, const PosArgs& P, const OutArgs& O,
                            int precision, void* stream) {
  lf_status st = check_plane(pl);
  if (st != LF_OK) return st;
  if (precision < LF_FP64 || precision > LF_FF) return fail(LF_EINVAL, "unknown precision");
  if (P.n == 0) return LF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  LF_CUDA(cudaGetDevice(&dev));
  int nsm = 0;
  LF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int block = 256;
  if (precision == LF_MIXED) {
    if (P.pts) LF_TRY(launch_anchor<false>(pl, P, O, nsm, s));
    else LF_TRY(launch_anchor<true>(pl, P, O, nsm, s));
  } else if (precision == LF_FF) {
    LF_TRY(launch_ff(pl, P, O, nsm, s));
  } else {
    PlaneLayout L = plane_layout<double>(pl->n_comp, pl->n_mem, 16);
    if (L.total > LF_SMEM_MAX) return fail(LF_EUNSUPPORTED, "plane too large for shared memory");
    LF_CUDA(cudaFuncSetAttribute(k_map_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)L.total));
    int occ = 0;
    LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_map_fp64, block, L.total));
    long long tiles = (P.n + block - 1) / block;
    long long grid = std::min<long long>(tiles, (long long)nsm * std::max(occ, 1));
    k_map_fp64<<<(unsigned)grid, block, L.total, s>>>(pl->comp, pl->n_comp, pl->mem, pl->n_mem,
                                                      pl->scaling, P, O);
  }
  LF_CUDA(cudaGetLastError());
  return LF_OK;
}

static lf_status check_grid(const lf_grid* g) {
  if (!g) return fail(LF_EINVAL, "grid is NULL");
  if (g->nx <= 0 || g->ny <= 0) return fail(LF_EINVAL, "grid must have nx, ny > 0");
  if (!(std::isfinite(g->x0) && std::isfinite(g->y0) && std::isfinite(g->dx) &&
        std::isfinite(g->dy)))
    return fail(LF_EINVAL, "grid geometry must be finite");
  return LF_OK;
}

}  // namespace lf

using namespace lf;

extern "C" lf_status lf_deflect_grid(const lf_plane* plane, const lf_grid* grid, int32_t precision,
                                     double* ax, double* ay, void* stream) {
  LF_TRY(check_grid(grid));
  if (!ax || !ay) return fail(LF_EINVAL, "ax and ay are required");
  PosArgs P{nullptr, grid->x0, grid->y0, grid->dx, grid->dy, grid->nx,
            (long long)grid->nx * grid->ny};
  OutArgs O{ax, ay, nullptr, nullptr, nullptr, nullptr, 1.0};
  return launch_map(plane, P, O, precision, stream);
}

extern "C" lf_status lf_jacobian_grid(const lf_plane* plane, const lf_grid* grid, double a_dis,
                                      int32_t precision, double* ax, double* ay, float* kappa,
                                      float* g1, float* g2, double* mu, void* stream) {
  LF_TRY(check_grid(grid));
  if (!(a_dis > 0.0 && a_dis <= 1.0)) return fail(LF_EINVAL, "a_dis must be in (0, 1]");
  PosArgs P{nullptr, grid->x0, grid->y0, grid->dx, grid->dy, grid->nx,
            (long long)grid->nx * grid->ny};
  OutArgs O{ax, ay, mu, kappa, g1, g2, a_dis};
  return launch_map(plane, P, O, precision, stream);
}

extern "C" lf_status lf_jacobian_points(const lf_plane* plane, const double* theta, int32_t n,
                                        double a_dis, int32_t precision, double* ax, double* ay,
                                        float* kappa, float* g1, float* g2, double* mu,
                                        void* stream) {
  if (n < 0) return fail(LF_EINVAL, "n must be >= 0");
  if (n > 0 && !theta) return fail(LF_EINVAL, "theta is NULL");
  if (!(a_dis > 0.0 && a_dis <= 1.0)) return fail(LF_EINVAL, "a_dis must be in (0, 1]");
  PosArgs P{theta, 0, 0, 0, 0, 1, (long long)n};
  OutArgs O{ax, ay, mu, kappa, g1, g2, a_dis};
  return launch_map(plane, P, O, precision, stream);
}
