// Lens-equation solver (Sec. 2.3): the images of a source beta are the common zeros of
// f(theta) = beta - theta + a alpha(theta).  Each component's zero contour is traced over an
// image-plane vertex grid by marching squares (linear interpolation along cell edges, saddle
// cells resolved by the cell-centre value), and the images are the exact intersections of
// pairs of piecewise-linear contour segments in the same cell.  An optional Newton polish on
// the lens equation follows (not part of the paper's solver).
//
// GPU layout of the work:
//  1. alpha on every vertex (the map kernels, any precision tier);
//  2. per cell, the [min, max] of alpha_x and alpha_y over its four corners, rounded outwards
//     to FP32 (independent of the source);
//  3. per (cell, source) an FP32 interval test that f1 and f2 can both vanish in the cell
//     (never rejects a cell the exact test accepts: the ranges are outward-rounded and a
//     margin covers the FP32 rounding of the test), then on the survivors the exact FP64
//     corner values, marching squares and segment intersections; candidates are appended
//     per source with a key (cell, segment pair) that fixes their order;
//  4. per source, the candidates sorted by key and merged when closer than 1e-6 h;
//  5. optionally one warp per image polishes it with Newton steps evaluated in FP64;
//  6. per source, polished images closer than 1e-7 merged, non-finite ones dropped.
#include "lf_internal.h"
#include "lf_eval.cuh"

namespace lf {

struct FinderWS {
  double *ax, *ay;   // alpha on the vertices, nx * ny each
  float4* rng;       // per cell: min ax, max ax, min ay, max ay
  double* cxy;       // n_src * max_cand * 2 candidate positions
  long long* ckey;   // n_src * max_cand keys
  int *ccnt, *kept;  // n_src each
};

static int finder_max_cand(int max_img) { return 4 * max_img + 16; }

static size_t finder_layout(long long nx, long long ny, long long n_src, int max_img, char* base,
                            FinderWS* w) {
  const long long nv = nx * ny, ncell = (nx - 1) * (ny - 1), mc = finder_max_cand(max_img);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = (o + bytes + 255) & ~(size_t)255;
    return base ? base + at : nullptr;
  };
  char* p;
  p = take((size_t)nv * 8); if (w) w->ax = (double*)p;
  p = take((size_t)nv * 8); if (w) w->ay = (double*)p;
  p = take((size_t)ncell * 16); if (w) w->rng = (float4*)p;
  p = take((size_t)(n_src * mc) * 16); if (w) w->cxy = (double*)p;
  p = take((size_t)(n_src * mc) * 8); if (w) w->ckey = (long long*)p;
  p = take((size_t)n_src * 4); if (w) w->ccnt = (int*)p;
  p = take((size_t)n_src * 4); if (w) w->kept = (int*)p;
  return o;
}

__global__ void k_cell_ranges(const double* __restrict__ ax, const double* __restrict__ ay, int nx,
                              long long ncell, float4* __restrict__ rng) {
  const long long cw = nx - 1;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const long long j = c / cw, i = c - j * cw;
    const long long v0 = j * nx + i, v1 = v0 + 1, v3 = v0 + nx, v2 = v3 + 1;
    const double x0 = ax[v0], x1 = ax[v1], x2 = ax[v2], x3 = ax[v3];
    const double y0 = ay[v0], y1 = ay[v1], y2 = ay[v2], y3 = ay[v3];
    float4 r;
    r.x = __double2float_rd(fmin(fmin(x0, x1), fmin(x2, x3)));
    r.y = __double2float_ru(fmax(fmax(x0, x1), fmax(x2, x3)));
    r.z = __double2float_rd(fmin(fmin(y0, y1), fmin(y2, y3)));
    r.w = __double2float_ru(fmax(fmax(y0, y1), fmax(y2, y3)));
    if (!(isfinite(x0) && isfinite(x1) && isfinite(x2) && isfinite(x3) && isfinite(y0) &&
          isfinite(y1) && isfinite(y2) && isfinite(y3)))
      r = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);   // never selected
    rng[c] = r;
  }
}

// Zero crossings of one field on the 4 edges of a cell (corners (0,0) (1,0) (1,1) (0,1);
// edge e joins corner e and e + 1) and the 0, 1 or 2 contour segments they form.
struct CellSegs {
  int n;
  double x[2][2], y[2][2];   // segment s: (x[s][0], y[s][0]) -> (x[s][1], y[s][1])
};

__device__ inline void cell_segments(const double v[4], const double X[4], const double Y[4],
                                     CellSegs& S) {
  double px[4], py[4];
  bool has[4];
  int ne = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int a = e, b = (e + 1) & 3;
    has[e] = (v[a] > 0.0) != (v[b] > 0.0);
    if (has[e]) {
      const double t = v[a] / (v[a] - v[b]);
      px[e] = X[a] + t * (X[b] - X[a]);
      py[e] = Y[a] + t * (Y[b] - Y[a]);
      ++ne;
    }
  }
  S.n = 0;
  if (ne == 2) {
    int e0 = -1, e1 = -1;
    for (int e = 0; e < 4; ++e)
      if (has[e]) { if (e0 < 0) e0 = e; else e1 = e; }
    S.x[0][0] = px[e0]; S.y[0][0] = py[e0]; S.x[0][1] = px[e1]; S.y[0][1] = py[e1];
    S.n = 1;
  } else if (ne == 4) {
    // saddle: each corner whose sign differs from the centre's is cut off by the segment
    // joining its two adjacent edges (edges k - 1 and k for corner k)
    const double centre = 0.25 * (((v[0] + v[1]) + v[2]) + v[3]);
    for (int k = 0; k < 4; ++k) {
      if ((v[k] > 0.0) != (centre > 0.0)) {
        const int ea = (k + 3) & 3;
        S.x[S.n][0] = px[ea]; S.y[S.n][0] = py[ea]; S.x[S.n][1] = px[k]; S.y[S.n][1] = py[k];
        ++S.n;
      }
    }
  }
}

// Exact intersection of segments p -> p2 and q -> q2 (parameters within [0, 1] up to 1e-12).
__device__ inline bool seg_intersect(double px, double py, double p2x, double p2y, double qx, double qy,
                                     double q2x, double q2y, double& ox, double& oy) {
  const double rx = p2x - px, ry = p2y - py, sx = q2x - qx, sy = q2y - qy;
  const double den = rx * sy - ry * sx;
  if (den == 0.0) return false;
  const double qpx = qx - px, qpy = qy - py;
  const double t = (qpx * sy - qpy * sx) / den;
  const double u = (qpx * ry - qpy * rx) / den;
  if (t >= -1e-12 && t <= 1.0 + 1e-12 && u >= -1e-12 && u <= 1.0 + 1e-12) {
    ox = px + t * rx;
    oy = py + t * ry;
    return true;
  }
  return false;
}

constexpr int LF_FIND_CHUNK = 512;   // sources staged in shared memory at a time

__global__ void __launch_bounds__(256) k_find_cells(const double* __restrict__ ax,
                                                    const double* __restrict__ ay,
                                                    const float4* __restrict__ rng, int nx,
                                                    long long ncell, double x0, double y0, double dx,
                                                    double dy, const double* __restrict__ beta,
                                                    const double* __restrict__ a_src, int n_src,
                                                    int max_cand, double* cxy, long long* ckey,
                                                    int* ccnt) {
  __shared__ double sb[LF_FIND_CHUNK][3];
  __shared__ float sf[LF_FIND_CHUNK][4];   // beta_x, beta_y, a, margin scale
  const long long cw = nx - 1;
  for (int s0 = 0; s0 < n_src; s0 += LF_FIND_CHUNK) {
    const int ns = min(LF_FIND_CHUNK, n_src - s0);
    __syncthreads();
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
      const double b1 = beta[2 * (s0 + k)], b2 = beta[2 * (s0 + k) + 1], a = a_src[s0 + k];
      const bool ok = a > 0.0 && a <= 1.0 && isfinite(b1) && isfinite(b2);
      if (!ok) lf_flag_error(LF_DEVERR_BADARG);
      sb[k][0] = b1; sb[k][1] = b2; sb[k][2] = a;
      sf[k][0] = (float)b1; sf[k][1] = (float)b2; sf[k][2] = ok ? (float)a : -1.f;
      sf[k][3] = 1.f + fabsf((float)b1) + fabsf((float)b2);
    }
    __syncthreads();
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
      const long long j = c / cw, i = c - j * cw;
      const float4 R = rng[c];
      const double xl = x0 + dx * (double)i, xr = x0 + dx * (double)(i + 1);
      const double yb = y0 + dy * (double)j, yt = y0 + dy * (double)(j + 1);
      const float xlf = (float)xl, xrf = (float)xr, ybf = (float)yb, ytf = (float)yt;
      const float scale_c = fabsf(xlf) + fabsf(xrf) + fabsf(ybf) + fabsf(ytf);
      const float amax = fmaxf(fmaxf(fabsf(R.x), fabsf(R.y)), fmaxf(fabsf(R.z), fabsf(R.w)));
      bool loaded = false;
      double X[4], Y[4], AX[4], AY[4];
      for (int k = 0; k < ns; ++k) {
        const float a = sf[k][2];
        if (!(a > 0.f)) continue;
        // f1 over the cell lies in [b1 - xr + a min ax, b1 - xl + a max ax]; same for f2
        const float m = 4e-6f * (sf[k][3] + scale_c + a * amax);
        const float lo1 = sf[k][0] - xrf + a * R.x, hi1 = sf[k][0] - xlf + a * R.y;
        const float lo2 = sf[k][1] - ytf + a * R.z, hi2 = sf[k][1] - ybf + a * R.w;
        if (lo1 > m || hi1 < -m || lo2 > m || hi2 < -m) continue;
        if (!loaded) {
          const long long v0 = j * nx + i;
          const long long vs[4] = {v0, v0 + 1, v0 + nx + 1, v0 + nx};
          X[0] = xl; X[1] = xr; X[2] = xr; X[3] = xl;
          Y[0] = yb; Y[1] = yb; Y[2] = yt; Y[3] = yt;
#pragma unroll
          for (int q = 0; q < 4; ++q) { AX[q] = ax[vs[q]]; AY[q] = ay[vs[q]]; }
          loaded = true;
        }
        const double b1 = sb[k][0], b2 = sb[k][1], ad = sb[k][2];
        double f1[4], f2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          f1[q] = __dadd_rn(__dsub_rn(b1, X[q]), __dmul_rn(ad, AX[q]));
          f2[q] = __dadd_rn(__dsub_rn(b2, Y[q]), __dmul_rn(ad, AY[q]));
        }
        const bool s0p = f1[0] > 0.0, t0p = f2[0] > 0.0;
        const bool ch1 = (f1[1] > 0.0) != s0p || (f1[2] > 0.0) != s0p || (f1[3] > 0.0) != s0p;
        const bool ch2 = (f2[1] > 0.0) != t0p || (f2[2] > 0.0) != t0p || (f2[3] > 0.0) != t0p;
        if (!(ch1 && ch2)) continue;
        CellSegs A, B;
        cell_segments(f1, X, Y, A);
        cell_segments(f2, X, Y, B);
        for (int sa = 0; sa < A.n; ++sa)
          for (int sbi = 0; sbi < B.n; ++sbi) {
            double ox, oy;
            if (!seg_intersect(A.x[sa][0], A.y[sa][0], A.x[sa][1], A.y[sa][1], B.x[sbi][0],
                               B.y[sbi][0], B.x[sbi][1], B.y[sbi][1], ox, oy))
              continue;
            const int s = s0 + k;
            const int slot = atomicAdd(&ccnt[s], 1);
            if (slot < max_cand) {
              const size_t at = (size_t)s * max_cand + slot;
              cxy[2 * at] = ox;
              cxy[2 * at + 1] = oy;
              ckey[at] = c * 4 + sa * 2 + sbi;
            }
          }
      }
    }
  }
}

// Per source: candidates in key order (row-major cell, then segment pair), merged when
// closer than tol; kept[s] = number kept, or -1 if the candidate buffer overflowed.
__global__ void k_sort_merge(int n_src, int max_cand, double tol, double* cxy, long long* ckey,
                             const int* ccnt, int* kept) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_src) return;
  const int n = ccnt[s];
  if (n > max_cand) { kept[s] = -1; return; }
  double* P = cxy + (size_t)s * max_cand * 2;
  long long* K = ckey + (size_t)s * max_cand;
  for (int i = 1; i < n; ++i) {   // insertion sort by key (a few candidates per source)
    const long long k = K[i];
    const double x = P[2 * i], y = P[2 * i + 1];
    int j = i - 1;
    while (j >= 0 && K[j] > k) {
      K[j + 1] = K[j]; P[2 * (j + 1)] = P[2 * j]; P[2 * (j + 1) + 1] = P[2 * j + 1];
      --j;
    }
    K[j + 1] = k; P[2 * (j + 1)] = x; P[2 * (j + 1) + 1] = y;
  }
  const double t2 = tol * tol;
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const double x = P[2 * i], y = P[2 * i + 1];
    bool keep = true;
    for (int q = 0; q < m && keep; ++q) {
      const double ex = x - P[2 * q], ey = y - P[2 * q + 1];
      keep = ex * ex + ey * ey > t2;
    }
    if (keep) { P[2 * m] = x; P[2 * m + 1] = y; K[m] = K[i]; ++m; }
  }
  kept[s] = m;
}

// Newton polish theta <- theta - A^-1 (beta(theta) - beta_s), one warp per image, the plane's
// alpha and psi_ij summed in FP64 across the lanes; stops when |beta(theta) - beta_s| < 1e-12.
__global__ void __launch_bounds__(256) k_polish(const lf_comp* __restrict__ comp, int nc,
                                                const lf_member* __restrict__ mem, int nm,
                                                lf_scaling sc, const double* __restrict__ beta,
                                                const double* __restrict__ a_src, int n_src,
                                                int max_cand, const int* __restrict__ kept,
                                                int iters, double* cxy) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  const PlaneLayout L = plane_layout<double>(nc, nm, 16);
  lf_comp* rawc = reinterpret_cast<lf_comp*>(smem + L.rawc);
  lf_member* rawm = reinterpret_cast<lf_member*>(smem + L.rawm);
  CompT<double>* dc = reinterpret_cast<CompT<double>*>(smem + L.dc);
  MemT<double>* dm = reinterpret_cast<MemT<double>*>(smem + L.dm);
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  bool ok = stage_to_smem(rawc, comp, (uint32_t)nc * 64u, bar, 0);
  if (ok) ok = stage_to_smem(rawm, mem, (uint32_t)nm * 32u, bar, nc > 0 ? 1 : 0);
  if (!ok) return;
  digest_plane<double>(rawc, nc, rawm, nm, sc, dc, dm);
  __syncthreads();

  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  const int K = nc + nm;
  const int k0 = (int)((long long)K * lane / 32), k1 = (int)((long long)K * (lane + 1) / 32);
  const long long n_slot = (long long)n_src * max_cand;
  for (long long slot = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); slot < n_slot;
       slot += (long long)gridDim.x * wpb) {
    const int s = (int)(slot / max_cand), q = (int)(slot - (long long)s * max_cand);
    if (q >= kept[s]) continue;
    const double a = a_src[s], bx = beta[2 * s], by = beta[2 * s + 1];
    double tx = cxy[2 * slot], ty = cxy[2 * slot + 1];
    for (int it = 0; it < iters; ++it) {
      double acc[5] = {0, 0, 0, 0, 0};
      accumulate_fp64(dc, nc, dm, nm, k0, k1, tx, ty, acc);
#pragma unroll
      for (int v = 0; v < 5; ++v)
        for (int off = 16; off > 0; off >>= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
      const double rx = (tx - a * acc[0]) - bx, ry = (ty - a * acc[1]) - by;
      if (hypot(rx, ry) < 1e-12) break;
      const double a11 = 1.0 - a * acc[2], a22 = 1.0 - a * acc[3], a12 = -a * acc[4];
      const double det = a11 * a22 - a12 * a12;
      tx -= (a22 * rx - a12 * ry) / det;
      ty -= (a11 * ry - a12 * rx) / det;
      if (!(isfinite(tx) && isfinite(ty))) break;
    }
    if (lane == 0) { cxy[2 * slot] = tx; cxy[2 * slot + 1] = ty; }
  }
}

// Per source: the kept images written to img; after a polish they are first merged greedily
// (an image is kept when it is finite and farther than tol from every image kept before it).
// n_img[s] = their number (may exceed max_img: only the first max_img are stored), or -1
// when the candidate buffer overflowed.
__global__ void k_find_finish(int n_src, int max_cand, int max_img, bool polished, double tol,
                              double* cxy, const int* __restrict__ kept, double* img, int* n_img) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_src) return;
  const int n = kept[s];
  if (n < 0) { n_img[s] = -1; return; }
  double* P = cxy + (size_t)s * max_cand * 2;
  int m = n;
  if (polished) {
    m = 0;
    for (int i = 0; i < n; ++i) {
      const double x = P[2 * i], y = P[2 * i + 1];
      bool keep = isfinite(x) && isfinite(y);
      for (int q = 0; q < m && keep; ++q) keep = hypot(x - P[2 * q], y - P[2 * q + 1]) > tol;
      if (keep) { P[2 * m] = x; P[2 * m + 1] = y; ++m; }
    }
  }
  double* O = img + (size_t)s * max_img * 2;
  for (int i = 0; i < m && i < max_img; ++i) { O[2 * i] = P[2 * i]; O[2 * i + 1] = P[2 * i + 1]; }
  n_img[s] = m;
}

}  // namespace lf

using namespace lf;

extern "C" size_t lf_find_images_workspace(int32_t nx, int32_t ny, int32_t n_src, int32_t max_img) {
  if (nx < 2 || ny < 2 || n_src < 0 || max_img < 1) return 0;
  return finder_layout(nx, ny, n_src, max_img, nullptr, nullptr);
}

extern "C" lf_status lf_find_images(const lf_plane* plane, const lf_grid* grid, int32_t precision,
                                    const double* beta, const double* a_src, int32_t n_src,
                                    int32_t max_img, int32_t polish_iters, void* workspace,
                                    size_t workspace_bytes, double* img, int32_t* n_img,
                                    void* stream) {
  LF_TRY(check_plane(plane));
  if (!grid) return fail(LF_EINVAL, "grid is NULL");
  if (grid->nx < 2 || grid->ny < 2) return fail(LF_EINVAL, "the vertex grid needs nx, ny >= 2");
  if (!(std::isfinite(grid->x0) && std::isfinite(grid->y0) && grid->dx > 0 && grid->dy > 0 &&
        std::isfinite(grid->dx) && std::isfinite(grid->dy)))
    return fail(LF_EINVAL, "grid origin must be finite and its steps positive");
  if (precision < LF_FP64 || precision > LF_FF) return fail(LF_EINVAL, "unknown precision");
  if (n_src < 0) return fail(LF_EINVAL, "n_src must be >= 0");
  if (max_img < 1) return fail(LF_EINVAL, "max_img must be >= 1");
  if (polish_iters < 0) return fail(LF_EINVAL, "polish_iters must be >= 0");
  if (n_src == 0) return LF_OK;
  if (!beta || !a_src || !img || !n_img) return fail(LF_EINVAL, "beta, a_src, img and n_img are required");
  const size_t need = finder_layout(grid->nx, grid->ny, n_src, max_img, nullptr, nullptr);
  if (!workspace || workspace_bytes < need)
    return fail(LF_EINVAL, "workspace of %zu bytes needed (lf_find_images_workspace)", need);
  if ((uintptr_t)workspace & 255u) return fail(LF_EINVAL, "workspace must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  FinderWS W;
  finder_layout(grid->nx, grid->ny, n_src, max_img, (char*)workspace, &W);
  const int max_cand = finder_max_cand(max_img);
  int dev = 0, nsm = 0;
  LF_CUDA(cudaGetDevice(&dev));
  LF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));

  // 1. alpha on the vertices
  PosArgs P{nullptr, grid->x0, grid->y0, grid->dx, grid->dy, grid->nx,
            (long long)grid->nx * grid->ny};
  OutArgs O{W.ax, W.ay, nullptr, nullptr, nullptr, nullptr, 1.0};
  LF_TRY(launch_map(plane, P, O, precision, stream));
  // 2. cell ranges
  const long long ncell = (long long)(grid->nx - 1) * (grid->ny - 1);
  const unsigned g2 = (unsigned)std::min<long long>((ncell + 255) / 256, (long long)nsm * 16);
  k_cell_ranges<<<g2, 256, 0, s>>>(W.ax, W.ay, grid->nx, ncell, W.rng);
  // 3. candidates
  LF_CUDA(cudaMemsetAsync(W.ccnt, 0, (size_t)n_src * 4, s));
  const unsigned g3 = (unsigned)std::min<long long>((ncell + 255) / 256, (long long)nsm * 8);
  k_find_cells<<<g3, 256, 0, s>>>(W.ax, W.ay, W.rng, grid->nx, ncell, grid->x0, grid->y0, grid->dx,
                                   grid->dy, beta, a_src, n_src, max_cand, W.cxy, W.ckey, W.ccnt);
  // 4. order and merge
  const unsigned gs = (unsigned)((n_src + 127) / 128);
  k_sort_merge<<<gs, 128, 0, s>>>(n_src, max_cand, 1e-6 * grid->dx, W.cxy, W.ckey, W.ccnt, W.kept);
  // 5. polish
  if (polish_iters > 0) {
    PlaneLayout L = plane_layout<double>(plane->n_comp, plane->n_mem, 16);
    if (L.total > LF_SMEM_MAX) return fail(LF_EUNSUPPORTED, "plane too large for shared memory");
    LF_CUDA(cudaFuncSetAttribute(k_polish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    const long long slots = (long long)n_src * max_cand;
    const unsigned gp = (unsigned)std::min<long long>((slots + 7) / 8, (long long)nsm * 2);
    k_polish<<<gp, 256, L.total, s>>>(plane->comp, plane->n_comp, plane->mem, plane->n_mem,
                                       plane->scaling, beta, a_src, n_src, max_cand, W.kept,
                                       polish_iters, W.cxy);
  }
  // 6. output
  k_find_finish<<<gs, 128, 0, s>>>(n_src, max_cand, max_img, polish_iters > 0, 1e-7, W.cxy, W.kept,
                                    img, n_img);
  LF_CUDA(cudaGetLastError());
  return LF_OK;
}

// ------------------------------------------------------------------ several planes -----
// Sources at one redshift behind several planes: beta(theta) is the recursion's (Sec. 2.2),
// so f = beta_s - beta(theta) = beta_s - theta + alpha_eff(theta) with the effective
// deflection alpha_eff = theta - beta(theta) on the vertices (the trace kernel, in the chosen
// tier) and a = 1; steps 2-4 and 6 are those above.  The polish alternates the recursion at
// the candidates (FP64 for the FP64 tier, else float-float: float-float deflections, about
// 1e-12 relative), traced in 32-thread blocks so that a few hundred rays spread over many
// SMs, with Newton steps theta <- theta - A^-1 (beta(theta) - beta_s) on its non-symmetric A.
namespace lf {

lf_status trace_rays(const lf_plane* planes, int32_t n_planes, const double* ratios, const double* theta,
                     int32_t n, const lf_grid* grid, int32_t precision, double* beta, double* A,
                     void* stream, int block);   // lf_trace.cu

struct FinderMPWS {
  double* bvert;   // beta on the vertices, nx * ny * 2
  double* ones;    // a = 1 per source
  double* pb;      // per polished candidate: beta (2) and A (4) of the recursion
  double* pA;
  double* pos;     // the kept candidates, compacted (2 each)
  int* map;        // their slot (source * max_cand + k)
  int* count;      // how many
};

static size_t finder_mp_layout(long long nx, long long ny, long long n_src, int max_img, char* base,
                               FinderWS* w, FinderMPWS* m) {
  size_t o = finder_layout(nx, ny, n_src, max_img, base, w);
  const long long slots = n_src * finder_max_cand(max_img);
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = (o + bytes + 255) & ~(size_t)255;
    return base ? base + at : nullptr;
  };
  char* p;
  p = take((size_t)(nx * ny) * 16); if (m) m->bvert = (double*)p;
  p = take((size_t)n_src * 8); if (m) m->ones = (double*)p;
  p = take((size_t)slots * 16); if (m) m->pb = (double*)p;
  p = take((size_t)slots * 32); if (m) m->pA = (double*)p;
  p = take((size_t)slots * 16); if (m) m->pos = (double*)p;
  p = take((size_t)slots * 4); if (m) m->map = (int*)p;
  p = take(4); if (m) m->count = (int*)p;
  return o;
}

__global__ void k_mp_alpha(const double* __restrict__ bvert, long long nv, int nx, double x0, double y0,
                           double dx, double dy, double* ax, double* ay, double* ones, int n_src) {
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
  for (long long v = t0; v < nv; v += nt) {
    const long long iy = v / nx, ix = v - iy * nx;
    ax[v] = (x0 + dx * (double)ix) - bvert[2 * v];
    ay[v] = (y0 + dy * (double)iy) - bvert[2 * v + 1];
  }
  for (long long i = t0; i < n_src; i += nt) ones[i] = 1.0;
}

// The kept candidates of every source into one list (order immaterial: each is polished alone).
__global__ void k_mp_compact(int n_src, int max_cand, const int* __restrict__ kept,
                             const double* __restrict__ cxy, double* pos, int* map, int* count) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)n_src * max_cand) return;
  const int src = (int)(q / max_cand), k = (int)(q - (long long)src * max_cand);
  if (k >= kept[src]) return;
  const int i = atomicAdd(count, 1);
  map[i] = (int)q;
  pos[2 * i] = cxy[2 * q];
  pos[2 * i + 1] = cxy[2 * q + 1];
}

__global__ void k_mp_scatter(int n, const int* __restrict__ map, const double* __restrict__ pos, double* cxy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cxy[2 * map[i]] = pos[2 * i];
  cxy[2 * map[i] + 1] = pos[2 * i + 1];
}

// A step longer than max_step (the grid step) leaves the candidate where it is: the raw
// candidate lies within O(h^2) of its root, so such a step means A is near-singular there (a
// critical curve) and the iteration has left the root's basin.
__global__ void k_mp_newton(int n, int max_cand, const int* __restrict__ map, const double* __restrict__ beta,
                            const double* __restrict__ pb, const double* __restrict__ pA, double max_step,
                            double* pos) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int src = map[i] / max_cand;
  const double rx = pb[2 * i] - beta[2 * src], ry = pb[2 * i + 1] - beta[2 * src + 1];
  const double* A = pA + 4 * i;
  const double id = 1.0 / (A[0] * A[3] - A[1] * A[2]);
  const double sx = (A[3] * rx - A[1] * ry) * id, sy = (A[0] * ry - A[2] * rx) * id;
  if (!(sx * sx + sy * sy <= max_step * max_step)) return;
  pos[2 * i] -= sx;
  pos[2 * i + 1] -= sy;
}

}  // namespace lf

extern "C" size_t lf_find_images_multiplane_workspace(int32_t nx, int32_t ny, int32_t n_src, int32_t max_img) {
  if (nx < 2 || ny < 2 || n_src < 0 || max_img < 1) return 0;
  return finder_mp_layout(nx, ny, n_src, max_img, nullptr, nullptr, nullptr);
}

extern "C" lf_status lf_find_images_multiplane(const lf_plane* planes, int32_t n_planes, const double* ratios,
                                               const lf_grid* grid, int32_t precision, const double* beta,
                                               int32_t n_src, int32_t max_img, int32_t polish_iters,
                                               void* workspace, size_t workspace_bytes, double* img,
                                               int32_t* n_img, void* stream) {
  if (!planes || n_planes < 1 || n_planes > LF_MAX_PLANES) return fail(LF_EINVAL, "need 1 <= n_planes <= 8 planes");
  if (!ratios) return fail(LF_EINVAL, "ratios is NULL");
  for (int j = 0; j < n_planes; ++j) LF_TRY(check_plane(&planes[j]));
  if (!grid) return fail(LF_EINVAL, "grid is NULL");
  if (grid->nx < 2 || grid->ny < 2) return fail(LF_EINVAL, "the vertex grid needs nx, ny >= 2");
  if (!(std::isfinite(grid->x0) && std::isfinite(grid->y0) && grid->dx > 0 && grid->dy > 0 &&
        std::isfinite(grid->dx) && std::isfinite(grid->dy)))
    return fail(LF_EINVAL, "grid origin must be finite and its steps positive");
  if (precision < LF_FP64 || precision > LF_FF) return fail(LF_EINVAL, "unknown precision");
  if (n_src < 0) return fail(LF_EINVAL, "n_src must be >= 0");
  if (max_img < 1) return fail(LF_EINVAL, "max_img must be >= 1");
  if (polish_iters < 0) return fail(LF_EINVAL, "polish_iters must be >= 0");
  if (n_src == 0) return LF_OK;
  if (!beta || !img || !n_img) return fail(LF_EINVAL, "beta, img and n_img are required");
  const size_t need = finder_mp_layout(grid->nx, grid->ny, n_src, max_img, nullptr, nullptr, nullptr);
  if (!workspace || workspace_bytes < need)
    return fail(LF_EINVAL, "workspace of %zu bytes needed (lf_find_images_multiplane_workspace)", need);
  if ((uintptr_t)workspace & 255u) return fail(LF_EINVAL, "workspace must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  FinderWS W;
  FinderMPWS M;
  finder_mp_layout(grid->nx, grid->ny, n_src, max_img, (char*)workspace, &W, &M);
  const int max_cand = finder_max_cand(max_img);
  int dev = 0, nsm = 0;
  LF_CUDA(cudaGetDevice(&dev));
  LF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // 1. alpha_eff = theta - beta(theta) on the vertices
  const long long nv = (long long)grid->nx * grid->ny;
  LF_TRY(lf_trace_multiplane(planes, n_planes, ratios, nullptr, 0, grid, precision, M.bvert, nullptr, stream));
  const unsigned g1 = (unsigned)std::min<long long>((nv + 255) / 256, (long long)nsm * 16);
  k_mp_alpha<<<g1, 256, 0, s>>>(M.bvert, nv, grid->nx, grid->x0, grid->y0, grid->dx, grid->dy, W.ax, W.ay,
                                M.ones, n_src);
  // 2-4. cell ranges, candidates, order and merge (a = 1)
  const long long ncell = (long long)(grid->nx - 1) * (grid->ny - 1);
  const unsigned g2 = (unsigned)std::min<long long>((ncell + 255) / 256, (long long)nsm * 16);
  k_cell_ranges<<<g2, 256, 0, s>>>(W.ax, W.ay, grid->nx, ncell, W.rng);
  LF_CUDA(cudaMemsetAsync(W.ccnt, 0, (size_t)n_src * 4, s));
  const unsigned g3 = (unsigned)std::min<long long>((ncell + 255) / 256, (long long)nsm * 8);
  k_find_cells<<<g3, 256, 0, s>>>(W.ax, W.ay, W.rng, grid->nx, ncell, grid->x0, grid->y0, grid->dx,
                                   grid->dy, beta, M.ones, n_src, max_cand, W.cxy, W.ckey, W.ccnt);
  const unsigned gs = (unsigned)((n_src + 127) / 128);
  k_sort_merge<<<gs, 128, 0, s>>>(n_src, max_cand, 1e-6 * grid->dx, W.cxy, W.ckey, W.ccnt, W.kept);
  // 5. polish: the kept candidates compacted (their count read back, one stream synchronisation),
  //    then the recursion at them and a Newton step, polish_iters times
  if (polish_iters > 0) {
    const long long slots = (long long)n_src * max_cand;
    LF_CUDA(cudaMemsetAsync(M.count, 0, sizeof(int), s));
    k_mp_compact<<<(unsigned)((slots + 255) / 256), 256, 0, s>>>(n_src, max_cand, W.kept, W.cxy, M.pos, M.map,
                                                                 M.count);
    int nk = 0;
    LF_CUDA(cudaMemcpyAsync(&nk, M.count, sizeof(int), cudaMemcpyDeviceToHost, s));
    LF_CUDA(cudaStreamSynchronize(s));
    if (nk > 0) {
      for (int it = 0; it < polish_iters; ++it) {
        LF_TRY(trace_rays(planes, n_planes, ratios, M.pos, nk, nullptr, precision == LF_FP64 ? LF_FP64 : LF_FF,
                          M.pb, M.pA, stream, 32));
        k_mp_newton<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(nk, max_cand, M.map, beta, M.pb, M.pA,
                                                                std::max(grid->dx, grid->dy), M.pos);
      }
      k_mp_scatter<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(nk, M.map, M.pos, W.cxy);
    }
  }
  // 6. output
  k_find_finish<<<gs, 128, 0, s>>>(n_src, max_cand, max_img, polish_iters > 0, 1e-7, W.cxy, W.kept,
                                    img, n_img);
  LF_CUDA(cudaGetLastError());
  return LF_OK;
}
