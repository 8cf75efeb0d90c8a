// Multi-plane ray tracing with the Jacobian product (Sec. 2.2).
//
// For each ray: theta_j = theta_1 - sum_{i<j} r_ij alpha_i(theta_i) and
// A_j = I - sum_{i<j} r_ij Psi_i(theta_i) A_i, then beta = theta_1 - sum_j rs_j alpha_j and
// A = I - sum_j rs_j Psi_j A_j.  All planes are staged into shared memory once per
// (persistent) block.  LF_MIXED evaluates each plane's components in FP32 on float-float
// offsets from theta_j and carries theta_j, the deflections, beta and the 2x2 Jacobian
// product in float-float (on the FP32 pipe); LF_FF evaluates in float-float and keeps the
// recursion in FP64; LF_FP64 does everything in FP64.
#include "lf_internal.h"
#include "lf_eval.cuh"

namespace lf {

struct MultiPlaneArgs {
  int np;
  const lf_comp* comp[LF_MAX_PLANES];
  const lf_member* mem[LF_MAX_PLANES];
  int nc[LF_MAX_PLANES], nm[LF_MAX_PLANES];
  lf_scaling sc[LF_MAX_PLANES];
  uint32_t base[LF_MAX_PLANES];     // shared-memory offset of each plane's layout
  double r[LF_MAX_PLANES][LF_MAX_PLANES];
  double rs[LF_MAX_PLANES];
  float2 rf[LF_MAX_PLANES][LF_MAX_PLANES];   // the same ratios as float-float (hi, lo)
  float2 rsf[LF_MAX_PLANES];
};

// Stages and digests every plane; returns false (all threads) if a bounded wait ran out.
template <class T, class M>
__device__ bool stage_planes(unsigned char* smem, uint64_t* bar, const MultiPlaneArgs& A) {
  uint32_t phase = 0;
  for (int j = 0; j < A.np; ++j) {
    PlaneLayout L = plane_layout<T, M>(A.nc[j], A.nm[j], A.base[j]);
    if (A.nc[j] > 0) {
      if (!stage_to_smem(smem + L.rawc, A.comp[j], (uint32_t)A.nc[j] * 64u, bar, phase & 1u))
        return false;
      ++phase;
    }
    if (A.nm[j] > 0) {
      if (!stage_to_smem(smem + L.rawm, A.mem[j], (uint32_t)A.nm[j] * 32u, bar, phase & 1u))
        return false;
      ++phase;
    }
    if constexpr (std::is_same<M, MemX>::value)
      digest_plane_x(reinterpret_cast<lf_comp*>(smem + L.rawc), A.nc[j],
                     reinterpret_cast<lf_member*>(smem + L.rawm), A.nm[j], A.sc[j],
                     reinterpret_cast<CompT<float>*>(smem + L.dc), reinterpret_cast<MemX*>(smem + L.dm));
    else
      digest_plane<T>(reinterpret_cast<lf_comp*>(smem + L.rawc), A.nc[j],
                      reinterpret_cast<lf_member*>(smem + L.rawm), A.nm[j], A.sc[j],
                      reinterpret_cast<CompT<T>*>(smem + L.dc), reinterpret_cast<MemT<T>*>(smem + L.dm));
  }
  __syncthreads();
  return true;
}

struct RayIO {
  const double* pts;
  double x0, y0, dx, dy;
  int nx;
  long long n;
  double* beta;
  double* A;
};

template <int MODE>   // LF_FP64, LF_MIXED or LF_FF
__global__ void __launch_bounds__(256) k_trace(MultiPlaneArgs MP, RayIO io, int chunk) {
  constexpr bool MIXED = MODE != LF_FP64;
  typedef typename std::conditional<MIXED, float, double>::type T;
  typedef typename std::conditional<MODE == LF_FF, MemX, MemT<T>>::type Mem;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  float2* tab = reinterpret_cast<float2*>(smem + 16);
  for (int j = 0; j < MP.np; ++j)
    if (!LF_CHECK(plane_layout<T, Mem>(MP.nc[j], MP.nm[j], MP.base[j]).total <= lf_dyn_smem())) return;
  if (threadIdx.x == 0) mbar_init(bar, 1);
  init_ff_tables(tab);
  __syncthreads();
  if (!stage_planes<T, Mem>(smem, bar, MP)) return;

  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < io.n;
       p += (long long)gridDim.x * blockDim.x) {
    double t1x, t1y;
    if (io.pts) {
      t1x = io.pts[2 * p];
      t1y = io.pts[2 * p + 1];
    } else {
      long long j = p / io.nx, i = p - j * io.nx;
      t1x = io.x0 + (double)i * io.dx;
      t1y = io.y0 + (double)j * io.dy;
    }
    if constexpr (MODE == LF_MIXED) {
      // The recursion on the FP32 pipe: theta_j, the deflections and beta in float-float, and
      // the Jacobian product Psi_j A_j and A_j in float-float as well (about 48 bits, the
      // precision of the FP64 product to within the FP32 rounding of each Psi_j).
      ff t1xf, t1yf;
      {
        float h, l;
        split_ff(t1x, h, l); t1xf = ff_make(h, l);
        split_ff(t1y, h, l); t1yf = ff_make(h, l);
      }
      ff alx[LF_MAX_PLANES], aly[LF_MAX_PLANES];
      ff PA[LF_MAX_PLANES][4];   // Psi_j A_j, row-major
      for (int j = 0; j < MP.np; ++j) {
        ff tx = t1xf, ty = t1yf;
        ff a00 = ff_make(1.f, 0.f), a01 = ff_zero(), a10 = ff_zero(), a11 = ff_make(1.f, 0.f);
        for (int i = 0; i < j; ++i) {
          const float2 r = MP.rf[i][j];
          const ff rr = ff_make(r.x, r.y);
          tx = ff_sub(tx, ff_mul(rr, alx[i]));
          ty = ff_sub(ty, ff_mul(rr, aly[i]));
          a00 = ff_sub(a00, ff_mul(rr, PA[i][0])); a01 = ff_sub(a01, ff_mul(rr, PA[i][1]));
          a10 = ff_sub(a10, ff_mul(rr, PA[i][2])); a11 = ff_sub(a11, ff_mul(rr, PA[i][3]));
        }
        PlaneLayout L = plane_layout<T, Mem>(MP.nc[j], MP.nm[j], MP.base[j]);
        const CompT<T>* dc = reinterpret_cast<const CompT<T>*>(smem + L.dc);
        const Mem* dm = reinterpret_cast<const Mem*>(smem + L.dm);
        float xh[1] = {tx.hi}, xl[1] = {tx.lo}, yh[1] = {ty.hi}, yl[1] = {ty.lo};
        ff acc[5][1];
        for (int v = 0; v < 5; ++v) acc[v][0] = ff_zero();
        accumulate_mixed<1>(dc, MP.nc[j], dm, MP.nm[j], 0, MP.nc[j] + MP.nm[j], chunk, xh, xl, yh, yl,
                            tab, acc);
        alx[j] = acc[0][0];
        aly[j] = acc[1][0];
        const ff pxx = acc[2][0], pyy = acc[3][0], pxy = acc[4][0];
        PA[j][0] = ff_add(ff_mul(pxx, a00), ff_mul(pxy, a10));
        PA[j][1] = ff_add(ff_mul(pxx, a01), ff_mul(pxy, a11));
        PA[j][2] = ff_add(ff_mul(pxy, a00), ff_mul(pyy, a10));
        PA[j][3] = ff_add(ff_mul(pxy, a01), ff_mul(pyy, a11));
      }
      ff bx = t1xf, by = t1yf;
      ff A00 = ff_make(1.f, 0.f), A01 = ff_zero(), A10 = ff_zero(), A11 = ff_make(1.f, 0.f);
      for (int j = 0; j < MP.np; ++j) {
        const float2 r = MP.rsf[j];
        const ff rr = ff_make(r.x, r.y);
        bx = ff_sub(bx, ff_mul(rr, alx[j]));
        by = ff_sub(by, ff_mul(rr, aly[j]));
        A00 = ff_sub(A00, ff_mul(rr, PA[j][0])); A01 = ff_sub(A01, ff_mul(rr, PA[j][1]));
        A10 = ff_sub(A10, ff_mul(rr, PA[j][2])); A11 = ff_sub(A11, ff_mul(rr, PA[j][3]));
      }
      if (io.beta) {
        io.beta[2 * p] = ff_to_double(bx);
        io.beta[2 * p + 1] = ff_to_double(by);
      }
      if (io.A) {
        io.A[4 * p] = ff_to_double(A00); io.A[4 * p + 1] = ff_to_double(A01);
        io.A[4 * p + 2] = ff_to_double(A10); io.A[4 * p + 3] = ff_to_double(A11);
      }
      continue;
    }
    double al[LF_MAX_PLANES][2];
    double PA[LF_MAX_PLANES][4];   // Psi_j A_j, row-major
    for (int j = 0; j < MP.np; ++j) {
      double tx = t1x, ty = t1y;
      double a00 = 1, a01 = 0, a10 = 0, a11 = 1;
      for (int i = 0; i < j; ++i) {
        double r = MP.r[i][j];
        tx -= r * al[i][0];
        ty -= r * al[i][1];
        a00 -= r * PA[i][0]; a01 -= r * PA[i][1];
        a10 -= r * PA[i][2]; a11 -= r * PA[i][3];
      }
      PlaneLayout L = plane_layout<T, Mem>(MP.nc[j], MP.nm[j], MP.base[j]);
      const CompT<T>* dc = reinterpret_cast<const CompT<T>*>(smem + L.dc);
      const Mem* dm = reinterpret_cast<const Mem*>(smem + L.dm);
      double s[5];
      if constexpr (MIXED) {
        float xh[1], xl[1], yh[1], yl[1];
        split_ff(tx, xh[0], xl[0]);
        split_ff(ty, yh[0], yl[0]);
        ff acc[5][1];
        for (int v = 0; v < 5; ++v) acc[v][0] = ff_zero();
        if constexpr (MODE == LF_FF)
          accumulate_ext<1>(dc, MP.nc[j], dm, MP.nm[j], 0, MP.nc[j] + MP.nm[j], xh, xl, yh, yl, tab, acc);
        else
          accumulate_mixed<1>(dc, MP.nc[j], dm, MP.nm[j], 0, MP.nc[j] + MP.nm[j], chunk, xh, xl, yh,
                              yl, tab, acc);
        for (int v = 0; v < 5; ++v) s[v] = ff_to_double(acc[v][0]);
      } else {
        for (int v = 0; v < 5; ++v) s[v] = 0.0;
        accumulate_fp64(dc, MP.nc[j], dm, MP.nm[j], 0, MP.nc[j] + MP.nm[j], tx, ty, s);
      }
      al[j][0] = s[0];
      al[j][1] = s[1];
      // Psi_j A_j with Psi = [[pxx, pxy], [pxy, pyy]]
      PA[j][0] = s[2] * a00 + s[4] * a10;
      PA[j][1] = s[2] * a01 + s[4] * a11;
      PA[j][2] = s[4] * a00 + s[3] * a10;
      PA[j][3] = s[4] * a01 + s[3] * a11;
    }
    double bx = t1x, by = t1y, A00 = 1, A01 = 0, A10 = 0, A11 = 1;
    for (int j = 0; j < MP.np; ++j) {
      double r = MP.rs[j];
      bx -= r * al[j][0];
      by -= r * al[j][1];
      A00 -= r * PA[j][0]; A01 -= r * PA[j][1];
      A10 -= r * PA[j][2]; A11 -= r * PA[j][3];
    }
    if (io.beta) {
      io.beta[2 * p] = bx;
      io.beta[2 * p + 1] = by;
    }
    if (io.A) {
      io.A[4 * p] = A00; io.A[4 * p + 1] = A01;
      io.A[4 * p + 2] = A10; io.A[4 * p + 3] = A11;
    }
  }
}

// Fills the plane part of MultiPlaneArgs and returns the shared-memory bytes needed.
lf_status check_plane(const lf_plane* pl);

template <class T, class M>
lf_status fill_planes(const lf_plane* planes, int np, MultiPlaneArgs& A, uint32_t& total) {
  A.np = np;
  uint32_t base = LF_MAP_BASE;
  for (int j = 0; j < np; ++j) {
    LF_TRY(check_plane(&planes[j]));
    A.comp[j] = planes[j].comp;
    A.mem[j] = planes[j].mem;
    A.nc[j] = planes[j].n_comp;
    A.nm[j] = planes[j].n_mem;
    A.sc[j] = planes[j].scaling;
    A.base[j] = base;
    base = plane_layout<T, M>(planes[j].n_comp, planes[j].n_mem, base).total;
  }
  total = base;
  if (total > LF_SMEM_MAX) return fail(LF_EUNSUPPORTED, "planes too large for shared memory");
  return LF_OK;
}

}  // namespace lf

using namespace lf;

// The trace with a chosen block size (small blocks spread a few rays over many SMs).
lf_status lf::trace_rays(const lf_plane* planes, int32_t n_planes, const double* ratios, const double* theta,
                         int32_t n, const lf_grid* grid, int32_t precision, double* beta, double* A,
                         void* stream, int block) {
  if (!planes) return fail(LF_EINVAL, "planes is NULL");
  if (n_planes < 1 || n_planes > LF_MAX_PLANES) return fail(LF_EINVAL, "need 1 <= n_planes <= 8");
  if (!ratios) return fail(LF_EINVAL, "ratios is NULL");
  if (precision < LF_FP64 || precision > LF_FF) return fail(LF_EINVAL, "unknown precision");
  RayIO io{};
  if (theta) {
    if (n < 0) return fail(LF_EINVAL, "n must be >= 0");
    io.pts = theta;
    io.n = n;
  } else {
    if (!grid || grid->nx <= 0 || grid->ny <= 0) return fail(LF_EINVAL, "need theta or a grid");
    io.x0 = grid->x0; io.y0 = grid->y0; io.dx = grid->dx; io.dy = grid->dy; io.nx = grid->nx;
    io.n = (long long)grid->nx * grid->ny;
  }
  io.beta = beta;
  io.A = A;
  MultiPlaneArgs MP{};
  for (int i = 0; i < n_planes; ++i)
    for (int j = 0; j < n_planes; ++j) {
      double v = ratios[i * n_planes + j];
      if (j > i && !(std::isfinite(v) && v >= 0.0)) return fail(LF_EINVAL, "invalid ratio r[%d][%d]", i, j);
      MP.r[i][j] = j > i ? v : 0.0;
    }
  for (int j = 0; j < n_planes; ++j) {
    double v = ratios[n_planes * n_planes + j];
    if (!(std::isfinite(v) && v >= 0.0)) return fail(LF_EINVAL, "invalid source ratio %d", j);
    MP.rs[j] = v;
  }
  for (int i = 0; i < n_planes; ++i) {
    for (int j = 0; j < n_planes; ++j) {
      const float h = (float)MP.r[i][j];
      MP.rf[i][j] = make_float2(h, (float)(MP.r[i][j] - (double)h));
    }
    const float h = (float)MP.rs[i];
    MP.rsf[i] = make_float2(h, (float)(MP.rs[i] - (double)h));
  }
  uint32_t total = 0;
  if (precision == LF_MIXED) LF_TRY((fill_planes<float, MemT<float>>(planes, n_planes, MP, total)));
  else if (precision == LF_FF) LF_TRY((fill_planes<float, MemX>(planes, n_planes, MP, total)));
  else LF_TRY((fill_planes<double, MemT<double>>(planes, n_planes, MP, total)));
  if (io.n == 0) return LF_OK;
  int dev = 0, nsm = 0, occ = 0;
  LF_CUDA(cudaGetDevice(&dev));
  LF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = (cudaStream_t)stream;
  long long tiles = (io.n + block - 1) / block;
  auto k = precision == LF_MIXED ? k_trace<LF_MIXED> : precision == LF_FF ? k_trace<LF_FF> : k_trace<LF_FP64>;
  LF_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total));
  LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, block, total));
  long long g = std::min<long long>(tiles, (long long)nsm * std::max(occ, 1));
  k<<<(unsigned)g, block, total, s>>>(MP, io, g_member_chunk);
  LF_CUDA(cudaGetLastError());
  return LF_OK;
}

extern "C" lf_status lf_trace_multiplane(const lf_plane* planes, int32_t n_planes,
                                         const double* ratios, const double* theta, int32_t n,
                                         const lf_grid* grid, int32_t precision, double* beta,
                                         double* A, void* stream) {
  return trace_rays(planes, n_planes, ratios, theta, n, grid, precision, beta, A, stream, 256);
}
