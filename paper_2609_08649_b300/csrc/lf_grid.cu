// Grid / point maps of alpha, kappa, gamma and mu (Sec. 2.1; Eq. lens_eq, Eq. jac).
//
// Persistent kernels: one block per SM slot stages the component and member tables
// into shared memory once with the bulk-copy engine, digests them (member scaling
// relations of Eq. scaling, trigonometry, float-float centres), then walks pixel tiles
// with a grid stride.  Every thread owns PPT positions so that each component read from
// shared memory (a broadcast) is reused PPT times.
//
//  LF_MIXED: per-component closed forms in FP32 on float-float offsets; per-chunk FP32 sums
//            folded into float-float accumulators every `chunk` members; FP64 det A and mu.
//  LF_FP64:  the same loop in FP64 throughout, one position per thread.
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

// ------------------------------------------------------------------- LF_MIXED ------
#ifndef LF_MAP_MINB
#define LF_MAP_MINB 3   // scalar and float-float variants: at most 85 registers, 3 blocks of 256
#endif
#ifndef LF_MAP_MINB_PACK
#define LF_MAP_MINB_PACK 4   // packed variant: 64 registers, 4 blocks of 256 per SM
#endif
#ifndef LF_MAP_PACK
#define LF_MAP_PACK 1   // members in packed pairs (f32x2)
#endif
#ifndef LF_MAP_PPT
#define LF_MAP_PPT 1
#endif
#ifndef LF_MAP_CHUNK
#define LF_MAP_CHUNK 16   // packed variant: member pairs per FP32 partial sum (16 terms per lane)
#endif
// Member record of each variant: float-float (EXT), packed pairs (PACK), or scalar.
template <bool EXT, bool PACK>
using MapMem = typename std::conditional<EXT, MemX,
                                         typename std::conditional<PACK, MemPair, MemT<float>>::type>::type;

template <int PPT, bool EXT, bool PACK>
__global__ void __launch_bounds__(256, PACK ? LF_MAP_MINB_PACK : LF_MAP_MINB) k_map_mixed(const lf_comp* __restrict__ comp, int nc,
                                                   const lf_member* __restrict__ mem, int nm,
                                                   lf_scaling sc, PosArgs P, OutArgs O, int chunk) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  typedef MapMem<EXT, PACK> Mem;
  const PlaneLayout L = plane_layout<float, Mem>(nc, nm, LF_MAP_BASE);
  lf_comp* rawc = reinterpret_cast<lf_comp*>(smem + L.rawc);
  lf_member* rawm = reinterpret_cast<lf_member*>(smem + L.rawm);
  CompT<float>* dc = reinterpret_cast<CompT<float>*>(smem + L.dc);
  Mem* dm = reinterpret_cast<Mem*>(smem + L.dm);
  float2* tab = reinterpret_cast<float2*>(smem + 16);
  if (threadIdx.x == 0) mbar_init(bar, 1);
  init_ff_tables(tab);
  __syncthreads();
  bool ok = stage_to_smem(rawc, comp, (uint32_t)nc * 64u + 0u, bar, 0);
  if (ok) ok = stage_to_smem(rawm, mem, (uint32_t)nm * 32u, bar, nc > 0 ? 1 : 0);
  if (!ok) return;
  if constexpr (EXT) digest_plane_x(rawc, nc, rawm, nm, sc, dc, dm);
  else if constexpr (PACK) digest_plane_pairs(rawc, nc, rawm, nm, sc, dc, dm);
  else digest_plane<float>(rawc, nc, rawm, nm, sc, dc, dm);
  __syncthreads();

  const long long per_tile = (long long)PPT * blockDim.x;
  const long long n_tiles = (P.n + per_tile - 1) / per_tile;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    float pxh[PPT], pxl[PPT], pyh[PPT], pyl[PPT];
    long long pid[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      pid[k] = tile * per_tile + threadIdx.x + (long long)k * blockDim.x;
      double x, y;
      position_of(P, pid[k] < P.n ? pid[k] : 0, x, y);
      split_ff(x, pxh[k], pxl[k]);
      split_ff(y, pyh[k], pyl[k]);
    }
    ff acc[5][PPT];
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int k = 0; k < PPT; ++k) acc[v][k] = ff_zero();

    if constexpr (EXT) accumulate_ext<PPT>(dc, nc, dm, nm, 0, nc + nm, pxh, pxl, pyh, pyl, tab, acc);
    else if constexpr (PACK)
      accumulate_packed<PPT>(dc, nc, dm, nm, 0, nc + (int)mem_records<MemPair>(nm), chunk, pxh, pxl,
                             pyh, pyl, tab, acc);
    else accumulate_mixed<PPT>(dc, nc, dm, nm, 0, nc + nm, chunk, pxh, pxl, pyh, pyl, tab, acc);
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if (pid[k] < P.n)
        write_out(O, pid[k], ff_to_double(acc[0][k]), ff_to_double(acc[1][k]),
                  ff_to_double(acc[2][k]), ff_to_double(acc[3][k]), ff_to_double(acc[4][k]));
    }
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

template <int PPT, bool EXT, bool PACK>
static lf_status launch_mixed(const lf_plane* pl, const PosArgs& P, const OutArgs& O, int nsm,
                              int block, cudaStream_t s) {
  typedef MapMem<EXT, PACK> Mem;
  PlaneLayout L = plane_layout<float, Mem>(pl->n_comp, pl->n_mem, LF_MAP_BASE);
  if (L.total > LF_SMEM_MAX) return fail(LF_EUNSUPPORTED, "plane too large for shared memory");
  auto k = k_map_mixed<PPT, EXT, PACK>;
  LF_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
  int occ = 0;
  LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, block, L.total));
  long long tiles = (P.n + (long long)PPT * block - 1) / ((long long)PPT * block);
  long long grid = std::min<long long>(tiles, (long long)nsm * std::max(occ, 1));
  k<<<(unsigned)grid, block, L.total, s>>>(pl->comp, pl->n_comp, pl->mem, pl->n_mem, pl->scaling, P, O,
                                           PACK ? LF_MAP_CHUNK : g_member_chunk);
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
#if LF_MAP_PACK
    LF_TRY((launch_mixed<LF_MAP_PPT, false, true>(pl, P, O, nsm, block, s)));
#else
    LF_TRY((launch_mixed<LF_MAP_PPT, false, false>(pl, P, O, nsm, block, s)));
#endif
  } else if (precision == LF_FF) {
    LF_TRY((launch_mixed<1, true, false>(pl, P, O, nsm, block, s)));
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
