// lf_chi2_batch_static: the batched source-plane chi^2 of one cluster without any device
// allocation.
//
// Who needs it: callers that cannot call cudaMalloc.  Examples are a process whose GPU
// memory is already reserved by another framework's caching allocator, and plug-in
// environments that forbid device allocation outright.  lf_plan_create allocates the plan's
// tables; this entry point instead keeps every derived table (the cluster descriptor, the
// member factors, the image arrays, the work counter) in one fixed array of device memory
// that is part of the library image.  The caller still provides the inputs and the output.
//
// The call uploads its host-side tables (the descriptor, the member-array pointers and the
// image arrays, read from the caller's host memory and this function's stack) with
// cudaMemcpyAsync from pageable memory.  Such a copy first waits for the stream's earlier
// work, so the call returns to the host only once the stream has drained up to it.  It
// cannot be captured into a CUDA graph either (the copies would record host addresses that
// are gone at replay): a call on a capturing stream returns LF_EUNSUPPORTED before any work.
//
// The array is LF_STATIC_SCRATCH_BYTES (1 MiB) per device.  Every GPU that loads the library
// holds it until the process exits.  Every call uses the same array and leaves its
// contents behind; the work counter is cleared at the start of each call.  Two calls that
// overlap on the GPU (on different streams, or from different host threads) race on the
// array and must not be issued.
//
// Host code only sees a host-side stand-in for the array's name, so the device address
// is looked up once per device with cudaGetSymbolAddress the first time the entry point
// runs on that device (with that device current).  That first call therefore does a
// little set-up and should come before any stream capture.
#include "lf_internal.h"

#include <mutex>

namespace lf {

constexpr size_t LF_STATIC_SCRATCH_BYTES = size_t(1) << 20;

static __device__ __align__(256) unsigned char g_lf_static_scratch[LF_STATIC_SCRATCH_BYTES];

constexpr int LF_STATIC_MAX_DEVICES = 64;
static void* g_static_ptr[LF_STATIC_MAX_DEVICES];
static std::mutex g_static_mu;

static lf_status static_scratch(void** out) {
  int dev = 0;
  LF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= LF_STATIC_MAX_DEVICES) return fail(LF_EUNSUPPORTED, "device index %d too large", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_lf_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(LF_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return LF_OK;
}

// Fills the member factor tables and the image -> family map inside the scratch array.
template <class MemPre>
__global__ void k_static_prep(ClusterDesc* C, const lf_member* const* mems, int* img_fam,
                              float4* theta_ff, float4* sinv_f, float2* ratio_ff) {
  const ClusterDesc& cd = *C;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int i = tid; i < cd.n_img; i += nth) {
    float4 t, v;
    split_ff(cd.theta[2 * i], t.x, t.y);
    split_ff(cd.theta[2 * i + 1], t.z, t.w);
    v = make_float4((float)cd.sinv[3 * i], (float)cd.sinv[3 * i + 1], (float)cd.sinv[3 * i + 2], 0.f);
    theta_ff[i] = t;
    sinv_f[i] = v;
  }
  for (int q = tid; q < cd.n_fam * cd.np; q += nth) {
    float2 r;
    split_ff(cd.fam_ratio[q], r.x, r.y);
    ratio_ff[q] = r;
  }
  for (int j = 0; j < cd.np; ++j) {
    const PlaneDesc& P = cd.pl[j];
    MemPre* pre = const_cast<MemPre*>(reinterpret_cast<const MemPre*>(P.mpre));
    for (int i = tid; i < P.nm; i += nth) {
      const lf_member& m = mems[j][i];
      const double lnl = m.log_l * 2.302585092994045684;
      const double fb = exp(2.0 * P.sc.lam * lnl), fs = exp(P.sc.beta * lnl), fa = exp(P.sc.alpha * lnl);
      if constexpr (std::is_same<MemPre, MemPreF>::value) {
        MemPreF r;
        split_ff(m.x, r.xh, r.xl);
        split_ff(m.y, r.yh, r.yl);
        split_ff(fb, r.fb, r.fbl);
        split_ff(fs, r.fs, r.fsl);
        split_ff(fa, r.fa, r.fal);
        r.lnl = (float)lnl;
        r.pad = 0.f;
        pre[i] = r;
      } else {
        pre[i] = MemPreD{m.x, m.y, fb, fs, fa, lnl, 0.0, 0.0};
      }
    }
  }
  for (int f = tid; f < cd.n_fam; f += nth)
    for (int i = cd.fam_off[f]; i < cd.fam_off[f + 1]; ++i) img_fam[i] = f;
}

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace lf

using namespace lf;

extern "C" lf_status lf_chi2_batch_static(const lf_cluster* cl, const double* theta, int32_t S,
                                          int32_t precision, double* chi2, void* stream) {
  if (!cl || !theta || !chi2) return fail(LF_EINVAL, "cluster, theta and chi2 are required");
  if (S < 1) return fail(LF_EINVAL, "S must be >= 1");
  {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LF_CUDA(cudaStreamIsCapturing((cudaStream_t)stream, &cap));
    if (cap != cudaStreamCaptureStatusNone)
      return fail(LF_EUNSUPPORTED, "lf_chi2_batch_static copies host tables and cannot be captured");
  }
  if (precision < LF_FP64 || precision > LF_FF) return fail(LF_EINVAL, "unknown precision");
  if (cl->n_planes < 1 || cl->n_planes > LF_MAX_PLANES || !cl->planes || !cl->arcsec_per_kpc)
    return fail(LF_EINVAL, "cluster needs 1..8 planes and arcsec_per_kpc");
  if (cl->n_planes > 1 && !cl->ratios) return fail(LF_EINVAL, "multi-plane cluster needs ratios");
  const lf_images& im = cl->images;
  if (im.n_img < 1 || im.n_img > LF_MAX_IMG || im.n_fam < 1 || !im.theta_obs || !im.sinv ||
      !im.fam_off || !im.fam_ratio)
    return fail(LF_EINVAL, "incomplete image set (1..%d images)", LF_MAX_IMG);
  if (im.fam_off[0] != 0 || im.fam_off[im.n_fam] != im.n_img)
    return fail(LF_EINVAL, "fam_off must run from 0 to n_img");
  if (im.mag || im.td)
    return fail(LF_EUNSUPPORTED, "the static entry point has no flux or time-delay terms (use a plan)");
  for (int f = 0; f < im.n_fam; ++f)
    if (im.fam_off[f + 1] <= im.fam_off[f]) return fail(LF_EINVAL, "family %d is empty", f);
  for (int i = 0; i < im.n_img; ++i) {
    double a = im.sinv[3 * i], b = im.sinv[3 * i + 1], c = im.sinv[3 * i + 2];
    if (!(std::isfinite(im.theta_obs[2 * i]) && std::isfinite(im.theta_obs[2 * i + 1]) && a > 0 && c > 0 &&
          a * c - b * b > 0))
      return fail(LF_EINVAL, "image %d: non-finite position or S^-1 not positive definite", i);
  }
  const int np = cl->n_planes;
  for (int f = 0; f < im.n_fam; ++f)
    for (int l = 0; l < np; ++l) {
      double v = im.fam_ratio[f * np + l];
      if (!(std::isfinite(v) && (np == 1 ? (v > 0.0 && v <= 1.0) : (v >= 0.0 && v <= 1.0))))
        return fail(LF_EINVAL, "family %d has an invalid distance ratio", f);
    }

  // descriptor (host side, on the stack) -------------------------------------------
  ClusterDesc C;
  memset(&C, 0, sizeof C);
  C.np = np;
  int comp_base[LF_MAX_PLANES + 1] = {0};
  const lf_member* mems[LF_MAX_PLANES] = {nullptr};
  for (int j = 0; j < np; ++j) {
    const lf_plane& src = cl->planes[j];
    LF_TRY(check_plane(&src));
    PlaneDesc& P = C.pl[j];
    P.comp = src.comp;                 // staged by the kernel straight from the caller's array
    P.nc = src.n_comp;
    P.nm = src.n_mem;
    P.sc = src.scaling;
    P.apk = cl->arcsec_per_kpc[j];
    if (!(std::isfinite(P.apk) && P.apk > 0)) return fail(LF_EINVAL, "invalid arcsec_per_kpc");
    mems[j] = src.mem;
    comp_base[j + 1] = comp_base[j] + P.nc;
    if (np > 1)
      for (int l = 0; l < np; ++l) C.r[j][l] = (l > j) ? cl->ratios[j * np + l] : 0.0;
  }
  C.n_img = im.n_img;
  C.n_fam = im.n_fam;
  LF_TRY(parse_params(*cl, comp_base, C));
  // carve the scratch array -------------------------------------------------------------
  const size_t pre_sz = precision == LF_MIXED ? sizeof(MemPreF) : sizeof(MemPreD);
  size_t off = 0;
  const size_t o_desc = off; off = align256(off + sizeof(ClusterDesc));
  const size_t o_ctr = off; off = align256(off + 2 * sizeof(int));        // counter, order
  size_t o_pre[LF_MAX_PLANES];
  for (int j = 0; j < np; ++j) { o_pre[j] = off; off = align256(off + C.pl[j].nm * pre_sz); }
  const size_t o_mems = off; off = align256(off + np * sizeof(lf_member*));
  const size_t o_theta = off; off = align256(off + 2 * sizeof(double) * im.n_img);
  const size_t o_sinv = off; off = align256(off + 3 * sizeof(double) * im.n_img);
  const size_t o_ratio = off; off = align256(off + sizeof(double) * im.n_fam * np);
  const size_t o_off = off; off = align256(off + sizeof(int) * (im.n_fam + 1));
  const size_t o_if = off; off = align256(off + sizeof(int) * im.n_img);
  const size_t o_tff = off; off = align256(off + sizeof(float4) * im.n_img);
  const size_t o_sf = off; off = align256(off + sizeof(float4) * im.n_img);
  const size_t o_rff = off; off = align256(off + sizeof(float2) * im.n_fam * np);
  if (off > LF_STATIC_SCRATCH_BYTES)
    return fail(LF_EINVAL, "cluster needs %zu bytes of scratch, more than the %zu-byte static array "
                "(too many members or images for this entry point; use a plan)", off,
                LF_STATIC_SCRATCH_BYTES);

  const int block = std::min(256, chi2_max_block(precision));
  layout_cluster(C, precision, block, 32);
  if (C.smem > LF_SMEM_MAX) return fail(LF_EUNSUPPORTED, "cluster too large for shared memory");

  void* vbase = nullptr;
  LF_TRY(static_scratch(&vbase));
  unsigned char* base = static_cast<unsigned char*>(vbase);
  for (int j = 0; j < np; ++j) C.pl[j].mpre = base + o_pre[j];
  C.theta = reinterpret_cast<const double*>(base + o_theta);
  C.sinv = reinterpret_cast<const double*>(base + o_sinv);
  C.fam_ratio = reinterpret_cast<const double*>(base + o_ratio);
  C.fam_off = reinterpret_cast<const int*>(base + o_off);
  C.img_fam = reinterpret_cast<const int*>(base + o_if);
  C.theta_ff = reinterpret_cast<const float4*>(base + o_tff);
  C.sinv_f = reinterpret_cast<const float4*>(base + o_sf);
  C.ratio_ff = reinterpret_cast<const float2*>(base + o_rff);

  cudaStream_t st = (cudaStream_t)stream;
  LF_CUDA(cudaMemcpyAsync(base + o_desc, &C, sizeof C, cudaMemcpyHostToDevice, st));
  LF_CUDA(cudaMemcpyAsync(base + o_mems, mems, np * sizeof(lf_member*), cudaMemcpyHostToDevice, st));
  LF_CUDA(cudaMemcpyAsync(base + o_theta, im.theta_obs, 2 * sizeof(double) * im.n_img, cudaMemcpyHostToDevice, st));
  LF_CUDA(cudaMemcpyAsync(base + o_sinv, im.sinv, 3 * sizeof(double) * im.n_img, cudaMemcpyHostToDevice, st));
  LF_CUDA(cudaMemcpyAsync(base + o_ratio, im.fam_ratio, sizeof(double) * im.n_fam * np, cudaMemcpyHostToDevice, st));
  LF_CUDA(cudaMemcpyAsync(base + o_off, im.fam_off, sizeof(int) * (im.n_fam + 1), cudaMemcpyHostToDevice, st));
  LF_CUDA(cudaMemsetAsync(base + o_ctr, 0, 2 * sizeof(int), st));   // work counter = 0, order = {0}
  ClusterDesc* dC = reinterpret_cast<ClusterDesc*>(base + o_desc);
  const lf_member* const* dm = reinterpret_cast<const lf_member* const*>(base + o_mems);
  int* dif = reinterpret_cast<int*>(base + o_if);
  float4* dtf = reinterpret_cast<float4*>(base + o_tff);
  float4* dsf = reinterpret_cast<float4*>(base + o_sf);
  float2* drf = reinterpret_cast<float2*>(base + o_rff);
  if (precision == LF_MIXED) k_static_prep<MemPreF><<<32, 256, 0, st>>>(dC, dm, dif, dtf, dsf, drf);
  else k_static_prep<MemPreD><<<32, 256, 0, st>>>(dC, dm, dif, dtf, dsf, drf);
  LF_CUDA(cudaGetLastError());

  int dev = 0, nsm = 0, occ = 0;
  LF_CUDA(cudaGetDevice(&dev));
  LF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int* counter = reinterpret_cast<int*>(base + o_ctr);
  const int* order = counter + 1;
  const void* kfn = precision == LF_MIXED ? (const void*)k_chi2<LF_MIXED, false>
                    : precision == LF_FF  ? (const void*)k_chi2<LF_FF, false>
                                          : (const void*)k_chi2<LF_FP64, false>;
  LF_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C.smem));
  LF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, block, C.smem));
  const int grid = std::min(nsm * std::max(occ, 1), S);
  if (precision == LF_MIXED)
    k_chi2<LF_MIXED, false><<<grid, block, C.smem, st>>>(dC, order, S, S, theta, chi2, nullptr, counter, g_member_chunk, nullptr, nullptr);
  else if (precision == LF_FF)
    k_chi2<LF_FF, false><<<grid, block, C.smem, st>>>(dC, order, S, S, theta, chi2, nullptr, counter, g_member_chunk, nullptr, nullptr);
  else
    k_chi2<LF_FP64, false><<<grid, block, C.smem, st>>>(dC, order, S, S, theta, chi2, nullptr, counter, g_member_chunk, nullptr, nullptr);
  LF_CUDA(cudaGetLastError());
  return LF_OK;
}
