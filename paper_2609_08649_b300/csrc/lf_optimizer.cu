// Multi-start Nelder-Mead (Nelder & Mead 1965), the paper's optimizer (Sec. 3.5), for M
// independent runs driving the batched chi^2 of a plan.  Coefficients and rules as in
// Lagarias et al. (1998): reflection 1, expansion 2, contraction 1/2, shrink 1/2; vertices
// ordered stably by chi^2 each iteration; a point outside the prior box [lo, hi] has
// chi^2 = +inf.  Every iteration evaluates the reflection point of every run in one chi^2
// launch and then the expansion or contraction point in a second; runs that shrink have
// their n new vertices evaluated in further launches (only when some run shrinks, which the
// host learns from a flag, once per iteration).  Vector arithmetic uses one IEEE operation
// per component (no contraction into fused multiply-adds), so the simplices follow the same
// operations as a plain implementation of the method.
#include "lf_internal.h"

namespace lf {

__device__ __forceinline__ bool in_box(const double* x, const double* lo, const double* hi, int P) {
  for (int p = 0; p < P; ++p)
    if (!(x[p] >= lo[p] && x[p] <= hi[p])) return false;
  return true;
}
__device__ __forceinline__ double boxed(double f, const double* x, const double* lo,
                                        const double* hi, int P) {
  return (isfinite(f) && in_box(x, lo, hi, P)) ? f : INFINITY;
}

// Orders each run's vertices stably by f, forms the centroid of the best n and the reflection
// point.  tmp: [M (P+1) P] scratch.
__global__ void k_nm_reflect(double* X, double* F, int M, int P, double* tmp, double* xb,
                             double* xr) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int n1 = P + 1;
  double* Xm = X + (size_t)m * n1 * P;
  double* Fm = F + (size_t)m * n1;
  int idx[LF_MAX_P + 1];
  for (int i = 0; i < n1; ++i) idx[i] = i;
  for (int i = 1; i < n1; ++i) {           // stable insertion sort of the vertex order
    const int k = idx[i];
    const double fk = Fm[k];
    int j = i - 1;
    while (j >= 0 && Fm[idx[j]] > fk) { idx[j + 1] = idx[j]; --j; }
    idx[j + 1] = k;
  }
  double* T = tmp + (size_t)m * n1 * P;
  double fs[LF_MAX_P + 1];
  for (int i = 0; i < n1; ++i) {
    for (int p = 0; p < P; ++p) T[(size_t)i * P + p] = Xm[(size_t)idx[i] * P + p];
    fs[i] = Fm[idx[i]];
  }
  for (int i = 0; i < n1; ++i) {
    for (int p = 0; p < P; ++p) Xm[(size_t)i * P + p] = T[(size_t)i * P + p];
    Fm[i] = fs[i];
  }
  const double dn = (double)P;
  for (int p = 0; p < P; ++p) {
    double s = Xm[p];
    for (int i = 1; i < P; ++i) s = __dadd_rn(s, Xm[(size_t)i * P + p]);
    const double c = __ddiv_rn(s, dn);
    xb[(size_t)m * P + p] = c;
    xr[(size_t)m * P + p] = __dadd_rn(c, __dsub_rn(c, Xm[(size_t)P * P + p]));
  }
}

// From f_r: the step of each run and its second point (expansion or contraction; the
// reflection point again when none is needed).  step: 0 reflect, 1 expand, 2 outside
// contraction, 3 inside contraction.
__global__ void k_nm_second(const double* X, const double* F, int M, int P, const double* lo,
                            const double* hi, const double* xb, const double* xr, double* fr,
                            double* x2, int* step) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int n1 = P + 1;
  const double* Xm = X + (size_t)m * n1 * P;
  const double* Fm = F + (size_t)m * n1;
  const double* b = xb + (size_t)m * P;
  const double* r = xr + (size_t)m * P;
  double* y = x2 + (size_t)m * P;
  const double f_r = boxed(fr[m], r, lo, hi, P);
  fr[m] = f_r;
  int s;
  if (f_r < Fm[0]) s = 1;
  else if (f_r < Fm[P - 1]) s = 0;
  else if (f_r < Fm[P]) s = 2;
  else s = 3;
  step[m] = s;
  for (int p = 0; p < P; ++p) {
    double v;
    if (s == 1) v = __dadd_rn(b[p], __dmul_rn(2.0, __dsub_rn(r[p], b[p])));
    else if (s == 2) v = __dadd_rn(b[p], __dmul_rn(0.5, __dsub_rn(r[p], b[p])));
    else if (s == 3) v = __dsub_rn(b[p], __dmul_rn(0.5, __dsub_rn(b[p], Xm[(size_t)P * P + p])));
    else v = r[p];
    y[p] = v;
  }
}

// Applies the step; runs that shrink get their new vertices in shrink[m][i - 1] (i = 1..n) and
// raise *any_shrink.  counts: per-step totals (0..4) or null.
__global__ void k_nm_apply(double* X, double* F, int M, int P, const double* lo, const double* hi,
                           const double* xr, const double* fr, const double* x2, const double* f2,
                           int* step, double* shrink, int* any_shrink, unsigned long long* counts) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int n1 = P + 1;
  double* Xm = X + (size_t)m * n1 * P;
  double* Fm = F + (size_t)m * n1;
  const double* r = xr + (size_t)m * P;
  const double* y = x2 + (size_t)m * P;
  const int s = step[m];
  const double f_r = fr[m];
  const double f_2 = s == 0 ? f_r : boxed(f2[m], y, lo, hi, P);
  const double* take = nullptr;
  double ftake = 0.0;
  bool shr = false;
  if (s == 0) { take = r; ftake = f_r; }
  else if (s == 1) { if (f_2 < f_r) { take = y; ftake = f_2; } else { take = r; ftake = f_r; } }
  else if (s == 2) { if (f_2 <= f_r) { take = y; ftake = f_2; } else shr = true; }
  else { if (f_2 < Fm[P]) { take = y; ftake = f_2; } else shr = true; }
  if (take) {
    for (int p = 0; p < P; ++p) Xm[(size_t)P * P + p] = take[p];
    Fm[P] = ftake;
  } else {
    for (int i = 1; i < n1; ++i)
      for (int p = 0; p < P; ++p) {
        const double v = __dadd_rn(Xm[p], __dmul_rn(0.5, __dsub_rn(Xm[(size_t)i * P + p], Xm[p])));
        Xm[(size_t)i * P + p] = v;
        shrink[((size_t)m * P + (i - 1)) * P + p] = v;
      }
    step[m] = 4;
    atomicOr(any_shrink, 1);
  }
  if (counts) atomicAdd(&counts[shr ? 4 : s], 1ull);
}

// The chi^2 of the shrunk vertices back into the simplices of the runs that shrank.
__global__ void k_nm_shrunk(double* F, int M, int P, const double* lo, const double* hi,
                            const int* step, const double* shrink, const double* fs) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= M * P) return;
  const int m = q / P, i = q - m * P;
  if (step[m] != 4) return;
  F[(size_t)m * (P + 1) + i + 1] = boxed(fs[q], shrink + (size_t)q * P, lo, hi, P);
}

}  // namespace lf

using namespace lf;

extern "C" lf_status lf_nm_run(lf_plan* plan, double* simplex, double* fvals, int32_t M,
                               int32_t n_iter, const double* lo, const double* hi,
                               unsigned long long* steps, void* stream) {
  if (!plan) return fail(LF_EINVAL, "plan is NULL");
  if (!simplex || !fvals || !lo || !hi) return fail(LF_EINVAL, "NULL argument");
  if (plan->n_clusters != 1) return fail(LF_EUNSUPPORTED, "the optimizer runs on single-cluster plans");
  if (M < 1 || M > plan->max_samples) return fail(LF_EINVAL, "need 1 <= M <= the plan's max_samples");
  if (n_iter < 0) return fail(LF_EINVAL, "n_iter must be >= 0");
  LF_TRY(ensure_nm_workspace(plan, M));
  cudaStream_t st = (cudaStream_t)stream;
  const int P = plan->P;
  NmWork& w = plan->nm;
  const int blk = 128, grd = (M + blk - 1) / blk;
  for (int it = 0; it < n_iter; ++it) {
    k_nm_reflect<<<grd, blk, 0, st>>>(simplex, fvals, M, P, w.tmp, w.xb, w.xr);
    LF_CUDA(cudaGetLastError());
    LF_TRY(launch_chi2(plan, w.xr, M, w.fr, nullptr, st));
    k_nm_second<<<grd, blk, 0, st>>>(simplex, fvals, M, P, lo, hi, w.xb, w.xr, w.fr, w.x2, w.step);
    LF_CUDA(cudaGetLastError());
    LF_TRY(launch_chi2(plan, w.x2, M, w.f2, nullptr, st));
    LF_CUDA(cudaMemsetAsync(w.flag, 0, sizeof(int), st));
    k_nm_apply<<<grd, blk, 0, st>>>(simplex, fvals, M, P, lo, hi, w.xr, w.fr, w.x2, w.f2, w.step,
                                    w.shrink, w.flag, steps);
    LF_CUDA(cudaGetLastError());
    LF_CUDA(cudaMemcpyAsync(w.flag_host, w.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LF_CUDA(cudaStreamSynchronize(st));
    if (*w.flag_host) {
      const long long n_pts = (long long)M * P;
      for (long long off = 0; off < n_pts; off += plan->max_samples) {
        const int cnt = (int)std::min<long long>(plan->max_samples, n_pts - off);
        LF_TRY(launch_chi2(plan, w.shrink + off * P, cnt, w.fs + off, nullptr, st));
      }
      k_nm_shrunk<<<(unsigned)((n_pts + blk - 1) / blk), blk, 0, st>>>(fvals, M, P, lo, hi, w.step,
                                                                      w.shrink, w.fs);
      LF_CUDA(cudaGetLastError());
    }
  }
  return LF_OK;
}
