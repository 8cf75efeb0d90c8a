// On-device posterior samplers of Sec. 3.5 driving the batched chi^2 of a plan: the
// affine-invariant ensemble sampler (Goodman & Weare 2010) and random-walk Metropolis-Hastings.
// AIES:  Likelihood exp(-chi^2/2), uniform
// priors on a box.  One step updates the two halves of the ensemble in turn: walker k of one
// half takes a partner j from the other half and z from g(z) ~ 1/sqrt(z) on [1/a, a],
// proposes y = x_j + z (x_k - x_j), and accepts with probability
// min(1, z^(P-1) exp(-(chi^2(y) - chi^2(x_k)) / 2)); proposals outside the box are rejected.
// The random numbers are inputs (three uniforms per walker and step), so that a run can be
// replayed exactly.  All of a step's work (proposals, the chi^2 of the proposals, the
// acceptance) stays on the device, on the caller's stream.
#include "lf_internal.h"

namespace lf {

// Proposals of one half.  u: this half's (u_partner, u_z, u_accept) rows.
__global__ void k_aies_propose(const double* __restrict__ x, int S, int P, int half,
                               const double* __restrict__ u, double a, const double* __restrict__ lo,
                               const double* __restrict__ hi, double* __restrict__ prop,
                               double* __restrict__ zs, int* __restrict__ inside) {
  const int h = S / 2;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= h) return;
  const int k = half == 0 ? n : h + n;
  const int oth = half == 0 ? h : 0;
  int j = (int)(u[3 * n] * h);
  j = j < h - 1 ? j : h - 1;
  const double t = (a - 1.0) * u[3 * n + 1] + 1.0;
  const double z = t * t / a;
  zs[n] = z;
  int in = 1;
  for (int p = 0; p < P; ++p) {
    const double xj = x[(size_t)(oth + j) * P + p];
    const double y = xj + z * (x[(size_t)k * P + p] - xj);
    prop[(size_t)n * P + p] = y;
    in &= (y >= lo[p]) && (y <= hi[p]);
  }
  inside[n] = in;
}

__global__ void k_aies_accept(double* __restrict__ x, double* __restrict__ chi2, int S, int P,
                              int half, const double* __restrict__ u, const double* __restrict__ prop,
                              const double* __restrict__ zs, const int* __restrict__ inside,
                              const double* __restrict__ chi2_new, unsigned long long* n_accept) {
  const int h = S / 2;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= h) return;
  const int k = half == 0 ? n : h + n;
  const double cn = chi2_new[n];
  bool acc = false;
  if (inside[n] && isfinite(cn)) {
    const double log_r = (P - 1) * log(zs[n]) - 0.5 * (cn - chi2[k]);
    acc = log(u[3 * n + 2]) < log_r;
  }
  if (acc) {
    for (int p = 0; p < P; ++p) x[(size_t)k * P + p] = prop[(size_t)n * P + p];
    chi2[k] = cn;
    if (n_accept) atomicAdd(n_accept, 1ull);
  }
}

// Random-walk Metropolis-Hastings (the paper's other sampler, Sec. 3.5): S independent
// chains, proposal y_k = x_k + step * z_k with caller-supplied standard normals z.
__global__ void k_mh_propose(const double* __restrict__ x, int S, int P, const double* __restrict__ z,
                             const double* __restrict__ step, const double* __restrict__ lo,
                             const double* __restrict__ hi, double* __restrict__ prop,
                             int* __restrict__ inside) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S) return;
  int in = 1;
  for (int p = 0; p < P; ++p) {
    const double y = x[(size_t)k * P + p] + step[p] * z[(size_t)k * P + p];
    prop[(size_t)k * P + p] = y;
    in &= (y >= lo[p]) && (y <= hi[p]);
  }
  inside[k] = in;
}

// Accepts y_k when it is in the box, chi^2(y_k) is finite and log u_k < -(chi^2(y) - chi^2(x))/2
// (a symmetric proposal has no Hastings factor).
__global__ void k_mh_accept(double* __restrict__ x, double* __restrict__ chi2, int S, int P,
                            const double* __restrict__ u, const double* __restrict__ prop,
                            const int* __restrict__ inside, const double* __restrict__ chi2_new,
                            unsigned long long* n_accept) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S) return;
  const double cn = chi2_new[k];
  if (inside[k] && isfinite(cn) && log(u[k]) < -0.5 * (cn - chi2[k])) {
    for (int p = 0; p < P; ++p) x[(size_t)k * P + p] = prop[(size_t)k * P + p];
    chi2[k] = cn;
    if (n_accept) atomicAdd(n_accept, 1ull);
  }
}

}  // namespace lf

using namespace lf;

extern "C" lf_status lf_mh_run(lf_plan* plan, double* chains, double* chi2, int32_t S,
                               int32_t n_steps, const double* normals, const double* uniforms,
                               const double* step, const double* lo, const double* hi, double* trace,
                               unsigned long long* n_accept, void* stream) {
  if (!plan) return fail(LF_EINVAL, "plan is NULL");
  if (!chains || !chi2 || !normals || !uniforms || !step || !lo || !hi)
    return fail(LF_EINVAL, "NULL argument");
  if (plan->n_clusters != 1) return fail(LF_EUNSUPPORTED, "the sampler runs on single-cluster plans");
  if (S < 1 || S > plan->max_samples) return fail(LF_EINVAL, "need 1 <= S <= the plan's max_samples");
  if (n_steps < 0) return fail(LF_EINVAL, "n_steps must be >= 0");
  LF_TRY(ensure_sampler_workspace(plan));
  cudaStream_t st = (cudaStream_t)stream;
  const int P = plan->P;
  const int blk = 128, grd = (S + blk - 1) / blk;
  for (int t = 0; t < n_steps; ++t) {
    k_mh_propose<<<grd, blk, 0, st>>>(chains, S, P, normals + (size_t)t * S * P, step, lo, hi,
                                      plan->d_prop, plan->d_inside);
    LF_CUDA(cudaGetLastError());
    LF_TRY(launch_chi2(plan, plan->d_prop, S, plan->d_chi2_prop, nullptr, st));
    k_mh_accept<<<grd, blk, 0, st>>>(chains, chi2, S, P, uniforms + (size_t)t * S, plan->d_prop,
                                     plan->d_inside, plan->d_chi2_prop, n_accept);
    LF_CUDA(cudaGetLastError());
    if (trace)
      LF_CUDA(cudaMemcpyAsync(trace + (size_t)t * S * P, chains, (size_t)S * P * sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
  }
  return LF_OK;
}

extern "C" lf_status lf_aies_run(lf_plan* plan, double* walkers, double* chi2, int32_t S,
                                 int32_t n_steps, const double* uniforms, double a,
                                 const double* lo, const double* hi, double* chain,
                                 unsigned long long* n_accept, void* stream) {
  if (!plan) return fail(LF_EINVAL, "plan is NULL");
  if (!walkers || !chi2 || !uniforms || !lo || !hi) return fail(LF_EINVAL, "NULL argument");
  if (plan->n_clusters != 1) return fail(LF_EUNSUPPORTED, "the sampler runs on single-cluster plans");
  if (S < 4 || (S & 1)) return fail(LF_EINVAL, "S must be even and >= 4");
  if (S / 2 > plan->max_samples) return fail(LF_EINVAL, "S/2 must not exceed the plan's max_samples");
  if (n_steps < 0) return fail(LF_EINVAL, "n_steps must be >= 0");
  if (!(a > 1.0 && std::isfinite(a))) return fail(LF_EINVAL, "the stretch scale a must be > 1");
  LF_TRY(ensure_sampler_workspace(plan));
  cudaStream_t st = (cudaStream_t)stream;
  const int P = plan->P, h = S / 2;
  const int blk = 128, grd = (h + blk - 1) / blk;
  for (int step = 0; step < n_steps; ++step) {
    for (int half = 0; half < 2; ++half) {
      const double* u = uniforms + ((size_t)step * S + (size_t)half * h) * 3;
      k_aies_propose<<<grd, blk, 0, st>>>(walkers, S, P, half, u, a, lo, hi, plan->d_prop,
                                          plan->d_z, plan->d_inside);
      LF_CUDA(cudaGetLastError());
      LF_TRY(launch_chi2(plan, plan->d_prop, h, plan->d_chi2_prop, nullptr, st));
      k_aies_accept<<<grd, blk, 0, st>>>(walkers, chi2, S, P, half, u, plan->d_prop, plan->d_z,
                                         plan->d_inside, plan->d_chi2_prop, n_accept);
      LF_CUDA(cudaGetLastError());
    }
    if (chain)
      LF_CUDA(cudaMemcpyAsync(chain + (size_t)step * S * P, walkers, (size_t)S * P * sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
  }
  return LF_OK;
}
