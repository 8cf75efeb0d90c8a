// Host-side helpers: error reporting, device error word, flat LCDM distances and the
// physical -> lensing unit conversions used to set up planes.
#include "lf_internal.h"

namespace lf {

#ifndef LF_CHUNK
#define LF_CHUNK 16
#endif
int g_member_chunk = LF_CHUNK;

static thread_local std::string g_last_error;

lf_status fail(lf_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

// 64-point Gauss-Legendre rule on [-1, 1], nodes found by Newton iteration on P_64.
struct GaussLegendre {
  static constexpr int N = 64;
  double x[N], w[N];
  GaussLegendre() {
    for (int i = 0; i < N; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (N + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= N; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        double dp = N * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) {
          x[i] = z;
          w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
          break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
      }
    }
  }
};

static const GaussLegendre& gl() {
  static GaussLegendre g;
  return g;
}

static double inv_E(double z, double Om) {
  return 1.0 / std::sqrt(Om * (1.0 + z) * (1.0 + z) * (1.0 + z) + 1.0 - Om);
}

// int_{z1}^{z2} dz / E(z), split into panels of width <= 0.5 for ~1e-15 accuracy.
static double comoving_integral(double z1, double z2, double Om) {
  if (z2 <= z1) return 0.0;
  const GaussLegendre& g = gl();
  int panels = std::max(1, (int)std::ceil((z2 - z1) / 0.5));
  double h = (z2 - z1) / panels, sum = 0.0;
  for (int p = 0; p < panels; ++p) {
    double a = z1 + p * h, c = a + 0.5 * h;
    for (int i = 0; i < GaussLegendre::N; ++i) sum += g.w[i] * inv_E(c + 0.5 * h * g.x[i], Om);
  }
  return sum * 0.5 * h;
}

constexpr double C_KMS = 299792.458;
constexpr double ARCSEC_PER_RAD = 180.0 / M_PI * 3600.0;
constexpr double G_MPC_MSUN_KMS2 = 4.300917270e-9;

}  // namespace lf

using namespace lf;

extern "C" double lf_angular_distance(double H0, double Om, double z1, double z2) {
  return C_KMS / H0 * comoving_integral(z1, z2, Om) / (1.0 + z2);
}

extern "C" double lf_adis(double H0, double Om, double z_l, double z_s) {
  if (z_s <= z_l) return 0.0;
  return lf_angular_distance(H0, Om, z_l, z_s) / lf_angular_distance(H0, Om, 0.0, z_s);
}

extern "C" double lf_arcsec_per_kpc(double H0, double Om, double z) {
  return ARCSEC_PER_RAD / (lf_angular_distance(H0, Om, 0.0, z) * 1000.0);
}

extern "C" double lf_td_scale(double H0, double Om, double z_d) {
  constexpr double KM_PER_MPC = 3.0856775814913673e19, S_PER_DAY = 86400.0;
  const double dd_km = lf_angular_distance(H0, Om, 0.0, z_d) * KM_PER_MPC;
  const double theta0 = 1.0 / ARCSEC_PER_RAD;
  return (1.0 + z_d) * dd_km / C_KMS * theta0 * theta0 / S_PER_DAY;
}

extern "C" double lf_b_from_vdisp(double v_kms) {
  double r = v_kms / C_KMS;
  return 4.0 * M_PI * r * r * ARCSEC_PER_RAD;
}

extern "C" lf_status lf_nfw_params(double H0, double Om, double z_l, double m200, double conc,
                                   double* kappa_s, double* theta_s) {
  if (!kappa_s || !theta_s) return fail(LF_EINVAL, "NULL output");
  if (!(m200 > 0 && conc > 0 && z_l > 0)) return fail(LF_EINVAL, "need m200, conc, z_l > 0");
  double Ez2 = Om * std::pow(1.0 + z_l, 3) + 1.0 - Om;
  double rho_c = 3.0 * H0 * H0 * Ez2 / (8.0 * M_PI * G_MPC_MSUN_KMS2);        // Msun / Mpc^3
  double r200 = std::cbrt(3.0 * m200 / (4.0 * M_PI * 200.0 * rho_c));          // Mpc
  double rs = r200 / conc;
  double delta_c = 200.0 / 3.0 * conc * conc * conc / (std::log1p(conc) - conc / (1.0 + conc));
  double dd = lf_angular_distance(H0, Om, 0.0, z_l);
  double sigma_cr = C_KMS * C_KMS / (4.0 * M_PI * G_MPC_MSUN_KMS2 * dd);        // Msun / Mpc^2
  *kappa_s = delta_c * rho_c * rs / sigma_cr;
  *theta_s = rs / dd * ARCSEC_PER_RAD;
  return LF_OK;
}

extern "C" lf_status lf_comp_from_physical(const lf_phys_comp* in, double H0, double Om, double z_l,
                                           lf_comp* out) {
  if (!in || !out) return fail(LF_EINVAL, "NULL argument");
  auto given = [](double v) { return !std::isnan(v); };
  lf_comp c;
  memset(&c, 0, sizeof c);
  c.kind = in->kind;
  c.x = in->x;
  c.y = in->y;
  c.pa = in->pa_deg * (M_PI / 180.0);
  switch (in->kind) {
    case LF_SIE:
    case LF_DPIE: {
      if (!(in->eps >= 0.0 && in->eps < 1.0)) return fail(LF_EINVAL, "eps must be in [0, 1)");
      const double q = (1.0 - in->eps) / (1.0 + in->eps);
      if (given(in->vdisp)) {
        c.b = lf_b_from_vdisp(in->vdisp);
      } else if (given(in->theta_e) && given(in->z_ref)) {
        // the area-equivalent Einstein radius at z_ref: theta_E = a_dis b sqrt(q)
        const double a = lf_adis(H0, Om, z_l, in->z_ref);
        if (!(a > 0.0)) return fail(LF_EINVAL, "z_ref must lie behind the lens");
        c.b = in->theta_e / (std::sqrt(q) * a);
      } else {
        return fail(LF_EINVAL, "an isothermal component needs vdisp or (theta_e, z_ref)");
      }
      const double apk = lf_arcsec_per_kpc(H0, Om, z_l);
      if (given(in->core_arcsec)) c.core = in->core_arcsec;
      else if (given(in->core_kpc)) c.core = in->core_kpc * apk;
      else return fail(LF_EINVAL, "an isothermal component needs a core radius");
      c.cut = given(in->cut_kpc) ? in->cut_kpc * apk : 0.0;
      c.eps = in->eps;
      break;
    }
    case LF_NFW:
    case LF_ENFW: {
      if (given(in->kappa_s) && given(in->theta_s)) {
        if (!(std::isfinite(in->kappa_s) && in->theta_s > 0.0 && std::isfinite(in->theta_s)))
          return fail(LF_EINVAL, "need a finite kappa_s and theta_s > 0");
        c.b = in->kappa_s;
        c.core = in->theta_s;
      } else {
        LF_TRY(lf_nfw_params(H0, Om, z_l, in->m200, in->conc, &c.b, &c.core));
      }
      if (in->kind == LF_NFW) {
        c.pa = 0.0;
      } else {
        if (!(in->eps >= 0.0 && in->eps < 1.0)) return fail(LF_EINVAL, "eps must be in [0, 1)");
        c.eps = in->eps;
      }
      break;
    }
    case LF_SHEAR: {
      // a shear quoted at source redshift z_ref carries that a_dis; the tables hold a_dis = 1
      c.b = in->gamma;
      if (given(in->z_ref)) {
        const double a = lf_adis(H0, Om, z_l, in->z_ref);
        if (!(a > 0.0)) return fail(LF_EINVAL, "z_ref must lie behind the lens");
        c.b /= a;
      }
      break;
    }
    case LF_MULTIPOLE3:
      c.b = in->amp;
      break;
    default:
      return fail(LF_EINVAL, "unknown component kind %d", in->kind);
  }
  *out = c;
  return LF_OK;
}

extern "C" lf_status lf_scaling_from_physical(double vstar_kms, double core_star_kpc, double cut_star_kpc,
                                              double lam, double beta, double alpha, double H0, double Om,
                                              double z_l, lf_scaling* out) {
  if (!out) return fail(LF_EINVAL, "NULL output");
  if (!(vstar_kms >= 0 && core_star_kpc >= 0 && cut_star_kpc > 0 && z_l > 0))
    return fail(LF_EINVAL, "need v* >= 0, core* >= 0, cut* > 0 and z_l > 0");
  const double apk = lf_arcsec_per_kpc(H0, Om, z_l);
  out->b_star = lf_b_from_vdisp(vstar_kms);
  out->core_star = core_star_kpc * apk;
  out->cut_star = cut_star_kpc * apk;
  out->lam = lam;
  out->beta = beta;
  out->alpha = alpha;
  return LF_OK;
}

extern "C" lf_status lf_multiplane_ratios(double H0, double Om, const double* z_planes, int32_t n_planes,
                                          double z_s, double* ratios) {
  if (!z_planes || !ratios || n_planes < 1 || n_planes > LF_MAX_PLANES)
    return fail(LF_EINVAL, "need 1..%d plane redshifts and an output table", LF_MAX_PLANES);
  for (int j = 0; j < n_planes; ++j) {
    if (!(z_planes[j] > 0.0) || (j > 0 && !(z_planes[j] > z_planes[j - 1])))
      return fail(LF_EINVAL, "plane redshifts must be positive and increasing");
  }
  const int n = n_planes;
  for (int j = 0; j < n; ++j) {
    const double dj = lf_angular_distance(H0, Om, 0.0, z_planes[j]);
    for (int i = 0; i < n; ++i)
      ratios[i * n + j] = i < j ? lf_angular_distance(H0, Om, z_planes[i], z_planes[j]) / dj : 0.0;
  }
  const double ds = lf_angular_distance(H0, Om, 0.0, z_s);
  for (int j = 0; j < n; ++j)
    ratios[n * n + j] = z_s > z_planes[j] ? lf_angular_distance(H0, Om, z_planes[j], z_s) / ds : 0.0;
  return LF_OK;
}

extern "C" lf_status lf_device_error(void* stream) {
  LF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned int v = 0, zero = 0;
  LF_CUDA(cudaMemcpyFromSymbol(&v, g_lf_err, sizeof v));
  LF_CUDA(cudaMemcpyToSymbol(g_lf_err, &zero, sizeof zero));
  if (v & LF_DEVERR_TIMEOUT) return fail(LF_ETIMEOUT, "a bounded device wait ran out");
  if (v & LF_DEVERR_BADCOMP) return fail(LF_EINVAL, "an invalid component was skipped on the device");
  if (v & LF_DEVERR_BADARG) return fail(LF_EINVAL, "an invalid per-source argument was skipped on the device");
  if (v & LF_DEVERR_BOUNDS) return fail(LF_EINVAL, "an index check failed on the device (LF_CHECK_BOUNDS build)");
  return LF_OK;
}

extern "C" const char* lf_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* lf_version(void) { return "lf-b300 0.1 (sm_103a)"; }
