/*
 * lf.h -- C ABI of the B300 (sm_103a) batched lens-equation / source-plane chi^2 library.
 *
 * The library evaluates the paper's strong-lensing forward model on the GPU:
 *   - deflection alpha and deformation tensor psi_ij summed over analytic components
 *     (cored isothermal ellipsoid, dPIE / pseudo-Jaffe ellipsoid, spherical NFW, external
 *     shear) and over cluster members on the luminosity scaling relations
 *     (Sec. 2.1; Sec. 3.4, Eq. scaling);
 *   - the lens map beta = theta - a_dis alpha (Eq. lens_eq), the Jacobian
 *     A = I - a_dis psi_ij (Eq. jac), kappa, gamma and mu = 1/det A (Sec. 2.1);
 *   - multi-plane ray tracing with the Jacobian product (Sec. 2.2);
 *   - the source-plane chi^2 with the analytic best-fit source (Eq. chi2_src, Sec. 3.1)
 *     for thousands of parameter samples per launch, and its gradient with respect to the
 *     parameters (the paper has no gradient; it is the hand-written adjoint of that chi^2).
 *
 * Conventions (Sec. 2.1): angles in arcsec; the potential carries no a_dis, so every
 * strength is its a_dis = 1 value; position angles are radians counter-clockwise from +x;
 * ellipticity eps = (1 - q)/(1 + q).  kappa and gamma returned by the grid calls are the
 * paper's a_dis-free values; mu includes a_dis.
 *
 * Memory: arrays documented "device" are caller-owned device memory, read or written
 * stream-ordered on `stream` (a cudaStream_t passed as void*; NULL = legacy default
 * stream).  Arrays documented "host" are read during the call only.  No call allocates
 * device memory except lf_plan_create, which owns everything it allocates until
 * lf_plan_destroy.  Every call is asynchronous with respect to the host.
 *
 * Errors: every call validates its arguments before launching anything and returns
 * LF_EINVAL (with a message in lf_last_error()) on a bad argument; LF_ECUDA when a CUDA
 * call fails (including an earlier asynchronous fault that surfaces at launch);
 * LF_EUNSUPPORTED for a valid request outside what the kernels implement.  Kernels never
 * trap: a bounded wait that runs out sets a device error word that lf_device_error()
 * reads and clears (LF_ETIMEOUT).  Nothing aborts the process.
 */
#ifndef LF_H_
#define LF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LF_OK = 0,
  LF_EINVAL = 1,
  LF_ECUDA = 2,
  LF_ENOMEM = 3,
  LF_ETIMEOUT = 4,
  LF_EUNSUPPORTED = 5
} lf_status;

/* Component kinds (Sec. 2.1 profile library; closed forms after Keeton 2001). */
typedef enum {
  LF_SIE = 1,    /* cored isothermal ellipsoid: b, eps, pa, core (= s)                 */
  LF_DPIE = 2,   /* dPIE / pseudo-Jaffe ellipsoid: b, eps, pa, core, cut; eps = 0 is round */
  LF_NFW = 3,    /* spherical NFW: b = kappa_s, core = theta_s (scale radius, arcsec)  */
  LF_SHEAR = 4,  /* external shear: b = gamma, pa = shear angle; x, y = reference point */
  LF_MULTIPOLE3 = 5, /* third-order multipole with a theta^2 potential (Sec. 4.2):
                        psi = b r^2 cos 3(phi - pa) about (x, y); eps, core, cut unused */
  LF_ENFW = 6        /* elliptical NFW (Sec. 4.1-4.2, approximated as in Oguri 2021): b = kappa_s,
                        core = theta_s, eps, pa; kappa = 2 kappa_s g(xi / theta_s),
                        xi^2 = u^2 + v^2/q^2, with g the spherical NFW's convergence written as a
                        sum of 38 cored steep ellipsoids (relative error < 2e-6 for
                        1e-4 < xi / theta_s < 1e3); cut unused */
} lf_kind;

/* LF_FP64: every operation in FP64, one thread per position (the plain comparator).
 * LF_MIXED: per-component closed forms in FP32 on offsets taken in float-float (the
 * deflection of elliptical isothermal components and of the shear in float-float), FP32
 * sums per member chunk folded into float-float accumulators, then FP64 for det A, mu, the
 * multi-plane Jacobian product and the chi^2 reduction.  The maps (lf_deflect_grid,
 * lf_jacobian_grid, lf_jacobian_points, lf_jacobian_grid_host) anchor each tile of 16 x 16
 * pixels (or 256 points) at its centre: every member's deflection there in float-float,
 * its change across the tile in FP32 from cancellation-free differences, members that
 * change fast across the tile and every explicit component in float-float; alpha within
 * 1e-6 arcsec of FP64 at cluster scale, psi_ij FP32.
 * LF_FF: as LF_MIXED, but the deflection of every member is also carried in float-float
 * (about 48 significant bits on the FP32 pipe) and accumulated in float-float; psi_ij
 * stays FP32.  Spherical NFW components stay FP32 in the mixed tier's chi^2 and trace
 * kernels. */
typedef enum { LF_FP64 = 0, LF_MIXED = 1, LF_FF = 2 } lf_precision;

/* One explicit component, 64 bytes (device arrays of these are staged into shared
 * memory by bulk copy, so the array must be 16-byte aligned). */
typedef struct {
  double x, y;     /* centre, arcsec */
  double b;        /* strength at a_dis = 1 (arcsec; kappa_s for NFW; gamma for shear) */
  double eps;      /* ellipticity (1-q)/(1+q), 0 <= eps < 1 */
  double pa;       /* position angle, radians CCW from +x */
  double core;     /* core radius s (arcsec); NFW scale radius theta_s */
  double cut;      /* dPIE truncation radius (arcsec), cut > core */
  int32_t kind;    /* lf_kind */
  int32_t pad;
} lf_comp;

/* One cluster member, 32 bytes: a round pseudo-Jaffe galaxy whose strength, core and
 * cut follow the scaling relations of Eq. scaling from its luminosity. */
typedef struct {
  double x, y;     /* centre, arcsec */
  double log_l;    /* log10(L / L*) */
  double pad;
} lf_member;

/* Eq. scaling in lensing units: v = v* (L/L*)^lam, so b = b* (L/L*)^(2 lam);
 * core = core* (L/L*)^beta; cut = cut* (L/L*)^alpha. */
typedef struct {
  double b_star;     /* arcsec, = 4 pi (v_star / c)^2 */
  double core_star;  /* arcsec */
  double cut_star;   /* arcsec */
  double lam, beta, alpha;
} lf_scaling;

/* One lens plane. */
typedef struct {
  int32_t n_comp;            /* >= 0 */
  int32_t n_mem;             /* >= 0 */
  const lf_comp* comp;       /* device [n_comp], 16-byte aligned (NULL if n_comp == 0) */
  const lf_member* mem;      /* device [n_mem], 16-byte aligned (NULL if n_mem == 0) */
  lf_scaling scaling;        /* host values, used when n_mem > 0 */
} lf_plane;

/* Pixel-centre grid: pixel (i, j) sits at (x0 + i dx, y0 + j dy); outputs are row-major
 * with y the slow index, element j * nx + i. */
typedef struct {
  double x0, y0, dx, dy;
  int32_t nx, ny;
} lf_grid;

/* ---------------------------------------------------------------- grid maps ------ */

/* alpha on a grid (Sec. 2.1, alpha = grad psi).  ax, ay: device [ny * nx] FP64. */
lf_status lf_deflect_grid(const lf_plane* plane, const lf_grid* grid, int32_t precision,
                          double* ax, double* ay, void* stream);

/* alpha, kappa, gamma1, gamma2 and mu = 1/det A with det A = (1 - a kappa)^2 - a^2 |gamma|^2
 * evaluated in FP64 (Eq. jac and the magnification below it).  Any output pointer may be
 * NULL to skip it.  ax, ay, mu: device FP64 [ny * nx]; kappa, g1, g2: device FP32.
 * a_dis in (0, 1]. */
lf_status lf_jacobian_grid(const lf_plane* plane, const lf_grid* grid, double a_dis,
                           int32_t precision, double* ax, double* ay, float* kappa,
                           float* g1, float* g2, double* mu, void* stream);

/* The maps of lf_jacobian_grid written to HOST memory, with the device-to-host copies
 * overlapped with the computation (the paper has no counterpart: this is the I/O path of the
 * Sec. 2.1 maps).  The grid is split into at most `bands` bands of whole rows, each a
 * multiple of 16 rows (the mixed maps' tile height; the last band may be shorter).  Each band is computed on `stream` into one of two device slots of
 * `workspace` while the previous band is copied to the host on a second stream owned by the
 * library (one per device, created on first use).
 * ax, ay, kappa, g1, g2, mu: HOST [ny * nx] row-major, types as in lf_jacobian_grid; any may
 *   be NULL (all NULL: nothing is computed).  Page-locked (pinned) memory lets the copies
 *   run concurrently with the computation; pageable memory gives the same results without
 *   the overlap.  The caller must not touch them until `stream` has been synchronised.
 * workspace: device, 256-byte aligned, at least lf_jacobian_grid_host_workspace(grid, bands)
 *   bytes, owned by the caller and reusable once the call's work on `stream` has finished.
 * The work is ordered on `stream`: it starts after the caller's earlier work there, and
 * later work there runs after the last copy.
 * Band k's rows start at y0 + r0 dy (r0 = its first row), so FP64 pixel positions may differ
 * from one lf_jacobian_grid call over the whole grid by one rounding (about 1e-16 relative);
 * the first band's are identical.
 * Errors: LF_EINVAL (invalid grid, plane, a_dis, precision, bands < 1, or a missing,
 * undersized or misaligned workspace) before any launch; LF_ECUDA from the CUDA runtime. */
size_t lf_jacobian_grid_host_workspace(const lf_grid* grid, int32_t bands);
lf_status lf_jacobian_grid_host(const lf_plane* plane, const lf_grid* grid, double a_dis,
                                int32_t precision, double* ax, double* ay, float* kappa,
                                float* g1, float* g2, double* mu, int32_t bands,
                                void* workspace, size_t workspace_bytes, void* stream);

/* Same quantities at arbitrary positions: theta device [n * 2] FP64 (x, y interleaved). */
lf_status lf_jacobian_points(const lf_plane* plane, const double* theta, int32_t n,
                             double a_dis, int32_t precision, double* ax, double* ay,
                             float* kappa, float* g1, float* g2, double* mu, void* stream);

/* ------------------------------------------------------------- multi-plane ------- */

/* Multi-plane lens equation and Jacobian (Sec. 2.2):
 *   theta_j = theta_1 - sum_{i<j} r[i][j] alpha_i(theta_i),
 *   A_j = I - sum_{i<j} r[i][j] psi_i(theta_i) A_i,
 *   beta = theta_1 - sum_j rs[j] alpha_j(theta_j),  A = I - sum_j rs[j] psi_j A_j,
 * with r[i][j] = D_ij / D_j and rs[j] = D_js / D_s.
 * planes: host [n_planes] (1 <= n_planes <= 8), ordered by redshift.
 * ratios: host [(n_planes + 1) * n_planes]: row i < n_planes holds r[i][0..n_planes-1]
 *   (only j > i is read), the last row holds rs[0..n_planes-1].
 * Positions: theta device [n * 2] FP64, or theta == NULL and `grid` (n ignored).
 * beta: device [n * 2] FP64; A: device [n * 4] FP64 row-major (A00, A01, A10, A11);
 * either may be NULL.
 * Precision: LF_FP64 computes everything in FP64.  LF_MIXED evaluates the components in FP32
 * on float-float offsets, carries theta_j, the deflections and beta in float-float, and
 * forms the Jacobian product in FP32.  LF_FF evaluates the deflections in float-float and
 * keeps the recursion in FP64. */
lf_status lf_trace_multiplane(const lf_plane* planes, int32_t n_planes, const double* ratios,
                              const double* theta, int32_t n, const lf_grid* grid,
                              int32_t precision, double* beta, double* A, void* stream);

/* ---------------------------------------------------------- image finder ------- */

/* Lens-equation solver of Sec. 2.3: the images of a source beta are the common zeros of
 * f(theta) = beta - theta + a alpha(theta).  Each component's zero contour is traced over the
 * vertex grid `grid` (vertices x0 + i dx, y0 + j dy, i < nx, j < ny; nx, ny >= 2) by marching
 * squares (linear interpolation along cell edges, a saddle cell resolved by its centre value,
 * f > 0 counted as positive), and the images are the exact intersections of pairs of contour
 * segments in one cell (segment parameters within [0, 1] up to 1e-12).  Candidates are
 * ordered by cell (row-major) and segment pair and merged when closer than 1e-6 dx.  With
 * polish_iters > 0 each image is then refined by up to polish_iters Newton steps
 * theta <- theta - A^-1 (theta - a alpha - beta), evaluated in FP64, stopping once the
 * residual is below 1e-12; images closer than 1e-7 (arcsec) after the polish are merged and
 * non-finite ones dropped (the polish is not part of the paper's solver).
 * precision selects the tier of the deflection grid (LF_FP64 / LF_MIXED / LF_FF).
 *   beta    device [n_src * 2] source positions, arcsec
 *   a_src   device [n_src] a_dis = D_ds / D_s of each source, in (0, 1]; a source outside
 *           that range is skipped with n_img = 0 and raises the device error word
 *   img     device [n_src * max_img * 2] images of source s at img[2 (s max_img + k)]
 *   n_img   device [n_src] number of images found (may exceed max_img: only the first
 *           max_img are stored), or -1 when more than 4 max_img + 16 raw candidates arose
 *   workspace  device, 256-byte aligned, at least lf_find_images_workspace(nx, ny, n_src,
 *           max_img) bytes; caller-owned, reusable after the stream reaches the call's end
 * Stream-ordered; LF_EINVAL for invalid host arguments (nothing launched). */
size_t lf_find_images_workspace(int32_t nx, int32_t ny, int32_t n_src, int32_t max_img);
lf_status lf_find_images(const lf_plane* plane, const lf_grid* grid, int32_t precision,
                         const double* beta, const double* a_src, int32_t n_src, int32_t max_img,
                         int32_t polish_iters, void* workspace, size_t workspace_bytes,
                         double* img, int32_t* n_img, void* stream);

/* The lens-equation solver above for sources behind several planes (Sec. 2.2, 2.3), all at the
 * one source redshift that the last row of `ratios` describes (ratios and planes as for
 * lf_trace_multiplane; call once per source redshift).  With beta(theta) the recursion's,
 * f = beta_s - theta + alpha_eff(theta), alpha_eff = theta - beta(theta) on the vertices
 * (traced in the chosen tier), and the zero contours, candidates, ordering and merging are
 * those of lf_find_images with a = 1.  The polish (polish_iters > 0) takes polish_iters
 * Newton steps theta <- theta - A^-1 (beta(theta) - beta_s) on the recursion (FP64 for
 * LF_FP64, else float-float: float-float deflections, about 1e-12 relative) with its
 * (non-symmetric) A; a step longer than the grid step is not taken (an image next to a
 * critical curve keeps its unpolished position).  The polish reads the number of kept
 * candidates back to the host: with polish_iters > 0 the call synchronises the stream once.
 *   beta, img, n_img  as for lf_find_images (no a_src)
 *   workspace  device, 256-byte aligned, at least lf_find_images_multiplane_workspace(nx, ny,
 *           n_src, max_img) bytes (the single-plane workspace plus the traced vertices and the
 *           polish state); caller-owned
 * LF_EINVAL for invalid host arguments (nothing launched). */
size_t lf_find_images_multiplane_workspace(int32_t nx, int32_t ny, int32_t n_src, int32_t max_img);
lf_status lf_find_images_multiplane(const lf_plane* planes, int32_t n_planes, const double* ratios,
                                    const lf_grid* grid, int32_t precision, const double* beta,
                                    int32_t n_src, int32_t max_img, int32_t polish_iters,
                                    void* workspace, size_t workspace_bytes, double* img,
                                    int32_t* n_img, void* stream);

/* ------------------------------------------------------------ chi^2 plans ------- */

/* Field codes a sampled parameter can target, and the transform applied first. */
typedef enum { LF_F_X = 0, LF_F_Y, LF_F_B, LF_F_EPS, LF_F_PA, LF_F_CORE, LF_F_CUT } lf_field;
typedef enum { LF_S_BSTAR = 0, LF_S_CORESTAR, LF_S_CUTSTAR, LF_S_LAM, LF_S_BETA, LF_S_ALPHA } lf_scaling_slot;
typedef enum {
  LF_XF_IDENT = 0,   /* value used as is                                  */
  LF_XF_VDISP = 1,   /* km/s -> b = 4 pi (v/c)^2 arcsec                   */
  LF_XF_DEG = 2,     /* degrees -> radians                                */
  LF_XF_KPC = 3      /* kpc -> arcsec with the plane's arcsec_per_kpc     */
} lf_xform;

/* Observed multiple images, grouped into families (CSR).  All host arrays. */
typedef struct {
  int32_t n_img, n_fam;
  const double* theta_obs;   /* [n_img * 2] observed positions, arcsec               */
  const double* sinv;        /* [n_img * 3] S_i^-1 as (xx, xy, yy) (Eq. chi2_img)    */
  const int32_t* fam_off;    /* [n_fam + 1] image offsets, fam_off[0] = 0            */
  const double* fam_ratio;   /* single plane: [n_fam] a_dis of each family;
                                multi-plane: [n_fam * n_planes] D_js/D_s per family  */
  /* Optional flux and time-delay measurements (Sec. 3.2-3.3; single-plane clusters; the
   * chi^2 of lf_chi2_batch then adds Eq. chi2_flux and Eq. chi2_td in their source-plane
   * forms, with m_src and Delta t_0 per family solved analytically, and lf_chi2_grad_batch
   * differentiates them).  An image takes part in a term when its value and its error are
   * finite and the error is > 0.                                                            */
  const double* mag;         /* [n_img] observed magnitudes, or NULL (no flux term)          */
  const double* mag_err;     /* [n_img] magnitude errors                                      */
  const double* td;          /* [n_img] observed time delays in days (any zero point per
                                family), or NULL (no time-delay term)                         */
  const double* td_err;      /* [n_img] time-delay errors in days                             */
  double td_scale;           /* (1 + z_d) D_d theta_0^2 / c in days (lf_td_scale); the factor
                                of a family is td_scale / a_dis                               */
} lf_images;

/* One cluster of a plan: its base model, images and parameter map.  The sampled
 * parameter vector of length P overwrites P fields of the base model per sample. */
typedef struct {
  int32_t n_planes;                 /* 1..8 */
  const lf_plane* planes;           /* host [n_planes]; comp/mem device pointers */
  const double* ratios;             /* host, multi-plane only: r[i][j] as in
                                       lf_trace_multiplane (rows 0..n_planes-1)   */
  const double* arcsec_per_kpc;     /* host [n_planes] for LF_XF_KPC             */
  lf_images images;
  int32_t P;                        /* parameters per sample, 1..64 */
  const int32_t* p_comp;            /* host [P]: component index counted over all planes
                                       in order, -1 for a scaling slot of the first
                                       plane that has members, or -2 for the a_dis =
                                       D_ds/D_s of one family, sampled directly (free
                                       source redshift, Sec. 3.5; single-plane
                                       clusters, transform LF_XF_IDENT; a sampled value
                                       outside (0, 1] gives chi^2 = +inf)          */
  const int32_t* p_field;           /* host [P]: lf_field; lf_scaling_slot if -1; the
                                       family index if -2                             */
  const int32_t* p_xform;           /* host [P]: lf_xform                            */
} lf_cluster;

typedef struct lf_plan lf_plan;

/* Builds a plan for n_clusters clusters that share P.  Copies everything it needs to the
 * device (the caller may free its arrays afterwards) and records the launch shape.
 * flags: bit 0 = capture the chi^2 launch in a CUDA graph; bit 1 = autotune the tile
 * shape on first use.  max_samples bounds S of later calls. */
lf_status lf_plan_create(lf_plan** out, const lf_cluster* clusters, int32_t n_clusters,
                         int32_t max_samples, int32_t precision, int32_t flags);

/* chi^2 of Eq. chi2_src (analytic source of Sec. 3.1) for S samples.
 * theta: device [S * P] FP64 in the parameters' own units; samples are cluster-major:
 * sample s belongs to cluster s / (S / n_clusters) (S must divide evenly).
 * chi2: device [S] FP64.  A sample with a non-finite magnification matrix or a singular
 * G in some family gets +inf; a one-image family contributes 0. */
lf_status lf_chi2_batch(lf_plan* plan, const double* theta, int32_t S, double* chi2,
                        void* stream);

/* chi^2 and its gradient d chi^2 / d theta (device [S * P] FP64).  For Eq. chi2_src the source
 * position is held at its optimum (d chi^2 / d beta_model = 0), so only the explicit
 * dependence is differentiated.  Multi-plane plans run the adjoint of the recursion of
 * Sec. 2.2 (reverse sweep over the planes with the third derivatives of psi at every later
 * plane's ray positions); their per-image records must fit in shared memory next to the
 * forward state (LF_EUNSUPPORTED otherwise).  Plans with flux or time-delay terms add those
 * terms to chi2 and their adjoint to grad: through the magnification (third derivatives of
 * psi and their parameter derivatives), the arrival time (psi and its parameter derivatives)
 * and beta_model, on which these terms do depend; such a plan whose parameters include a
 * family's a_dis returns LF_EUNSUPPORTED.
 * Precision: the cotangents are weighted by the offsets beta_i - beta_model (~ the position
 * errors), so the member deflections need more than FP32.  An LF_MIXED plan with one plane per
 * cluster and no flux / time-delay terms anchors them at the plan's own fields: every image's
 * member sum at the fields given to lf_plan_create, once, in FP64; per sample the change of
 * each member from those fields in FP32, in a form whose rounding is relative to the change.
 * Its precision is best for samples near the plan's fields (the usual case of a sampler or
 * optimizer around a mode).  Any other LF_MIXED plan runs its gradient on an LF_FF plan over
 * the same clusters, built with it. */
lf_status lf_chi2_grad_batch(lf_plan* plan, const double* theta, int32_t S, double* chi2,
                             double* grad, void* stream);

/* Image-plane chi^2 of Eq. chi2_img: for every image the model image is found by `iters`
 * Newton-Raphson steps theta <- theta - A(theta)^-1 (beta(theta) - beta_model) started at the
 * observed position (the paper's image-plane scheme, Sec. 3.5), towards the family's analytic
 * source beta_model = G^-1 g of Sec. 3.1; then chi2_img = sum_i (theta_obs - theta_model)^T
 * S_i^-1 (theta_obs - theta_model) and rms = sqrt(mean_i |theta_obs - theta_model|^2), the
 * image-plane rms the paper reports.  chi2_img, rms: device [S] FP64 (rms may be NULL).
 * 1 <= iters <= 64.  Multi-plane plans take beta(theta) and the non-symmetric A(theta) of the
 * recursion of Sec. 2.2 to each family's source plane.  A plan whose Newton state does not fit
 * in shared memory next to its tables returns LF_EUNSUPPORTED.  A sample whose Newton
 * iteration leaves the finite range gets chi2_img = +inf. */
lf_status lf_chi2_img_batch(lf_plan* plan, const double* theta, int32_t S, int32_t iters,
                            double* chi2_img, double* rms, void* stream);

/* Affine-invariant ensemble sampler (Goodman & Weare 2010; the paper's posterior sampler,
 * Sec. 3.5) on a single-cluster plan: likelihood exp(-chi^2/2) with the plan's chi^2, uniform
 * priors on the box [lo, hi].  Each of n_steps steps updates the two halves of the S walkers
 * in turn with the stretch move: walker k of one half takes partner j = floor(u0 S/2) of the
 * other half and z = ((a - 1) u1 + 1)^2 / a, proposes y = x_j + z (x_k - x_j), and accepts if
 * log u2 < (P - 1) log z - (chi^2(y) - chi^2(x_k)) / 2 (FP64); proposals outside the box are
 * rejected.  walkers: device [S * P] in/out; chi2: device [S] in/out (chi^2 of the walkers on
 * entry, e.g. from lf_chi2_batch); uniforms: device [n_steps * S * 3] in [0, 1), rows of the
 * first S/2 walkers drive the first half; lo, hi: device [P]; chain: device
 * [n_steps * S * P] (the walkers after each step) or NULL; n_accept: device counter added to,
 * or NULL.  S even, S/2 <= max_samples, a > 1.  The first call allocates the sampler's
 * workspace inside the plan. */
lf_status lf_aies_run(lf_plan* plan, double* walkers, double* chi2, int32_t S, int32_t n_steps,
                      const double* uniforms, double a, const double* lo, const double* hi,
                      double* chain, unsigned long long* n_accept, void* stream);

/* Random-walk Metropolis-Hastings (the paper's other sampler, Sec. 3.5) on a single-cluster
 * plan: S independent chains, likelihood exp(-chi^2/2), uniform priors on [lo, hi].  Each of
 * n_steps steps proposes y_k = x_k + step (.) z_k for every chain (z: standard normals) and
 * accepts if y_k is in the box, chi^2(y_k) is finite and log u_k < -(chi^2(y_k) - chi^2(x_k))/2
 * (FP64).  chains: device [S * P] in/out; chi2: device [S] in/out (chi^2 of the chains on
 * entry); normals: device [n_steps * S * P]; uniforms: device [n_steps * S] in (0, 1);
 * step, lo, hi: device [P]; trace: device [n_steps * S * P] (the chains after each step) or
 * NULL; n_accept: device counter added to, or NULL.  1 <= S <= max_samples.  The first call
 * allocates the sampler's workspace inside the plan. */
lf_status lf_mh_run(lf_plan* plan, double* chains, double* chi2, int32_t S, int32_t n_steps,
                    const double* normals, const double* uniforms, const double* step,
                    const double* lo, const double* hi, double* trace,
                    unsigned long long* n_accept, void* stream);

/* Multi-start Nelder-Mead downhill simplex (Nelder & Mead 1965; the paper's optimizer,
 * Sec. 3.5) for M independent runs on a single-cluster plan, minimising the plan's chi^2 with
 * chi^2 = +inf outside the prior box [lo, hi].  Coefficients and rules of Lagarias et al.
 * (1998): each iteration orders a run's P + 1 vertices stably by chi^2, reflects the worst
 * through the centroid of the others (summed in vertex order), then expands (2), contracts
 * outside or inside (1/2) or shrinks towards the best vertex (1/2); vector arithmetic is one
 * IEEE operation per component.  simplex: device [M * (P+1) * P] in/out; fvals: device
 * [M * (P+1)] in/out, the vertices' chi^2 on entry (finite or +inf); steps: device [5]
 * counters of reflections, expansions, outside and inside contractions and shrinks added to,
 * or NULL.  1 <= M <= max_samples.  Synchronises the stream once per iteration (to learn
 * whether some run shrinks).  The first call allocates the workspace inside the plan. */
lf_status lf_nm_run(lf_plan* plan, double* simplex, double* fvals, int32_t M, int32_t n_iter,
                    const double* lo, const double* hi, unsigned long long* steps, void* stream);

lf_status lf_plan_destroy(lf_plan* plan);

/* lf_chi2_batch for one cluster with no device allocation (the paper has no counterpart;
 * it exists for callers that cannot call cudaMalloc: a process whose GPU memory is already
 * reserved by another framework's caching allocator, or a plug-in host that forbids device
 * allocation).  The call uploads its host-side tables with cudaMemcpyAsync from pageable
 * memory, which waits for the stream's earlier work (the host returns once the stream has
 * drained up to the call), and it cannot be captured into a CUDA graph: on a capturing
 * stream it returns LF_EUNSUPPORTED before any work.
 * Arguments are those of one lf_cluster (host arrays read during the call; comp / mem device
 * arrays read on `stream`), theta device [S * P], chi2 device [S], all samples belonging to
 * that cluster.  Every derived table lives in one fixed 1 MiB array of device memory inside
 * the library (held by every GPU that loads the library until the process exits); a
 * cluster that needs more returns LF_EINVAL with the size in lf_last_error().  All calls
 * share that array and its contents persist between calls: calls that overlap on the GPU
 * race and must not be issued.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress), so it should come before any stream capture.  Host-side
 * validation as in lf_plan_create; component fields are validated on the device
 * (lf_device_error). */
lf_status lf_chi2_batch_static(const lf_cluster* cluster, const double* theta, int32_t S,
                               int32_t precision, double* chi2, void* stream);

/* Tile shape chosen by the plan (components per thread slice, threads per block). */
lf_status lf_plan_info(const lf_plan* plan, int32_t* kslices, int32_t* block, int32_t* graph);

/* ------------------------------------------------------------- host helpers ------ */

/* Flat LCDM angular-diameter distance D_A(z1, z2) in Mpc (Gauss-Legendre quadrature). */
double lf_angular_distance(double H0, double Om, double z1, double z2);
/* a_dis = D_ds / D_s. */
double lf_adis(double H0, double Om, double z_l, double z_s);
/* Angular size of one kpc at redshift z, arcsec. */
double lf_arcsec_per_kpc(double H0, double Om, double z);
/* (1 + z_d) D_d theta_0^2 / c in days with theta_0 = 1 arcsec: the time-delay factor of
 * Eq. time_delay at a_dis = 1 (a family's factor is this over its a_dis). */
double lf_td_scale(double H0, double Om, double z_d);
/* b = 4 pi (v/c)^2 in arcsec for a velocity dispersion v in km/s. */
double lf_b_from_vdisp(double v_kms);
/* Spherical NFW (M200 [Msun], concentration c) at z_l -> kappa_s and theta_s [arcsec]
 * (200 x the critical density at z_l; Sigma_cr at a_dis = 1). */
lf_status lf_nfw_params(double H0, double Om, double z_l, double m200, double conc,
                        double* kappa_s, double* theta_s);

/* One explicit component in physical units, for lf_comp_from_physical.  A field that is
 * not given holds NaN. */
typedef struct {
  int32_t kind;              /* lf_kind */
  int32_t pad;
  double x, y;               /* centre, arcsec */
  double vdisp;              /* isothermal: velocity dispersion, km/s */
  double theta_e, z_ref;     /* isothermal (instead of vdisp): area-equivalent Einstein radius
                                in arcsec at source redshift z_ref; shear: z_ref at which gamma
                                is quoted */
  double eps, pa_deg;        /* ellipticity (1-q)/(1+q); position angle in degrees */
  double core_kpc, core_arcsec, cut_kpc;   /* isothermal core (either unit), dPIE cut */
  double m200, conc;         /* NFW / elliptical NFW: M200 [Msun] (200 x rho_crit(z_l)), c */
  double kappa_s, theta_s;   /* NFW / elliptical NFW given in lensing units instead */
  double gamma;              /* shear */
  double amp;                /* multipole amplitude A of psi = A theta^2 cos 3(phi - pa) */
} lf_phys_comp;

/* Physical description -> lensing-unit component at a_dis = 1 (the unit conversions of the
 * A1 set-up, Sec. 3.4-3.5): b = 4 pi (v/c)^2 from vdisp, or b = theta_E / (a sqrt(q)) with
 * q = (1 - eps)/(1 + eps) and a = a_dis(z_l, z_ref); kpc -> arcsec at z_l; NFW through
 * lf_nfw_params; a shear quoted at z_ref divided by a_dis(z_l, z_ref); degrees -> radians.
 * Host only.  Errors: LF_EINVAL for a missing or invalid field. */
lf_status lf_comp_from_physical(const lf_phys_comp* in, double H0, double Om, double z_l,
                                lf_comp* out);

/* Eq. scaling from physical units: b_star = 4 pi (v_star / c)^2, core_star and cut_star from kpc to arcsec at
 * z_l; the exponents are copied.  Host only.  Errors: LF_EINVAL. */
lf_status lf_scaling_from_physical(double vstar_kms, double core_star_kpc, double cut_star_kpc,
                                   double lam, double beta, double alpha, double H0, double Om,
                                   double z_l, lf_scaling* out);

/* The distance-ratio table of the Sec. 2.2 recursion for planes at increasing redshifts
 * z_planes[0..n-1] and a source at z_s: ratios[i * n + j] = D_ij / D_j for i < j (0 else),
 * and the last row ratios[n * n + j] = D_js / D_s (0 for a plane behind the source); the
 * (n + 1) x n row-major layout that lf_trace_multiplane takes.  Host only.  Errors: LF_EINVAL
 * (n outside 1..8, redshifts not positive and increasing, NULL pointers). */
lf_status lf_multiplane_ratios(double H0, double Om, const double* z_planes, int32_t n_planes,
                               double z_s, double* ratios);

/* Failure-detection self-test (the paper has no counterpart): a one-block kernel arms a
 * shared-memory mbarrier for 16 bytes of bulk-copy transactions, issues no copy, and waits
 * with the library's bounded wait limited to `polls` polls (1..65536).  The wait runs out,
 * the kernel records the timeout in the device error word and returns, so the next
 * lf_device_error(stream) reports LF_ETIMEOUT (and clears the word).  No copy is ever in
 * flight and no thread spins past the limit.  Errors: LF_EINVAL for polls outside the range. */
lf_status lf_selftest_wait_timeout(uint32_t polls, void* stream);

/* Measured arithmetic rates of the current GPU (the roofline denominators of the
 * lens-equation kernels): FP32 fused multiply-adds, MUFU reciprocal square roots and FP64
 * fused multiply-adds per second, each from a kernel of independent dependency chains on
 * every SM timed with CUDA events on `stream` (synchronises it; allocates and frees a
 * scratch buffer). */
lf_status lf_probe_alu(double* fp32_fma_per_s, double* mufu_rsqrt_per_s, double* fp64_fma_per_s,
                       void* stream);

/* lf_probe_alu with one more rate: FP32 lane-operations per second of packed f32x2 FMA chains
 * (two lanes' FMAs per instruction), or NULL to skip it.  Equal to the scalar FMA rate where the
 * packed instructions share the FP32 datapath and save issue slots only. */
lf_status lf_probe_alu2(double* fp32_fma_per_s, double* fp32_fma2_lanes_per_s,
                        double* mufu_rsqrt_per_s, double* fp64_fma_per_s, void* stream);

/* Reads and clears the device error word (waits for `stream`): LF_OK or LF_ETIMEOUT. */
lf_status lf_device_error(void* stream);

/* Message of the last failing call on this host thread. */
const char* lf_last_error(void);

/* Library version string. */
const char* lf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LF_H_ */
