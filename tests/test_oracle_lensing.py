"""Pins of the oracle's lens map, magnification, multi-plane recursion, source-plane
chi^2, gradient, cosmology and image finder against closed forms, finite differences,
brute-force minimisation and limiting cases."""
import math

import numpy as np
import pytest
import torch
from scipy.optimize import minimize

from oracle import cosmology as cz
from oracle import images as im
from oracle import lensing as L
from oracle import model as om
from oracle import profiles as pr
from paper_2609_08649_b300 import workloads as W

torch.set_default_dtype(torch.float64)


def small_cluster(seed=0, n_mem=12):
    rng = np.random.default_rng(seed)
    comps = [W.PhysComp(W.DPIE, 0.5, -0.3, vdisp=700.0, eps=0.25, pa_deg=35.0, core_kpc=20.0, cut_kpc=800.0),
             W.PhysComp(W.SIE, 6.0, 4.0, vdisp=300.0, eps=0.1, pa_deg=-10.0, core_arcsec=0.3),
             W.PhysComp(W.NFW, -8.0, 3.0, m200=3e13, conc=6.0),
             W.PhysComp(W.SHEAR, gamma=0.04, pa_deg=20.0)]
    mem = W.PhysMembers(rng.uniform(-20, 20, n_mem), rng.uniform(-20, 20, n_mem), rng.uniform(-2, 1, n_mem),
                        vstar=220.0, core_star_kpc=0.2, cut_star_kpc=40.0, lam=0.25, beta=0.5, alpha=0.5)
    return W.Workload("small", W.Cosmo(), [W.PhysPlane(0.4, comps, mem)], z_s=2.5)


def plane_fn(pl):
    def fn(tx, ty):
        out = L.plane_sum(pl, torch.as_tensor(tx)[None], torch.as_tensor(ty)[None])
        return [o[0].numpy() for o in out]
    return fn


def test_mu_is_inverse_det_of_finite_difference_lens_map():
    wl = small_cluster()
    pl = om.build_planes(wl)[0]
    a = cz.a_dis(0.4, 2.5)
    tx = torch.tensor([[1.0, -7.5, 12.0, 3.3]])
    ty = torch.tensor([[2.0, 5.5, -9.0, -14.0]])
    ax, ay, pxx, pyy, pxy = L.plane_sum(pl, tx, ty)
    kappa, g1, g2, mu, det = L.jacobian_maps(ax, ay, pxx, pyy, pxy, a)
    h = 1e-5
    beta = lambda x, y: L.lens_map(x, y, *L.plane_sum(pl, x, y)[:2], a)
    bxp, byp = beta(tx + h, ty); bxm, bym = beta(tx - h, ty)
    bxq, byq = beta(tx, ty + h); bxn, byn = beta(tx, ty - h)
    fd_det = ((bxp - bxm) * (byq - byn) - (bxq - bxn) * (byp - bym)) / (4 * h * h)
    assert torch.allclose(det, fd_det, atol=1e-8)
    assert torch.allclose(mu, 1 / fd_det, rtol=1e-6)
    # eigenvalue form: mu = 1/((1 - a e1)(1 - a e2)), e1,2 = kappa +- |gamma|
    g = torch.hypot(g1, g2)
    assert torch.allclose(mu, 1 / ((1 - a * (kappa + g)) * (1 - a * (kappa - g))), rtol=1e-12)


def test_member_scaling_relation():
    """A member at L = L* is the spherical PJE of (b*, core*, cut*); at other L its strength
    is the isothermal b of v = v* (L/L*)^lam (b ~ v^2)."""
    wl = small_cluster()
    pl = om.build_planes(wl)[0]
    bm, cm, tm = L.member_fields(pl)
    m = wl.planes[0].members
    for k in range(len(m.x)):
        v = m.vstar * 10 ** (m.lam * m.log_l[k])
        assert abs(float(bm[0, k]) - L.b_from_vdisp(v)) < 1e-12
        apk = cz.arcsec_per_kpc(0.4)
        assert abs(float(tm[0, k]) - m.cut_star_kpc * apk * 10 ** (m.alpha * m.log_l[k])) < 1e-12
        assert abs(float(cm[0, k]) - m.core_star_kpc * apk * 10 ** (m.beta * m.log_l[k])) < 1e-12


@pytest.mark.parametrize("lam,alpha", [(0.25, 0.5), (0.3, 0.8)])
def test_member_mass_scales_as_luminosity_power(lam, alpha):
    """A consequence of the scaling relations that the power laws do not restate: a core-less
    pseudo-Jaffe member's deflection far outside its cut radius tends to b a / r (its total
    lensing mass is proportional to b a), and b ~ v^2, so with v ~ L^lam and a ~ L^alpha the mass
    grows as L^(2 lam + alpha), a constant mass-to-light ratio for the paper's lam = 1/4,
    alpha = 1/2.  Measured from the full lens evaluation of one member at two luminosities."""
    far = []
    for log_l in (0.0, 1.0):
        mem = W.PhysMembers(np.array([0.0]), np.array([0.0]), np.array([log_l]), vstar=220.0,
                            core_star_kpc=0.0, cut_star_kpc=40.0, lam=lam, beta=0.5, alpha=alpha)
        wl = W.Workload("one_member", W.Cosmo(), [W.PhysPlane(0.4, [], mem)], z_s=2.5)
        pl = om.build_planes(wl)[0]
        r = 1e6
        ax = L.plane_sum(pl, torch.tensor([[r]]), torch.tensor([[0.0]]))[0]
        far.append(float(ax[0, 0]) * r)
    assert abs(far[1] / far[0] - 10.0 ** (2 * lam + alpha)) < 1e-4 * 10.0 ** (2 * lam + alpha)


def test_isothermal_strength_from_velocity_dispersion():
    # b = 4 pi sigma^2 / c^2 in radians: sigma = 900 km/s -> 23.3603"
    assert abs(L.b_from_vdisp(900.0) - 23.3603) < 1e-4


def test_one_plane_multiplane_equals_single_plane():
    wl = small_cluster()
    pl = om.build_planes(wl)[0]
    a = cz.a_dis(0.4, 2.5)
    tx = torch.tensor([[1.0, -7.5, 12.0]]); ty = torch.tensor([[2.0, 5.5, -9.0]])
    beta, A = L.trace_multiplane([pl], [[0.0]], [a], tx, ty)
    ax, ay, pxx, pyy, pxy = L.plane_sum(pl, tx, ty)
    bx, by = L.lens_map(tx, ty, ax, ay, a)
    assert torch.allclose(beta[..., 0], bx, atol=1e-13) and torch.allclose(beta[..., 1], by, atol=1e-13)
    assert torch.allclose(A, L.jac_matrix(pxx, pyy, pxy, a), atol=1e-13)
    assert torch.allclose(A, A.transpose(-1, -2), atol=1e-15)       # single plane: symmetric


def _three_planes():
    wl = W.multiplane_c3(n_grid=8, n_samples=1)
    for p in wl.planes:
        p.comps = p.comps[:6]
    wl.planes[0].members.x = wl.planes[0].members.x[:10]
    wl.planes[0].members.y = wl.planes[0].members.y[:10]
    wl.planes[0].members.log_l = wl.planes[0].members.log_l[:10]
    planes = om.build_planes(wl)
    r, rs = cz.multiplane_ratios([p.z for p in wl.planes], wl.z_s)
    return wl, planes, r, rs


def test_multiplane_jacobian_is_derivative_of_lens_map():
    wl, planes, r, rs = _three_planes()
    tx = torch.tensor([[3.0, -20.0, 41.0]]); ty = torch.tensor([[-4.0, 7.5, 10.0]])
    beta, A = L.trace_multiplane(planes, r, rs, tx, ty)
    h = 1e-5
    bp, _ = L.trace_multiplane(planes, r, rs, tx + h, ty)
    bm, _ = L.trace_multiplane(planes, r, rs, tx - h, ty)
    bq, _ = L.trace_multiplane(planes, r, rs, tx, ty + h)
    bn, _ = L.trace_multiplane(planes, r, rs, tx, ty - h)
    fd = torch.stack([(bp - bm) / (2 * h), (bq - bn) / (2 * h)], -1)   # d beta_i / d theta_j
    assert torch.allclose(A, fd, atol=1e-8)
    # two or more massive planes: the Jacobian is not symmetric (Sec. 2.2)
    assert float((A[..., 0, 1] - A[..., 1, 0]).abs().max()) > 1e-6


def test_massless_planes_are_no_ops():
    wl, planes, r, rs = _three_planes()
    tx = torch.tensor([[3.0, -20.0]]); ty = torch.tensor([[-4.0, 7.5]])
    b1, A1 = L.trace_multiplane(planes[:1], [[0.0]], [rs[0]], tx, ty)
    empty = L.LPlane([], *[torch.zeros(1, 0)] * 7)
    b3, A3 = L.trace_multiplane([planes[0], empty, empty], r, rs, tx, ty)
    assert torch.allclose(b1, b3, atol=1e-13) and torch.allclose(A1, A3, atol=1e-13)


def test_cosmology_einstein_de_sitter_closed_form():
    # Om = 1: D_A(z1, z2) = 2c/H0 / (1+z2) ((1+z1)^-1/2 - (1+z2)^-1/2)
    for z1, z2 in [(0.0, 1.0), (0.5, 2.0), (0.39, 4.0)]:
        ref = 2 * cz.C_KMS / 70.0 / (1 + z2) * ((1 + z1) ** -0.5 - (1 + z2) ** -0.5)
        assert abs(cz.d_ang(z1, z2, 70.0, 1.0) - ref) < 1e-9 * ref
    assert abs(682.80248 - cz.d_ang(0.5, 2.0, 70.0, 1.0)) < 1e-5
    # low-redshift Hubble law
    assert abs(cz.d_ang(0.0, 1e-4) / (cz.C_KMS / 70.0 * 1e-4) - 1) < 2e-4
    assert cz.a_dis(0.5, 0.5) == 0.0 and 0 < cz.a_dis(0.5, 2.0) < cz.a_dis(0.5, 9.0) < 1


def test_cosmology_flat_lcdm_against_independent_quadrature():
    """Omega_m = 0.3: the oracle's adaptive quadrature against mpmath's tanh-sinh quadrature
    of the same integral at 30 digits, for the redshift pairs of the workloads."""
    import mpmath
    mpmath.mp.dps = 30
    c_h0 = mpmath.mpf(cz.C_KMS) / 70
    E = lambda z: mpmath.sqrt(mpmath.mpf("0.3") * (1 + z) ** 3 + mpmath.mpf("0.7"))
    for z1, z2 in [(0.0, 0.5), (0.0, 2.0), (0.5, 2.0), (0.39, 4.0), (0.9, 4.0), (2.1, 4.0), (0.5, 9.0)]:
        ref = c_h0 / (1 + mpmath.mpf(z2)) * mpmath.quad(lambda z: 1 / E(z), [mpmath.mpf(z1), mpmath.mpf(z2)])
        assert abs(cz.d_ang(z1, z2) / float(ref) - 1) < 1e-12, (z1, z2)
    # a_dis and the kpc scale from the same distances
    dd = c_h0 / mpmath.mpf("1.5") * mpmath.quad(lambda z: 1 / E(z), [0, mpmath.mpf("0.5")])
    assert abs(cz.arcsec_per_kpc(0.5) / float(mpmath.mpf(cz.ARCSEC_PER_RAD) / (dd * 1000)) - 1) < 1e-12


def _sheet_plane(k0):
    t = lambda v: torch.tensor([[float(v)]])
    return L.LPlane([L.SHEET], t(0), t(0), t(k0), t(0), t(0), t(0), t(0))


def test_mass_sheet_closed_forms():
    """A uniform sheet kappa_0: alpha = kappa_0 theta, gamma = 0, beta = (1 - a kappa_0) theta
    and mu = 1 / (1 - a kappa_0)^2, through plane_sum, lens_map and jacobian_maps; added to
    another lens it shifts kappa by kappa_0 and leaves gamma alone."""
    k0, a = 0.37, 0.62
    tx = torch.tensor([[1.5, -7.25, 12.0, 0.0]]); ty = torch.tensor([[2.0, 5.5, -9.0, 0.0]])
    ax, ay, pxx, pyy, pxy = L.plane_sum(_sheet_plane(k0), tx, ty)
    assert torch.equal(ax, k0 * tx) and torch.equal(ay, k0 * ty)
    kappa, g1, g2, mu, det = L.jacobian_maps(ax, ay, pxx, pyy, pxy, a)
    assert torch.allclose(kappa, torch.full_like(kappa, k0), rtol=0, atol=1e-15)
    assert float(g1.abs().max()) == 0.0 and float(g2.abs().max()) == 0.0
    assert torch.allclose(mu, torch.full_like(mu, 1 / (1 - a * k0) ** 2), rtol=1e-14, atol=0)
    bx, by = L.lens_map(tx, ty, ax, ay, a)
    assert torch.allclose(bx, (1 - a * k0) * tx, rtol=1e-15, atol=1e-15)
    assert torch.allclose(by, (1 - a * k0) * ty, rtol=1e-15, atol=1e-15)
    op = om.build_planes(small_cluster())[0]
    both = L.LPlane(op.kind + [L.SHEET], *[torch.cat([getattr(op, f), getattr(_sheet_plane(k0), f)], 1)
                                            for f in ("x", "y", "b", "eps", "pa", "core", "cut")],
                    op.mx, op.my, op.log_l, op.b_star, op.core_star, op.cut_star, op.lam, op.beta, op.alpha)
    k1, a1, b1, _, _ = L.jacobian_maps(*L.plane_sum(op, tx, ty), a)
    k2, a2, b2, _, _ = L.jacobian_maps(*L.plane_sum(both, tx, ty), a)
    assert torch.allclose(k2 - k1, torch.full_like(k1, k0), atol=1e-13)
    assert torch.allclose(a1, a2, atol=1e-13) and torch.allclose(b1, b2, atol=1e-13)


def test_mass_sheet_planes_multiplane_closed_form():
    """Two sheet planes kappa_1, kappa_2: theta_2 = (1 - r_12 kappa_1) theta_1, so
    beta = c theta_1 and A = c I with c = 1 - rs_1 kappa_1 - rs_2 kappa_2 (1 - r_12 kappa_1)."""
    k1, k2 = 0.21, 0.34
    r, rs = cz.multiplane_ratios([0.4, 1.0], 3.0)
    tx = torch.tensor([[1.5, -7.25, 12.0]]); ty = torch.tensor([[2.0, 5.5, -9.0]])
    beta, A = L.trace_multiplane([_sheet_plane(k1), _sheet_plane(k2)], r, rs, tx, ty)
    c = 1 - rs[0] * k1 - rs[1] * k2 * (1 - r[0][1] * k1)
    assert torch.allclose(beta[..., 0], c * tx, rtol=1e-14, atol=1e-14)
    assert torch.allclose(beta[..., 1], c * ty, rtol=1e-14, atol=1e-14)
    eye = torch.eye(2, dtype=torch.float64).expand_as(A)
    assert torch.allclose(A, c * eye, rtol=0, atol=1e-15)


def test_source_plane_chi2_is_invariant_under_a_mass_sheet():
    """With a pure sheet lens, beta_i = (1 - a kappa_0) theta_i and mu_i = I / (1 - a kappa_0),
    so M_i = S_i^-1 / (1 - a kappa_0)^2 and the factors cancel in Eq. chi2_src: the chi^2 is that
    of the observed positions about their S^-1-weighted family mean, for every kappa_0."""
    rng = np.random.default_rng(4)
    fam_off = [0, 2, 5, 9]
    th = torch.tensor(rng.uniform(-10, 10, (9, 2)))
    sinv = torch.tensor(np.column_stack([rng.uniform(20, 200, 9), rng.uniform(-5, 5, 9), rng.uniform(20, 200, 9)]))
    Sm = L.sinv_matrix(sinv)
    ref = 0.0
    for f in range(3):
        i0, i1 = fam_off[f], fam_off[f + 1]
        mean = torch.linalg.solve(Sm[i0:i1].sum(0), (Sm[i0:i1] @ th[i0:i1, :, None]).sum(0))[:, 0]
        d = th[i0:i1] - mean
        ref += float((d[:, None, :] @ Sm[i0:i1] @ d[:, :, None]).sum())
    for k0 in (0.0, 0.3, -0.4):
        beta, A = L.single_plane_source_terms(_sheet_plane(k0), th, fam_off, [0.7] * 3)
        c = L.chi2_src(beta, A, sinv, fam_off)
        assert abs(float(c.reshape(-1)[0]) - ref) <= 1e-12 * ref, k0


def _chi2_model(theta_obs, fam_off, a, pl, sinv):
    beta, A = L.single_plane_source_terms(pl, theta_obs, fam_off, [a] * (len(fam_off) - 1))
    return beta, A, L.chi2_src(beta, A, sinv, fam_off)


def sis_like_plane():
    wl = W.Workload("g", W.Cosmo(), [W.PhysPlane(0.5, [
        W.PhysComp(W.SIE, 0.0, 0.0, theta_e=1.2, z_ref=2.0, eps=0.15, pa_deg=30.0, core_arcsec=0.05),
        W.PhysComp(W.SHEAR, gamma=0.05, z_ref=2.0, pa_deg=0.0)])], z_s=2.0)
    return om.build_planes(wl)[0], cz.a_dis(0.5, 2.0)


def test_noise_free_images_give_zero_chi2():
    pl, a = sis_like_plane()
    fn = plane_fn(pl)
    imgs = im.find_images(fn, a, (0.05, 0.03), -2.5, -2.5, 0.02, 251, newton=True)
    assert len(imgs) == 5           # four bright images and the central one of the cored SIE
    theta = torch.tensor(imgs)
    sinv = torch.tensor([[400.0, 0.0, 400.0]] * 5)
    _, _, chi2 = _chi2_model(theta, [0, 5], a, pl, sinv)
    assert float(chi2[0]) < 1e-18


def test_analytic_source_minimises_chi2():
    """beta_model = G^-1 g agrees with a brute-force minimisation of Eq. chi2_src over
    the source position, and the minimum equals the closed-form chi^2."""
    pl, a = sis_like_plane()
    theta = torch.tensor([[1.1, 0.4], [-0.9, -0.6], [0.3, -1.2], [-0.2, 1.0]])
    sinv = torch.tensor([[400.0, 30.0, 250.0], [100.0, 0.0, 100.0], [300.0, -20.0, 150.0], [90.0, 5.0, 60.0]])
    beta, A, chi2 = _chi2_model(theta, [0, 4], a, pl, sinv)
    mu = torch.linalg.inv(A[0])
    Sinv = L.sinv_matrix(sinv)

    def chi2_at(bm):
        d = beta[0] - torch.tensor(bm)
        dt = (mu @ d[..., None])
        return float((dt.transpose(-1, -2) @ Sinv @ dt).sum())
    res = minimize(chi2_at, x0=[0.0, 0.0], method="Nelder-Mead",
                   options={"xatol": 1e-12, "fatol": 1e-14, "maxiter": 20000})
    assert abs(res.fun - float(chi2[0])) < 1e-8 * max(1.0, res.fun)


def test_chi2_statistics_with_small_noise():
    """With Gaussian noise of covariance S on noise-free images, E[chi2_src] is close to
    2 sum_f (n_f - 1) (chi^2 with 2(n-1) degrees of freedom per family, to first order,
    Eq. delta)."""
    pl, a = sis_like_plane()
    fn = plane_fn(pl)
    rng = np.random.default_rng(7)
    fams, offs = [], [0]
    while len(fams) < 12:
        b = rng.uniform(-0.08, 0.08, 2)
        imgs = im.find_images(fn, a, tuple(b), -2.5, -2.5, 0.02, 251, newton=True)
        if len(imgs) == 5:
            fams.append(imgs)
            offs.append(offs[-1] + 5)
    clean = torch.tensor(np.concatenate(fams))
    sig = 1e-4
    sinv = torch.tensor([[1 / sig ** 2, 0.0, 1 / sig ** 2]] * len(clean))
    vals = []
    for t in range(40):
        noisy = clean + torch.tensor(rng.normal(0, sig, clean.shape))
        vals.append(float(_chi2_model(noisy, offs, a, pl, sinv)[2][0]))
    dof = 2 * sum(len(f) - 1 for f in fams)
    assert abs(np.mean(vals) - dof) < 4 * math.sqrt(2 * dof / len(vals))


def test_gradient_autograd_matches_central_differences():
    from oracle.gradient import chi2_and_grad, chi2_only
    wl = small_cluster(n_mem=6)
    wl.params = [W.ParamSpec(0, W.F_X, W.XF_IDENT, 0.5, 0.1, False),
                 W.ParamSpec(0, W.F_B, W.XF_VDISP, 700.0, 0.01, True),
                 W.ParamSpec(0, W.F_EPS, W.XF_IDENT, 0.25, 0.02, False),
                 W.ParamSpec(0, W.F_PA, W.XF_DEG, 35.0, 2.0, False),
                 W.ParamSpec(0, W.F_CORE, W.XF_KPC, 20.0, 0.01, True),
                 W.ParamSpec(3, W.F_B, W.XF_IDENT, 0.04, 0.005, False),
                 W.ParamSpec(-1, 0, W.XF_VDISP, 220.0, 0.01, True),
                 W.ParamSpec(-1, 3, W.XF_IDENT, 0.25, 0.01, False)]
    wl.n_samples = 2
    theta = torch.tensor(W.sample_thetas(wl, 3))
    tobs = torch.tensor([[10.0, 3.0], [-9.0, -4.0], [2.0, 12.0], [4.0, -11.0], [-13.0, 1.0]])
    sinv = torch.tensor([[100.0, 0.0, 100.0]] * 5)
    fam_off, fam_adis = [0, 3, 5], [0.6, 0.7]
    chi2, grad = chi2_and_grad(wl, theta, tobs, sinv, fam_off, fam_adis)
    for p in range(theta.shape[1]):
        h = 1e-4 * max(abs(float(theta[0, p])), 1.0)
        tp, tm = theta.clone(), theta.clone()
        tp[:, p] += h; tm[:, p] -= h
        tpp, tmm = theta.clone(), theta.clone()
        tpp[:, p] += 2 * h; tmm[:, p] -= 2 * h
        f = lambda t: chi2_only(wl, t, tobs, sinv, fam_off, fam_adis)
        fd = (8 * (f(tp) - f(tm)) - (f(tpp) - f(tmm))) / (12 * h)    # 4th-order central
        assert torch.allclose(grad[:, p], fd, rtol=1e-7, atol=1e-7 * float(chi2.abs().max())), p


def test_image_finder_sis_closed_form_and_second_order_error():
    """SIS images: theta = beta_hat (|beta| + a b) and -beta_hat (a b - |beta|); without the
    Newton polish the error of the marching-squares construction falls as h^2."""
    b, a = 1.0, 0.6
    pl = L.LPlane([L.SIE], *[torch.tensor([[v]]) for v in (0.0, 0.0, b, 0.0, 0.0, 0.0, 0.0)])
    fn = plane_fn(pl)
    beta = np.array([0.13, 0.07])
    bh = beta / np.linalg.norm(beta)
    exact = np.array([bh * (np.linalg.norm(beta) + a * b), -bh * (a * b - np.linalg.norm(beta))])
    errs = []
    for h in (0.04, 0.02, 0.01):
        n = int(round(3.0 / h)) + 1
        imgs = im.find_images(fn, a, beta, -1.5 + h / 3, -1.5 + h / 7, h, n)
        # alpha of the singular SIS flips direction across the centre: the cell that
        # holds it shows a spurious sign change, which is not an image
        imgs = imgs[np.hypot(imgs[:, 0], imgs[:, 1]) > 2 * h]
        assert len(imgs) == 2
        err = max(min(np.hypot(*(e - p)) for p in imgs) for e in exact)
        errs.append(err)
    assert errs[0] / errs[2] > 8.0          # ~ 16 for O(h^2)
    imgs = im.find_images(fn, a, beta, -1.5 + 0.01 / 3, -1.5 + 0.01 / 7, 0.01, 301, newton=True)
    assert max(min(np.hypot(*(e - p)) for p in imgs) for e in exact) < 1e-12


def test_image_finder_agrees_with_brute_force_roots():
    """All roots of the lens equation of an SIE + shear found by Newton from a dense
    set of starting points match the marching-squares images."""
    pl, a = sis_like_plane()
    fn = plane_fn(pl)
    beta = (0.04, -0.02)
    imgs = im.find_images(fn, a, beta, -2.5, -2.5, 0.05, 101, newton=True)
    roots = []
    for x in np.linspace(-2.2, 2.2, 23):
        for y in np.linspace(-2.2, 2.2, 23):
            p = im.polish(fn, a, beta, (x, y), iters=60)
            ax, ay = fn(np.array([p[0]]), np.array([p[1]]))[:2]
            if np.all(np.isfinite(p)) and np.hypot(p[0] - a * ax[0] - beta[0], p[1] - a * ay[0] - beta[1]) < 1e-11 \
                    and np.hypot(*p) > 0.2 and all(np.hypot(*(p - q)) > 1e-6 for q in roots):
                roots.append(p)
    # the central (demagnified) image of a cored SIE sits near the core; ignore |theta| < 0.2
    found = [p for p in imgs if np.hypot(*p) > 0.2]
    assert len(found) == len(roots) == 4
    for r in roots:
        assert min(np.hypot(*(r - p)) for p in found) < 1e-9
