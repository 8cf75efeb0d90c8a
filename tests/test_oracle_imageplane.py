"""Pins of the oracle's image-plane chi^2 (Eq. chi2_img, Newton from the observed images):
zero on noise-free images, model images equal to the marching-squares solver's images of
beta_model, the lens equation satisfied at the model images, and chi^2_src close to
chi^2_img for small offsets (Eq. delta)."""
import numpy as np
import pytest
import torch

from oracle import images as im
from oracle import imageplane as ip
from oracle import lensing as L
from oracle import model as om
from paper_2609_08649_b300 import workloads as W

torch.set_default_dtype(torch.float64)


def galaxy():
    wl = W.galaxy_c0()
    wl.params = [W.ParamSpec(0, W.F_X, W.XF_IDENT, 0.0, 0.01, False),
                 W.ParamSpec(0, W.F_EPS, W.XF_IDENT, wl.planes[0].comps[0].eps, 0.01, False)]
    wl.n_samples = 3
    return wl


def test_noise_free_images_give_zero_image_plane_chi2():
    wl = galaxy()
    cat = W.load_catalogue("galaxy_sie_shear")
    th = torch.tensor(W.sample_thetas(wl, 1))[:1]
    adis = om.single_plane_adis(wl, cat.fam_zs)
    sinv = torch.tensor(np.tile([400.0, 0, 400.0], (len(cat.theta_obs), 1)))
    chi2, rms, tm = ip.chi2_img(wl, th, torch.tensor(cat.theta_true), sinv, list(cat.fam_off), adis)
    assert float(chi2[0]) < 1e-16 and float(rms[0]) < 1e-9


def test_model_images_solve_the_lens_equation_and_match_the_grid_solver():
    wl = galaxy()
    cat = W.load_catalogue("galaxy_sie_shear")
    th = torch.tensor(W.sample_thetas(wl, 2))
    adis = om.single_plane_adis(wl, cat.fam_zs)
    tobs = torch.tensor(cat.theta_obs)
    sinv = torch.tensor(np.tile([400.0, 0, 400.0], (len(tobs), 1)))
    chi2, rms, tm = ip.chi2_img(wl, th, tobs, sinv, list(cat.fam_off), adis, iters=12)
    planes = om.apply_params(wl, th)
    beta, A = L.single_plane_source_terms(planes[0], tobs, list(cat.fam_off), adis)
    bm = ip.source_models(beta, A, sinv, list(cat.fam_off))
    for s in range(th.shape[0]):
        pl = om.apply_params(wl, th[s:s + 1])[0]

        def fn(x, y):
            out = L.plane_sum(pl, torch.as_tensor(x)[None], torch.as_tensor(y)[None])
            return [o[0].numpy() for o in out]
        for f in range(len(cat.fam_off) - 1):
            a = adis[f]
            src = bm[s, f].numpy()
            grid_imgs = im.find_images(fn, a, src, -2.5, -2.5, 0.01, 501, newton=True)
            for i in range(cat.fam_off[f], cat.fam_off[f + 1]):
                p = tm[s, i].numpy()
                ax, ay = fn(np.array([p[0]]), np.array([p[1]]))[:2]
                assert np.hypot(p[0] - a * ax[0] - src[0], p[1] - a * ay[0] - src[1]) < 1e-12
                assert min(np.hypot(*(p - q)) for q in grid_imgs) < 1e-9


def test_source_plane_chi2_approximates_image_plane_chi2():
    """Eq. delta: for small offsets theta_obs - theta_model ~ A^-1 (beta_obs - beta_model),
    so chi^2_src ~ chi^2_img; with 1 mas noise the two agree to a few per cent."""
    wl = galaxy()
    cat = W.load_catalogue("galaxy_sie_shear")
    th = torch.tensor(W.sample_thetas(wl, 1))[:1]
    adis = om.single_plane_adis(wl, cat.fam_zs)
    rng = np.random.default_rng(3)
    sig = 1e-3
    tobs = torch.tensor(cat.theta_true + rng.normal(0, sig, cat.theta_true.shape))
    sinv = torch.tensor(np.tile([1 / sig ** 2, 0, 1 / sig ** 2], (len(tobs), 1)))
    from oracle import gradient as OG
    csrc = OG.chi2_only(wl, th, tobs, sinv, list(cat.fam_off), adis)
    cimg, _, _ = ip.chi2_img(wl, th, tobs, sinv, list(cat.fam_off), adis)
    assert abs(float(csrc[0]) / float(cimg[0]) - 1) < 0.05


@pytest.fixture(scope="module")
def three_plane():
    from tests.helpers import three_plane_images
    return three_plane_images()


def test_multiplane_reduces_to_single_plane_with_massless_later_planes():
    """Three planes whose second and third carry nothing: the multi-plane chi2_img equals the
    single-plane one with a_dis = D_ds/D_s of each family."""
    from oracle import cosmology as cz
    wl3 = W.multiplane_c3(n_grid=8, n_samples=3)
    wl3 = W.replace(wl3, planes=[wl3.planes[0]] + [W.replace(p, comps=[], members=None) for p in wl3.planes[1:]])
    wl1 = W.replace(wl3, planes=[wl3.planes[0]])
    cat = W.load_catalogue("cluster_200")
    zs = np.where(np.arange(len(cat.fam_zs)) % 2 == 0, 4.0, 2.5)
    th = torch.tensor(W.sample_thetas(wl3, wl3.seed))
    th[:, :] = th[0]                     # the unjittered model: Newton from the catalogue stays tame
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1e4, 0, 1e4], (n, 1)))
    tobs = torch.tensor(cat.theta_true)
    c3, r3, t3 = ip.chi2_img(wl3, th, tobs, sinv, list(cat.fam_off), iters=8, fam_zs=list(zs))
    z = [p.z for p in wl3.planes]
    adis = [cz.multiplane_ratios(z, zf, wl3.cosmo.H0, wl3.cosmo.Om)[1][0] for zf in zs]
    c1, r1, t1 = ip.chi2_img(wl1, th, tobs, sinv, list(cat.fam_off), adis, iters=8)
    fin = torch.isfinite(c1)
    assert fin.all()
    assert torch.allclose(c3, c1, rtol=1e-11, atol=0)
    assert torch.allclose(t3, t1, rtol=0, atol=1e-10)


def test_multiplane_noise_free_images_give_zero(three_plane):
    """True images of the three-plane model (found on a grid and polished with the multi-plane
    lens equation): with the model that made them, the model images are the observed ones."""
    wl, cat = three_plane
    th = torch.tensor(W.sample_thetas(wl, wl.seed)[:1])
    n = len(cat.theta_true)
    sinv = torch.tensor(np.tile([1e6, 0, 1e6], (n, 1)))
    c, r, tm = ip.chi2_img(wl, th, torch.tensor(cat.theta_true), sinv, list(cat.fam_off), iters=6,
                           fam_zs=list(cat.fam_zs))
    assert float(r[0]) < 1e-10 and float(c[0]) < 1e-12


def test_multiplane_model_images_solve_the_lens_equation(three_plane):
    """With 1 mas noise, every model image satisfies the multi-plane lens equation for its
    family's analytic source to 1e-10 arcsec, within a few mas of the observed image."""
    from oracle import cosmology as cz
    wl, cat = three_plane
    th = torch.tensor(W.sample_thetas(wl, wl.seed)[:1])
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1e6, 0, 1e6], (n, 1)))
    tobs = torch.tensor(cat.theta_obs)
    c, r, tm = ip.chi2_img(wl, th, tobs, sinv, list(cat.fam_off), iters=8, fam_zs=list(cat.fam_zs))
    planes = om.apply_params(wl, th)
    zs = [p.z for p in wl.planes]
    rr, _ = cz.multiplane_ratios(zs, zs[-1] + 1.0, wl.cosmo.H0, wl.cosmo.Om)
    fam_rs = [cz.multiplane_ratios(zs, z, wl.cosmo.H0, wl.cosmo.Om)[1] for z in cat.fam_zs]
    beta, A = L.multi_plane_source_terms(planes, rr, fam_rs, tobs, list(cat.fam_off))
    bm = ip.source_models(beta, A, sinv, list(cat.fam_off))[0]
    rs = L.image_ratios(fam_rs, list(cat.fam_off), len(planes))
    b, _ = L.multi_plane_beta_A(planes, rr, rs, tm[:, :, 0], tm[:, :, 1])
    for f in range(len(cat.fam_off) - 1):
        i0, i1 = cat.fam_off[f], cat.fam_off[f + 1]
        assert float((b[0, i0:i1] - bm[f]).abs().max()) < 1e-10
    assert float((tm[0] - tobs).norm(dim=-1).max()) < 0.01
    assert 0 < float(r[0]) < 0.005
