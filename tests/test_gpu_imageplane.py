"""Parity of lf_chi2_img_batch (image-plane chi^2 of Eq. chi2_img, Newton model images from
the observed positions towards the analytic source) with the oracle.

Tolerances: FP64 tier 1e-9 relative (the Newton iterates agree to rounding); the float-float
tier 1e-5 relative (the stated chi^2 target).  The mixed tier's model images move by
a |A^-1| |d alpha| with its FP32-level |d alpha| of a few 1e-6", against image offsets of
sigma = 1 mas in the parity case, so chi^2_img carries ~2 a |mu| |d alpha| / sigma, up to
5e-3 relative (measured 2.6e-4; values are printed)."""
import numpy as np
import pytest
import torch

from oracle import imageplane as ip
from oracle import model as OM

pytestmark = pytest.mark.gpu
W = pytest.importorskip("paper_2609_08649_b300.workloads")
TOL = {"fp64": 1e-9, "ff": 1e-5, "mixed": 5e-3}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import api, model
    return api, model


def oracle(wl, cat, th, tobs=None, iters=8):
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1 / wl.sigma_pos ** 2, 0, 1 / wl.sigma_pos ** 2], (n, 1)))
    t = torch.tensor(cat.theta_obs if tobs is None else tobs)
    c, r, _ = ip.chi2_img(wl, torch.tensor(th), t, sinv, list(cat.fam_off),
                          OM.single_plane_adis(wl, cat.fam_zs), iters=iters)
    return c.numpy(), r.numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_cluster_image_plane_chi2_matches_oracle(lib, prec):
    """The regime the scheme is meant for (the paper notes the model must already be good):
    images 1 mas from the model's images and parameters jittered by 1 % of the sampler's
    widths.  Far from a good model, plain Newton from the observed image can cross a critical
    curve and land on another image; there the iteration is chaotic and the tiers (and the
    oracle) legitimately end at different roots."""
    api, PM = lib
    wl = W.cluster_c2(n_samples=6)
    wl.params = [W.replace(p, jitter=p.jitter * 0.01) for p in wl.params]
    wl.sigma_pos = 0.001
    base = W.load_catalogue("cluster_200")
    tobs = base.theta_true + W.position_noise(31, len(base.theta_true), 0.001)
    cat = W.Catalogue(tobs, base.theta_true, base.fam_off, base.fam_zs)
    th = W.sample_thetas(wl, wl.seed)
    plan = api.Plan([PM.cluster_input(wl, cat)], 6, prec)
    c, r = plan.chi2_img(torch.tensor(th, device="cuda"), iters=8)
    cref, rref = oracle(wl, cat, th)
    rel = np.abs(c.cpu().numpy() - cref) / cref
    print(f"image-plane chi^2 ({prec}): relative error {rel.max():.3e}; rms {r.cpu().numpy()[:3]}")
    assert np.all(rel <= TOL[prec])
    assert np.allclose(r.cpu().numpy(), rref, rtol=TOL[prec], atol=0)
    api.device_error()


def test_full_size_image_plane_sampled(lib):
    """The benchmark's image-plane chi^2: 4096 samples x 200 images in one launch (mixed tier,
    8 Newton steps), in the regime of the parity test above; 8 seeded samples against the
    oracle one by one."""
    api, PM = lib
    wl = W.cluster_c2()
    wl.params = [W.replace(p, jitter=p.jitter * 0.01) for p in wl.params]
    wl.sigma_pos = 0.001
    base = W.load_catalogue("cluster_200")
    tobs = base.theta_true + W.position_noise(31, len(base.theta_true), 0.001)
    cat = W.Catalogue(tobs, base.theta_true, base.fam_off, base.fam_zs)
    th = W.sample_thetas(wl, wl.seed)
    plan = api.Plan([PM.cluster_input(wl, cat)], th.shape[0], "mixed", flags=api.FLAG_GRAPH)
    c, r = plan.chi2_img(torch.tensor(th, device="cuda"), iters=8)
    c, r = c.cpu().numpy(), r.cpu().numpy()
    idx = np.concatenate([[0, th.shape[0] - 1], np.random.default_rng(37).integers(0, th.shape[0], 6)])
    cref, rref = oracle(wl, cat, th[idx])
    assert np.all(np.abs(c[idx] - cref) <= TOL["mixed"] * cref)
    assert np.allclose(r[idx], rref, rtol=TOL["mixed"], atol=0)
    api.device_error()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_noise_free_images_give_zero(lib, prec):
    api, PM = lib
    wl = W.galaxy_c0()
    cat = W.load_catalogue("galaxy_sie_shear")
    wl.params = [W.ParamSpec(0, W.F_X, W.XF_IDENT, 0.0, 0.01, False)]
    wl.n_samples = 2
    th = W.sample_thetas(wl, 1)[:1].repeat(2, 0)
    clean = W.Catalogue(cat.theta_true, cat.theta_true, cat.fam_off, cat.fam_zs)
    plan = api.Plan([PM.cluster_input(wl, clean)], 2, prec)
    c, r = plan.chi2_img(torch.tensor(th, device="cuda"), iters=6)
    assert float(r.max()) < {"fp64": 1e-10, "ff": 1e-9, "mixed": 1e-6}[prec]


def test_image_plane_entry_point_validation(lib):
    api, PM = lib
    from paper_2609_08649_b300 import _lib as L
    wl = W.cluster_c2(n_samples=2)
    cat = W.load_catalogue("cluster_200")
    th = torch.tensor(W.sample_thetas(wl, wl.seed), device="cuda")
    plan = api.Plan([PM.cluster_input(wl, cat)], 2, "mixed")
    with pytest.raises(L.LFError):
        plan.chi2_img(th, iters=0)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_three_plane_image_plane_chi2_matches_oracle(lib, prec):
    """Three lens planes: true images of the three-plane model (made by the oracle, 11
    families at z = 4) observed with 1 mas noise, parameters jittered by 1 % of the sampler's
    widths; Newton with the recursion's beta and non-symmetric A against the oracle's.  The
    later planes hold spherical NFW and round dPIE components: FP32 deflections in the mixed
    tier, float-float in the float-float tier."""
    api, PM = lib
    from tests.helpers import three_plane_images
    wl, cat = three_plane_images()
    wl = W.replace(wl, n_samples=4, sigma_pos=0.001,
                   params=[W.replace(p, jitter=p.jitter * 0.01) for p in wl.params])
    th = W.sample_thetas(wl, wl.seed)
    plan = api.Plan([PM.cluster_input(wl, cat)], 4, prec)
    c, r = plan.chi2_img(torch.tensor(th, device="cuda"), iters=8)
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1 / wl.sigma_pos ** 2, 0, 1 / wl.sigma_pos ** 2], (n, 1)))
    cref, rref, _ = ip.chi2_img(wl, torch.tensor(th), torch.tensor(cat.theta_obs), sinv, list(cat.fam_off),
                                iters=8, fam_zs=list(cat.fam_zs))
    cref, rref = cref.numpy(), rref.numpy()
    rel = np.abs(c.cpu().numpy() - cref) / cref
    print(f"three-plane image-plane chi^2 ({prec}): relative error {rel.max():.3e}; rms {rref}")
    assert np.all(np.isfinite(cref)) and np.all(rref < 0.01)
    assert np.all(rel <= TOL[prec])
    assert np.allclose(r.cpu().numpy(), rref, rtol=TOL[prec], atol=0)
    api.device_error()
