"""Pins of the oracle's flux and time-delay terms (Sec. 3.2-3.3, source-plane forms):
the singular isothermal sphere's closed-form time delay and magnifications, invariance
under the per-family nuisances (m_src, Delta t_0), and the linearisation against the exact
values at the image-plane model images."""
import math

import numpy as np
import torch

from oracle import auxterms as AX
from oracle import cosmology as cz
from oracle import imageplane as ip
from oracle import lensing as L
from oracle import model as OM
from paper_2609_08649_b300 import workloads as W

torch.set_default_dtype(torch.float64)


def sis_workload(b_e):
    """An SIS (round, coreless) of Einstein radius b_e at a = 1, at the origin."""
    comps = [W.PhysComp(W.SIE, 0.0, 0.0, vdisp=300.0, eps=0.0, pa_deg=0.0, core_arcsec=0.0)]
    wl = W.Workload("sis", W.Cosmo(), [W.PhysPlane(0.5, comps)], params=[W.ParamSpec(0, W.F_X, W.XF_IDENT, 0.0, 0.0, False)],
                    n_samples=1)
    return wl


def test_sis_time_delay_and_magnification_closed_forms():
    b, beta, a = 1.3, 0.4, 0.6
    wl = sis_workload(1.0)
    pl = OM.build_planes(wl)[0]
    pl.b = torch.full_like(pl.b, b)        # strength b at a = 1 (Einstein radius a b)
    t = torch.tensor([[beta + a * b, 0.0], [beta - a * b, 0.0]])
    ax, ay, *_ = L.plane_sum(pl, t[None, :, 0], t[None, :, 1])
    assert torch.allclose(t[:, 0] - a * ax[0], torch.full((2,), beta), atol=1e-14)   # both are images
    K0 = cz.td_scale(0.5)
    wl.params = [W.ParamSpec(0, W.F_B, W.XF_IDENT, b, 0.0, False)]
    th = torch.tensor([[b]])
    sinv = torch.tensor([[1e4, 0.0, 1e4]] * 2)
    mu, mu_model, T = AX.linearised(wl, th, t, sinv, [0, 2], [a], K0)
    K = K0 / a
    assert abs(float(T[0, 0] - T[0, 1]) - (-2.0 * K * a * b * beta)) < 1e-9 * K
    mu_ref = torch.tensor([(beta + a * b) / beta, -(a * b - beta) / beta])
    assert torch.allclose(mu[0], mu_ref, rtol=1e-12) and torch.allclose(mu_model[0], mu_ref, rtol=1e-9)
    m_src = 25.0
    mag = m_src - 2.5 * torch.log10(mu_ref.abs())
    cf = AX.chi2_flux(mu_model, mag, torch.tensor([0.1, 0.1]), [0, 2])
    assert float(cf[0]) < 1e-18


def cluster(noise=0.0, seed=31):
    wl = W.cluster_c2(n_samples=3)
    cat = W.load_catalogue("cluster_200")
    tobs = cat.theta_true + (W.position_noise(seed, len(cat.theta_true), noise) if noise else 0.0)
    base = OM.single_plane_adis(wl, cat.fam_zs)
    sinv = torch.tensor(np.tile([1e6, 0.0, 1e6], (len(tobs), 1)))
    return wl, cat, torch.tensor(tobs), base, sinv


def test_nuisance_invariance():
    wl, cat, tobs, base, sinv = cluster(noise=0.01)
    th = W.sample_thetas(wl, 3)
    n = len(tobs)
    rng = np.random.default_rng(2)
    mag, me = rng.uniform(22, 27, n), np.full(n, 0.1)
    td, te = rng.uniform(-500, 500, n), np.full(n, 2.0)
    K0 = cz.td_scale(wl.planes[0].z)
    cf, ct = AX.chi2_aux(wl, th, tobs, sinv, list(cat.fam_off), base, K0, mag, me, td, te)
    off = cat.fam_off
    mag2, td2 = mag.copy(), td.copy()
    mag2[off[3]:off[4]] += 1.7
    td2[off[10]:off[11]] -= 333.0
    cf2, ct2 = AX.chi2_aux(wl, th, tobs, sinv, list(cat.fam_off), base, K0, mag2, me, td2, te)
    assert torch.allclose(cf, cf2, rtol=1e-10) and torch.allclose(ct, ct2, rtol=1e-10)
    assert float(cf.min()) > 0 and float(ct.min()) > 0


def test_linearisation_tracks_the_image_plane_values():
    """With 1 mas noise, the exact magnification and arrival time at the model images
    (Newton from the observed images towards beta_model) differ from the observed-image
    values at first order; the linearised values remove most of that difference."""
    wl, cat, tobs, base, sinv = cluster(noise=0.001)
    th = torch.tensor(W.sample_thetas(wl, 1))[:1]
    K0 = cz.td_scale(wl.planes[0].z)
    mu_obs, mu_lin, T_lin = AX.linearised(wl, th, tobs, sinv, list(cat.fam_off), base, K0)
    _, _, tm = ip.chi2_img(wl, th, tobs, sinv, list(cat.fam_off), base, iters=12)
    pl = OM.apply_params(wl, th)[0]
    N = len(tobs)
    fam = np.repeat(np.arange(len(cat.fam_off) - 1), np.diff(cat.fam_off))
    a = torch.tensor(np.asarray(base)[fam])[None]
    ax, ay, pxx, pyy, pxy = L.plane_sum(pl, tm[..., 0], tm[..., 1])
    mu_ex = 1.0 / ((1 - a * pxx) * (1 - a * pyy) - (a * pxy) ** 2)
    bmx, bmy = tm[..., 0] - a * ax, tm[..., 1] - a * ay      # = beta_model at convergence
    psi = L.plane_potential(pl, tm[..., 0], tm[..., 1])
    K = K0 / a
    T_ex = K * (0.5 * ((tm[..., 0] - bmx) ** 2 + (tm[..., 1] - bmy) ** 2) - a * psi)
    # the first-order terms of each image: compare both approximations on every image
    e0 = (mu_obs - mu_ex).abs()
    e1 = (mu_lin - mu_ex).abs()
    big = e0 > 1e-6 * mu_ex.abs()
    assert big.sum() > 100
    assert float((e1[big] / e0[big]).median()) < 0.05
    T_obs0 = K * (0.5 * ((tobs[None, :, 0] - (tobs[None, :, 0] - a * L.plane_sum(pl, tobs[None, :, 0], tobs[None, :, 1])[0])) ** 2
                         + (tobs[None, :, 1] - (tobs[None, :, 1] - a * L.plane_sum(pl, tobs[None, :, 0], tobs[None, :, 1])[1])) ** 2)
                  - a * L.plane_potential(pl, tobs[None, :, 0], tobs[None, :, 1]))
    d0 = (T_obs0 - T_ex).abs()
    d1 = (T_lin - T_ex).abs()
    bigt = d0 > 1e-6
    assert bigt.sum() > 100
    assert float((d1[bigt] / d0[bigt]).median()) < 0.05


def test_catalogue_measurements_have_the_noise_chi2():
    """On the unjittered model at the noise-free images the linear terms vanish, so each chi^2
    is the noise's: E = sum over measured families of (n_f - 1), variance 2 E."""
    wl, cat, tobs, base, sinv = cluster(noise=0.0)
    mag, me, td, te = W.load_aux("cluster_200")
    th = W.sample_thetas(wl, 1)[:1]
    K0 = cz.td_scale(wl.planes[0].z)
    cf, ct = AX.chi2_aux(wl, th, tobs, sinv, list(cat.fam_off), base, K0, mag, me, td, te)
    sizes = np.diff(cat.fam_off)
    ef = sum(sizes[f] - 1 for f in range(len(sizes)) if np.isfinite(mag[cat.fam_off[f]]))
    et = sum(sizes[f] - 1 for f in range(len(sizes)) if np.isfinite(td[cat.fam_off[f]]))
    assert ef > 20 and et > 20
    assert abs(float(cf[0]) - ef) < 5 * math.sqrt(2 * ef), (float(cf[0]), ef)
    assert abs(float(ct[0]) - et) < 5 * math.sqrt(2 * et), (float(ct[0]), et)


def test_total_chi2_gradient_matches_central_differences():
    """d (chi2_src + chi2_flux + chi2_td) / d theta by autograd (grad mu through a
    differentiable second pass) against fourth-order central differences of the same FP64
    total, on the first 20 families of the 200-image cluster with its synthetic magnitudes and
    delays (h = 1e-4 max(|theta_p|, 1))."""
    wl = W.cluster_c2(n_samples=1)
    cat = W.load_catalogue("cluster_200")
    mag, me, td, te = W.load_aux("cluster_200")
    n = int(cat.fam_off[20])
    off = list(cat.fam_off[:21])
    tobs = torch.tensor(cat.theta_obs[:n])
    sinv = torch.tensor(np.tile([100.0, 0.0, 100.0], (n, 1)))
    base = OM.single_plane_adis(wl, cat.fam_zs[:20])
    K0 = cz.td_scale(wl.planes[0].z)
    args = (tobs, sinv, off, base, K0, mag[:n], me[:n], td[:n], te[:n])
    th = torch.tensor(W.sample_thetas(wl, wl.seed))
    c, g = AX.chi2_total_and_grad(wl, th, *args)

    def total(t):
        beta, A = L.single_plane_source_terms(OM.apply_params(wl, t)[0], tobs, off, OM.family_adis(wl, t, base))
        cf, ct = AX.chi2_aux(wl, t, tobs, sinv, off, base, K0, mag[:n], me[:n], td[:n], te[:n])
        return float((L.chi2_src(beta, A, sinv, off) + cf + ct)[0])

    with torch.no_grad():
        assert abs(total(th) - float(c[0])) <= 1e-12 * float(c[0])
        fd = []
        for p in range(th.shape[1]):
            h = 1e-4 * max(abs(float(th[0, p])), 1.0)
            f = []
            for k in (1, -1, 2, -2):
                t = th.clone()
                t[0, p] += k * h
                f.append(total(t))
            fd.append((8 * (f[0] - f[1]) - (f[2] - f[3])) / (12 * h))
    fd = np.array(fd)
    gg = g[0].numpy()
    scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    assert np.all(np.abs(gg - fd) <= 1e-6 * scale), np.abs(gg - fd) / scale
    # the flux and delay terms carry gradient of their own
    th2 = th.clone().requires_grad_(True)
    beta, A = L.single_plane_source_terms(OM.apply_params(wl, th2)[0], tobs, off, OM.family_adis(wl, th2, base))
    (g_src,) = torch.autograd.grad(L.chi2_src(beta, A, sinv, off).sum(), th2)
    assert float((g[0] - g_src[0]).abs().max()) > 1e-3 * float(g[0].abs().max())
