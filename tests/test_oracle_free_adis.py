"""Pins of the oracle's sampled family distance ratios (free source redshifts sampled in
a_dis, Sec. 3.5): the fixed-ratio chi^2 as a special case, equivalence with a family moved to
another redshift through the cosmology, the zero of chi^2 at the true ratio for noise-free
images, and autograd against finite differences for the new gradient entries."""
import numpy as np
import torch

from oracle import cosmology as cz
from oracle import gradient as OG
from oracle import model as OM
from paper_2609_08649_b300 import workloads as W

torch.set_default_dtype(torch.float64)


def setup(free=(0, 20, 40, 59), n_samples=3, noise_free=False):
    wl = W.cluster_c2(n_samples=n_samples)
    cat = W.load_catalogue("cluster_200")
    base = OM.single_plane_adis(wl, cat.fam_zs)
    wl2 = W.with_free_adis(wl, free, [base[f] for f in free])
    tobs = cat.theta_true if noise_free else cat.theta_obs
    n = len(tobs)
    sinv = torch.tensor(np.tile([100.0, 0.0, 100.0], (n, 1)))
    return wl, wl2, cat, base, torch.tensor(tobs), sinv


def test_fixed_values_reproduce_the_fixed_ratio_chi2():
    wl, wl2, cat, base, tobs, sinv = setup()
    th = torch.tensor(W.sample_thetas(wl, 5))
    th2 = torch.cat([th, torch.tensor([[base[f] for f in (0, 20, 40, 59)]] * th.shape[0])], 1)
    c1 = OG.chi2_only(wl, th, tobs, sinv, list(cat.fam_off), base)
    c2 = OG.chi2_only(wl2, th2, tobs, sinv, list(cat.fam_off), base)
    assert torch.equal(c1, c2)


def test_sampled_ratio_equals_a_family_moved_in_redshift():
    wl, wl2, cat, base, tobs, sinv = setup()
    th = torch.tensor(W.sample_thetas(wl, 6))[:2]
    zs = np.array(cat.fam_zs, dtype=float)
    zs[20] = 3.7
    moved = OM.single_plane_adis(wl, zs)
    a20 = cz.a_dis(wl.planes[0].z, 3.7, wl.cosmo.H0, wl.cosmo.Om)
    th2 = torch.cat([th, torch.tensor([[base[0], a20, base[40], base[59]]] * 2)], 1)
    c_moved = OG.chi2_only(wl, th, tobs, sinv, list(cat.fam_off), moved)
    c_free = OG.chi2_only(wl2, th2, tobs, sinv, list(cat.fam_off), base)
    assert torch.allclose(c_moved, c_free, rtol=1e-13, atol=0)
    assert not torch.allclose(c_moved, OG.chi2_only(wl, th, tobs, sinv, list(cat.fam_off), base))


def test_noise_free_chi2_vanishes_at_the_true_ratio_only():
    wl, wl2, cat, base, tobs, sinv = setup(free=(30,), noise_free=True)
    th = torch.tensor(W.sample_thetas(wl, 1))[:1]
    vals = []
    for da in (-0.01, 0.0, 0.01):
        th2 = torch.cat([th, torch.tensor([[base[30] + da]])], 1)
        vals.append(float(OG.chi2_only(wl2, th2, tobs, sinv, list(cat.fam_off), base)[0]))
    assert vals[1] < 1e-12 and vals[0] > 1e-3 and vals[2] > 1e-3


def test_gradient_in_the_ratios_matches_finite_differences():
    wl, wl2, cat, base, tobs, sinv = setup()
    th = torch.tensor(W.sample_thetas(wl2, 7))[1:2]
    _, g = OG.chi2_and_grad(wl2, th, tobs, sinv, list(cat.fam_off), base)
    P = th.shape[1]
    for p in range(P - 4, P):
        h = 1e-4 * max(abs(float(th[0, p])), 1.0)
        vals = []
        for k in (-2, -1, 1, 2):
            t = th.clone()
            t[0, p] += k * h
            vals.append(float(OG.chi2_only(wl2, t, tobs, sinv, list(cat.fam_off), base)[0]))
        fd = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
        assert abs(fd - float(g[0, p])) <= 1e-6 * max(abs(fd), 1.0), (p, fd, float(g[0, p]))
