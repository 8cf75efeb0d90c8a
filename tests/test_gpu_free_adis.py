"""Parity of sampled family distance ratios (p_comp = -2: a free source redshift sampled
directly in a_dis, Sec. 3.5) in the chi^2 plans against the oracle: chi^2 and gradient in
every tier, the static entry point, the image-plane chi^2, out-of-range values and invalid
parameter maps.  Tolerances as in test_gpu_chi2.py (the mixed bound takes each sample's
ratios)."""
import numpy as np
import pytest
import torch

from oracle import gradient as OG
from oracle import imageplane as OIP
from oracle import model as OM
from tests.helpers import chi2_mixed_bound

pytestmark = pytest.mark.gpu
W = pytest.importorskip("paper_2609_08649_b300.workloads")
FREE = (0, 7, 20, 33, 41, 59)
CHI2_TOL = {"fp64": 1e-10, "mixed": 1e-5, "ff": 1e-5}


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import api, model
    wl = W.cluster_c2(n_samples=24)
    cat = W.load_catalogue("cluster_200")
    base = OM.single_plane_adis(wl, cat.fam_zs)
    wl2 = W.with_free_adis(wl, FREE, [base[f] for f in FREE], jitter=0.005)
    th = W.sample_thetas(wl2, 77)
    return api, model, wl2, cat, base, th


def oracle(wl2, cat, base, th, grad=False):
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1 / wl2.sigma_pos ** 2, 0, 1 / wl2.sigma_pos ** 2], (n, 1)))
    fn = OG.chi2_and_grad if grad else OG.chi2_only
    return fn(wl2, torch.tensor(th), torch.tensor(cat.theta_obs), sinv, list(cat.fam_off), base)


def grad_err(g, ref):
    scale = np.maximum(np.abs(ref), 1e-2 * np.abs(ref).max(axis=1, keepdims=True))
    return (np.abs(g - ref) / scale).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_chi2_and_gradient_with_free_ratios(setup, prec):
    api, PM, wl2, cat, base, th = setup
    S = 8
    plan = api.Plan([PM.cluster_input(wl2, cat)], S, prec)
    c, g = plan.chi2_grad(torch.tensor(th[:S], device="cuda"))
    c, g = c.cpu().numpy(), g.cpu().numpy()
    cref, gref = oracle(wl2, cat, base, th[:S], grad=True)
    cref, gref = cref.numpy(), gref.numpy()
    assert np.all(np.abs(c - cref) <= CHI2_TOL[prec] * np.abs(cref))
    c1 = plan.chi2(torch.tensor(th[:S], device="cuda")).cpu().numpy()
    if prec == "mixed":      # the forward launch (FP32 member sums)
        assert np.all(np.abs(c1 - cref) <= chi2_mixed_bound(wl2, cat, th[:S]))
    P0 = len(wl2.params) - len(FREE)
    ga, gra = g[:, P0:], gref[:, P0:]
    err = grad_err(g, gref)
    norm = (np.linalg.norm(g - gref, axis=1) / np.linalg.norm(gref, axis=1)).max()
    print(f"free a_dis ({prec}): chi2 rel {np.abs(c / cref - 1).max():.2e}, grad per-comp {err:.2e}, "
          f"norm {norm:.2e}, d chi2/d a range {np.abs(gra).min():.2e}..{np.abs(gra).max():.2e}")
    assert np.all(np.abs(gra) > 0)
    if prec == "fp64":
        assert err < 1e-8
    else:      # mixed and float-float: the float-float adjoint
        assert err < 1e-4
    api.device_error()


def test_out_of_range_ratio_gives_infinite_chi2(setup):
    api, PM, wl2, cat, base, th = setup
    t = th[:4].copy()
    P0 = len(wl2.params) - len(FREE)
    t[1, P0 + 2] = 1.2
    t[2, P0 + 4] = 0.0
    plan = api.Plan([PM.cluster_input(wl2, cat)], 4, "mixed")
    c = plan.chi2(torch.tensor(t, device="cuda")).cpu().numpy()
    assert np.isfinite(c[0]) and np.isfinite(c[3]) and np.isinf(c[1]) and np.isinf(c[2])


def test_static_entry_point_with_free_ratios(setup):
    api, PM, wl2, cat, base, th = setup
    from paper_2609_08649_b300 import _lib as L
    import ctypes as C
    ci = PM.cluster_input(wl2, cat)
    S = 6
    t = torch.tensor(th[:S], device="cuda")
    ref = api.Plan([ci], S, "fp64").chi2(t)
    out = torch.empty(S, dtype=torch.float64, device="cuda")
    cs = ci.c_struct()
    L.check(L.lib.lf_chi2_batch_static(C.byref(cs), api._ptr(t), S, L.LF_FP64, api._ptr(out), api._stream()))
    assert torch.allclose(out, ref, rtol=1e-12, atol=0)


def test_image_plane_chi2_with_free_ratios(setup):
    api, PM, wl2, cat, base, th = setup
    wl3 = W.replace(wl2, sigma_pos=0.001,
                    params=[W.replace(p, jitter=p.jitter * 0.01) for p in wl2.params])
    tobs = cat.theta_true + W.position_noise(31, len(cat.theta_true), 0.001)
    cat3 = W.Catalogue(tobs, cat.theta_true, cat.fam_off, cat.fam_zs)
    t = W.sample_thetas(wl3, 5)[:4]
    plan = api.Plan([PM.cluster_input(wl3, cat3)], 4, "fp64")
    c, r = plan.chi2_img(torch.tensor(t, device="cuda"), iters=8)
    n = len(tobs)
    sinv = torch.tensor(np.tile([1e6, 0, 1e6], (n, 1)))
    cref, rref, _ = OIP.chi2_img(wl3, torch.tensor(t), torch.tensor(tobs), sinv, list(cat.fam_off), base)
    assert np.allclose(c.cpu().numpy(), cref.numpy(), rtol=1e-9, atol=0)


def test_invalid_ratio_maps(setup):
    api, PM, wl2, cat, base, th = setup
    from paper_2609_08649_b300 import _lib as L
    bad = [W.with_free_adis(wl2, [len(cat.fam_zs)], [0.7]),                  # family out of range
           W.with_free_adis(wl2, [FREE[0]], [0.7]),                           # targeted twice
           W.replace(wl2, params=list(wl2.params[:-1]) +
                     [W.replace(wl2.params[-1], xform=W.XF_VDISP)])]          # not sampled directly
    for w in bad:
        with pytest.raises(L.LFError):
            api.Plan([PM.cluster_input(w, cat)], 2, "mixed")
    w3 = W.multiplane_c3(n_grid=8, n_samples=2)
    w3 = W.with_free_adis(w3, [0], [0.5])
    cat3 = W.Catalogue(cat.theta_obs, cat.theta_true, cat.fam_off, np.full(len(cat.fam_zs), 4.0))
    with pytest.raises(L.LFError) as e:
        api.Plan([PM.cluster_input(w3, cat3)], 2, "mixed")
    assert e.value.status == L.LF_EUNSUPPORTED
