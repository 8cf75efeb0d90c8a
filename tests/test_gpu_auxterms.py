"""Parity of the flux and time-delay chi^2 terms (Eq. chi2_flux, Eq. chi2_td in their
source-plane forms, Sec. 3.2-3.3) in lf_chi2_batch against the oracle, on the 200-image
cluster with the synthetic measurement set (75 images with magnitudes, 15 families with
delays).  The plan's chi^2 with measurements minus the plan's chi^2 without them is the
added term; it is compared with the oracle's chi2_flux + chi2_td.

The gradient of the total chi^2 (lf_chi2_grad_batch with the measurements) is compared with
the oracle's reverse-mode autograd through the same FP64 computation.

Tolerances: FP64 tier 1e-9 relative.  The mixed tiers evaluate each component's potential in
FP32, so the arrival time carries |dT_i| ~ K a 4u sum_k |psi_k(theta_i)| (about 6e-3 days on
this cluster, against 2-day delay errors); the added chi^2 is held to 1e-3 relative
(measured 3.3e-4)."""
import numpy as np
import pytest
import torch

from oracle import auxterms as AX
from oracle import cosmology as cz
from oracle import model as OM

pytestmark = pytest.mark.gpu
W = pytest.importorskip("paper_2609_08649_b300.workloads")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import api, model
    wl = W.cluster_c2(n_samples=8)
    cat = W.load_catalogue("cluster_200")
    aux = W.load_aux("cluster_200")
    th = W.sample_thetas(wl, wl.seed)
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1 / wl.sigma_pos ** 2, 0, 1 / wl.sigma_pos ** 2], (n, 1)))
    base = OM.single_plane_adis(wl, cat.fam_zs)
    cf, ct = AX.chi2_aux(wl, th, torch.tensor(cat.theta_obs), sinv, list(cat.fam_off), base,
                         cz.td_scale(wl.planes[0].z), *aux)
    return api, model, wl, cat, aux, th, cf.numpy(), ct.numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_flux_and_delay_terms_match_oracle(setup, prec):
    api, PM, wl, cat, aux, th, cf, ct = setup
    S = th.shape[0]
    t = torch.tensor(th, device="cuda")
    c0 = api.Plan([PM.cluster_input(wl, cat)], S, prec).chi2(t).cpu().numpy()
    c1 = api.Plan([PM.cluster_input(wl, cat, aux=aux)], S, prec).chi2(t).cpu().numpy()
    add, ref = c1 - c0, cf + ct
    rel = np.abs(add - ref) / ref
    print(f"flux+delay ({prec}): added chi2 {add[:3]}, oracle {ref[:3]}, relative error {rel.max():.2e}")
    tol = {"fp64": 1e-9, "ff": 1e-3, "mixed": 1e-3}[prec]
    assert np.all(rel <= tol)
    # each term alone
    mag, me, td, te = aux
    c_f = api.Plan([PM.cluster_input(wl, cat, aux=(mag, me, None, None))], S, prec).chi2(t).cpu().numpy()
    assert np.all(np.abs((c_f - c0) - cf) <= tol * cf)
    api.device_error()


def _grad_err(g, ref):
    scale = np.maximum(np.abs(ref), 1e-2 * np.abs(ref).max(axis=1, keepdims=True))
    return (np.abs(g - ref) / scale).max()


# Gradient bounds per component (relative to the larger of |g_p| and 1e-2 max_p |g_p|).  FP64:
# the adjoint is the oracle's derivative in another order of rounding, 1e-7.  Float-float
# adjoint (ff, and mixed through its float-float plan): psi and its third derivatives per
# component in FP32 put |dT_i| ~ 6e-3 days on the arrival times (see the module's note), so
# the time-delay cotangent -2 w_t (d_i - Delta t_0) carries ~6e-3 / sigma_t ~ 3e-3 relative
# error where the residual is ~sigma_t, and the magnification's third derivatives ~1e-6
# relative: 1e-2.
GRAD_TOL = {"fp64": 1e-7, "ff": 1e-2, "mixed": 1e-2}


@pytest.mark.parametrize("prec", ["fp64", "ff", "mixed"])
def test_gradient_with_flux_and_delay_terms_matches_oracle(setup, prec):
    """lf_chi2_grad_batch on a plan with magnitudes and delays: chi^2 = chi2_src + chi2_flux +
    chi2_td and its gradient against the oracle's autograd through the same FP64 computation
    (grad mu differentiated by a second pass); the plan without the measurements is far from
    that gradient, so the comparison sees the added terms."""
    api, PM, wl, cat, aux, th, cf, ct = setup
    S = 4
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1 / wl.sigma_pos ** 2, 0, 1 / wl.sigma_pos ** 2], (n, 1)))
    base = OM.single_plane_adis(wl, cat.fam_zs)
    cref, gref = AX.chi2_total_and_grad(wl, th[:S], torch.tensor(cat.theta_obs), sinv, list(cat.fam_off),
                                        base, cz.td_scale(wl.planes[0].z), *aux)
    cref, gref = cref.numpy(), gref.numpy()
    t = torch.tensor(th[:S], device="cuda")
    c, g = api.Plan([PM.cluster_input(wl, cat, aux=aux)], S, prec).chi2_grad(t)
    c, g = c.cpu().numpy(), g.cpu().numpy()
    c0, g0 = api.Plan([PM.cluster_input(wl, cat)], S, prec).chi2_grad(t)
    c0, g0 = c0.cpu().numpy(), g0.cpu().numpy()
    add = cf[:S] + ct[:S]
    e, e0 = _grad_err(g, gref), _grad_err(g0, gref)
    print(f"total chi2 ({prec}): {c[:2]} oracle {cref[:2]}; gradient error {e:.2e} "
          f"(without the terms {e0:.2e})")
    tol_c = {"fp64": 1e-9 * cref, "ff": 1e-5 * (cref - add) + 1e-3 * add, "mixed": 1e-5 * (cref - add) + 1e-3 * add}
    assert np.all(np.abs(c - cref) <= tol_c[prec])
    assert e < GRAD_TOL[prec]
    assert e0 > 100 * GRAD_TOL[prec]
    api.device_error()


@pytest.mark.parametrize("which", ["flux", "delay"])
def test_gradient_of_each_term(setup, which):
    """Each term alone (FP64): magnitudes only, delays only."""
    api, PM, wl, cat, aux, th, cf, ct = setup
    S = 2
    mag, me, td, te = aux
    sub = (mag, me, None, None) if which == "flux" else (None, None, td, te)
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1 / wl.sigma_pos ** 2, 0, 1 / wl.sigma_pos ** 2], (n, 1)))
    nan = np.full(n, np.nan)
    ox = (mag, me, nan, nan) if which == "flux" else (nan, nan, td, te)
    cref, gref = AX.chi2_total_and_grad(wl, th[:S], torch.tensor(cat.theta_obs), sinv, list(cat.fam_off),
                                        OM.single_plane_adis(wl, cat.fam_zs), cz.td_scale(wl.planes[0].z), *ox)
    c, g = api.Plan([PM.cluster_input(wl, cat, aux=sub)], S, "fp64").chi2_grad(torch.tensor(th[:S], device="cuda"))
    e = _grad_err(g.cpu().numpy(), gref.numpy())
    print(f"{which}: gradient error {e:.2e}")
    assert np.all(np.abs(c.cpu().numpy() - cref.numpy()) <= 1e-9 * cref.numpy())
    assert e < GRAD_TOL["fp64"]


def test_refusals(setup):
    """Flux / time-delay terms: single-plane clusters only; values need their errors; no
    gradient when a family's a_dis is sampled."""
    api, PM, wl, cat, aux, th, cf, ct = setup
    from paper_2609_08649_b300 import _lib as L
    w3 = W.multiplane_c3(n_grid=8, n_samples=2)
    cat3 = W.Catalogue(cat.theta_obs, cat.theta_true, cat.fam_off, np.full(len(cat.fam_zs), 4.0))
    with pytest.raises(L.LFError) as e:
        api.Plan([PM.cluster_input(w3, cat3, aux=aux)], 2, "mixed")
    assert e.value.status == L.LF_EUNSUPPORTED
    mag, me, td, te = aux
    with pytest.raises(L.LFError):   # values without errors
        api.Plan([PM.cluster_input(wl, cat, aux=(mag, None, None, None))], 2, "mixed")
    base = OM.single_plane_adis(wl, cat.fam_zs)
    wl2 = W.with_free_adis(wl, (0, 7), [base[0], base[7]], jitter=0.005)
    th2 = W.sample_thetas(wl2, 5)
    plan = api.Plan([PM.cluster_input(wl2, cat, aux=aux)], 2, "fp64")
    plan.chi2(torch.tensor(th2[:2], device="cuda"))      # the chi^2 itself is supported
    with pytest.raises(L.LFError) as e:
        plan.chi2_grad(torch.tensor(th2[:2], device="cuda"))
    assert e.value.status == L.LF_EUNSUPPORTED
