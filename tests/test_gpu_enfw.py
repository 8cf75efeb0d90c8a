"""Parity of the elliptical NFW component (LF_ENFW: Sec. 4.1-4.2, approximated as in Oguri
2021 by a sum of cored steep ellipsoids) with the oracle, in the maps, the chi^2 and its
gradient, and the flux / time-delay terms.

Tolerances.  The two sides use independent fits of the same recipe (tests/test_cse_table.py:
their profiles agree to 1e-12 on the fitted range 1e-4 <= xi / r_s <= 1e3, to 1e-8 outside
it), so FP64 parity is limited by rounding of the 38-term sums, |d alpha| <= 1e-12 (1 + S_a),
|d psi| <= 1e-12 (1 + S_p) with S_a, S_p the sums of the terms' magnitudes, plus 1e-8 S at
positions outside a halo's fitted range.  The mixed and float-float tiers evaluate this halo's deflection in float-float
(|d alpha| <= 1e-10 + 2^-40 S_a) and its psi_ij in FP32 term by term (|d psi| <= 8 u S_p).
chi^2 and gradient: the tiers' targets of tests/test_gpu_chi2.py, on the families whose
images keep |det A| >= 0.02 (the catalogue is not made of images of this model)."""
import numpy as np
import pytest
import torch

from oracle import auxterms as AX
from oracle import cosmology as cz
from oracle import cse_nfw as C
from oracle import model as OM
from oracle import profiles as pr
from tests.helpers import U32, families_off_critical, grid_xy, mu_det
from tests.test_gpu_chi2 import CHI2_TOL, grad_ok, oracle

pytestmark = pytest.mark.gpu
W = pytest.importorskip("paper_2609_08649_b300.workloads")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import api, model
    return api, model


def term_sums(pl, x, y):
    """Oracle alpha, psi of a members-free plane and the sums of the magnitudes of every
    term (each CSE of the elliptical NFW halos counted separately)."""
    tx, ty = torch.tensor(x)[None], torch.tensor(y)[None]
    from oracle import lensing as OL
    tot = [torch.zeros_like(tx) for _ in range(5)]
    sa, sp = torch.zeros_like(tx), torch.zeros_like(tx)
    out = torch.zeros_like(tx, dtype=torch.bool)      # outside some halo's fitted range
    s_tab, a_tab = C.table()
    for k, kind in enumerate(pl.kind):
        col = lambda f: f[:, k:k + 1]
        dx, dy = tx - col(pl.x), ty - col(pl.y)
        o = OL.component(kind, dx, dy, col(pl.b), col(pl.eps), col(pl.pa), col(pl.core), col(pl.cut))
        tot = [t + v for t, v in zip(tot, o)]
        if kind == OL.ENFW:
            q, pa, rs, ks = OL.q_from_eps(col(pl.eps)), col(pl.pa), col(pl.core), col(pl.b)
            c, s = torch.cos(pa), torch.sin(pa)
            u, v = (c * dx + s * dy) / rs, (-s * dx + c * dy) / rs
            xi = torch.sqrt(u * u + v * v / (q * q))
            out |= (xi < 1e-4) | (xi > 1e3)
            t = pr.cse_uv(u[..., None], v[..., None], q[..., None], torch.tensor(s_tab))
            at = torch.tensor(a_tab)
            sa += 2 * ks * rs * (torch.hypot(t[0], t[1]) * at).sum(-1)
            sp += 2 * ks * ((t[2].abs() + t[3].abs() + t[4].abs()) * at).sum(-1)
        else:
            sa += torch.hypot(o[0], o[1])
            sp += o[2].abs() + o[3].abs() + o[4].abs()
    return [t[0].numpy() for t in tot], sa[0].numpy(), sp[0].numpy(), out[0].numpy()


def halo_plane_workload():
    wl = W.cluster_c5_enfw(n_samples=1)
    pl = wl.planes[0]
    return W.replace(wl, planes=[W.replace(pl, comps=list(pl.comps[:3]), members=None)], params=[])


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_enfw_map_matches_oracle(lib, prec):
    """Two elliptical NFW halos and a shear on a ragged 301 x 263 grid spanning the halos'
    centres (one pixel centre 1 mas from a halo centre) and out to 2.5 theta_s."""
    api, PM = lib
    wl = halo_plane_workload()
    grid = W.Grid(-79.999, -80.001, 0.533333, 0.61068702, 301, 263)
    a = cz.a_dis(0.5, 3.0)
    dp = PM.device_planes(wl)[0]
    X, Y = grid_xy(grid)
    (ax, ay, pxx, pyy, pxy), sa, sp, out = term_sums(OM.build_planes(wl)[0], X.ravel(), Y.ravel())
    assert out.sum() >= 1                 # the pixel 1 mas from the first halo's centre
    g = {k: v.cpu().numpy().ravel().astype(np.float64) for k, v in api.jacobian_grid(dp, grid, a, prec).items()}
    api.device_error()
    if prec == "fp64":
        ta = 1e-12 * (1 + sa) + np.where(out, 1e-8 * sa, 0.0)
        tp = 1e-12 * (1 + sp) + np.where(out, 1e-8 * sp, 0.0)
    else:
        ta, tp = 1e-10 + 2.0 ** -40 * sa, 8 * U32 * sp + 1e-9
    ea, eb = np.abs(g["ax"] - ax), np.abs(g["ay"] - ay)
    print(f"eNFW map ({prec}): max |d alpha| {max(ea.max(), eb.max()):.2e}, max |alpha| {np.hypot(ax, ay).max():.1f}")
    assert np.all(ea <= ta) and np.all(eb <= ta)
    k0, g10, g20 = 0.5 * (pxx + pyy), 0.5 * (pxx - pyy), pxy
    for key, ref in (("kappa", k0), ("g1", g10), ("g2", g20)):
        assert np.all(np.abs(g[key] - ref) <= tp + U32 * np.abs(ref)), (key, np.abs(g[key] - ref).max())
    mu0, det0 = mu_det(pxx, pyy, pxy, a)
    m = np.abs(det0) >= 1e-3
    ddet = 2 * a * np.abs(1 - a * k0) * tp + 2 * a * a * np.hypot(g10, g20) * tp + 2 * a * a * tp * tp
    rel = np.abs(g["mu"][m] - mu0[m]) / np.abs(mu0[m])
    assert np.all(rel <= 1e-12 + ddet[m] / np.abs(det0[m]) * 1.5 + 1e-9), rel.max()


@pytest.fixture(scope="module")
def hera():
    wl = W.cluster_c5_enfw(n_samples=4)
    th = W.sample_thetas(wl, wl.seed)
    th[3, 2] = 0.0                      # one sample with a round first halo (eps = 0 exactly)
    cat = families_off_critical(wl, W.load_catalogue("cluster_200"), th, 0.02)
    return wl, cat, th


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_enfw_chi2_and_gradient_match_oracle(lib, hera, prec):
    """The Hera-like model (14 parameters: kappa_s, theta_s, eps, pa of both halos, shear,
    multipole, scaling relation) against the oracle's chi^2 and autograd gradient."""
    api, PM = lib
    wl, cat, th = hera
    assert len(cat.theta_obs) >= 60
    plan = api.Plan([PM.cluster_input(wl, cat)], th.shape[0], prec)
    c, g = plan.chi2_grad(torch.tensor(th, device="cuda"))
    cref, gref = oracle(wl, cat, th, grad=True)
    c1 = plan.chi2(torch.tensor(th, device="cuda"))
    assert torch.equal(c, c1) or prec != "fp64" or torch.allclose(c, c1, rtol=1e-14)
    rel = np.abs(c.cpu().numpy() - cref.numpy()) / np.abs(cref.numpy())
    print(f"eNFW chi2 ({prec}): relative error {rel.max():.2e}")
    assert np.all(rel <= CHI2_TOL[prec])
    assert grad_ok(g.cpu().numpy(), gref.numpy(), prec)
    api.device_error()


def test_enfw_gradient_matches_central_differences(lib, hera):
    """Float-float adjoint vs fourth-order central differences of the library's FP64 chi^2."""
    api, PM = lib
    wl, cat, th = hera
    plan = api.Plan([PM.cluster_input(wl, cat)], 1, "ff")
    P = th.shape[1]
    plan64 = api.Plan([PM.cluster_input(wl, cat)], 4 * P, "fp64")
    t0 = torch.tensor(th[1:2], device="cuda")
    _, g = plan.chi2_grad(t0)
    hs = [1e-4 * max(abs(float(t0[0, p])), 1.0) for p in range(P)]
    rows = []
    for p in range(P):
        for k in (1, -1, 2, -2):
            t = t0.clone()
            t[0, p] += k * hs[p]
            rows.append(t)
    f = plan64.chi2(torch.cat(rows)).cpu().numpy().reshape(P, 4)
    fd = np.array([(8 * (f[p, 0] - f[p, 1]) - (f[p, 2] - f[p, 3])) / (12 * hs[p]) for p in range(P)])
    assert grad_ok(g.cpu().numpy(), fd[None], "ff")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_enfw_flux_and_delay_terms(lib, hera, prec):
    """The flux / time-delay pass (potential and third derivatives of the halos) on the
    200-image catalogue's measurement set: FP64 1e-9 relative, mixed 1e-3 (FP32 potentials)."""
    api, PM = lib
    wl = W.cluster_c5_enfw(n_samples=4)
    th = W.sample_thetas(wl, wl.seed)
    cat = W.load_catalogue("cluster_200")
    aux = W.load_aux("cluster_200")
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1 / wl.sigma_pos ** 2, 0, 1 / wl.sigma_pos ** 2], (n, 1)))
    cf, ct = AX.chi2_aux(wl, th, torch.tensor(cat.theta_obs), sinv, list(cat.fam_off),
                         OM.single_plane_adis(wl, cat.fam_zs), cz.td_scale(wl.planes[0].z), *aux)
    t = torch.tensor(th, device="cuda")
    c0 = api.Plan([PM.cluster_input(wl, cat)], 4, prec).chi2(t).cpu().numpy()
    c1 = api.Plan([PM.cluster_input(wl, cat, aux=aux)], 4, prec).chi2(t).cpu().numpy()
    ref = (cf + ct).numpy()
    rel = np.abs((c1 - c0) - ref) / ref
    print(f"eNFW flux+delay ({prec}): relative error {rel.max():.2e}")
    assert np.all(rel <= {"fp64": 1e-9, "mixed": 1e-3}[prec])
    api.device_error()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-7), ("ff", 1e-2)])
def test_enfw_gradient_with_flux_and_delay_terms(lib, prec, tol):
    """lf_chi2_grad_batch with the measurements on the eNFW + shear + m = 3 multipole model:
    the potentials and third derivatives of every sampled component kind on dual numbers,
    against the oracle's autograd of the total chi^2 (bounds as in test_gpu_auxterms.py)."""
    api, PM = lib
    wl = W.cluster_c5_enfw(n_samples=2)
    th = W.sample_thetas(wl, wl.seed)[:2]
    cat = W.load_catalogue("cluster_200")
    aux = W.load_aux("cluster_200")
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1 / wl.sigma_pos ** 2, 0, 1 / wl.sigma_pos ** 2], (n, 1)))
    cref, gref = AX.chi2_total_and_grad(wl, th, torch.tensor(cat.theta_obs), sinv, list(cat.fam_off),
                                        OM.single_plane_adis(wl, cat.fam_zs), cz.td_scale(wl.planes[0].z), *aux)
    c, g = api.Plan([PM.cluster_input(wl, cat, aux=aux)], 2, prec).chi2_grad(torch.tensor(th, device="cuda"))
    g, gref = g.cpu().numpy(), gref.numpy()
    scale = np.maximum(np.abs(gref), 1e-2 * np.abs(gref).max(axis=1, keepdims=True))
    e = (np.abs(g - gref) / scale).max()
    print(f"eNFW total chi2 gradient ({prec}): error {e:.2e}")
    assert np.all(np.abs(c.cpu().numpy() - cref.numpy()) <= {"fp64": 1e-9, "ff": 1e-3}[prec] * cref.numpy())
    assert e < tol
    api.device_error()


def test_invalid_enfw_components_are_refused(lib):
    """A scale radius <= 0 or an ellipticity >= 1: a plan refuses the cluster before any launch;
    a map skips the component and raises the device error word."""
    api, PM = lib
    from paper_2609_08649_b300 import _lib as L
    good = W.PhysComp(W.ENFW, 0.0, 0.0, kappa_s=0.3, theta_s=20.0, eps=0.2, pa_deg=10.0)
    grid = W.Grid(-10.0, -10.0, 1.0, 1.0, 21, 21)
    ref = api.jacobian_grid(PM.device_plane(W.PhysPlane(0.5, [good]), W.Cosmo()), grid, 0.5, "mixed")
    api.device_error()
    for field, value in (("core", 0.0), ("core", -3.0), ("eps", 1.0)):
        # the host converter refuses such a component, so write it into the table directly
        dp = PM.device_plane(W.PhysPlane(0.5, [good, good]), W.Cosmo())
        dp.comp_host[field][1] = value
        dp.to("cuda")
        o = api.jacobian_grid(dp, grid, 0.5, "mixed")
        with pytest.raises(L.LFError):
            api.device_error()
        assert torch.equal(o["ax"], ref["ax"]) and torch.equal(o["mu"], ref["mu"])
        wl = W.Workload("bad", W.Cosmo(), [W.PhysPlane(0.5, [good, good])],
                        params=[W.ParamSpec(0, W.F_B, W.XF_IDENT, 0.3, 0.01, True)], n_samples=2)
        cat = W.load_catalogue("galaxy_sie_shear")
        ci = PM.cluster_input(wl, cat)
        ci.planes[0].comp_host[field][1] = value
        ci.planes[0].to("cuda")
        with pytest.raises(L.LFError) as e:
            api.Plan([ci], 2, "mixed")
        assert e.value.status == L.LF_EINVAL
        bad = W.replace(good, **({"theta_s": value} if field == "core" else {"eps": value}))
        with pytest.raises(L.LFError):      # the host converter refuses it too
            PM.device_plane(W.PhysPlane(0.5, [bad]), W.Cosmo())
