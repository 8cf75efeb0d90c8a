"""Parity of lf_chi2_batch / lf_chi2_grad_batch with the FP64 oracle (Eq. chi2_src with the
analytic source of Sec. 3.1; gradient by the oracle's autograd and by central finite
differences), plus the plan's edge cases.

Tolerances: FP64 path 1e-10 relative on chi^2 and 1e-8 on the gradient; the mixed and
float-float tiers the stated targets, 1e-5 relative on chi^2 and 1e-4 on every gradient
component (relative to the larger of |g_p| and 1e-2 max_p |g_p| of the sample).  The cotangents
of the adjoint are weighted by d_i = beta_i - beta_model ~ sigma_pos, so FP32 member deflections
would put ~1e-4 relative errors on them: the mixed tier's lf_chi2_grad_batch anchors its member
sums at the plan's fields (FP64 sums per image once, the sample's change per member in FP32,
rounded relative to the change) on single-plane plans, and runs the float-float adjoint on the
others, so its chi^2 and gradient share the float-float bounds.
The forward chi^2 (lf_chi2_batch) of the mixed tiers keeps M in float-float words and is held
to 1e-5 on every sample, near critical curves included.  The adjoint launch forms A from FP32
psi_ij (M in float-float words as well), so its gradient moves by ~u/|det A|^3 near a
critical curve: a
sample with an image at |det A| < 1e-3 is held to the near-critical bounds (norm 1e-3, 1e-2
per component)."""
import numpy as np
import pytest
import torch

from oracle import gradient as OG
from oracle import model as OM
from tests.helpers import chi2_mixed_bound, families_off_critical

pytestmark = pytest.mark.gpu
W = pytest.importorskip("paper_2609_08649_b300.workloads")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import api, model
    return api, model


def oracle(wl, cat, theta, grad=False, sigma=None):
    sig = wl.sigma_pos if sigma is None else sigma
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([1 / sig ** 2, 0, 1 / sig ** 2], (n, 1)))
    tobs = torch.tensor(cat.theta_obs)
    th = torch.as_tensor(theta)
    kw = {}
    if len(wl.planes) == 1:
        kw["fam_adis"] = OM.single_plane_adis(wl, cat.fam_zs)
    else:
        kw["fam_zs"] = list(cat.fam_zs)
    fn = OG.chi2_and_grad if grad else OG.chi2_only
    return fn(wl, th, tobs, sinv, list(cat.fam_off), **kw)


def grad_err(g, ref):
    scale = np.maximum(np.abs(ref), 1e-2 * np.abs(ref).max(axis=1, keepdims=True))
    return (np.abs(g - ref) / scale).max()


def grad_ok(g, ref, prec):
    norm = (np.linalg.norm(g - ref, axis=1) / np.linalg.norm(ref, axis=1)).max()
    comp = grad_err(g, ref)
    print(f"gradient error ({prec}): per-component {comp:.3e}, norm {norm:.3e}")
    if prec == "fp64":
        return comp < 1e-8
    if prec in ("ff", "mixed"):
        return comp < 1e-4
    assert prec == "near_critical"
    return norm < 1e-3 and comp < 1e-2


CHI2_TOL = {"fp64": 1e-10, "mixed": 1e-5, "ff": 1e-5}


@pytest.fixture(scope="module")
def c2():
    wl = W.cluster_c2()
    return wl, W.load_catalogue("cluster_200"), W.sample_thetas(wl, wl.seed)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5), ("ff", 1e-5)])
def test_cluster_chi2_matches_oracle(lib, c2, prec, tol):
    api, PM = lib
    wl, cat, th = c2
    plan = api.Plan([PM.cluster_input(wl, cat)], 64, prec)
    S = 24
    c = plan.chi2(torch.tensor(th[:S], device="cuda")).cpu().numpy()
    ref = oracle(wl, cat, th[:S]).numpy()
    assert np.all(np.abs(c - ref) <= tol * np.abs(ref))
    if prec == "mixed":
        assert np.all(np.abs(c - ref) <= chi2_mixed_bound(wl, cat, th[:S]))
    api.device_error()


def test_full_size_chi2_sampled(lib, c2):
    """The benchmark configuration: 4096 samples in one persistent launch (graph + tuner),
    12 seeded samples checked against the oracle one by one."""
    api, PM = lib
    wl, cat, th = c2
    plan = api.Plan([PM.cluster_input(wl, cat)], 4096, "mixed", flags=api.FLAG_GRAPH | api.FLAG_AUTOTUNE)
    out = plan.chi2(torch.tensor(th, device="cuda"))
    out2 = plan.chi2(torch.tensor(th, device="cuda"))      # graph re-capture (new theta buffer)
    assert torch.equal(out, out2)
    idx = np.concatenate([[0, 4095], np.random.default_rng(9).integers(0, 4096, 10)])
    ref = oracle(wl, cat, th[idx]).numpy()
    c = out.cpu().numpy()[idx]
    assert np.all(np.abs(c - ref) <= 1e-5 * np.abs(ref))
    api.device_error()


@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_every_benchmark_sample_within_tolerance(lib, c2, prec):
    """All 4096 samples of the benchmark launch (graph + tuner) within the stated 1e-5 of the
    FP64 kernel, not a subset: about 3 % of them put an image within |det A| < 3e-3 of a
    critical curve, where M kept in FP32 words would miss it by up to 3e-3 (its weak
    direction is lost; the tiers keep M in float-float words).  The FP64 kernel is held to the
    oracle at 1e-10 by test_cluster_chi2_matches_oracle; the eight samples with the image
    nearest a critical curve are also compared with the oracle directly."""
    api, PM = lib
    wl, cat, th = c2
    t = torch.tensor(th, device="cuda")
    ref = api.Plan([PM.cluster_input(wl, cat)], 4096, "fp64").chi2(t).cpu().numpy()
    plan = api.Plan([PM.cluster_input(wl, cat)], 4096, prec, flags=api.FLAG_GRAPH | api.FLAG_AUTOTUNE)
    got = plan.chi2(t).cpu().numpy()
    rel = np.abs(got - ref) / np.abs(ref)
    print(f"{prec}: max rel {rel.max():.3e}, median {np.median(rel):.3e}")
    assert rel.max() <= 1e-5
    kw = {"fam_adis": OM.single_plane_adis(wl, cat.fam_zs)}
    with torch.no_grad():
        _, A = OG._terms(wl, torch.as_tensor(th), torch.tensor(cat.theta_obs), list(cat.fam_off), **kw)
    near = np.argsort(torch.linalg.det(A).abs().min(1).values.numpy())[:8]
    o = oracle(wl, cat, th[near]).numpy()
    assert np.all(np.abs(got[near] - o) <= 1e-5 * np.abs(o))
    api.device_error()


def test_graph_and_tuner_do_not_change_results(lib, c2):
    api, PM = lib
    wl, cat, th = c2
    t = torch.tensor(th[:256], device="cuda")
    base = api.Plan([PM.cluster_input(wl, cat)], 256, "fp64").chi2(t)
    for flags in (api.FLAG_GRAPH, api.FLAG_AUTOTUNE, api.FLAG_GRAPH | api.FLAG_AUTOTUNE):
        p = api.Plan([PM.cluster_input(wl, cat)], 256, "fp64", flags=flags)
        a = p.chi2(t)
        b = p.chi2(t)                     # replay
        assert torch.equal(a, b)
        assert torch.allclose(a, base, rtol=1e-12, atol=0)


@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_graph_slots_alternate_chi2_and_gradient(lib, c2, prec):
    """A graph-captured plan keeps one graph for the chi^2 launch and one for the gradient
    launch: alternating the two calls replays each and gives the results of a plan without
    graphs (chi^2 bit for bit; the gradient to the order of its shared-memory atomics)."""
    api, PM = lib
    wl, cat, th = c2
    t = torch.tensor(th[:64], device="cuda")
    ref = api.Plan([PM.cluster_input(wl, cat)], 64, prec)
    c0 = ref.chi2(t)
    cg0, g0 = ref.chi2_grad(t)
    p = api.Plan([PM.cluster_input(wl, cat)], 64, prec, flags=api.FLAG_GRAPH)
    c, cg, g = torch.empty_like(c0), torch.empty_like(cg0), torch.empty_like(g0)
    for _ in range(3):                    # fixed buffers: the second and third rounds replay
        c.zero_(); cg.zero_(); g.zero_()
        p.chi2(t, out=c)
        p.chi2_grad(t, out=cg, grad=g)
        assert torch.equal(c, c0) and torch.equal(cg, cg0)
        # the parameter terms reach shared memory by atomics in run-dependent order
        assert float((g - g0).abs().max()) <= 1e-12 * float(g0.abs().max())


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_gradient_matches_oracle_autograd(lib, c2, prec):
    api, PM = lib
    wl, cat, th = c2
    plan = api.Plan([PM.cluster_input(wl, cat)], 16, prec)
    S = 4
    c, g = plan.chi2_grad(torch.tensor(th[:S], device="cuda"))
    cref, gref = oracle(wl, cat, th[:S], grad=True)
    assert grad_ok(g.cpu().numpy(), gref.numpy(), prec)
    assert np.all(np.abs(c.cpu().numpy() - cref.numpy()) <= CHI2_TOL[prec] * np.abs(cref.numpy()))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_gradient_at_round_halo(lib, c2, prec):
    """A sampled ellipticity at exactly eps = 0 (the round profile in the forward pass): the
    adjoint takes the round branch with its exact derivative in eps there.  The mixed tier's
    anchored launch evaluates that round halo in the float-float tier's form."""
    api, PM = lib
    wl, cat, th = c2
    t = th[:3].copy()
    k_eps = [i for i, p in enumerate(wl.params) if p.comp == 0 and p.field == W.F_EPS][0]
    t[:, k_eps] = 0.0
    plan = api.Plan([PM.cluster_input(wl, cat)], 4, prec)
    c, g = plan.chi2_grad(torch.tensor(t, device="cuda"))
    cref, gref = oracle(wl, cat, t, grad=True)
    assert np.all(np.abs(c.cpu().numpy() - cref.numpy()) <= CHI2_TOL[prec] * np.abs(cref.numpy()))
    assert grad_ok(g.cpu().numpy(), gref.numpy(), prec)


@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_gradient_matches_central_differences(lib, c2, prec):
    """Adjoint vs central differences (h = 1e-4 max(|theta_p|, 1), fourth order) of the FP64
    chi^2 of the library."""
    api, PM = lib
    wl, cat, th = c2
    plan = api.Plan([PM.cluster_input(wl, cat)], 64, prec)
    plan64 = api.Plan([PM.cluster_input(wl, cat)], 128, "fp64")
    t0 = torch.tensor(th[:1], device="cuda")
    _, g = plan.chi2_grad(t0)
    P = t0.shape[1]
    rows = []
    for p in range(P):
        h = 1e-4 * max(abs(float(t0[0, p])), 1.0)
        for k in (1, -1, 2, -2):
            t = t0.clone()
            t[0, p] += k * h
            rows.append(t)
    f = plan64.chi2(torch.cat(rows)).cpu().numpy().reshape(P, 4)
    fd = np.array([(8 * (f[p, 0] - f[p, 1]) - (f[p, 2] - f[p, 3])) /
                   (12 * 1e-4 * max(abs(float(t0[0, p])), 1.0)) for p in range(P)])
    assert grad_ok(g.cpu().numpy(), fd[None], prec)


@pytest.mark.parametrize("move", [0.1, 0.3])
def test_mixed_gradient_far_from_plan_fields(lib, c2, move):
    """The mixed tier anchors its gradient's member sums at the plan's fields: each image's sum
    at the fields given to the plan in FP64, each member's change to the sample's fields in
    FP32, rounded relative to the change.  Samples whose scaling amplitudes (v*, cut*) sit 10 %
    and 30 % from the plan's still meet the stated chi^2 and gradient bounds (measured 4.3e-6
    per component with the amplitudes 30 % rms away)."""
    api, PM = lib
    wl, cat, th = c2
    base = np.array([p.base for p in wl.params])
    ks = [i for i, p in enumerate(wl.params) if p.comp == -1]
    t = th[1:4].copy()
    signs = np.array([[1.0, -1.0], [-1.0, 1.0], [1.0, 1.0]])
    for col, k in enumerate(ks):
        t[:, k] = base[k] * (1.0 + move * signs[:, col])
    plan = api.Plan([PM.cluster_input(wl, cat)], 8, "mixed")
    c, g = plan.chi2_grad(torch.tensor(t, device="cuda"))
    cref, gref = oracle(wl, cat, t, grad=True)
    rel = np.abs(c.cpu().numpy() - cref.numpy()) / np.abs(cref.numpy())
    print(f"amplitudes {move:.0%} from the plan's: chi2 rel {rel.max():.2e}")
    assert np.all(rel <= CHI2_TOL["mixed"])
    assert grad_ok(g.cpu().numpy(), gref.numpy(), "mixed")


def test_mixed_gradient_sampled_exponents_far_from_plan(lib, c4):
    """All six scaling slots sampled (one cluster of the 16-cluster workload), the exponents
    lambda, beta, alpha moved by +-0.05 and the amplitudes by +-10 % from the plan's fields: the
    anchored member changes (expm1 of the exponent change times ln L) against the oracle."""
    api, PM = lib
    wls, cats = c4
    w, cat = wls[0], cats[0]
    base = np.array([p.base for p in w.params])
    t = np.tile(base, (3, 1))
    sl = {p.field: i for i, p in enumerate(w.params) if p.comp == -1}
    sg = np.array([1.0, -1.0, 1.0])
    for f in (0, 1, 2):
        t[:, sl[f]] = base[sl[f]] * (1.0 + 0.1 * sg * (1 if f != 1 else -1))
    for f in (3, 4, 5):
        t[:, sl[f]] = base[sl[f]] + 0.05 * sg * (1 if f != 4 else -1)
    plan = api.Plan([PM.cluster_input(w, cat)], 4, "mixed")
    c, g = plan.chi2_grad(torch.tensor(t, device="cuda"))
    cref, gref = oracle(w, cat, t, grad=True)
    rel = np.abs(c.cpu().numpy() - cref.numpy()) / np.abs(cref.numpy())
    with torch.no_grad():
        _, A = OG._terms(w, torch.tensor(t), torch.tensor(cat.theta_obs), list(cat.fam_off),
                         fam_adis=OM.single_plane_adis(w, cat.fam_zs))
    det = torch.linalg.det(A).abs().min(1).values.numpy()
    print(f"exponents moved: chi2 rel {rel.max():.2e}, min |det A| per sample {det}")
    for s_ in range(3):
        assert rel[s_] <= max(CHI2_TOL["mixed"], chi2_mixed_bound(w, cat, t[s_:s_ + 1])[0] / abs(float(cref[s_])))
        assert grad_ok(g[s_:s_ + 1].cpu().numpy(), gref[s_:s_ + 1].numpy(),
                       "mixed" if det[s_] >= 1e-3 else "near_critical")


@pytest.fixture(scope="module")
def c4():
    wls = W.multicluster_c4()
    n = 4
    cats = [W.load_catalogue(f"multicluster_{c:02d}") for c in range(n)]
    return wls[:n], cats


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_multicluster_gradient_one_launch(lib, c4, prec):
    """Four clusters of different sizes (22 parameters incl. all six scaling-relation
    slots) in one launch; 2 samples per cluster against the oracle."""
    api, PM = lib
    wls, cats = c4
    spc = 2
    ths = [W.sample_thetas(W.replace(w, n_samples=spc), w.seed) for w in wls]
    plan = api.Plan([PM.cluster_input(w, c) for w, c in zip(wls, cats)], spc * len(wls), prec)
    c, g = plan.chi2_grad(torch.tensor(np.concatenate(ths), device="cuda"))
    c, g = c.cpu().numpy(), g.cpu().numpy()
    for k, (w, cat) in enumerate(zip(wls, cats)):
        cref, gref = oracle(w, cat, ths[k], grad=True)
        sl = slice(k * spc, (k + 1) * spc)
        rel = np.abs(c[sl] - cref.numpy()) / np.abs(cref.numpy())
        print(f"cluster {k} ({prec}): chi2 rel {rel.max():.2e}")
        assert np.all(rel <= CHI2_TOL[prec])
        assert grad_ok(g[sl], gref.numpy(), prec)


def test_multicluster_forward_every_sample_ff(lib):
    """The float-float tier's forward chi^2 on all 16 synthetic clusters x 64 samples in one
    launch, every sample within the stated 1e-5 of the FP64 kernel.  Its M is kept in
    float-float words: with FP32 words, whose weak direction is lost already at |det A| ~ 0.02,
    one sample missed by 1.0e-5 (the mixed tier's forward launch misses on 13 samples, 3.3e-4
    worst, from its FP32 member sums; see the design notes)."""
    api, PM = lib
    wls = W.multicluster_c4()
    cats = [W.load_catalogue(f"multicluster_{c:02d}") for c in range(len(wls))]
    spc = 64
    th = torch.tensor(np.concatenate([W.sample_thetas(W.replace(w, n_samples=spc), w.seed) for w in wls]),
                      device="cuda")
    ins = [PM.cluster_input(w, c) for w, c in zip(wls, cats)]
    ref = api.Plan(ins, spc * len(wls), "fp64").chi2(th).cpu().numpy()
    got = api.Plan(ins, spc * len(wls), "ff", flags=api.FLAG_GRAPH | api.FLAG_AUTOTUNE).chi2(th).cpu().numpy()
    rel = np.abs(got - ref) / np.abs(ref)
    print(f"ff, 16 clusters: max rel {rel.max():.3e}")
    assert rel.max() <= 1e-5
    api.device_error()


def multiplane_case(n_samples=6):
    """Three planes; besides the main plane's halos and scaling relation, the sampled
    parameters include components of both later planes (an NFW's position, a dPIE's
    position, strength and cut), so the gradient runs through the recursion's positions."""
    wl = W.multiplane_c3(n_grid=8, n_samples=n_samples)
    n1, n2 = len(wl.planes[0].comps), len(wl.planes[1].comps)
    nfw2, pje2 = n1, n1 + 30                  # plane 2: 30 NFW then 30 dPIE
    nfw3, pje3 = n1 + n2, n1 + n2 + 20        # plane 3: 20 NFW then 20 dPIE
    extra = []
    for ci in (nfw2, nfw3):
        c = wl.planes[1 if ci == nfw2 else 2].comps[ci - (n1 if ci == nfw2 else n1 + n2)]
        extra += [W.ParamSpec(ci, W.F_X, W.XF_IDENT, c.x, 0.3, False),
                  W.ParamSpec(ci, W.F_Y, W.XF_IDENT, c.y, 0.3, False)]
    for ci, pl in ((pje2, 1), (pje3, 2)):
        c = wl.planes[pl].comps[ci - (n1 if pl == 1 else n1 + n2)]
        extra += [W.ParamSpec(ci, W.F_X, W.XF_IDENT, c.x, 0.3, False),
                  W.ParamSpec(ci, W.F_Y, W.XF_IDENT, c.y, 0.3, False),
                  W.ParamSpec(ci, W.F_B, W.XF_VDISP, c.vdisp, 0.01, True),
                  W.ParamSpec(ci, W.F_CUT, W.XF_KPC, c.cut_kpc, 0.01, True)]
    return W.replace(wl, params=list(wl.params) + extra)


@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_full_size_gradient_sampled(lib, prec):
    """The benchmark's gradient: all 16 clusters x 64 samples (22 parameters) in one
    graph-captured launch; 6 seeded samples (and the first and last) against the oracle's
    autograd one by one.  Both mixed tiers form A from FP32 psi_ij, so an image near a
    critical curve (these catalogues are the models' own images, magnified ones included)
    moves chi^2 by ~u/|det A|: chi^2 is held to the larger of the stated 1e-5 and the
    first-order bound of tests/helpers.chi2_mixed_bound, and the gradient (which grows like
    1/det^3 there) to the stated 1e-4 per component on samples whose images all keep
    |det A| >= 1e-3 (the mask of the magnification checks), to the near-critical bounds on
    the others (measured: 1.1e-3 per component on a sample with an image at |det A| = 3.9e-4,
    <= 2.4e-5 on the rest)."""
    api, PM = lib
    wls = W.multicluster_c4()
    cats = [W.load_catalogue(f"multicluster_{c:02d}") for c in range(len(wls))]
    ths = [W.sample_thetas(w, w.seed) for w in wls]
    th = np.concatenate(ths)
    plan = api.Plan([PM.cluster_input(w, c) for w, c in zip(wls, cats)], th.shape[0], prec,
                    flags=api.FLAG_GRAPH)
    c, g = plan.chi2_grad(torch.tensor(th, device="cuda"))
    c, g = c.cpu().numpy(), g.cpu().numpy()
    spc = wls[0].n_samples
    idx = np.concatenate([[0, th.shape[0] - 1], np.random.default_rng(29).integers(0, th.shape[0], 6)])
    near = 0
    for s in idx:
        k, j = int(s) // spc, int(s) % spc
        cref, gref = oracle(wls[k], cats[k], ths[k][j:j + 1], grad=True)
        bound = chi2_mixed_bound(wls[k], cats[k], ths[k][j:j + 1])[0]
        bound = max(bound, CHI2_TOL[prec] * abs(float(cref[0])))
        assert abs(c[s] - float(cref[0])) <= bound, (s, c[s], float(cref[0]), bound)
        tier = prec
        with torch.no_grad():
            _, A = OG._terms(wls[k], torch.tensor(ths[k][j:j + 1]), torch.tensor(cats[k].theta_obs),
                             list(cats[k].fam_off), fam_adis=OM.single_plane_adis(wls[k], cats[k].fam_zs))
        if float(torch.linalg.det(A).abs().min()) < 1e-3:
            tier = "near_critical"
            near += 1
        assert grad_ok(g[s:s + 1], gref.numpy(), tier)
    print(f"full-size gradient ({prec}): {near} of {len(idx)} samples with an image at |det A| < 1e-3")
    api.device_error()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5), ("ff", 1e-5)])
def test_multiplane_chi2(lib, c2, prec, tol):
    """Three planes, families at z = 4, every family of the 200-image catalogue kept.  Its
    images are not images of this synthetic model and many sit near its critical curves; the
    forward chi^2 holds the stated bound there because the mixed tiers keep M in float-float
    words (with FP32 words, 94 of 1024 samples of the benchmark's three-plane launch missed
    1e-5, up to 4.3e-3)."""
    api, PM = lib
    _, cat, _ = c2
    wl = W.multiplane_c3(n_grid=8, n_samples=6)
    th = W.sample_thetas(wl, wl.seed)
    cat3 = W.Catalogue(cat.theta_obs, cat.theta_true, cat.fam_off, np.full(len(cat.fam_zs), 4.0))
    plan = api.Plan([PM.cluster_input(wl, cat3)], 6, prec)
    c = plan.chi2(torch.tensor(th, device="cuda")).cpu().numpy()
    ref = oracle(wl, cat3, th).numpy()
    assert np.all(np.abs(c - ref) <= tol * np.abs(ref))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_multiplane_gradient_matches_oracle_autograd(lib, c2, prec):
    """The adjoint of the multi-plane recursion (reverse sweep over the planes, third
    derivatives at every later plane's positions) against the oracle's autograd through
    the same recursion; the families sit at z = 2.5 (behind two planes) and z = 4.  The
    catalogue's images are not images of this synthetic model, and many of them fall near
    its critical curves: the families kept are those with |det A| >= 0.05 at every image."""
    api, PM = lib
    _, cat, _ = c2
    wl = multiplane_case()
    zs = np.where(np.arange(len(cat.fam_zs)) % 2 == 0, 4.0, 2.5)
    th = W.sample_thetas(wl, wl.seed)
    cat3 = families_off_critical(wl, W.Catalogue(cat.theta_obs, cat.theta_true, cat.fam_off, zs), th, 0.05)
    assert len(cat3.theta_obs) >= 30
    plan = api.Plan([PM.cluster_input(wl, cat3)], 6, prec)
    c, g = plan.chi2_grad(torch.tensor(th, device="cuda"))
    cref, gref = oracle(wl, cat3, th, grad=True)
    assert np.all(np.abs(c.cpu().numpy() - cref.numpy()) <= CHI2_TOL[prec] * np.abs(cref.numpy()))
    assert grad_ok(g.cpu().numpy(), gref.numpy(), prec)
    # the later planes' parameters carry gradient
    P0 = len(W.multiplane_c3(n_grid=8, n_samples=6).params)
    assert np.all(np.abs(gref.numpy()[:, P0:]).max(axis=0) > 0)
    api.device_error()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_multiplane_true_images(lib, prec):
    """Three planes with a catalogue of true images of the model itself
    (tests/helpers.three_plane_images: 44 images in 11 families at z = 4, every family kept,
    magnified images with |det A| down to ~0.01 and cond A up to ~60 included), on the
    unperturbed model (chi^2 ~ 4e-3, the catalogue's noise) and seven jittered samples.
    FP64: the stated bounds.  Float-float tier: the forward chi^2 (M in float-float words) to the
    stated 1e-5.  Mixed tier's forward chi^2: at the unperturbed model chi^2 is the
    catalogue's noise (~4e-3), and the FP32 member deflections' rounding (~1e-6") moves it by
    more than 1e-5 of that, so it is held to 1e-5 relative plus the first-order rounding bound
    of tests/helpers.chi2_rounding_bound with FP32 deflections.  The adjoint launch's chi^2,
    whose M is FP32, to 1e-5 relative plus that bound without the deflection term; the
    float-float adjoint's gradient to the stated 1e-4 per component (no image here reaches
    |det A| < 1e-3)."""
    api, PM = lib
    from tests.helpers import chi2_rounding_bound, three_plane_images
    wl, cat = three_plane_images()
    th = W.sample_thetas(wl, wl.seed)[:8]
    plan = api.Plan([PM.cluster_input(wl, cat)], 8, prec)
    t = torch.tensor(th, device="cuda")
    c1 = plan.chi2(t).cpu().numpy()
    c, g = plan.chi2_grad(t)
    c = c.cpu().numpy()
    cref, gref = oracle(wl, cat, th, grad=True)
    cref, gref = cref.numpy(), gref.numpy()
    r1, r = np.abs(c1 - cref) / cref, np.abs(c - cref) / cref
    print(f"three planes, true images ({prec}): chi2 relative error per sample, forward {np.array2string(r1, precision=1)}, "
          f"adjoint launch {np.array2string(r, precision=1)}")
    if prec == "fp64":
        assert r1.max() <= CHI2_TOL[prec] and r.max() <= CHI2_TOL[prec]
    else:
        b_ff = chi2_rounding_bound(wl, cat, th)
        print(f"  bound / chi2 (adjoint launch): {np.array2string(b_ff / cref, precision=1)}")
        if prec == "ff":
            assert r1.max() <= CHI2_TOL[prec]
        else:
            b_fwd = chi2_rounding_bound(wl, cat, th, alpha_coef=4.0)
            assert np.all(np.abs(c1 - cref) <= CHI2_TOL[prec] * cref + b_fwd)
        assert np.all(np.abs(c - cref) <= CHI2_TOL["ff"] * cref + b_ff)
    assert grad_ok(g.cpu().numpy(), gref, prec)
    api.device_error()


def test_multiplane_gradient_matches_central_differences(lib, c2):
    """Float-float adjoint vs fourth-order central differences of the library's FP64 chi^2."""
    api, PM = lib
    _, cat, _ = c2
    wl = multiplane_case(n_samples=1)
    th = W.sample_thetas(wl, wl.seed)
    cat3 = families_off_critical(wl, W.Catalogue(cat.theta_obs, cat.theta_true, cat.fam_off,
                                                 np.full(len(cat.fam_zs), 4.0)), th, 0.05)
    plan = api.Plan([PM.cluster_input(wl, cat3)], 1, "ff")
    plan64 = api.Plan([PM.cluster_input(wl, cat3)], 4 * th.shape[1], "fp64")
    t0 = torch.tensor(th[:1], device="cuda")
    _, g = plan.chi2_grad(t0)
    P = t0.shape[1]
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


def test_single_image_family_contributes_zero_and_galaxy_chi2(lib):
    api, PM = lib
    wl = W.galaxy_c0()
    cat = W.load_catalogue("galaxy_sie_shear")
    wl.params = [W.ParamSpec(0, W.F_X, W.XF_IDENT, 0.0, 0.01, False),
                 W.ParamSpec(0, W.F_Y, W.XF_IDENT, 0.0, 0.01, False),
                 W.ParamSpec(0, W.F_EPS, W.XF_IDENT, wl.planes[0].comps[0].eps, 0.01, False),
                 W.ParamSpec(0, W.F_PA, W.XF_DEG, 30.0, 1.0, False),
                 W.ParamSpec(1, W.F_B, W.XF_IDENT, 0.05 / 0.6353908, 0.002, False)]
    wl.n_samples = 8
    th = W.sample_thetas(wl, 3)
    # add a one-image family at the end
    one = W.Catalogue(np.vstack([cat.theta_obs, [[0.3, 0.2]]]), np.vstack([cat.theta_true, [[0.3, 0.2]]]),
                      np.append(cat.fam_off, cat.fam_off[-1] + 1), np.append(cat.fam_zs, 2.0))
    for prec in ("fp64", "mixed", "ff"):
        p1 = api.Plan([PM.cluster_input(wl, cat)], 8, prec)
        p2 = api.Plan([PM.cluster_input(wl, one)], 8, prec)
        t = torch.tensor(th, device="cuda")
        a, b = p1.chi2(t), p2.chi2(t)
        assert torch.equal(a, b)
        ref = oracle(wl, cat, th).numpy()
        assert np.all(np.abs(a.cpu().numpy() - ref) <= CHI2_TOL[prec] * ref)
        _, g = p2.chi2_grad(t)
        _, gref = oracle(wl, cat, th, grad=True)
        assert grad_ok(g.cpu().numpy(), gref.numpy(), prec)


def test_plan_validation(lib, c2):
    api, PM = lib
    from paper_2609_08649_b300 import _lib as L
    wl, cat, th = c2
    plan = api.Plan([PM.cluster_input(wl, cat)], 8, "mixed")
    with pytest.raises(L.LFError):
        plan.chi2(torch.tensor(th[:9], device="cuda"))          # S > max_samples
    ci = PM.cluster_input(wl, cat)
    ci.fam_ratio[0] = 1.5
    with pytest.raises(L.LFError) as e:
        api.Plan([ci], 8, "mixed")
    assert e.value.status == L.LF_EINVAL
    ci = PM.cluster_input(wl, cat)
    ci.p_field[0] = 9
    with pytest.raises(L.LFError):
        api.Plan([ci], 8, "mixed")
    plan2 = api.Plan([PM.cluster_input(wl, cat), PM.cluster_input(wl, cat)], 8, "mixed")
    with pytest.raises(L.LFError):
        plan2.chi2(torch.tensor(th[:3], device="cuda"))         # not a multiple of 2 clusters


def test_autograd_function(lib, c2):
    api, PM = lib
    wl, cat, th = c2
    plan = api.Plan([PM.cluster_input(wl, cat)], 4, "fp64")
    t = torch.tensor(th[:4], device="cuda", requires_grad=True)
    y = api.chi2(t, plan)
    y.sum().backward()
    _, g = plan.chi2_grad(t.detach())
    assert torch.allclose(t.grad, g)
    # without a gradient requested, forward is the plain chi^2 launch (same values)
    with torch.no_grad():
        y2 = api.chi2(t, plan)
    assert not y2.requires_grad and torch.equal(y2, plan.chi2(t.detach()))
    y3 = api.chi2(t.detach(), plan)
    assert torch.equal(y3, y2)
