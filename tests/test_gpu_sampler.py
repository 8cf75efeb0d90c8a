"""lf_aies_run (stretch-move sampler on the device) against the oracle's sampler with the
same random numbers.  FP64 tier: identical walkers after several steps (the chi^2 values
agree to ~1e-14, so every accept decision is the same).  Mixed tier: identical proposals;
accept decisions can differ only where |log u - log r| is inside the chi^2 tolerance, and
everywhere else the walkers are identical."""
import numpy as np
import pytest
import torch

from oracle import gradient as OG
from oracle import model as OM
from oracle import sampler as OS

pytestmark = pytest.mark.gpu
W = pytest.importorskip("paper_2609_08649_b300.workloads")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import api, model
    wl = W.cluster_c2(n_samples=32)
    cat = W.load_catalogue("cluster_200")
    th = W.sample_thetas(wl, 41)
    base = th[0]
    lo = base - 20 * np.array([p.jitter * (abs(p.base) if p.relative else 1) for p in wl.params])
    hi = base + 20 * np.array([p.jitter * (abs(p.base) if p.relative else 1) for p in wl.params])
    n = len(cat.theta_obs)
    sinv = torch.tensor(np.tile([100.0, 0, 100.0], (n, 1)))
    adis = OM.single_plane_adis(wl, cat.fam_zs)
    f = lambda x: OG.chi2_only(wl, torch.tensor(x), torch.tensor(cat.theta_obs), sinv,
                               list(cat.fam_off), adis).numpy()
    return api, model, wl, cat, th, lo, hi, f


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sampler_matches_oracle(setup, prec):
    api, PM, wl, cat, th, lo, hi, f = setup
    S, steps, a = th.shape[0], 3, 2.0
    u = W.sampler_uniforms(7, steps, S)
    plan = api.Plan([PM.cluster_input(wl, cat)], S, prec)
    x = torch.tensor(th, device="cuda")
    c = plan.chi2(x)
    acc, chain = plan.aies_run(x, c, torch.tensor(u, device="cuda"), a,
                               torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda"), chain=True)
    xo, co = th.copy(), f(th)
    if prec == "fp64":
        n_acc = OS.run(xo, co, u, a, lo, hi, f)
        assert int(acc) == n_acc and n_acc > 0
        assert np.allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-12)
        assert np.allclose(c.cpu().numpy(), co, rtol=1e-10, atol=0)
        assert np.allclose(chain[-1].cpu().numpy(), xo, rtol=0, atol=1e-12)
    else:
        # one step: proposals are FP64 arithmetic on identical inputs; decisions may differ
        # only inside the chi^2 tolerance band around the threshold
        x1 = torch.tensor(th, device="cuda")
        c1 = plan.chi2(x1)
        plan.aies_run(x1, c1, torch.tensor(u[:1], device="cuda"), a, torch.tensor(lo, device="cuda"),
                      torch.tensor(hi, device="cuda"))
        xo, co = th.copy(), f(th)
        OS.run(xo, co, u[:1], a, lo, hi, f)
        same = np.all(np.abs(x1.cpu().numpy() - xo) <= 1e-12, axis=1)
        assert same.mean() >= 0.9
        h = S // 2
        P = th.shape[1]
        for k in np.nonzero(~same[:h])[0]:   # first half: a differing walker is a band decision
            j = OS.partner_of(u[0, k, 0], h)
            z = OS.z_of(u[0, k, 1], a)
            y = th[h + j] + z * (th[k] - th[h + j])
            cy, ck = f(y[None])[0], f(th[k:k + 1])[0]
            log_r = (P - 1) * np.log(z) - 0.5 * (cy - ck)
            assert abs(np.log(u[0, k, 2]) - log_r) < 1e-5 * (abs(cy) + abs(ck))


def test_sampler_validation(setup):
    api, PM, wl, cat, th, lo, hi, f = setup
    from paper_2609_08649_b300 import _lib as L
    plan = api.Plan([PM.cluster_input(wl, cat)], 32, "mixed")
    x = torch.tensor(th[:5], device="cuda")
    c = plan.chi2(x)
    with pytest.raises(L.LFError):        # odd number of walkers
        plan.aies_run(x, c, torch.zeros(1, 5, 3, dtype=torch.float64, device="cuda"), 2.0,
                      torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda"))


# ------------------------------------------------------------ Metropolis-Hastings ----
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mh_matches_oracle(setup, prec):
    api, PM, wl, cat, th, lo, hi, f = setup
    S, steps = 16, 4
    sd = np.array([p.jitter * (abs(p.base) if p.relative else 1) for p in wl.params])
    step = 0.7 * sd
    z, u = W.mh_randoms(9, steps, S, th.shape[1])
    plan = api.Plan([PM.cluster_input(wl, cat)], S, prec)
    x = torch.tensor(th[:S], device="cuda")
    c = plan.chi2(x)
    dev = lambda a: torch.tensor(a, device="cuda")
    acc, tr = plan.mh_run(x, c, dev(z), dev(u), dev(step), dev(lo), dev(hi), trace=True)
    xo, co = th[:S].copy(), f(th[:S])
    if prec == "fp64":
        n_acc = OS.mh_run(xo, co, z, u, step, lo, hi, f)
        assert int(acc) == n_acc and 0 < n_acc < S * steps
        assert np.allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-12)
        assert np.allclose(c.cpu().numpy(), co, rtol=1e-10, atol=0)
        assert np.allclose(tr[-1].cpu().numpy(), xo, rtol=0, atol=1e-12)
    else:
        # one step: identical proposals; a decision may differ only inside the chi^2 band
        x1 = torch.tensor(th[:S], device="cuda")
        c1 = plan.chi2(x1)
        plan.mh_run(x1, c1, dev(z[:1]), dev(u[:1]), dev(step), dev(lo), dev(hi))
        xo, co = th[:S].copy(), f(th[:S])
        OS.mh_run(xo, co, z[:1], u[:1], step, lo, hi, f)
        same = np.all(np.abs(x1.cpu().numpy() - xo) <= 1e-12, axis=1)
        assert same.mean() >= 0.9
        for k in np.nonzero(~same)[0]:
            y = th[k] + step * z[0, k]
            cy, ck = f(y[None])[0], f(th[k:k + 1])[0]
            assert abs(np.log(u[0, k]) + 0.5 * (cy - ck)) < 1e-5 * (abs(cy) + abs(ck))


def test_mh_validation(setup):
    api, PM, wl, cat, th, lo, hi, f = setup
    from paper_2609_08649_b300 import _lib as L
    plan = api.Plan([PM.cluster_input(wl, cat)], 4, "mixed")
    x = torch.tensor(th[:8], device="cuda")
    c = torch.zeros(8, dtype=torch.float64, device="cuda")
    P = th.shape[1]
    z = torch.zeros(1, 8, P, dtype=torch.float64, device="cuda")
    u = torch.full((1, 8), 0.5, dtype=torch.float64, device="cuda")
    s = torch.ones(P, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LFError):      # more chains than the plan's max_samples
        plan.mh_run(x, c, z, u, s, torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda"))
    with pytest.raises(TypeError):      # float32 input refused by the binding
        plan.mh_run(x[:4], c[:4], z[:, :4].float(), u[:, :4], s, torch.tensor(lo, device="cuda"),
                    torch.tensor(hi, device="cuda"))
