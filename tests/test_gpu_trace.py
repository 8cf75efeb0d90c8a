"""Parity of lf_trace_multiplane with the oracle's multi-plane recursion (Sec. 2.2)."""
import numpy as np
import pytest
import torch

from oracle import cosmology as cz
from oracle import lensing as OL
from oracle import model as OM
from tests.helpers import U32, grid_xy

pytestmark = pytest.mark.gpu
W = pytest.importorskip("paper_2609_08649_b300.workloads")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import api, model
    return api, model


def _oracle_trace(wl, x, y):
    planes = OM.build_planes(wl)
    r, rs = cz.multiplane_ratios([p.z for p in wl.planes], wl.z_s)
    beta, A = OL.trace_multiplane(planes, r, rs, torch.tensor(x)[None], torch.tensor(y)[None])
    return beta[0].numpy(), A[0].numpy()


def _jac_bound(wl, x, y):
    """First-order bound on |A - A_oracle| per ray for the mixed tiers.  Each plane's Psi_j is
    the FP32 sum of its components, |d Psi_j| <= d_j = 16 u S_j with S_j = sum_k |psi_k(theta_j)|
    (16 u covers the FP32 NFW), while the recursion and the products Psi_j A_j are carried in
    float-float or FP64.  Linearising the recursion, with infinity norms a_j = |A_j|,
    p_j = |Psi_j| and |d Psi_j| <= 2 d_j:
      e_j = |d A_j| <= sum_{i<j} r_ij (2 d_i a_i + p_i e_i),
      |d A| <= sum_j rs_j (2 d_j a_j + p_j e_j)."""
    from tests.helpers import oracle_plane_terms
    planes = OM.build_planes(wl)
    r, rs = cz.multiplane_ratios([p.z for p in wl.planes], wl.z_s)
    _, alphas, psis, As = OL.multiplane_parts(planes, r, torch.tensor(x)[None], torch.tensor(y)[None])
    t1 = np.stack([x, y], -1)
    inf = lambda M: M[0].abs().sum(-1).amax(-1).numpy()
    d, a, pn = [], [], []
    for j, pl in enumerate(planes):
        tj = t1.copy()
        for i in range(j):
            tj = tj - r[i][j] * alphas[i][0].numpy()
        d.append(16 * U32 * oracle_plane_terms(pl, tj[:, 0], tj[:, 1])[2])
        a.append(inf(As[j]))
        pn.append(inf(psis[j]))
    e = []
    for j in range(len(planes)):
        e.append(sum((r[i][j] * (2 * d[i] * a[i] + pn[i] * e[i]) for i in range(j)), np.zeros_like(x)))
    tot = sum(rs[j] * (2 * d[j] * a[j] + pn[j] * e[j]) for j in range(len(planes)))
    return 1e-12 + tot


def _check_mu(A, A0):
    """mu = 1/det A where |det A| >= 1e-3, relative error bounded by the error of det A: with
    |dA_ij| <= e and |A_ij| <= m, |d det| <= 4 m e + 2 e^2 (four products of the 2x2
    determinant), and |1/det - 1/det0| |det0| = |d det| / |det| <= |d det| / (|det0| - |d det|)."""
    det = A[:, 0, 0] * A[:, 1, 1] - A[:, 0, 1] * A[:, 1, 0]
    det0 = A0[:, 0, 0] * A0[:, 1, 1] - A0[:, 0, 1] * A0[:, 1, 0]
    m = np.abs(det0) >= 1e-3
    dA = np.abs(A - A0).max((1, 2))
    ddet = 4 * np.abs(A0).max((1, 2)) * dA + 2 * dA * dA
    rel = np.abs(1 / det[m] - 1 / det0[m]) * np.abs(det0[m])
    assert np.all(rel <= 1e-12 + ddet[m] / (np.abs(det0[m]) - ddet[m])), rel.max()


def _abs_scale(wl, x, y):
    """sum over planes and components of |alpha_k| at the unlensed position (error scale)."""
    from tests.helpers import oracle_plane_terms
    tot = np.zeros_like(x)
    for p in OM.build_planes(wl):
        tot += oracle_plane_terms(p, x, y)[1]
    return tot


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_three_plane_grid_matches_oracle(lib, prec):
    api, PM = lib
    wl = W.multiplane_c3(n_grid=8)
    grid = W.Grid(-80.0, -79.0, 2.3, 2.1, 71, 77)
    X, Y = grid_xy(grid)
    planes = PM.device_planes(wl)
    r = PM.multiplane_ratios(wl.cosmo, [p.z for p in wl.planes], wl.z_s)
    beta, A = api.trace_multiplane(planes, r, grid=grid, precision=prec)
    b0, A0 = _oracle_trace(wl, X.ravel(), Y.ravel())
    beta, A = beta.cpu().numpy(), A.cpu().numpy()
    if prec == "fp64":
        assert np.abs(beta - b0).max() < 1e-10
        assert np.abs(A - A0).max() < 1e-10
    else:
        sa = _abs_scale(wl, X.ravel(), Y.ravel())
        tol = 1e-6 + 16 * U32 * sa
        assert np.all(np.abs(beta - b0).max(1) <= tol)
        ta = _jac_bound(wl, X.ravel(), Y.ravel())
        dA = np.abs(A - A0).max((1, 2))
        print(f"{prec}: max |dA| = {dA.max():.3e}, max |dA| / bound = {(dA / ta).max():.3f}")
        assert np.all(dA <= ta)
        _check_mu(A, A0)
    # the Jacobian of a multi-plane lens is not symmetric
    assert np.abs(A[:, 0, 1] - A[:, 1, 0]).max() > 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_single_plane_trace_equals_lens_map(lib, prec):
    api, PM = lib
    wl = W.cluster_c1()
    dp = PM.device_planes(wl)
    a = cz.a_dis(0.5, 2.0)
    r = np.array([[0.0], [a]])
    pts = torch.tensor(np.random.default_rng(5).uniform(-60, 60, (333, 2)), device="cuda")
    beta, A = api.trace_multiplane(dp, r, theta=pts, precision=prec)
    o = api.jacobian_points(dp[0], pts, a, prec)
    bx = pts[:, 0] - a * o["ax"]
    # the two kernels may contract multiply-adds differently: FP32-level differences in mixed
    tol = {"fp64": 1e-12, "mixed": 5e-5, "ff": 1e-9}[prec]
    assert torch.allclose(beta[:, 0], bx, rtol=0, atol=tol)
    # A11 = 1 - a psi_xx and kappa = (psi_xx + psi_yy)/2 -> trace check
    tr = A[:, 0, 0] + A[:, 1, 1]
    assert torch.allclose(tr, 2 - 2 * a * o["kappa"].double(), atol=1e-5)
    assert torch.allclose(A[:, 0, 1], A[:, 1, 0], atol=1e-15)


def test_trace_images_of_chi2_workload(lib):
    """The 200-image set traced through the 3 planes to z_s = 4 (mixed) vs the oracle."""
    api, PM = lib
    wl = W.multiplane_c3(n_grid=8)
    cat = W.load_catalogue("cluster_200")
    planes = PM.device_planes(wl)
    r = PM.multiplane_ratios(wl.cosmo, [p.z for p in wl.planes], wl.z_s)
    pts = torch.tensor(cat.theta_obs, device="cuda")
    beta, A = api.trace_multiplane(planes, r, theta=pts, precision="mixed")
    b0, A0 = _oracle_trace(wl, cat.theta_obs[:, 0].copy(), cat.theta_obs[:, 1].copy())
    sa = _abs_scale(wl, cat.theta_obs[:, 0].copy(), cat.theta_obs[:, 1].copy())
    assert np.all(np.abs(beta.cpu().numpy() - b0).max(1) <= 1e-6 + 16 * U32 * sa)
    api.device_error()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_three_plane_trace_with_elliptical_nfw_halos(lib, prec):
    """The three-plane model with the main plane's two halos replaced by the elliptical NFW
    halos of the Hera-like workload (38-term cored-steep-ellipsoid sums), against the
    oracle's recursion; tolerances as for the three-plane grid (one ray lands 0.04" from an
    NFW centre on the second plane, where the Jacobian magnifies errors in psi_ij)."""
    api, PM = lib
    wl = W.multiplane_c3(n_grid=8)
    halos = [c for c in W.cluster_c5_enfw(n_samples=1).planes[0].comps if c.kind == W.ENFW]
    p0 = wl.planes[0]
    wl = W.replace(wl, planes=[W.replace(p0, comps=halos + list(p0.comps[2:]))] + list(wl.planes[1:]),
                   params=[])
    grid = W.Grid(-80.0, -79.0, 2.3, 2.1, 71, 77)
    X, Y = grid_xy(grid)
    planes = PM.device_planes(wl)
    r = PM.multiplane_ratios(wl.cosmo, [p.z for p in wl.planes], wl.z_s)
    beta, A = api.trace_multiplane(planes, r, grid=grid, precision=prec)
    b0, A0 = _oracle_trace(wl, X.ravel(), Y.ravel())
    beta, A = beta.cpu().numpy(), A.cpu().numpy()
    api.device_error()
    if prec == "fp64":
        assert np.abs(beta - b0).max() < 1e-10
        assert np.abs(A - A0).max() < 1e-10
    else:
        sa = _abs_scale(wl, X.ravel(), Y.ravel())
        assert np.all(np.abs(beta - b0).max(1) <= 1e-6 + 16 * U32 * sa)
        ta = _jac_bound(wl, X.ravel(), Y.ravel())
        dA = np.abs(A - A0).max((1, 2))
        print(f"{prec}: max |dA| = {dA.max():.3e}, max |dA| / bound = {(dA / ta).max():.3f}")
        assert np.all(dA <= ta)
        _check_mu(A, A0)


def test_full_size_trace_sampled(lib):
    """The benchmark's trace: the 2048^2 grid at 0.08" through the three planes in one launch
    (mixed tier); 400 seeded pixels against the oracle's recursion one by one."""
    api, PM = lib
    wl = W.multiplane_c3()
    planes = PM.device_planes(wl)
    r = PM.multiplane_ratios(wl.cosmo, [p.z for p in wl.planes], wl.z_s)
    beta, A = api.trace_multiplane(planes, r, grid=wl.grid, precision="mixed")
    api.device_error()
    n = wl.grid.nx * wl.grid.ny
    idx = np.random.default_rng(23).integers(0, n, 400)
    idx[:2] = [0, n - 1]
    X = wl.grid.x0 + wl.grid.dx * (idx % wl.grid.nx)
    Y = wl.grid.y0 + wl.grid.dy * (idx // wl.grid.nx)
    b0, A0 = _oracle_trace(wl, X, Y)
    bt = torch.as_tensor(idx, device=beta.device)
    b, Ag = beta[bt].cpu().numpy(), A[bt].cpu().numpy()
    sa = _abs_scale(wl, X, Y)
    assert np.all(np.abs(b - b0).max(1) <= 1e-6 + 16 * U32 * sa)
    dA = np.abs(Ag - A0).max((1, 2))
    ta = _jac_bound(wl, X, Y)
    print(f"2048^2 mixed trace: max |dA| = {dA.max():.3e}, max |dA| / bound = {(dA / ta).max():.3f}")
    assert np.all(dA <= ta)
    _check_mu(Ag, A0)
