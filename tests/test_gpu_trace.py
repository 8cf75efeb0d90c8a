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
        assert np.abs(A - A0).max() < 1e-4
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
        assert np.abs(A - A0).max() < 1e-4


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
    assert np.abs(Ag - A0).max() < 1e-4
