"""Pins of the oracle's per-component closed forms against what the mathematics fixes
(not against the oracle itself): the SIS constant deflection, scale freedom of the
singular ellipsoid, Hessian = derivative of alpha (curl-free), kappa from the surface
density definitions, the elliptical deflection integral, the point-mass far field, and
branch continuity of the NFW forms."""
import math

import numpy as np
import pytest
import torch
from scipy.integrate import quad

from oracle import cse_nfw as C
from oracle import profiles as pr

T = lambda *v: torch.tensor(v, dtype=torch.float64)
PTS_X = T(0.3, -1.2, 2.5, 0.01, -3.3, 4.0)
PTS_Y = T(0.7, 0.1, -1.9, -0.02, 2.2, 0.5)


def fd_jac(fn, x, y, h=1e-5):
    axp, axm, ayp, aym = fn(x + h, y), fn(x - h, y), fn(x, y + h), fn(x, y - h)
    return ((axp[0] - axm[0]) / (2 * h), (ayp[1] - aym[1]) / (2 * h),
            (ayp[0] - aym[0]) / (2 * h), (axp[1] - axm[1]) / (2 * h))


PROFILES = {
    "sie": lambda x, y: pr.sie(x, y, 1.3, 0.7, 0.5, 0.2),
    "sie_round": lambda x, y: pr.sie(x, y, 1.3, 1.0, 0.5, 0.2),
    "sie_nearly_round": lambda x, y: pr.sie(x, y, 1.3, 1 - 1e-7, 0.5, 0.2),
    "dpie": lambda x, y: pr.dpie(x, y, 1.0, 0.6, -0.3, 0.1, 3.0),
    "dpie_round": lambda x, y: pr.dpie(x, y, 1.0, 1.0, -0.3, 0.1, 3.0),
    "pje_sph": lambda x, y: pr.pje_sph(x, y, 1.0, 0.1, 3.0),
    "nfw": lambda x, y: pr.nfw_sph(x, y, 0.2, 1.5),
    "shear": lambda x, y: pr.shear(x, y, 0.07, 0.4),
    "cse": lambda x, y: pr.cse_uv(x, y, 0.7, 0.3),
    "enfw": lambda x, y: pr.enfw(x, y, 0.2, 0.75, 0.5, 2.5, *C.table()),
}


def test_sis_deflection_is_constant():
    th = torch.linspace(0, 2 * math.pi, 17)[:-1].double()
    for rad in (0.05, 1.7, 40.0):
        dx, dy = rad * torch.cos(th), rad * torch.sin(th)
        # q = 1 exactly takes the round limit; q = 1 - 1e-12 goes through atan/atanh
        # and differs from the SIS by O(1 - q) only
        for q in (1.0, 1 - 1e-12):
            ax, ay, *_ = pr.sie(dx, dy, 1.3, q, 0.4, 0.0)
            assert torch.allclose(torch.hypot(ax, ay), torch.full_like(ax, 1.3), rtol=0, atol=1e-11)


def test_singular_ellipsoid_is_scale_free():
    for lam in (0.1, 3.0, 77.0):
        a = pr.sie(PTS_X, PTS_Y, 1.3, 0.6, 0.2, 0.0)
        b = pr.sie(lam * PTS_X, lam * PTS_Y, 1.3, 0.6, 0.2, 0.0)
        assert torch.allclose(a[0], b[0], atol=1e-12) and torch.allclose(a[1], b[1], atol=1e-12)
        # psi_ij scales as 1/lambda
        for i in (2, 3, 4):
            assert torch.allclose(a[i], lam * b[i], atol=1e-12)


@pytest.mark.parametrize("name", sorted(PROFILES))
def test_hessian_is_derivative_of_alpha_and_curl_free(name):
    fn = PROFILES[name]
    out = fn(PTS_X, PTS_Y)
    dxax, dyay, dyax, dxay = fd_jac(fn, PTS_X, PTS_Y)
    assert torch.allclose(out[2], dxax, atol=2e-9)
    assert torch.allclose(out[3], dyay, atol=2e-9)
    assert torch.allclose(out[4], dyax, atol=2e-9)
    assert torch.allclose(dxay, dyax, atol=2e-9)      # curl-free: d_x alpha_y = d_y alpha_x


def test_sie_kappa_matches_density():
    b, q, pa, s = 1.3, 0.7, 0.5, 0.2
    out = pr.sie(PTS_X, PTS_Y, b, q, pa, s)
    c, sn = math.cos(pa), math.sin(pa)
    u, v = c * PTS_X + sn * PTS_Y, -sn * PTS_X + c * PTS_Y
    kappa = 0.5 * b / torch.sqrt(s * s + u * u + v * v / (q * q))
    assert torch.allclose(0.5 * (out[2] + out[3]), kappa, atol=1e-13)


def test_dpie_kappa_matches_density():
    b, q, pa, s, a = 1.0, 0.6, -0.3, 0.1, 3.0
    out = pr.dpie(PTS_X, PTS_Y, b, q, pa, s, a)
    c, sn = math.cos(pa), math.sin(pa)
    u, v = c * PTS_X + sn * PTS_Y, -sn * PTS_X + c * PTS_Y
    xi2 = u * u + v * v / (q * q)
    kappa = 0.5 * b * (1 / torch.sqrt(s * s + xi2) - 1 / torch.sqrt(a * a + xi2))
    assert torch.allclose(0.5 * (out[2] + out[3]), kappa, atol=1e-13)


def test_sie_deflection_equals_elliptical_integral():
    """alpha of an elliptical density kappa(xi), xi^2 = u^2 + v^2/q^2, from the
    potential-theory integrals alpha_u = q u J0, alpha_v = q v J1 with
    J_n = int_0^1 kappa(xi(w)) / (1 - (1 - q^2) w)^(n + 1/2) dw,
    xi(w)^2 = w (u^2 + v^2 / (1 - (1 - q^2) w)); evaluated by quadrature."""
    b, q, s = 1.3, 0.65, 0.25
    kap = lambda xi2: 0.5 * b / math.sqrt(s * s + xi2)
    for u, v in [(0.3, 0.7), (-1.2, 0.1), (2.5, -1.9), (0.05, 3.0)]:
        def J(n):
            f = lambda w: kap(w * (u * u + v * v / (1 - (1 - q * q) * w))) / (1 - (1 - q * q) * w) ** (n + 0.5)
            return quad(f, 0, 1, epsabs=1e-14, epsrel=1e-13)[0]
        au, av = q * u * J(0), q * v * J(1)
        o = pr.sie(T(u), T(v), b, q, 0.0, s)
        assert abs(float(o[0]) - au) < 1e-11 and abs(float(o[1]) - av) < 1e-11


def test_rotation_convention():
    """The position angle rotates the whole field counter-clockwise."""
    pa = 0.7
    c, s = math.cos(pa), math.sin(pa)
    u, v = T(1.1, -0.4), T(0.3, 2.0)
    x, y = c * u - s * v, s * u + c * v
    o0 = pr.sie(u, v, 1.0, 0.6, 0.0, 0.1)
    o1 = pr.sie(x, y, 1.0, 0.6, pa, 0.1)
    assert torch.allclose(o1[0], c * o0[0] - s * o0[1], atol=1e-13)
    assert torch.allclose(o1[1], s * o0[0] + c * o0[1], atol=1e-13)
    # major axis along the position angle: kappa falls slower along it
    k_major = pr.sie(T(2 * c), T(2 * s), 1.0, 0.6, pa, 0.1)
    k_minor = pr.sie(T(-2 * s), T(2 * c), 1.0, 0.6, pa, 0.1)
    assert float(k_major[2] + k_major[3]) > float(k_minor[2] + k_minor[3])


def _mean_kappa(kappa_fn, r):
    return 2.0 / r ** 2 * quad(lambda t: t * kappa_fn(t), 0, r, epsabs=0, epsrel=1e-13, limit=200)[0]


def test_pje_sph_mean_convergence_from_density():
    b, s, a = 1.0, 0.1, 3.0
    kappa = lambda r: 0.5 * b * (1 / math.sqrt(s * s + r * r) - 1 / math.sqrt(a * a + r * r))
    for r in (0.01, 0.5, 3.0, 40.0):
        o = pr.pje_sph(T(r), T(0.0), b, s, a)
        assert abs(float(o[0]) / r - _mean_kappa(kappa, r)) < 1e-12
        assert abs(0.5 * float(o[2] + o[3]) - kappa(r)) < 1e-13


def test_pje_far_field_is_point_mass():
    """For r >> cut, |alpha| r -> b (cut - core) (point mass of theta_E^2 = b(cut - core)),
    with the next term -(cut + core)/(2 r) relative."""
    b, s, a = 1.2, 0.2, 5.0
    for r in (1e3, 1e4, 1e5):
        o = pr.pje_sph(T(r), T(0.0), b, s, a)
        ratio = float(o[0]) * r / (b * (a - s))
        assert abs(ratio - 1 + (a + s) / (2 * r)) < 5 * ((a + s) / r) ** 2


def test_nfw_kappa_from_3d_density():
    """kappa(x) = kappa_s int dz / (t (1 + t)^2), t = sqrt(x^2 + z^2): the projected NFW
    density (rho = rho_s / ((r/rs)(1 + r/rs)^2), kappa_s = rho_s rs / Sigma_cr)."""
    ks, rs = 0.2, 1.5
    for x in (0.05, 0.5, 0.999, 1.0, 1.0004, 2.0, 9.0):
        f = lambda z: 1.0 / (math.sqrt(x * x + z * z) * (1 + math.sqrt(x * x + z * z)) ** 2)
        kap = 2 * ks * quad(f, 0, math.inf, epsabs=0, epsrel=1e-13, limit=400)[0]
        o = pr.nfw_sph(T(x * rs), T(0.0), ks, rs)
        assert abs(0.5 * float(o[2] + o[3]) - kap) < 1e-11 * max(1.0, kap)


def test_nfw_mean_convergence_from_density():
    ks, rs = 0.2, 1.5
    kappa = lambda r: 0.5 * float(sum(pr.nfw_sph(T(r), T(0.0), ks, rs)[2:4]))
    for r in (0.3, 1.5, 1.5 * (1 + 5e-4), 6.0):
        o = pr.nfw_sph(T(r), T(0.0), ks, rs)
        assert abs(float(o[0]) / r - _mean_kappa(kappa, r)) < 1e-10


def test_nfw_branches_are_continuous_at_x_equal_one():
    ks, rs = 0.2, 1.5
    for w in (1e-3, 1e-6):
        xs = T(rs * math.sqrt(1 - w * (1 + 1e-9)), rs * math.sqrt(1 - w * (1 - 1e-9)),
               rs * math.sqrt(1 + w * (1 - 1e-9)), rs * math.sqrt(1 + w * (1 + 1e-9)))
        o = pr.nfw_sph(xs, torch.zeros_like(xs), ks, rs)
        k = 0.5 * (o[2] + o[3])
        assert abs(float(k[0] - k[1])) < 1e-12 and abs(float(k[2] - k[3])) < 1e-12
        assert abs(float(o[0][0] - o[0][1])) < 1e-12 and abs(float(o[0][2] - o[0][3])) < 1e-12
    o = pr.nfw_sph(T(rs), T(0.0), ks, rs)
    assert abs(0.5 * float(o[2] + o[3]) - 2 * ks / 3) < 1e-14          # kappa(1) = 2 ks / 3
    assert abs(float(o[0]) / rs - 4 * ks * (1 + math.log(0.5))) < 1e-14   # h(1) = 1 + ln 1/2


def test_shear_is_linear_and_traceless():
    g, pa = 0.07, 0.4
    o = pr.shear(PTS_X, PTS_Y, g, pa)
    assert torch.allclose(o[2] + o[3], torch.zeros(1, dtype=torch.float64), atol=1e-16)
    assert abs(float(torch.hypot(o[2], o[4])[0]) - g) < 1e-15
    o2 = pr.shear(2 * PTS_X, 2 * PTS_Y, g, pa)
    assert torch.allclose(o2[0], 2 * o[0]) and torch.allclose(o2[1], 2 * o[1])
    # the shear stretches along pa + 90 deg is compressive: psi = (g/2) r^2 cos 2(phi - pa)
    r = 1.7
    psi = lambda phi: 0.5 * g * r * r * math.cos(2 * (phi - pa))
    phi = 0.9
    x, y = r * math.cos(phi), r * math.sin(phi)
    h = 1e-6
    dpsi_dx = (0.5 * g * ((x + h) ** 2 + y * y) * math.cos(2 * (math.atan2(y, x + h) - pa))
               - 0.5 * g * ((x - h) ** 2 + y * y) * math.cos(2 * (math.atan2(y, x - h) - pa))) / (2 * h)
    ox = pr.shear(T(x), T(y), g, pa)
    assert abs(float(ox[0]) - dpsi_dx) < 1e-8
    assert abs(psi(phi) - 0.5 * g * r * r * math.cos(2 * (phi - pa))) == 0


# ---------------------------------------------------------------- m = 3 multipole ----
def _mp_potential(x, y, amp, pa):
    """The definition, psi = amp r^2 cos 3(phi - pa)."""
    return amp * (x * x + y * y) * np.cos(3.0 * (np.arctan2(y, x) - pa))


def test_multipole3_alpha_is_the_gradient_of_its_potential():
    rng = np.random.default_rng(5)
    x, y = rng.uniform(-40, 40, 50), rng.uniform(-40, 40, 50)
    amp, pa = 0.004, 0.3
    ax, ay, *_ = pr.multipole3(torch.tensor(x), torch.tensor(y), amp, pa)
    h = 1e-4
    fx = (_mp_potential(x + h, y, amp, pa) - _mp_potential(x - h, y, amp, pa)) / (2 * h)
    fy = (_mp_potential(x, y + h, amp, pa) - _mp_potential(x, y - h, amp, pa)) / (2 * h)
    assert np.allclose(ax.numpy(), fx, rtol=1e-7, atol=1e-9)
    assert np.allclose(ay.numpy(), fy, rtol=1e-7, atol=1e-9)


def test_multipole3_hessian_and_convergence():
    rng = np.random.default_rng(6)
    x, y = torch.tensor(rng.uniform(-40, 40, 50)), torch.tensor(rng.uniform(-40, 40, 50))
    amp, pa = 0.004, -0.7
    ax, ay, pxx, pyy, pxy = pr.multipole3(x, y, amp, pa)
    h = 1e-5
    axp, ayp, *_ = pr.multipole3(x + h, y, amp, pa)
    axm, aym, *_ = pr.multipole3(x - h, y, amp, pa)
    bxp, byp, *_ = pr.multipole3(x, y + h, amp, pa)
    bxm, bym, *_ = pr.multipole3(x, y - h, amp, pa)
    assert torch.allclose(pxx, (axp - axm) / (2 * h), rtol=1e-6, atol=1e-9)
    assert torch.allclose(pyy, (byp - bym) / (2 * h), rtol=1e-6, atol=1e-9)
    assert torch.allclose(pxy, (ayp - aym) / (2 * h), rtol=1e-6, atol=1e-9)
    assert torch.allclose(pxy, (bxp - bxm) / (2 * h), rtol=1e-6, atol=1e-9)   # curl-free
    # Laplacian of amp r^2 cos 3D: (n^2 - m^2) amp cos 3D with n = 2, m = 3
    kappa = 0.5 * (pxx + pyy)
    ref = -2.5 * amp * torch.cos(3.0 * (torch.atan2(y, x) - pa))
    assert torch.allclose(kappa, ref, rtol=1e-12, atol=1e-15)


def test_multipole3_threefold_symmetry_and_orientation():
    x = torch.tensor([3.0, -7.0, 12.5], dtype=torch.float64)
    y = torch.tensor([4.0, 1.0, -9.0], dtype=torch.float64)
    amp, pa = 0.01, 0.2
    t = 2.0 * math.pi / 3.0
    xr, yr = math.cos(t) * x - math.sin(t) * y, math.sin(t) * x + math.cos(t) * y
    a0 = pr.multipole3(x, y, amp, pa)
    a1 = pr.multipole3(xr, yr, amp, pa)
    assert torch.allclose(a1[0], math.cos(t) * a0[0] - math.sin(t) * a0[1], atol=1e-13)
    assert torch.allclose(a1[1], math.sin(t) * a0[0] + math.cos(t) * a0[1], atol=1e-13)
    # along the orientation axis the deflection is radial and outward, 2 amp r
    ax, ay, *_ = pr.multipole3(torch.tensor([5.0 * math.cos(pa)], dtype=torch.float64),
                               torch.tensor([5.0 * math.sin(pa)], dtype=torch.float64), amp, pa)
    ref = torch.tensor([10 * amp * math.cos(pa), 10 * amp * math.sin(pa)], dtype=torch.float64)
    assert torch.allclose(torch.stack([ax, ay]).flatten(), ref, atol=1e-14)


@pytest.mark.parametrize("prof", ["sie", "dpie"])
def test_round_branch_derivative_in_q_is_the_elliptical_limit(prof):
    """At q = 1 the closed forms take the round branch; its derivative in q (autograd) must
    equal the one-sided limit q -> 1- of the elliptical branch's derivative, here by
    Richardson extrapolation of difference quotients of the elliptical values (the
    derivative in eps = (1 - q)/(1 + q) follows by dq/deps = -2 at eps = 0)."""
    fn = (lambda q: pr.sie(PTS_X, PTS_Y, 1.3, q, 0.5, 0.2)) if prof == "sie" else \
         (lambda q: pr.dpie(PTS_X, PTS_Y, 1.0, q, -0.3, 0.1, 3.0))
    q1 = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    out = fn(q1)
    f1 = [o.detach() for o in out]
    for k in range(5):
        g = torch.stack([torch.autograd.grad(out[k][i], q1, retain_graph=True)[0]
                         for i in range(len(PTS_X))])
        # D(h) = (f(1) - f(1 - h)) / h = f' - h f''/2 + ...; two Richardson levels
        D = lambda h: (f1[k] - fn(torch.tensor(1.0 - h, dtype=torch.float64))[k]) / h
        h = 1e-3
        d1, d2, d4 = D(h), D(h / 2), D(h / 4)
        r1, r2 = 2 * d2 - d1, 2 * d4 - d2
        lim = (4 * r2 - r1) / 3
        scale = max(float(g.abs().max()), 1e-3)
        assert float((g - lim).abs().max()) < 1e-7 * scale, (k, g, lim)


def test_nfw_mean_convergence_near_the_centre_to_full_precision():
    """alpha = 4 ks rs h(x) / x with h = ln(x/2) + arccosh(1/x)/sqrt(1 - x^2) (x < 1), or
    ln(x/2) + arccos(1/x)/sqrt(x^2 - 1) (x > 1), against the same formula evaluated with 50
    digits (mpmath): near the centre the two terms of h cancel, and h must still carry full
    FP64 precision (the multi-plane Jacobian multiplies its error by 1/x^2)."""
    import mpmath as mp
    mp.mp.dps = 50
    ks, rs = 0.3, 4.0
    for x in (1e-4, 1e-3, 3.6e-3, 1e-2, 0.1, 0.4, 0.49, 0.51, 0.8, 1.5, 4.0):
        X = mp.mpf(x)
        if x < 1:
            h = mp.log(X / 2) + mp.acosh(1 / X) / mp.sqrt(1 - X * X)
        else:
            h = mp.log(X / 2) + mp.acos(1 / X) / mp.sqrt(X * X - 1)
        ref = float(4 * ks * rs * h / X)
        o = pr.nfw_sph(T(x * rs), T(0.0), ks, rs)
        assert abs(float(o[0]) / ref - 1) < 1e-13, (x, float(o[0]), ref)
