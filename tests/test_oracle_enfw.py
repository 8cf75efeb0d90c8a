"""Pins of the oracle's elliptical NFW (Sec. 4.1, 4.2: approximated as in Oguri 2021 by a sum
of cored steep ellipsoids) against what the mathematics fixes: the CSE deflection from the
potential-theory integrals of its density, kappa = tr Psi / 2 against the CSE density, the
fit of the spherical NFW convergence, the spherical limit against the closed-form NFW, the
elliptical deflection against the integrals of the exact elliptical NFW density, and the
potential's gradient."""
import math

import numpy as np
import pytest
import torch
from scipy.integrate import quad

from oracle import cse_nfw as C
from oracle import lensing as L
from oracle import profiles as pr

T = lambda *v: torch.tensor(v, dtype=torch.float64)


def schramm(kappa, u, v, q):
    """alpha_u = q u J0, alpha_v = q v J1, J_n = int_0^1 kappa(xi^2(w)) / (1 - (1 - q^2) w)^(n + 1/2) dw,
    xi^2(w) = w (u^2 + v^2 / (1 - (1 - q^2) w)) (homoeoidal density kappa(u^2 + v^2 / q^2))."""
    def J(n):
        f = lambda w: kappa(w * (u * u + v * v / (1 - (1 - q * q) * w))) / (1 - (1 - q * q) * w) ** (n + 0.5)
        pts = [1e-6, 1e-4, 1e-2] if u * u + v * v > 1 else None
        return quad(f, 0, 1, epsabs=0, epsrel=1e-12, limit=400, points=pts)[0]
    return q * u * J(0), q * v * J(1)


@pytest.mark.parametrize("q,s", [(0.6, 0.3), (0.85, 0.02), (1.0, 0.5)])
def test_cse_deflection_equals_elliptical_integral(q, s):
    kap = lambda xi2: 0.5 / (s * s + xi2) ** 1.5
    for u, v in [(0.3, 0.7), (-1.2, 0.1), (2.5, -1.9), (0.05, 3.0), (0.01, -0.004)]:
        au, av = schramm(kap, u, v, q)
        o = pr.cse_uv(T(u), T(v), q, s)
        assert abs(float(o[0]) - au) < 1e-10 * max(1.0, abs(au)), (u, v, float(o[0]), au)
        assert abs(float(o[1]) - av) < 1e-10 * max(1.0, abs(av)), (u, v, float(o[1]), av)


def test_cse_hessian_trace_is_the_density():
    q, s = 0.7, 0.4
    u, v = T(0.3, -1.2, 2.5, 0.01, -3.3), T(0.7, 0.1, -1.9, -0.02, 2.2)
    o = pr.cse_uv(u, v, q, s)
    kappa = 0.5 / (s * s + u * u + v * v / (q * q)) ** 1.5
    assert torch.allclose(0.5 * (o[2] + o[3]), kappa, rtol=1e-13, atol=0)


def test_nfw_fit_accuracy():
    """The CSE sum reproduces the spherical NFW g(x) to 2e-6 relative on 1e-4 <= x <= 1e3
    (between the fit's nodes too), with non-negative coefficients."""
    s, a = C.table()
    assert np.all(a > 0) and len(a) >= 30
    x = np.logspace(-4, 3, 9973)
    rel = np.abs(C.g_approx(x) / C.nfw_g(x).numpy() - 1)
    assert rel.max() < 2e-6


def test_spherical_limit_is_the_closed_form_nfw():
    """q = 1: alpha and Psi of the CSE sum against nfw_sph, 0.01 <= r / r_s <= 100.  The
    convergence error of the fit (<= 2e-6 relative) bounds both."""
    ks, rs = 0.3, 12.0
    r = rs * torch.logspace(-2, 2, 57, dtype=torch.float64)
    ang = torch.linspace(0.1, 6.0, 57, dtype=torch.float64)
    dx, dy = r * torch.cos(ang), r * torch.sin(ang)
    a = pr.enfw(dx, dy, ks, 1.0, 0.4, rs, *C.table())
    b = pr.nfw_sph(dx, dy, ks, rs)
    amag = torch.hypot(b[0], b[1])
    assert float((torch.hypot(a[0] - b[0], a[1] - b[1]) / amag).max()) < 3e-6
    kb = 0.5 * (b[2] + b[3])
    for k in (2, 3, 4):
        assert float(((a[k] - b[k]).abs() / kb.abs()).max()) < 1e-5


@pytest.mark.parametrize("q", [0.55, 0.8])
def test_elliptical_deflection_matches_the_exact_elliptical_nfw(q):
    """alpha of the CSE sum against the integrals of the exact elliptical NFW density
    kappa = 2 ks g(xi / rs), at radii 0.05-20 rs: the fit error bounds the difference."""
    ks, rs = 0.25, 2.0
    g = lambda x: float(C.nfw_g(T(x))[0])
    kap = lambda xi2: 2 * ks * g(max(math.sqrt(xi2), 1e-300) / rs)
    for u, v in [(0.1, 0.05), (1.5, -0.7), (-3.0, 2.2), (0.02, 9.0), (25.0, 30.0)]:
        au, av = schramm(kap, u, v, q)
        o = pr.enfw(T(u), T(v), ks, q, 0.0, rs, *C.table())
        m = math.hypot(au, av)
        assert math.hypot(float(o[0]) - au, float(o[1]) - av) < 5e-6 * m, (u, v, float(o[0]), au)


def test_enfw_rotation_and_component_dispatch():
    """The dispatched component (kind 6: b = kappa_s, core = r_s, eps, pa) rotates the
    principal-frame result by the position angle."""
    ks, rs, eps, pa = 0.2, 3.0, 0.25, 0.6
    q = L.q_from_eps(eps)
    x, y = T(1.3, -0.4), T(0.2, 2.1)
    o = L.component(L.ENFW, x, y, ks, eps, pa, rs, 0.0)
    c, s = math.cos(pa), math.sin(pa)
    u, v = c * x + s * y, -s * x + c * y
    p = pr.enfw(u, v, ks, q, 0.0, rs, *C.table())
    assert torch.allclose(o[0], c * p[0] - s * p[1], rtol=1e-13, atol=1e-15)
    assert torch.allclose(o[1], s * p[0] + c * p[1], rtol=1e-13, atol=1e-15)
    assert torch.allclose(o[2] + o[3], p[2] + p[3], rtol=1e-13, atol=1e-15)   # trace invariant


def test_potential_gradient_is_alpha_and_vanishes_at_the_centre():
    ks, rs, eps, pa = 0.2, 3.0, 0.3, -0.4
    x, y = T(1.3, -0.4, 7.0, 0.05, 40.0), T(0.2, 2.1, -3.0, 0.02, -25.0)
    h = 1e-5      # central differences converge as h^2 (near the centre psi''' is large)
    f = lambda x, y: L.component_potential(L.ENFW, x, y, ks, eps, pa, rs, 0.0)
    gx = (f(x + h, y) - f(x - h, y)) / (2 * h)
    gy = (f(x, y + h) - f(x, y - h)) / (2 * h)
    o = L.component(L.ENFW, x, y, ks, eps, pa, rs, 0.0)
    assert torch.allclose(gx, o[0], rtol=1e-7, atol=1e-9)
    assert torch.allclose(gy, o[1], rtol=1e-7, atol=1e-9)
    assert abs(float(f(T(0.0), T(0.0)))) < 1e-12
    # the unit CSE alone, against its density: psi_uu + psi_vv = 2 kappa by differences
    q, s = 0.6, 0.05
    p = lambda u, v: pr.cse_potential_uv(u, v, q, s)
    u, v = T(0.3, -1.1, 0.02), T(0.2, 0.4, -0.03)
    hh = 1e-4
    lap = (p(u + hh, v) + p(u - hh, v) + p(u, v + hh) + p(u, v - hh) - 4 * p(u, v)) / hh ** 2
    kap = 0.5 / (s * s + u * u + v * v / (q * q)) ** 1.5
    assert torch.allclose(lap, 2 * kap, rtol=1e-5)
