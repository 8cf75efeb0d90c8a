"""Pins of the oracle's lens potentials: grad psi = alpha by central differences of psi for
every profile (each is defined only up to a constant), and the time-delay scale against the
Einstein-de Sitter closed form of the distance."""
import math

import numpy as np
import torch

from oracle import cosmology as cz
from oracle import profiles as pr

torch.set_default_dtype(torch.float64)
RNG = np.random.default_rng(8)
X = torch.tensor(RNG.uniform(-30, 30, 200))
Y = torch.tensor(RNG.uniform(-30, 30, 200))


def check(pot, alpha, h=1e-5, rtol=1e-6, atol=1e-8):
    ax, ay = alpha(X, Y)[:2]
    fx = (pot(X + h, Y) - pot(X - h, Y)) / (2 * h)
    fy = (pot(X, Y + h) - pot(X, Y - h)) / (2 * h)
    assert torch.allclose(fx, ax, rtol=rtol, atol=atol), (fx - ax).abs().max()
    assert torch.allclose(fy, ay, rtol=rtol, atol=atol), (fy - ay).abs().max()


def test_sie_potential():
    for q, s in ((0.7, 0.5), (0.45, 2.0), (0.999, 0.1)):
        check(lambda x, y: pr.sie_potential(x, y, 20.0, q, 0.6, s),
              lambda x, y: pr.sie(x, y, 20.0, q, 0.6, s))


def test_dpie_and_round_pje_potentials():
    check(lambda x, y: pr.dpie_potential(x, y, 15.0, 0.6, -0.4, 1.0, 80.0),
          lambda x, y: pr.dpie(x, y, 15.0, 0.6, -0.4, 1.0, 80.0))
    check(lambda x, y: pr.pje_sph_potential(x, y, 0.8, 0.05, 7.0),
          lambda x, y: pr.pje_sph(x, y, 0.8, 0.05, 7.0))


def test_nfw_potential_both_branches():
    check(lambda x, y: pr.nfw_potential(x, y, 0.3, 12.0), lambda x, y: pr.nfw_sph(x, y, 0.3, 12.0))
    check(lambda x, y: pr.nfw_potential(x, y, 0.3, 60.0), lambda x, y: pr.nfw_sph(x, y, 0.3, 60.0))


def test_shear_and_multipole_potentials():
    check(lambda x, y: pr.shear_potential(x, y, 0.07, 0.3), lambda x, y: pr.shear(x, y, 0.07, 0.3))
    check(lambda x, y: pr.multipole3_potential(x, y, 0.004, 0.3),
          lambda x, y: pr.multipole3(x, y, 0.004, 0.3))


def test_td_scale_einstein_de_sitter():
    """Om = 1: D_d = (2c/H0) (1 - (1+z)^-1/2) / (1+z)."""
    z, H0 = 0.5, 70.0
    dd = 2 * cz.C_KMS / H0 * (1 - (1 + z) ** -0.5) / (1 + z)
    ref = (1 + z) * dd * cz.M_PER_MPC / (cz.C_KMS * 1e3) * (math.pi / 180 / 3600) ** 2 / 86400
    assert abs(cz.td_scale(z, H0, 1.0) / ref - 1) < 1e-12
