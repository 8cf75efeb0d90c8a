"""Flat LCDM distances (oracle).  TEST INFRASTRUCTURE ONLY.

The paper works in a flat cosmology with (H0, Om, Ow) = (70, 0.3, 0.7) and w = -1
(Sec. 1, last paragraph).  Angular-diameter distance between redshifts z1 < z2:
    D_A(z1, z2) = c/H0 / (1 + z2) * int_{z1}^{z2} dz / E(z),
    E(z) = sqrt(Om (1+z)^3 + 1 - Om).
a_dis = D_ds / D_s (Sec. 2.1, below the lensing potential).
"""
import math

from scipy.integrate import quad

C_KMS = 299792.458
ARCSEC_PER_RAD = 180.0 / math.pi * 3600.0
G_MPC_MSUN_KMS2 = 4.300917270e-9      # G in Mpc (km/s)^2 / Msun


def E(z, Om):
    return math.sqrt(Om * (1.0 + z) ** 3 + 1.0 - Om)


def comoving(z1, z2, H0=70.0, Om=0.3):
    """Line-of-sight comoving distance in Mpc."""
    val, _ = quad(lambda z: 1.0 / E(z, Om), z1, z2, epsabs=0.0, epsrel=1e-13, limit=200)
    return C_KMS / H0 * val


def d_ang(z1, z2, H0=70.0, Om=0.3):
    """Angular-diameter distance from z1 to z2 (flat universe), Mpc."""
    return comoving(z1, z2, H0, Om) / (1.0 + z2)


def a_dis(z_l, z_s, H0=70.0, Om=0.3):
    """Distance ratio D_ds / D_s."""
    if z_s <= z_l:
        return 0.0
    return d_ang(z_l, z_s, H0, Om) / d_ang(0.0, z_s, H0, Om)


def arcsec_per_kpc(z, H0=70.0, Om=0.3):
    """Angular size of 1 kpc at redshift z, in arcsec."""
    return ARCSEC_PER_RAD / (d_ang(0.0, z, H0, Om) * 1000.0)


M_PER_MPC = 3.0856775814913673e22
SECONDS_PER_DAY = 86400.0


def td_scale(z_d, H0=70.0, Om=0.3):
    """(1 + z_d) D_d theta_0^2 / c in days, theta_0 = 1 arcsec: the time-delay factor of
    Eq. time_delay at a_dis = 1 (the factor of a family is this over its a_dis, since
    D_d D_s / D_ds = D_d / a_dis)."""
    dd_m = d_ang(0.0, z_d, H0, Om) * M_PER_MPC
    theta0 = 1.0 / ARCSEC_PER_RAD
    return (1.0 + z_d) * dd_m * theta0 * theta0 / (C_KMS * 1e3) / SECONDS_PER_DAY


def rho_crit(z, H0=70.0, Om=0.3):
    """Critical density 3 H(z)^2 / (8 pi G) in Msun / Mpc^3."""
    Hz = H0 * E(z, Om)
    return 3.0 * Hz * Hz / (8.0 * math.pi * G_MPC_MSUN_KMS2)


def multiplane_ratios(zs_planes, z_s, H0=70.0, Om=0.3):
    """Ratios for the recursion of Sec. 2.2: r[i][j] = D_ij / D_j for i < j (planes),
    and the last row r_s[i] = D_is / D_s."""
    n = len(zs_planes)
    r = [[0.0] * n for _ in range(n)]
    for j in range(n):
        dj = d_ang(0.0, zs_planes[j], H0, Om)
        for i in range(j):
            r[i][j] = d_ang(zs_planes[i], zs_planes[j], H0, Om) / dj
    ds = d_ang(0.0, z_s, H0, Om)
    rs = [d_ang(zi, z_s, H0, Om) / ds if z_s > zi else 0.0 for zi in zs_planes]
    return r, rs
