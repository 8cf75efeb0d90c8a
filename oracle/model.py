"""Physical workload description -> oracle lensing units.  TEST INFRASTRUCTURE ONLY.

Conversions (each side of the parity check has its own):
* isothermal strength from a velocity dispersion, b = 4 pi (v/c)^2 (a_dis = 1);
* an area-equivalent Einstein radius theta_E quoted at source redshift z_ref:
  the tangential critical curve of an isothermal ellipsoid is the kappa = 1/2 contour
  of a_dis kappa, an ellipse of semi-axes a b and q a b, so theta_E = a b sqrt(q);
* kpc -> arcsec at the plane's redshift;
* spherical NFW (M200, c) -> (kappa_s, theta_s) with 200 x the critical density at
  z_l and Sigma_cr at a_dis = 1, c^2 / (4 pi G D_d);
* an external shear quoted at z_ref is divided by a_dis(z_l, z_ref) (paper convention,
  the potential carries no a_dis);
* sampled parameters: km/s -> b, degrees -> radians, kpc -> arcsec.
"""
import math

import numpy as np
import torch

from . import cosmology as cz
from .lensing import LPlane, b_from_vdisp, q_from_eps

SIE, DPIE, NFW, SHEAR, MPOLE3, ENFW = 1, 2, 3, 4, 5, 6
XF_IDENT, XF_VDISP, XF_DEG, XF_KPC = 0, 1, 2, 3
FIELDS = ("x", "y", "b", "eps", "pa", "core", "cut")
SCALING = ("b_star", "core_star", "cut_star", "lam", "beta", "alpha")


def nfw_lensing(m200, conc, z_l, H0=70.0, Om=0.3):
    rc = cz.rho_crit(z_l, H0, Om)
    r200 = (3.0 * m200 / (4.0 * math.pi * 200.0 * rc)) ** (1.0 / 3.0)       # Mpc
    rs = r200 / conc
    delta_c = 200.0 / 3.0 * conc ** 3 / (math.log(1.0 + conc) - conc / (1.0 + conc))
    dd = cz.d_ang(0.0, z_l, H0, Om)
    sigma_cr = cz.C_KMS ** 2 / (4.0 * math.pi * cz.G_MPC_MSUN_KMS2 * dd)    # Msun / Mpc^2
    ks = delta_c * rc * rs / sigma_cr
    theta_s = rs / dd * cz.ARCSEC_PER_RAD
    return ks, theta_s


def comp_fields(c, z_l, cosmo):
    """Lensing-unit fields (x, y, b, eps, pa, core, cut) of one physical component."""
    H0, Om = cosmo.H0, cosmo.Om
    apk = cz.arcsec_per_kpc(z_l, H0, Om)
    pa = math.radians(c.pa_deg)
    if c.kind in (SIE, DPIE):
        q = q_from_eps(c.eps)
        if c.vdisp is not None:
            b = b_from_vdisp(c.vdisp)
        else:
            b = c.theta_e / (math.sqrt(q) * cz.a_dis(z_l, c.z_ref, H0, Om))
        core = c.core_arcsec if c.core_arcsec is not None else c.core_kpc * apk
        cut = c.cut_kpc * apk if c.cut_kpc is not None else 0.0
        return [c.x, c.y, b, c.eps, pa, core, cut]
    if c.kind == NFW:
        ks, ts = nfw_lensing(c.m200, c.conc, z_l, H0, Om)
        return [c.x, c.y, ks, 0.0, 0.0, ts, 0.0]
    if c.kind == ENFW:   # the spherical normalisation, with the ellipticity on xi
        ks, ts = (c.kappa_s, c.theta_s) if c.kappa_s is not None else nfw_lensing(c.m200, c.conc, z_l, H0, Om)
        return [c.x, c.y, ks, c.eps, pa, ts, 0.0]
    if c.kind == SHEAR:
        g = c.gamma
        if c.z_ref is not None:
            g = g / cz.a_dis(z_l, c.z_ref, H0, Om)
        return [c.x, c.y, g, 0.0, pa, 0.0, 0.0]
    if c.kind == MPOLE3:
        return [c.x, c.y, c.amp, 0.0, pa, 0.0, 0.0]
    raise ValueError(c.kind)


def build_planes(wl, S=1):
    """LPlane list (sample axis of length S, all samples equal) for a workload."""
    out = []
    for pl in wl.planes:
        fields = np.array([comp_fields(c, pl.z, wl.cosmo) for c in pl.comps], dtype=np.float64)
        if fields.size == 0:
            fields = np.zeros((0, 7))
        t = lambda j: torch.tensor(fields[:, j], dtype=torch.float64)[None, :].repeat(S, 1)
        lp = LPlane([c.kind for c in pl.comps], t(0), t(1), t(2), t(3), t(4), t(5), t(6))
        if pl.members is not None:
            m = pl.members
            apk = cz.arcsec_per_kpc(pl.z, wl.cosmo.H0, wl.cosmo.Om)
            full = lambda v: torch.full((S,), float(v), dtype=torch.float64)
            lp.mx = torch.tensor(m.x, dtype=torch.float64)
            lp.my = torch.tensor(m.y, dtype=torch.float64)
            lp.log_l = torch.tensor(m.log_l, dtype=torch.float64)
            lp.b_star = full(b_from_vdisp(m.vstar))
            lp.core_star = full(m.core_star_kpc * apk)
            lp.cut_star = full(m.cut_star_kpc * apk)
            lp.lam, lp.beta, lp.alpha = full(m.lam), full(m.beta), full(m.alpha)
        out.append(lp)
    return out


def transform(xform, v, apk):
    if xform == XF_IDENT:
        return v
    if xform == XF_VDISP:
        return 4.0 * math.pi * (v / cz.C_KMS) ** 2 * cz.ARCSEC_PER_RAD
    if xform == XF_DEG:
        return v * (math.pi / 180.0)
    if xform == XF_KPC:
        return v * apk
    raise ValueError(xform)


def apply_params(wl, theta):
    """Planes with the sampled parameters (S, P) written into their targets (the A1
    component-preparation step).  `theta` may require grad; the result is
    differentiable with respect to it."""
    S = theta.shape[0]
    planes = build_planes(wl, S)
    offs = np.cumsum([0] + [len(p.comps) for p in wl.planes])
    for p, spec in enumerate(wl.params):
        if spec.comp >= 0:
            j = int(np.searchsorted(offs, spec.comp, side="right") - 1)
            k = spec.comp - offs[j]
            apk = cz.arcsec_per_kpc(wl.planes[j].z, wl.cosmo.H0, wl.cosmo.Om)
            pl = planes[j]
            name = FIELDS[spec.field]
            col = getattr(pl, name).clone()
            col[:, k] = transform(spec.xform, theta[:, p], apk)
            setattr(pl, name, col)
        elif spec.comp == -2:
            continue   # a family's distance ratio: see family_adis
        else:
            # scaling slots live on the first plane that has members
            j = next(i for i, pp in enumerate(wl.planes) if pp.members is not None)
            apk = cz.arcsec_per_kpc(wl.planes[j].z, wl.cosmo.H0, wl.cosmo.Om)
            setattr(planes[j], SCALING[spec.field], transform(spec.xform, theta[:, p], apk))
    return planes


def family_adis(wl, theta, base_adis):
    """(S, F) distance ratios a_dis of the families for each sample: the fixed values
    `base_adis`, except the families whose a_dis is itself a sampled parameter (comp = -2,
    field = family index; sampled directly in a_dis, Sec. 3.5).  Differentiable in theta."""
    S = theta.shape[0]
    cols = [torch.full((S,), float(a), dtype=torch.float64) for a in base_adis]
    for p, spec in enumerate(wl.params):
        if spec.comp == -2:
            cols[spec.field] = theta[:, p]
    return torch.stack(cols, 1)


def single_plane_adis(wl, family_zs):
    z_l = wl.planes[0].z
    return [cz.a_dis(z_l, z, wl.cosmo.H0, wl.cosmo.Om) for z in family_zs]
