"""Host-side set-up: physical model descriptions -> lensing-unit component tables in
device memory (the lf_plane of the C ABI).  Unit conversions call the library's host
helpers (distances, velocity dispersion -> strength, NFW normalisation).
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import torch

from . import _lib as L
from . import workloads as W

COMP_DTYPE = np.dtype([("x", "<f8"), ("y", "<f8"), ("b", "<f8"), ("eps", "<f8"), ("pa", "<f8"),
                       ("core", "<f8"), ("cut", "<f8"), ("kind", "<i4"), ("pad", "<i4")])
MEM_DTYPE = np.dtype([("x", "<f8"), ("y", "<f8"), ("log_l", "<f8"), ("pad", "<f8")])
assert COMP_DTYPE.itemsize == 64 and MEM_DTYPE.itemsize == 32


def adis(cosmo, z_l, z_s):
    return L.lib.lf_adis(cosmo.H0, cosmo.Om, z_l, z_s)


def td_scale(cosmo, z_d):
    """(1 + z_d) D_d theta_0^2 / c in days (the library's cosmology)."""
    return L.lib.lf_td_scale(cosmo.H0, cosmo.Om, z_d)


def arcsec_per_kpc(cosmo, z):
    return L.lib.lf_arcsec_per_kpc(cosmo.H0, cosmo.Om, z)


def b_from_vdisp(v):
    return L.lib.lf_b_from_vdisp(v)


def nfw_params(cosmo, z_l, m200, conc):
    ks, ts = C.c_double(), C.c_double()
    L.check(L.lib.lf_nfw_params(cosmo.H0, cosmo.Om, z_l, m200, conc, C.byref(ks), C.byref(ts)))
    return ks.value, ts.value


def comp_record(c: W.PhysComp, z_l, cosmo):
    """(x, y, b, eps, pa, core, cut, kind) in lensing units."""
    pa = math.radians(c.pa_deg)
    if c.kind in (W.SIE, W.DPIE):
        q = (1 - c.eps) / (1 + c.eps)
        if c.vdisp is not None:
            b = b_from_vdisp(c.vdisp)
        else:   # area-equivalent Einstein radius at z_ref: theta_E = a b sqrt(q)
            b = c.theta_e / (math.sqrt(q) * adis(cosmo, z_l, c.z_ref))
        apk = arcsec_per_kpc(cosmo, z_l)
        core = c.core_arcsec if c.core_arcsec is not None else c.core_kpc * apk
        cut = c.cut_kpc * apk if c.cut_kpc is not None else 0.0
        return (c.x, c.y, b, c.eps, pa, core, cut, c.kind)
    if c.kind == W.NFW:
        ks, ts = nfw_params(cosmo, z_l, c.m200, c.conc)
        return (c.x, c.y, ks, 0.0, 0.0, ts, 0.0, c.kind)
    if c.kind == W.ENFW:   # spherical NFW normalisation, ellipticity applied to xi
        ks, ts = (c.kappa_s, c.theta_s) if c.kappa_s is not None else nfw_params(cosmo, z_l, c.m200, c.conc)
        return (c.x, c.y, ks, c.eps, pa, ts, 0.0, c.kind)
    if c.kind == W.SHEAR:
        g = c.gamma if c.z_ref is None else c.gamma / adis(cosmo, z_l, c.z_ref)
        return (c.x, c.y, g, 0.0, pa, 0.0, 0.0, c.kind)
    if c.kind == W.MPOLE3:
        return (c.x, c.y, c.amp, 0.0, pa, 0.0, 0.0, c.kind)
    raise ValueError(c.kind)


@dataclass
class DevicePlane:
    """A lens plane whose tables live in device memory (kept alive by this object)."""
    z: float
    comp_host: np.ndarray
    mem_host: np.ndarray
    scaling: tuple
    comp_dev: Optional[torch.Tensor] = None
    mem_dev: Optional[torch.Tensor] = None

    def to(self, device):
        if len(self.comp_host):
            self.comp_dev = torch.from_numpy(self.comp_host.view(np.uint8).copy()).to(device)
        if len(self.mem_host):
            self.mem_dev = torch.from_numpy(self.mem_host.view(np.uint8).copy()).to(device)
        return self

    def c_struct(self) -> L.lf_plane:
        p = L.lf_plane()
        p.n_comp = len(self.comp_host)
        p.n_mem = len(self.mem_host)
        p.comp = self.comp_dev.data_ptr() if self.comp_dev is not None else None
        p.mem = self.mem_dev.data_ptr() if self.mem_dev is not None else None
        p.scaling = L.lf_scaling(*self.scaling)
        return p


def device_plane(pl: W.PhysPlane, cosmo, device="cuda") -> DevicePlane:
    recs = [comp_record(c, pl.z, cosmo) for c in pl.comps]
    comp = np.zeros(len(recs), dtype=COMP_DTYPE)
    for i, r in enumerate(recs):
        comp[i] = r + (0,)
    if pl.members is not None:
        m = pl.members
        mem = np.zeros(len(m.x), dtype=MEM_DTYPE)
        mem["x"], mem["y"], mem["log_l"] = m.x, m.y, m.log_l
        apk = arcsec_per_kpc(cosmo, pl.z)
        scaling = (b_from_vdisp(m.vstar), m.core_star_kpc * apk, m.cut_star_kpc * apk,
                   m.lam, m.beta, m.alpha)
    else:
        mem = np.zeros(0, dtype=MEM_DTYPE)
        scaling = (0.0, 0.0, 1.0, 0.0, 0.0, 0.0)
    return DevicePlane(pl.z, comp, mem, scaling).to(device)


def device_planes(wl: W.Workload, device="cuda") -> List[DevicePlane]:
    return [device_plane(p, wl.cosmo, device) for p in wl.planes]


def grid_struct(g: W.Grid) -> L.lf_grid:
    return L.lf_grid(g.x0, g.y0, g.dx, g.dy, g.nx, g.ny)


def multiplane_ratios(cosmo, zs_planes, z_s):
    """(n+1) x n table: r[i][j] = D_ij/D_j for i < j, last row D_js/D_s."""
    n = len(zs_planes)
    r = np.zeros((n + 1, n))
    for j in range(n):
        dj = L.lib.lf_angular_distance(cosmo.H0, cosmo.Om, 0.0, zs_planes[j])
        for i in range(j):
            r[i, j] = L.lib.lf_angular_distance(cosmo.H0, cosmo.Om, zs_planes[i], zs_planes[j]) / dj
    ds = L.lib.lf_angular_distance(cosmo.H0, cosmo.Om, 0.0, z_s)
    for j in range(n):
        r[n, j] = (L.lib.lf_angular_distance(cosmo.H0, cosmo.Om, zs_planes[j], z_s) / ds
                   if z_s > zs_planes[j] else 0.0)
    return r


def cluster_input(wl: W.Workload, cat: W.Catalogue, sigma_pos=None, device="cuda", aux=None):
    """ClusterInput for a workload and its image catalogue: circular S_i = sigma^2 I
    (Eq. chi2_img with sigma_1 = sigma_2), per-family distance ratios from the library's
    cosmology, and the parameter map of the workload."""
    from .api import ClusterInput
    planes = device_planes(wl, device)
    sig = wl.sigma_pos if sigma_pos is None else sigma_pos
    n = len(cat.theta_obs)
    sinv = np.tile([1.0 / sig ** 2, 0.0, 1.0 / sig ** 2], (n, 1))
    zl = [p.z for p in wl.planes]
    apk = [arcsec_per_kpc(wl.cosmo, z) for z in zl]
    if len(planes) == 1:
        fam_ratio = np.array([adis(wl.cosmo, zl[0], z) for z in cat.fam_zs])
        ratios = None
    else:
        fam_ratio = np.array([multiplane_ratios(wl.cosmo, zl, z)[-1] for z in cat.fam_zs])
        ratios = multiplane_ratios(wl.cosmo, zl, max(zl) + 1.0)[:-1]
    p_comp = [p.comp for p in wl.params]
    p_field = [p.field for p in wl.params]
    p_xform = [p.xform for p in wl.params]
    ts = td_scale(wl.cosmo, zl[0]) if aux is not None else 0.0
    return ClusterInput(planes, apk, cat.theta_obs, sinv, cat.fam_off, fam_ratio, p_comp, p_field,
                        p_xform, ratios, aux=aux, td_scale=ts)
