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


_PHYS_FIELDS = ("vdisp", "theta_e", "z_ref", "core_kpc", "core_arcsec", "cut_kpc", "m200", "conc",
                "kappa_s", "theta_s", "gamma", "amp")


def comp_record(c: W.PhysComp, z_l, cosmo):
    """(x, y, b, eps, pa, core, cut, kind) in lensing units, converted by the library's
    lf_comp_from_physical (fields not given are passed as NaN)."""
    p = L.lf_phys_comp()
    p.kind, p.x, p.y, p.eps, p.pa_deg = c.kind, c.x, c.y, c.eps, c.pa_deg
    for f in _PHYS_FIELDS:
        v = getattr(c, f)
        setattr(p, f, math.nan if v is None else float(v))
    out = L.lf_comp()
    L.check(L.lib.lf_comp_from_physical(C.byref(p), cosmo.H0, cosmo.Om, z_l, C.byref(out)))
    return (out.x, out.y, out.b, out.eps, out.pa, out.core, out.cut, out.kind)


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
        sc = L.lf_scaling()
        L.check(L.lib.lf_scaling_from_physical(m.vstar, m.core_star_kpc, m.cut_star_kpc, m.lam, m.beta,
                                               m.alpha, cosmo.H0, cosmo.Om, pl.z, C.byref(sc)))
        scaling = (sc.b_star, sc.core_star, sc.cut_star, sc.lam, sc.beta, sc.alpha)
    else:
        mem = np.zeros(0, dtype=MEM_DTYPE)
        scaling = (0.0, 0.0, 1.0, 0.0, 0.0, 0.0)
    return DevicePlane(pl.z, comp, mem, scaling).to(device)


def device_planes(wl: W.Workload, device="cuda") -> List[DevicePlane]:
    return [device_plane(p, wl.cosmo, device) for p in wl.planes]


def grid_struct(g: W.Grid) -> L.lf_grid:
    return L.lf_grid(g.x0, g.y0, g.dx, g.dy, g.nx, g.ny)


def multiplane_ratios(cosmo, zs_planes, z_s):
    """(n+1) x n table (lf_multiplane_ratios): r[i][j] = D_ij/D_j for i < j, last row D_js/D_s."""
    n = len(zs_planes)
    r = np.zeros((n + 1, n))
    z = np.ascontiguousarray(zs_planes, dtype=np.float64)
    L.check(L.lib.lf_multiplane_ratios(cosmo.H0, cosmo.Om, z.ctypes.data_as(C.c_void_p), n, float(z_s),
                                       r.ctypes.data_as(C.c_void_p)))
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
