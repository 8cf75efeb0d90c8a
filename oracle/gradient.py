"""Batched source-plane chi^2 and its parameter gradient (oracle, FP64).

TEST INFRASTRUCTURE ONLY.  chi^2 per sample follows Eq. chi2_src with the analytic
source of Sec. 3.1 after writing each sample's parameters into the model (Eq. scaling
for the members).  The gradient d chi^2 / d theta is PyTorch reverse-mode autograd
through exactly that FP64 computation: a library primitive, independent of any
hand-derived adjoint.
"""
import torch

from . import cosmology as cz
from . import lensing as L
from . import model as om


def _terms(wl, theta, tobs, fam_off, fam_adis=None, fam_zs=None):
    planes = om.apply_params(wl, theta)
    if len(planes) == 1:
        return L.single_plane_source_terms(planes[0], tobs, fam_off, om.family_adis(wl, theta, fam_adis))
    zs = [p.z for p in wl.planes]
    r, _ = cz.multiplane_ratios(zs, zs[-1] + 1.0, wl.cosmo.H0, wl.cosmo.Om)
    fam_rs = [cz.multiplane_ratios(zs, z, wl.cosmo.H0, wl.cosmo.Om)[1] for z in fam_zs]
    return L.multi_plane_source_terms(planes, r, fam_rs, tobs, fam_off)


def chi2_only(wl, theta, tobs, sinv, fam_off, fam_adis=None, fam_zs=None):
    with torch.no_grad():
        beta, A = _terms(wl, theta, tobs, fam_off, fam_adis, fam_zs)
        return L.chi2_src(beta, A, sinv, fam_off)


def chi2_and_grad(wl, theta, tobs, sinv, fam_off, fam_adis=None, fam_zs=None):
    th = theta.clone().detach().requires_grad_(True)
    beta, A = _terms(wl, th, tobs, fam_off, fam_adis, fam_zs)
    chi2 = L.chi2_src(beta, A, sinv, fam_off)
    (g,) = torch.autograd.grad(chi2.sum(), th)
    return chi2.detach(), g
