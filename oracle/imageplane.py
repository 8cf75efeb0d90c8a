"""Image-plane chi^2 (Eq. chi2_img) with model images found by Newton-Raphson from the
observed positions (oracle, FP64).  TEST INFRASTRUCTURE ONLY.

For each family the source is the analytic source-plane solution beta_model = G^-1 g
(Sec. 3.1); each model image solves beta(theta) = beta_model by Newton steps
theta <- theta - A(theta)^-1 (beta(theta) - beta_model) started at theta_obs (Sec. 3.5,
image-plane scheme); then chi^2_img = sum_i (theta_obs,i - theta_model,i)^T S_i^-1 (...)
and the image-plane rms = sqrt(mean_i |theta_obs,i - theta_model,i|^2) (Sec. 4, 5).
With several lens planes, beta(theta) and A(theta) are those of the multi-plane recursion
(Sec. 2.2) to each family's source plane; A is then not symmetric.
"""
import math

import torch

from . import cosmology as cz
from . import lensing as L
from . import model as om


def source_models(beta, A, sinv, fam_off):
    """beta_model per family (S, F, 2) from Eq. chi2_src's analytic minimiser."""
    Sinv = L.sinv_matrix(sinv)
    mu = torch.linalg.inv(A)
    M = mu.transpose(-1, -2) @ Sinv[None] @ mu
    out = []
    for f in range(len(fam_off) - 1):
        i0, i1 = int(fam_off[f]), int(fam_off[f + 1])
        G = M[:, i0:i1].sum(1)
        g = (M[:, i0:i1] @ beta[:, i0:i1, :, None]).sum(1)
        out.append(torch.linalg.solve(G, g)[..., 0])
    return torch.stack(out, 1)


def chi2_img(wl, theta, tobs, sinv, fam_off, fam_adis=None, iters=8, fam_zs=None):
    """(chi2_img (S,), rms (S,), theta_model (S, N, 2)) for sampled parameters theta (S, P).
    One plane: fam_adis (the families' a_dis).  Several planes: fam_zs (source redshifts)."""
    with torch.no_grad():
        theta = torch.as_tensor(theta)
        planes = om.apply_params(wl, theta)
        N = tobs.shape[0]
        fam = torch.empty(N, dtype=torch.long)
        for f in range(len(fam_off) - 1):
            fam[int(fam_off[f]):int(fam_off[f + 1])] = f
        if len(planes) == 1:
            pl = planes[0]
            fa = om.family_adis(wl, theta, fam_adis)                  # (S, F)
            beta, A = L.single_plane_source_terms(pl, tobs, fam_off, fa)
            a = fa[:, fam]                                            # (S, N)

            def terms(th):
                ax, ay, pxx, pyy, pxy = L.plane_sum(pl, th[..., 0], th[..., 1])
                b = torch.stack([th[..., 0] - a * ax, th[..., 1] - a * ay], -1)
                return b, L.jac_matrix(pxx, pyy, pxy, a)
        else:
            zs = [p.z for p in wl.planes]
            r, _ = cz.multiplane_ratios(zs, zs[-1] + 1.0, wl.cosmo.H0, wl.cosmo.Om)
            fam_rs = [cz.multiplane_ratios(zs, z, wl.cosmo.H0, wl.cosmo.Om)[1] for z in fam_zs]
            beta, A = L.multi_plane_source_terms(planes, r, fam_rs, tobs, fam_off)
            rs = L.image_ratios(fam_rs, fam_off, len(planes))

            def terms(th):
                return L.multi_plane_beta_A(planes, r, rs, th[..., 0], th[..., 1])
        bm = source_models(beta, A, sinv, fam_off)
        target = bm[:, fam]                                   # (S, N, 2)
        th = tobs[None].expand(beta.shape[0], N, 2).clone()
        for _ in range(iters):
            b, Aj = terms(th)
            th = th - torch.linalg.solve(Aj, (b - target)[..., None])[..., 0]
        d = tobs[None] - th
        Sm = L.sinv_matrix(sinv)
        chi2 = (d[..., None, :] @ Sm[None] @ d[..., None])[..., 0, 0].sum(1)
        rms = torch.sqrt((d * d).sum(-1).mean(1))
        chi2 = torch.where(torch.isfinite(chi2), chi2, torch.full_like(chi2, math.inf))
        return chi2, rms, th
