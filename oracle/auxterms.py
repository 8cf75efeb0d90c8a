"""Flux and time-delay chi^2 terms in their source-plane forms (oracle, FP64).

TEST INFRASTRUCTURE ONLY.  Single lens plane.

The total chi^2 of Sec. 3 adds to the image positions the fluxes (Eq. chi2_flux) and the
time delays (Eq. chi2_td).  In the source-plane scheme both are evaluated at the observed
images only:
  * beta_i = theta_i - a alpha(theta_i), A_i = I - a Psi(theta_i), mu_i = 1 / det A_i, and
    beta_model of the family from the analytic source of Sec. 3.1 (Eq. chi2_src);
  * magnification linearised about the observed image (Sec. 3.2):
      mu_model,i = mu_i + [A_i^-1 (beta_model - beta_i)] . grad mu(theta_i),
    with grad mu by automatic differentiation of mu(theta) through the closed forms;
  * time delay linearised about (theta_i, beta_i) (Eq. td_approx, Fermat's principle makes the
    image-plane gradient vanish):
      T_model,i = K [(theta_i - beta_i)^2 / 2 - a psi(theta_i)] + K (beta_model - beta_i).(beta_i - theta_i),
    K = (1 + z_d) D_d D_s / (c D_ds) theta_0^2 = td_scale / a for the family;
  * nuisances by linear minimisation per family: m_src (Eq. msrc) and Delta t_0 (Eq. dt0);
  * chi2_flux = sum_i (m_i + 2.5 log10|mu_model,i| - m_src)^2 / sigma_m,i^2,
    chi2_td = sum_i (dt_obs,i - T_model,i - Delta t_0)^2 / sigma_t,i^2,
    over the images that carry the measurement (finite value, positive error).
"""
import math

import torch

from . import imageplane as ip
from . import lensing as L
from . import model as om


def linearised(wl, theta, tobs, sinv, fam_off, fam_adis, td_scale, create_graph=False):
    """Per image (S, N): mu at the observed image, the linearised mu_model, and the
    linearised model arrival time T_model (days).  With create_graph the results stay
    differentiable in theta (grad mu by a second autograd pass), for the gradient of the
    total chi^2; otherwise they are plain values."""
    theta = torch.as_tensor(theta, dtype=torch.float64)
    tobs = torch.as_tensor(tobs, dtype=torch.float64)
    S, N = theta.shape[0], tobs.shape[0]
    with torch.set_grad_enabled(create_graph):
        pl = om.apply_params(wl, theta)[0]
        fa = om.family_adis(wl, theta, fam_adis)
    fam = torch.empty(N, dtype=torch.long)
    for f in range(len(fam_off) - 1):
        fam[int(fam_off[f]):int(fam_off[f + 1])] = f
    a = fa[:, fam]
    tx = tobs[:, 0].expand(S, N).clone().requires_grad_(True)
    ty = tobs[:, 1].expand(S, N).clone().requires_grad_(True)
    with torch.enable_grad():
        ax, ay, pxx, pyy, pxy = L.plane_sum(pl, tx, ty)
        det = (1.0 - a * pxx) * (1.0 - a * pyy) - (a * pxy) ** 2
        mu = 1.0 / det
        gx, gy = torch.autograd.grad(mu.sum(), (tx, ty), create_graph=create_graph)
    with torch.set_grad_enabled(create_graph):
        if not create_graph:
            ax, ay, pxx, pyy, pxy, mu = [v.detach() for v in (ax, ay, pxx, pyy, pxy, mu)]
        tx, ty = tobs[:, 0].expand(S, N), tobs[:, 1].expand(S, N)
        bx, by = tx - a * ax, ty - a * ay
        beta = torch.stack([bx, by], -1)
        A = L.jac_matrix(pxx, pyy, pxy, a)
        bm = ip.source_models(beta, A, sinv, fam_off)[:, fam]          # (S, N, 2)
        dbeta = bm - beta
        dtheta = torch.linalg.solve(A, dbeta[..., None])[..., 0]      # A^-1 (beta_model - beta_i)
        mu_model = mu + dtheta[..., 0] * gx + dtheta[..., 1] * gy
        psi = L.plane_potential(pl, tx, ty)
        K = td_scale / a
        geo = 0.5 * ((tx - bx) ** 2 + (ty - by) ** 2)
        T = K * (geo - a * psi) + K * (dbeta[..., 0] * (bx - tx) + dbeta[..., 1] * (by - ty))
    return mu, mu_model, T


def _weighted(res, err, fam_off):
    """sum over images of (res - c_f)^2 / err^2 with c_f the weighted mean per family, over
    the images with a finite res and err > 0.  res: (S, N)."""
    ok = torch.isfinite(torch.as_tensor(err)) & (torch.as_tensor(err) > 0)
    S = res.shape[0]
    out = torch.zeros(S, dtype=torch.float64)
    for f in range(len(fam_off) - 1):
        i0, i1 = int(fam_off[f]), int(fam_off[f + 1])
        idx = [i for i in range(i0, i1) if bool(ok[i])]
        if not idx:
            continue
        r = res[:, idx]
        w = 1.0 / torch.as_tensor(err)[idx] ** 2
        c = (r * w).sum(1, keepdim=True) / w.sum()
        out = out + (((r - c) ** 2) * w).sum(1)
    return torch.where(torch.isfinite(out), out, torch.full_like(out, math.inf))


def chi2_flux(mu_model, mag, mag_err, fam_off):
    """Eq. chi2_flux with m_src of Eq. msrc (log is base 10: magnitudes)."""
    mag = torch.as_tensor(mag, dtype=torch.float64)
    y = mag[None] + 2.5 * torch.log10(mu_model.abs())
    err = torch.as_tensor(mag_err, dtype=torch.float64)
    err = torch.where(torch.isfinite(mag), err, torch.zeros_like(err))
    return _weighted(y, err, fam_off)


def chi2_td(T_model, td, td_err, fam_off):
    """Eq. chi2_td with Delta t_0 of Eq. dt0 per family."""
    td = torch.as_tensor(td, dtype=torch.float64)
    d = td[None] - T_model
    err = torch.as_tensor(td_err, dtype=torch.float64)
    err = torch.where(torch.isfinite(td), err, torch.zeros_like(err))
    return _weighted(d, err, fam_off)


def chi2_aux(wl, theta, tobs, sinv, fam_off, fam_adis, td_scale, mag, mag_err, td, td_err):
    """(chi2_flux, chi2_td) per sample."""
    _, mu_model, T = linearised(wl, theta, tobs, sinv, fam_off, fam_adis, td_scale)
    return chi2_flux(mu_model, mag, mag_err, fam_off), chi2_td(T, td, td_err, fam_off)


def chi2_total_and_grad(wl, theta, tobs, sinv, fam_off, fam_adis, td_scale, mag, mag_err, td, td_err):
    """The total chi^2 of Sec. 3 in its source-plane form, chi2_src + chi2_flux + chi2_td (S,),
    and its gradient in the sampled parameters (S, P) by reverse-mode autograd through exactly
    that FP64 computation (grad mu included, by a differentiable second pass)."""
    th = torch.as_tensor(theta, dtype=torch.float64).clone().detach().requires_grad_(True)
    tobs_t = torch.as_tensor(tobs, dtype=torch.float64)
    pl = om.apply_params(wl, th)[0]
    beta, A = L.single_plane_source_terms(pl, tobs_t, fam_off, om.family_adis(wl, th, fam_adis))
    c_src = L.chi2_src(beta, A, sinv, fam_off)
    _, mu_model, T = linearised(wl, th, tobs_t, sinv, fam_off, fam_adis, td_scale, create_graph=True)
    total = c_src + chi2_flux(mu_model, mag, mag_err, fam_off) + chi2_td(T, td, td_err, fam_off)
    (g,) = torch.autograd.grad(total.sum(), th)
    return total.detach(), g
