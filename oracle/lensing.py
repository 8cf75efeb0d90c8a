"""Lens map, Jacobian, magnification, multi-plane recursion and source-plane chi^2
(oracle, FP64).  TEST INFRASTRUCTURE ONLY.

All tensors are float64 on the CPU.  A plane is an `LPlane` in lensing units
(strengths at a_dis = 1, arcsec, radians) whose component fields carry a leading
sample axis S (S = 1 for a single model).  Positions have shape (S or 1, N).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional

import torch

from . import profiles as pr
from . import cse_nfw

SIE, DPIE, NFW, SHEAR, MPOLE3, ENFW = 1, 2, 3, 4, 5, 6
SHEET = 101   # oracle-only test profile: a uniform mass sheet of convergence b
C_KMS = 299792.458
ARCSEC_PER_RAD = 180.0 / math.pi * 3600.0


@dataclass
class LPlane:
    kind: List[int]                    # K component kinds
    x: torch.Tensor                    # (S, K) each
    y: torch.Tensor
    b: torch.Tensor
    eps: torch.Tensor
    pa: torch.Tensor
    core: torch.Tensor
    cut: torch.Tensor
    mx: Optional[torch.Tensor] = None  # (M,) member geometry
    my: Optional[torch.Tensor] = None
    log_l: Optional[torch.Tensor] = None
    b_star: Optional[torch.Tensor] = None   # (S,) scaling relation, lensing units
    core_star: Optional[torch.Tensor] = None
    cut_star: Optional[torch.Tensor] = None
    lam: Optional[torch.Tensor] = None
    beta: Optional[torch.Tensor] = None
    alpha: Optional[torch.Tensor] = None

    @property
    def n_members(self):
        return 0 if self.mx is None else int(self.mx.numel())


def b_from_vdisp(v_kms):
    """Isothermal strength at a_dis = 1: b = 4 pi (v/c)^2, in arcsec."""
    return 4.0 * math.pi * (v_kms / C_KMS) ** 2 * ARCSEC_PER_RAD


def q_from_eps(eps):
    """eps = (1 - q)/(1 + q)  =>  q = (1 - eps)/(1 + eps) (Sec. 2.1)."""
    return (1.0 - eps) / (1.0 + eps)


def member_fields(pl: LPlane):
    """Eq. scaling: v = v* (L/L*)^lam, core = core* (L/L*)^beta, cut = cut* (L/L*)^alpha;
    b scales as v^2, so b_m = b* (L/L*)^(2 lam).  Returns (S, M) tensors."""
    ll = pl.log_l[None, :] * math.log(10.0)
    b = pl.b_star[:, None] * torch.exp(2.0 * pl.lam[:, None] * ll)
    core = pl.core_star[:, None] * torch.exp(pl.beta[:, None] * ll)
    cut = pl.cut_star[:, None] * torch.exp(pl.alpha[:, None] * ll)
    return b, core, cut


def component(kind, dx, dy, b, eps, pa, core, cut):
    if kind == SIE:
        return pr.sie(dx, dy, b, q_from_eps(eps), pa, core)
    if kind == DPIE:
        return pr.dpie(dx, dy, b, q_from_eps(eps), pa, core, cut)
    if kind == NFW:
        return pr.nfw_sph(dx, dy, b, core)
    if kind == SHEAR:
        return pr.shear(dx, dy, b, pa)
    if kind == MPOLE3:
        return pr.multipole3(dx, dy, b, pa)
    if kind == ENFW:     # b = kappa_s, core = r_s
        return pr.enfw(dx, dy, b, q_from_eps(eps), pa, core, *cse_nfw.table())
    if kind == SHEET:
        return pr.mass_sheet(dx, dy, b)
    raise ValueError(f"unknown component kind {kind}")


def component_potential(kind, dx, dy, b, eps, pa, core, cut):
    if kind == SIE:
        return pr.sie_potential(dx, dy, b, q_from_eps(eps), pa, core)
    if kind == DPIE:
        return pr.dpie_potential(dx, dy, b, q_from_eps(eps), pa, core, cut)
    if kind == NFW:
        return pr.nfw_potential(dx, dy, b, core)
    if kind == SHEAR:
        return pr.shear_potential(dx, dy, b, pa)
    if kind == MPOLE3:
        return pr.multipole3_potential(dx, dy, b, pa)
    if kind == ENFW:
        return pr.enfw_potential(dx, dy, b, q_from_eps(eps), pa, core, *cse_nfw.table())
    if kind == SHEET:
        return pr.mass_sheet_potential(dx, dy, b)
    raise ValueError(f"unknown component kind {kind}")


def plane_potential(pl: LPlane, tx, ty):
    """psi (up to a constant per component) summed over the plane's components and members,
    (S, N) for positions (1, N) or (S, N)."""
    out = torch.zeros(torch.broadcast_shapes(tx.shape, (pl.x.shape[0], 1)), dtype=torch.float64)
    for k, kind in enumerate(pl.kind):
        col = lambda f: f[:, k:k + 1]
        out = out + component_potential(kind, tx - col(pl.x), ty - col(pl.y), col(pl.b), col(pl.eps),
                                         col(pl.pa), col(pl.core), col(pl.cut))
    if pl.n_members:
        bm, cm, tm = member_fields(pl)
        for m in range(pl.n_members):
            out = out + pr.pje_sph_potential(tx - pl.mx[m], ty - pl.my[m], bm[:, m:m + 1],
                                             cm[:, m:m + 1], tm[:, m:m + 1])
    return out


def plane_sum(pl: LPlane, tx, ty):
    """alpha and psi_ij summed over every component and member of one plane
    (Sec. 2.1: the potential of a composite lens is the sum of its parts).
    Returns five tensors of shape broadcast(S, N)."""
    S = pl.x.shape[0]
    shape = torch.broadcast_shapes((S, 1), tx.shape)
    acc = [torch.zeros(shape, dtype=torch.float64) for _ in range(5)]
    for k, kind in enumerate(pl.kind):
        col = lambda f: f[:, k:k + 1]
        out = component(kind, tx - col(pl.x), ty - col(pl.y), col(pl.b), col(pl.eps),
                        col(pl.pa), col(pl.core), col(pl.cut))
        acc = [a + o for a, o in zip(acc, out)]
    if pl.n_members:
        bm, cm, tm = member_fields(pl)
        for m in range(pl.n_members):
            out = pr.pje_sph(tx - pl.mx[m], ty - pl.my[m], bm[:, m:m + 1], cm[:, m:m + 1],
                             tm[:, m:m + 1])
            acc = [a + o for a, o in zip(acc, out)]
    return tuple(acc)


def jacobian_maps(ax, ay, pxx, pyy, pxy, a_dis):
    """kappa, gamma1, gamma2 from psi_ij (Sec. 2.1; a_dis-free, as in the paper), and
    mu = 1/det A with det A = (1 - a kappa)^2 - a^2 |gamma|^2 (Eq. jac and the
    eigenvalue form of mu)."""
    kappa = 0.5 * (pxx + pyy)
    g1 = 0.5 * (pxx - pyy)
    g2 = pxy
    det = (1.0 - a_dis * kappa) ** 2 - a_dis * a_dis * (g1 * g1 + g2 * g2)
    return kappa, g1, g2, 1.0 / det, det


def lens_map(tx, ty, ax, ay, a_dis):
    """Eq. lens_eq: beta = theta - a_dis alpha(theta)."""
    return tx - a_dis * ax, ty - a_dis * ay


def jac_matrix(pxx, pyy, pxy, a_dis):
    """Eq. jac: A_ij = delta_ij - a_dis psi_ij, returned as (..., 2, 2)."""
    a11 = 1.0 - a_dis * pxx
    a22 = 1.0 - a_dis * pyy
    a12 = -a_dis * pxy
    return torch.stack([torch.stack([a11, a12], -1), torch.stack([a12, a22], -1)], -2)


def trace_multiplane(planes: List[LPlane], r, rs, tx, ty):
    """Sec. 2.2 recursion.  theta_j = theta_1 - sum_{i<j} (D_ij/D_j) alpha_i(theta_i);
    beta = theta_1 - sum_j (D_js/D_s) alpha_j(theta_j).  The Jacobian follows by the
    chain rule: A_j = I - sum_{i<j} (D_ij/D_j) Psi_i(theta_i) A_i, A = I - sum_j
    (D_js/D_s) Psi_j A_j (not symmetric in general).  r[i][j] = D_ij/D_j, rs[j] = D_js/D_s.
    Returns beta (..., 2) and A (..., 2, 2)."""
    t1, alphas, psis, As = multiplane_parts(planes, r, tx, ty)
    beta = t1.clone()
    A = torch.eye(2, dtype=torch.float64).expand_as(As[0]).clone()
    for j in range(len(planes)):
        beta = beta - rs[j] * alphas[j]
        A = A - rs[j] * (psis[j] @ As[j])
    return beta, A


def multiplane_parts(planes: List[LPlane], r, tx, ty):
    """The source-independent part of the recursion: per plane theta_j, alpha_j, Psi_j, A_j."""
    S = planes[0].x.shape[0]
    shape = torch.broadcast_shapes((S, 1), tx.shape)
    t1 = torch.stack([tx.expand(shape), ty.expand(shape)], -1)
    eye = torch.eye(2, dtype=torch.float64).expand(*shape, 2, 2)
    alphas, psis, As = [], [], []
    for j, pl in enumerate(planes):
        tj = t1.clone()
        Aj = eye.clone()
        for i in range(j):
            tj = tj - r[i][j] * alphas[i]
            Aj = Aj - r[i][j] * (psis[i] @ As[i])
        ax, ay, pxx, pyy, pxy = plane_sum(pl, tj[..., 0], tj[..., 1])
        alphas.append(torch.stack([ax, ay], -1))
        psis.append(torch.stack([torch.stack([pxx, pxy], -1), torch.stack([pxy, pyy], -1)], -2))
        As.append(Aj)
    return t1, alphas, psis, As


def sinv_matrix(sinv):
    """(N, 3) [S^-1_xx, S^-1_xy, S^-1_yy] -> (N, 2, 2)."""
    return torch.stack([torch.stack([sinv[:, 0], sinv[:, 1]], -1),
                        torch.stack([sinv[:, 1], sinv[:, 2]], -1)], -2)


def covariance_inverse(sig1, sig2, phi):
    """S_i = R^T diag(sig1^2, sig2^2) R with R = [[cos, sin], [-sin, cos]] (Eq. chi2_img
    and below); returns S_i^-1 as [xx, xy, yy]."""
    c, s = math.cos(phi), math.sin(phi)
    R = torch.tensor([[c, s], [-s, c]], dtype=torch.float64)
    Sm = R.T @ torch.diag(torch.tensor([sig1 ** 2, sig2 ** 2], dtype=torch.float64)) @ R
    Si = torch.linalg.inv(Sm)
    return [float(Si[0, 0]), float(Si[0, 1]), float(Si[1, 1])]


def chi2_src(beta, A, sinv, fam_off):
    """Eq. chi2_src with the analytic source of Sec. 3.1.

    beta: (S, N, 2) source positions of the observed images; A: (S, N, 2, 2) Jacobians;
    sinv: (N, 3); fam_off: CSR offsets (F + 1).  For each family:
      mu_i = A_i^-1, M_i = mu_i^T S_i^-1 mu_i, G = sum M_i, g = sum M_i beta_i,
      beta_model = G^-1 g, chi^2 = sum (beta_i - beta_model)^T M_i (beta_i - beta_model).
    A sample with a non-finite value anywhere in a family gets chi^2 = +inf.
    Returns (S,) chi^2."""
    Sinv = sinv_matrix(sinv)
    mu = torch.linalg.inv(A)
    M = mu.transpose(-1, -2) @ Sinv[None] @ mu
    S = beta.shape[0]
    chi2 = torch.zeros(S, dtype=torch.float64)
    for f in range(len(fam_off) - 1):
        i0, i1 = int(fam_off[f]), int(fam_off[f + 1])
        Mf = M[:, i0:i1]
        bf = beta[:, i0:i1]
        G = Mf.sum(1)
        g = (Mf @ bf[..., None]).sum(1)
        bm = torch.linalg.solve(G, g)                              # (S, 2, 1)
        d = bf[..., None] - bm[:, None]
        chi2 = chi2 + (d.transpose(-1, -2) @ Mf @ d)[..., 0, 0].sum(1)
    return torch.where(torch.isfinite(chi2), chi2, torch.full_like(chi2, math.inf))


def single_plane_source_terms(pl: LPlane, theta_obs, fam_off, fam_adis):
    """beta_i = theta_i - a_f alpha(theta_i), A_i = I - a_f Psi(theta_i) for every
    observed image i of family f (Eq. lens_eq, Eq. jac).  fam_adis: one a_dis per family,
    or an (S, F) tensor of per-sample values."""
    N = theta_obs.shape[0]
    fam = torch.empty(N, dtype=torch.long)
    for f in range(len(fam_off) - 1):
        fam[int(fam_off[f]):int(fam_off[f + 1])] = f
    if torch.is_tensor(fam_adis) and fam_adis.dim() == 2:
        a = fam_adis[:, fam]
    else:
        a = torch.tensor([float(v) for v in fam_adis], dtype=torch.float64)[fam]
    tx, ty = theta_obs[None, :, 0], theta_obs[None, :, 1]
    ax, ay, pxx, pyy, pxy = plane_sum(pl, tx, ty)
    bx, by = tx - a * ax, ty - a * ay
    beta = torch.stack([bx, by], -1)
    A = jac_matrix(pxx, pyy, pxy, a)
    return beta, A


def image_ratios(fam_rs, fam_off, n_planes):
    """(n_planes, N) ratios D_js/D_s of each image's family."""
    N = int(fam_off[-1])
    rs = torch.zeros(n_planes, N, dtype=torch.float64)
    for f in range(len(fam_off) - 1):
        for j in range(n_planes):
            rs[j, int(fam_off[f]):int(fam_off[f + 1])] = float(fam_rs[f][j])
    return rs


def multi_plane_source_terms(planes, r, fam_rs, theta_obs, fam_off):
    """Per image, beta and A traced through all planes to its family's source
    (fam_rs[f][j] = D_js/D_s for that family's redshift)."""
    rs = image_ratios(fam_rs, fam_off, len(planes))
    return multi_plane_beta_A(planes, r, rs, theta_obs[None, :, 0], theta_obs[None, :, 1])


def multi_plane_beta_A(planes, r, rs, tx, ty):
    """beta (S, N, 2) and A (S, N, 2, 2) of the recursion at positions (tx, ty) of shape
    (S or 1, N), each position traced to its own source plane with ratios rs (n_planes, N)."""
    t1, alphas, psis, As = multiplane_parts(planes, r, tx, ty)
    beta = t1.clone()
    eye = torch.eye(2, dtype=torch.float64)
    A = eye.expand_as(As[0]).clone()
    for j in range(len(planes)):
        beta = beta - rs[j][None, :, None] * alphas[j]
        A = A - rs[j][None, :, None, None] * (psis[j] @ As[j])
    return beta, A
