"""Shared test helpers: oracle evaluation of the same seeded inputs, error metrics."""
import functools
import math

import numpy as np
import torch

from oracle import cosmology as cz
from oracle import lensing as OL
from oracle import model as OM
from oracle import profiles as pr
from paper_2609_08649_b300 import workloads as W

U32 = 2.0 ** -24


def oracle_plane_terms(pl, x, y):
    """Oracle alpha, psi and the sum over components of |alpha_k| and |psi_k| (the scale
    that FP32 rounding errors of the mixed path are proportional to)."""
    tx = torch.as_tensor(np.asarray(x, dtype=np.float64))[None]
    ty = torch.as_tensor(np.asarray(y, dtype=np.float64))[None]
    tot = [torch.zeros_like(tx) for _ in range(5)]
    absa = torch.zeros_like(tx)
    absp = torch.zeros_like(tx)
    for k, kind in enumerate(pl.kind):
        col = lambda f: f[:, k:k + 1]
        o = OL.component(kind, tx - col(pl.x), ty - col(pl.y), col(pl.b), col(pl.eps), col(pl.pa),
                         col(pl.core), col(pl.cut))
        tot = [t + v for t, v in zip(tot, o)]
        absa += torch.hypot(o[0], o[1])
        absp += o[2].abs() + o[3].abs() + o[4].abs()
    if pl.n_members:
        bm, cm, tm = OL.member_fields(pl)
        for m in range(pl.n_members):
            o = pr.pje_sph(tx - pl.mx[m], ty - pl.my[m], bm[:, m:m + 1], cm[:, m:m + 1], tm[:, m:m + 1])
            tot = [t + v for t, v in zip(tot, o)]
            absa += torch.hypot(o[0], o[1])
            absp += o[2].abs() + o[3].abs() + o[4].abs()
    return [t[0].numpy() for t in tot], absa[0].numpy(), absp[0].numpy()


def grid_xy(g):
    xs = g.x0 + g.dx * np.arange(g.nx)
    ys = g.y0 + g.dy * np.arange(g.ny)
    X, Y = np.meshgrid(xs, ys)
    return X, Y


def mu_det(pxx, pyy, pxy, a):
    k = 0.5 * (pxx + pyy)
    g1 = 0.5 * (pxx - pyy)
    det = (1 - a * k) ** 2 - a * a * (g1 * g1 + pxy * pxy)
    return 1 / det, det


def chi2_mixed_bound(wl, cat, theta, sigma=None, coef=4.0):
    """First-order bound on |chi2_mixed - chi2| per sample from the FP32 rounding of each
    component (relative coef * u): d chi2 = sum_i 2 a_f [-w_i . d alpha_i + w_i^T d Psi_i z_i]
    (w = M d, z = mu d, d = beta_i - beta_model), with |d alpha_i| <= coef u sum_k |alpha_k|
    and |d Psi_i| <= coef u sum_k |psi_k| at image i."""
    from oracle import lensing as OLL
    sig = wl.sigma_pos if sigma is None else sigma
    th = torch.as_tensor(theta)
    pl = OM.apply_params(wl, th)[0]
    a_f = OM.family_adis(wl, th, OM.single_plane_adis(wl, cat.fam_zs))   # (S, F)
    off = list(cat.fam_off)
    n = len(cat.theta_obs)
    tx = torch.tensor(cat.theta_obs[:, 0])[None]
    ty = torch.tensor(cat.theta_obs[:, 1])[None]
    S = th.shape[0]
    sa = torch.zeros(S, n, dtype=torch.float64)
    sp = torch.zeros(S, n, dtype=torch.float64)
    for k, kind in enumerate(pl.kind):
        col = lambda f: f[:, k:k + 1]
        o = OLL.component(kind, tx - col(pl.x), ty - col(pl.y), col(pl.b), col(pl.eps), col(pl.pa),
                          col(pl.core), col(pl.cut))
        sa += torch.hypot(o[0], o[1])
        sp += o[2].abs() + o[3].abs() + o[4].abs()
    if pl.n_members:
        bm, cm, tm = OLL.member_fields(pl)
        for m in range(pl.n_members):
            o = pr.pje_sph(tx - pl.mx[m], ty - pl.my[m], bm[:, m:m + 1], cm[:, m:m + 1], tm[:, m:m + 1])
            sa += torch.hypot(o[0], o[1])
            sp += o[2].abs() + o[3].abs() + o[4].abs()
    beta, A = OLL.single_plane_source_terms(pl, torch.tensor(cat.theta_obs), off, a_f)
    sinv = torch.tensor(np.tile([1 / sig ** 2, 0, 1 / sig ** 2], (n, 1)))
    Sm = OLL.sinv_matrix(sinv)
    mu = torch.linalg.inv(A)
    M = mu.transpose(-1, -2) @ Sm[None] @ mu
    bound = torch.zeros(S, dtype=torch.float64)
    for f in range(len(off) - 1):
        i0, i1 = off[f], off[f + 1]
        if i1 - i0 < 2:
            continue
        Mf, bf = M[:, i0:i1], beta[:, i0:i1]
        bmod = torch.linalg.solve(Mf.sum(1), (Mf @ bf[..., None]).sum(1))
        d = bf[..., None] - bmod[:, None]
        w = (Mf @ d)[..., 0]
        z = (mu[:, i0:i1] @ d)[..., 0]
        wn, zn = w.norm(dim=-1), z.norm(dim=-1)
        da = coef * U32 * sa[:, i0:i1]
        dp = coef * U32 * sp[:, i0:i1]
        bound += (2 * a_f[:, f:f + 1] * (wn * da + wn * zn * dp)).sum(1)
    return bound.numpy()


def families_off_critical(wl, cat, theta, thr):
    """The catalogue restricted to the families whose images all keep |det A_i| >= thr for
    every sample (oracle FP64 source-plane terms).  Near a critical curve the chi^2 gradient
    grows like 1/det^3 and the FP32 arithmetic of the mixed tiers no longer resolves it."""
    from oracle import gradient as OG
    kw = {"fam_zs": list(cat.fam_zs)} if len(wl.planes) > 1 else \
        {"fam_adis": OM.single_plane_adis(wl, cat.fam_zs)}
    with torch.no_grad():
        _, A = OG._terms(wl, torch.as_tensor(theta), torch.tensor(cat.theta_obs), list(cat.fam_off), **kw)
    det = torch.linalg.det(A).abs().min(0).values.numpy()
    keep = [f for f in range(len(cat.fam_off) - 1)
            if det[cat.fam_off[f]:cat.fam_off[f + 1]].min() >= thr]
    idx = np.concatenate([np.arange(cat.fam_off[f], cat.fam_off[f + 1]) for f in keep])
    off = np.concatenate([[0], np.cumsum([cat.fam_off[f + 1] - cat.fam_off[f] for f in keep])])
    return W.Catalogue(cat.theta_obs[idx], cat.theta_true[idx], off, np.asarray(cat.fam_zs)[keep])


@functools.lru_cache(maxsize=2)
def three_plane_field(z_src=4.0, x0=-80.0, h=0.4, n=401):
    """The three-plane model (multiplane_c3) and, on an n^2 vertex grid from (x0, x0) with step
    h, the effective deflection alpha_eff = theta - beta(theta) of its recursion to z_src
    (oracle code only).  Returns (wl, planes, r, rs, ax, ay)."""
    from oracle import cosmology as cz
    wl = W.multiplane_c3(n_grid=8)
    planes = OM.build_planes(wl)
    zs = [p.z for p in wl.planes]
    r, _ = cz.multiplane_ratios(zs, zs[-1] + 1.0, wl.cosmo.H0, wl.cosmo.Om)
    rs1 = cz.multiplane_ratios(zs, z_src, wl.cosmo.H0, wl.cosmo.Om)[1]
    xs = x0 + h * np.arange(n)
    X, Y = np.meshgrid(xs, xs)
    rs = torch.tensor([[float(v)] * (n * n) for v in rs1], dtype=torch.float64)
    beta, _ = OL.multi_plane_beta_A(planes, r, rs, torch.tensor(X.ravel())[None], torch.tensor(Y.ravel())[None])
    ax = (X.ravel() - beta[0, :, 0].numpy()).reshape(n, n)
    ay = (Y.ravel() - beta[0, :, 1].numpy()).reshape(n, n)
    return wl, planes, r, rs1, ax, ay


def three_plane_polish(planes, r, rs1, src, th, iters=20, max_step=None):
    """Newton steps of the multi-plane lens equation beta(theta) = src from positions th (k, 2);
    with max_step, a longer step is not taken (the position stays)."""
    th = torch.tensor(np.asarray(th, dtype=np.float64))
    rsk = torch.tensor([[float(v)] * len(th) for v in rs1], dtype=torch.float64)
    for _ in range(iters):
        b, A = OL.multi_plane_beta_A(planes, r, rsk, th[None, :, 0], th[None, :, 1])
        step = torch.linalg.solve(A[0], (b[0] - torch.tensor(src))[..., None])[..., 0]
        if max_step is not None:
            ok = (step * step).sum(-1) <= max_step * max_step
            step = torch.where(ok[:, None], step, torch.zeros_like(step))
        th = th - step
    return th.numpy()


@functools.lru_cache(maxsize=2)
def three_plane_images(n_src=12, seed=41, z_src=4.0, sigma=0.001):
    """A catalogue of true images of the three-plane model (multiplane_c3) for sources at
    z_src, made with oracle code only: marching squares on the effective deflection of
    three_plane_field (oracle images.find_images with a = 1), then Newton steps of the
    multi-plane lens equation toward each image's own source.  Families keep the sources
    with 2-5 images; the observed positions carry seeded Gaussian noise of sigma.  Returns
    (workload, Catalogue)."""
    from oracle import images as OI
    wl, planes, r, rs1, ax, ay = three_plane_field(z_src)
    fams = []
    for src in W.source_candidates(seed, n_src, 10.0, 2.0, -2.0):
        imgs = OI.find_images(None, 1.0, src, -80.0, -80.0, 0.4, 401, newton=False, alpha_grid=(ax, ay))
        if len(imgs) < 2:
            continue
        fams.append(three_plane_polish(planes, r, rs1, src, imgs[:5]))
    true = np.concatenate(fams)
    off = np.concatenate([[0], np.cumsum([len(f) for f in fams])]).astype(np.int32)
    obs = true + W.position_noise(seed + 1, len(true), sigma)
    return wl, W.Catalogue(obs, true, off, np.full(len(fams), z_src))


def _abs_sums(pl, tx, ty):
    """Per sample and position: sum_k |alpha_k| and sum_k max(|psi_xx|, |psi_yy|, |psi_xy|)_k
    over a plane's components and members (oracle FP64).  tx, ty: (S, N)."""
    sa = torch.zeros_like(tx)
    sp = torch.zeros_like(tx)
    for k, kind in enumerate(pl.kind):
        col = lambda f: f[:, k:k + 1]
        o = OL.component(kind, tx - col(pl.x), ty - col(pl.y), col(pl.b), col(pl.eps), col(pl.pa),
                         col(pl.core), col(pl.cut))
        sa += torch.hypot(o[0], o[1])
        sp += torch.maximum(torch.maximum(o[2].abs(), o[3].abs()), o[4].abs())
    if pl.n_members:
        bm, cm, tm = OL.member_fields(pl)
        for m in range(pl.n_members):
            o = pr.pje_sph(tx - pl.mx[m], ty - pl.my[m], bm[:, m:m + 1], cm[:, m:m + 1], tm[:, m:m + 1])
            sa += torch.hypot(o[0], o[1])
            sp += torch.maximum(torch.maximum(o[2].abs(), o[3].abs()), o[4].abs())
    return sa, sp


def chi2_rounding_bound(wl, cat, theta, alpha_coef=0.0, psi_coef=4.0, alg_coef=4.0, sigma=None):
    """First-order bound on |chi2_tier - chi2| per sample from the FP32 arithmetic of the mixed
    tiers, single- or multi-plane, from the oracle's chi^2 differentiated (autograd) in each
    image's beta_i and A_i:
      |d chi2| <= sum_i |dchi2/dbeta_i| . e_i + |dchi2/dA_i| : E_i + alg_coef u sum_i |d_i|^T |M_i| |d_i|
    with e_i = alpha_coef u sum_j rs_j sum_k |alpha_k(theta_j)| (FP32 deflections, the mixed
    forward launch's members), E_i = psi_coef u [sum_j rs_j sum_k |psi_k(theta_j)| max|A_j| + |A_i|]
    elementwise (psi_ij of every component in FP32; A rounded to FP32 before mu = A^-1 and
    M = mu^T S^-1 mu, a backward error of order u |A|), and the last term the FP32 rounding of M
    itself (d_i = beta_i - beta_model)."""
    from oracle import gradient as OG
    sig = wl.sigma_pos if sigma is None else sigma
    th = torch.as_tensor(theta)
    n = len(cat.theta_obs)
    off = list(cat.fam_off)
    tobs = torch.tensor(cat.theta_obs)
    planes = OM.apply_params(wl, th)
    zs = [p.z for p in wl.planes]
    if len(planes) == 1:
        a_f = OM.family_adis(wl, th, OM.single_plane_adis(wl, cat.fam_zs))
        fam = np.concatenate([[f] * (off[f + 1] - off[f]) for f in range(len(off) - 1)])
        rs = [a_f[:, fam]]                                     # (S, N)
        r = [[0.0]]
    else:
        r, _ = cz.multiplane_ratios(zs, zs[-1] + 1.0, wl.cosmo.H0, wl.cosmo.Om)
        fam_rs = [cz.multiplane_ratios(zs, z, wl.cosmo.H0, wl.cosmo.Om)[1] for z in cat.fam_zs]
        rs = [v[None] for v in OL.image_ratios(fam_rs, off, len(planes))]
    with torch.no_grad():
        t1, alphas, psis, As = OL.multiplane_parts(planes, r, tobs[None, :, 0], tobs[None, :, 1])
        ea = torch.zeros(th.shape[0], n, dtype=torch.float64)
        EA = torch.zeros(th.shape[0], n, dtype=torch.float64)
        for j, pl in enumerate(planes):
            tj = t1.clone()
            for i in range(j):
                tj = tj - r[i][j] * alphas[i]
            sa, sp = _abs_sums(pl, tj[..., 0], tj[..., 1])
            ea += rs[j] * sa
            EA += rs[j] * sp * As[j].abs().amax((-1, -2))
    beta, A = OG._terms(wl, th, tobs, off, **({"fam_adis": OM.single_plane_adis(wl, cat.fam_zs)}
                                               if len(planes) == 1 else {"fam_zs": list(cat.fam_zs)}))
    beta = beta.detach().requires_grad_(True)
    A = A.detach().requires_grad_(True)
    sinv = torch.tensor(np.tile([1 / sig ** 2, 0, 1 / sig ** 2], (n, 1)))
    c = OL.chi2_src(beta, A, sinv, off)
    gb, gA = torch.autograd.grad(c.sum(), (beta, A))
    with torch.no_grad():
        Sm = OL.sinv_matrix(sinv)
        mu = torch.linalg.inv(A)
        M = mu.transpose(-1, -2) @ Sm[None] @ mu
        alg = torch.zeros(th.shape[0], dtype=torch.float64)
        for f in range(len(off) - 1):
            i0, i1 = off[f], off[f + 1]
            if i1 - i0 < 2:
                continue
            Mf, bf = M[:, i0:i1], beta[:, i0:i1]
            bm = torch.linalg.solve(Mf.sum(1), (Mf @ bf[..., None]).sum(1))
            d = (bf[..., None] - bm[:, None]).abs()
            alg += (d.transpose(-1, -2) @ Mf.abs() @ d)[..., 0, 0].sum(1)
        E = psi_coef * U32 * (EA[..., None, None] + A.abs())
        bound = (gb.abs().sum(-1) * alpha_coef * U32 * ea).sum(1) + (gA.abs() * E).sum((-1, -2, -3)) \
            + alg_coef * U32 * alg
    return bound.numpy()
