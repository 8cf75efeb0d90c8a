"""Shared test helpers: oracle evaluation of the same seeded inputs, error metrics."""
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
