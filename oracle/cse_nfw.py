"""Elliptical NFW as a sum of cored steep ellipsoids (oracle, FP64).  TEST INFRASTRUCTURE ONLY.

The paper models its cluster halos with elliptical NFW profiles approximated by the method of
Oguri (2021, PASP 133, 074504) (Sec. 4.1, 4.2): the spherical NFW convergence is written as a
sum of cored steep ellipsoids (CSE), whose lensing quantities have closed forms, and the
ellipticity is then applied to every term.  The coefficients here are our own fit (Oguri's
printed table is not reproduced): with x = r / r_s and the NFW convergence
kappa_NFW = 2 kappa_s g(x), g = (F(x) - 1) / (1 - x^2) (Bartelmann 1996),

    g(x) ~ sum_i a_i / (2 (s_i^2 + x^2)^(3/2)),

s_i = 10^(-5 + 9 i / 39), i = 0..39, and a_i >= 0 the non-negative least-squares solution of
the relative residual on 2000 log-spaced x in [1e-4, 1e3]; terms with a_i = 0 are dropped.
The fit's relative error on g is below 2e-6 over that range (pinned in
tests/test_oracle_enfw.py).
"""
import functools

import numpy as np
import torch
from scipy.optimize import nnls

from . import profiles as pr

S_LOG10_LO, S_LOG10_HI, N_TERMS = -5.0, 4.0, 40
X_LOG10_LO, X_LOG10_HI, N_NODES = -4.0, 3.0, 2000


def nfw_g(x):
    """g(x) = kappa_NFW / (2 kappa_s) from the oracle's spherical NFW (kappa = tr Psi / 2)."""
    x = torch.as_tensor(x, dtype=torch.float64)
    o = pr.nfw_sph(x, torch.zeros_like(x), 0.5, 1.0)
    return 0.5 * (o[2] + o[3])


@functools.lru_cache(maxsize=1)
def table():
    """(s_i, a_i) of the CSE sum, float64 numpy arrays (non-zero terms only)."""
    s = 10.0 ** np.linspace(S_LOG10_LO, S_LOG10_HI, N_TERMS)
    x = 10.0 ** np.linspace(X_LOG10_LO, X_LOG10_HI, N_NODES)
    g = nfw_g(x).numpy()
    basis = 0.5 / (s[None, :] ** 2 + x[:, None] ** 2) ** 1.5
    a, _ = nnls(basis / g[:, None], np.ones_like(g), maxiter=50 * N_TERMS * N_TERMS)
    keep = a > 0
    return s[keep].copy(), a[keep].copy()


def g_approx(x):
    s, a = table()
    x = np.asarray(x, dtype=np.float64)
    return (0.5 / (s[None, :] ** 2 + x.reshape(-1, 1) ** 2) ** 1.5 @ a).reshape(x.shape)
