"""Nelder-Mead downhill simplex (Nelder & Mead 1965), the paper's optimizer (Sec. 3.5), for many
independent runs (oracle, FP64).  TEST INFRASTRUCTURE ONLY.

Coefficients and rules as in Lagarias et al. (1998): reflection 1, expansion 2, contraction 1/2,
shrink 1/2.  One iteration of one run, with its n + 1 vertices ordered by f (stable: equal
values keep their order):
  xbar = (x_1 + ... + x_n) / n (summed in vertex order), x_r = xbar + (xbar - x_{n+1});
  f_1 <= f_r < f_n              -> x_r replaces x_{n+1};
  f_r < f_1                     -> x_e = xbar + 2 (x_r - xbar); the better of x_e (if f_e < f_r)
                                   and x_r replaces x_{n+1};
  f_n <= f_r < f_{n+1}          -> x_c = xbar + (x_r - xbar) / 2; if f_c <= f_r it replaces
                                   x_{n+1}, else shrink;
  f_r >= f_{n+1}                -> x_cc = xbar - (xbar - x_{n+1}) / 2; if f_cc < f_{n+1} it replaces
                                   x_{n+1}, else shrink;
  shrink                        -> x_i = x_1 + (x_i - x_1) / 2 for i = 2 .. n + 1, all re-evaluated.
A point outside the prior box [lo, hi] has f = +inf.  Every vector operation is one IEEE
operation per component (no fused multiply-add), so that an implementation that performs the
same operations reproduces the simplices exactly.
"""
import numpy as np


def _boxed(fn, lo, hi):
    def g(pts):
        pts = np.asarray(pts, dtype=np.float64)
        if len(pts) == 0:
            return np.zeros(0)
        v = np.asarray(fn(pts), dtype=np.float64).copy()
        out = ~np.all((pts >= lo) & (pts <= hi), axis=1)
        v[out] = np.inf
        v[~np.isfinite(v)] = np.inf
        return v
    return g


def order(X, F):
    """Sort each run's vertices by f, stably (in place)."""
    for m in range(X.shape[0]):
        idx = np.argsort(F[m], kind="stable")
        X[m] = X[m][idx]
        F[m] = F[m][idx]


def centroid(X):
    """(M, n): mean of the best n vertices, summed in vertex order."""
    M, n1, n = X.shape
    s = X[:, 0].copy()
    for i in range(1, n1 - 1):
        s = s + X[:, i]
    return s / float(n1 - 1)


def iterate(X, F, fn, lo, hi):
    """One iteration of every run, in place.  X: (M, n + 1, n), F: (M, n + 1).
    Returns the per-run step taken: 0 reflect, 1 expand, 2 outside contraction,
    3 inside contraction, 4 shrink."""
    f = _boxed(fn, lo, hi)
    M, n1, n = X.shape
    order(X, F)
    xb = centroid(X)
    xw = X[:, n1 - 1]
    xr = xb + (xb - xw)
    fr = f(xr)
    step = np.zeros(M, dtype=np.int64)
    # second point per run: expansion or contraction
    x2 = xr.copy()
    need2 = np.zeros(M, dtype=bool)
    for m in range(M):
        f1, fn_, fw = F[m, 0], F[m, n1 - 2], F[m, n1 - 1]
        if fr[m] < f1:
            step[m] = 1
            x2[m] = xb[m] + 2.0 * (xr[m] - xb[m])
            need2[m] = True
        elif fr[m] < fn_:
            step[m] = 0
        elif fr[m] < fw:
            step[m] = 2
            x2[m] = xb[m] + 0.5 * (xr[m] - xb[m])
            need2[m] = True
        else:
            step[m] = 3
            x2[m] = xb[m] - 0.5 * (xb[m] - xw[m])
            need2[m] = True
    f2 = np.full(M, np.inf)
    if need2.any():
        f2[need2] = f(x2[need2])
    shrink = np.zeros(M, dtype=bool)
    for m in range(M):
        w = n1 - 1
        if step[m] == 0:
            X[m, w], F[m, w] = xr[m], fr[m]
        elif step[m] == 1:
            if f2[m] < fr[m]:
                X[m, w], F[m, w] = x2[m], f2[m]
            else:
                X[m, w], F[m, w] = xr[m], fr[m]
        elif step[m] == 2:
            if f2[m] <= fr[m]:
                X[m, w], F[m, w] = x2[m], f2[m]
            else:
                shrink[m] = True
        else:
            if f2[m] < F[m, w]:
                X[m, w], F[m, w] = x2[m], f2[m]
            else:
                shrink[m] = True
    if shrink.any():
        ms = np.nonzero(shrink)[0]
        for m in ms:
            for i in range(1, n1):
                X[m, i] = X[m, 0] + 0.5 * (X[m, i] - X[m, 0])
        pts = X[ms, 1:].reshape(-1, n)
        F[ms, 1:] = f(pts).reshape(len(ms), n1 - 1)
        step[ms] = 4
    return step


def run(X, F, fn, lo, hi, n_iter):
    steps = np.zeros(5, dtype=np.int64)
    for _ in range(n_iter):
        s = iterate(X, F, fn, lo, hi)
        steps += np.bincount(s, minlength=5)
    return steps
