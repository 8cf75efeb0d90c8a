"""Writes csrc/lf_cse_table.h: the cored-steep-ellipsoid (CSE) expansion of the spherical NFW
convergence that the elliptical NFW component (LF_ENFW) evaluates.

With x = r / r_s, the NFW convergence is 2 kappa_s g(x), g = (F(x) - 1) / (1 - x^2),
F = atanh(sqrt(1 - x^2)) / sqrt(1 - x^2) (x < 1) or atan(sqrt(x^2 - 1)) / sqrt(x^2 - 1) (x > 1)
(Bartelmann 1996).  Following the method of Oguri (2021, PASP 133, 074504) it is approximated
by sum_i a_i / (2 (s_i^2 + x^2)^(3/2)) with 40 fixed scales s_i = 10^(-5 + 9 i / 39) and a_i >= 0
from non-negative least squares on the relative residual at 2000 log-spaced x in
[1e-4, 1e3]; zero terms are dropped.  Run: python -m paper_2609_08649_b300.gen_cse_table
"""
import os

import numpy as np
from scipy.optimize import nnls

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "lf_cse_table.h")


def nfw_g(x):
    x = np.asarray(x, dtype=np.float64)
    w = (1.0 - x) * (1.0 + x)
    out = np.empty_like(x)
    near = np.abs(w) < 1e-3
    n = np.arange(1, 13)
    out[near] = (w[near, None] ** (n - 1) / (2 * n + 1)).sum(1)     # sum_{n>=1} w^(n-1) / (2n+1)
    lt, gt = (w > 0) & ~near, (w < 0) & ~near
    r = np.sqrt(w[lt])
    out[lt] = (np.arctanh(r) / r - 1.0) / w[lt]
    r = np.sqrt(-w[gt])
    out[gt] = (np.arctan(r) / r - 1.0) / w[gt]
    return out


def fit():
    s = 10.0 ** np.linspace(-5.0, 4.0, 40)
    x = 10.0 ** np.linspace(-4.0, 3.0, 2000)
    g = nfw_g(x)
    A = 0.5 / (x[:, None] ** 2 + s[None, :] ** 2) ** 1.5
    a, _ = nnls(A / g[:, None], np.ones_like(g), maxiter=50 * 40 * 40)
    return s[a > 0], a[a > 0]


def ff_pairs(v):
    """float-float pairs (hi, lo) of FP64 values, hi = float32(v), lo = float32(v - hi)."""
    hi = np.asarray(v, dtype=np.float64).astype(np.float32)
    lo = (np.asarray(v, dtype=np.float64) - hi.astype(np.float64)).astype(np.float32)
    return [f"{{{float(h):.9e}f, {float(l):.9e}f}}" for h, l in zip(hi, lo)]


def main():
    s, a = fit()
    rows = lambda v: [", ".join(f"{t:.17e}" for t in v[i:i + 3]) for i in range(0, len(v), 3)]
    body = lambda v: ", \\\n  ".join(rows(v))
    pairs = lambda v: ", \\\n  ".join(ff_pairs(v))
    with open(OUT, "w") as f:
        f.write("// Generated by gen_cse_table.py: the cored-steep-ellipsoid expansion of the spherical\n"
                "// NFW convergence, g(x) = sum_i a_i / (2 (s_i^2 + x^2)^(3/2)), x = r / r_s.\n"
                "#pragma once\n\n"
                f"#define LF_CSE_N {len(s)}\n"
                f"#define LF_CSE_S_LIST \\\n  {body(s)}\n"
                f"#define LF_CSE_A_LIST \\\n  {body(a)}\n"
                "// float-float (hi, lo) of s_i and of a_i / s_i\n"
                f"#define LF_CSE_S_FF_LIST \\\n  {pairs(s)}\n"
                f"#define LF_CSE_C_FF_LIST \\\n  {pairs(a / s)}\n")
    print(OUT, len(s))


if __name__ == "__main__":
    main()
