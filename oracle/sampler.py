"""Posterior samplers of Sec. 3.5 (oracle): the affine-invariant ensemble sampler's stretch
move and random-walk Metropolis-Hastings.  TEST INFRASTRUCTURE ONLY.

The paper samples the posterior with the AIES of Goodman & Weare (2010) (Sec. 3.5), with
likelihood L ~ exp(-chi^2/2) (Sec. 3) and uniform priors.  One step updates the two halves
of the ensemble in turn: walker k of one half picks a partner j from the other half, draws
z from g(z) ~ 1/sqrt(z) on [1/a, a], proposes y = x_j + z (x_k - x_j), and accepts with
probability min(1, z^(P-1) exp(-(chi^2(y) - chi^2(x_k))/2)); a proposal outside the prior
box is rejected.  The random numbers are inputs: u[k] = (u_partner, u_z, u_accept) for each
walker of the half, so that the GPU sampler can be replayed exactly.
"""
import math

import numpy as np


def z_of(u, a):
    """Inverse CDF of g(z) ~ 1/sqrt(z) on [1/a, a]: z = ((a - 1) u + 1)^2 / a."""
    return ((a - 1.0) * u + 1.0) ** 2 / a


def partner_of(u, n_other):
    return min(int(u * n_other), n_other - 1)


def half_step(x, chi2, half, u, a, lo, hi, chi2_fn):
    """Updates walkers of `half` (0: first S/2, 1: second S/2) in place; returns accepts."""
    S, P = x.shape
    h = S // 2
    me = range(0, h) if half == 0 else range(h, S)
    other = x[h:] if half == 0 else x[:h]
    props = np.empty((h, P))
    zs = np.empty(h)
    for n, k in enumerate(me):
        j = partner_of(u[n, 0], h)
        zs[n] = z_of(u[n, 1], a)
        props[n] = other[j] + zs[n] * (x[k] - other[j])
    inside = np.all((props >= lo) & (props <= hi), axis=1)
    c_new = chi2_fn(props)
    acc = np.zeros(h, dtype=bool)
    for n, k in enumerate(me):
        if not inside[n] or not np.isfinite(c_new[n]):
            continue
        log_r = (P - 1) * math.log(zs[n]) - 0.5 * (c_new[n] - chi2[k])
        if math.log(u[n, 2]) < log_r:
            x[k] = props[n]
            chi2[k] = c_new[n]
            acc[n] = True
    return acc


def run(x, chi2, uniforms, a, lo, hi, chi2_fn):
    """uniforms: (n_steps, S, 3); the first S/2 rows drive half 0, the rest half 1."""
    S = x.shape[0]
    h = S // 2
    n_acc = 0
    for step in range(uniforms.shape[0]):
        n_acc += half_step(x, chi2, 0, uniforms[step, :h], a, lo, hi, chi2_fn).sum()
        n_acc += half_step(x, chi2, 1, uniforms[step, h:], a, lo, hi, chi2_fn).sum()
    return n_acc


def mh_step(x, chi2, z, u, step, lo, hi, chi2_fn):
    """One Metropolis-Hastings step of S independent chains with the symmetric Gaussian
    random-walk proposal y_k = x_k + step * z_k (z: (S, P) standard normals, step: (P,)):
    y_k is accepted when it lies in the prior box, chi^2(y_k) is finite and
    log u_k < -(chi^2(y_k) - chi^2(x_k)) / 2 (u: (S,) uniforms); a symmetric proposal has no
    Hastings factor.  Updates x, chi2 in place; returns the accept flags."""
    props = x + step[None, :] * z
    inside = np.all((props >= lo) & (props <= hi), axis=1)
    c_new = chi2_fn(props)
    acc = np.zeros(x.shape[0], dtype=bool)
    for k in range(x.shape[0]):
        if not inside[k] or not np.isfinite(c_new[k]):
            continue
        if math.log(u[k]) < -0.5 * (c_new[k] - chi2[k]):
            x[k] = props[k]
            chi2[k] = c_new[k]
            acc[k] = True
    return acc


def mh_run(x, chi2, normals, uniforms, step, lo, hi, chi2_fn):
    """normals: (n_steps, S, P); uniforms: (n_steps, S).  Returns the number accepted."""
    n_acc = 0
    for t in range(normals.shape[0]):
        n_acc += mh_step(x, chi2, normals[t], uniforms[t], step, lo, hi, chi2_fn).sum()
    return n_acc

