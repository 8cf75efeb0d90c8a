"""Pins of the oracle's stretch-move sampler: the z distribution (density 1/sqrt(z) on
[1/a, a], mean known in closed form), and the stationary distribution on a Gaussian target
(mean and covariance), which fails without the z^(P-1) factor of the acceptance."""
import math

import numpy as np

from oracle import sampler as smp


def test_z_draws_follow_inverse_sqrt_density():
    a = 2.0
    u = np.random.default_rng(0).uniform(0, 1, 200000)
    z = smp.z_of(u, a)
    assert z.min() >= 1 / a - 1e-12 and z.max() <= a + 1e-12
    # g(z) = 1/(2 sqrt z (sqrt a - 1/sqrt a)) on [1/a, a]; E[z] = (a^1.5 - a^-1.5) / (3 (sqrt a - 1/sqrt a))
    mean = (a ** 1.5 - a ** -1.5) / (3 * (math.sqrt(a) - 1 / math.sqrt(a)))
    assert abs(z.mean() - mean) < 4 * z.std() / math.sqrt(len(z))


def _gauss_chi2(mu, cinv):
    def f(x):
        d = x - mu
        return np.einsum("ni,ij,nj->n", d, cinv, d)
    return f


def test_stationary_distribution_is_the_target():
    rng = np.random.default_rng(1)
    P, S, steps = 3, 64, 1500
    mu = np.array([1.0, -2.0, 0.5])
    C = np.array([[1.0, 0.6, 0.0], [0.6, 2.0, -0.3], [0.0, -0.3, 0.5]])
    f = _gauss_chi2(mu, np.linalg.inv(C))
    x = mu + rng.normal(0, 0.1, (S, P))
    c = f(x)
    lo, hi = np.full(P, -1e9), np.full(P, 1e9)
    samples = []
    for t in range(steps):
        smp.run(x, c, rng.uniform(0, 1, (1, S, 3)), 2.0, lo, hi, f)
        if t >= 300:
            samples.append(x.copy())
    s = np.concatenate(samples)
    assert np.allclose(s.mean(0), mu, atol=0.12)
    assert np.allclose(np.cov(s.T), C, atol=0.2)
    # without the z^(P-1) factor the ensemble contracts: the target covariance is not reached
    def half_no_jacobian(x, chi2, half, u, a, lo, hi, chi2_fn):
        S_, P_ = x.shape
        h = S_ // 2
        me = range(0, h) if half == 0 else range(h, S_)
        other = x[h:] if half == 0 else x[:h]
        for n, k in enumerate(me):
            j = smp.partner_of(u[n, 0], h)
            z = smp.z_of(u[n, 1], a)
            y = other[j] + z * (x[k] - other[j])
            cy = chi2_fn(y[None])[0]
            if math.log(u[n, 2]) < -0.5 * (cy - chi2[k]):
                x[k] = y
                chi2[k] = cy
    x = mu + rng.normal(0, 0.1, (S, P))
    c = f(x)
    wrong = []
    for t in range(steps):
        u = rng.uniform(0, 1, (S, 3))
        half_no_jacobian(x, c, 0, u[:S // 2], 2.0, lo, hi, f)
        half_no_jacobian(x, c, 1, u[S // 2:], 2.0, lo, hi, f)
        if t >= 300:
            wrong.append(x.copy())
    w = np.concatenate(wrong)
    assert np.abs(np.cov(w.T) - C).max() > 0.2


def test_prior_box_rejects():
    """With u_accept ~ 0 every finite proposal inside the box is accepted; the ones that
    leave the box are not."""
    f = _gauss_chi2(np.zeros(2), 1e-6 * np.eye(2))
    x = np.array([[0.0, 0.0], [0.5, 0.5], [0.9, 0.9], [-0.9, 0.2]])
    c = f(x)
    u = np.array([[0.0, 1.0, 1e-300], [0.0, 1.0, 1e-300]])   # partner 0 of the other half, z = a
    lo, hi = np.full(2, -1.0), np.full(2, 1.0)
    a = 4.0
    props = x[2] + a * (x[:2] - x[2])                       # y = x_j + z (x_k - x_j)
    inside = np.all((props >= lo) & (props <= hi), axis=1)
    x0 = x.copy()
    acc = smp.half_step(x, c, 0, u, a, lo, hi, f)
    assert list(acc) == list(inside)
    for n in range(2):
        assert np.array_equal(x[n], props[n] if inside[n] else x0[n])


# ------------------------------------------------------------ Metropolis-Hastings ----
def test_mh_acceptance_rate_on_a_standard_normal():
    """For a N(0, 1) target and a N(0, s^2) random-walk proposal, the stationary acceptance
    probability is (2 / pi) arctan(2 / s)."""
    rng = np.random.default_rng(3)
    f = _gauss_chi2(np.zeros(1), np.eye(1))
    S, steps = 2000, 60
    x = rng.normal(0, 1, (S, 1))         # start in the stationary distribution
    c = f(x)
    lo, hi = np.full(1, -1e9), np.full(1, 1e9)
    for s in (0.5, 2.0, 6.0):
        acc = smp.mh_run(x, c, rng.normal(0, 1, (steps, S, 1)), rng.uniform(0, 1, (steps, S)),
                         np.array([s]), lo, hi, f)
        rate = acc / (steps * S)
        ref = 2 / math.pi * math.atan(2 / s)
        assert abs(rate - ref) < 0.01, (s, rate, ref)


def test_mh_stationary_distribution_is_the_target():
    rng = np.random.default_rng(4)
    mu = np.array([1.0, -2.0])
    C = np.array([[1.0, 0.5], [0.5, 2.0]])
    f = _gauss_chi2(mu, np.linalg.inv(C))
    S = 400
    x = mu + rng.normal(0, 0.1, (S, 2))
    c = f(x)
    lo, hi = np.full(2, -1e9), np.full(2, 1e9)
    smp.mh_run(x, c, rng.normal(0, 1, (300, S, 2)), rng.uniform(0, 1, (300, S)), np.array([1.2, 1.6]),
               lo, hi, f)
    samples = []
    for _ in range(30):
        smp.mh_run(x, c, rng.normal(0, 1, (10, S, 2)), rng.uniform(0, 1, (10, S)), np.array([1.2, 1.6]),
                   lo, hi, f)
        samples.append(x.copy())
    s = np.concatenate(samples)
    assert np.allclose(s.mean(0), mu, atol=0.08)
    assert np.allclose(np.cov(s.T), C, atol=0.15)


def test_mh_prior_box_and_acceptance_rule():
    f = _gauss_chi2(np.zeros(2), np.eye(2))
    x = np.array([[0.0, 0.0], [0.9, 0.0], [0.0, 0.0]])
    c = f(x)
    z = np.array([[0.5, 0.0], [1.0, 0.0], [0.0, 2.0]])
    u = np.array([1e-300, 1e-300, 0.999])
    lo, hi = np.full(2, -1.0), np.full(2, 1.5)
    acc = smp.mh_step(x, c, z, u, np.array([1.0, 1.0]), lo, hi, f)
    # chain 0: y = (0.5, 0) inside, accepted; chains 1 and 2: y = (1.9, 0) and (0, 2) leave
    # the box (hi = 1.5), rejected whatever u
    assert list(acc) == [True, False, False]
    x2 = np.array([[0.0, 0.0]]); c2 = f(x2)
    u_acc = math.exp(-0.5 * 0.25) * 0.999          # just below exp(-d chi^2 / 2) for y = (0.5, 0)
    u_rej = math.exp(-0.5 * 0.25) * 1.001
    assert smp.mh_step(x2.copy(), c2.copy(), np.array([[0.5, 0.0]]), np.array([u_acc]), np.ones(2), lo, hi, f)[0]
    assert not smp.mh_step(x2.copy(), c2.copy(), np.array([[0.5, 0.0]]), np.array([u_rej]), np.ones(2), lo, hi, f)[0]
