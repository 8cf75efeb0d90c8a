"""Pins of the oracle's Nelder-Mead (Sec. 3.5): each step of the method forced on a crafted
2-D case and compared with its defining formula, convergence on Rosenbrock's function and on
a quadratic, and the prior box."""
import numpy as np

from oracle import optimizer as NM

BIG = np.full(2, 1e9)


def one(X, F, fn, lo=-BIG, hi=BIG):
    X = np.array(X, dtype=float)[None]
    F = np.array(F, dtype=float)[None]
    s = NM.iterate(X, F, fn, lo, hi)
    return int(s[0]), X[0], F[0]


def sq(c):
    c = np.asarray(c, dtype=float)
    return lambda p: ((np.asarray(p) - c) ** 2).sum(-1)


def test_reflection():
    f = sq([1.0, 1.8])
    X = [[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]
    F = f(np.array(X))
    step, Xn, Fn = one(X, F, f)
    # ordered: (0,1) f=1.64, (1,0) f=3.24, (0,0) f=4.24; xbar = (0.5, 0.5); x_r = (1, 1), f_r = 0.64 < f_1
    # -> expansion x_e = (1.5, 1.5), f_e = 0.34 < f_r: expansion taken
    assert step == 1
    assert np.allclose(Xn[2], [1.5, 1.5]) and np.isclose(Fn[2], f(np.array([1.5, 1.5])))
    g = sq([0.4, 0.9])
    # ordered: (0,1) 0.17, (1,0) 1.17, (0,0) 0.97 -> (0,1) 0.17, (0,0) 0.97, (1,0) 1.17
    # xbar = (0, 0.5), x_r = (-1, 1): f_r = 1.97 >= f_n = 0.97, < f_w? no (1.97 > 1.17) -> inside
    step, Xn, Fn = one(X, g(np.array(X)), g)
    assert step == 3
    assert np.allclose(Xn[2], [0.5, 0.25])                      # xbar - (xbar - x_w)/2, x_w = (1, 0)
    h = sq([0.45, 0.45])
    # f: (0,0) 0.405, (1,0) 0.505, (0,1) 0.505; xbar = (0.5, 0); x_r = (1, -1): 2.405 >= f_w
    step, Xn, Fn = one(X, h(np.array(X)), h)
    assert step in (3, 4)


def test_plain_reflection_and_outside_contraction():
    f = sq([0.6, 0.55])
    X = [[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]
    # f: (0,0) 0.6625, (1,0) 0.4625, (0,1) 0.5625 -> order (1,0), (0,1), (0,0)
    # xbar = (0.5, 0.5), x_r = (1, 1): f_r = 0.3625 < f_1 = 0.4625 -> expansion (2, 2): 3.5 > f_r -> x_r
    step, Xn, Fn = one(X, f(np.array(X)), f)
    assert step == 1 and np.allclose(Xn[2], [1.0, 1.0])
    g = sq([1.2, 1.2])
    # f: (0,0) 2.88, (1,0) 1.48, (0,1) 1.48 -> order (1,0), (0,1), (0,0); x_r = (1, 1): 0.08 < f_1 ->
    # expansion (1.5, 1.5): 0.18 > 0.08 -> x_r
    step, Xn, Fn = one(X, g(np.array(X)), g)
    assert step == 1 and np.allclose(Xn[2], [1.0, 1.0])
    k = lambda p: np.where(np.asarray(p)[..., 0] > 0.9, 10.0, 0.0) + sq([0.0, 0.0])(p)
    # f: (0,0) 0, (0,1) 1, (1,0) 11 -> order (0,0), (0,1), (1,0); xbar = (0, 0.5); x_r = (-1, 1):
    # f_r = 2 >= f_n = 1, < f_w = 11 -> outside contraction x_c = (-0.5, 0.75): 0.8125 <= 2
    step, Xn, Fn = one(X, k(np.array(X)), k)
    assert step == 2 and np.allclose(Xn[2], [-0.5, 0.75])
    r = lambda p: sq([0.0, 0.0])(p) + np.where(np.asarray(p)[..., 0] < -0.05, 5.0, 0.0)
    # f: (0,0) 0, (0,1) 1, (1,0) 1 -> stable order (0,0), (1,0), (0,1); xbar = (0.5, 0);
    # x_r = (1, -1): 2 >= f_n = 1 and < f_w? no: 2 > 1 -> inside x_cc = (0.25, 0.5): 0.3125 < 1
    step, Xn, Fn = one(X, r(np.array(X)), r)
    assert step == 3 and np.allclose(Xn[2], [0.25, 0.5])


def test_shrink():
    # a function whose every trial point is worse than the worst vertex forces the shrink
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    F0 = np.array([0.0, 1.0, 2.0])
    lut = {tuple(X[i]): F0[i] for i in range(3)}

    def f(p):
        p = np.atleast_2d(p)
        return np.array([lut.get(tuple(q), 100.0 + q.sum()) for q in p])
    step, Xn, Fn = one(X, F0, f)
    assert step == 4
    assert np.allclose(Xn, [[0, 0], [0.5, 0.0], [0.0, 0.5]])
    assert np.allclose(Fn[1:], [100.5, 100.5])


def test_rosenbrock_and_quadratic_convergence():
    ros = lambda p: 100.0 * (np.asarray(p)[..., 1] - np.asarray(p)[..., 0] ** 2) ** 2 + (1 - np.asarray(p)[..., 0]) ** 2
    x0 = np.array([-1.2, 1.0])
    X = np.array([[x0, x0 + [0.1, 0], x0 + [0, 0.1]]])
    F = ros(X[0])[None]
    NM.run(X, F, ros, -BIG, BIG, 400)
    assert np.allclose(X[0, 0], [1.0, 1.0], atol=1e-4)
    c = np.array([0.3, -1.0, 2.0, 0.5, -0.7])
    q = sq(c)
    rng = np.random.default_rng(0)
    X = rng.normal(0, 1, (3, 6, 5))
    F = np.stack([q(X[m]) for m in range(3)])
    NM.run(X, F, q, np.full(5, -1e9), np.full(5, 1e9), 1500)
    assert np.allclose(X[:, 0], c[None], atol=1e-5)


def test_prior_box():
    f = sq([2.0, 2.0])        # minimum outside the box [-1, 1]^2
    X = np.array([[[0.0, 0.0], [0.5, 0.0], [0.0, 0.5]]])
    F = f(X[0])[None]
    NM.run(X, F, f, np.full(2, -1.0), np.full(2, 1.0), 200)
    assert np.all(X <= 1.0) and np.all(X >= -1.0)
    assert np.allclose(X[0, 0], [1.0, 1.0], atol=1e-3)
