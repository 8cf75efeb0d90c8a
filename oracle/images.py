"""Lens-equation solver (oracle, FP64).  TEST INFRASTRUCTURE ONLY.

Sec. 2.3: with f(theta) = beta - theta + a alpha(theta), the images are the common
zeros of f1 and f2.  Each component's zero contour is traced over an image-plane
grid by marching squares (linear interpolation along cell edges, saddle cells
resolved by the cell-centre value), and the images are the exact intersections of
pairs of piecewise-linear contour segments that share a cell.  The position error
of that construction is O(h^2) for a grid step h.  `newton=True` then polishes each
image with Newton steps on the lens equation (not part of the paper's solver).

`alpha_fn(tx, ty)` must return (ax, ay, pxx, pyy, pxy) as float64 numpy arrays.
"""
import numpy as np


def _edge_points(v, X, Y):
    """Zero crossings of a field on the 4 edges of one cell (corners in the order
    (0,0) (1,0) (1,1) (0,1)); returns dict edge -> point."""
    pts = {}
    for e in range(4):
        a, b = e, (e + 1) % 4
        va, vb = v[a], v[b]
        if (va > 0) != (vb > 0):
            t = va / (va - vb)
            pts[e] = (X[a] + t * (X[b] - X[a]), Y[a] + t * (Y[b] - Y[a]))
    return pts


def _segments(v, X, Y):
    pts = _edge_points(v, X, Y)
    if len(pts) == 2:
        e = sorted(pts)
        return [(pts[e[0]], pts[e[1]])]
    if len(pts) == 4:
        centre = 0.25 * sum(v)
        segs = []
        # isolate each corner whose sign differs from the centre: it is cut off by
        # the segment joining its two adjacent edges (edges k-1 and k for corner k)
        for k in range(4):
            if (v[k] > 0) != (centre > 0):
                segs.append((pts[(k - 1) % 4], pts[k]))
        return segs
    return []


def _intersect(p, p2, q, q2):
    r = (p2[0] - p[0], p2[1] - p[1])
    s = (q2[0] - q[0], q2[1] - q[1])
    den = r[0] * s[1] - r[1] * s[0]
    if den == 0.0:
        return None
    qp = (q[0] - p[0], q[1] - p[1])
    t = (qp[0] * s[1] - qp[1] * s[0]) / den
    u = (qp[0] * r[1] - qp[1] * r[0]) / den
    if -1e-12 <= t <= 1 + 1e-12 and -1e-12 <= u <= 1 + 1e-12:
        return (p[0] + t * r[0], p[1] + t * r[1])
    return None


def find_images(alpha_fn, a, beta_s, x0, y0, h, n, newton=False, alpha_grid=None):
    """Images of source beta_s on an n x n vertex grid (x0 + i h, y0 + j h).

    alpha_grid: optional precomputed (ax, ay) on the vertices (n, n) [y, x] to reuse the
    deflection field for many sources at one a."""
    xs = x0 + h * np.arange(n)
    ys = y0 + h * np.arange(n)
    TX, TY = np.meshgrid(xs, ys)
    if alpha_grid is None:
        ax, ay = alpha_fn(TX.ravel(), TY.ravel())[:2]
        ax, ay = ax.reshape(n, n), ay.reshape(n, n)
    else:
        ax, ay = alpha_grid
    f1 = beta_s[0] - TX + a * ax
    f2 = beta_s[1] - TY + a * ay
    s1 = f1 > 0
    s2 = f2 > 0
    ch1 = (s1[:-1, :-1] != s1[:-1, 1:]) | (s1[:-1, :-1] != s1[1:, :-1]) | (s1[:-1, :-1] != s1[1:, 1:])
    ch2 = (s2[:-1, :-1] != s2[:-1, 1:]) | (s2[:-1, :-1] != s2[1:, :-1]) | (s2[:-1, :-1] != s2[1:, 1:])
    found = []
    for j, i in zip(*np.nonzero(ch1 & ch2)):
        X = [xs[i], xs[i + 1], xs[i + 1], xs[i]]
        Y = [ys[j], ys[j], ys[j + 1], ys[j + 1]]
        v1 = [f1[j, i], f1[j, i + 1], f1[j + 1, i + 1], f1[j + 1, i]]
        v2 = [f2[j, i], f2[j, i + 1], f2[j + 1, i + 1], f2[j + 1, i]]
        for sa in _segments(v1, X, Y):
            for sb in _segments(v2, X, Y):
                p = _intersect(sa[0], sa[1], sb[0], sb[1])
                if p is not None:
                    found.append(p)
    imgs = []
    for p in found:
        if all((p[0] - q[0]) ** 2 + (p[1] - q[1]) ** 2 > (1e-6 * h) ** 2 for q in imgs):
            imgs.append(p)
    imgs = np.array(imgs, dtype=np.float64).reshape(-1, 2)
    if newton and len(imgs):
        imgs = np.array([polish(alpha_fn, a, beta_s, p) for p in imgs])
        keep = []
        for p in imgs:
            if np.all(np.isfinite(p)) and all(np.hypot(*(p - q)) > 1e-7 for q in keep):
                keep.append(p)
        imgs = np.array(keep).reshape(-1, 2)
    return imgs


def polish(alpha_fn, a, beta_s, p, tol=1e-12, iters=50):
    """Newton iteration theta <- theta - A^-1 (beta(theta) - beta_s)."""
    th = np.array(p, dtype=np.float64)
    for _ in range(iters):
        ax, ay, pxx, pyy, pxy = [float(np.asarray(v).ravel()[0]) for v in
                                 alpha_fn(np.array([th[0]]), np.array([th[1]]))]
        r = np.array([th[0] - a * ax - beta_s[0], th[1] - a * ay - beta_s[1]])
        if np.hypot(*r) < tol:
            break
        A = np.array([[1 - a * pxx, -a * pxy], [-a * pxy, 1 - a * pyy]])
        th = th - np.linalg.solve(A, r)
    return th
