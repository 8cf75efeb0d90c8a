"""Write the synthetic multiple-image catalogues used as chi^2 inputs.

TEST INFRASTRUCTURE: calls only the oracle and the seeded generators.  Run from the
repository root:  python -m oracle.make_catalogues [name ...]

Images are made by forward ray-shooting (the lens-equation solver of Sec. 2.3 on the
unjittered model, with Newton polish): a seeded candidate source is kept when it has at
least as many images as its family needs; the most magnified images are kept, and
seeded Gaussian astrometric noise of sigma_pos is added.  Output: one text file per
workload under tests/golden/catalogues/ with columns
    family  z_s  x_obs  y_obs  x_true  y_true
"""
import os
import sys

import numpy as np
import torch

from paper_2609_08649_b300 import workloads as W

from . import cosmology as cz
from . import images as im
from . import lensing as L
from . import model as om

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden", "catalogues")


def _alpha_fn(pl):
    def fn(tx, ty):
        out = L.plane_sum(pl, torch.as_tensor(np.asarray(tx, dtype=np.float64))[None],
                          torch.as_tensor(np.asarray(ty, dtype=np.float64))[None])
        return [o[0].numpy() for o in out]
    return fn


def _alpha_grid(fn, x0, h, n, chunk=1 << 18):
    xs = x0 + h * np.arange(n)
    TX, TY = np.meshgrid(xs, xs)
    tx, ty = TX.ravel(), TY.ravel()
    ax = np.empty_like(tx)
    ay = np.empty_like(ty)
    for i in range(0, tx.size, chunk):
        o = fn(tx[i:i + chunk], ty[i:i + chunk])
        ax[i:i + chunk], ay[i:i + chunk] = o[0], o[1]
    return ax.reshape(n, n), ay.reshape(n, n)


def make(wl, seed, src_radius, src_centre, half, h, drop_central=False):
    pl = om.build_planes(wl)[0]
    fn = _alpha_fn(pl)
    n = int(round(2 * half / h)) + 1
    agrid = _alpha_grid(fn, -half, h, n)
    z_l = wl.planes[0].z
    rows = []
    cands = W.source_candidates(seed, 100000, src_radius, *src_centre)
    ci = 0
    for f, (size, zs) in enumerate(zip(wl.family_sizes, wl.family_zs)):
        a = cz.a_dis(z_l, zs, wl.cosmo.H0, wl.cosmo.Om)
        while True:
            beta = cands[ci]
            ci += 1
            imgs = im.find_images(fn, a, beta, -half, -half, h, n, newton=True, alpha_grid=agrid)
            if len(imgs) == 0:
                continue
            o = fn(imgs[:, 0], imgs[:, 1])
            kappa, g1, g2, mu, det = L.jacobian_maps(*[torch.tensor(v) for v in o], a)
            mu = np.abs(mu.numpy())
            ok = np.isfinite(mu) & (np.abs(imgs).max(1) < half - 2 * h)
            imgs, mu = imgs[ok], mu[ok]
            order = np.argsort(-mu)
            if drop_central and len(imgs) >= 5:
                order = order[:-1]
            if len(order) >= size:
                chosen = imgs[order[:size]]
                break
        noise = W.position_noise(seed * 1000 + f, size, wl.sigma_pos)
        for k in range(size):
            rows.append((f, zs, chosen[k, 0] + noise[k, 0], chosen[k, 1] + noise[k, 1], chosen[k, 0], chosen[k, 1]))
    return np.array(rows)


def write(name, rows, header):
    os.makedirs(OUT, exist_ok=True)
    np.savetxt(os.path.join(OUT, name + ".txt"), rows, fmt=["%d", "%.10f", "%.12f", "%.12f", "%.12f", "%.12f"],
               header=header + "\nfamily z_s x_obs y_obs x_true y_true")
    print("wrote", name, rows.shape)


def make_aux(wl, cat, seed, flux_fams, td_fams, sig_m=0.1, sig_t=2.0):
    """Flux and time-delay measurements of a catalogue's noise-free images on the unjittered
    model (Sec. 3.2-3.3): m_i = m_src - 2.5 log10|mu_i| + N(0, sig_m) with m_src ~ U[24, 27]
    per family, and delays T_i - T_first + N(0, sig_t) days with T the arrival time of
    Eq. time_delay about the family's true source; NaN where a family has no measurement."""
    pl = om.build_planes(wl)[0]
    t = torch.tensor(cat.theta_true)
    ax, ay, pxx, pyy, pxy = [o[0] for o in L.plane_sum(pl, t[None, :, 0], t[None, :, 1])]
    psi = L.plane_potential(pl, t[None, :, 0], t[None, :, 1])[0]
    adis = om.single_plane_adis(wl, cat.fam_zs)
    K0 = cz.td_scale(wl.planes[0].z, wl.cosmo.H0, wl.cosmo.Om)
    rng = np.random.default_rng(seed)
    n = len(cat.theta_true)
    mag, me, td, te = (np.full(n, np.nan) for _ in range(4))
    for f in range(len(cat.fam_off) - 1):
        i0, i1 = cat.fam_off[f], cat.fam_off[f + 1]
        a = adis[f]
        m_src = rng.uniform(24.0, 27.0)
        det = (1 - a * pxx[i0:i1]) * (1 - a * pyy[i0:i1]) - (a * pxy[i0:i1]) ** 2
        bx = t[i0:i1, 0] - a * ax[i0:i1]
        by = t[i0:i1, 1] - a * ay[i0:i1]
        T = (K0 / a) * (0.5 * ((t[i0:i1, 0] - bx) ** 2 + (t[i0:i1, 1] - by) ** 2) - a * psi[i0:i1])
        nm, nt = rng.normal(0, sig_m, i1 - i0), rng.normal(0, sig_t, i1 - i0)
        if f in flux_fams:
            mag[i0:i1] = m_src + 2.5 * np.log10(np.abs(det.numpy())) + nm
            me[i0:i1] = sig_m
        if f in td_fams:
            td[i0:i1] = (T - T[0]).numpy() + nt
            te[i0:i1] = sig_t
    return np.stack([mag, me, td, te], 1)


def main(names):
    if not names or "galaxy" in names:
        wl = W.galaxy_c0()
        rows = make(wl, seed=10, src_radius=0.12, src_centre=(0.0, 0.0), half=2.5, h=0.01, drop_central=True)
        write("galaxy_sie_shear", rows, "C0-shaped galaxy lens: 5 sources x 4 images, sigma_pos = 0.05")
    if not names or "cluster" in names:
        wl = W.cluster_c2()
        rows = make(wl, seed=11, src_radius=12.0, src_centre=(4.0, -3.0), half=80.0, h=0.1)
        write("cluster_200", rows, "C2-shaped cluster: 60 families / 200 images, z_s ~ U[1, 6], sigma_pos = 0.1")
    if not names or "cluster_aux" in names:
        wl = W.cluster_c2()
        cat = W.load_catalogue("cluster_200", OUT)
        rows = make_aux(wl, cat, seed=12, flux_fams=range(0, 30), td_fams=range(40, 55))
        np.savetxt(os.path.join(OUT, "cluster_200_aux.txt"), rows, fmt="%.10f",
                   header="flux and time-delay measurements of cluster_200 (rows = its images)\n"
                          "mag mag_err td_days td_err_days (nan: no measurement)")
        print("wrote cluster_200_aux", rows.shape)
    if not names or "multicluster" in names:
        for c, wl in enumerate(W.multicluster_c4()):
            x2, y2 = wl.planes[0].comps[1].x, wl.planes[0].comps[1].y
            rows = make(wl, seed=100 + c, src_radius=12.0, src_centre=(0.3 * x2, 0.3 * y2), half=80.0, h=0.2)
            write(f"multicluster_{c:02d}", rows, f"C4 cluster {c}: {len(wl.family_sizes)} families")


if __name__ == "__main__":
    torch.set_num_threads(os.cpu_count() or 1)
    main(sys.argv[1:])
