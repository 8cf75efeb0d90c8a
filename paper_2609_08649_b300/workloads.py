"""Seeded synthetic workloads for the batched lens-equation / chi^2 path.

This module only draws random numbers and writes down model descriptions in
*physical* units (arcsec, km/s, kpc, degrees, solar masses, redshifts).  It
holds none of the lensing arithmetic: no distances, no unit conversion to
lensing strengths, no deflections.  Both the CUDA path (through the package's
host-side builders) and the FP64 oracle consume these descriptions and convert
them with their own code.

The shapes follow the paper's cluster workloads (Sec. 4-5: 49-242 images,
62-340 members, 2-5 images per family, sigma_pos 0.1-0.5 arcsec, members as
pseudo-Jaffe galaxies on the luminosity scaling relations of Eq. scaling) since
the paper's own catalogues are not public inputs here.

Component kinds (shared numeric codes): 1 SIE (cored isothermal ellipsoid),
2 DPIE (pseudo-Jaffe / dPIE ellipsoid), 3 NFW (spherical), 4 SHEAR, 5 MPOLE3 (third-order
multipole with a theta^2 potential), 6 ENFW (elliptical NFW as a sum of cored steep ellipsoids).
"""
from __future__ import annotations

import dataclasses
import os
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SIE, DPIE, NFW, SHEAR, MPOLE3, ENFW = 1, 2, 3, 4, 5, 6

# Parameter-field codes of a component and transforms applied to a sampled
# parameter before it lands in that field (shared by the param map of both sides).
FIELDS = ("x", "y", "b", "eps", "pa", "core", "cut")
F_X, F_Y, F_B, F_EPS, F_PA, F_CORE, F_CUT = range(7)
SCALING_SLOTS = ("b_star", "core_star", "cut_star", "lam", "beta", "alpha")
XF_IDENT, XF_VDISP, XF_DEG, XF_KPC = 0, 1, 2, 3


@dataclass
class PhysComp:
    """One analytic component in physical units.

    kind: SIE/DPIE: x, y [arcsec], vdisp [km/s] (or theta_e [arcsec], the
    area-equivalent Einstein radius at source redshift z_ref), eps, pa_deg,
    core_kpc / core_arcsec, cut_kpc.  NFW: m200 [Msun], conc.  ENFW: m200, conc (or kappa_s,
    theta_s [arcsec]), eps, pa_deg.  SHEAR: gamma, pa_deg.
    """
    kind: int
    x: float = 0.0
    y: float = 0.0
    vdisp: Optional[float] = None
    theta_e: Optional[float] = None
    z_ref: Optional[float] = None
    eps: float = 0.0
    pa_deg: float = 0.0
    core_kpc: Optional[float] = None
    core_arcsec: Optional[float] = None
    cut_kpc: Optional[float] = None
    m200: Optional[float] = None
    conc: Optional[float] = None
    gamma: Optional[float] = None
    amp: Optional[float] = None      # MPOLE3 amplitude A of psi = A theta^2 cos 3(phi - pa)
    kappa_s: Optional[float] = None  # ENFW given in lensing units (instead of m200, conc)
    theta_s: Optional[float] = None  # ENFW scale radius [arcsec]


@dataclass
class PhysMembers:
    """Cluster members on the scaling relations of Eq. scaling (spherical PJE)."""
    x: np.ndarray
    y: np.ndarray
    log_l: np.ndarray            # log10(L/L*)
    vstar: float                 # km/s
    core_star_kpc: float
    cut_star_kpc: float
    lam: float
    beta: float
    alpha: float


@dataclass
class PhysPlane:
    z: float
    comps: List[PhysComp]
    members: Optional[PhysMembers] = None


@dataclass
class Grid:
    """Pixel-centre grid, row-major with y the slow index."""
    x0: float
    y0: float
    dx: float
    dy: float
    nx: int
    ny: int


@dataclass
class Cosmo:
    H0: float = 70.0
    Om: float = 0.3


@dataclass
class ParamSpec:
    """One sampled parameter: its target and its jitter recipe."""
    comp: int            # index into the concatenated components, -1 = scaling slot
    field: int           # F_* for components, index into SCALING_SLOTS for -1
    xform: int           # XF_*
    base: float          # central value in the parameter's own (physical) unit
    jitter: float        # standard deviation of the Gaussian jitter
    relative: bool       # jitter relative to base


@dataclass
class Workload:
    name: str
    cosmo: Cosmo
    planes: List[PhysPlane]
    z_s: Optional[float] = None
    grid: Optional[Grid] = None
    params: List[ParamSpec] = field(default_factory=list)
    n_samples: int = 0
    seed: int = 0
    sigma_pos: float = 0.1
    family_sizes: List[int] = field(default_factory=list)
    family_zs: List[float] = field(default_factory=list)


def sample_thetas(wl: Workload, seed: int) -> np.ndarray:
    """(S, P) float64 parameter samples: base + Gaussian jitter (physical units)."""
    rng = np.random.default_rng(seed)
    P = len(wl.params)
    base = np.array([p.base for p in wl.params], dtype=np.float64)
    sd = np.array([p.jitter * (abs(p.base) if p.relative else 1.0) for p in wl.params])
    z = rng.standard_normal((wl.n_samples, P))
    th = base[None, :] + sd[None, :] * z
    th[0] = base          # sample 0 is the unjittered model
    return th


def _cluster_halos(x2=25.0, y2=-15.0):
    return [
        PhysComp(DPIE, 0.0, 0.0, vdisp=900.0, eps=0.2, pa_deg=30.0, core_kpc=30.0, cut_kpc=1000.0),
        PhysComp(DPIE, x2, y2, vdisp=600.0, eps=0.3, pa_deg=-20.0, core_kpc=15.0, cut_kpc=1000.0),
    ]


def _members(rng, n, half=75.0, vstar=250.0):
    return PhysMembers(x=rng.uniform(-half, half, n), y=rng.uniform(-half, half, n),
                       log_l=rng.uniform(-2.0, 1.0, n), vstar=vstar, core_star_kpc=0.15,
                       cut_star_kpc=45.0, lam=0.25, beta=0.5, alpha=0.5)


def galaxy_c0() -> Workload:
    """Plain single-plane galaxy lens: SIE + external shear, 64x64 grid at 0.1"."""
    q = 0.7
    eps = (1 - q) / (1 + q)
    comps = [PhysComp(SIE, 0.0, 0.0, theta_e=1.2, z_ref=2.0, eps=eps, pa_deg=30.0, core_arcsec=0.05),
             PhysComp(SHEAR, gamma=0.05, z_ref=2.0, pa_deg=0.0)]
    return Workload("galaxy_sie_shear_64", Cosmo(), [PhysPlane(0.5, comps)], z_s=2.0,
                    grid=Grid(-3.15, -3.15, 0.1, 0.1, 64, 64), seed=0, sigma_pos=0.05,
                    family_sizes=[4] * 5, family_zs=[2.0] * 5)


def cluster_c1(n_grid: int = 4096, seed: int = 1) -> Workload:
    """Cluster single plane: 2 elliptical dPIE halos + 300 PJE members; grid maps at z_s=9."""
    rng = np.random.default_rng(seed)
    pl = PhysPlane(0.5, _cluster_halos(), _members(rng, 300))
    d = 0.04 * 4096 / n_grid
    x0 = -(n_grid - 1) / 2 * d
    return Workload(f"cluster_dpie302_grid{n_grid}", Cosmo(), [pl], z_s=9.0,
                    grid=Grid(x0, x0, d, d, n_grid, n_grid), seed=seed)


def _halo_params(ci: int, h: PhysComp) -> List[ParamSpec]:
    return [ParamSpec(ci, F_X, XF_IDENT, h.x, 0.3, False),
            ParamSpec(ci, F_Y, XF_IDENT, h.y, 0.3, False),
            ParamSpec(ci, F_B, XF_VDISP, h.vdisp, 0.01, True),
            ParamSpec(ci, F_EPS, XF_IDENT, h.eps, 0.02, False),
            ParamSpec(ci, F_PA, XF_DEG, h.pa_deg, 2.0, False),
            ParamSpec(ci, F_CORE, XF_KPC, h.core_kpc, 0.01, True),
            ParamSpec(ci, F_CUT, XF_KPC, h.cut_kpc, 0.01, True)]


def cluster_c2(n_samples: int = 4096, seed: int = 2) -> Workload:
    """Batched source-plane chi^2: C1's model + shear, 18 jittered parameters,
    60 families (15x2 + 20x3 + 15x4 + 10x5 = 200 images), z_s ~ U[1, 6]."""
    c1 = cluster_c1()
    comps = _cluster_halos() + [PhysComp(SHEAR, gamma=0.05, pa_deg=0.0)]
    pl = PhysPlane(0.5, comps, c1.planes[0].members)
    params = _halo_params(0, comps[0]) + _halo_params(1, comps[1]) + [
        ParamSpec(2, F_B, XF_IDENT, 0.05, 0.005, False),
        ParamSpec(2, F_PA, XF_DEG, 0.0, 5.0, False),
        ParamSpec(-1, 0, XF_VDISP, 250.0, 0.01, True),
        ParamSpec(-1, 2, XF_KPC, 45.0, 0.01, True)]
    rng = np.random.default_rng(seed + 1000)
    sizes = [2] * 15 + [3] * 20 + [4] * 15 + [5] * 10
    zs = list(rng.uniform(1.0, 6.0, len(sizes)))
    return Workload("cluster_chi2_4096x200", Cosmo(), [pl], params=params, n_samples=n_samples,
                    seed=seed, sigma_pos=0.1, family_sizes=sizes, family_zs=zs)


def cluster_c2_mpole(n_samples: int = 4096, seed: int = 2) -> Workload:
    """C2's model plus an m = 3 multipole at the centre (amplitude 0.004, orientation 10
    deg), both sampled: 20 parameters (the angular-structure term of the paper's Hera
    model)."""
    wl = cluster_c2(n_samples, seed)
    pl = wl.planes[0]
    comps = list(pl.comps) + [PhysComp(MPOLE3, 0.0, 0.0, amp=0.004, pa_deg=10.0)]
    k = len(comps) - 1
    params = list(wl.params) + [ParamSpec(k, F_B, XF_IDENT, 0.004, 0.0005, False),
                                ParamSpec(k, F_PA, XF_DEG, 10.0, 5.0, False)]
    return dataclasses.replace(wl, name="cluster_mpole_4096x200",
                               planes=[dataclasses.replace(pl, comps=comps)], params=params)


def cluster_c5_enfw(n_samples: int = 4096, seed: int = 6) -> Workload:
    """A cluster shaped like the paper's Hera model (Sec. 4.2): two elliptical NFW halos at
    fixed positions (kappa_s, theta_s of M200 = 1.2e15 and 3e14 Msun with c = 5 and 6 at
    z = 0.5), external shear, an m = 3 multipole and C1's 300 members on the scaling
    relations.  14 sampled parameters as in that model: per halo kappa_s, theta_s, eps and pa;
    the shear's strength and angle; the multipole's amplitude and angle; v* and cut*.  The
    families are C2's (200 images)."""
    c1 = cluster_c1()
    halos = [PhysComp(ENFW, 0.0, 0.0, kappa_s=0.5618, theta_s=60.03, eps=0.2, pa_deg=30.0),
             PhysComp(ENFW, 25.0, -15.0, kappa_s=0.4486, theta_s=31.51, eps=0.3, pa_deg=-20.0)]
    comps = halos + [PhysComp(SHEAR, gamma=0.05, pa_deg=0.0),
                     PhysComp(MPOLE3, 0.0, 0.0, amp=0.004, pa_deg=10.0)]
    params = []
    for k, h in enumerate(halos):
        params += [ParamSpec(k, F_B, XF_IDENT, h.kappa_s, 0.01, True),
                   ParamSpec(k, F_CORE, XF_IDENT, h.theta_s, 0.01, True),
                   ParamSpec(k, F_EPS, XF_IDENT, h.eps, 0.02, False),
                   ParamSpec(k, F_PA, XF_DEG, h.pa_deg, 2.0, False)]
    params += [ParamSpec(2, F_B, XF_IDENT, 0.05, 0.005, False),
               ParamSpec(2, F_PA, XF_DEG, 0.0, 5.0, False),
               ParamSpec(3, F_B, XF_IDENT, 0.004, 0.0005, False),
               ParamSpec(3, F_PA, XF_DEG, 10.0, 5.0, False),
               ParamSpec(-1, 0, XF_VDISP, 250.0, 0.01, True),
               ParamSpec(-1, 2, XF_KPC, 45.0, 0.01, True)]
    c2 = cluster_c2()
    return Workload("cluster_enfw_4096x200", Cosmo(), [PhysPlane(0.5, comps, c1.planes[0].members)],
                    params=params, n_samples=n_samples, seed=seed, sigma_pos=0.1,
                    family_sizes=c2.family_sizes, family_zs=c2.family_zs)


def multiplane_c3(n_grid: int = 2048, n_samples: int = 1024, seed: int = 4) -> Workload:
    """Three planes (z = 0.39, 0.9, 2.1) traced to z_s = 4."""
    rng = np.random.default_rng(seed)
    p1 = PhysPlane(0.39, _cluster_halos(), _members(rng, 148))

    def los_plane(z, n_nfw, n_pje):
        comps = []
        for _ in range(n_nfw):
            comps.append(PhysComp(NFW, rng.uniform(-75, 75), rng.uniform(-75, 75),
                                  m200=10 ** rng.uniform(12.0, 14.0), conc=rng.uniform(4.0, 8.0)))
        for _ in range(n_pje):
            comps.append(PhysComp(DPIE, rng.uniform(-75, 75), rng.uniform(-75, 75),
                                  vdisp=rng.uniform(100.0, 250.0), eps=0.0, pa_deg=0.0,
                                  core_kpc=0.1, cut_kpc=rng.uniform(10.0, 50.0)))
        return PhysPlane(z, comps)

    p2 = los_plane(0.9, 30, 30)
    p3 = los_plane(2.1, 20, 20)
    d = 0.08 * 2048 / n_grid
    x0 = -(n_grid - 1) / 2 * d
    params = _halo_params(0, p1.comps[0]) + _halo_params(1, p1.comps[1]) + [
        ParamSpec(-1, 0, XF_VDISP, 250.0, 0.01, True),
        ParamSpec(-1, 2, XF_KPC, 45.0, 0.01, True)]
    return Workload(f"multiplane3_grid{n_grid}", Cosmo(), [p1, p2, p3], z_s=4.0,
                    grid=Grid(x0, x0, d, d, n_grid, n_grid), params=params,
                    n_samples=n_samples, seed=seed)


def multicluster_c4(n_clusters: int = 16, samples_per_cluster: int = 64, seed: int = 5):
    """16 clusters, 50-500 members, 20-300 images in 2-5 image families, 22 parameters."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_clusters):
        n_mem = int(rng.integers(50, 501))
        n_img = int(rng.integers(20, 301))
        sizes = []
        while sum(sizes) < n_img:
            sizes.append(int(rng.integers(2, 6)))
        excess = sum(sizes) - n_img
        while excess > 0:               # trim the last families (never below 2 images)
            for i in range(len(sizes) - 1, -1, -1):
                if excess > 0 and sizes[i] > 2:
                    sizes[i] -= 1
                    excess -= 1
            if all(s == 2 for s in sizes) and excess > 0:
                sizes.pop()
                excess -= 2
        zs = list(rng.uniform(1.0, 6.0, len(sizes)))
        x2, y2 = rng.uniform(-30, 30), rng.uniform(-30, 30)
        halos = _cluster_halos(x2, y2)
        halos[0].vdisp = float(rng.uniform(800.0, 1000.0))
        halos[1].vdisp = float(rng.uniform(500.0, 700.0))
        comps = halos + [PhysComp(SHEAR, gamma=float(rng.uniform(0.02, 0.08)),
                                  pa_deg=float(rng.uniform(-90, 90)))]
        mem = _members(rng, n_mem)
        mem.core_star_kpc = 0.3
        z_l = float(rng.uniform(0.3, 0.6))
        params = _halo_params(0, comps[0]) + _halo_params(1, comps[1]) + [
            ParamSpec(2, F_B, XF_IDENT, comps[2].gamma, 0.005, False),
            ParamSpec(2, F_PA, XF_DEG, comps[2].pa_deg, 5.0, False),
            ParamSpec(-1, 0, XF_VDISP, 250.0, 0.01, True),
            ParamSpec(-1, 1, XF_KPC, 0.3, 0.01, True),
            ParamSpec(-1, 2, XF_KPC, 45.0, 0.01, True),
            ParamSpec(-1, 3, XF_IDENT, 0.25, 0.005, False),
            ParamSpec(-1, 4, XF_IDENT, 0.5, 0.005, False),
            ParamSpec(-1, 5, XF_IDENT, 0.5, 0.005, False)]
        out.append(Workload(f"multicluster_{c}", Cosmo(), [PhysPlane(z_l, comps, mem)], params=params,
                            n_samples=samples_per_cluster, seed=seed * 100 + c, sigma_pos=0.1,
                            family_sizes=sizes, family_zs=zs))
    return out


def source_candidates(seed: int, n: int, radius: float, cx: float = 0.0, cy: float = 0.0) -> np.ndarray:
    """(n, 2) source positions uniform in a disk (candidates for forward ray-shooting)."""
    rng = np.random.default_rng(seed)
    r = radius * np.sqrt(rng.uniform(0, 1, n))
    t = rng.uniform(0, 2 * np.pi, n)
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], axis=1)


def position_noise(seed: int, n: int, sigma: float) -> np.ndarray:
    """(n, 2) Gaussian astrometric noise."""
    return np.random.default_rng(seed).normal(0.0, sigma, (n, 2))


def sampler_uniforms(seed: int, n_steps: int, n_walkers: int) -> np.ndarray:
    """(n_steps, n_walkers, 3) uniforms in [0, 1) for the stretch-move sampler
    (partner choice, stretch factor, acceptance)."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, (n_steps, n_walkers, 3))


def mh_randoms(seed: int, n_steps: int, n_chains: int, P: int):
    """(normals (n_steps, n_chains, P), uniforms (n_steps, n_chains)) for the random-walk
    Metropolis-Hastings chains."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_steps, n_chains, P)), rng.uniform(0.0, 1.0, (n_steps, n_chains))


def random_positions(seed: int, n: int, half: float) -> np.ndarray:
    """(n, 2) positions uniform in a square of half-width `half` (sampled-pixel checks)."""
    return np.random.default_rng(seed).uniform(-half, half, (n, 2))


F_ADIS = -2   # ParamSpec.comp of a family's sampled distance ratio (field = family index)


def with_free_adis(wl: Workload, families, base_adis, jitter=0.01) -> Workload:
    """A copy of `wl` whose listed families have their a_dis = D_ds/D_s sampled directly
    (free source redshifts), jittered by `jitter` around the caller's `base_adis` (one value
    per listed family, from the caller's cosmology)."""
    extra = [ParamSpec(F_ADIS, int(f), XF_IDENT, float(a), float(jitter), False)
             for f, a in zip(families, base_adis)]
    return dataclasses.replace(wl, params=list(wl.params) + extra)


def replace(obj, **kw):
    return dataclasses.replace(obj, **kw)


# ----------------------------------------------------------- stored catalogues -----
CATALOGUE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                             "tests", "golden", "catalogues")


@dataclass
class Catalogue:
    theta_obs: np.ndarray      # (N, 2) observed positions (noisy)
    theta_true: np.ndarray     # (N, 2) noise-free images
    fam_off: np.ndarray        # (F + 1,)
    fam_zs: np.ndarray         # (F,)


def load_aux(name: str, directory: str = CATALOGUE_DIR):
    """Flux and time-delay measurements of a catalogue's images written by
    oracle/make_catalogues.py: (mag, mag_err, td_days, td_err_days), NaN where absent."""
    a = np.loadtxt(os.path.join(directory, name + "_aux.txt"), ndmin=2)
    return a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy(), a[:, 3].copy()


def load_catalogue(name: str, directory: str = CATALOGUE_DIR) -> Catalogue:
    """Multiple-image catalogue written by oracle/make_catalogues.py (forward ray-shooting
    on the unjittered model); columns family, z_s, x_obs, y_obs, x_true, y_true."""
    a = np.loadtxt(os.path.join(directory, name + ".txt"), ndmin=2)
    fam = a[:, 0].astype(np.int64)
    F = int(fam.max()) + 1
    counts = np.bincount(fam, minlength=F)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    zs = np.array([a[fam == f, 1][0] for f in range(F)])
    return Catalogue(a[:, 2:4].copy(), a[:, 4:6].copy(), off, zs)
