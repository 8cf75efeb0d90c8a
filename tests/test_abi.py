"""The C-ABI library loads on a machine without a GPU and exports every symbol that
include/lf.h declares; host helpers agree with the oracle; argument validation returns
LF_EINVAL before any launch."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lf_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2609_08649_b300 import _lib as L
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L.lib, s), s
    assert set(L.EXPORTS) == set(syms)


def test_host_distances_match_oracle():
    from oracle import cosmology as cz
    from paper_2609_08649_b300 import _lib as L
    for z1, z2 in [(0.0, 0.5), (0.5, 2.0), (0.39, 4.0), (2.1, 9.0)]:
        assert abs(L.lib.lf_angular_distance(70.0, 0.3, z1, z2) - cz.d_ang(z1, z2)) < 1e-9
    assert abs(L.lib.lf_adis(70.0, 0.3, 0.5, 2.0) - 0.6353908) < 1e-7
    assert abs(L.lib.lf_b_from_vdisp(900.0) - 23.3603) < 1e-4
    assert L.lib.lf_adis(70.0, 0.3, 0.5, 0.4) == 0.0


def test_nfw_normalisation_matches_oracle():
    from oracle import model as om
    from paper_2609_08649_b300 import model as pm
    from paper_2609_08649_b300 import workloads as W
    ks, ts = pm.nfw_params(W.Cosmo(), 0.9, 3e13, 6.0)
    ks0, ts0 = om.nfw_lensing(3e13, 6.0, 0.9)
    assert abs(ks / ks0 - 1) < 1e-9 and abs(ts / ts0 - 1) < 1e-9


def test_invalid_arguments_are_rejected_before_launch():
    from paper_2609_08649_b300 import _lib as L
    g = L.lf_grid(0, 0, 0.1, 0.1, 4, 4)
    p = L.lf_plane()
    p.n_comp, p.n_mem = 1, 0
    p.comp = None
    st = L.lib.lf_deflect_grid(C.byref(p), C.byref(g), L.LF_MIXED, C.c_void_p(16), C.c_void_p(16), None)
    assert st == L.LF_EINVAL and b"NULL" in L.lib.lf_last_error()
    p.comp = C.c_void_p(8)      # misaligned
    st = L.lib.lf_deflect_grid(C.byref(p), C.byref(g), L.LF_MIXED, C.c_void_p(16), C.c_void_p(16), None)
    assert st == L.LF_EINVAL and b"aligned" in L.lib.lf_last_error()
    p.n_comp = 0
    st = L.lib.lf_jacobian_grid(C.byref(p), C.byref(g), 1.5, L.LF_MIXED, None, None, None, None, None, None, None)
    assert st == L.LF_EINVAL
    bad = L.lf_grid(0, 0, 0.1, 0.1, 0, 4)
    st = L.lib.lf_deflect_grid(C.byref(p), C.byref(bad), L.LF_MIXED, C.c_void_p(16), C.c_void_p(16), None)
    assert st == L.LF_EINVAL
    st = L.lib.lf_deflect_grid(C.byref(p), C.byref(g), 7, C.c_void_p(16), C.c_void_p(16), None)
    assert st == L.LF_EINVAL
    st = L.lib.lf_trace_multiplane(C.byref(p), 9, None, None, 0, None, L.LF_MIXED, None, None, None)
    assert st == L.LF_EINVAL


def test_python_layer_rejects_tensors_the_abi_would_misread():
    """The C ABI reads raw double pointers on the device: float32 or host tensors must be
    refused by the binding, not reinterpreted."""
    import torch
    from paper_2609_08649_b300 import api
    with pytest.raises(TypeError):
        api._dev64(torch.zeros(3, dtype=torch.float32), "x")
    with pytest.raises(TypeError):
        api._dev64(torch.zeros(3, dtype=torch.float64), "x")   # host memory
    with pytest.raises(TypeError):
        api._dev64([1.0, 2.0], "x")


def test_host_maps_workspace_and_validation():
    """lf_jacobian_grid_host: the workspace size follows the band split (two slots of
    ceil(ny / bands) rows, 36 bytes a pixel rounded to 256 per map), and invalid arguments
    are refused before any CUDA call."""
    from paper_2609_08649_b300 import _lib as L
    up = lambda b: (b + 255) // 256 * 256
    g = L.lf_grid(0, 0, 0.1, 0.1, 100, 263)
    for bands, rows in [(1, 263), (5, 64), (16, 32), (263, 16), (1000, 16)]:   # multiples of 16 rows
        px = 100 * rows
        assert L.lib.lf_jacobian_grid_host_workspace(C.byref(g), bands) == 2 * (3 * up(8 * px) + 3 * up(4 * px))
    assert L.lib.lf_jacobian_grid_host_workspace(C.byref(g), 0) == 0
    assert L.lib.lf_jacobian_grid_host_workspace(None, 4) == 0
    p = L.lf_plane()
    p.n_comp, p.n_mem = 0, 0
    need = L.lib.lf_jacobian_grid_host_workspace(C.byref(g), 4)
    host = C.c_void_p(64)
    call = lambda grid, a, prec, bands, ws, nbytes: L.lib.lf_jacobian_grid_host(
        C.byref(p), grid, a, prec, host, None, None, None, None, None, bands, ws, nbytes, None)
    assert call(C.byref(g), 0.5, L.LF_MIXED, 0, C.c_void_p(256), need) == L.LF_EINVAL           # bands
    assert b"bands" in L.lib.lf_last_error()
    assert call(C.byref(g), 0.5, L.LF_MIXED, 4, None, need) == L.LF_EINVAL                       # no workspace
    assert call(C.byref(g), 0.5, L.LF_MIXED, 4, C.c_void_p(256), need - 1) == L.LF_EINVAL        # undersized
    assert b"workspace" in L.lib.lf_last_error()
    assert call(C.byref(g), 0.5, L.LF_MIXED, 4, C.c_void_p(128), need) == L.LF_EINVAL            # misaligned
    assert call(C.byref(g), 1.5, L.LF_MIXED, 4, C.c_void_p(256), need) == L.LF_EINVAL            # a_dis
    assert call(C.byref(g), 0.5, 7, 4, C.c_void_p(256), need) == L.LF_EINVAL                     # precision
    bad = L.lf_grid(0, 0, 0.1, 0.1, 100, 0)
    assert call(C.byref(bad), 0.5, L.LF_MIXED, 4, C.c_void_p(256), need) == L.LF_EINVAL          # grid


def test_host_maps_binding_rejects_wrong_outputs():
    """api.jacobian_grid_host checks the host tensors before any CUDA call: dtype, device,
    size, contiguity and the output names."""
    import torch
    from paper_2609_08649_b300 import api
    from paper_2609_08649_b300 import workloads as W
    grid = W.Grid(0.0, 0.0, 0.1, 0.1, 8, 4)
    n = 32
    bad = [{"ax": torch.zeros(n, dtype=torch.float32)},                 # alpha is FP64
           {"kappa": torch.zeros(n, dtype=torch.float64)},              # kappa is FP32
           {"mu": torch.zeros(n - 1, dtype=torch.float64)},             # wrong size
           {"ay": torch.zeros(2 * n, dtype=torch.float64)[::2]},        # not contiguous
           {"beta": torch.zeros(n, dtype=torch.float64)}]               # not a map
    for out in bad:
        with pytest.raises(TypeError):
            api.jacobian_grid_host(None, grid, 0.5, "mixed", out=out)


def test_host_unit_conversions_match_the_oracle():
    """lf_comp_from_physical, lf_scaling_from_physical and lf_multiplane_ratios (host-only set-up
    helpers) against the oracle's own conversions, on every component kind of the workloads."""
    import numpy as np
    from oracle import cosmology as cz
    from oracle import lensing as OLL
    from oracle import model as OM
    from paper_2609_08649_b300 import _lib as L
    from paper_2609_08649_b300 import model as PM
    from paper_2609_08649_b300 import workloads as W
    wls = [W.galaxy_c0(), W.cluster_c2(n_samples=1), W.multiplane_c3(n_grid=8, n_samples=1),
           W.cluster_c5_enfw(n_samples=1), W.cluster_c2_mpole(n_samples=1)]
    kinds = set()
    for wl in wls:
        for pl in wl.planes:
            for c in pl.comps:
                a = np.array(PM.comp_record(c, pl.z, wl.cosmo)[:7])
                b = np.array(OM.comp_fields(c, pl.z, wl.cosmo))
                assert np.all(np.abs(a - b) <= 1e-13 * np.maximum(1, np.abs(b))), (c.kind, a, b)
                kinds.add(c.kind)
            if pl.members is not None:
                m = pl.members
                sc = PM.device_plane(pl, wl.cosmo, device="cpu").scaling
                apk = cz.arcsec_per_kpc(pl.z)
                ref = (OLL.b_from_vdisp(m.vstar), m.core_star_kpc * apk, m.cut_star_kpc * apk, m.lam, m.beta, m.alpha)
                assert np.allclose(sc, ref, rtol=1e-13, atol=0)
    assert kinds >= {W.SIE, W.DPIE, W.NFW, W.SHEAR, W.MPOLE3, W.ENFW}
    zs = [0.39, 0.9, 2.1]
    r = PM.multiplane_ratios(W.Cosmo(), zs, 4.0)
    r0, rs0 = cz.multiplane_ratios(zs, 4.0)
    assert np.allclose(r[:3], np.array(r0), rtol=1e-13, atol=0) and np.allclose(r[3], rs0, rtol=1e-13, atol=0)
    bad = L.lf_phys_comp()
    bad.kind = W.SIE
    for f in ("vdisp", "theta_e", "z_ref", "core_kpc", "core_arcsec", "cut_kpc"):
        setattr(bad, f, float("nan"))
    out = L.lf_comp()
    assert L.lib.lf_comp_from_physical(C.byref(bad), 70.0, 0.3, 0.5, C.byref(out)) == L.LF_EINVAL
