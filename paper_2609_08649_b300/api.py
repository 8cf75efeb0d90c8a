"""PyTorch-facing calls of the C ABI: device tensors in, device tensors out, on the
current CUDA stream.  Every computation runs in the library's kernels."""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from .model import DevicePlane, grid_struct

PRECISION = {"fp64": L.LF_FP64, "mixed": L.LF_MIXED, "ff": L.LF_FF}


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev64(t: torch.Tensor, name: str, inplace=False) -> torch.Tensor:
    """A float64 CUDA tensor for the C ABI (which reads raw double pointers): other dtypes or
    host tensors are rejected rather than reinterpreted."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if inplace and not t.is_contiguous():
        raise ValueError(f"{name} is updated in place and must be contiguous")
    return t.contiguous()


def _prec(p):
    return PRECISION[p] if isinstance(p, str) else int(p)


def deflect_grid(plane: DevicePlane, grid, precision="mixed"):
    n = grid.nx * grid.ny
    ax = torch.empty(n, dtype=torch.float64, device="cuda")
    ay = torch.empty_like(ax)
    ps, gs = plane.c_struct(), grid_struct(grid)
    L.check(L.lib.lf_deflect_grid(C.byref(ps), C.byref(gs), _prec(precision), _ptr(ax), _ptr(ay),
                                  _stream()))
    return ax.view(grid.ny, grid.nx), ay.view(grid.ny, grid.nx)


def _jac_outputs(n, outputs):
    out = {}
    for k in outputs:
        dt = torch.float32 if k in ("kappa", "g1", "g2") else torch.float64
        out[k] = torch.empty(n, dtype=dt, device="cuda")
    return out


ALL_OUTPUTS = ("ax", "ay", "kappa", "g1", "g2", "mu")


def jacobian_grid(plane: DevicePlane, grid, a_dis, precision="mixed", outputs=ALL_OUTPUTS):
    n = grid.nx * grid.ny
    o = _jac_outputs(n, outputs)
    ps, gs = plane.c_struct(), grid_struct(grid)
    L.check(L.lib.lf_jacobian_grid(C.byref(ps), C.byref(gs), float(a_dis), _prec(precision),
                                   *[_ptr(o.get(k)) for k in ALL_OUTPUTS], _stream()))
    return {k: v.view(grid.ny, grid.nx) for k, v in o.items()}


def jacobian_grid_host_workspace(grid, bands=32) -> int:
    gs = grid_struct(grid)
    return int(L.lib.lf_jacobian_grid_host_workspace(C.byref(gs), int(bands)))


def jacobian_grid_host(plane: DevicePlane, grid, a_dis, precision="mixed", out=None, bands=32,
                       workspace=None, outputs=ALL_OUTPUTS):
    """The maps of jacobian_grid written to host tensors (`out`: name -> contiguous CPU tensor
    of ny*nx elements, float64 for ax, ay, mu and float32 for kappa, g1, g2, pinned for
    overlap; allocated pinned when None), computed in `bands` row bands whose device-to-host
    copies overlap the computation.  `workspace`: uint8 CUDA tensor of at least
    jacobian_grid_host_workspace(grid, bands) bytes (allocated when None).  Returns `out`
    after synchronising the current stream."""
    n = grid.nx * grid.ny
    if out is None:
        out = {k: torch.empty(n, dtype=torch.float32 if k in ("kappa", "g1", "g2") else torch.float64,
                              pin_memory=True) for k in outputs}
    for k, t in out.items():
        want = torch.float32 if k in ("kappa", "g1", "g2") else torch.float64
        if k not in ALL_OUTPUTS or t.is_cuda or t.dtype != want or not t.is_contiguous() or t.numel() != n:
            raise TypeError(f"out[{k!r}] must be a contiguous CPU {want} tensor of {n} elements")
    need = jacobian_grid_host_workspace(grid, bands)
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")
    ps, gs = plane.c_struct(), grid_struct(grid)
    L.check(L.lib.lf_jacobian_grid_host(C.byref(ps), C.byref(gs), float(a_dis), _prec(precision),
                                        *[_ptr(out.get(k)) for k in ALL_OUTPUTS], int(bands),
                                        _ptr(workspace), workspace.numel(), _stream()))
    torch.cuda.current_stream().synchronize()
    return out


def jacobian_points(plane: DevicePlane, theta: torch.Tensor, a_dis, precision="mixed",
                    outputs=ALL_OUTPUTS):
    theta = _dev64(theta, "theta")
    n = theta.shape[0]
    o = _jac_outputs(n, outputs)
    ps = plane.c_struct()
    L.check(L.lib.lf_jacobian_points(C.byref(ps), _ptr(theta), n, float(a_dis), _prec(precision),
                                     *[_ptr(o.get(k)) for k in ALL_OUTPUTS], _stream()))
    return o


def trace_multiplane(planes: Sequence[DevicePlane], ratios: np.ndarray, theta=None, grid=None,
                     precision="mixed"):
    """beta (n, 2) and A (n, 2, 2) traced through all planes (ratios: (n+1) x n table)."""
    arr = (L.lf_plane * len(planes))(*[p.c_struct() for p in planes])
    rat = np.ascontiguousarray(ratios, dtype=np.float64)
    if theta is not None:
        theta = _dev64(theta, "theta")
        n = theta.shape[0]
        gptr = None
    else:
        n = grid.nx * grid.ny
        gs = grid_struct(grid)
        gptr = C.byref(gs)
    beta = torch.empty(n, 2, dtype=torch.float64, device="cuda")
    A = torch.empty(n, 2, 2, dtype=torch.float64, device="cuda")
    L.check(L.lib.lf_trace_multiplane(arr, len(planes), rat.ctypes.data_as(C.c_void_p), _ptr(theta),
                                      n, gptr, _prec(precision), _ptr(beta), _ptr(A), _stream()))
    return beta, A


def find_images(plane: DevicePlane, grid, beta: torch.Tensor, a_src: torch.Tensor, max_img=8,
                polish_iters=0, precision="fp64", workspace: Optional[torch.Tensor] = None):
    """Images of n_src sources (beta (n_src, 2), a_src (n_src,)) on a vertex grid.
    Returns (img (n_src, max_img, 2), n_img (n_src,) int32); n_img = -1 flags an overflow of
    the candidate buffer.  `workspace` (uint8, from find_images_workspace) may be reused."""
    beta = _dev64(beta, "beta")
    a_src = _dev64(a_src, "a_src")
    n = beta.shape[0]
    need = find_images_workspace(grid, n, max_img)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
    img = torch.full((n, max_img, 2), float("nan"), dtype=torch.float64, device="cuda")
    n_img = torch.zeros(n, dtype=torch.int32, device="cuda")
    ps, gs = plane.c_struct(), grid_struct(grid)
    L.check(L.lib.lf_find_images(C.byref(ps), C.byref(gs), _prec(precision), _ptr(beta), _ptr(a_src),
                                 n, int(max_img), int(polish_iters), _ptr(workspace),
                                 workspace.numel(), _ptr(img), _ptr(n_img), _stream()))
    return img, n_img


def find_images_workspace(grid, n_src, max_img=8):
    return int(L.lib.lf_find_images_workspace(grid.nx, grid.ny, n_src, max_img))


def find_images_multiplane_workspace(grid, n_src, max_img=8):
    return int(L.lib.lf_find_images_multiplane_workspace(grid.nx, grid.ny, n_src, max_img))


def find_images_multiplane(planes: Sequence[DevicePlane], ratios: np.ndarray, grid, beta: torch.Tensor,
                           max_img=8, polish_iters=0, precision="fp64",
                           workspace: Optional[torch.Tensor] = None):
    """Images of n_src sources (beta (n_src, 2)) behind several planes, all at the source
    redshift of the ratios table ((n+1) x n, as for trace_multiplane).  Returns
    (img (n_src, max_img, 2), n_img (n_src,) int32) as find_images does."""
    beta = _dev64(beta, "beta")
    n = beta.shape[0]
    need = find_images_multiplane_workspace(grid, n, max_img)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
    img = torch.full((n, max_img, 2), float("nan"), dtype=torch.float64, device="cuda")
    n_img = torch.zeros(n, dtype=torch.int32, device="cuda")
    arr = (L.lf_plane * len(planes))(*[p.c_struct() for p in planes])
    rat = np.ascontiguousarray(ratios, dtype=np.float64)
    gs = grid_struct(grid)
    L.check(L.lib.lf_find_images_multiplane(arr, len(planes), rat.ctypes.data_as(C.c_void_p), C.byref(gs),
                                            _prec(precision), _ptr(beta), n, int(max_img), int(polish_iters),
                                            _ptr(workspace), workspace.numel(), _ptr(img), _ptr(n_img),
                                            _stream()))
    return img, n_img


def probe_alu():
    """Measured (FP32 FMA, MUFU rsqrt, FP64 FMA) operations per second of the current GPU."""
    r = [C.c_double() for _ in range(3)]
    L.check(L.lib.lf_probe_alu(*[C.byref(v) for v in r], _stream()))
    return tuple(v.value for v in r)


def probe_alu2():
    """Measured (FP32 FMA, packed f32x2 FMA in lane-operations, MUFU rsqrt, FP64 FMA) per second."""
    r = [C.c_double() for _ in range(4)]
    L.check(L.lib.lf_probe_alu2(*[C.byref(v) for v in r], _stream()))
    return tuple(v.value for v in r)


def device_error():
    L.check(L.lib.lf_device_error(_stream()))


# ------------------------------------------------------------------ chi^2 plans -----
class ClusterInput:
    """Everything one cluster of a plan needs, in lensing units (host arrays)."""

    def __init__(self, planes, arcsec_per_kpc, theta_obs, sinv, fam_off, fam_ratio,
                 p_comp, p_field, p_xform, ratios=None, aux=None, td_scale=0.0):
        """aux: optional (mag, mag_err, td, td_err) per image (NaN where absent; either pair
        may be None) for the flux and time-delay terms; td_scale from model.td_scale."""
        f64 = lambda v: None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        self.aux = tuple(f64(v) for v in aux) if aux is not None else (None, None, None, None)
        self.td_scale = float(td_scale)
        self.planes = planes
        self.apk = np.ascontiguousarray(arcsec_per_kpc, dtype=np.float64)
        self.theta_obs = np.ascontiguousarray(theta_obs, dtype=np.float64)
        self.sinv = np.ascontiguousarray(sinv, dtype=np.float64)
        self.fam_off = np.ascontiguousarray(fam_off, dtype=np.int32)
        self.fam_ratio = np.ascontiguousarray(fam_ratio, dtype=np.float64)
        self.p_comp = np.ascontiguousarray(p_comp, dtype=np.int32)
        self.p_field = np.ascontiguousarray(p_field, dtype=np.int32)
        self.p_xform = np.ascontiguousarray(p_xform, dtype=np.int32)
        n = len(planes)
        self.ratios = (np.ascontiguousarray(ratios, dtype=np.float64).reshape(-1)[: n * n]
                       if ratios is not None else None)

    def c_struct(self):
        self._planes_arr = (L.lf_plane * len(self.planes))(*[p.c_struct() for p in self.planes])
        c = L.lf_cluster()
        c.n_planes = len(self.planes)
        c.planes = C.cast(self._planes_arr, C.c_void_p)
        c.ratios = self.ratios.ctypes.data_as(C.c_void_p) if self.ratios is not None else None
        c.arcsec_per_kpc = self.apk.ctypes.data_as(C.c_void_p)
        im = L.lf_images()
        im.n_img = len(self.theta_obs)
        im.n_fam = len(self.fam_off) - 1
        im.theta_obs = self.theta_obs.ctypes.data_as(C.c_void_p)
        im.sinv = self.sinv.ctypes.data_as(C.c_void_p)
        im.fam_off = self.fam_off.ctypes.data_as(C.c_void_p)
        im.fam_ratio = self.fam_ratio.ctypes.data_as(C.c_void_p)
        ptr = lambda v: None if v is None else v.ctypes.data_as(C.c_void_p)
        im.mag, im.mag_err, im.td, im.td_err = (ptr(v) for v in self.aux)
        im.td_scale = self.td_scale
        c.images = im
        c.P = len(self.p_comp)
        c.p_comp = self.p_comp.ctypes.data_as(C.c_void_p)
        c.p_field = self.p_field.ctypes.data_as(C.c_void_p)
        c.p_xform = self.p_xform.ctypes.data_as(C.c_void_p)
        return c


FLAG_GRAPH, FLAG_AUTOTUNE = 1, 2


class Plan:
    """lf_plan_create / lf_chi2_batch / lf_chi2_grad_batch / lf_plan_destroy."""

    def __init__(self, clusters: Sequence[ClusterInput], max_samples, precision="mixed", flags=0):
        arr = (L.lf_cluster * len(clusters))(*[c.c_struct() for c in clusters])
        self._keep = clusters
        self.handle = C.c_void_p()
        self.n_clusters = len(clusters)
        self.P = len(clusters[0].p_comp)
        L.check(L.lib.lf_plan_create(C.byref(self.handle), arr, len(clusters), int(max_samples),
                                     _prec(precision), int(flags)))

    def chi2(self, theta: torch.Tensor, out: Optional[torch.Tensor] = None):
        theta = _dev64(theta, "theta")
        S = theta.shape[0]
        out = torch.empty(S, dtype=torch.float64, device="cuda") if out is None else _dev64(out, "out", True)
        L.check(L.lib.lf_chi2_batch(self.handle, _ptr(theta), S, _ptr(out), _stream()))
        return out

    def chi2_grad(self, theta: torch.Tensor, out=None, grad=None):
        theta = _dev64(theta, "theta")
        S = theta.shape[0]
        out = torch.empty(S, dtype=torch.float64, device="cuda") if out is None else _dev64(out, "out", True)
        grad = (torch.empty(S, self.P, dtype=torch.float64, device="cuda") if grad is None
                else _dev64(grad, "grad", True))
        L.check(L.lib.lf_chi2_grad_batch(self.handle, _ptr(theta), S, _ptr(out), _ptr(grad), _stream()))
        return out, grad

    def chi2_img(self, theta: torch.Tensor, iters=8):
        """Image-plane chi^2 and rms per sample (Newton model images)."""
        theta = _dev64(theta, "theta")
        S = theta.shape[0]
        out = torch.empty(S, dtype=torch.float64, device="cuda")
        rms = torch.empty(S, dtype=torch.float64, device="cuda")
        L.check(L.lib.lf_chi2_img_batch(self.handle, _ptr(theta), S, int(iters), _ptr(out), _ptr(rms),
                                        _stream()))
        return out, rms

    def aies_run(self, walkers: torch.Tensor, chi2: torch.Tensor, uniforms: torch.Tensor, a: float,
                 lo: torch.Tensor, hi: torch.Tensor, chain=False):
        """Stretch-move steps in place on (walkers, chi2); uniforms (n_steps, S, 3) on the device.
        Returns (n_accepted, chain or None)."""
        walkers = _dev64(walkers, "walkers", True)
        chi2 = _dev64(chi2, "chi2", True)
        uniforms, lo, hi = _dev64(uniforms, "uniforms"), _dev64(lo, "lo"), _dev64(hi, "hi")
        S = walkers.shape[0]
        n_steps = uniforms.shape[0]
        ch = torch.empty(n_steps, S, self.P, dtype=torch.float64, device="cuda") if chain else None
        acc = torch.zeros(1, dtype=torch.int64, device="cuda")
        L.check(L.lib.lf_aies_run(self.handle, _ptr(walkers), _ptr(chi2), S, n_steps,
                                  _ptr(uniforms), float(a), _ptr(lo), _ptr(hi), _ptr(ch), _ptr(acc),
                                  _stream()))
        return acc, ch

    def mh_run(self, chains: torch.Tensor, chi2: torch.Tensor, normals: torch.Tensor,
               uniforms: torch.Tensor, step: torch.Tensor, lo: torch.Tensor, hi: torch.Tensor,
               trace=False):
        """Random-walk Metropolis-Hastings steps in place on (chains, chi2); normals
        (n_steps, S, P), uniforms (n_steps, S) on the device.  Returns (n_accepted, trace)."""
        chains = _dev64(chains, "chains", True)
        chi2 = _dev64(chi2, "chi2", True)
        normals, uniforms = _dev64(normals, "normals"), _dev64(uniforms, "uniforms")
        step, lo, hi = _dev64(step, "step"), _dev64(lo, "lo"), _dev64(hi, "hi")
        S, n_steps = chains.shape[0], normals.shape[0]
        tr = torch.empty(n_steps, S, self.P, dtype=torch.float64, device="cuda") if trace else None
        acc = torch.zeros(1, dtype=torch.int64, device="cuda")
        L.check(L.lib.lf_mh_run(self.handle, _ptr(chains), _ptr(chi2), S, n_steps, _ptr(normals),
                                _ptr(uniforms), _ptr(step), _ptr(lo), _ptr(hi), _ptr(tr), _ptr(acc),
                                _stream()))
        return acc, tr

    def nm_run(self, simplex: torch.Tensor, fvals: torch.Tensor, n_iter: int, lo: torch.Tensor,
               hi: torch.Tensor):
        """Nelder-Mead iterations in place on simplex (M, P+1, P) and fvals (M, P+1) (the
        vertices' chi^2).  Returns the step counts (reflect, expand, outside contraction,
        inside contraction, shrink)."""
        simplex = _dev64(simplex, "simplex", True)
        fvals = _dev64(fvals, "fvals", True)
        lo, hi = _dev64(lo, "lo"), _dev64(hi, "hi")
        steps = torch.zeros(5, dtype=torch.int64, device="cuda")
        L.check(L.lib.lf_nm_run(self.handle, _ptr(simplex), _ptr(fvals), simplex.shape[0], int(n_iter),
                                _ptr(lo), _ptr(hi), _ptr(steps), _stream()))
        return steps

    def info(self):
        ks, blk, g = C.c_int32(), C.c_int32(), C.c_int32()
        L.check(L.lib.lf_plan_info(self.handle, C.byref(ks), C.byref(blk), C.byref(g)))
        return {"kslices": ks.value, "block": blk.value, "graph": bool(g.value)}

    def close(self):
        if self.handle:
            L.lib.lf_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Chi2Function(torch.autograd.Function):
    """chi^2 per sample with d chi^2 / d theta from the library's adjoint kernel.  The adjoint
    runs in forward (with the chi^2) only when theta needs a gradient; otherwise forward is one
    lf_chi2_batch call."""

    @staticmethod
    def forward(ctx, theta, plan):
        if not ctx.needs_input_grad[0]:
            ctx.save_for_backward(None)
            return plan.chi2(theta.detach())
        chi2, grad = plan.chi2_grad(theta.detach())
        ctx.save_for_backward(grad)
        return chi2

    @staticmethod
    def backward(ctx, g_out):
        (grad,) = ctx.saved_tensors
        return g_out[:, None] * grad, None


def chi2(theta, plan):
    return Chi2Function.apply(theta, plan)
