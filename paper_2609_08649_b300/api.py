"""PyTorch-facing calls of the C ABI: device tensors in, device tensors out, on the
current CUDA stream.  Every computation runs in the library's kernels."""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from .model import DevicePlane, grid_struct

PRECISION = {"fp64": L.LF_FP64, "mixed": L.LF_MIXED}


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


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


def jacobian_points(plane: DevicePlane, theta: torch.Tensor, a_dis, precision="mixed",
                    outputs=ALL_OUTPUTS):
    theta = theta.contiguous()
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
        theta = theta.contiguous()
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


def device_error():
    L.check(L.lib.lf_device_error(_stream()))
