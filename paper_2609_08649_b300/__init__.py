"""Batched lens equation, multi-plane tracing and source-plane chi^2 with its gradient, on the
GPU (the method of LensFactory.jl: Sec. 2 lens maps and multi-plane recursion, Sec. 3 chi^2).

The compute path is the C-ABI library `liblf.so` (CUDA kernels for sm_103a, built in-tree
by `build.py`; declarations and argument conventions in `include/lf.h`).  This package is its
Python binding and imports nothing on its own:

  api        calls on torch CUDA tensors, on the current stream:
               deflect_grid, jacobian_grid, jacobian_points  -- alpha, kappa, gamma, mu maps
               jacobian_grid_host                            -- the same into pinned host memory
               trace_multiplane                              -- beta and A through several planes
               find_images, find_images_multiplane           -- lens-equation solver
               Plan(...).chi2 / chi2_grad / chi2_img         -- batched chi^2, its gradient,
                                                                the image-plane chi^2
               Plan(...).aies_run / mh_run / nm_run          -- samplers and optimiser
               chi2(theta, plan)                             -- autograd wrapper
  model      lens planes and clusters from physical descriptions (DevicePlane, ClusterInput)
  workloads  seeded synthetic models, catalogues and parameter samples
  _lib       the ctypes structs and signatures of the library

Precision tiers ("fp64", "mixed", "ff") select the kernels' arithmetic.  There is no CPU
fallback: importing `api` without the built library raises.
"""
