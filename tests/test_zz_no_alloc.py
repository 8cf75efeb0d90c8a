"""lf_chi2_batch_static: the allocation-free chi^2 entry point for callers that cannot call
cudaMalloc (GPU memory owned by another allocator, hosts that forbid device allocation).  Its
output must match the plan-based lf_chi2_batch on the same inputs within the tests' chi^2
tolerances, on two calls in a row (the shared static array keeps the previous call's
contents, so the second call checks that everything that must start from zero is cleared);
the device's free memory must not change across calls; a capturing stream is refused.  Kept
in its own file so that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-9), ("ff", 1e-12)])
def test_static_entry_point_matches_plan(prec, tol):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import _lib as L
    from paper_2609_08649_b300 import api
    from paper_2609_08649_b300 import model as PM
    from paper_2609_08649_b300 import workloads as W
    wl = W.cluster_c2(n_samples=64)
    cat = W.load_catalogue("cluster_200")
    th = torch.tensor(W.sample_thetas(wl, wl.seed), device="cuda")
    ci = PM.cluster_input(wl, cat)
    plan = api.Plan([ci], th.shape[0], prec)
    ref = plan.chi2(th)
    cs = ci.c_struct()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full((th.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        L.check(L.lib.lf_chi2_batch_static(C.byref(cs), C.c_void_p(th.data_ptr()), th.shape[0],
                                           api.PRECISION[prec], C.c_void_p(out.data_ptr()), stream))
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert torch.allclose(out, ref, rtol=tol, atol=0), (call, (out - ref).abs().max().item())
    # a second, smaller cluster through the same array, then the first again
    wl4 = W.multicluster_c4()[3]
    cat4 = W.load_catalogue("multicluster_03")
    th4 = torch.tensor(W.sample_thetas(wl4, wl4.seed), device="cuda")
    ci4 = PM.cluster_input(wl4, cat4)
    ref4 = api.Plan([ci4], th4.shape[0], prec).chi2(th4)
    cs4 = ci4.c_struct()
    out4 = torch.empty(th4.shape[0], dtype=torch.float64, device="cuda")
    L.check(L.lib.lf_chi2_batch_static(C.byref(cs4), C.c_void_p(th4.data_ptr()), th4.shape[0],
                                       api.PRECISION[prec], C.c_void_p(out4.data_ptr()), stream))
    out = torch.empty_like(ref)
    L.check(L.lib.lf_chi2_batch_static(C.byref(cs), C.c_void_p(th.data_ptr()), th.shape[0],
                                       api.PRECISION[prec], C.c_void_p(out.data_ptr()), stream))
    torch.cuda.synchronize()
    assert torch.allclose(out4, ref4, rtol=tol, atol=0)
    assert torch.allclose(out, ref, rtol=tol, atol=0)
    # no device allocation: free memory (2 MiB granularity) is unchanged by further calls
    free0 = torch.cuda.mem_get_info()[0]
    for c_, t_, o_ in ((cs4, th4, out4), (cs, th, out)):
        L.check(L.lib.lf_chi2_batch_static(C.byref(c_), C.c_void_p(t_.data_ptr()), t_.shape[0],
                                           api.PRECISION[prec], C.c_void_p(o_.data_ptr()), stream))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    api.device_error()


def test_static_entry_point_refuses_stream_capture():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import _lib as L
    from paper_2609_08649_b300 import model as PM
    from paper_2609_08649_b300 import workloads as W
    wl = W.cluster_c2(n_samples=2)
    cat = W.load_catalogue("cluster_200")
    cs = PM.cluster_input(wl, cat).c_struct()
    th = torch.tensor(W.sample_thetas(wl, wl.seed), device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        out.add_(1.0)
        st = L.lib.lf_chi2_batch_static(C.byref(cs), C.c_void_p(th.data_ptr()), 2, L.LF_MIXED,
                                        C.c_void_p(out.data_ptr()), C.c_void_p(s.cuda_stream))
    assert st == L.LF_EUNSUPPORTED and b"captur" in L.lib.lf_last_error()


def test_static_entry_point_rejects_oversized_cluster():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import _lib as L
    from paper_2609_08649_b300 import model as PM
    from paper_2609_08649_b300 import workloads as W
    wl = W.cluster_c2(n_samples=1)
    cat = W.load_catalogue("cluster_200")
    m = wl.planes[0].members
    n = 30000        # 30000 member records need more than the 1 MiB array
    rng = np.random.default_rng(0)
    wl.planes[0].members = W.PhysMembers(rng.uniform(-75, 75, n), rng.uniform(-75, 75, n),
                                         rng.uniform(-2, 1, n), m.vstar, m.core_star_kpc,
                                         m.cut_star_kpc, m.lam, m.beta, m.alpha)
    ci = PM.cluster_input(wl, cat)
    cs = ci.c_struct()
    th = torch.tensor(W.sample_thetas(wl, wl.seed), device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    st = L.lib.lf_chi2_batch_static(C.byref(cs), C.c_void_p(th.data_ptr()), 1, L.LF_MIXED,
                                    C.c_void_p(out.data_ptr()), None)
    assert st == L.LF_EINVAL and b"static" in L.lib.lf_last_error()
