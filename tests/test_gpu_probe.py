"""lf_probe_alu: measured arithmetic rates (the roofline denominators) are positive, ordered
as the hardware orders them (FP32 FMA > MUFU > FP64 FMA on this part), and within the
nominal per-SM lane counts at the maximum clock."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2609_08649_b300 import api
    fma, rsq, dfma = api.probe_alu()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    clock_max = 2.2e9        # above the part's maximum SM clock
    print(f"probe: FP32 FMA {fma / 1e12:.2f} T/s, rsqrt {rsq / 1e12:.2f} T/s, FP64 FMA {dfma / 1e12:.3f} T/s")
    assert 0 < dfma < rsq < fma
    assert fma <= nsm * 128 * clock_max and rsq <= nsm * 32 * clock_max
    assert fma > 0.3 * nsm * 128 * 1.0e9
    # packed f32x2 FMA chains: lane-operations per second, on the same 128 FP32 lanes per SM
    fma_b, fma2, rsq_b, dfma_b = api.probe_alu2()
    print(f"probe: packed f32x2 FMA {fma2 / 1e12:.2f} T lane-ops/s (scalar {fma_b / 1e12:.2f})")
    assert 0 < fma2 <= nsm * 128 * clock_max and 0 < fma_b <= nsm * 128 * clock_max


def test_bounded_wait_runs_out_and_is_reported():
    """The failure-detection path: a kernel whose mbarrier phase can never complete (16 bytes
    of transactions expected, no copy issued) gives up after 64 polls, the device error word
    reports LF_ETIMEOUT once, and the context stays usable."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import ctypes as C
    from paper_2609_08649_b300 import _lib as L
    from paper_2609_08649_b300 import api
    api.device_error()                                   # start from a clean word
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(L.lib.lf_selftest_wait_timeout(64, stream))
    with pytest.raises(L.LFError) as e:
        api.device_error()
    assert e.value.status == L.LF_ETIMEOUT
    api.device_error()                                   # the word was cleared
    assert L.lib.lf_selftest_wait_timeout(0, stream) == L.LF_EINVAL
    x = torch.arange(8.0, device="cuda")
    assert float(x.sum()) == 28.0                        # the context still runs work
