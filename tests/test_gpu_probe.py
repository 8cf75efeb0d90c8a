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
