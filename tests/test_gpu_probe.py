"""ak_probe_fp64_rate: the measured FP64 rate that the FP64 form's roofline divides by."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ak():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2409_16053_gb300 import build
    build.build()
    from paper_2409_16053_gb300 import ak as mod
    return mod


def test_fp64_rate_is_plausible_and_repeatable(ak):
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    a = ak.ak_probe_fp64_rate(0)
    b = ak.ak_probe_fp64_rate(0)
    # per SM and clock at most the unit's width (a few DFMA), at least a small fraction
    # of it, at clocks between 0.5 and 2.5 GHz
    for r in (a, b):
        per_sm = r / nsm
        assert 0.1 * 0.5e9 < per_sm < 64 * 2.5e9, r
    assert abs(a - b) / max(a, b) < 0.2, (a, b)
