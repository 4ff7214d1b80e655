"""The FP64 throughput probe (GPU): it must return a rate of the order the
hardware can issue -- GB300 issues a few FP64 lane-operations per SM per
cycle -- so that the FP64 roofline of the sweep has a measured denominator."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_rate_is_plausible():
    import torch

    from paper_1702_04910_gb300 import binding as B
    props = torch.cuda.get_device_properties(0)
    rate = B.lbm_measure_fp64_rate(torch.cuda.current_stream().cuda_stream)
    per_sm_cycle = rate / props.multi_processor_count / 2.1e9
    # between a quarter of one lane-op and 64 lane-ops per SM per cycle at
    # any clock up to 2.1 GHz: catches a probe whose chains were optimised
    # away (far above) or that measured the wrong thing (far below)
    assert 0.25 < per_sm_cycle < 64.0, (rate, per_sm_cycle)
