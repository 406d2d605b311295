"""The FP64 rate probe (swnmg_fp64_rate), the roofline denominator of the
kernels bound by the FP64 pipe: a positive rate of the right order for this
GPU class (one to a few FP64 lane operations per clock per SM), and bad
arguments refused."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fp64_rate_plausible():
    from paper_1608_06721_gb300 import swnmg
    props = torch.cuda.get_device_properties(0)
    for op in (0, 1):
        r = swnmg.fp64_rate(op)
        per_sm_clock = r / props.multi_processor_count / 2.1e9
        assert 0.25 <= per_sm_clock <= 64.0, (op, r, per_sm_clock)
    with pytest.raises(swnmg.SwnmgError):
        swnmg.fp64_rate(2)
