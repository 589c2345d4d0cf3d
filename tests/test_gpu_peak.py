"""The FP32 FMA-rate probe (the ALU roofline's measured denominator) lands
between half and just above the nominal rate SMs x 128 lanes x 2 x the
maximum SM clock."""
import pytest
import torch

from paper_2310_04676_gb300 import sg

pytestmark = pytest.mark.gpu


def test_fma_rate_probe_is_near_nominal():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    props = torch.cuda.get_device_properties(0)
    rate = sg.fp32_fma_rate(iters=1024, repeats=3)
    clock_khz = getattr(props, "clock_rate", 0) or 2070000
    nominal = props.multi_processor_count * 128 * 2 * clock_khz * 1e3 / 1e12
    assert 0.5 * nominal <= rate <= 1.05 * nominal, (rate, nominal)
    lib = sg.load_library()
    assert lib.sg_measure_fp32_fma_rate(None, 0, 1, None) == sg.SG_ERR_INVALID_ARG
