"""The peak-rate probes the benchmark's rooflines divide by (corr_probe_rate)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_peak_probes_run_and_are_plausible():
    """The peak-rate probes the benchmark divides by: each returns a positive
    rate below what the part could possibly do (its tensor and ALU counts at
    2.1 GHz), and the tensor-core probe's completion wait does not expire."""
    from paper_1501_05992_gb300 import corr
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceilings = {"tc_fp8": sms * 32768 * 2.1e9, "mma_s8": sms * 32768 * 2.1e9,
                "dp4a": sms * 128 * 8 * 2.1e9, "ffma": sms * 128 * 2 * 2.1e9}
    for kind, ceiling in ceilings.items():
        try:
            rate, ms = corr.probe_rate(kind)
        except corr.CorrError as e:
            if e.status == corr.CORR_E_UNSUPPORTED:
                continue
            raise
        assert 0 < rate < ceiling and ms > 0, (kind, rate)
