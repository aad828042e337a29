"""The issue-rate probe that checks the sweep kernel's derived roofline peak
(SMs x 128 lanes x SM clock): every kind runs and reports a rate that a GPU
of this many SMs can reach."""
import pytest

pytestmark = pytest.mark.gpu


def test_issue_rates_are_physical():
    import torch
    from paper_1409_3901_gb300 import probe

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 128 * 2.3e9     # above the maximum SM clock of the part
    floor = sms * 128 * 0.5e9       # a quarter of the issue rate at 2 GHz
    rates = {}
    for kind in probe.ISSUE_KINDS:
        rate, ms = probe.issue_rate(kind)
        assert ms > 0.1
        assert floor < rate < ceiling, (kind, rate, floor, ceiling)
        rates[kind] = rate
    print({k: "%.1f T/s" % (v / 1e12) for k, v in rates.items()})
