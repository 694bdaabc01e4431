"""The int32 issue-rate probe that sits beside the enumeration's roofline:
positive rates, none above the derived issue peak (152 SMs x 128 lanes x
the maximum SM clock, with 5% margin for clock reporting), so that a probe
the compiler had folded away would fail here."""
import pytest

from paper_1806_10113_gb300 import tm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_int32_rates_are_positive_and_below_the_issue_peak():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 128 * 2070e6 * 1.05
    r = tm.tm_measure_int32_rates()
    assert set(r) == {"max", "add", "max_add"}
    for k, v in r.items():
        assert 0.05 * peak < v < peak, (k, v, peak)
