"""The ceiling probes the roofline divides by (lj_measure_peak): each returns
a rate that its own timing supports and that lies below what the unit counts
allow at the GPU's maximum clock, and the rates keep the ratios the hardware
fixes (packed FP32 FMA >= scalar FP32 FMA >> FP64 FMA)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.fixture(scope="module")
def rates(cuda_lib):
    lj = cuda_lib
    buf = torch.zeros(16 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for name, kind, work, b in (("dfma", lj.LJ_PEAK_DFMA, 40, None),
                                ("ffma", lj.LJ_PEAK_FFMA, 2000, None),
                                ("ffma2", lj.LJ_PEAK_FFMA2, 2000, None),
                                ("l2", lj.LJ_PEAK_L2_READ, 200, buf)):
        out[name] = lj.lj_measure_peak(kind, work, b)
    # the L2 probe only reads a zero-filled buffer
    assert int(buf.count_nonzero()) == 0
    return out


def test_rates_match_their_own_timing(rates):
    sms, threads = _sms(), 8 * 256
    for name, per_lane in (("dfma", 2), ("ffma", 2), ("ffma2", 4)):
        rate, ms = rates[name]
        work = {"dfma": 40, "ffma": 2000, "ffma2": 2000}[name]
        flops = sms * threads * 8 * 16 * work * per_lane
        assert ms > 0 and rate == pytest.approx(flops / (ms * 1e-3), rel=1e-6)
    rate, ms = rates["l2"]
    assert rate == pytest.approx((16 << 20) * 200 / (ms * 1e-3), rel=1e-6)


def test_rates_are_physical(rates):
    sms = _sms()
    clock_hz = 2.2e9        # above the 2.07 GHz maximum SM clock of the part
    assert 0 < rates["dfma"][0] <= sms * 2 * 2 * clock_hz        # 2 DFMA / clk / SM
    assert 0 < rates["ffma"][0] <= sms * 128 * 2 * clock_hz      # 128 FFMA / clk / SM
    assert 0 < rates["ffma2"][0] <= sms * 128 * 2 * clock_hz
    assert rates["ffma"][0] > 20 * rates["dfma"][0]
    assert rates["ffma2"][0] >= 0.9 * rates["ffma"][0]
    assert rates["l2"][0] > 1e12                                   # bytes/s, a resident buffer
