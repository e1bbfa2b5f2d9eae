"""The library's microbenchmarks (mcx_peak_measure) give rates in the range
the hardware's unit counts and clock allow: FFMA at most 128 lanes per SM
per clock (and at least half of that), IMAD at most that, FP64 well below
FP32, the 3-atomic monitor hit at most a third of the u64 atomic rate, and
footprints outside the documented range refused."""

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_08747_gb300 import build
    build.build()
    from paper_2410_08747_gb300 import mcx
    return mcx, torch


def test_peak_rates_are_physical(env):
    mcx, torch = env
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clock_hz = 2.2e9                      # above GB300's 2070 MHz maximum SM clock
    lane_peak = 128 * sms * clock_hz
    ffma = mcx.peak_measure("ffma")
    imad = mcx.peak_measure("imad")
    dfma = mcx.peak_measure("dfma")
    philox = mcx.peak_measure("philox")
    assert 0.4 * 128 * sms * 1.0e9 < ffma <= lane_peak   # at least 40 % of the lanes at 1 GHz
    assert 0.0 < imad <= ffma * 1.05
    assert 0.0 < dfma < 0.2 * ffma
    assert 0.0 < philox < ffma / 60          # a block is well over 60 lane instructions
    mb = 16 * 1024 * 1024
    hit = mcx.peak_measure("hit", 0, mb // 24 * 24)
    red = mcx.peak_measure("red_u64", 0, mb)
    assert 0.0 < hit <= red / 3 * 1.1
    with pytest.raises(mcx.McxError):
        mcx.peak_measure("hit", 0, 100)       # fewer than 64 bins
