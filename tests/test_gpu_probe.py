"""The unit-peak microbenchmarks (ddsp_probe_unit_peaks) run on the device
and return rates within what one SM can physically do: at most 4 warp
instructions per clock (128 lane operations), shared-memory loads within
twice the 128-byte port, and the dedispersion inner loop no faster than
the shared-memory bytes it reads (one byte per add)."""
import pytest

from paper_2605_03531_b300 import DdspError, build, probe_unit_peaks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def test_unit_peaks_are_physical():
    r = probe_unit_peaks(0)
    assert r["sms"] > 0 and all(b >= 1 for b in r["blocks_per_sm"])
    assert 16 <= r["smem_bytes_per_clk"] <= 256
    for k in ("iadd3_per_clk", "prmt_per_clk"):
        assert 8 <= r[k] <= 128, (k, r[k])
    assert 16 <= r["swar_adds_per_clk"] <= 1.05 * r["smem_bytes_per_clk"]


def test_bad_device_refused():
    with pytest.raises(DdspError):
        probe_unit_peaks(-1)
