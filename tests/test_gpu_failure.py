"""Failure detection on the GPU without a fault: every device wait of the
default (interleaved) dedispersion kernel is bounded.  The copy-issuing warp
is told to stop before one chunk of channels (a hand-off nothing will ever
complete), with a short hand-off bound; the computing warps' wait runs out,
the kernel records DDSP_E_TIMEOUT, lets the copies it issued land and
returns.  The plan then reports the timeout, and with the switch off and the
default bound restored the next dedispersion is bit-exact against the oracle
again: the context stayed usable."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import DdspError, Plan, _lib, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _c1_plan():
    cfg = synth.config1()
    p = Plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
             cfg.widths, nbits=8, norm_window=cfg.norm_window,
             cand_capacity=1 << 16)
    return cfg, p


@pytest.mark.parametrize("chunk", [0, 3])
def test_withheld_copy_times_out_then_recovers(chunk):
    cfg, p = _c1_plan()
    assert p.get_tile()["flags"] & 16, "default tile is the interleaved kernel"
    x = synth.filterbank(cfg, 16384)
    ref = oracle.dedisperse(x.numpy(), p.delays())
    xd = x.cuda()
    p.set_wait_limit(2_000_000)          # about 1 ms of SM clock
    p.withhold_copy(chunk)
    p.dedisperse(xd)
    with pytest.raises(DdspError) as e:
        p.check()
    assert e.value.code == _lib.DDSP_E_TIMEOUT
    p.check()                            # the error word was cleared
    p.withhold_copy(-1)
    p.set_wait_limit(0)
    out = p.dedisperse(xd)
    p.check()
    assert np.array_equal(out.cpu().numpy(), ref)
    # the search after it runs and finds the injected pulse
    p.single_pulse_search(out, cfg.threshold)
    cands, n = p.fetch()
    best = cands[np.argmax(cands["snr"])]
    assert n > 0 and int(best["dm_idx"]) == 100


def test_wait_limit_arguments():
    _, p = _c1_plan()
    with pytest.raises(DdspError):
        p.set_wait_limit(-1)
    with pytest.raises(DdspError):
        p.withhold_copy(-2)
    p.set_wait_limit(0)
    p.withhold_copy(-1)


def test_short_bound_alone_keeps_results_exact():
    """A hand-off bound far above a copy's latency (50 us) with no switch:
    every wait completes, the output is exact and no error is reported."""
    cfg, p = _c1_plan()
    x = synth.filterbank(cfg, 16384)
    ref = oracle.dedisperse(x.numpy(), p.delays())
    p.set_wait_limit(100_000)
    out = p.dedisperse(x.cuda())
    p.check()
    assert np.array_equal(out.cpu().numpy(), ref)
