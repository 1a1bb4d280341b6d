"""Pins of the oracle's gptool-style RFI mitigation (Sec.2.1).

* a pure bandpass shape (every channel a fixed gain times one time series)
  comes out flat across the band, with no flags;
* a constant block is left as it is (its MAD is 0: no flags);
* planted narrowband RFI is flagged exactly, planted broadband bursts are
  among the time flags, and noise-only channels stay unflagged (4 sigma);
* doubling the data (no clipping) flags the same channels and samples;
* a second round only adds flags; the fill level replaces flagged data.
"""
import numpy as np
import pytest

import oracle
from paper_2605_03531_b300 import synth


def test_bandpass_shape_is_flattened():
    """A gain rising steadily across the band: the 21-channel moving median
    of a monotone spectrum is the channel's own value away from the band
    edges, so those channels come out flat (up to 8-bit rounding)."""
    nt, nc = 512, 128
    rng = np.random.default_rng(2)
    gain = 0.5 + 1.5 * np.arange(nc) / (nc - 1)
    base = 80 + 20 * rng.random(nt)
    x = np.round(gain[None, :] * base[:, None]).astype(np.uint8)
    out, fc, ft = oracle.rfi_clean(x)
    assert not fc.any() and not ft.any()
    inner = slice(10, nc - 10)
    assert x[:, inner].astype(float).std(1).mean() > 15   # the input is not flat
    y = out[:, inner].astype(float)
    assert np.percentile(y.max(1) - y.min(1), 90) <= 3     # the output is


def test_constant_block_unchanged():
    x = np.full((300, 64), 93, np.uint8)
    out, fc, ft = oracle.rfi_clean(x)
    assert np.array_equal(out, x) and not fc.any() and not ft.any()


def _rfi_block(seed=3):
    x = synth.noise_u8_np(4096, 256, seed).astype(np.int64)
    rfi_c = [17, 40, 41, 200]
    rfi_t = [100, 2000, 3001]
    x[:, rfi_c] += 60
    x[rfi_t, :] += 40
    return np.minimum(x, 255).astype(np.uint8), rfi_c, rfi_t


def test_planted_rfi_is_flagged():
    x, rfi_c, rfi_t = _rfi_block()
    out, fc, ft = oracle.rfi_clean(x)
    assert list(np.nonzero(fc)[0]) == rfi_c
    assert set(rfi_t) <= set(np.nonzero(ft)[0])
    assert ft.sum() < 0.01 * x.shape[0]                 # ~0.3 % at 3 sigma
    fill = out[rfi_t[0], 0]
    assert (out[:, rfi_c] == fill).all() and (out[rfi_t, :] == fill).all()
    assert abs(int(fill) - 128) <= 2                    # the band's level


def test_flags_scale_invariant_and_monotone_in_rounds():
    x, _, _ = _rfi_block(5)
    x = (x // 2).astype(np.uint8)                       # room to double
    _, fc1, ft1 = oracle.rfi_clean(x)
    _, fc2, ft2 = oracle.rfi_clean((2 * x.astype(np.int64)).astype(np.uint8))
    assert np.array_equal(fc1, fc2) and np.array_equal(ft1, ft2)
    _, fa, ta = oracle.rfi_clean(x, rounds=1)
    _, fb, tb = oracle.rfi_clean(x, rounds=2)
    assert not (fa & ~fb).any() and not (ta & ~tb).any()


def test_bad_arguments():
    with pytest.raises(ValueError):
        oracle.rfi_clean(np.zeros((4, 4), np.uint8), rounds=0)
