"""Pins of the oracle's resampling for frequency derivatives (Sec.3.4).

* f1 = f2 = 0 leaves the series unchanged;
* a constant series c gives every kept bin c times its width in input
  samples, 1 + f' k tau0 / f0 + f'' (k tau0)^2 / (2 f0) (closed form), in
  reversed order and with the reversed-series parameters when f1 > 0;
* a pulse train whose frequency drifts as f0 + f1 t + f2 t^2 / 2 comes out
  with pulses at a constant spacing, for f1 < 0 and for f1 > 0;
* the output never holds more power than the input, and bad arguments fail.
"""
import numpy as np
import pytest

import oracle


def test_identity_without_derivatives():
    x = np.random.default_rng(1).integers(-100, 100, 1000).astype(np.int32)
    y = oracle.resample(x, 5.0, 0.0, 0.0, 1e-3)
    assert np.array_equal(y, x.astype(np.float64))


@pytest.mark.parametrize("f1,f2", [(-0.02, 0.0), (-0.01, -0.001), (0.02, 0.0),
                                   (0.01, 0.002)])
def test_constant_series_closed_form(f1, f2):
    n, c, f0, ts = 5000, 7, 3.0, 1e-3
    y = oracle.resample(np.full(n, c, np.int32), f0, f1, f2, ts)
    T = n * ts
    if f1 > 0:
        F0, fp, fpp = f0 + f1 * T + f2 * T * T / 2, f1 + f2 * T, -f2
    else:
        F0, fp, fpp = f0, -f1, -f2
    k = np.arange(y.size)
    w = 1 + fp * k * ts / F0 + fpp * (k * ts) ** 2 / (2 * F0)
    ref = c * (w[::-1] if f1 > 0 else w)
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-9)
    assert y.size <= n and (y.size == n or np.sum(w) <= n)


@pytest.mark.parametrize("f1,f2", [(-0.01, 0.0), (-0.008, -1e-5), (0.01, 0.0),
                                   (0.008, 1e-5)])
def test_drifting_pulse_train_becomes_periodic(f1, f2):
    """Drifts of ~1.6 % over the series (the interval law is first order in
    f' t / f0, so the residual phase error stays well under a period)."""
    ts, n, f0 = 1e-3, 40000, 25.0          # 40 samples per period at the start
    t = np.arange(n) * ts
    phase = f0 * t + f1 * t ** 2 / 2 + f2 * t ** 3 / 6
    x = np.zeros(n, np.int32)
    x[np.nonzero(np.diff(np.floor(phase)) > 0)[0] + 1] = 1000
    y = oracle.resample(x, f0, f1, f2, ts)

    def positions(v):
        idx = np.nonzero(v > 300)[0]
        return idx[np.concatenate([[True], np.diff(idx) > 5])]

    def residual(pos):
        k = np.arange(pos.size)
        fit = np.polyval(np.polyfit(k, pos, 1), k)
        return np.abs(pos - fit).max()

    # the input drifts by many samples from any constant period; the
    # resampled train keeps one period to within a few samples
    assert residual(positions(x)) > 20
    assert residual(positions(y)) <= 3
    T = n * ts
    F = f0 + f1 * T + f2 * T * T / 2 if f1 > 0 else f0
    assert abs(np.median(np.diff(positions(y))) - 1 / (F * ts)) <= 1.0
    assert y.sum() <= x.sum() + 1e-6


def test_bad_arguments():
    x = np.ones(10, np.int32)
    with pytest.raises(ValueError):
        oracle.resample(x, 0.0, 0.0, 0.0, 1e-3)
    with pytest.raises(ValueError):
        oracle.resample(x[:0], 1.0, 0.0, 0.0, 1e-3)
