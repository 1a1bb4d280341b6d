"""Pins of the oracle's downsampling (Sec.3.2) and running-median
de-reddening (Sec.3.3) to things other than itself.

* downsampling: numpy's reshape-and-sum (a library routine), the identity
  at factor 1, the dropped partial group, int32 overflow;
* running median: numpy's partition (a library selection) over every
  clamped window of small series with many ties; closed forms: a constant
  series gives zeros, a ramp gives zeros inside and
  t - floor((t + h) / 2) at the left end, a lone spike on a constant keeps
  its height and leaves the rest at zero; removal of a slow baseline.
"""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("n,f", [(1000, 1), (1000, 4), (1003, 7), (5, 8), (64, 64)])
def test_downsample_is_reshape_sum(n, f):
    rng = np.random.default_rng(n + f)
    x = rng.integers(-1000, 1000, size=n).astype(np.int32)
    y = oracle.downsample(x, f)
    m = n // f
    ref = x[:m * f].astype(np.int64).reshape(m, f).sum(1) if m else np.zeros(0)
    assert y.size == m and np.array_equal(y, ref)
    if f == 1:
        assert np.array_equal(y, x)


def test_downsample_overflow_and_bad_factor():
    x = np.full(8, 2 ** 30, np.int32)
    with pytest.raises(OverflowError):
        oracle.downsample(x, 2)
    assert np.array_equal(oracle.downsample(x[:2], 1), x[:2])
    with pytest.raises(OverflowError):
        oracle.downsample(x, 0)


def _brute(x, h):
    n = x.size
    out = np.empty(n, np.int64)
    for t in range(n):
        w = x[max(0, t - h):min(n, t + h + 1)]
        k = (w.size - 1) // 2
        out[t] = int(x[t]) - int(np.partition(w, k)[k])
    return out


@pytest.mark.parametrize("n,h,vals", [(300, 7, 5), (257, 20, 1000), (64, 0, 9),
                                      (40, 100, 3), (1, 3, 10)])
def test_running_median_vs_partition(n, h, vals):
    rng = np.random.default_rng(n * 31 + h)
    x = rng.integers(-vals, vals + 1, size=n).astype(np.int32)
    assert np.array_equal(oracle.dered(x, h), _brute(x, h))
    for t in (0, n // 2, n - 1):
        assert oracle.running_median(x, h, t) == int(x[t]) - _brute(x, h)[t]


def test_running_median_closed_forms():
    n, h = 200, 9
    assert (oracle.dered(np.full(n, -7, np.int32), h) == 0).all()
    t = np.arange(n)
    z = oracle.dered(t.astype(np.int32), h)
    assert (z[h:n - h] == 0).all()
    left = t[:h] - (t[:h] + h) // 2
    assert np.array_equal(z[:h], left)
    x = np.full(n, 50, np.int32)
    x[100] = 1050
    z = oracle.dered(x, h)
    assert z[100] == 1000 and (np.delete(z, 100) == 0).all()


def test_dered_removes_a_slow_baseline():
    rng = np.random.default_rng(5)
    n, h = 20000, 200
    t = np.arange(n)
    base = (3000 * np.sin(2 * np.pi * t / 8000)).astype(np.int64)
    noise = rng.normal(0, 100, n).astype(np.int64)
    x = (base + noise).astype(np.int32)
    z = oracle.dered(x, h)
    inner = slice(h, n - h)
    assert np.std(z[inner]) < 1.5 * np.std(noise) and np.std(x) > 15 * np.std(noise)
