"""Pins of the oracle's folding transform and folded-profile boxcar search
(Sec.3.5) to things other than itself.

* transform: profile 0 is the plain fold (numpy reshape-and-sum), profile
  m - 1 shifts row i by i samples (numpy roll), every profile keeps the
  total power, m = 1 and m = 2 by hand, linearity, and a pulse train whose
  period is p + s0/(m - 1) folds best at s0 with its pulses stacked;
* profile S/N: numpy's cyclic sums (roll) in a brute-force scan, closed
  forms for a flat profile and a lone spike, ties to the smaller width and
  phase.
"""
import numpy as np
import pytest

import oracle


def rows(x, p, m):
    return x[:m * p].astype(np.int64).reshape(m, p)


@pytest.mark.parametrize("n,p", [(4096, 37), (1000, 7), (64, 64), (100, 33), (4096, 1)])
def test_fold_closed_forms(n, p):
    rng = np.random.default_rng(n + p)
    x = rng.integers(-500, 500, size=n).astype(np.int32)
    F = oracle.ffa(x, p)
    m = oracle.ffa_rows(n, p)
    assert F.shape == (m, p) and m * p <= n < 2 * m * p
    R = rows(x, p, m)
    assert np.array_equal(F[0], R.sum(0))
    shifted = np.stack([np.roll(R[i], -i) for i in range(m)])
    assert np.array_equal(F[m - 1], shifted.sum(0))
    assert (F.sum(1) == R.sum()).all()


def test_fold_small_stacks_by_hand():
    x = np.array([1, 2, 3, 10, 20, 30], np.int32)
    assert np.array_equal(oracle.ffa(x[:3], 3), [[1, 2, 3]])          # m = 1
    F = oracle.ffa(x, 3)                                               # m = 2
    assert np.array_equal(F, [[11, 22, 33], [21, 32, 13]])
    with pytest.raises(ValueError):
        oracle.ffa(x[:2], 3)


def test_fold_linear():
    rng = np.random.default_rng(4)
    a = rng.integers(-99, 99, size=2000).astype(np.int32)
    b = rng.integers(-99, 99, size=2000).astype(np.int32)
    Fa, Fb = oracle.ffa(a, 29), oracle.ffa(b, 29)
    assert np.array_equal(oracle.ffa(3 * a - 2 * b, 29), 3 * Fa - 2 * Fb)


@pytest.mark.parametrize("s0", [0, 5, 17, 31])
def test_pulse_train_folds_at_its_period(s0):
    """3-sample pulses every p + s0/(m - 1) samples: trial s0 stacks all m
    pulses in one bin (the transform's integer shifts stay within a sample
    of the true drift), trials 4 or more away do not."""
    p, m = 50, 32
    n = m * p
    period = p + s0 / (m - 1)
    x = np.zeros(n, np.int32)
    at = np.floor(7 + np.arange(int(n / period) + 1) * period).astype(np.int64)
    for d in range(3):
        x[(at + d)[at + d < n]] = 100
    peaks = oracle.ffa(x, p).max(1)
    assert peaks[s0] == 100 * m
    assert max(peaks[s] for s in range(m) if abs(s - s0) >= 4) < peaks[s0]


def _brute_snr(P, m, widths, sigma):
    p = P.size
    mu = P.sum() / p
    best = (-1, 0.0, 0)
    for wi, w in enumerate(widths):
        if w < 1 or w > p:
            continue
        B = sum(np.roll(P, -i) for i in range(w))
        snr = (B - w * mu) / (sigma * np.sqrt(m * w))
        j = int(np.argmax(snr))
        if best[0] < 0 or snr[j] > best[1]:
            best = (wi, float(snr[j]), j)
    return best


@pytest.mark.parametrize("p,m", [(50, 8), (97, 32), (16, 1)])
def test_fold_snr_vs_roll_sums(p, m):
    rng = np.random.default_rng(p * m)
    P = rng.integers(-3000, 3000, size=p).astype(np.int64)
    P[p // 3:p // 3 + 4] += 20000
    widths = [1, 2, 4, 8, 16, 32, 64, 128]
    wi, s, ph = oracle.fold_snr(P, m, widths, 12.5)
    bw, bs, bj = _brute_snr(P, m, widths, 12.5)
    assert (wi, ph) == (bw, bj) and abs(s - bs) <= 1e-9 * abs(bs)


def test_fold_snr_closed_forms():
    flat = np.full(40, 7, np.int64)
    assert oracle.fold_snr(flat, 4, [2, 1], 1.0) == (0, 0.0, 0)
    spike = np.zeros(40, np.int64)
    spike[11] = 400
    wi, s, ph = oracle.fold_snr(spike, 16, [1, 2], 2.0)
    assert (wi, ph) == (0, 11) and abs(s - (400 - 10.0) / (2.0 * 4.0)) < 1e-12
    assert oracle.fold_snr(spike, 16, [64], 1.0)[0] == -1       # no width fits
