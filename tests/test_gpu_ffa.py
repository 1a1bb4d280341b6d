"""GPU parity of the folding transform and the folded-profile search
(Sec.3.5) with the CPU oracle.

* transform: integer sums, bit-exact;
* search: the FP32 S/N within 1e-5 relative of the oracle's FP64 value;
  width and phase equal unless the oracle's S/N at the GPU's choice is
  within 1e-5 of its best (a near tie decided in a different precision).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import DdspError, Plan, build

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _plan():
    return Plan(16, 500.0, -1.0, 1e-3, np.zeros(4), [1, 2], nbits=8,
                norm_window=8192, cand_capacity=1024)


def _series(rows, n, seed, lo=-3000, hi=3000):
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi, size=(rows, n), endpoint=True).astype(np.int32)


@pytest.mark.parametrize("rows,n,p", [(2, 4096, 37), (3, 16384, 1), (2, 1000, 7),
                                      (2, 5000, 3000), (1, 16384, 128),
                                      (2, 999, 999)])
def test_transform_matches_oracle(rows, n, p):
    x = _series(rows, n, n + p)
    pl = _plan()
    F = pl.ffa(torch.from_numpy(x).cuda(), p).cpu().numpy()
    pl.check()
    for r in range(rows):
        assert np.array_equal(F[r].astype(np.int64), oracle.ffa(x[r], p)), r


def check_search(x, p_lo, p_hi, widths, sigma):
    pl = _plan()
    snr, wi, ph = pl.ffa_search(torch.from_numpy(x).cuda(), p_lo, p_hi,
                                widths, sigma)
    pl.check()
    snr, wi, ph = snr.cpu().numpy(), wi.cpu().numpy(), ph.cpu().numpy()
    rows, n = x.shape
    nchecked = 0
    for r in range(rows):
        for pi, p in enumerate(range(p_lo, p_hi)):
            F = oracle.ffa(x[r], p)
            m = F.shape[0]
            assert (snr[r, pi, m:] == -np.inf).all() and (wi[r, pi, m:] == -1).all()
            for s in range(m):
                owi, osn, oph = oracle.fold_snr(F[s], m, widths, sigma)
                g = snr[r, pi, s]
                assert abs(g - osn) <= RTOL * max(abs(osn), 1.0), (r, p, s)
                if (wi[r, pi, s], ph[r, pi, s]) != (owi, oph):
                    w = widths[wi[r, pi, s]]
                    P = F[s]
                    B = sum(int(P[(ph[r, pi, s] + i) % p]) for i in range(w))
                    alt = (B - w * P.sum() / p) / (sigma * np.sqrt(m * w))
                    assert abs(alt - osn) <= RTOL * max(abs(osn), 1.0), (r, p, s)
                nchecked += 1
    return nchecked


def test_search_matches_oracle():
    x = _series(2, 4096, 11)
    assert check_search(x, 30, 41, [1, 2, 4, 8, 16], 1500.0) > 1000


def test_search_widths_wider_than_small_periods():
    x = _series(1, 2000, 12)
    check_search(x, 3, 9, [1, 2, 4, 8], 900.0)          # w = 4, 8 skipped where > p


def test_search_finds_planted_pulsar():
    n, p0, s0 = 16384, 200, 23
    m = Plan.ffa_rows(n, p0)
    period = p0 + s0 / (m - 1)
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1024, size=(1, n))
    at = np.floor(50 + np.arange(int(n / period) + 1) * period).astype(np.int64)
    for d in range(4):
        a = at + d
        x[0, a[a < n]] += 900          # folded S/N about 12
    x = np.round(x).astype(np.int32)
    pl = _plan()
    snr, wi, ph = pl.ffa_search(torch.from_numpy(x).cuda(), 190, 210,
                                [1, 2, 4, 8, 16], 1024.0)
    snr = snr.cpu().numpy()[0]
    pi, s = np.unravel_index(np.argmax(snr), snr.shape)
    assert 190 + pi == p0 and abs(s - s0) <= 2 and snr[pi, s] > 10


def test_bench_size_sampled():
    rows, n, p_lo, p_hi = 256, 16384, 128, 256
    widths = [1, 2, 4, 8, 16, 32]
    x = _series(rows, n, 21, -4000, 4000)
    pl = _plan()
    snr, wi, ph = pl.ffa_search(torch.from_numpy(x).cuda(), p_lo, p_hi,
                                widths, 1024.0)
    pl.check()
    snr, wi, ph = snr.cpu().numpy(), wi.cpu().numpy(), ph.cpu().numpy()
    rng = np.random.default_rng(5)
    for _ in range(30):
        r = int(rng.integers(rows))
        p = int(rng.integers(p_lo, p_hi))
        F = oracle.ffa(x[r], p)
        m = F.shape[0]
        for s in (0, m - 1, int(rng.integers(m))):
            owi, osn, oph = oracle.fold_snr(F[s], m, widths, 1024.0)
            assert abs(snr[r, p - p_lo, s] - osn) <= RTOL * max(abs(osn), 1.0)


def test_overflow_and_argument_errors():
    pl = _plan()
    big = np.full((1, 4096), 2 ** 29, np.int32)
    pl.ffa(torch.from_numpy(big).cuda(), 256)          # m = 16: sums reach 2^33
    with pytest.raises(DdspError) as e:
        pl.check()
    assert e.value.code == -7
    x = torch.zeros((1, 40000), dtype=torch.int32, device="cuda")
    with pytest.raises(DdspError):
        pl.ffa(x, 9000)                                 # m * p > 16384
    y = torch.zeros((1, 4096), dtype=torch.int32, device="cuda")
    with pytest.raises(DdspError):
        pl.ffa_search(y, 30, 40, [2, 1], 1.0)           # unsorted widths
    with pytest.raises(DdspError):
        pl.ffa_search(y, 40, 40, [1], 1.0)              # empty period range
    with pytest.raises(DdspError):
        pl.ffa(y, 5000)                                 # p > nsamp
    pl.check()
