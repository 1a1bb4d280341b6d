"""GPU parity of downsampling (Sec.3.2) and running-median de-reddening
(Sec.3.3) with the CPU oracle: integer work, so bit-exact, on small series
in full and on the beam's 1024 x 262144 series at sampled outputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import DdspError, Plan, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _plan():
    return Plan(16, 500.0, -1.0, 1e-3, np.zeros(4), [1, 2], nbits=8,
                norm_window=8192, cand_capacity=1024)


def _series(rows, n, seed, lo, hi):
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi, size=(rows, n), endpoint=True).astype(np.int32)


@pytest.mark.parametrize("rows,n,f", [(3, 1000, 1), (4, 1003, 3), (2, 4096, 32),
                                      (3, 5000, 100), (2, 7, 8), (1, 64, 64)])
def test_downsample_matches_oracle(rows, n, f):
    x = _series(rows, n, rows * n + f, -50000, 50000)
    p = _plan()
    y = p.downsample(torch.from_numpy(x).cuda(), f).cpu().numpy()
    p.check()
    assert y.shape == (rows, n // f)
    for r in range(rows):
        assert np.array_equal(y[r], oracle.downsample(x[r], f))


def test_downsample_overflow_is_reported():
    x = np.full((1, 64), 2 ** 30, np.int32)
    p = _plan()
    p.downsample(torch.from_numpy(x).cuda(), 4)
    with pytest.raises(DdspError) as e:
        p.check()
    assert e.value.code == -7
    p.check()                                    # the error word was cleared
    with pytest.raises(DdspError):
        p.downsample(torch.from_numpy(x).cuda(), 0)


@pytest.mark.parametrize("rows,n,h,lo,hi", [
    (3, 3000, 0, -5, 5),            # h = 0: all zeros
    (3, 3000, 1, -3, 3),            # many ties
    (2, 9001, 37, -1000, 1000),     # ragged last chunk
    (2, 20000, 700, 0, 4000),       # several chunks, 12-bit values
    (2, 5000, 3000, -2 ** 29, 2 ** 29),   # window wider than a chunk
    (2, 300, 1000, -9, 9),          # window wider than the row
    (1, 1, 5, 7, 7),                # one sample
    (2, 2500, 64, 123, 123),        # constant rows (no wavelet levels)
])
def test_dered_matches_oracle(rows, n, h, lo, hi):
    x = _series(rows, n, n + h, lo, hi)
    p = _plan()
    z = p.dered(torch.from_numpy(x).cuda(), h).cpu().numpy()
    p.check()
    for r in range(rows):
        assert np.array_equal(z[r], oracle.dered(x[r], h)), r


def test_dered_full_int32_range_and_spikes():
    x = _series(2, 4000, 9, -2 ** 31, 2 ** 31 - 1)
    x[1] = 17
    x[1, ::500] = 2 ** 31 - 1                   # lone spikes on a constant
    p = _plan()
    h = 40
    xd = torch.from_numpy(x).cuda()
    z = p.dered(xd, h).cpu().numpy()
    with pytest.raises(DdspError) as e:          # residuals beyond int32
        p.check()
    assert e.value.code == -7
    assert (z[1][::500] == 2 ** 31 - 1 - 17).all()
    # rows whose residuals fit int32 are exact
    x2 = _series(2, 4000, 10, -2 ** 30, 2 ** 30 - 1)
    z2 = p.dered(torch.from_numpy(x2).cuda(), h).cpu().numpy()
    p.check()
    for r in range(2):
        assert np.array_equal(z2[r], oracle.dered(x2[r], h))


def test_dered_beam_series_sampled():
    ndm, n, h = 1024, 262144, 1024
    x = synth.gaussian_series(ndm, n, seed=14, device="cuda")
    p = _plan()
    z = p.dered(x, h)
    p.check()
    rng = np.random.default_rng(3)
    rows = rng.integers(0, ndm, 40)
    xs = x[torch.from_numpy(rows).cuda()].cpu().numpy()
    zs = z[torch.from_numpy(rows).cuda()].cpu().numpy()
    for i, r in enumerate(rows):
        for t in np.concatenate([[0, 1, h, n - 1], rng.integers(0, n, 6)]):
            m = oracle.running_median(xs[i], h, int(t))
            assert zs[i, t] == int(xs[i, t]) - m, (r, t)


def test_dered_after_dedispersion_matches_oracle_chain():
    cfg = synth.config1()
    x = synth.filterbank(cfg, 16384)
    p = Plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
             cfg.widths, nbits=8, norm_window=cfg.norm_window,
             cand_capacity=1 << 16)
    series = p.dedisperse(x.cuda())
    z = p.dered(series, 256).cpu().numpy()
    y = p.downsample(series, 4).cpu().numpy()
    p.check()
    d, _ = oracle.delay_table(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp,
                              cfg.dm_list())
    ks = [0, 100, 255]
    ref = oracle.dedisperse(x.numpy(), d[ks])
    for i, k in enumerate(ks):
        assert np.array_equal(z[k], oracle.dered(ref[i], 256))
        assert np.array_equal(y[k], oracle.downsample(ref[i], 4))


def test_dered_argument_errors():
    p = _plan()
    x = torch.zeros((2, 100), dtype=torch.int32, device="cuda")
    with pytest.raises(DdspError):
        p.dered(x, -1)
    with pytest.raises(DdspError):
        p.dered(x, 7000)
    p.dered(x, 6700)
    with pytest.raises(DdspError):
        p.dered(x, 3, out=x)                     # in place is not allowed
    p.check()
