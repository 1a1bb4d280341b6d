"""GPU parity of the single-pulse search against the CPU oracle.

* window statistics (2*median, 4*MAD): bit-exact;
* per-sample best boxcar sum: bit-exact; best S/N: within 1e-5 relative of
  the FP64 oracle; best width: equal unless two widths tie within 1e-5;
* candidate lists: identical after removing events whose oracle S/N is
  within 1e-4*thr of the threshold;
* the 2048 x 1048576 stress configuration at full size: statistics and
  candidates of sampled DM rows against the oracle run on those rows.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import CAND_DTYPE, DdspError, Plan, build, synth
from parity import SNR_RTOL, THR_EXEMPT, compare_candidates, sps_parallel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _plan(ndm, widths, L, cap=1 << 20):
    # the delay parameters do not matter for the search on a given series
    return Plan(16, 500.0, -1.0, 1e-3, np.zeros(ndm), widths, nbits=8,
                norm_window=L, cand_capacity=cap)


def oracle_dense(x, widths, L):
    """Best width index and S/N at every (k, t) from the oracle (a search with
    a threshold below every possible S/N returns every sample)."""
    ndm, n = x.shape
    c, cnt = oracle.sps(x, widths, L, -1e300, cap=ndm * n)
    assert cnt == c.size
    bw = np.full((ndm, n), -1, np.int64)
    bs = np.zeros((ndm, n))
    bw[c["dm_idx"], c["t"]] = c["w_idx"]
    bs[c["dm_idx"], c["t"]] = c["snr"]
    return bw, bs


def check_dense(x, widths, L):
    ndm, n = x.shape
    p = _plan(ndm, widths, L)
    xd = torch.from_numpy(x).cuda()
    bw, bs, bsum = p.search_dense(xd)
    torch.cuda.synchronize()
    bw, bs, bsum = bw.cpu().numpy(), bs.cpu().numpy(), bsum.cpu().numpy()
    # statistics, bit-exact
    m2, mad4 = p.stats()
    for k in range(ndm):
        rm2, rmad4 = oracle.window_stats(x[k], L)
        assert np.array_equal(m2[k], rm2) and np.array_equal(mad4[k], rmad4), k
    rbw, rbs = oracle_dense(x, widths, L)
    valid = rbw >= 0
    assert np.array_equal(bw >= 0, valid)
    # S/N of the GPU's chosen width vs the oracle's best S/N
    err = np.abs(bs[valid] - rbs[valid])
    assert (err <= SNR_RTOL * np.abs(rbs[valid]) + 1e-30).all(), err.max()
    # width: equal, or the oracle's S/N at both widths agrees within 1e-5
    diff = valid & (bw != rbw)
    for k, t in zip(*np.nonzero(diff)):
        w_gpu = widths[bw[k, t]]
        B = int(x[k, t:t + w_gpu].astype(np.int64).sum())
        j = min(t // L, max(1, n // L) - 1) if L else 0
        rm2, rmad4 = oracle.window_stats(x[k], L)
        s_gpu_w = oracle.snr(B, w_gpu, rm2[j], rmad4[j])
        assert abs(s_gpu_w - rbs[k, t]) <= SNR_RTOL * abs(rbs[k, t]), (k, t)
    # boxcar sum at the GPU's width, bit-exact
    for k in range(ndm):
        for wi, w in enumerate(widths):
            sel = np.nonzero(bw[k] == wi)[0]
            if sel.size:
                ref = oracle.boxcar(x[k], w)[sel]
                assert np.array_equal(bsum[k, sel].astype(np.int64), ref), (k, w)
    return p


@pytest.mark.parametrize("n,L,widths", [
    (40000, 8192, [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024]),
    (15158, 8192, [1, 2, 4, 8, 16, 32]),      # one window longer than L
    (8192, 8192, [1, 2, 4]),
    (5000, 0, [1, 4, 16]),                    # one window over the series
    (9001, 1000, [2, 8, 64]),                 # ragged last window, odd widths set
    (33, 8, [1, 2, 4, 8, 16, 32]),            # widths longer than windows
])
def test_dense_matches_oracle(n, L, widths):
    x = synth.gaussian_series(4, n, seed=n + L).numpy()
    check_dense(x, widths, L)


def test_dense_on_dedispersed_series():
    cfg = synth.config1()
    x = synth.filterbank(cfg, 16384).numpy()
    d, _ = oracle.delay_table(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp,
                              cfg.dm_list())
    ks = np.array([0, 1, 99, 100, 101, 255])
    series = oracle.dedisperse(x, d[ks])
    check_dense(series, cfg.widths, 8192)


_compare_candidates = compare_candidates


@pytest.mark.parametrize("thr", [5.0, 6.5, 9.0])
def test_candidates_match_oracle(thr):
    widths = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024]
    x = synth.gaussian_series(8, 1 << 16, seed=21).numpy()
    p = _plan(8, widths, 8192)
    p.single_pulse_search(torch.from_numpy(x).cuda(), thr)
    got, n_got = p.fetch()
    ref, n_ref = oracle.sps(x, widths, 8192, thr)
    assert n_ref > 0
    _compare_candidates(got, n_got, ref, n_ref, thr, x, widths, 8192)


def test_candidates_c1_series():
    cfg = synth.config1()
    x = synth.filterbank(cfg, 16384).numpy()
    d, _ = oracle.delay_table(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp,
                              cfg.dm_list())
    series = oracle.dedisperse(x, d)
    p = _plan(cfg.ndm, cfg.widths, cfg.norm_window)
    p.single_pulse_search(torch.from_numpy(series).cuda(), cfg.threshold)
    got, n_got = p.fetch()
    ref, n_ref = oracle.sps(series, cfg.widths, cfg.norm_window, cfg.threshold)
    _compare_candidates(got, n_got, ref, n_ref, cfg.threshold, series,
                        cfg.widths, cfg.norm_window)


def _stats_match(x, L):
    p = _plan(x.shape[0], [1, 2, 4], L)
    p.single_pulse_search(torch.from_numpy(x).cuda(), 1e6)
    m2, mad4 = p.stats()
    for k in range(x.shape[0]):
        rm2, rmad4 = oracle.window_stats(x[k], L)
        assert np.array_equal(m2[k], rm2), ("median", k)
        assert np.array_equal(mad4[k], rmad4), ("mad", k)


def test_window_stats_across_spreads():
    """Gaussian windows whose middle half is far narrower, near, and far wider
    than the single-value bins of the one-pass median, and windows whose
    whole range sits near the series minimum: bit-exact against the oracle."""
    L, n = 8192, 3 * 8192 + 1001
    rows = [synth.gaussian_series(2, n, seed=60 + i, mean=m, sd=sd,
                                  event_rate=0.0).numpy()
            for i, (m, sd) in enumerate([(0.0, 3.0), (1000.0, 300.0),
                                         (5e5, 1024.0), (5e5, 2000.0),
                                         (5e5, 2100.0), (5e5, 2300.0),
                                         (5e5, 5000.0), (-7e8, 4e7)])]
    _stats_match(np.concatenate(rows), L)


def test_window_stats_misleading_estimate():
    """Rows built so that an estimate from 32 evenly spaced samples of each
    window is wrong: (a) the sampled positions hold 0 and the rest of the
    window lies 10^4 above, so the median leaves any bin range centred on
    the estimate; (b) thirds at -6000, 0 and +6000 with the sampled positions
    at 0, so the median is right but the MAD (6000) is far outside; (c) two
    equal halves 2000 apart (median between them, every deviation 1000)."""
    L, n = 8192, 3 * 8192 + 1000     # even-length windows
    nwin = oracle.num_windows(n, L)
    noise = synth.gaussian_series(3, n, seed=77, mean=0.0, sd=2.0,
                                  event_rate=0.0).numpy()
    x = np.zeros((3, n), np.int32)
    t = np.arange(n)
    x[0] = 10000 + noise[0]
    x[1] = np.where(t % 3 == 0, -6000, np.where(t % 3 == 1, 0, 6000)) + noise[1]
    x[2] = np.where(t % 2 == 0, 0, 2000)
    for j in range(nwin):
        lo, hi = oracle.window_bounds(n, L, j)
        pos = lo + (np.arange(32, dtype=np.int64) * (hi - lo)) // 32
        x[0, pos] = 0
        x[1, pos] = noise[1, pos]
    _stats_match(x, L)
    # the planted structure really is what the docstring says
    m2, mad4 = oracle.window_stats(x[1], L)
    assert (np.abs(m2) <= 8).all() and (mad4 >= 4 * 5990).all()
    m2, mad4 = oracle.window_stats(x[2], L)
    assert (m2 == 2000).all() and (mad4 == 4000).all()


def test_mad_zero_gives_no_candidates():
    x = np.full((3, 20000), 7, np.int32)
    x[1, 5000] = 10 ** 6
    x[2, ::2] = 9                      # two values: MAD 1
    x[2, 100:104] = 400
    p = _plan(3, [1, 2, 4], 8192)
    p.single_pulse_search(torch.from_numpy(x).cuda(), 5.0)
    got, n = p.fetch()
    ref, n_ref = oracle.sps(x, [1, 2, 4], 8192, 5.0)
    assert n == n_ref
    assert set(got["dm_idx"].tolist()) <= {2}
    m2, mad4 = p.stats()
    assert (mad4[0] == 0).all() and (mad4[1] == 0).all()


def test_truncation_reports_true_count():
    widths = [1, 2, 4]
    x = synth.gaussian_series(4, 1 << 15, seed=5).numpy()
    ref, n_ref = oracle.sps(x, widths, 8192, 3.0)
    assert n_ref > 50
    p = _plan(4, widths, 8192, cap=16)
    p.single_pulse_search(torch.from_numpy(x).cuda(), 3.0)
    with pytest.raises(DdspError) as e:
        p.fetch()
    assert e.value.code == -6
    got, n = p.fetch(allow_truncated=True)
    assert n == n_ref and got.size == 16


def test_argument_errors():
    p = _plan(2, [1, 2], 8192)
    x = torch.zeros((2, 1000), dtype=torch.int32, device="cuda")
    with pytest.raises(DdspError):
        p.single_pulse_search(x, 0.0)
    with pytest.raises(DdspError):
        p.single_pulse_search(x, float("nan"))
    # a window longer than the on-chip limit takes the long mode (no error)
    big = _plan(1, [1, 1024], 0)
    big.single_pulse_search(torch.zeros((1, 60000), dtype=torch.int32,
                                        device="cuda"), 5.0)
    assert big.fetch()[1] == 0          # MAD 0: no candidates


def test_stress_config_full_size_64_rows():
    """2048 x 1048576 int32 series, widths 1..1024, L = 8192, thr 6.5, in the
    launch configuration the benchmark times; the oracle on 64 rows: both
    edges, the 16 rows holding the strongest widest (1024-sample) boxcars,
    and evenly spaced rows.  Window statistics bit-exact and candidate lists
    identical under the tolerance rule, row by row."""
    ndm, n, L, thr = 2048, 1 << 20, 8192, 6.5
    widths = [1 << i for i in range(11)]
    x = synth.gaussian_series(ndm, n, seed=4, device="cuda")
    # no peak merging: the wide events light up ~1/3 of all samples
    p = _plan(ndm, widths, L, cap=1 << 30)
    p.single_pulse_search(x, thr)
    m2, mad4 = p.stats()
    # rows by the largest 1024-sample sum of their input (torch, on the
    # input only): the rows with the widest events
    top = torch.empty(ndm, dtype=torch.int64, device="cuda")
    for r0 in range(0, ndm, 128):
        q = torch.cumsum(x[r0:r0 + 128].to(torch.int64), dim=1)
        top[r0:r0 + 128] = (q[:, 1024:] - q[:, :-1024]).max(dim=1).values
        del q
    wide = torch.argsort(top, descending=True)[:16].cpu().numpy()
    chosen = set([0, 1, 2, 3, ndm - 4, ndm - 3, ndm - 2, ndm - 1])
    chosen |= set(int(k) for k in wide)
    for k in range(5, ndm - 5, 29):          # evenly spaced, up to 64 rows
        if len(chosen) >= 64:
            break
        chosen.add(k)
    rows = sorted(chosen)
    assert len(rows) == 64
    dev, n_total = p.candidates_device()
    assert dev.shape[0] == n_total, "candidate capacity exceeded"
    sel = torch.isin(dev[:, 0], torch.tensor(rows, dtype=torch.int32,
                                             device="cuda"))
    mine_all = dev[sel].cpu().numpy().view(CAND_DTYPE).reshape(-1)
    xh = x[rows].cpu().numpy()
    ref_all, _ = sps_parallel(xh, widths, L, thr, cap=1 << 21)
    for i, k in enumerate(rows):
        rm2, rmad4 = oracle.window_stats(xh[i], L)
        assert np.array_equal(m2[k], rm2) and np.array_equal(mad4[k], rmad4), k
        mine = mine_all[mine_all["dm_idx"] == k].copy()
        mine["dm_idx"] = 0
        ref = ref_all[ref_all["dm_idx"] == i].copy()
        ref["dm_idx"] = 0
        _compare_candidates(mine, mine.size, ref, ref.size, thr,
                            xh[i][None, :], widths, L)
    assert 0.1 * ndm * n < n_total < 0.6 * ndm * n


def test_dense_snr_bits_with_large_sums():
    """The S/N numerator 2*B_y - w*odd is rounded to FP32 exactly once: with
    boxcar sums between 2^24 and 2^30 (where the rounding matters) the dense
    S/N equals, bit for bit, the FP32 product rebuilt from the reported sum
    and the window's exact statistics with the same IEEE operations."""
    rng = np.random.default_rng(7)
    ndm, n, L = 3, 16384, 4096
    widths = [1, 4, 16, 64, 256]
    x = rng.integers(-3_000_000, 3_000_000, size=(ndm, n)).astype(np.int32)
    p = Plan(16, 500.0, -1.0, 1e-3, np.zeros(ndm), widths, nbits=8,
             norm_window=L, cand_capacity=1024)
    bw, bs, bsum = (t.cpu().numpy() for t in p.search_dense(torch.from_numpy(x).cuda()))
    m2, mad4 = p.stats()
    big = 0
    for k in range(ndm):
        for t in range(0, n - 256, 29):
            j = min(t // L, m2.shape[1] - 1)
            wi = int(bw[k, t])
            w, M2, MAD4 = widths[wi], int(m2[k, j]), int(mad4[k, j])
            odd, mfloor = M2 & 1, M2 >> 1
            by = (int(bsum[k, t]) - w * mfloor + 2**31) % 2**32 - 2**31
            big += abs(by) > 2**24
            num = 2 * by - w * odd
            two_sigma = np.float32(1.482602218505602) * np.float32(MAD4) * np.float32(0.5)
            inv = np.float32(1.0) / (two_sigma * np.sqrt(np.float32(w)))
            ref = np.float32(num) * inv
            assert np.float32(bs[k, t]).view(np.uint32) == ref.view(np.uint32), (k, t)
    assert big > 100


@pytest.mark.parametrize("n,L,widths", [
    (300000, 0, [1, 2, 4, 8, 16, 32, 64, 128, 256]),  # one window, whole series
    (200001, 60000, [1, 4, 16, 64, 1024]),            # long windows, ragged last
    (49152, 0, [1, 2, 4]),                             # just past the limit
])
def test_long_windows_dense_match_oracle(n, L, widths):
    """Windows longer than the on-chip limit: exact statistics by a pass over
    global memory, then the search in 8192-sample segments; statistics,
    best widths, S/N and boxcar sums as the oracle's."""
    x = synth.gaussian_series(3, n, seed=n % 1000 + 7).numpy()
    check_dense(x, widths, L)


def test_long_window_candidates_match_oracle():
    """Normalisation over the whole series (L = 0) of 16 beam-length rows."""
    widths = [1 << i for i in range(9)]
    x = synth.gaussian_series(16, 262144, seed=41).numpy()
    p = _plan(16, widths, 0)
    p.single_pulse_search(torch.from_numpy(x).cuda(), 6.0)
    got, n_got = p.fetch()
    ref, n_ref = sps_parallel(x, widths, 0, 6.0)
    assert n_ref > 0
    compare_candidates(got, n_got, ref, n_ref, 6.0, x, widths, 0)
    m2, mad4 = p.stats()
    for k in (0, 15):
        rm2, rmad4 = oracle.window_stats(x[k], 0)
        assert np.array_equal(m2[k], rm2) and np.array_equal(mad4[k], rmad4)
