"""Pins for the CPU oracle: it is checked against things other than itself.

* delay table: exact rational arithmetic of Ch.1 Eq.1 (no floating point),
  the paper's own constant and units (4.14881 ms GHz^2), hand-checkable
  values, and the law's invariants;
* dedispersion: the DM = 0 trial is the channel sum (the "0-DM" series of
  Sec.3.2), an impulse reappears at its delay only, linearity, brute force by
  a dense shift-matrix product on tiny inputs, and an injected pulse peaking
  at its true DM and width;
* median / MAD: numpy's median (a library routine) and a closed form;
* boxcar: numpy's convolution and the constant-series closed form;
* S/N: unit variance on pure noise, MAD = 0 gives no candidates.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2605_03531_b300 import synth

K_EXACT = Fraction("4148.808")


def exact_delay(nchan, f_top, bw, tsamp, dm, c):
    """Delay of Ch.1 Eq.1 in exact rational arithmetic, rounded half away."""
    f_top, bw, tsamp, dm = (Fraction(str(v)) for v in (f_top, bw, tsamp, dm))
    fr = max(f_top, f_top + (nchan - 1) * bw)
    f = f_top + c * bw
    x = K_EXACT * dm * (1 / (f * f) - 1 / (fr * fr)) / tsamp
    return math.floor(x + Fraction(1, 2)) if x >= 0 else -math.floor(-x + Fraction(1, 2))


# ----------------------------------------------------------------- delays
def test_delay_hand_values():
    """Hand-checkable values of the law (both computed in exact arithmetic):
    256 ch over 550-750 MHz at 1.31072 ms: DM 100 at the lowest channel is 481
    samples and DM 255 gives D = 1226; 4096 ch over 300-500 MHz at 81.92 us:
    DM 250 gives D = 89989."""
    d, D = oracle.delay_table(256, 750.0, -0.78125, 1.31072e-3, [100.0, 255.0])
    assert d[0, -1] == 481
    assert D == 1226
    _, D2 = oracle.delay_table(4096, 500.0, -0.048828125, 81.92e-6, [250.0])
    assert D2 == 89989


def test_delay_table_equals_exact_rational():
    """Every entry of a small table equals the exact rational value."""
    nchan, f_top, bw, ts = 64, 750.0, -3.125, 1.31072e-3
    dms = [0.0, 0.5, 7.25, 100.0, 333.3]
    d, _ = oracle.delay_table(nchan, f_top, bw, ts, dms)
    for k, dm in enumerate(dms):
        for c in range(nchan):
            assert d[k, c] == exact_delay(nchan, f_top, bw, ts, dm, c), (k, c)


def golden(name):
    """key -> list of floats from a fixture under tests/golden/."""
    out = {}
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    for line in open(path):
        line = line.split("#", 1)[0].split()
        if line:
            out[line[0]] = [float(v) for v in line[1:]]
    return out


def test_delay_paper_units():
    """The paper writes the law with the constant 4.14881 ms GHz^2 (Ch.1
    Eq.1; tests/golden/dispersion_law.txt).  Evaluated in those units (ms,
    GHz), over the paper's trial-DM range (Sec.2.1), the continuous delay
    matches the oracle's within the 6-figure precision of that constant."""
    g = golden("dispersion_law.txt")
    kc = g["constant_ms_ghz2"][0]
    dm_lo, dm_hi = g["dm_range"]
    nchan, f_top, bw, ts = 128, 1460.0, -1.5625, 1.31072e-3
    for dm in (dm_lo + 10.0, 250.0, dm_hi - 1.0):
        f_ref_ghz = f_top / 1000.0
        for c in (1, 40, 127):
            f_ghz = (f_top + c * bw) / 1000.0
            ms = kc * dm * (1 / f_ghz ** 2 - 1 / f_ref_ghz ** 2)
            samples = ms * 1e-3 / ts
            x = oracle.delay_exact(nchan, f_top, bw, ts, dm, c)
            assert abs(samples - x) <= 2e-6 * abs(x) + 1e-9


def test_delay_invariants():
    nchan, f_top, bw, ts = 256, 750.0, -0.78125, 1.31072e-3
    dms = np.linspace(0, 500, 41)
    d, D = oracle.delay_table(nchan, f_top, bw, ts, dms)
    assert (d[0] == 0).all()                       # DM 0: no delay
    assert (d[:, 0] == 0).all()                    # reference channel: no delay
    assert (np.diff(d, axis=0) >= 0).all()         # monotone in DM
    assert (np.diff(d, axis=1) >= 0).all()         # monotone toward low f
    assert D == d.max()
    # linear in DM up to the two roundings
    d2, _ = oracle.delay_table(nchan, f_top, bw, ts, 2 * dms)
    assert np.abs(d2 - 2 * d).max() <= 1


def test_delay_ascending_band():
    """chan_bw > 0: the reference is the last (highest) channel."""
    d, D = oracle.delay_table(32, 400.0, 2.0, 1e-3, [50.0])
    assert d[0, -1] == 0 and d[0, 0] == D > 0
    for c in range(32):
        assert d[0, c] == exact_delay(32, 400.0, 2.0, 1e-3, 50.0, c)


def test_delay_rejects_bad_args():
    with pytest.raises(ValueError):
        oracle.delay_table(16, 500.0, -1.0, 1e-3, [-1.0])
    with pytest.raises(ValueError):
        oracle.delay_table(16, 500.0, 0.0, 1e-3, [1.0])
    with pytest.raises(ValueError):
        oracle.delay_table(16, 500.0, -1.0, 0.0, [1.0])


# ---------------------------------------------------------- dedispersion
def test_dm0_is_channel_sum():
    """I1: the DM = 0 trial equals the plain channel sum (the 0-DM series)."""
    rng = np.random.default_rng(0)
    x = rng.integers(0, 256, size=(700, 48), dtype=np.uint8)
    d, D = oracle.delay_table(48, 500.0, -2.0, 1e-3, [0.0, 30.0])
    out = oracle.dedisperse(x, d)
    nout = 700 - D
    assert np.array_equal(out[0], x[:nout].astype(np.int64).sum(axis=1))


def test_impulse_reappears_at_its_delay():
    """I2: a unit impulse at (c, s0) shows up in trial k at t = s0 - d[k][c]
    and nowhere else."""
    nchan, nin = 32, 600
    dms = np.linspace(0, 80, 9)
    d, D = oracle.delay_table(nchan, 400.0, -1.0, 1e-3, dms)
    nout = nin - D
    for c, s0 in [(0, 50), (31, 500), (17, 333)]:
        x = np.zeros((nin, nchan), dtype=np.uint8)
        x[s0, c] = 1
        out = oracle.dedisperse(x, d)
        for k in range(len(dms)):
            t = s0 - d[k, c]
            expect = np.zeros(nout, dtype=np.int32)
            if 0 <= t < nout:
                expect[t] = 1
            assert np.array_equal(out[k], expect), (c, k)


def test_linearity_uint16():
    """I3: D(a*x + b*y) = a*D(x) + b*D(y) (uint16 inputs kept in range)."""
    rng = np.random.default_rng(1)
    x = rng.integers(0, 1000, size=(900, 20), dtype=np.uint16)
    y = rng.integers(0, 1000, size=(900, 20), dtype=np.uint16)
    d, _ = oracle.delay_table(20, 450.0, -5.0, 1e-3, [0.0, 12.0, 40.0])
    lhs = oracle.dedisperse((3 * x + 7 * y).astype(np.uint16), d)
    rhs = 3 * oracle.dedisperse(x, d).astype(np.int64) + 7 * oracle.dedisperse(y, d)
    assert np.array_equal(lhs, rhs)


def test_brute_force_shift_matrix_tiny():
    """I5: on tiny inputs, every trial equals a dense product with 0/1 shift
    matrices S_c (S_c[t, s] = 1 iff s = t + d[k][c]), built by enumeration."""
    rng = np.random.default_rng(2)
    for nchan in (1, 2, 3, 4):
        for nin in (17, 40, 64):
            dms = np.arange(0, 6, dtype=np.float64) * 3.0
            d, D = oracle.delay_table(nchan, 300.0, -8.0, 1e-3, dms)
            if nin - D <= 0:
                continue
            x = rng.integers(0, 256, size=(nin, nchan), dtype=np.uint8)
            out = oracle.dedisperse(x, d)
            nout = nin - D
            for k in range(len(dms)):
                acc = np.zeros(nout, dtype=np.int64)
                for c in range(nchan):
                    S = np.zeros((nout, nin), dtype=np.int64)
                    for t in range(nout):
                        S[t, t + d[k, c]] = 1
                    acc += S @ x[:, c].astype(np.int64)
                assert np.array_equal(out[k], acc)


def test_dedisperse_at_matches_full():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 256, size=(300, 16), dtype=np.uint8)
    d, _ = oracle.delay_table(16, 500.0, -4.0, 1e-3, [0.0, 9.0, 25.0])
    out = oracle.dedisperse(x, d)
    for k in range(3):
        for t in (0, 7, out.shape[1] - 1):
            assert oracle.dedisperse_at(x, d, k, t) == out[k, t]


def test_injected_pulse_peaks_at_true_dm_and_width():
    """I4 (the injection test of Sec.2.4): the 256-channel block with one
    pulse at DM 100, width 4, gives its strongest candidate at DM index 100
    and width 4."""
    cfg = synth.config1()
    x = synth.filterbank(cfg, 16384).numpy()
    d, D = oracle.delay_table(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp,
                              cfg.dm_list())
    assert D == 1226
    # a band of DMs around the pulse keeps this test quick
    ks = np.arange(90, 111)
    series = oracle.dedisperse(x, d[ks])
    cands, n = oracle.sps(series, cfg.widths, cfg.norm_window, cfg.threshold)
    assert n > 0
    best = cands[np.argmax(cands["snr"])]
    assert ks[best["dm_idx"]] == 100
    assert cfg.widths[best["w_idx"]] == 4
    assert abs(best["t"] - 8000) <= 1
    assert best["snr"] > 30


# -------------------------------------------------------------- statistics
@pytest.mark.parametrize("n", [1, 2, 7, 8, 1001, 4096])
def test_median_mad_vs_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.integers(-5000, 5000, size=n).astype(np.int32)
    m2, mad4 = oracle.median_mad(x)
    med = np.median(x.astype(np.float64))
    assert m2 == 2 * med
    assert mad4 == 4 * np.median(np.abs(x - med))


def test_median_mad_closed_form():
    """Alternating +a/-a: median 0, MAD a."""
    a = 37
    x = np.array([a, -a] * 500, dtype=np.int32)
    assert oracle.median_mad(x) == (0, 4 * a)
    # constant series: MAD 0
    assert oracle.median_mad(np.full(9, 12, np.int32)) == (24, 0)


def test_window_layout():
    """n_win = max(1, floor(n/L)); the last window runs to the end."""
    assert oracle.num_windows(10, 8192) == 1
    assert oracle.num_windows(20000, 8192) == 2
    assert oracle.window_bounds(20000, 8192, 1) == (8192, 20000)
    assert oracle.window_bounds(5, 0, 0) == (0, 5)
    rng = np.random.default_rng(5)
    x = rng.integers(0, 100, size=20000).astype(np.int32)
    m2, mad4 = oracle.window_stats(x, 8192)
    assert m2[1] == 2 * np.median(x[8192:])


def test_boxcar_vs_convolution_and_constant():
    rng = np.random.default_rng(6)
    x = rng.integers(-1000, 1000, size=500).astype(np.int32)
    for w in (1, 2, 4, 32, 64):
        ref = np.convolve(x.astype(np.int64), np.ones(w, dtype=np.int64), "valid")
        assert np.array_equal(oracle.boxcar(x, w), ref)
    c = np.full(100, 17, np.int32)
    assert (oracle.boxcar(c, 8) == 8 * 17).all()


def test_snr_unit_variance_on_noise():
    """Width-1 S/N of Gaussian noise has mean ~0 and sd ~1 (MAD*1.4826 is
    the Gaussian sigma)."""
    x = synth.gaussian_series(1, 1 << 16, seed=11, event_rate=0.0).numpy()[0]
    m2, mad4 = oracle.median_mad(x)
    s = np.array([oracle.snr(int(v), 1, m2, mad4) for v in x[:20000]])
    n = s.size
    assert abs(s.mean()) < 3 / math.sqrt(n) + 0.01
    assert abs(s.std() - 1.0) < 3 / math.sqrt(n) + 0.01


def test_sps_noise_and_degenerate():
    x = synth.gaussian_series(2, 1 << 15, seed=12, event_rate=0.0).numpy()
    _, n = oracle.sps(x, [1, 2, 4, 8], 8192, 7.0)
    assert n == 0
    # MAD = 0 -> S/N = 0 -> no candidate, even with a spike
    c = np.full((1, 1000), 5, np.int32)
    c[0, 500] = 10 ** 6
    _, n0 = oracle.sps(c, [1, 2], 0, 1.0)
    assert n0 == 0


def test_sps_best_width_and_ties():
    """A clean boxcar event of width 8 on an alternating baseline: the best
    width is 8 and the event is found at its start."""
    n = 4096
    x = np.array([10, -10] * (n // 2), dtype=np.int32)
    x[1000:1008] += 200
    cands, cnt = oracle.sps(x, [1, 2, 4, 8, 16], 0, 10.0)
    best = cands[np.argmax(cands["snr"])]
    assert best["t"] == 1000 and best["w_idx"] == 3
    wi, s = oracle.best_at(x, 0, [1, 2, 4, 8, 16], 1000)
    assert wi == 3 and abs(s - best["snr"]) < 1e-12


# ----------------------------------------------------------------- unpack
@pytest.mark.parametrize("dtype,shape", [(np.uint8, (37, 19)),
                                         (np.uint16, (5, 64)),
                                         (np.uint8, (1, 1))])
def test_unpack_is_numpy_transpose(dtype, shape):
    """Time-major spectra -> channel-major rows: numpy's transpose (a
    library routine) of the same array."""
    rng = np.random.default_rng(3)
    x = rng.integers(0, np.iinfo(dtype).max + 1, size=shape).astype(dtype)
    assert np.array_equal(oracle.unpack(x), np.ascontiguousarray(x.T))
