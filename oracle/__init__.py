"""CPU oracle for dedispersion and the boxcar single-pulse search.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package.  The product path (the
CUDA library and its Python binding) never imports, links or runs it, and the
two share no code: only the seeded input generators feed both.

The arithmetic lives in ``oracle.c`` (plain C, FP64 where floating point is
involved); this module is ctypes marshalling around it.  Each wrapper cites
the passage of the paper its C function writes out:

* ``delay_table``   -- dispersion delay law, Ch.1 Eq.1;
* ``dedisperse``    -- brute-force shift-and-sum, Sec.3.2;
* ``window_stats``  -- median / MAD noise estimate, Sec.3.3;
* ``boxcar``, ``sps`` -- boxcar single-pulse search above a threshold, Sec.2.1;
* ``peaks``, ``dbscan``, ``cluster_reps``, ``peaks_cluster`` -- peaks
  filtering with square DM-time stencils, DBSCAN clustering in the DM-time
  plane and the strongest candidate of each cluster, Sec.2.1;
* ``downsample``, ``running_median``, ``dered`` -- downsampling by a user
  factor (Sec.3.2) and running-median de-reddening (Sec.3.3);
* ``ffa``, ``fold_snr`` -- the folding transform by the fast folding
  algorithm and the boxcar search of a folded profile, Sec.3.5;
* ``resample`` -- resampling for the frequency derivatives, Sec.3.4;
* ``rfi_clean`` -- gptool-style bandpass correction and channel / time
  flagging of 8-bit spectra, Sec.2.1.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class Cand(C.Structure):
    _fields_ = [("dm_idx", C.c_int32), ("w_idx", C.c_int32),
                ("t", C.c_int64), ("snr", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_delay_table.restype = C.c_int32
        L.orc_delay_table.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                      P, C.c_int, P]
        L.orc_delay_exact.restype = C.c_double
        L.orc_delay_exact.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_int]
        L.orc_unpack_u8.restype = None
        L.orc_unpack_u8.argtypes = [P, C.c_int64, C.c_int, P]
        L.orc_unpack_u16.restype = None
        L.orc_unpack_u16.argtypes = [P, C.c_int64, C.c_int, P]
        L.orc_dedisperse.restype = C.c_int
        L.orc_dedisperse.argtypes = [P, C.c_int, C.c_int64, C.c_int, P, C.c_int,
                                     C.c_int64, P]
        L.orc_dedisperse_at.restype = C.c_int64
        L.orc_dedisperse_at.argtypes = [P, C.c_int, C.c_int64, C.c_int, P, C.c_int64]
        L.orc_num_windows.restype = C.c_int64
        L.orc_num_windows.argtypes = [C.c_int64, C.c_int64]
        L.orc_window_bounds.restype = None
        L.orc_window_bounds.argtypes = [C.c_int64, C.c_int64, C.c_int64, P, P]
        L.orc_median_mad.restype = None
        L.orc_median_mad.argtypes = [P, C.c_int64, P, P]
        L.orc_window_stats.restype = None
        L.orc_window_stats.argtypes = [P, C.c_int64, C.c_int64, P, P]
        L.orc_boxcar.restype = C.c_int
        L.orc_boxcar.argtypes = [P, C.c_int64, C.c_int, P]
        L.orc_snr.restype = C.c_double
        L.orc_snr.argtypes = [C.c_int64, C.c_int, C.c_int64, C.c_int64]
        L.orc_best_at.restype = C.c_int
        L.orc_best_at.argtypes = [P, C.c_int64, C.c_int64, P, C.c_int, C.c_int64,
                                  C.POINTER(C.c_double)]
        L.orc_sps.restype = C.c_int64
        L.orc_sps.argtypes = [P, C.c_int, C.c_int64, P, C.c_int, C.c_int64,
                              C.c_double, P, C.c_int64]
        L.orc_peaks.restype = C.c_int
        L.orc_peaks.argtypes = [P, P, P, P, C.c_int64, P, C.c_int, P, C.c_int64, P]
        L.orc_dbscan.restype = C.c_int
        L.orc_dbscan.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, P]
        L.orc_cluster_reps.restype = None
        L.orc_cluster_reps.argtypes = [P, P, C.c_int64, P]
        L.orc_downsample.restype = C.c_int
        L.orc_downsample.argtypes = [P, C.c_int64, C.c_int64, P]
        L.orc_running_median_at.restype = C.c_int64
        L.orc_running_median_at.argtypes = [P, C.c_int64, C.c_int64, C.c_int64, P]
        L.orc_running_median_subtract.restype = C.c_int
        L.orc_running_median_subtract.argtypes = [P, C.c_int64, C.c_int64, P]
        L.orc_ffa.restype = C.c_int64
        L.orc_ffa.argtypes = [P, C.c_int64, C.c_int64, P]
        L.orc_fold_snr.restype = C.c_int
        L.orc_fold_snr.argtypes = [P, C.c_int64, C.c_int64, P, C.c_int,
                                   C.c_double, C.POINTER(C.c_double),
                                   C.POINTER(C.c_int64)]
        L.orc_resample.restype = C.c_int64
        L.orc_resample.argtypes = [P, C.c_int64, C.c_double, C.c_double,
                                   C.c_double, C.c_double, P, C.c_int64]
        L.orc_rfi_clean.restype = C.c_int
        L.orc_rfi_clean.argtypes = [P, C.c_int64, C.c_int64, C.c_int, C.c_int,
                                    C.c_int, C.c_int, P, P, P]
        L.orc_set_threads.restype = None
        L.orc_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def set_threads(n: int) -> None:
    """Number of OpenMP threads the DM loop of ``dedisperse`` uses from now
    on (timing only; results do not depend on it)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))
    lib().orc_set_threads(int(n))


def delay_table(nchan, f_top, chan_bw, tsamp, dm_list):
    """Integer delay table d[k][c] and the largest delay D (Ch.1 Eq.1)."""
    dm = np.ascontiguousarray(dm_list, dtype=np.float64)
    d = np.empty((dm.size, nchan), dtype=np.int32)
    D = lib().orc_delay_table(int(nchan), float(f_top), float(chan_bw),
                              float(tsamp), _ptr(dm), int(dm.size), _ptr(d))
    if D < 0:
        raise ValueError("invalid delay-table arguments")
    return d, int(D)


def delay_exact(nchan, f_top, chan_bw, tsamp, dm, c):
    """Unrounded delay in samples for one (DM, channel)."""
    return lib().orc_delay_exact(int(nchan), float(f_top), float(chan_bw),
                                 float(tsamp), float(dm), int(c))


def unpack(x):
    """Time-major [nin][nchan] spectra -> channel-major [nchan][nin]."""
    x = np.ascontiguousarray(x)
    nin, nchan = x.shape
    out = np.empty((nchan, nin), dtype=x.dtype)
    if x.dtype == np.uint8:
        lib().orc_unpack_u8(_ptr(x), nin, nchan, _ptr(out))
    elif x.dtype == np.uint16:
        lib().orc_unpack_u16(_ptr(x), nin, nchan, _ptr(out))
    else:
        raise TypeError("uint8 or uint16 spectra expected")
    return out


def _nbits(x):
    if x.dtype == np.uint8:
        return 8
    if x.dtype == np.uint16:
        return 16
    raise TypeError("uint8 or uint16 spectra expected")


def dedisperse(x, d):
    """Brute-force dedispersion of time-major spectra x[nin][nchan] (Sec.3.2).

    Returns int32 out[ndm][nout], nout = nin - max(d)."""
    x = np.ascontiguousarray(x)
    d = np.ascontiguousarray(d, dtype=np.int32)
    nin, nchan = x.shape
    ndm = d.shape[0]
    nout = nin - int(d.max())
    if nout <= 0:
        raise ValueError("input shorter than the largest delay")
    out = np.empty((ndm, nout), dtype=np.int32)
    rc = lib().orc_dedisperse(_ptr(x), _nbits(x), nin, nchan, _ptr(d), ndm, nout,
                              _ptr(out))
    if rc != 0:
        raise ValueError("dedispersion sum out of int32 range")
    return out


def dedisperse_at(x, d, k, t):
    """One dedispersed sample out[k][t] (same definition as ``dedisperse``)."""
    x = np.ascontiguousarray(x)
    nin, nchan = x.shape
    row = np.ascontiguousarray(d[k], dtype=np.int32)
    v = lib().orc_dedisperse_at(_ptr(x), _nbits(x), nin, nchan, _ptr(row), int(t))
    if v == np.iinfo(np.int64).min:
        raise IndexError("sample outside the input")
    return int(v)


def num_windows(n, L):
    return int(lib().orc_num_windows(int(n), int(L)))


def window_bounds(n, L, j):
    lo, hi = C.c_int64(), C.c_int64()
    lib().orc_window_bounds(int(n), int(L), int(j), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def median_mad(x):
    """(2*median, 4*MAD) of a 1-D int32 array, exact (Sec.3.3)."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    m2, mad4 = C.c_int64(), C.c_int64()
    lib().orc_median_mad(_ptr(x), x.size, C.byref(m2), C.byref(mad4))
    return m2.value, mad4.value


def window_stats(x, L):
    """Per-window (2*median, 4*MAD) arrays of one int32 series."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    nwin = num_windows(x.size, L)
    m2 = np.empty(nwin, dtype=np.int64)
    mad4 = np.empty(nwin, dtype=np.int64)
    lib().orc_window_stats(_ptr(x), x.size, int(L), _ptr(m2), _ptr(mad4))
    return m2, mad4


def boxcar(x, w):
    """B_w(t) = sum_{i<w} x[t+i] for t <= n-w, by direct summation (int64)."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    n = x.size
    out = np.empty(max(n - w + 1, 0), dtype=np.int64)
    if out.size and lib().orc_boxcar(_ptr(x), n, int(w), _ptr(out)) != 0:
        raise OverflowError("boxcar sum leaves int32")
    return out


def snr(B, w, m2, mad4):
    return lib().orc_snr(int(B), int(w), int(m2), int(mad4))


def best_at(x, L, widths, t):
    """(best width index, best S/N) at one sample of one series."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    ws = np.ascontiguousarray(widths, dtype=np.int32)
    s = C.c_double()
    wi = lib().orc_best_at(_ptr(x), x.size, int(L), _ptr(ws), ws.size, int(t),
                           C.byref(s))
    return wi, s.value


CAND_DTYPE = np.dtype([("dm_idx", np.int32), ("w_idx", np.int32),
                       ("t", np.int64), ("snr", np.float64)])


def sps(series, widths, L, thr, cap=None):
    """Boxcar single-pulse search over series[ndm][n] (Sec.2.1).

    Returns (candidates sorted by (dm_idx, t), true count)."""
    series = np.ascontiguousarray(series, dtype=np.int32)
    if series.ndim == 1:
        series = series[None, :]
    ndm, n = series.shape
    ws = np.ascontiguousarray(widths, dtype=np.int32)
    if cap is None:
        cap = 1 << 20
    out = np.zeros(cap, dtype=CAND_DTYPE)
    cnt = lib().orc_sps(_ptr(series), ndm, n, _ptr(ws), ws.size, int(L),
                        float(thr), _ptr(out), int(cap))
    return out[:min(cnt, cap)].copy(), int(cnt)


# ------------------------------------------------ peaks filtering, clustering
# Candidate records as the search emits them: FP32 S/N, so both sides take
# every comparison on the same values.
CAND32_DTYPE = np.dtype([("dm_idx", np.uint32), ("t", np.uint32),
                         ("w_idx", np.uint32), ("snr", np.float32)])


def _cand_fields(c):
    c = np.ascontiguousarray(c)
    return (np.ascontiguousarray(c["dm_idx"], dtype=np.uint32),
            np.ascontiguousarray(c["t"], dtype=np.uint32),
            np.ascontiguousarray(c["w_idx"], dtype=np.uint32),
            np.ascontiguousarray(c["snr"], dtype=np.float32))


def peaks(cands, half, idx=None):
    """Keep flags of the peaks filter (Sec.2.1, square stencils of half-size
    half[w_idx]), for every candidate or for the indices ``idx``."""
    k, t, w, s = _cand_fields(cands)
    hf = np.ascontiguousarray(half, dtype=np.int32)
    n = k.size
    if idx is None:
        m, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        m, ip = idx.size, _ptr(idx)
    keep = np.zeros(max(m, 1), dtype=np.uint8)
    rc = lib().orc_peaks(_ptr(k), _ptr(t), _ptr(w), _ptr(s), n, _ptr(hf),
                         hf.size, ip, m, _ptr(keep))
    if rc != 0:
        raise ValueError("width index or stencil size out of range")
    return keep[:m].astype(bool)


def dbscan(k, t, eps_dm, eps_t, min_pts):
    """DBSCAN labels of points sorted by (k, t): the sorted index of the point
    that started each cluster, -1 for noise."""
    k = np.ascontiguousarray(k, dtype=np.uint32)
    t = np.ascontiguousarray(t, dtype=np.uint32)
    lab = np.empty(max(k.size, 1), dtype=np.int64)
    rc = lib().orc_dbscan(_ptr(k), _ptr(t), k.size, int(eps_dm), int(eps_t),
                          int(min_pts), _ptr(lab))
    if rc != 0:
        raise ValueError("points not sorted and distinct, or bad parameters")
    return lab[:k.size]


def cluster_reps(labels, snr):
    """rep[c]: index of the strongest point with label c (ties to the smaller
    index), -1 where c is not a label."""
    labels = np.ascontiguousarray(labels, dtype=np.int64)
    snr = np.ascontiguousarray(snr, dtype=np.float32)
    rep = np.empty(max(labels.size, 1), dtype=np.int64)
    lib().orc_cluster_reps(_ptr(labels), _ptr(snr), labels.size, _ptr(rep))
    return rep[:labels.size]


def peaks_cluster(cands, half, eps_dm, eps_t, min_pts):
    """The whole step of Sec.2.1 after the search: peaks filtering, the kept
    candidates sorted by (dm_idx, t), DBSCAN labels of those, and the index
    (into the sorted peaks) of each cluster's strongest member, clusters in
    increasing label order.  Returns (peaks, labels, reps)."""
    cands = np.ascontiguousarray(cands)
    keep = peaks(cands, half)
    kept = cands[keep]
    order = np.lexsort((kept["t"], kept["dm_idx"]))
    pk = kept[order]
    labels = dbscan(pk["dm_idx"], pk["t"], eps_dm, eps_t, min_pts)
    rep = cluster_reps(labels, pk["snr"])
    reps = rep[rep >= 0]
    return pk, labels, reps


# ------------------------------------------- downsampling and de-reddening
def downsample(x, f):
    """y[j] = sum of x[j*f .. j*f + f - 1] for j < len(x) // f (Sec.3.2)."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    f = int(f)
    y = np.empty(max(x.size // f, 1) if f >= 1 else 1, dtype=np.int32)
    if lib().orc_downsample(_ptr(x), x.size, f, _ptr(y)) != 0:
        raise OverflowError("factor < 1 or a sum leaves int32")
    return y[:x.size // f]


def running_median(x, h, t):
    """Lower median of x over [t - h, t + h] clamped to the series."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    work = np.empty(max(min(2 * int(h) + 1, x.size), 1), dtype=np.int32)
    return int(lib().orc_running_median_at(_ptr(x), x.size, int(h), int(t),
                                           _ptr(work)))


def dered(x, h):
    """z[t] = x[t] - running median over [t - h, t + h] (Sec.3.3)."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    z = np.empty(max(x.size, 1), dtype=np.int32)
    if lib().orc_running_median_subtract(_ptr(x), x.size, int(h), _ptr(z)) != 0:
        raise OverflowError("h < 0 or a residual leaves int32")
    return z[:x.size]


# ------------------------------------------------------- folding transform
def ffa_rows(n, p):
    """m: the largest power of two with m * p <= n (0 if p > n)."""
    if p < 1 or n < p:
        return 0
    m = 1
    while 2 * m * p <= n:
        m *= 2
    return m


def ffa(x, p):
    """Folding transform F[m][p] (int64) of series x at base period p."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    m = ffa_rows(x.size, int(p))
    if m == 0:
        raise ValueError("p < 1 or the series is shorter than p")
    out = np.empty((m, int(p)), dtype=np.int64)
    lib().orc_ffa(_ptr(x), x.size, int(p), _ptr(out))
    return out


def fold_snr(P, m, widths, sigma):
    """(best width index, best S/N, phase) of one folded profile."""
    P = np.ascontiguousarray(P, dtype=np.int64)
    ws = np.ascontiguousarray(widths, dtype=np.int32)
    s = C.c_double()
    ph = C.c_int64()
    wi = lib().orc_fold_snr(_ptr(P), P.size, int(m), _ptr(ws), ws.size,
                            float(sigma), C.byref(s), C.byref(ph))
    return wi, s.value, ph.value


# ---------------------------------------------------------------- resampling
def resample(x, f0, f1, f2, tsamp):
    """Series resampled for f = f0 + f1 t + f2 t^2 / 2 (Sec.3.4), FP64."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    cap = 2 * x.size + 16
    out = np.empty(cap, dtype=np.float64)
    k = lib().orc_resample(_ptr(x), x.size, float(f0), float(f1), float(f2),
                           float(tsamp), _ptr(out), cap)
    if k < 0:
        raise ValueError("bad resampling arguments")
    return out[:k]


# ---------------------------------------------------------- RFI mitigation
def rfi_clean(x, hw=10, kc=4, kt=3, rounds=2):
    """(cleaned uint8 [nt][nc], channel flags, time flags) of a time-major
    uint8 block (Sec.2.1, gptool style)."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    nt, nc = x.shape
    out = np.empty_like(x)
    fc = np.empty(nc, dtype=np.uint8)
    ft = np.empty(nt, dtype=np.uint8)
    if lib().orc_rfi_clean(_ptr(x), nt, nc, int(hw), int(kc), int(kt),
                           int(rounds), _ptr(out), _ptr(fc), _ptr(ft)) != 0:
        raise ValueError("bad RFI arguments")
    return out, fc.astype(bool), ft.astype(bool)
