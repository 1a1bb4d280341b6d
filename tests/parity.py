"""Helpers the parity tests share: the tolerance rule for candidate lists,
row digests of large outputs, the oracle's search run over row chunks on
several host threads, and the text format of stored oracle results.

Nothing here computes a result of the method: expected values come from
``oracle`` (directly, or from files under ``tests/golden/`` that
``tests/golden/make_golden.py`` writes by calling the oracle)."""
from __future__ import annotations

import hashlib
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle

SNR_RTOL = 1e-5      # S/N relative tolerance against the FP64 oracle
THR_EXEMPT = 1e-4    # events within this fraction of thr of it are exempt

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Streaming blocks whose input window still reaches before the stream's
# first sample (read as zeros) light up hundreds of thousands of candidates
# (the dedispersed series ramps up as channels come in); their stored
# candidates are kept for these DM rows only.
C5_EARLY_ROWS = (0, 682)


def row_digests(a, group=1):
    """blake2b-64 hex digest of each group of `group` consecutive rows of a
    2-D int32 array (little-endian bytes)."""
    a = np.ascontiguousarray(a, dtype="<i4")
    return [hashlib.blake2b(a[r:r + group].tobytes(), digest_size=8).hexdigest()
            for r in range(0, a.shape[0], group)]


def sps_parallel(series, widths, L, thr, cap=None, threads=None):
    """oracle.sps over row chunks on several threads (the C call releases
    the GIL); each row's candidates depend on that row alone, so the
    concatenation in row order is the oracle's list for the whole array."""
    series = np.ascontiguousarray(series, dtype=np.int32)
    ndm = series.shape[0]
    threads = threads or os.cpu_count() or 1
    step = max(1, -(-ndm // (4 * threads)))
    chunks = [(r, min(ndm, r + step)) for r in range(0, ndm, step)]

    def run(rr):
        c, n = oracle.sps(series[rr[0]:rr[1]], widths, L, thr,
                          cap=cap or (1 << 22))
        assert c.size == n, "oracle candidate capacity exceeded"
        c = c.copy()
        c["dm_idx"] += rr[0]
        return c

    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(run, chunks))
    out = np.concatenate(parts) if parts else np.zeros(0, oracle.CAND_DTYPE)
    return out, int(out.size)


def _keys(c, n):
    return c["dm_idx"].astype(np.int64) * (int(n) + 1) + c["t"].astype(np.int64)


def compare_candidates(got, n_got, ref, n_ref, thr, x, widths, L):
    """GPU list vs the oracle's list for series x (numpy [ndm][n]): the same
    (dm_idx, t) pairs except events whose oracle S/N is within THR_EXEMPT*thr
    of thr; S/N within SNR_RTOL; the same best width unless the oracle's S/N
    at the GPU's width equals the best within SNR_RTOL."""
    assert n_got == got.size and n_ref == ref.size
    n = x.shape[1]
    kg, kr = _keys(got, n), _keys(ref, n)
    assert np.unique(kg).size == kg.size, "repeated (dm_idx, t) in the GPU list"
    og, orr = np.argsort(kg, kind="stable"), np.argsort(kr, kind="stable")
    g, r = got[og], ref[orr]
    kg, kr = kg[og], kr[orr]
    common, ig, ir = np.intersect1d(kg, kr, assume_unique=True,
                                    return_indices=True)
    gs = g["snr"][ig].astype(np.float64)
    rs = r["snr"][ir].astype(np.float64)
    bad = np.abs(gs - rs) > SNR_RTOL * np.abs(rs)
    assert not bad.any(), ("S/N", g[ig][bad][:5], r[ir][bad][:5])
    for i in np.nonzero(g["w_idx"][ig] != r["w_idx"][ir])[0]:
        k, t = int(g["dm_idx"][ig[i]]), int(g["t"][ig[i]])
        wg = widths[int(g["w_idx"][ig[i]])]
        B = int(x[k, t:t + wg].astype(np.int64).sum())
        rm2, rmad4 = oracle.window_stats(x[k], L)
        j = min(t // L, max(1, n // L) - 1) if L else 0
        s_w = oracle.snr(B, wg, rm2[j], rmad4[j])
        assert abs(s_w - rs[i]) <= SNR_RTOL * abs(rs[i]), ("width", k, t)
    only = np.concatenate([np.setdiff1d(kg, common, assume_unique=True),
                           np.setdiff1d(kr, common, assume_unique=True)])
    for key in only:
        k, t = int(key // (n + 1)), int(key % (n + 1))
        _, s = oracle.best_at(x[k], L, widths, t)
        assert abs(s - thr) <= THR_EXEMPT * thr, ("not exempt", k, t, s)


def compare_to_stored(got, stored, thr, width_check=None):
    """GPU list vs a stored oracle list taken at threshold thr*(1 - THR_EXEMPT)
    (so it holds every exempt event too).  Every GPU candidate must be
    stored; every stored event with S/N > thr*(1 + THR_EXEMPT) must be found;
    S/N within SNR_RTOL; a different best width is passed to width_check(k,
    t, w_idx_gpu, snr_oracle), which must confirm the tie.  Returns the number
    of exempt events."""
    sk = {(int(c["dm_idx"]), int(c["t"])): c for c in stored}
    gk = {(int(c["dm_idx"]), int(c["t"])): c for c in got}
    assert len(gk) == got.size, "repeated (dm_idx, t) in the GPU list"
    for key, g in gk.items():
        assert key in sk, ("GPU candidate the oracle does not have", key,
                           float(g["snr"]))
        r = sk[key]
        assert abs(float(g["snr"]) - r["snr"]) <= SNR_RTOL * abs(r["snr"]), key
        if int(g["w_idx"]) != int(r["w_idx"]):
            assert width_check is not None, ("best width differs", key)
            width_check(key[0], key[1], int(g["w_idx"]), float(r["snr"]))
    exempt = 0
    for key, r in sk.items():
        if abs(r["snr"] - thr) <= THR_EXEMPT * thr:
            exempt += 1
            continue
        assert key in gk, ("oracle candidate the GPU missed", key, r["snr"])
    return exempt


STORED_DTYPE = np.dtype([("block", np.int64), ("dm_idx", np.int64),
                         ("t", np.int64), ("w_idx", np.int64),
                         ("snr", np.float64)])


def write_candidates(path, header, recs):
    """Text file: '#' header lines, then 'block dm_idx t w_idx snr' rows
    (S/N with 17 significant digits, enough to read back the double)."""
    with open(path, "w") as f:
        for line in header:
            f.write(f"# {line}\n")
        for r in recs:
            f.write(f"{int(r['block'])} {int(r['dm_idx'])} {int(r['t'])} "
                    f"{int(r['w_idx'])} {float(r['snr']):.17g}\n")


def read_candidates(path):
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            b, k, t, w, s = line.split()
            rows.append((int(b), int(k), int(t), int(w), float(s)))
    out = np.zeros(len(rows), STORED_DTYPE)
    if rows:
        a = np.array(rows, dtype=object)
        for i, f in enumerate(STORED_DTYPE.names):
            out[f] = a[:, i].astype(STORED_DTYPE[f])
    return out


def write_digests(path, header, items):
    """Text file: '#' header lines, then 'key digest' rows."""
    with open(path, "w") as f:
        for line in header:
            f.write(f"# {line}\n")
        for key, dg in items:
            f.write(f"{key} {dg}\n")


def read_digests(path):
    out = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, dg = line.split()
            out[key] = dg
    return out
