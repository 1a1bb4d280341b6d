"""Write the stored oracle results the full-size GPU parity tests compare
against.  Calls only the CPU oracle (``oracle``) and the seeded input
generators (``synth``); nothing here runs on a GPU or loads the CUDA library.

    python tests/golden/make_golden.py c2 c5     (about half an hour on 8 cores)

c2: the single full-size beam (4096 channels, 262144 + D samples, 1024 DM
    trials over 0-250, widths 1..256, L 8192, threshold 7): a digest of every
    dedispersed row, and every candidate whose oracle S/N is at least
    7*(1 - 1e-4) (the exempt band of the tolerance rule included).
c5: ten 16384-sample blocks of one streaming beam of that shape
    (synth.config5_stream): block j's result is the plain path on the input
    window [j*B - D16 - C, (j+1)*B - (D16 - D)) with zeros before the stream
    (D16 = D rounded up to 16, C = the widest boxcar minus one rounded up to
    4), i.e. C + B output columns whose candidates are reported for start
    times t < B; a digest of every 16 dedispersed rows and the candidates
    (for the first blocks, whose windows reach before the stream, those of
    a few DM rows).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle                                     # noqa: E402
from paper_2605_03531_b300 import synth           # noqa: E402
from parity import (THR_EXEMPT, C5_EARLY_ROWS, row_digests,  # noqa: E402
                    sps_parallel, write_candidates, write_digests,
                    STORED_DTYPE)


def _stored(c, block=0, keep=None):
    if keep is not None:
        c = c[keep]
    out = np.zeros(c.size, STORED_DTYPE)
    out["block"] = block
    for f in ("dm_idx", "t", "w_idx", "snr"):
        out[f] = c[f]
    return out


def make_c2():
    t0 = time.time()
    cfg = synth.config2()
    d, D = oracle.delay_table(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp,
                              cfg.dm_list())
    nin = cfg.nsamp_out + D
    x = synth.filterbank(cfg, nin).numpy()
    series = oracle.dedisperse(x, d)
    assert series.shape == (cfg.ndm, cfg.nsamp_out)
    head = [f"c2: {cfg.name}, nin {nin}, D {D}, seed {cfg.seed}, "
            f"{len(cfg.pulses)} pulses",
            "oracle.dedisperse of synth.filterbank(config2(), 262144 + D)",
            "key = DM-trial row, value = blake2b-64 of its int32 LE bytes",
            "written by tests/golden/make_golden.py c2"]
    write_digests(os.path.join(HERE, "c2_series_rows.txt"), head,
                  list(enumerate(row_digests(series))))
    thr_lo = cfg.threshold * (1.0 - THR_EXEMPT)
    c, n = sps_parallel(series, cfg.widths, cfg.norm_window, thr_lo)
    write_candidates(
        os.path.join(HERE, "c2_candidates.txt"),
        [f"c2: oracle.sps(series, widths 1..256, L {cfg.norm_window}, "
         f"thr 7*(1-1e-4)) -> {n} records",
         "columns: block(0) dm_idx t w_idx snr(FP64 oracle)",
         "written by tests/golden/make_golden.py c2"], _stored(c))
    print(f"c2: {n} candidates, {time.time() - t0:.0f} s", flush=True)


def make_c5(nblocks=10):
    t0 = time.time()
    cfg, x = synth.config5_stream(nblocks)
    x = x.numpy()
    B = cfg.nsamp_out
    d, D = oracle.delay_table(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp,
                              cfg.dm_list())
    D16 = -(-D // 16) * 16
    C = -(-(max(cfg.widths) - 1) // 4) * 4
    pre = D16 + C
    warm = -(-pre // B)     # blocks whose window reaches before the stream
    xz = np.concatenate([np.zeros((pre, cfg.nchan), np.uint8), x])
    thr_lo = cfg.threshold * (1.0 - THR_EXEMPT)
    digests, cands = [], []
    for j in range(nblocks):
        win = xz[j * B: j * B + C + B + D]
        s = oracle.dedisperse(win, d)
        assert s.shape == (cfg.ndm, C + B)
        for g, dg in enumerate(row_digests(s, 16)):
            digests.append((f"{j}:{16 * g}", dg))
        c, _ = sps_parallel(s, cfg.widths, cfg.norm_window, thr_lo)
        keep = c["t"] < B
        if j < warm:
            keep &= np.isin(c["dm_idx"], C5_EARLY_ROWS)
        cands.append(_stored(c, j, keep))
        print(f"c5 block {j}: {int((c['t'] < B).sum())} candidates, "
              f"{int(keep.sum())} kept, {time.time() - t0:.0f} s", flush=True)
    head = [f"c5: {cfg.name}, B {B}, D {D}, D16 {D16}, C {C}, seed {cfg.seed}, "
            f"{len(cfg.pulses)} pulses",
            "block j = oracle.dedisperse of the input window "
            "[j*B - D16 - C, (j+1)*B - (D16 - D)), zeros before the stream",
            "key = block:first row of 16, value = blake2b-64 of the 16 rows",
            "written by tests/golden/make_golden.py c5"]
    write_digests(os.path.join(HERE, "c5_series_rows.txt"), head, digests)
    allc = np.concatenate(cands)
    write_candidates(
        os.path.join(HERE, "c5_candidates.txt"),
        [f"c5: oracle.sps per block (C + B columns, L {cfg.norm_window}, "
         f"thr 7*(1-1e-4)), start times t < B kept -> {allc.size} records",
         f"blocks 0..{warm - 1} (windows reaching before the stream): DM rows "
         f"{list(C5_EARLY_ROWS)} only",
         "columns: block dm_idx t(column of the block's series) w_idx snr",
         "written by tests/golden/make_golden.py c5"], allc)


if __name__ == "__main__":
    what = sys.argv[1:] or ["c2", "c5"]
    oracle.set_threads(os.cpu_count() or 1)
    if "c2" in what:
        make_c2()
    if "c5" in what:
        make_c5()
