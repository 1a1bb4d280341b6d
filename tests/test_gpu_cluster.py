"""GPU parity of the peaks filter and DM-time clustering (Sec.2.1) with the
CPU oracle, on the same seeded candidate records.

Every decision is taken on the same FP32 S/N values on both sides, and the
labelling rule is deterministic, so the sorted peaks, their cluster labels
and the representatives must be identical.  At a million candidates the
oracle decides a sample of the peak flags one by one, and the clustering is
checked through properties that hold at any size.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import Cluster, DdspError, Plan, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def run_gpu(c, ndm, nsamp, half, eps_dm, eps_t, min_pts, cap=None):
    cl = Cluster(ndm, nsamp, cap or max(c.size, 1))
    cl.run(Cluster.to_device(c), half, eps_dm, eps_t, min_pts)
    pk, lab = cl.peaks()
    reps, idx = cl.reps()
    cl.close()
    return pk, lab, reps, idx


def check_parity(c, ndm, nsamp, half, eps_dm, eps_t, min_pts):
    pk, lab, reps, idx = run_gpu(c, ndm, nsamp, half, eps_dm, eps_t, min_pts)
    opk, olab, oreps = oracle.peaks_cluster(c, half, eps_dm, eps_t, min_pts)
    assert pk.size == opk.size
    for f in ("dm_idx", "t", "w_idx", "snr"):
        assert np.array_equal(pk[f], opk[f]), f
    assert np.array_equal(lab.astype(np.int64), olab)
    assert np.array_equal(idx.astype(np.int64), oreps)
    assert np.array_equal(reps, opk[oreps])
    return pk, lab, reps


@pytest.mark.parametrize("ndm,nsamp,nev,noise,quantum,half,eps,min_pts", [
    (64, 5000, 10, 200, 0.0, [1, 2, 4, 8], (2, 6), 3),
    (128, 20000, 30, 1000, 0.25, [2, 4, 8, 16, 32], (3, 20), 4),
    (33, 1001, 6, 100, 1 / 64, [0, 1, 2], (1, 1), 2),          # ties, odd plane
    (256, 65536, 40, 3000, 0.0, [3, 6, 12, 24, 48, 96], (6, 64), 1),
    (16, 40, 3, 60, 0.5, [40, 40], (16, 40), 2),                # stencils > plane
])
def test_parity_with_oracle(ndm, nsamp, nev, noise, quantum, half, eps, min_pts):
    c = synth.candidate_list(ndm, nsamp, len(half), nev, ndm + nsamp,
                             dm_half=(1, max(2, ndm // 8)),
                             t_half=(1, max(2, nsamp // 200)), noise=noise,
                             quantum=quantum)
    assert c.size > 0
    pk, lab, reps = check_parity(c, ndm, nsamp, half, eps[0], eps[1], min_pts)
    assert pk.size < c.size or not any(half)


def test_half_zero_keeps_all_and_min_pts_one_clusters_all():
    c = synth.candidate_list(40, 3000, 3, 300, 5, dm_half=(1, 4),
                             t_half=(1, 20))
    pk, lab, reps = check_parity(c, 40, 3000, [0, 0, 0], 2, 8, 1)
    assert pk.size == c.size and (lab >= 0).all()


def test_empty_single_and_counts():
    cl = Cluster(8, 100, 16)
    empty = torch.zeros((16, 4), dtype=torch.int32, device="cuda")
    cl.run(empty, [1], 1, 1, 1, n=0)
    pk, lab = cl.peaks()
    reps, idx = cl.reps()
    assert pk.size == 0 and reps.size == 0
    c = np.zeros(3, dtype=synth.CAND_DTYPE)
    c[0] = (3, 50, 0, 9.0)
    c[1] = (3, 52, 0, 8.0)
    c[2] = (7, 99, 0, 7.5)
    d = Cluster.to_device(c)
    # a device counter selects the first records only
    cnt = torch.tensor([1], dtype=torch.int32, device="cuda")
    cl.run(d, [1], 1, 1, 1, n=3, count=cnt.data_ptr())
    pk, lab = cl.peaks()
    assert pk.size == 1 and pk["t"][0] == 50 and lab[0] == 0
    cl.run(d, [2], 1, 1, 1)
    pk, lab = cl.peaks()
    assert list(pk["t"]) == [50, 99] and list(lab) == [0, 1]
    # truncated fetch keeps the true count
    cl.run(d, [0], 1, 1, 1)
    with pytest.raises(DdspError) as e:
        cl.peaks(cap=2)
    assert e.value.code == -6
    cl.close()


def test_bad_records_and_arguments():
    cl = Cluster(8, 100, 4)
    c = np.zeros(2, dtype=synth.CAND_DTYPE)
    c[0] = (1, 10, 0, 9.0)
    c[1] = (1, 10, 0, 8.0)                      # repeated (dm_idx, t)
    cl.run(Cluster.to_device(c), [1], 1, 1, 1)
    with pytest.raises(DdspError) as e:
        cl.peaks()
    assert e.value.code == -1
    c[1] = (8, 10, 0, 8.0)                      # outside the plane
    cl.run(Cluster.to_device(c), [1], 1, 1, 1)
    with pytest.raises(DdspError):
        cl.reps()
    c[1] = (2, 10, 3, 8.0)                      # width index >= nwidths
    cl.run(Cluster.to_device(c), [1], 1, 1, 1)
    with pytest.raises(DdspError):
        cl.peaks()
    ok = Cluster.to_device(c[:1])
    for args in ([-1], 1, 1, 1), ([1], -1, 1, 1), ([1], 1, 1, 0):
        with pytest.raises(DdspError):
            cl.run(ok, *args)
    big = torch.zeros((5, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(DdspError):
        cl.run(big, [1], 1, 1, 1)               # more than the capacity
    with pytest.raises(DdspError):
        Cluster(0, 100, 4)
    cl.close()


def test_chained_on_search_output_matches_explicit_call():
    cfg = synth.config1()
    x = synth.filterbank(cfg, 16384)
    p = Plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
             cfg.widths, nbits=8, norm_window=cfg.norm_window,
             cand_capacity=1 << 16)
    series = p.dedisperse(x.cuda())
    p.single_pulse_search(series, 5.0)
    half = list(cfg.widths)
    cl = Cluster(cfg.ndm, series.shape[1], 1 << 16)
    cl.run_plan(p, half, 4, 16, 1)
    pk1, lab1 = cl.peaks()
    reps1, _ = cl.reps()
    got, n = p.fetch()
    assert n > 0
    cl.run(Cluster.to_device(got), half, 4, 16, 1)
    pk2, lab2 = cl.peaks()
    reps2, _ = cl.reps()
    assert np.array_equal(pk1, pk2) and np.array_equal(lab1, lab2)
    assert np.array_equal(reps1, reps2) and reps1.size >= 1
    # the injected pulse (DM trial 100) is among the representatives
    assert (np.abs(reps1["dm_idx"].astype(int) - 100) <= 2).any()
    cl.close()
    p.close()


def test_million_candidates_sampled_and_properties():
    ndm, nsamp = 1024, 262144
    half = np.array([1, 2, 4, 8, 16, 32, 64, 128, 256], np.int32)
    eps_dm, eps_t, min_pts = 4, 32, 3
    c = synth.candidate_list(ndm, nsamp, half.size, 3000, 99, dm_half=(1, 30),
                             t_half=(1, 120), noise=200000, quantum=1 / 128)
    assert c.size > 1_000_000
    cl = Cluster(ndm, nsamp, c.size)
    cl.run(Cluster.to_device(c), half, eps_dm, eps_t, min_pts)
    pk, lab = cl.peaks()
    reps, idx = cl.reps()
    cl.close()
    # peak flags of a sample of the input, decided one by one by the oracle
    rng = np.random.default_rng(7)
    sample = rng.choice(c.size, 600, replace=False)
    keep = oracle.peaks(c, half, sample)
    key_pk = pk["dm_idx"].astype(np.int64) * nsamp + pk["t"]
    key_s = c["dm_idx"][sample].astype(np.int64) * nsamp + c["t"][sample]
    assert np.array_equal(np.isin(key_s, key_pk), keep)
    assert np.all(np.diff(key_pk) > 0)
    # DBSCAN properties on a sample of the peaks
    k, t = pk["dm_idx"].astype(np.int64), pk["t"].astype(np.int64)
    row_start = np.searchsorted(k, np.arange(ndm + 1))

    def nbrs(i):
        out = []
        for kk in range(max(0, k[i] - eps_dm), min(ndm - 1, k[i] + eps_dm) + 1):
            a, b = row_start[kk], row_start[kk + 1]
            lo = a + np.searchsorted(t[a:b], t[i] - eps_t)
            hi = a + np.searchsorted(t[a:b], t[i] + eps_t, side="right")
            out.extend(range(lo, hi))
        return np.array(out, dtype=np.int64)

    core = {}

    def is_core(i):
        if i not in core:
            core[i] = nbrs(i).size >= min_pts
        return core[i]

    for i in rng.choice(pk.size, 400, replace=False):
        nb = nbrs(i)
        if is_core(i):
            assert lab[i] >= 0 and lab[i] <= i and lab[lab[i]] == lab[i]
            assert is_core(lab[i])
            for j in nb:
                if is_core(j):
                    assert lab[j] == lab[i]
        else:
            adj = [lab[j] for j in nb if is_core(j)]
            assert lab[i] == (min(adj) if adj else -1)
    # representatives: one per label, the strongest member, ties to the
    # earlier peak, in increasing label order
    labels = np.unique(lab[lab >= 0])
    assert np.array_equal(np.sort(lab[idx]), lab[idx])
    assert np.array_equal(lab[idx], labels)
    order = np.lexsort((np.arange(pk.size), -pk["snr"].astype(np.float64), lab))
    first = np.ones(order.size, bool)
    first[1:] = lab[order][1:] != lab[order][:-1]
    best = order[first & (lab[order] >= 0)]
    assert np.array_equal(np.sort(best), np.sort(idx.astype(np.int64)))
    assert np.array_equal(reps, pk[idx])
