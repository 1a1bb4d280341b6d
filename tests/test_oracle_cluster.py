"""Pins of the oracle's peaks filter and DM-time clustering (Sec.2.1) to
things other than itself.

* DBSCAN: the core points, the partition of the core points into clusters
  and the noise points equal scikit-learn's DBSCAN (Chebyshev metric on
  integer-scaled coordinates, so its eps-ball is the oracle's rectangle);
  border points, which DBSCAN may give to any adjacent cluster, must sit
  next to a core point of their cluster, and the oracle's canonical choice
  (the adjacent cluster with the smallest label) is checked too.  With
  min_pts = 1 the clusters are the connected components of the
  neighbourhood graph (networkx).  Hand-built chains and borders pin the
  boundary cases (spacing exactly eps, eps + 1, a border between two
  clusters, min_pts - 1 neighbours).
* Peaks filter: hand-built lists with known answers (exact ties, a stronger
  neighbour exactly on and just outside the stencil edge), and invariants a
  plausible slip breaks: the strongest candidate always stays, half-size 0
  keeps everything, a larger stencil keeps a subset, one isolated event
  keeps exactly its peak.
* The whole step on well separated synthetic events returns one cluster per
  event whose strongest member is the event's centre.
"""
import itertools

import networkx as nx
import numpy as np
import pytest

import oracle
from paper_2605_03531_b300 import synth

C32 = oracle.CAND32_DTYPE


def cands(rows):
    """rows: (k, t, w_idx, snr) tuples -> candidate records."""
    c = np.zeros(len(rows), dtype=C32)
    for i, (k, t, w, s) in enumerate(rows):
        c[i] = (k, t, w, s)
    return c


def sorted_points(c):
    o = np.lexsort((c["t"], c["dm_idx"]))
    return c[o]


# ------------------------------------------------------------------- DBSCAN
def _sk_dbscan(k, t, eps_dm, eps_t, min_pts):
    from sklearn.cluster import DBSCAN
    X = np.stack([k.astype(np.float64) * eps_t, t.astype(np.float64) * eps_dm], 1)
    db = DBSCAN(eps=float(eps_dm * eps_t), min_samples=min_pts,
                metric="chebyshev").fit(X)
    core = np.zeros(k.size, dtype=bool)
    core[db.core_sample_indices_] = True
    return db.labels_, core


def _neighbours(k, t, i, eps_dm, eps_t):
    return np.nonzero((np.abs(k.astype(np.int64) - int(k[i])) <= eps_dm)
                      & (np.abs(t.astype(np.int64) - int(t[i])) <= eps_t))[0]


@pytest.mark.parametrize("seed,eps_dm,eps_t,min_pts", [
    (1, 2, 6, 3), (2, 1, 1, 2), (3, 4, 20, 5), (4, 3, 3, 4), (5, 6, 40, 8)])
def test_dbscan_matches_sklearn(seed, eps_dm, eps_t, min_pts):
    c = synth.candidate_list(64, 4000, 5, 12, seed, dm_half=(1, 6),
                             t_half=(1, 30), noise=300)
    p = sorted_points(c)
    k, t = p["dm_idx"], p["t"]
    lab = oracle.dbscan(k, t, eps_dm, eps_t, min_pts)
    sk_lab, sk_core = _sk_dbscan(k, t, eps_dm, eps_t, min_pts)
    counts = np.array([_neighbours(k, t, i, eps_dm, eps_t).size
                       for i in range(k.size)])
    core = counts >= min_pts
    assert np.array_equal(core, sk_core)
    # noise: exactly the points with no core neighbour
    assert np.array_equal(lab == -1, sk_lab == -1)
    # the partition of the core points
    pairs = {}
    for i in np.nonzero(core)[0]:
        a, b = int(lab[i]), int(sk_lab[i])
        assert pairs.setdefault(a, b) == b
    assert len(set(pairs.values())) == len(pairs)
    # labels are the smallest core index of each cluster
    for a in pairs:
        members = np.nonzero(core & (lab == a))[0]
        assert a == members.min()
    # border points: next to a core point of their cluster, smallest label
    for i in np.nonzero(~core & (lab >= 0))[0]:
        nb = _neighbours(k, t, i, eps_dm, eps_t)
        adj = sorted({int(lab[j]) for j in nb if core[j]})
        assert adj and lab[i] == adj[0]
    assert k.size > 500 and core.sum() > 50 and (lab == -1).sum() > 10


def test_dbscan_min_pts_one_is_connected_components():
    c = synth.candidate_list(48, 3000, 4, 10, 11, dm_half=(1, 4),
                             t_half=(1, 12), noise=200)
    p = sorted_points(c)
    k, t = p["dm_idx"], p["t"]
    lab = oracle.dbscan(k, t, 2, 5, 1)
    g = nx.Graph()
    g.add_nodes_from(range(k.size))
    for i in range(k.size):
        for j in _neighbours(k, t, i, 2, 5):
            if j > i:
                g.add_edge(i, int(j))
    for comp in nx.connected_components(g):
        comp = sorted(comp)
        assert all(lab[i] == comp[0] for i in comp)
    assert (lab >= 0).all()


def test_dbscan_hand_chains_and_borders():
    # a row of points 3 samples apart: one cluster with eps_t = 3, none with 2
    k = np.zeros(6, np.uint32)
    t = np.arange(6, dtype=np.uint32) * 3
    assert list(oracle.dbscan(k, t, 0, 3, 2)) == [0] * 6
    assert list(oracle.dbscan(k, t, 0, 2, 2)) == [-1] * 6
    # min_pts = 3: the two ends have 2 neighbours (border points), so the
    # first core point, and the cluster's label, is index 1
    assert list(oracle.dbscan(k, t, 0, 3, 3)) == [1] * 6
    assert list(oracle.dbscan(k, t, 0, 3, 4)) == [-1] * 6
    # DM axis: rows 0 and 2 are neighbours only with eps_dm >= 2
    k2 = np.array([0, 2], np.uint32)
    t2 = np.array([5, 5], np.uint32)
    assert list(oracle.dbscan(k2, t2, 1, 0, 2)) == [-1, -1]
    assert list(oracle.dbscan(k2, t2, 2, 0, 2)) == [0, 0]
    # a border point between two clusters joins the smaller label
    # (eps_t 3, min_pts 4): t = 0..3 and 9..12 are core, t = 6 has only
    # 3 neighbours (3, 6, 9) and touches a core point of each cluster
    t3 = np.array([0, 1, 2, 3, 6, 9, 10, 11, 12], np.uint32)
    k3 = np.zeros(9, np.uint32)
    lab = oracle.dbscan(k3, t3, 0, 3, 4)
    assert list(lab) == [0, 0, 0, 0, 0, 5, 5, 5, 5]
    with pytest.raises(ValueError):
        oracle.dbscan(np.array([0, 0], np.uint32), np.array([3, 3], np.uint32), 1, 1, 1)


def test_cluster_reps_hand():
    lab = np.array([0, 0, -1, 3, 3, 3, 0])
    s = np.array([5, 7, 99, 4, 6, 6, 7], np.float32)
    rep = oracle.cluster_reps(lab, s)
    assert rep[0] == 1 and rep[3] == 4          # ties go to the smaller index
    assert (rep[[1, 2, 4, 5, 6]] == -1).all()


# -------------------------------------------------------------- peaks filter
def test_peaks_hand_cases():
    # centre (10, 100) S/N 9 with width index 1 (half-size 3): a stronger
    # candidate exactly on the stencil corner removes it; just outside does not
    half = [1, 3]
    on = cands([(10, 100, 1, 9.0), (13, 97, 0, 9.5)])
    assert list(oracle.peaks(on, half)) == [False, True]
    off_t = cands([(10, 100, 1, 9.0), (13, 96, 0, 9.5)])
    assert list(oracle.peaks(off_t, half)) == [True, True]
    off_k = cands([(10, 100, 1, 9.0), (14, 100, 0, 9.5)])
    assert list(oracle.peaks(off_k, half)) == [True, True]
    # the stencil is the candidate's own: the weak one (half 3) sees the
    # strong one 2 samples away, the strong one (half 1) does not reach it
    asym = cands([(0, 50, 1, 8.0), (0, 52, 0, 12.0)])
    assert list(oracle.peaks(asym, half)) == [False, True]
    # exact ties: the one earlier in (dm_idx, t) order stays; (5, 20) sees
    # only (5, 21), which it precedes, and (4, 22) precedes (5, 21)
    tie = cands([(5, 20, 0, 7.0), (5, 21, 0, 7.0), (4, 22, 0, 7.0)])
    assert list(oracle.peaks(tie, [1])) == [True, False, True]
    tie2 = cands([(5, 20, 0, 7.0), (5, 21, 0, 7.0)])
    assert list(oracle.peaks(tie2, [1])) == [True, False]
    with pytest.raises(ValueError):
        oracle.peaks(cands([(0, 0, 2, 7.0)]), [1, 1])


def test_peaks_invariants():
    c = synth.candidate_list(128, 20000, 6, 25, 21, dm_half=(1, 10),
                             t_half=(1, 60), noise=400, quantum=0.25)
    half = np.array([1, 2, 4, 8, 16, 32], np.int32)
    keep = oracle.peaks(c, half)
    assert keep[np.argmax(c["snr"])]
    assert oracle.peaks(c, np.zeros(6, np.int32)).all()
    keep_big = oracle.peaks(c, 2 * half)
    assert not (keep_big & ~keep).any()
    assert keep_big.sum() < keep.sum() < c.size
    # deciding a subset answers the same as deciding everything
    idx = np.arange(0, c.size, 7)
    assert np.array_equal(oracle.peaks(c, half, idx), keep[idx])


def test_peaks_single_event_keeps_its_peak():
    # one event; every stencil at least as large as the event, so only the
    # centre (the unique maximum) survives
    c = synth.candidate_list(200, 5000, 3, 1, 31, dm_half=(5, 5),
                             t_half=(9, 9), thr=1.0)
    keep = oracle.peaks(c, [20, 20, 20])
    kept = c[keep]
    assert kept.size == 1 and kept["snr"][0] == c["snr"].max()


# ------------------------------------------------------------- whole step
def test_peaks_cluster_recovers_separated_events():
    ndm, nsamp, ne = 256, 200000, 12
    u = synth.uniform_np(np.arange(8 * ne, dtype=np.uint64), 40).reshape(ne, 8)
    centres = {(int(u[e, 0] * ndm), int(u[e, 1] * nsamp)) for e in range(ne)}
    # the generator's centres must be far apart for this pin (checked)
    cs = sorted(centres)
    for a, b in itertools.combinations(cs, 2):
        assert abs(a[0] - b[0]) > 30 or abs(a[1] - b[1]) > 600
    c = synth.candidate_list(ndm, nsamp, 4, ne, 40, dm_half=(3, 8),
                             t_half=(10, 200), thr=6.5, snr_range=(20, 40))
    pk, lab, reps = oracle.peaks_cluster(c, [2, 2, 2, 2], 12, 250, 1)
    got = sorted((int(pk["dm_idx"][r]), int(pk["t"][r])) for r in reps)
    assert got == cs
