"""Batched multi-beam search: one persistent dedispersion launch over uneven
beams (replayed from a CUDA graph, with an autotuned tile), or the per-beam
interleaved mode, gives every beam exactly what its plan gives alone, and
matches the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import Batch, Plan, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _plan(cfg, cap=1 << 18):
    return Plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
                cfg.widths, nbits=8, norm_window=cfg.norm_window,
                cand_capacity=cap)


def _block(cfg, plan):
    nin = cfg.nsamp_out + plan.max_delay
    x = synth.noise_u8(nin, cfg.nchan, cfg.seed, device="cuda")
    synth.inject_pulses(x, cfg.pulses, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.seed)
    return x


def small_mix(n=10, seed=13):
    return synth.config3(nbeams=n, seed=seed, nsamp_range=(8192, 24576),
                         nchan_choices=(256, 256, 512, 1024),
                         dm_hi_choices=(20.0, 60.0, 150.0),
                         ndm_choices=(16, 37, 64, 128))


def _same_candidates(a, b):
    assert a.size == b.size
    for f in ("dm_idx", "t", "w_idx"):
        assert np.array_equal(a[f], b[f])
    assert np.array_equal(a["snr"], b["snr"])   # same kernel, same arithmetic


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_plain_per_beam(use_graph):
    cfgs = small_mix()
    plans = [_plan(c) for c in cfgs]
    blocks = [_block(c, p) for c, p in zip(cfgs, plans)]
    ref_series, ref_cands = [], []
    for c, p, x in zip(cfgs, plans, blocks):
        s = p.dedisperse(x)
        p.single_pulse_search(s, c.threshold)
        ref_series.append(s.clone())
        ref_cands.append(p.fetch()[0])
    batch = Batch(plans, [x.shape[0] for x in blocks])
    for b, x in enumerate(blocks):
        batch.ingest(b, x)
    for rep in range(3):                       # direct, capture + replay, replay
        for s in batch.series:
            s.fill_(-1)
        batch.run(7.0, use_graph=use_graph)
        batch.check()
        for b in range(len(cfgs)):
            assert torch.equal(batch.series[b], ref_series[b]), (rep, b)
            _same_candidates(plans[b].fetch()[0], ref_cands[b])


def test_batch_autotune_keeps_results():
    cfgs = small_mix(6, seed=17)
    plans = [_plan(c) for c in cfgs]
    blocks = [_block(c, p) for c, p in zip(cfgs, plans)]
    batch = Batch(plans, [x.shape[0] for x in blocks])
    for b, x in enumerate(blocks):
        batch.ingest(b, x)
    batch.run(7.0, use_graph=False)
    before = [s.clone() for s in batch.series]
    ms, best = batch.autotune(reps=1)
    assert best >= 0 and ms[best] > 0
    assert all(m < 0 or m >= ms[best] for m in ms)
    batch.run(7.0, use_graph=True)
    batch.run(7.0, use_graph=True)
    batch.check()
    for b in range(len(cfgs)):
        assert torch.equal(batch.series[b], before[b])


def test_batch_beam_matches_oracle():
    cfgs = small_mix(4, seed=19)
    plans = [_plan(c) for c in cfgs]
    blocks = [_block(c, p) for c, p in zip(cfgs, plans)]
    batch = Batch(plans, [x.shape[0] for x in blocks])
    for b, x in enumerate(blocks):
        batch.ingest(b, x)
    batch.run(7.0, use_graph=True)
    batch.check()
    for b in (0, 3):
        d = plans[b].delays()
        ref = oracle.dedisperse(blocks[b].cpu().numpy(), d)
        assert np.array_equal(batch.series[b].cpu().numpy(), ref)
        got, n = plans[b].fetch()
        rc, rn = oracle.sps(ref, cfgs[b].widths, cfgs[b].norm_window, 7.0)
        keys = {(int(c["dm_idx"]), int(c["t"])) for c in got}
        rkeys = {(int(c["dm_idx"]), int(c["t"])) for c in rc}
        for k in keys ^ rkeys:   # only events at the threshold may differ
            _, s = oracle.best_at(ref[k[0]], cfgs[b].norm_window, cfgs[b].widths, k[1])
            assert abs(s - 7.0) <= 7e-4


def test_batch_full_160_beams_sampled():
    """The full uneven mix: 160 beams, 1024-4096 channels, 65536-262144
    samples, DM grids up to 0-500 with 256-2048 trials, in one persistent
    launch under a CUDA graph; sampled beams against their plain path and
    sampled outputs against the oracle."""
    cfgs = synth.config3()
    plans = [_plan(c, cap=1 << 16) for c in cfgs]
    nins = [c.nsamp_out + p.max_delay for c, p in zip(cfgs, plans)]
    batch = Batch(plans, nins)
    for b, (c, p) in enumerate(zip(cfgs, plans)):
        x = _block(c, p)
        batch.ingest(b, x)
        del x
    batch.run(7.0, use_graph=True)
    batch.run(7.0, use_graph=True)
    batch.check()
    rng = np.random.default_rng(3)
    for b in rng.choice(len(cfgs), 3, replace=False):
        c, p = cfgs[b], plans[b]
        x = _block(c, p)
        s = p.dedisperse(x)
        assert torch.equal(batch.series[b], s), b
        xh = x.cpu().numpy()
        d = p.delays()
        for k, t in zip(rng.integers(0, c.ndm, 40), rng.integers(0, c.nsamp_out, 40)):
            assert int(s[k, t]) == oracle.dedisperse_at(xh, d, int(k), int(t))
        del x, s


def test_batch_per_beam_chunks_and_groups():
    """Beams whose delay spans inside a DM tile differ by ~40x share one
    step: the fine beams stage up to the tile's chunk limit in the main
    launch, the coarse one goes to the second launch with a narrower DM
    tile, and every beam stays exact for several limits."""
    coarse = synth.config3(nbeams=1, seed=23, nsamp_range=(8192, 8192),
                           nchan_choices=(256,), dm_hi_choices=(100.0,),
                           ndm_choices=(64,))
    fine = synth.config3(nbeams=2, seed=29, nsamp_range=(8192, 16384),
                         nchan_choices=(1024,), dm_hi_choices=(10.0,),
                         ndm_choices=(128,))
    cfgs = coarse + fine
    plans = [_plan(c) for c in cfgs]
    blocks = [_block(c, p) for c, p in zip(cfgs, plans)]
    ref = [p.dedisperse(x).clone() for p, x in zip(plans, blocks)]
    refc = []
    for c, p, r in zip(cfgs, plans, ref):
        p.single_pulse_search(r, c.threshold)
        refc.append(p.fetch()[0])
    batch = Batch(plans, [x.shape[0] for x in blocks])
    for b, x in enumerate(blocks):
        batch.ingest(b, x)
    for cap in (8, 3, 1):
        batch.set_tile(16, 8, cap, 2)
        t = [batch.beam_tile(b) for b in range(len(cfgs))]
        # spans per 16-trial tile: ~8500 samples (coarse), ~440 (fine)
        assert t[0]["group"] == 1 and t[0]["dm_tile"] < 16, (cap, t)
        assert t[1]["group"] == t[2]["group"] == 0
        assert t[1]["chan_chunk"] == t[2]["chan_chunk"] >= min(cap, 3)
        assert all(x["chan_chunk"] >= 1 for x in t)
        for s_ in batch.series:
            s_.fill_(-1)
        batch.run(7.0, use_graph=True)
        batch.run(7.0, use_graph=True)
        batch.check()
        for b in range(len(cfgs)):
            assert torch.equal(batch.series[b], ref[b]), (cap, b)
            _same_candidates(plans[b].fetch()[0], refc[b])


def test_batch_autotune_with_two_groups_keeps_results():
    cfgs = (synth.config3(nbeams=2, seed=41, nsamp_range=(8192, 8192),
                          nchan_choices=(256,), dm_hi_choices=(100.0,),
                          ndm_choices=(64,))
            + small_mix(4, seed=43))
    plans = [_plan(c) for c in cfgs]
    blocks = [_block(c, p) for c, p in zip(cfgs, plans)]
    ref = [p.dedisperse(x).clone() for p, x in zip(plans, blocks)]
    batch = Batch(plans, [x.shape[0] for x in blocks])
    for b, x in enumerate(blocks):
        batch.ingest(b, x)
    batch.set_tile(16, 8, 8, 2)
    assert any(batch.beam_tile(b)["group"] == 1 for b in range(len(cfgs)))
    ms, best = batch.autotune(reps=1)     # candidates with and without a split
    assert best >= 0 and ms[best] > 0
    batch.run(7.0, use_graph=True)
    batch.run(7.0, use_graph=True)
    batch.check()
    for b in range(len(cfgs)):
        assert torch.equal(batch.series[b], ref[b]), b


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_per_beam_mode_equals_plain(use_graph):
    """The per-beam interleaved mode (each beam's rows interleaved into the
    batch's one staging area, then its plan's default tile) reproduces every
    beam's series and candidates; set_tile returns to the persistent mode,
    which still agrees."""
    cfgs = small_mix(8, seed=17)
    plans = [_plan(c) for c in cfgs]
    blocks = [_block(c, p) for c, p in zip(cfgs, plans)]
    ref_series, ref_cands = [], []
    for c, p, x in zip(cfgs, plans, blocks):
        s = p.dedisperse(x)
        p.single_pulse_search(s, c.threshold)
        ref_series.append(s.clone())
        ref_cands.append(p.fetch()[0])
    batch = Batch(plans, [x.shape[0] for x in blocks])
    for b, x in enumerate(blocks):
        batch.ingest(b, x)
    assert batch.get_mode() == Batch.PERSISTENT
    batch.set_mode(Batch.PER_BEAM)
    assert batch.get_mode() == Batch.PER_BEAM
    for rep in range(3):
        for s_ in batch.series:
            s_.fill_(-1)
        batch.run(7.0, use_graph=use_graph)
        batch.check()
        for b in range(len(cfgs)):
            assert torch.equal(batch.series[b], ref_series[b]), (rep, b)
            _same_candidates(plans[b].fetch()[0], ref_cands[b])
    batch.set_tile(16, 8, 8, 2)
    assert batch.get_mode() == Batch.PERSISTENT
    for s_ in batch.series:
        s_.fill_(-1)
    batch.run(7.0, use_graph=use_graph)
    batch.check()
    for b in range(len(cfgs)):
        assert torch.equal(batch.series[b], ref_series[b]), b


def test_batch_mode_refused_for_unknown_value():
    cfgs = small_mix(2, seed=19)
    plans = [_plan(c) for c in cfgs]
    batch = Batch(plans, [c.nsamp_out + p.max_delay for c, p in zip(cfgs, plans)])
    from paper_2605_03531_b300 import DdspError
    with pytest.raises(DdspError):
        batch.set_mode(7)
    assert batch.get_mode() == Batch.PERSISTENT
