"""Streaming server: every block of every beam gives, bit for bit, what the
plain path (ddsp_dedisperse + ddsp_single_pulse_search) gives on the same
input window, whether the beam is stepped alone or with others, in any
interleaving of pushes and steps; the ring's back-pressure, admission by
free device memory and the result-window rules hold; the serving loop runs
against the real server."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import DdspError, Plan, Server, _lib, build, synth
from paper_2605_03531_b300.serve import DeviceStager, ServingLoop

pytestmark = pytest.mark.gpu

NCHAN, B, NBLK = 256, 4096, 6
WIDTHS = [1, 2, 4, 8, 16, 32, 64]
THR = 6.0


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    build.build()


def _plan(cap=1 << 16):
    # 300-500 MHz, 81.92 us, DM 0-10 in 64 trials: D = 3602 samples
    return Plan(NCHAN, 500.0, -200.0 / NCHAN, 81.92e-6,
                np.linspace(0.0, 10.0, 64), WIDTHS, nbits=8, norm_window=2048,
                cand_capacity=cap)


def _stream(seed, nblk=NBLK):
    """One beam's continuous time-major stream with pulses across block
    boundaries."""
    x = synth.noise_u8(nblk * B, NCHAN, seed, device="cuda")
    pulses = [synth.Pulse(dm=dm, width=w, amp=a, t0=t0) for dm, w, a, t0 in
              ((3.0, 4, 30.0, B - 700), (7.5, 16, 12.0, 2 * B + 900),
               (5.0, 1, 60.0, 4 * B - 50))]
    synth.inject_pulses(x, pulses, 500.0, -200.0 / NCHAN, 81.92e-6, seed)
    return x


def _reference(plan, srv, x, j):
    """Plain path on block j's window: input global samples
    [j*B - D16 - C, (j+1)*B) with zeros before the stream."""
    pre = srv.first_delay + srv.carry
    xz = torch.cat([torch.zeros((pre, NCHAN), dtype=torch.uint8, device="cuda"),
                    x[: (j + 1) * B]])
    win = xz[j * B: j * B + srv.series_cols + plan.max_delay]
    s = plan.dedisperse(win)
    assert s.shape[1] == srv.series_cols
    plan.single_pulse_search(s, THR)
    c, _ = plan.fetch()
    return s, c[c["t"] < B]


def _same(got, ref):
    assert got.size == ref.size
    for f in ("dm_idx", "t", "w_idx", "snr"):
        assert np.array_equal(got[f], ref[f]), f


def test_server_shape():
    p = _plan()
    srv = Server(p, B, 4)
    assert srv.carry == 64 and srv.series_cols == B + 64
    assert srv.first_delay == (p.max_delay + 15) // 16 * 16
    assert srv.ring_samples == (-(-srv.first_delay // B) + 1) * B
    assert srv.max_waiting == 1
    t = srv.get_tile()
    assert B % t["time_tile"] == 0 and t["chan_chunk"] >= 1
    srv.close()


@pytest.mark.parametrize("mode", ["relayout", "interleaved"])
def test_server_blocks_equal_plain_path_in_any_mix(mode):
    """Both dedispersion modes; the interleaved one with 2 staging slots,
    so a step of three beam-blocks takes two groups."""
    plan, ref_plan = _plan(), _plan()
    srv = Server(plan, B, 4)
    if mode == "interleaved":
        srv.set_mode(Server.INTERLEAVED, 2)
        assert srv.get_mode() == (Server.INTERLEAVED, 2)
    beams = [srv.admit() for _ in range(3)]
    xs = [_stream(100 + i) for i in range(3)]
    refs = [[_reference(ref_plan, srv, xs[i], j) for j in range(NBLK)]
            for i in range(3)]
    pushed = [0, 0, 0]
    stepped = [0, 0, 0]
    got_any = 0
    series_checked = 0

    def push(i):
        assert srv.push(beams[i], xs[i][pushed[i] * B:(pushed[i] + 1) * B])
        pushed[i] += 1

    def step_and_check(expect):
        nonlocal got_any, series_checked
        sid, sb = srv.step(THR)
        assert sorted(sb) == sorted(beams[i] for i in expect)
        torch.cuda.synchronize()
        assert srv.done(sid)
        for i in expect:
            j = stepped[i]
            s_ref, c_ref = refs[i][j]
            try:      # the series of the step's last group stay in their slots
                s_got = srv.series(beams[i])
            except DdspError as e:
                assert e.code == _lib.DDSP_E_STATE
                s_got = None
            if s_got is not None:
                assert torch.equal(s_got, s_ref), (i, j)
                series_checked += 1
            c, n, t0 = srv.fetch(beams[i], j)
            assert t0 == j * B - srv.first_delay - srv.carry
            _same(c, c_ref)
            got_any += n
            stepped[i] += 1

    push(0); step_and_check([0])                      # alone
    push(1); push(2); step_and_check([1, 2])           # two together
    push(0); push(1)
    # beam 0's next block waits until a step took the one before it
    assert not srv.push(beams[0], xs[0][2 * B:3 * B])
    step_and_check([0, 1])
    push(0); step_and_check([0])
    push(2); push(1); push(0); step_and_check([0, 1, 2])
    while min(pushed) < NBLK:
        for i in range(3):
            if pushed[i] < NBLK and pushed[i] - stepped[i] < 1:
                push(i)
        step_and_check([i for i in range(3) if pushed[i] > stepped[i]])
    while max(p - s for p, s in zip(pushed, stepped)) > 0:
        step_and_check([i for i in range(3) if pushed[i] > stepped[i]])
    assert got_any > 0 and series_checked >= NBLK
    srv.check()
    srv.close()


def test_server_beam_alone_equals_beam_in_mix():
    plan = _plan()
    x = _stream(7)
    solo = Server(plan, B, 1)
    b = solo.admit()
    alone = []
    for j in range(4):
        solo.push(b, x[j * B:(j + 1) * B])
        solo.step(THR)
        alone.append(solo.fetch(b, j)[0])
    solo.close()
    mix = Server(plan, B, 5)
    bs = [mix.admit() for _ in range(5)]
    others = [_stream(20 + i, 4) for i in range(4)]
    for j in range(4):
        for i, ob in enumerate(bs[1:]):
            mix.push(ob, others[i][j * B:(j + 1) * B])
        mix.push(bs[0], x[j * B:(j + 1) * B])
        _, sb = mix.step(THR)
        assert len(sb) == 5
        _same(mix.fetch(bs[0], j)[0], alone[j])
    mix.close()


def test_server_step_limit_takes_oldest_push():
    plan = _plan()
    srv = Server(plan, B, 3)
    bs = [srv.admit() for _ in range(3)]
    x = _stream(3, 1)
    for b in (bs[2], bs[0], bs[1]):
        srv.push(b, x)
    order = []
    for _ in range(3):
        _, sb = srv.step(THR, max_beams_in_step=1)
        order += sb
    assert order == [bs[2], bs[0], bs[1]]
    assert srv.step(THR) == (-1, [])
    srv.close()


def test_server_fetch_window_and_errors():
    plan = _plan()
    srv = Server(plan, B, 1)
    b = srv.admit()
    x = _stream(5, 4)
    with pytest.raises(DdspError) as e:
        srv.fetch(b, 0)                    # not stepped yet
    assert e.value.code == _lib.DDSP_E_STATE
    for j in range(4):
        srv.push(b, x[j * B:(j + 1) * B])
        srv.step(THR)
    srv.fetch(b, 3)
    srv.fetch(b, 2)
    with pytest.raises(DdspError) as e:
        srv.fetch(b, 1)                    # its buffer was reused
    assert e.value.code == _lib.DDSP_E_STATE
    with pytest.raises(DdspError):         # not 16-byte aligned
        srv.push(b, x.view(-1)[1:1 + B * NCHAN].view(B, NCHAN))
    with pytest.raises(DdspError):
        srv.step(0.0)
    with pytest.raises(DdspError) as e:
        srv.admit()                        # max_beams reached
    assert e.value.code == _lib.DDSP_E_RANGE
    srv.evict(b)
    assert srv.admit() == b
    srv.close()


def test_server_admission_by_free_memory():
    plan = _plan()
    probe = Server(plan, B, 8)
    need = probe.beam_bytes
    torch.cuda.synchronize()
    # free memory with a server's own buffers (series slots) in place
    free, _ = torch.cuda.mem_get_info()
    probe.close()
    torch.cuda.synchronize()
    # leave room for exactly one more beam (plus slack for allocator rounding)
    srv = Server(plan, B, 8, hbm_reserve_bytes=free - need - need // 2)
    srv.admit()
    with pytest.raises(DdspError) as e:
        srv.admit()
    assert e.value.code == _lib.DDSP_E_NOMEM
    srv.close()


def test_server_rejects_bad_shapes():
    plan = _plan()
    with pytest.raises(DdspError):
        Server(plan, 4000, 2)          # not a multiple of the time tile
    with pytest.raises(DdspError):
        Server(plan, 48, 2)            # shorter than the boxcar carry
    with pytest.raises(DdspError):
        Server(plan, B, 0)


def test_serving_loop_on_the_server():
    """A short real-time run: 6 beams, 5 blocks each at a 40 ms period;
    every block completes, its candidates equal the plain path's."""
    plan, ref_plan = _plan(), _plan()
    srv = Server(plan, B, 6)
    beams = [srv.admit() for _ in range(6)]
    xs = [_stream(300 + i, 5) for i in range(6)]
    host = [x.cpu().pin_memory() for x in xs]
    compute = torch.cuda.Stream()
    stager = DeviceStager(4, (B, NCHAN), compute)
    got = {}

    def keep(i, k, cands, t_start):
        got[(i, k)] = (cands, t_start)

    loop = ServingLoop(srv, beams, lambda i, k: host[i][k * B:(k + 1) * B], THR,
                       stager=stager, compute_stream=compute, on_candidates=keep)
    arr = synth.arrival_times(6, 5, period=0.04, seed=11, jitter_mean=0.005)
    res = loop.run(arr, time_limit=60.0)
    assert np.isfinite(res.latency).all() and (res.latency > 0).all()
    assert sum(res.step_sizes) == 30
    for i in (0, 5):
        for k in range(5):
            _, c_ref = _reference(ref_plan, srv, xs[i], k)
            _same(got[(i, k)][0], c_ref)
    srv.check(compute)
    srv.close()


def test_server_mode_arguments():
    srv = Server(_plan(), B, 2)
    for mode, slots in ((2, 4), (1, 0), (1, 17)):
        with pytest.raises(DdspError):
            srv.set_mode(mode, slots)
    assert srv.get_mode() == (Server.RELAYOUT, 0)
    srv.set_mode(Server.INTERLEAVED, 3)
    srv.set_mode(Server.RELAYOUT)
    assert srv.get_mode()[0] == Server.RELAYOUT
    srv.close()


@pytest.mark.parametrize("mode", ["relayout", "interleaved"])
def test_c5_shape_blocks_match_oracle(mode):
    """The streaming shape itself (4096 channels, 1024 DM trials over 0-250,
    widths 1..256, L 8192, 16384-sample blocks): ten blocks of one beam,
    stepped together with a second beam, past the point where its ring
    wraps.  Block j's series (C + B columns) is bit-exact against the
    oracle's dedispersion of the input window [j*B - D16 - C, (j+1)*B -
    (D16 - D)) with zeros before the stream, and its candidates (start
    times t < B) equal the oracle's search of those columns under the
    tolerance rule (for the first blocks, whose windows reach before the
    stream and light up ~5e5 candidates, on a few DM rows); both stored by
    tests/golden/make_golden.py."""
    import os
    from parity import (C5_EARLY_ROWS, GOLDEN, compare_to_stored,
                        read_candidates, read_digests, row_digests)
    cfg, x = synth.config5_stream(10)
    Bc = cfg.nsamp_out
    plan = Plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
                cfg.widths, nbits=8, norm_window=cfg.norm_window,
                cand_capacity=1 << 23)
    srv = Server(plan, Bc, 2)
    if mode == "interleaved":
        srv.set_mode(Server.INTERLEAVED, 2)
    assert srv.ring_samples < 10 * Bc          # the ring wraps in the run
    beam, other = srv.admit(), srv.admit()
    noise = synth.noise_u8(Bc, cfg.nchan, 77, device="cuda")
    xd = x.cuda()
    stored = read_digests(os.path.join(GOLDEN, "c5_series_rows.txt"))
    ref_all = read_candidates(os.path.join(GOLDEN, "c5_candidates.txt"))
    D16, Cc, D = srv.first_delay, srv.carry, plan.max_delay
    d = plan.delays()
    xh = x.numpy()
    xz = np.concatenate([np.zeros((D16 + Cc, cfg.nchan), np.uint8), xh])
    for j in range(10):
        assert srv.push(beam, xd[j * Bc:(j + 1) * Bc])
        assert srv.push(other, noise)
        _, sb = srv.step(cfg.threshold)
        assert sorted(sb) == sorted([beam, other])
        torch.cuda.synchronize()
        s = srv.series(beam).cpu().numpy()
        assert s.shape == (cfg.ndm, Cc + Bc)
        mine = row_digests(s, 16)
        bad = [16 * g for g in range(len(mine))
               if mine[g] != stored[f"{j}:{16 * g}"]]
        assert not bad, (j, bad[:8])
        got, n, t0 = srv.fetch(beam, j)
        assert t0 == j * Bc - D16 - Cc
        if j * Bc < D16 + Cc:
            # the window reaches before the stream: the stored candidates
            # are those of a few DM rows
            got = got[np.isin(got["dm_idx"], C5_EARLY_ROWS)]
        win = xz[j * Bc: j * Bc + Cc + Bc + D]

        def width_check(k, t, wg, s_ref):
            row = oracle.dedisperse(win, d[k:k + 1])[0]
            w = cfg.widths[wg]
            Bsum = int(row[t:t + w].astype(np.int64).sum())
            m2, mad4 = oracle.window_stats(row, cfg.norm_window)
            jj = min(t // cfg.norm_window, m2.size - 1)
            sn = oracle.snr(Bsum, w, m2[jj], mad4[jj])
            assert abs(sn - s_ref) <= 1e-5 * abs(s_ref), ("width", j, k, t)

        compare_to_stored(got, ref_all[ref_all["block"] == j], cfg.threshold,
                          width_check)
    srv.check()
    srv.close()


def test_server_interleave_on_unaligned_ring_positions():
    """Widths up to 8 make the carry 8 samples, so the ring position of a
    block's window is a multiple of 8 but not of 16: the interleave then
    takes its 4-sample path instead of the 16-byte one.  Every block's
    series and candidates equal the plain path's."""
    widths = [1, 2, 4, 8]

    def plan():
        return Plan(NCHAN, 500.0, -200.0 / NCHAN, 81.92e-6,
                    np.linspace(0.0, 10.0, 64), widths, nbits=8,
                    norm_window=2048, cand_capacity=1 << 16)

    srv_plan, ref_plan = plan(), plan()
    srv = Server(srv_plan, B, 2)
    srv.set_mode(Server.INTERLEAVED, 2)
    assert srv.carry == 8
    beams = [srv.admit() for _ in range(2)]
    xs = [_stream(300 + i) for i in range(2)]
    unaligned = 0
    for j in range(NBLK):
        for i in range(2):
            assert srv.push(beams[i], xs[i][j * B:(j + 1) * B])
        sid, sb = srv.step(THR)
        torch.cuda.synchronize()
        assert sorted(sb) == sorted(beams)
        for i in range(2):
            s_ref, c_ref = _reference(ref_plan, srv, xs[i], j)
            s_got = srv.series(beams[i])
            assert torch.equal(s_got, s_ref), (i, j)
            c, n, t0 = srv.fetch(beams[i], j)
            _same(c, c_ref)
            unaligned += (t0 % 16) != 0
    assert unaligned > 0
    srv.close()
