"""Host side of the streaming search: the seeded arrival schedule, the
continuous-batching loop and the real-time limit search, run against a fake
server on a simulated clock (no GPU).  The fake enforces the same rules as
the library's server: at most one block per beam waiting for a step, a step takes the
waiting block of the beams pushed first, a block's results can be read only
while it is one of the beam's two latest stepped blocks."""
import math

import numpy as np
import pytest

from paper_2605_03531_b300 import synth
from paper_2605_03531_b300.serve import ServingLoop, realtime_limit

T = synth.BLOCK_PERIOD_S


class SimClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeServer:
    """Step time = overhead + per_beam * beams, on the simulated clock."""

    def __init__(self, clock, nbeams, overhead=2e-3, per_beam=5e-3):
        self.clock = clock
        self.overhead, self.per_beam = overhead, per_beam
        self.pushed = [0] * nbeams
        self.processed = [0] * nbeams
        self.push_seq = {}
        self.nseq = 0
        self.steps = []          # (t_done, [(beam, block)])
        self.busy_until = 0.0
        self.step_of = {}
        self.fetched = []
        self.max_waiting = 1

    def push(self, beam, x, stream=None):
        j = self.pushed[beam]
        assert x == (beam, j)
        if j >= 1 and self.processed[beam] < j:
            return False
        self.push_seq[(beam, j)] = self.nseq
        self.nseq += 1
        self.pushed[beam] = j + 1
        return True

    def step(self, thr, max_beams_in_step=0, stream=None):
        ready = [b for b in range(len(self.pushed)) if self.processed[b] < self.pushed[b]]
        ready.sort(key=lambda b: self.push_seq[(b, self.processed[b])])
        if max_beams_in_step > 0:
            ready = ready[:max_beams_in_step]
        if not ready:
            return -1, []
        start = max(self.clock(), self.busy_until)
        self.busy_until = start + self.overhead + self.per_beam * len(ready)
        members = []
        for b in ready:
            members.append((b, self.processed[b]))
            self.step_of[(b, self.processed[b])] = len(self.steps)
            self.processed[b] += 1
        self.steps.append((self.busy_until, members))
        return len(self.steps) - 1, ready

    def done(self, sid):
        return self.clock() >= self.steps[sid][0]

    def fetch(self, beam, block, allow_truncated=False):
        assert self.processed[beam] - 2 <= block < self.processed[beam]
        assert self.done(self.step_of[(beam, block)])
        self.fetched.append((beam, block))
        return np.zeros(0), beam + block, block * 100


def _run(nbeams, nblocks, per_beam, max_beams_in_step=0, arrivals=None,
         time_limit=None, overhead=2e-3, max_inflight=1, min_batch=1,
         max_wait=0.0):
    clock = SimClock()
    srv = FakeServer(clock, nbeams, overhead=overhead, per_beam=per_beam)
    arr = arrivals if arrivals is not None else synth.arrival_times(nbeams, nblocks, seed=5)
    loop = ServingLoop(srv, list(range(nbeams)), lambda i, k: (i, k), 7.0,
                       max_beams_in_step=max_beams_in_step, clock=clock,
                       sleep=clock.sleep, max_inflight=max_inflight,
                       min_batch=min_batch, max_wait=max_wait)
    return loop.run(arr, time_limit=time_limit), srv


def test_minimum_batch_waits_at_most_max_wait():
    """Steps wait for 4 pushed blocks unless the oldest has waited 60 ms:
    every block completes, steps are larger than without the minimum, and
    no block waits for its step much beyond the limit."""
    # 256 beams: about 11 blocks arrive in 60 ms
    res, srv = _run(256, 3, per_beam=5e-4, min_batch=4, max_wait=0.06)
    base, _ = _run(256, 3, per_beam=5e-4)
    assert np.isfinite(res.latency).all()
    assert sum(res.step_sizes) == 256 * 3
    assert np.mean(res.step_sizes) > np.mean(base.step_sizes)
    small = [n for n in res.step_sizes if n < 4]
    assert len(small) < len(res.step_sizes) // 4
    # a block's latency: its wait (<= 60 ms plus one step in flight) and
    # its own step
    assert res.latency.max() < 0.06 + 2 * (2e-3 + 64 * 5e-4) + 0.01


def test_arrival_schedule():
    a = synth.arrival_times(64, 12, seed=5)
    assert a.shape == (64, 12)
    assert np.array_equal(a, synth.arrival_times(64, 12, seed=5))
    assert not np.array_equal(a, synth.arrival_times(64, 12, seed=6))
    assert (np.diff(a, axis=1) >= 0).all()
    # block 0: phase U[0, T) plus an exponential delay
    big = synth.arrival_times(4000, 6, seed=9)
    k = np.arange(6)[None, :] * T
    e = big - k
    assert (e >= 0).all()
    phase_free = big[:, 1:] - big[:, :-1]           # T + e_k - e_{k-1} (mostly)
    assert abs(np.median(phase_free) - T) < 0.01
    # jitter: the first block's delay beyond its phase has mean ~ 50 ms
    ph = synth.uniform_np(np.arange(4000, dtype=np.uint64) + np.uint64(1 << 44), 9) * T
    d0 = big[:, 0] - ph
    assert abs(d0.mean() - 0.05) < 0.004 and d0.min() >= 0


def test_every_block_completes_once_in_order():
    res, srv = _run(24, 6, per_beam=5e-3)
    assert np.isfinite(res.latency).all() and (res.latency > 0).all()
    done = {}
    for t, members in srv.steps:
        for b, j in members:
            assert (b, j) not in done
            done[(b, j)] = t
    assert len(done) == 24 * 6
    for b in range(24):
        ts = [done[(b, j)] for j in range(6)]
        assert ts == sorted(ts)
    assert sorted(srv.fetched) == sorted(done)
    assert res.ncand[3, 2] == 5       # what the fake reported
    assert sum(res.step_sizes) == 24 * 6


def test_batching_keeps_up_where_per_beam_steps_fall_behind():
    # 40 beams x 25 ms = 1.0 s of work per period plus per-step overhead
    # 150 ms: batched steps amortise the overhead, one-beam steps cannot
    batched, _ = _run(40, 8, per_beam=25e-3, overhead=0.15)
    plain, _ = _run(40, 8, per_beam=25e-3, overhead=0.15, max_beams_in_step=1)
    assert batched.percentile(99) < T
    assert plain.percentile(99) > T
    assert max(batched.step_sizes) > 1 and set(plain.step_sizes) == {1}


def test_overload_shows_in_latency():
    ok, _ = _run(20, 10, per_beam=10e-3)
    over, _ = _run(20, 10, per_beam=90e-3)      # 1.8 s of work per 1.34 s
    assert ok.percentile(99) < T < over.percentile(99)
    # latencies grow along the run when the server cannot keep up
    assert np.nanmean(over.latency[:, -1]) > np.nanmean(over.latency[:, 1])


def test_missing_block_stops_at_time_limit():
    arr = synth.arrival_times(6, 5, seed=5)
    arr[2, 3] = math.inf                       # this block never arrives
    res, srv = _run(6, 5, per_beam=5e-3, arrivals=arr, time_limit=10 * T)
    assert np.isnan(res.latency[2, 3:]).all()   # the beam stalls behind it
    others = np.delete(res.latency, 2, axis=0)
    assert np.isfinite(others).all()
    assert srv.pushed[2] == 3


def test_refused_push_is_an_error():
    clock = SimClock()
    srv = FakeServer(clock, 2)
    srv.push = lambda beam, x, stream=None: False
    loop = ServingLoop(srv, [0, 1], lambda i, k: (i, k), 7.0, clock=clock,
                       sleep=clock.sleep)
    with pytest.raises(RuntimeError):
        loop.run(synth.arrival_times(2, 2, seed=1))


def test_schedule_rows_must_match_beams():
    clock = SimClock()
    loop = ServingLoop(FakeServer(clock, 2), [0, 1], lambda i, k: (i, k), 7.0,
                       clock=clock, sleep=clock.sleep)
    with pytest.raises(ValueError):
        loop.run(np.zeros((3, 2)))


def test_realtime_limit_bisection():
    calls = []

    def p99(n):
        calls.append(n)
        return math.inf if n > 300 else 0.004 * n   # not admitted above 300

    n, seen = realtime_limit(p99, 64, 320, 16, T)
    assert n == 288 and len(calls) <= 6 and seen[304] == math.inf
    n, seen = realtime_limit(lambda n: 0.006 * n, 64, 320, 16, T)
    assert n == 208                      # 0.006*208 = 1.248 < 1.342 < 1.344
    assert realtime_limit(lambda n: 2.0, 64, 320, 16, T)[0] == 0


def test_two_steps_in_flight_read_results_in_time():
    """With a second step queued the loop reads each finished block while
    the fake server still holds its results (it asserts the window), and
    every block completes once."""
    res, srv = _run(30, 8, per_beam=20e-3, overhead=0.05, max_inflight=2)
    assert np.isfinite(res.latency).all()
    assert sorted(srv.fetched) == sorted((b, j) for b in range(30) for j in range(8))
    assert max(len(m) for _, m in srv.steps) > 1
