"""Real-time serving loop over a :class:`Server` (the streaming design of
Sec.2.1 and Ch.3: every beam delivers a block of spectra per period and each
block must be searched before the next one is due).

Continuous batching: blocks are ingested as they arrive (host -> device copy
on a copy stream, then the server's push on the compute stream); whenever no
step is running (and, optionally, once a few blocks wait or the oldest has
waited long enough), one step takes the waiting block of every ready beam
(or only the longest-waiting beam, for the per-beam sequential comparison).  The
latency of a block is the time from its arrival to the moment the host sees
its step complete.

The loop only sequences calls: every step of the search runs in the server's
kernels.  The server, the staging of blocks and the clock are passed in, so
the same loop runs against a fake server and a simulated clock on the CPU.
"""
from __future__ import annotations

import heapq
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class ServeResult:
    latency: np.ndarray            # [beams, blocks] seconds (nan: not done)
    ncand: np.ndarray              # [beams, blocks] candidates found
    step_sizes: list = field(default_factory=list)  # beams per step
    wall: float = 0.0              # seconds from start to the last completion
    busy: float = float("nan")     # device seconds of the pushes and steps
                                   # (with device timing), nan otherwise

    def percentile(self, q):
        v = self.latency[np.isfinite(self.latency)]
        return float(np.percentile(v, q)) if v.size else float("nan")


class DeviceStager:
    """Copies pinned host blocks into a ring of device staging buffers on
    `h2d_stream`; the consumer (the server's push on `compute_stream`) waits
    for the copy, and a staging buffer is reused only after that push ran."""

    def __init__(self, nslots, shape, compute_stream, h2d_stream=None):
        import torch
        self.torch = torch
        self.compute = compute_stream
        self.h2d = h2d_stream or torch.cuda.Stream()
        self.buf = [torch.empty(shape, dtype=torch.uint8, device="cuda")
                    for _ in range(nslots)]
        self.ready = [torch.cuda.Event() for _ in range(nslots)]
        self.free = [torch.cuda.Event() for _ in range(nslots)]
        for e in self.free:
            e.record(self.compute)
        self.next = 0

    def stage(self, host_block):
        """Start the copy; returns (device tensor, slot).  The compute stream
        is made to wait for the copy."""
        s = self.next
        self.next = (s + 1) % len(self.buf)
        with self.torch.cuda.stream(self.h2d):
            self.h2d.wait_event(self.free[s])
            self.buf[s].copy_(host_block, non_blocking=True)
            self.ready[s].record(self.h2d)
        self.compute.wait_event(self.ready[s])
        return self.buf[s], s

    def consumed(self, slot):
        """The push that reads `slot` has been enqueued on the compute
        stream."""
        self.free[slot].record(self.compute)


class ServingLoop:
    """Drive `server` with blocks arriving at given times.

    server: push(beam, x, stream) -> bool, step(threshold, max_beams_in_step,
        stream) -> (step id, beams), done(step id) -> bool,
        fetch(beam, block, allow_truncated) -> (cands, count, t_start),
        max_waiting: blocks a beam may have pushed but not yet stepped
    beams: the server's beam index for each schedule row
    source(i, k): host block k of schedule row i
    stager: stage(host) -> (device block, token), consumed(token); None
        passes the source's block through unchanged
    first_block: the server's block number of schedule column 0 (blocks
        the beams received before this run)
    """

    def __init__(self, server, beams, source, threshold, stager=None,
                 max_beams_in_step=0, max_inflight=1, compute_stream=None,
                 clock=time.monotonic, sleep=time.sleep, poll=2e-4,
                 on_candidates=None, first_block=0, device_timing=False,
                 min_batch=1, max_wait=0.0):
        self.server = server
        self.beams = list(beams)
        self.source = source
        self.threshold = float(threshold)
        self.stager = stager
        self.max_beams_in_step = int(max_beams_in_step)
        self.max_inflight = int(max_inflight)
        self.stream = compute_stream
        self.clock = clock
        self.sleep = sleep
        self.poll = float(poll)
        self.on_candidates = on_candidates
        self.first_block = int(first_block)
        self.max_waiting = int(getattr(server, "max_waiting", 1))
        # device_timing: CUDA events around every push and step on the
        # compute stream, summed into ServeResult.busy (the device time the
        # schedule needed: above the schedule's span the load is not
        # sustainable however short the run)
        self.device_timing = bool(device_timing)
        self._spans = []
        # a step waits for min_batch pushed blocks (a device launch of a few
        # beam-blocks leaves its last wave of work items mostly empty) unless
        # the oldest pushed block has waited max_wait seconds, or no more
        # blocks are due
        self.min_batch = max(1, int(min_batch))
        self.max_wait = float(max_wait)

    def _timed(self, fn):
        if not self.device_timing:
            return fn()
        import torch
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        out = fn()
        e1.record(self.stream)
        self._spans.append((e0, e1))
        return out

    def run(self, arrivals, time_limit=None):
        """Serve the schedule (arrivals[i][k] = seconds after the start at
        which block k of row i is available; inf = never).  Stops when every
        block completed, or at `time_limit` seconds with the blocks not done
        left at nan latency (their steps may still be running)."""
        arrivals = np.asarray(arrivals, dtype=np.float64)
        nb, nk = arrivals.shape
        if nb != len(self.beams):
            raise ValueError("one schedule row per beam")
        row_of = {b: i for i, b in enumerate(self.beams)}
        flat = arrivals.reshape(-1)
        order = np.argsort(flat, kind="stable")
        total = nb * nk
        waiting = [[] for _ in range(nb)]        # arrived, not pushed (heaps)
        has_waiting = set()                     # rows with a waiting block
        pushed = [0] * nb
        stepped = [0] * nb
        unstepped = 0                           # pushed blocks not in a step
        lat = np.full((nb, nk), np.nan)
        ncand = np.zeros((nb, nk), dtype=np.int64)
        inflight = deque()
        # push times of the blocks not yet in a step (a step takes the
        # oldest pushes first, so the front is the oldest)
        push_time = deque()

        def oldest_push():
            return push_time[0] if push_time else float("inf")

        res = ServeResult(lat, ncand)
        nexta, ndone = 0, 0
        t0 = self.clock()
        while ndone < total:
            now = self.clock() - t0
            if time_limit is not None and now > time_limit:
                break
            busy = False
            # arrivals that are due
            while nexta < total and flat[order[nexta]] <= now:
                i, k = divmod(int(order[nexta]), nk)
                heapq.heappush(waiting[i], k)
                has_waiting.add(i)
                nexta += 1
                busy = True
            # ingest in block order (a later block waits in host memory for
            # a missing one, or for a step to take the beam's block before
            # it: the server holds max_waiting blocks per beam)
            for i in sorted(has_waiting):
                while (waiting[i] and waiting[i][0] == pushed[i]
                       and pushed[i] - stepped[i] < self.max_waiting):
                    k = waiting[i][0]
                    host = self.source(i, k)
                    if self.stager is not None:
                        x, token = self.stager.stage(host)
                    else:
                        x, token = host, None
                    ok = self._timed(lambda: self.server.push(
                        self.beams[i], x, stream=self.stream))
                    if self.stager is not None:
                        self.stager.consumed(token)
                    if not ok:
                        raise RuntimeError("server refused a block the loop "
                                           "counted as admissible")
                    heapq.heappop(waiting[i])
                    pushed[i] += 1
                    unstepped += 1
                    push_time.append(self.clock() - t0)
                    busy = True
                if not waiting[i]:
                    has_waiting.discard(i)
            # completions
            finished = []
            while inflight and self.server.done(inflight[0][0]):
                _, members = inflight.popleft()
                tdone = self.clock() - t0
                for i, k in members:
                    lat[i, k] = tdone - arrivals[i, k]
                finished.extend(members)
                ndone += len(members)
                res.wall = tdone
                busy = True
            # with one step in flight, launch the next before reading the
            # finished blocks' results so the device stays busy; with more,
            # read first (a step launched now could reuse the candidate
            # buffer of a block finished but not yet read), the queued step
            # keeps the device busy meanwhile
            if self.max_inflight > 1:
                self._fetch(finished, res)
                finished = []
            full = (unstepped >= self.min_batch or nexta >= total or
                    (unstepped > 0 and
                     now - oldest_push() >= self.max_wait))
            if len(inflight) < self.max_inflight and unstepped > 0 and full:
                sid, sbeams = self._timed(lambda: self.server.step(
                    self.threshold, self.max_beams_in_step, stream=self.stream))
                if sbeams:
                    members = []
                    for b in sbeams:
                        i = row_of[b]
                        members.append((i, stepped[i]))
                        stepped[i] += 1
                        unstepped -= 1
                        if push_time:
                            push_time.popleft()
                    inflight.append((sid, members))
                    res.step_sizes.append(len(sbeams))
                    busy = True
            self._fetch(finished, res)
            if not busy:
                wait = self.poll
                if nexta < total and np.isfinite(flat[order[nexta]]):
                    wait = min(wait, max(0.0, flat[order[nexta]] - now))
                self.sleep(wait)
        if self.device_timing:
            import torch
            torch.cuda.current_stream().synchronize()
            if self.stream is not None:
                self.stream.synchronize()
            res.busy = sum(a.elapsed_time(b) for a, b in self._spans) * 1e-3
            self._spans = []
        return res


    def _fetch(self, finished, res):
        for i, k in finished:
            # a block over the candidate capacity keeps its first records
            # and reports the true count
            cands, n, t_start = self.server.fetch(
                self.beams[i], self.first_block + k, allow_truncated=True)
            res.ncand[i, k] = n
            if self.on_candidates is not None:
                self.on_candidates(i, k, cands, t_start)


def realtime_limit(run_at, lo, hi, step, deadline):
    """Largest beam count n in [lo, hi] (multiples of `step`) with
    run_at(n) <= deadline, by bisection assuming the p99 latency grows with
    n; run_at(n) returns the p99 latency (inf if n beams cannot be
    admitted).  Returns (n or 0, {n: p99})."""
    seen = {}

    def ok(n):
        if n not in seen:
            seen[n] = run_at(n)
        return seen[n] <= deadline

    a, b = lo // step, hi // step
    if not ok(a * step):
        return 0, seen
    while a < b:
        m = (a + b + 1) // 2
        if ok(m * step):
            a = m
        else:
            b = m - 1
    return a * step, seen
