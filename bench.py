#!/usr/bin/env python
"""Benchmark of the dedispersion + single-pulse-search path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one pass of the whole path over one beam block: unpack
(time-major -> channel-major), brute-force dedispersion of every DM trial,
the fused median/MAD + boxcar S/N + candidate-compaction kernel, and the
candidate fetch (device -> host, sorted).  Workload: one full-size beam,
4096 channels over 300-500 MHz at 81.92 us, a 262144-sample block plus the
89989-sample maximum-delay overlap, 1024 DM trials over 0-250 pc cm^-3,
boxcar widths 1..256, median/MAD windows of 8192 samples, threshold 7
(seeded synthetic 8-bit noise with 20 injected dispersed pulses).

Metric: dedispersion channel*sample*DM adds per second, N_c * N_out * N_dm
per step divided by the step time (whole job, all ranks).  The input block
(1.44 GB) is larger than L2, so no flush is needed between steps.

For N > 1 (torchrun, one rank per GPU) every rank processes its own beam:
weak scaling with no data-path collective; the barrier and the max-over-
ranks of the timings use the process group only.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dedispersion chan·sample·DM adds/s"
UNIT = "adds/s"
SM_COUNT_B300 = 148
ADDS_PER_SM_CLK = 128  # one byte operand per add through the 128 B/clk shared-memory port


def workload():
    from paper_2605_03531_b300 import synth
    return synth.config2()


def workload_config(cfg, nout):
    return {"workload": "single full-size beam: 4096 ch x 81.92 us, 300-500 MHz, "
                        "262144-sample block + max-delay overlap, 1024 DMs 0-250, "
                        "widths 1-256, L=8192, thr 7",
            "nchan": cfg.nchan, "nsamp_out": nout, "ndm": cfg.ndm,
            "widths": [int(w) for w in cfg.widths], "norm_window": cfg.norm_window,
            "threshold": cfg.threshold, "input_bits": 8,
            "l2": "inputs larger than L2 (1.44 GB block per step)"}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------- distributed
def dist_setup(n_gpus):
    from paper_2605_03531_b300 import shard
    return shard.init()


def barrier(world):
    from paper_2605_03531_b300 import shard
    shard.barrier(world)


def max_over_ranks(v, world):
    from paper_2605_03531_b300 import shard
    return shard.max_over_ranks(v, world)


# ------------------------------------------------------------- oracle CPU
def oracle_sample_rate(x_host, d, widths, L, target_s, min_t=8):
    """Time the oracle (dedispersion + search) on all DM trials x the first T
    output samples, T sized to about target_s seconds; returns adds/s,
    T, elapsed seconds."""
    import oracle
    cal_t = min_t
    D = int(d.max())

    def run(T):
        xs = np.ascontiguousarray(x_host[:T + D])
        t0 = time.perf_counter()
        series = oracle.dedisperse(xs, d)
        oracle.sps(series, widths, L, 7.0, cap=1 << 16)
        return time.perf_counter() - t0

    avail = x_host.shape[0] - D
    el = run(cal_t)
    T = int(max(min_t, min(avail, cal_t * target_s / max(el, 1e-3))))
    el = run(T)
    # a tiny calibration run is dominated by fixed costs: rescale once more
    if el < 0.6 * target_s and T < avail:
        T = int(max(min_t, min(avail, T * target_s / max(el, 1e-3))))
        el = run(T)
    adds = d.shape[0] * d.shape[1] * T
    return adds / el, T, el


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ----------------------------------------------------------------- arms
def run_reference(args):
    from paper_2605_03531_b300 import shard
    world, rank, _ = shard.world_from_env()
    if not shard.runs_reference(world, rank):
        return 0    # the CPU reference runs once, on rank 0
    cores = cpu_cores()
    os.environ["OMP_NUM_THREADS"] = str(cores)
    import oracle
    from paper_2605_03531_b300 import synth
    cfg = workload()
    d, D = oracle.delay_table(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp,
                              cfg.dm_list())
    budget = max(1.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    # one bounded slice of the block, regenerated on the host
    xfull = synth.noise_u8(32768 + D, cfg.nchan, cfg.seed).numpy()
    rate0, T, _ = oracle_sample_rate(xfull, d, cfg.widths, cfg.norm_window,
                                     target_s=budget)
    x = np.ascontiguousarray(xfull[:T + D])
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        series = oracle.dedisperse(x, d)
        oracle.sps(series, cfg.widths, cfg.norm_window, cfg.threshold, cap=1 << 16)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    step_s = sum(times) / len(times)
    adds = cfg.ndm * cfg.nchan * T
    value = adds / step_s
    sample = (f"all {cfg.ndm} DM trials x first {T} output samples x "
              f"{cfg.nchan} channels of the block per step (dedispersion + search)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": workload_config(cfg, cfg.nsamp_out),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def traffic_record(kernel, field="dram_bytes_per_launch"):
    """A per-launch figure (DRAM bytes, warp instructions) of the full-size
    launch from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(path))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    h = hashlib.sha256()
    try:
        for name in rec["sources"]:
            h.update(open(os.path.join(ROOT, "paper_2605_03531_b300", "csrc",
                                       name), "rb").read())
    except (OSError, KeyError):
        return None
    if h.hexdigest() != rec.get("sources_sha256"):
        return None
    return rec.get(field)


def run_ours(args):
    import torch
    from paper_2605_03531_b300 import Plan, build, shard, synth
    build.build()
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    cfg = workload()
    if world > 1:
        cfg.seed = shard.rank_seed(cfg.seed, rank)   # each rank its own beam
    plan = Plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
                cfg.widths, nbits=8, norm_window=cfg.norm_window,
                cand_capacity=1 << 20)
    if args.tile:
        plan.set_tile(*(int(v) for v in args.tile.split(",")))
    D = plan.max_delay
    nout = args.nsamp_out or cfg.nsamp_out
    nin = nout + D
    tile = plan.get_tile()
    kname = ("dedisp_il_kernel" if tile["flags"] & 16 else
             "dedisp_ws_kernel" if tile["flags"] & 8 else
             "dedisp_kernel" if tile["dm_tile"] > 0 else "dedisp_direct_kernel")
    x = synth.noise_u8(nin, cfg.nchan, cfg.seed, device=dev)
    synth.inject_pulses(x, cfg.pulses, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.seed)
    series = torch.empty((cfg.ndm, nout), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    adds = cfg.nchan * nout * cfg.ndm

    def step(ev=None):
        # stage (time-major block -> the rows the dedispersion tile reads),
        # dedispersion, search: the three launches ddsp_dedisperse plus
        # ddsp_sps make, timed one by one
        if ev is not None:
            ev[0].record(stream)
        plan.stage(x, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        plan.dedisperse_staged(nout, out=series, stream=stream)
        if ev is not None:
            ev[2].record(stream)
        plan.single_pulse_search(series, cfg.threshold, stream=stream)
        if ev is not None:
            ev[3].record(stream)
        return plan.fetch()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)]
           for _ in range(args.steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    idx = dev.index if dev.index is not None else 0
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[idx] if vis and vis.split(",")[idx].isdigit() else idx
    clocks = ClockSampler(smi_index)
    if not args.profile:
        clocks.start()
        time.sleep(0.5)
    barrier(world)
    torch.cuda.synchronize(dev)
    start.record(stream)
    ncand = 0
    for i in range(args.steps):
        _, ncand = step(evs[i])
    end.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    ck = clocks.stop()
    ms_total = start.elapsed_time(end)
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    k_stage = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    k_dedisp = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    k_sps = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    value = world * adds / (ms_step * 1e-3)

    if args.profile:   # kernels only (for profiler captures)
        if rank == 0:
            print(json.dumps({"profile": True, "workload": "beam", "nsamp_out": nout,
                              "ms_per_step": ms_step, "dedisp_ms": k_dedisp,
                              "sps_ms": k_sps, "stage_ms": k_stage,
                              "tile": tile}), flush=True)
        return 0

    # ---- end to end through the public calls with host buffers: every step
    # copies its block from pinned host memory and reads its candidates
    # back; the copy of step k+1 (own stream, two device buffers) overlaps
    # step k's kernels, as a streaming pipeline runs
    xh = torch.empty((nin, cfg.nchan), dtype=torch.uint8, pin_memory=True)
    xh.copy_(x.cpu())
    xd2 = [torch.empty_like(x) for _ in range(2)]
    series2 = [torch.empty_like(series) for _ in range(2)]
    copy_stream = torch.cuda.Stream(dev)
    ev_copied = [torch.cuda.Event() for _ in range(2)]
    ev_read = [torch.cuda.Event() for _ in range(2)]
    for e in ev_read:
        e.record(stream)

    def start_copy(k):
        b = k % 2
        copy_stream.wait_event(ev_read[b])      # the buffer's last reader ran
        with torch.cuda.stream(copy_stream):
            xd2[b].copy_(xh, non_blocking=True)
        ev_copied[b].record(copy_stream)

    def e2e_run(nsteps):
        ncs = []
        start_copy(0)
        for k in range(nsteps):
            b = k % 2
            stream.wait_event(ev_copied[b])
            plan.dedisperse(xd2[b], out=series2[b], stream=stream)
            ev_read[b].record(stream)
            if k + 1 < nsteps:
                start_copy(k + 1)
            if k > 0:                            # step k-1's search is done
                ncs.append(plan.fetch()[1])      # before step k's is queued
            plan.single_pulse_search(series2[b], cfg.threshold, stream=stream)
        ncs.append(plan.fetch()[1])
        return ncs

    e2e_run(max(1, args.warmup))
    torch.cuda.synchronize(dev)
    barrier(world)
    t0 = time.perf_counter()
    ncs = e2e_run(args.steps)
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world) / args.steps
    e2e = {"value": world * adds / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(nin * cfg.nchan),
           "d2h_bytes_per_step": int(4 + 16 * ncs[-1]), "ms_per_step": e2e_s * 1e3,
           "overlap": "host-to-device copy of step k+1 runs during step k"}

    sm_mhz = ck["sm_mhz"] if ck else None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    clk = sm_mhz or peaks.get("sm_max_mhz", 2032.0)
    peak = SM_COUNT_B300 * ADDS_PER_SM_CLK * clk * 1e6 / 1e12
    achieved = adds / (k_dedisp * 1e-3) / 1e12
    traffic = traffic_record(kname) if nout == cfg.nsamp_out else None
    # issue slots: warp instructions of the launch (ncu record) over the
    # 4 schedulers x 148 SMs x the sampled clock x the measured duration
    winst = (traffic_record(kname, "warp_inst_per_launch")
             if nout == cfg.nsamp_out else None)
    issue_frac = (winst / (k_dedisp * 1e-3 * SM_COUNT_B300 * 4 * clk * 1e6)
                  if winst else None)
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    sps_bytes = 4.0 * cfg.ndm * nout + 16 * ncand
    # staging reads the block once and writes 4 bytes per sample (the
    # interleaved rows) or 1 (channel-major rows)
    stage_bytes = (1.0 + (4 if tile["flags"] & 16 else 1)) * nin * cfg.nchan
    result = None
    if rank == 0:
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": workload_config(cfg, nout),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "Tadd/s", "frac": achieved / peak,
                         "issue_frac": issue_frac,
                         "traffic": traffic,
                         "kernel": kname, "tile": tile,
                         "peak_basis": f"{SM_COUNT_B300} SMs x {ADDS_PER_SM_CLK} "
                                       f"adds/clk x {clk:.0f} MHz "
                                       "(median SM clock sampled in the timed region)"},
            "kernels": {
                "stage_ms": k_stage, "dedisp_ms": k_dedisp, "sps_ms": k_sps,
                "stage_hbm_frac": stage_bytes / (k_stage * 1e-3) / 1e9 / hbm_peak,
                "sps_hbm_frac": sps_bytes / (k_sps * 1e-3) / 1e9 / hbm_peak,
                "hbm_peak_gbs": hbm_peak},
            "candidates_per_step": int(ncand),
            "e2e": e2e,
            "gpu_launches": 3 * args.steps,
            "clocks": ck,
        }
    if rank == 0 and not args.no_cpu_baseline:
        cores = cpu_cores()
        os.environ["OMP_NUM_THREADS"] = str(cores)
        d = plan.delays()
        xs = x[:min(nin, 65536 + D)].cpu().numpy()
        import oracle
        oracle.set_threads(cores)
        rate, T, el = oracle_sample_rate(xs, d, cfg.widths, cfg.norm_window,
                                         target_s=args.cpu_seconds)
        oracle.set_threads(1)
        rate1, T1, el1 = oracle_sample_rate(xs, d, cfg.widths, cfg.norm_window,
                                            target_s=max(2.0, args.cpu_seconds / 3))
        oracle.set_threads(cores)
        result["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all {cfg.ndm} DM trials x first {T} output samples x "
                      f"{cfg.nchan} channels (dedispersion + search), "
                      f"{el:.1f} s",
            "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": f"all {cfg.ndm} DM trials x first {T1} "
                                        f"output samples, {el1:.1f} s"}}
    if rank == 0 and world == 1 and not args.no_serving:
        del x, series, xd2, series2, xh
        plan.close()
        torch.cuda.empty_cache()
        try:
            result["serving"] = serving_check(
                dev, log=lambda m: print(m, file=sys.stderr, flush=True))
        except Exception as e:            # reported, never fatal to the line
            result["serving"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ------------------------------------------------ serving check (default run)
def serving_check(dev, blocks_per_beam=5, log=None):
    """The streaming target in bounded time: beams of the 4096-channel shape
    (16384-spectrum blocks every 1.342 s, Poisson-jittered arrivals) served
    by batched steps (every waiting beam-block, interleaved mode, 8 staging
    slots) and by the plain per-beam path (one beam per step, a second step
    queued), each from the real-time count an untimed calibration of its
    step time per beam-block suggests, then in steps of 16 beams up or down
    until the runs bracket its limit.  Rings are filled first (untimed), then
    `blocks_per_beam` blocks per beam arrive in real time; p50/p99 latency
    from arrival to the host seeing the block's step complete, and the
    device time the pushes and steps took per second of stream (duty): a
    count is real time if p99 < 1.342 s and the duty is below 1 (a short
    run cannot show a slowly growing backlog in its latencies).  The full
    bisection is `--workload serve`."""
    import torch
    from paper_2605_03531_b300 import Plan, Server, synth
    from paper_2605_03531_b300.serve import DeviceStager, ServingLoop
    cfg = synth.config5(1)[0]
    B, T = cfg.nsamp_out, synth.BLOCK_PERIOD_S
    plan = Plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
                cfg.widths, nbits=8, norm_window=cfg.norm_window,
                cand_capacity=1 << 18)
    pool = []
    for i in range(8):
        x = synth.noise_u8(B, cfg.nchan, cfg.seed + 17 * i, device=dev)
        synth.inject_pulses(x, synth.random_pulses(2, cfg.nchan, B - 4096, seed=i,
                                                   dm_range=(10.0, 240.0), wmax=64,
                                                   snr_range=(10.0, 30.0),
                                                   spacing=4096),
                            cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.seed + i)
        pool.append(x.cpu().pin_memory())
        del x
    compute = torch.cuda.Stream(dev)
    stager = DeviceStager(16, (B, cfg.nchan), compute)
    reserve, slots = 4 << 30, 8

    def make(n):
        srv = Server(plan, B, n, reserve)
        srv.set_mode(Server.INTERLEAVED, slots)
        return srv

    # calibration (untimed): device time per beam-block of a 32-beam step
    # and of a one-beam step
    def step_ms(nb):
        srv = make(nb)
        bs = [srv.admit() for _ in range(nb)]
        ms = []
        for rep in range(4):
            for i, b in enumerate(bs):
                xb, tok = stager.stage(pool[(i + rep) % 8])
                srv.push(b, xb, stream=compute)
                stager.consumed(tok)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(compute)
            srv.step(cfg.threshold, stream=compute)
            e1.record(compute)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        srv.close()
        torch.cuda.synchronize(dev)
        return min(ms[1:]) / nb
    ms_b, ms_p = step_ms(8), step_ms(1)
    per_beam_bytes = make(1).beam_bytes
    free, _ = torch.cuda.mem_get_info(dev)
    n_mem = int((free - reserve - slots * 4 * cfg.nchan * (B + 90112)) //
                per_beam_bytes) // 16 * 16
    # the count each path's step time allows, rounded down to 16 (the
    # runs decide)
    est_b = int(T * 1e3 / ms_b) // 16 * 16
    est_p = int(T * 1e3 / ms_p) // 16 * 16
    runs = {"batched": {}, "plain_per_beam": {}}

    def run_at(n, per_step, inflight, min_batch=1):
        srv = make(n)
        beams = []
        try:
            for _ in range(n):
                beams.append(srv.admit())
        except Exception as e:           # not admitted: memory
            srv.close()
            return {"admitted": len(beams), "error": str(e)}
        warm = -(-(srv.first_delay + srv.carry) // B)
        for k in range(warm):            # fill every ring (untimed)
            for i, b in enumerate(beams):
                xb, tok = stager.stage(pool[(3 * i + k) % 8])
                srv.push(b, xb, stream=compute)
                stager.consumed(tok)
            srv.step(cfg.threshold, stream=compute)
        srv.check(compute)
        arr = synth.arrival_times(n, blocks_per_beam, seed=5)
        loop = ServingLoop(srv, beams,
                           lambda i, k: pool[(3 * i + warm + k) % 8],
                           cfg.threshold, stager=stager, compute_stream=compute,
                           max_beams_in_step=per_step, first_block=warm,
                           max_inflight=inflight, device_timing=True,
                           min_batch=min_batch, max_wait=0.05)
        res = loop.run(arr, time_limit=blocks_per_beam * T + 30.0)
        srv.check(compute)
        srv.close()
        torch.cuda.synchronize(dev)
        lat = res.latency
        p99 = float("inf") if not np.isfinite(lat).all() else res.percentile(99)
        # device time the run's blocks needed per second of stream: at or
        # above 1 the backlog grows without bound, however short the run
        duty = res.busy / (blocks_per_beam * T)
        return {"p50_s": res.percentile(50), "p99_s": p99,
                "max_s": float(np.nanmax(lat)) if np.isfinite(lat).any() else None,
                "blocks": int(np.isfinite(lat).sum()),
                "mean_beams_per_step": float(np.mean(res.step_sizes)),
                "device_duty": duty,
                "real_time": bool(p99 < T and duty < 1.0)}

    # each path from its own estimate in steps of 16 beams: up while the
    # count is real time (at most two steps), down until it is (at most
    # three), so the runs bracket the path's limit
    paths = {
        # batched: a step waits for 4 beam-blocks (a launch of fewer leaves
        # its last wave of work items mostly empty) or 50 ms
        "batched": (est_b, lambda n: run_at(n, 0, 1, min_batch=4)),
        "plain_per_beam": (est_p, lambda n: run_at(n, 1, 2)),
    }
    for path, (start, run) in paths.items():
        n = max(16, min(start, n_mem))
        r = runs[path][str(n)] = run(n)
        if log:
            log(f"serving {path} {n}: {r}")
        up = r.get("real_time", False)
        for _ in range(2 if up else 3):
            n = n + 16 if up else n - 16
            if n < 16 or n > n_mem:
                break
            r = runs[path][str(n)] = run(n)
            if log:
                log(f"serving {path} {n}: {r}")
            if r.get("real_time", False) != up:
                break

    def best(path):
        ok = [int(n) for n, r in runs[path].items() if r.get("real_time")]
        return max(ok) if ok else 0
    return {
        "metric": "real-time beams per B300 at p99 (of the beam counts run)",
        "unit": "beams", "deadline_s": T, "blocks_per_beam": blocks_per_beam,
        "beams_tested": {p: sorted(int(n) for n in runs[p]) for p in runs},
        "real_time_beams": {"batched": best("batched"),
                            "plain_per_beam": best("plain_per_beam")},
        "step_ms_per_beam_block": {"batched_8": ms_b, "plain_1": ms_p},
        "beam_bytes": per_beam_bytes, "beams_fit_in_memory": n_mem,
        "workload": "streaming 4096-ch beams (300-500 MHz, 81.92 us), "
                    "16384-spectrum blocks, 1024 DMs 0-250, widths 1-256; "
                    "batched = interleaved mode with 8 staging slots, every "
                    "waiting beam-block per step once 4 wait or the oldest "
                    "waited 50 ms; plain = one beam per step, two steps in "
                    "flight",
        "runs": runs}


# ------------------------------------------------ one serving step (profiling)
def run_servestep(args):
    """One streaming server of the 4096-channel shape in the interleaved
    mode (8 staging slots) with --nbeams beams (0 = 8), stepped --steps
    times after --warmup steps, each step taking one fresh block of every
    beam: the device time of a step and per beam-block, by CUDA events (the
    workload that the serving launch list and its profile are taken on)."""
    import torch
    from paper_2605_03531_b300 import Plan, Server, build, synth
    build.build()
    dev = torch.device("cuda", 0)
    cfg = synth.config5(1)[0]
    B = cfg.nsamp_out
    plan = Plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
                cfg.widths, nbits=8, norm_window=cfg.norm_window,
                cand_capacity=1 << 18)
    nb = args.nbeams or 8
    srv = Server(plan, B, nb, 4 << 30)
    srv.set_mode(Server.INTERLEAVED, 8)
    beams = [srv.admit() for _ in range(nb)]
    blocks = [synth.noise_u8(B, cfg.nchan, 100 + i, device=dev)
              for i in range(4)]
    stream = torch.cuda.current_stream(dev)
    ms = []
    for k in range(args.warmup + args.steps):
        for i, b in enumerate(beams):
            srv.push(b, blocks[(i + k) % 4], stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        srv.step(cfg.threshold, stream=stream)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            ms.append(e0.elapsed_time(e1))
    srv.check(stream)
    srv.close()
    step = float(np.median(ms))
    print(json.dumps({"workload": "one serving step", "beams": nb,
                      "block": B, "nchan": cfg.nchan, "ndm": cfg.ndm,
                      "mode": "interleaved, 8 staging slots",
                      "ms_per_step": step, "ms_per_beam_block": step / nb,
                      "steps": args.steps, "warmup": args.warmup}),
          flush=True)
    return 0


# ------------------------------------------------ unit peaks (measurement)
def run_peaks(args):
    """Microbenchmarks of the on-chip units the dedispersion is bound by
    (ddsp_probe_unit_peaks): shared-memory load bytes, 3-input adds and byte
    permutes per SM clock, and the dedispersion inner loop on resident
    data, with the add rates each implies (1 shared byte per add; 4 ALU
    operations per pair of 4-sample words)."""
    from paper_2605_03531_b300 import build, probe_unit_peaks
    build.build()
    r = probe_unit_peaks(0)
    alu = min(r["iadd3_per_clk"], r["prmt_per_clk"])
    out = {"metric": "unit peaks per SM clock", "workload": "peaks",
           "impl": "ours", **r,
           "adds_per_clk_bounds": {
               "shared_memory": r["smem_bytes_per_clk"],
               "alu": 2.0 * alu,
               "inner_loop_resident": r["swar_adds_per_clk"],
               "nominal_used_for_roofline": ADDS_PER_SM_CLK}}
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------ search-only stress workload
SPS_METRIC = "single-pulse search series samples/s"


def run_sps(args):
    """2048 DM trials x 1048576 int32 samples (seeded Gaussian, mean 524288,
    sd 1024, 0.1% boxcar events of width 1..1024 and S/N 6..50), widths
    1..1024, median/MAD windows of 8192, FP32 S/N, threshold 6.5.  A step is
    the search kernel plus the read-back of the candidate count; the
    candidate records (about a third of all samples: no peak merging) stay on
    the device.  HBM-bound: 4 bytes per series sample read once plus 16 bytes
    per candidate record written."""
    import torch
    from paper_2605_03531_b300 import Plan, build, shard, synth
    build.build()
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    ndm, n = args.ndm or 2048, args.nsamp or (1 << 20)
    widths = [1 << i for i in range(11)]
    L, thr = 8192, 6.5
    x = synth.gaussian_series(ndm, n, seed=shard.rank_seed(4, rank), device=dev)
    cap = min(1 << 30, ndm * n)
    plan = Plan(16, 500.0, -1.0, 1e-3, np.zeros(ndm), widths, nbits=8,
                norm_window=L, cand_capacity=cap)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.single_pulse_search(x, thr, stream=stream)
        return plan.count()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier(world)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    ncand = 0
    for _ in range(args.steps):
        ncand = step()
    end.record(stream)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(start.elapsed_time(end), world) / args.steps
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    nbytes = 4.0 * ndm * n + 16.0 * min(ncand, cap)
    achieved = nbytes / (ms * 1e-3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": SPS_METRIC, "value": world * ndm * n / (ms * 1e-3),
            "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"single-pulse search stress: {ndm} DM trials x "
                                   f"{n} int32 samples, widths 1-1024, L=8192, "
                                   "thr 6.5", "ndm": ndm, "nsamp": n,
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "kernel": "sps_kernel"},
            "candidates_per_step": int(ncand), "gpu_launches": args.steps,
            "profile": bool(args.profile)}), flush=True)
    return 0


# ------------------------------------------- peaks filter + DM-time clustering
CLUSTER_METRIC = "single-pulse candidates filtered and clustered/s"
CLUSTER_HALF = [1, 2, 4, 8, 16, 32, 64, 128, 256]   # stencil = boxcar width
CLUSTER_EPS = (4, 32, 3)                            # eps_dm, eps_t, min_pts


def cluster_candidates(seed):
    """The beam's DM-time plane (1024 trials x 262144 samples, its 9 widths)
    with 3000 events (half extents 1-30 trials x 1-120 samples, peak S/N
    8-50, S/N on a 1/128 grid) and 200000 isolated noise candidates: about
    110 times the list one search of the beam block emits."""
    from paper_2605_03531_b300 import synth
    return synth.candidate_list(1024, 262144, len(CLUSTER_HALF), 3000, seed,
                                dm_half=(1, 30), t_half=(1, 120), noise=200000,
                                quantum=1 / 128)


def cluster_config(n):
    return {"workload": "peaks filter (square stencils, half-size = boxcar "
                        "width) + DBSCAN (4 trials x 32 samples, min_pts 3) of "
                        f"{n} single-pulse candidates on the beam's 1024 x "
                        "262144 DM-time plane (3000 events + 200000 noise)",
            "candidates": int(n), "ndm": 1024, "nsamp": 262144,
            "l2": "flushed between steps (256 MB write, outside the timed "
                  "intervals)"}


def cluster_oracle_rate(c, target_s):
    """Oracle candidates/s on the candidates of the first R DM trials taken
    as a list of their own, R sized to about target_s seconds (the filter
    is quadratic in the list size)."""
    import oracle
    R, el, m = 4, 0.0, 0
    for _ in range(3):
        sub = c[c["dm_idx"] < R]
        t0 = time.perf_counter()
        oracle.peaks_cluster(sub, CLUSTER_HALF, *CLUSTER_EPS)
        el, m = time.perf_counter() - t0, sub.size
        if el > 0.5 * target_s or R >= 1024:
            break
        R = int(min(1024, max(R + 1, R * (target_s / max(el, 1e-3)) ** 0.5)))
    return m / el, R, m, el


def run_cluster(args):
    import torch
    from paper_2605_03531_b300 import Cluster, build, shard
    build.build()
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    c = cluster_candidates(shard.rank_seed(6, rank))
    n = c.size
    d = Cluster.to_device(c, dev)
    cl = Cluster(1024, 262144, n, device=dev.index or 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)

    def step():
        cl.run(d, CLUSTER_HALF, *CLUSTER_EPS, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index or 0)
    if not args.profile:
        clocks.start()
        time.sleep(0.3)
    barrier(world)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for e0, e1 in evs:
        flush.fill_(1)
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / args.steps, world)
    peaks_n = cl.peaks()[0].size
    reps, _ = cl.reps()
    if args.profile:     # kernels only (for profiler captures)
        if rank == 0:
            print(json.dumps({"profile": True, "workload": "cluster",
                              "candidates": int(n), "ms_per_step": ms,
                              "peaks": int(peaks_n), "clusters": int(reps.size)}),
                  flush=True)
        cl.close()
        return 0
    # end to end through the public calls: records from pinned host memory,
    # the run, the representatives back on the host
    ch = torch.from_numpy(np.ascontiguousarray(c).view(np.int32).reshape(-1, 4).copy())
    ch = ch.pin_memory()

    def e2e_step():
        d.copy_(ch, non_blocking=True)
        step()
        return cl.reps()[0].size

    e2e_step()
    torch.cuda.synchronize(dev)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        nr = e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world) / args.steps
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    nbytes = 16.0 * n + 20.0 * peaks_n
    achieved = nbytes / (ms * 1e-3) / 1e9
    result = None
    if rank == 0:
        result = {
            "metric": CLUSTER_METRIC, "value": world * n / (ms * 1e-3),
            "unit": "candidates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32+f32",
            "data": "synthetic", "config": cluster_config(n),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "kernel": "ddsp_peaks_cluster (all 25 launches of the "
                                   "step, timed together)",
                         "bytes_basis": "16 B per input record read once + 20 B "
                                        "per peak (record + label) written"},
            "peaks_per_step": int(peaks_n), "clusters_per_step": int(reps.size),
            "e2e": {"value": world * n / e2e_s, "unit": "candidates/s",
                    "h2d_bytes_per_step": int(16 * n),
                    "d2h_bytes_per_step": int(16 * nr + 16),
                    "ms_per_step": e2e_s * 1e3},
            "gpu_launches": 25 * args.steps, "clocks": ck,
            "profile": bool(args.profile)}
        if not args.no_cpu_baseline and not args.profile:
            cores = cpu_cores()
            rate, R, m, el = cluster_oracle_rate(c, args.cpu_seconds)
            result["cpu_baseline"] = {
                "value": rate, "unit": "candidates/s", "cores": 1,
                "kind": "oracle",
                "sample": f"the {m} candidates of DM trials 0-{R - 1} as their "
                          f"own list ({el:.1f} s; the oracle is single-threaded "
                          f"and quadratic in the list size; {cores} cores seen)"}
        print(json.dumps(result), flush=True)
    cl.close()
    return 0


# ------------------------------------------------ downsampling + de-reddening
DERED_METRIC = "series samples de-reddened/s"


def dered_oracle_rate(x_row, h, target_s):
    """Oracle samples/s of the running-median subtraction on the first S
    samples of one row, S sized to about target_s seconds."""
    import oracle
    S, el = 2048, 0.0
    for _ in range(3):
        t0 = time.perf_counter()
        oracle.dered(x_row[:S], h)
        el = time.perf_counter() - t0
        if el > 0.5 * target_s or S >= x_row.size:
            break
        S = int(min(x_row.size, max(S + 1, S * target_s / max(el, 1e-3))))
    return S / el, S, el


def run_dered(args):
    """The beam's series shape, 1024 DM trials x 262144 int32 samples
    (seeded Gaussian, sd 1024, with 0.1% boxcar events and a slow sinusoidal
    baseline of amplitude 3000 and period 40000-200000 samples per row),
    de-reddened by subtracting the running median over 2049 samples
    (h = 1024: the window exceeds twice the widest boxcar, 256 samples, as
    Sec.3.3 asks).  A step is one ddsp_dered call over all rows; beside it
    the downsampling by 4 is timed on the same rows."""
    import torch
    from paper_2605_03531_b300 import Plan, build, shard, synth
    build.build()
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    ndm, n, h, f = 1024, 262144, 1024, 4
    x = synth.red_series(ndm, n, shard.rank_seed(15, rank), device=dev)
    z = torch.empty_like(x)
    y = torch.empty((ndm, n // f), dtype=torch.int32, device=dev)
    plan = Plan(16, 500.0, -1.0, 1e-3, np.zeros(4), [1, 2], nbits=8,
                norm_window=8192, cand_capacity=1024)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        plan.dered(x, h, out=z, stream=stream)
        plan.downsample(x, f, out=y, stream=stream)
    torch.cuda.synchronize(dev)
    plan.check()
    clocks = ClockSampler(dev.index or 0)
    if not args.profile:
        clocks.start()
        time.sleep(0.3)
    barrier(world)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    for _ in range(args.steps):
        plan.dered(x, h, out=z, stream=stream)
    ev[1].record(stream)
    for _ in range(args.steps):
        plan.downsample(x, f, out=y, stream=stream)
    ev[2].record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    plan.check()
    ms = max_over_ranks(ev[0].elapsed_time(ev[1]) / args.steps, world)
    ms_ds = ev[1].elapsed_time(ev[2]) / args.steps
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    nbytes = 8.0 * ndm * n
    achieved = nbytes / (ms * 1e-3) / 1e9
    ds_frac = (4.0 * ndm * n + 4.0 * ndm * (n // f)) / (ms_ds * 1e-3) / 1e9 / hbm
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile": True, "workload": "dered",
                              "ms_per_step": ms, "downsample_ms": ms_ds}),
                  flush=True)
        return 0
    # end to end: the rows from pinned host memory, the de-reddened rows back
    xh = x.cpu().pin_memory()
    zh = torch.empty_like(xh).pin_memory()

    def e2e_step():
        x.copy_(xh, non_blocking=True)
        plan.dered(x, h, out=z, stream=stream)
        zh.copy_(z, non_blocking=True)
        torch.cuda.synchronize(dev)

    e2e_step()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world) / args.steps
    if rank == 0:
        result = {
            "metric": DERED_METRIC, "value": world * ndm * n / (ms * 1e-3),
            "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"running-median de-reddening of {ndm} x {n} "
                                   f"int32 series (window {2 * h + 1} samples, "
                                   "slow sinusoidal baselines)", "ndm": ndm,
                       "nsamp": n, "half_window": h,
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "kernel": "dered_kernel",
                         "bytes_basis": "4 B read + 4 B written per sample"},
            "kernels": {"downsample_ms": ms_ds, "downsample_factor": f,
                        "downsample_hbm_frac": ds_frac},
            "e2e": {"value": world * ndm * n / e2e_s, "unit": "samples/s",
                    "h2d_bytes_per_step": int(4 * ndm * n),
                    "d2h_bytes_per_step": int(4 * ndm * n),
                    "ms_per_step": e2e_s * 1e3},
            "gpu_launches": args.steps, "clocks": ck}
        if not args.no_cpu_baseline:
            rate, S, el = dered_oracle_rate(x[0].cpu().numpy(), h, args.cpu_seconds)
            result["cpu_baseline"] = {
                "value": rate, "unit": "samples/s", "cores": 1, "kind": "oracle",
                "sample": f"the first {S} samples of one row ({el:.1f} s; the "
                          "oracle sorts every window, single-threaded)"}
        print(json.dumps(result), flush=True)
    return 0


# ------------------------------------------------ folding transform + search
FFA_METRIC = "FFA trial periods folded and searched/s"


def ffa_work(n, p_lo, p_hi, wmax):
    """(trial periods, algorithmic adds) of one row: per base period m*p*
    log2(m) transform adds and m*p*wmax running-window adds."""
    trials = adds = 0
    for p in range(p_lo, p_hi):
        m = 1
        while 2 * m * p <= n:
            m *= 2
        trials += m
        adds += m * p * (m.bit_length() - 1) + m * p * wmax
    return trials, adds


def run_ffa(args):
    """1024 DM-trial series of 16384 samples (a downsampled, de-reddened
    stretch of the beam: seeded Gaussian, mean 0, sd 1024, 0.1% boxcar
    events), folded at the base periods 128..255 (trial periods 128-256
    samples, one octave) and searched with boxcars of 1-32 samples."""
    import torch
    from paper_2605_03531_b300 import Plan, build, shard, synth
    build.build()
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    rows, n, p_lo, p_hi = 1024, 16384, 128, 256
    widths = [1, 2, 4, 8, 16, 32]
    x = synth.gaussian_series(rows, n, seed=shard.rank_seed(16, rank), mean=0.0,
                              device=dev)
    plan = Plan(16, 500.0, -1.0, 1e-3, np.zeros(4), [1, 2], nbits=8,
                norm_window=8192, cand_capacity=1024)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        out = plan.ffa_search(x, p_lo, p_hi, widths, 1024.0, stream=stream)
    torch.cuda.synchronize(dev)
    plan.check()
    clocks = ClockSampler(dev.index or 0)
    if not args.profile:
        clocks.start()
        time.sleep(0.3)
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out = plan.ffa_search(x, p_lo, p_hi, widths, 1024.0, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    plan.check()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    trials, adds = ffa_work(n, p_lo, p_hi, widths[-1])
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile": True, "workload": "ffa", "ms_per_step": ms}),
                  flush=True)
        return 0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    clk = (ck or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    peak = SM_COUNT_B300 * ADDS_PER_SM_CLK * clk * 1e6 / 1e12
    achieved = rows * adds / (ms * 1e-3) / 1e12
    # end to end: the rows from pinned host memory, the S/N back
    xh = x.cpu().pin_memory()

    def e2e_step():
        x.copy_(xh, non_blocking=True)
        snr, wi, ph = plan.ffa_search(x, p_lo, p_hi, widths, 1024.0, stream=stream)
        return snr.cpu()

    e2e_step()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world) / args.steps
    snr = out[0]
    best = float(snr.max())
    if rank == 0:
        result = {
            "metric": FFA_METRIC, "value": world * rows * trials / (ms * 1e-3),
            "unit": "trials/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"FFA search of {rows} x {n}-sample series, "
                                   f"base periods {p_lo}-{p_hi - 1}, boxcars 1-32",
                       "rows": rows, "nsamp": n, "p_lo": p_lo, "p_hi": p_hi,
                       "l2": "each row's stack is folded on chip; the 64 MB "
                             "input stays in L2 across periods"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "Tadd/s", "frac": achieved / peak, "traffic": None,
                         "kernel": "ffa_search_kernel",
                         "peak_basis": f"{SM_COUNT_B300} SMs x {ADDS_PER_SM_CLK} "
                                       f"adds/clk x {clk:.0f} MHz",
                         "adds_basis": "m p log2(m) transform adds + m p w_max "
                                       "window adds per (row, base period)"},
            "trials_per_step": rows * trials, "best_snr": best,
            "e2e": {"value": world * rows * trials / e2e_s, "unit": "trials/s",
                    "h2d_bytes_per_step": int(4 * rows * n),
                    "d2h_bytes_per_step": int(res.numel() * 4),
                    "ms_per_step": e2e_s * 1e3},
            "gpu_launches": args.steps, "clocks": ck}
        if not args.no_cpu_baseline:
            import oracle
            xr = x[0].cpu().numpy()
            t0 = time.perf_counter()
            done = 0
            p = p_lo
            while time.perf_counter() - t0 < args.cpu_seconds and p < p_hi:
                F = oracle.ffa(xr, p)
                for s_ in range(F.shape[0]):
                    oracle.fold_snr(F[s_], F.shape[0], widths, 1024.0)
                done += F.shape[0]
                p += 1
            el = time.perf_counter() - t0
            result["cpu_baseline"] = {
                "value": done / el, "unit": "trials/s", "cores": 1,
                "kind": "oracle",
                "sample": f"row 0, base periods {p_lo}-{p - 1} ({done} trials, "
                          f"{el:.1f} s, one thread)"}
        print(json.dumps(result), flush=True)
    return 0


# ------------------------------------------------------------------ resample
RESAMPLE_METRIC = "series samples resampled/s"


def run_resample(args):
    """1024 series of 262144 int32 samples (the beam's series shape, seeded
    Gaussian with events) resampled for a signal of f0 = 3 Hz, f1 = -2e-4
    Hz/s, f2 = -1e-8 Hz/s^2 at 81.92 us per sample (a drift of ~0.15 % over
    the 21.5 s block).  One step: one ddsp_resample call over all rows."""
    import torch
    from paper_2605_03531_b300 import Plan, build, shard, synth
    build.build()
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    rows, n, ts, f0, f1, f2 = 1024, 262144, 81.92e-6, 3.0, -2e-4, -1e-8
    x = synth.gaussian_series(rows, n, seed=shard.rank_seed(17, rank), device=dev)
    plan = Plan(16, 500.0, -1.0, 1e-3, np.zeros(4), [1, 2], nbits=8,
                norm_window=8192, cand_capacity=1024)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        y = plan.resample(x, ts, f0, f1, f2, stream=stream)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index or 0)
    if not args.profile:
        clocks.start()
        time.sleep(0.3)
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        y = plan.resample(x, ts, f0, f1, f2, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile": True, "workload": "resample",
                              "ms_per_step": ms}), flush=True)
        return 0
    K = y.shape[1]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    nbytes = 4.0 * rows * n + 4.0 * rows * K
    achieved = nbytes / (ms * 1e-3) / 1e9
    xh = x.cpu().pin_memory()
    yh = torch.empty((rows, K), dtype=torch.float32).pin_memory()

    def e2e_step():
        x.copy_(xh, non_blocking=True)
        yy = plan.resample(x, ts, f0, f1, f2, stream=stream)
        yh.copy_(yy, non_blocking=True)
        torch.cuda.synchronize(dev)

    e2e_step()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world) / args.steps
    if rank == 0:
        result = {
            "metric": RESAMPLE_METRIC, "value": world * rows * n / (ms * 1e-3),
            "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"resampling of {rows} x {n} int32 series for "
                                   "f0 3 Hz, f1 -2e-4 Hz/s, f2 -1e-8 Hz/s^2",
                       "rows": rows, "nsamp": n, "nout": K,
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "kernel": "resample_kernel",
                         "bytes_basis": "4 B read per input + 4 B written per output"},
            "e2e": {"value": world * rows * n / e2e_s, "unit": "samples/s",
                    "h2d_bytes_per_step": int(4 * rows * n),
                    "d2h_bytes_per_step": int(4 * rows * K),
                    "ms_per_step": e2e_s * 1e3},
            "gpu_launches": args.steps, "clocks": ck}
        if not args.no_cpu_baseline:
            import oracle
            xr = x[0].cpu().numpy()
            t0 = time.perf_counter()
            reps = 0
            while time.perf_counter() - t0 < args.cpu_seconds:
                oracle.resample(xr, f0, f1, f2, ts)
                reps += 1
            el = time.perf_counter() - t0
            result["cpu_baseline"] = {
                "value": reps * n / el, "unit": "samples/s", "cores": 1,
                "kind": "oracle",
                "sample": f"row 0 resampled {reps} times ({el:.1f} s, one thread)"}
        print(json.dumps(result), flush=True)
    return 0


# ------------------------------------------------------------ RFI mitigation
RFI_METRIC = "spectra samples cleaned/s"


def run_rfi(args):
    """One streaming block of 16384 spectra x 4096 channels (uint8, 67 MB):
    seeded noise (128 +- 16) with a gentle bandpass slope, 12 channels of
    narrowband RFI (+60) and 6 broadband bursts (+40); gptool-style
    cleaning with the paper's parameters (21-channel bandpass median, 4
    sigma channels, 3 sigma samples, two rounds)."""
    import torch
    from paper_2605_03531_b300 import Rfi, build, shard, synth
    build.build()
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    nt, nc = 16384, 4096
    seed = shard.rank_seed(18, rank)
    x = synth.noise_u8(nt, nc, seed, device=dev).to(torch.int32)
    g = torch.linspace(0.8, 1.2, nc, device=dev)
    x = torch.round(x.float() * g[None, :]).to(torch.int32)
    u = synth.uniform_np(np.arange(18, dtype=np.uint64), seed + 9)
    rfi_c = sorted({int(v * nc) for v in u[:12]})
    rfi_t = sorted({int(v * nt) for v in u[12:]})
    x[:, rfi_c] += 60
    x[rfi_t, :] += 40
    x = x.clamp(0, 255).to(torch.uint8).contiguous()
    out = torch.empty_like(x)
    r = Rfi(nt, nc, device=dev.index or 0)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        r.clean(x, out=out, stream=stream)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index or 0)
    if not args.profile:
        clocks.start()
        time.sleep(0.3)
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        r.clean(x, out=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    fc, ft, fill = r.flags()
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile": True, "workload": "rfi", "ms_per_step": ms}),
                  flush=True)
        return 0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    nbytes = 2.0 * 2 * nt * nc + 2.0 * nt * nc   # two reads per round, in + out
    achieved = nbytes / (ms * 1e-3) / 1e9
    xh = x.cpu().pin_memory()
    oh = torch.empty_like(xh).pin_memory()

    def e2e_step():
        x.copy_(xh, non_blocking=True)
        r.clean(x, out=out, stream=stream)
        oh.copy_(out, non_blocking=True)
        torch.cuda.synchronize(dev)

    e2e_step()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world) / args.steps
    if rank == 0:
        result = {
            "metric": RFI_METRIC, "value": world * nt * nc / (ms * 1e-3),
            "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8+int64",
            "data": "synthetic",
            "config": {"workload": f"gptool-style RFI cleaning of a {nt} x {nc} "
                                   "uint8 block (21-channel bandpass, 4/3 sigma, "
                                   "two rounds)", "nsamp": nt, "nchan": nc,
                       "planted_channels": len(rfi_c), "planted_samples": len(rfi_t),
                       "l2": "the 67 MB block stays in L2 across the passes"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "kernel": "ddsp_rfi_clean (all launches of the step)",
                         "bytes_basis": "two block reads per round + one read "
                                        "and one write"},
            "flags": {"channels": int(fc.sum()), "samples": int(ft.sum()),
                      "planted_channels_found": int(fc[rfi_c].sum()),
                      "planted_samples_found": int(ft[rfi_t].sum()),
                      "fill": int(fill)},
            "e2e": {"value": world * nt * nc / e2e_s, "unit": "samples/s",
                    "h2d_bytes_per_step": int(nt * nc),
                    "d2h_bytes_per_step": int(nt * nc),
                    "ms_per_step": e2e_s * 1e3},
            "gpu_launches": args.steps * 9, "clocks": ck}
        if not args.no_cpu_baseline:
            import oracle
            sub = xh.numpy()[:2048]
            t0 = time.perf_counter()
            oracle.rfi_clean(sub)
            el = time.perf_counter() - t0
            result["cpu_baseline"] = {
                "value": sub.size / el, "unit": "samples/s", "cores": 1,
                "kind": "oracle",
                "sample": f"the first 2048 spectra of the block ({el:.1f} s, "
                          "one thread)"}
        print(json.dumps(result), flush=True)
    r.close()
    return 0


# ----------------------------------------------------- uneven multi-beam batch
def run_batch(args):
    """160 beams of uneven shape (1024/2048/4096 channels in a 2:1:1 mix,
    65536-262144-sample blocks, DM ranges 0-100/0-250/0-500 with 256-2048
    trials, 0-5 injected pulses each).  One step = the dedispersion of all
    beams (persistent relayout launches over a work queue, or beam after
    beam through the interleaved kernel: the autotuner picks the mode and
    the tile) + one batched search launch, replayed from a CUDA graph; the
    rows are ingested (unpacked) once beforehand, as a ring buffer holds
    them.  Beside it: the plain path, each beam's dedispersion and search as
    separate launches with the persistent mode's relayout tile, and the
    plain path with each plan's default (interleaved) tile on the beams
    whose staging rows fit beside the batch, compared by adds per second."""
    import ctypes as C
    import torch
    from paper_2605_03531_b300 import Batch, Plan, _lib, build, shard, synth
    build.build()
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    cfgs = synth.config3(nbeams=args.nbeams or 160, seed=shard.rank_seed(3, rank))
    plans = [Plan(c.nchan, c.f_top, c.chan_bw, c.tsamp, c.dm_list(), c.widths,
                  nbits=8, norm_window=c.norm_window, cand_capacity=1 << 16)
             for c in cfgs]
    nins = [c.nsamp_out + p.max_delay for c, p in zip(cfgs, plans)]
    batch = Batch(plans, nins)
    stream = torch.cuda.current_stream(dev)
    for b, (c, p) in enumerate(zip(cfgs, plans)):
        x = synth.noise_u8(nins[b], c.nchan, c.seed, device=dev)
        synth.inject_pulses(x, c.pulses, c.f_top, c.chan_bw, c.tsamp, c.seed)
        batch.ingest(b, x, stream=stream)
        torch.cuda.synchronize(dev)
        del x
    adds = sum(c.nchan * c.nsamp_out * c.ndm for c in cfgs)
    tune_ms, best = batch.autotune(reps=1, stream=stream)
    tile = batch.get_tile()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(e0.elapsed_time(e1), world) / steps

    def batched():
        batch.run(7.0, use_graph=True, stream=stream)

    L = _lib.lib()
    rows = [batch.input_rows(b) for b in range(len(plans))]
    # the plain path runs every plan with the batch's own kernel shape (the
    # relayout tile and the beam's chunk), so the comparison is launch
    # structure only; it also needs no staging rows beside the batch's
    # channel-major pool (the interleaved tile's 4 bytes per sample for all
    # 160 plans would not fit in HBM)
    for b, p in enumerate(plans):
        bt = batch.beam_tile(b)
        p.set_tile(bt["dm_tile"], bt["dm_per_thread"], bt["chan_chunk"],
                   tile["stages"], 8)

    def plain():
        for b, p in enumerate(plans):
            ptr, pitch, _ = rows[b]
            _lib.check(L.ddsp_dedisperse_cm(
                p._h, C.c_void_p(ptr), pitch, cfgs[b].nsamp_out,
                C.c_void_p(batch.series[b].data_ptr()),
                C.c_void_p(stream.cuda_stream)), "ddsp_dedisperse_cm")
            p.single_pulse_search(batch.series[b], 7.0, stream=stream)

    ms_batch = timed(batched, args.steps, max(args.warmup, 2))
    batch.check(stream)
    ncand = sum(p.count() for p in plans)
    ms_plain = timed(plain, max(1, args.steps // 2), 1)
    value = world * adds / (ms_batch * 1e-3)

    # the plain path with each plan's default tile (the interleaved kernel:
    # 4-byte staging rows per plan, interleaved from the channel-major rows
    # first), on the first beams whose staging fits beside the batch in
    # HBM; compared by adds per second
    free, _ = torch.cuda.mem_get_info(dev)
    budget = free - (8 << 30)
    dplans, dsel = [], []
    for b, c in enumerate(cfgs):
        q = Plan(c.nchan, c.f_top, c.chan_bw, c.tsamp, c.dm_list(), c.widths,
                 nbits=8, norm_window=c.norm_window, cand_capacity=1 << 16)
        need = 4 * c.nchan * (nins[b] + 4096)
        if need > budget or q.cm_pitch(c.nsamp_out) > rows[b][1]:
            q.close()
            continue
        budget -= need
        dplans.append(q)
        dsel.append(b)
    adds_sel = sum(cfgs[b].nchan * cfgs[b].nsamp_out * cfgs[b].ndm
                   for b in dsel)

    def plain_default():
        for q, b in zip(dplans, dsel):
            ptr, pitch, _ = rows[b]
            _lib.check(L.ddsp_dedisperse_cm(
                q._h, C.c_void_p(ptr), pitch, cfgs[b].nsamp_out,
                C.c_void_p(batch.series[b].data_ptr()),
                C.c_void_p(stream.cuda_stream)), "ddsp_dedisperse_cm")
            q.single_pulse_search(batch.series[b], 7.0, stream=stream)

    ms_pd = timed(plain_default, max(1, args.steps // 2), 1) if dsel else None
    plain_default_rec = None
    if dsel:
        plain_default_rec = {
            "beams": len(dsel), "adds_per_step": adds_sel,
            "value": world * adds_sel / (ms_pd * 1e-3), "ms_per_step": ms_pd,
            "kernel": "each plan's default tile (interleaved), per beam"}
    for q in dplans:
        q.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"{len(cfgs)} uneven beams in one batched step "
                                   "(CUDA graph, autotuned mode and tile): 1024/2048/"
                                   "4096 ch, 65536-262144 samples, DM 0-100/250/500 "
                                   "x 256-2048 trials", "beams": len(cfgs),
                       "adds_per_step": adds,
                       "l2": "inputs larger than L2"},
            "mode": "per_beam" if batch.get_mode() == Batch.PER_BEAM
                    else "persistent",
            "plain_per_beam": {"value": world * adds / (ms_plain * 1e-3),
                               "ms_per_step": ms_plain,
                               "launches_per_step": 2 * len(cfgs),
                               "kernel": "relayout tile of the persistent "
                                         "mode, per beam"},
            "batched_over_plain": ms_plain / ms_batch,
            "plain_default_tile": plain_default_rec,
            "batched_over_plain_default": (
                value / plain_default_rec["value"] if plain_default_rec
                else None),
            "tile": tile, "autotune_ms": tune_ms, "autotune_best": best,
            "candidates_per_step": int(ncand), "gpu_launches": 3 * args.steps}),
            flush=True)
    return 0


# ------------------------------------------------ streaming serving (c5)
def run_serve(args):
    """Beams of the 4096-channel config2 shape stream 16384-spectrum blocks
    (67 MB, one per 1.342 s per beam) with seeded Poisson-jittered arrivals;
    the server ingests them into per-beam rings and searches every waiting
    block in continuous-batching steps.  Reported: the largest beam count
    (multiple of 16 in 64..448) whose p99 block latency stays below the
    1.342 s period, for batched steps and for one beam per step (the plain
    per-beam path), found by bisection on real-time runs of --steps blocks
    per beam.  Blocks come from a pool of pinned host blocks (noise plus
    pulses) and reach the device through a separate copy stream."""
    import torch
    from paper_2605_03531_b300 import Plan, Server, build, synth
    from paper_2605_03531_b300.serve import (DeviceStager, ServingLoop,
                                             realtime_limit)
    build.build()
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    cfg = synth.config5(1)[0]
    B, T = cfg.nsamp_out, synth.BLOCK_PERIOD_S
    plan = Plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
                cfg.widths, nbits=8, norm_window=cfg.norm_window,
                cand_capacity=1 << 18)
    adds_block = cfg.nchan * B * cfg.ndm
    # pool of host blocks
    pool = []
    for i in range(8):
        x = synth.noise_u8(B, cfg.nchan, cfg.seed + 17 * i, device=dev)
        synth.inject_pulses(x, synth.random_pulses(2, cfg.nchan, B - 4096, seed=i,
                                                   dm_range=(10.0, 240.0), wmax=64,
                                                   snr_range=(10.0, 30.0),
                                                   spacing=4096),
                            cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.seed + i)
        pool.append(x.cpu().pin_memory())
        del x
    compute = torch.cuda.Stream(dev)
    stager = DeviceStager(16, (B, cfg.nchan), compute)
    reserve = 4 << 30

    # dedispersion: the fastest full step of 32 beams among the server's
    # relayout shapes and its interleaved mode (8 staging slots)
    tiles = [(16, 8, 8, 2), (8, 8, 4, 2), (16, 8, 4, 2), (8, 8, 6, 2),
             (16, 8, 4, 4), (8, 4, 4, 2), (16, 4, 6, 2), (8, 4, 8, 2),
             ("interleaved", 8)]

    def make_server(t, n):
        if t[0] == "interleaved":
            srv = Server(plan, B, n, reserve)
            srv.set_mode(Server.INTERLEAVED, t[1])
            return srv
        return Server(plan, B, n, reserve, tile=t)

    tune = {}
    for t in tiles:
        try:
            srv = make_server(t, 32)
        except Exception:
            continue
        bs = [srv.admit() for _ in range(32)]
        blocks = [stager.stage(pool[i % 8]) for i in range(2)]
        ms = []
        for rep in range(3):
            for b in bs:
                x, tok = blocks[rep % 2]
                srv.push(b, x, stream=compute)
                stager.consumed(tok)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(compute)
            srv.step(cfg.threshold, stream=compute)
            e1.record(compute)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        tune[t] = min(ms[1:])
        srv.close()
        torch.cuda.synchronize(dev)
    tile = min(tune, key=tune.get)

    def run_at(n, per_step, inflight, min_batch=1):
        try:
            srv = make_server(tile, n)
        except Exception:
            return float("inf")
        beams = []
        try:
            for _ in range(n):
                beams.append(srv.admit())
        except Exception:
            srv.close()
            return float("inf")
        # fill every ring first (untimed): the first timed block's window
        # then holds only stream data, as in steady operation
        warm = -(-(srv.first_delay + srv.carry) // B)
        for k in range(warm):
            for i, b in enumerate(beams):
                x, tok = stager.stage(pool[(3 * i + k) % 8])
                srv.push(b, x, stream=compute)
                stager.consumed(tok)
            srv.step(cfg.threshold, stream=compute)
        srv.check(compute)
        arr = synth.arrival_times(n, args.steps, seed=5)
        loop = ServingLoop(srv, beams, lambda i, k: pool[(3 * i + warm + k) % 8],
                           cfg.threshold, stager=stager, compute_stream=compute,
                           max_beams_in_step=per_step, first_block=warm,
                           max_inflight=inflight, device_timing=True,
                           min_batch=min_batch, max_wait=0.05)
        res = loop.run(arr, time_limit=args.steps * T + 60.0)
        srv.check(compute)
        srv.close()
        torch.cuda.synchronize(dev)
        lat = res.latency
        p99 = float("inf") if not np.isfinite(lat).all() else res.percentile(99)
        duty = res.busy / (args.steps * T)
        runs[(n, per_step)] = {
            "p50_s": res.percentile(50), "p99_s": p99,
            "max_s": float(np.nanmax(lat)),
            "mean_beams_per_step": float(np.mean(res.step_sizes)),
            "steps": len(res.step_sizes), "device_duty": duty,
            "sustained_adds_per_s": n * args.steps * adds_block / res.wall,
            "candidates_per_block": float(res.ncand.mean())}
        # a device busier than the stream's own time falls behind without
        # bound, whatever the run's latencies show
        return p99 if duty < 1.0 else float("inf")

    runs = {}
    clk = ClockSampler(local if world > 1 else 0)
    clk.start()
    # each path at its own best queue depth: batched steps already keep the
    # device busy, one-beam steps need a second step queued to hide the
    # host's turnaround between launches
    n_batched, _ = realtime_limit(lambda n: run_at(n, 0, args.inflight, 4),
                                  64, 448, 16, T)
    n_plain, _ = realtime_limit(lambda n: run_at(n, 1, args.plain_inflight),
                                64, 448, 16, T)
    clocks = clk.stop()
    if rank == 0:
        def table(per_step):
            return {str(n): v for (n, ps), v in sorted(runs.items()) if ps == per_step}
        print(json.dumps({
            "metric": "real-time beams per B300 at p99", "value": n_batched * world,
            "unit": "beams", "n_gpus": world, "steps": args.steps,
            "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "streaming 4096-ch beams (300-500 MHz, "
                                   "81.92 us), 16384-spectrum blocks every "
                                   f"{T:.4f} s, 1024 DMs 0-250, widths 1-256, "
                                   "Poisson-jittered arrivals",
                       "deadline_s": T, "blocks_per_beam": args.steps,
                       "steps_in_flight": {"batched": args.inflight,
                                           "plain_per_beam": args.plain_inflight},
                       "adds_per_block": adds_block,
                       "dedispersion": ({"mode": "interleaved",
                                         "staging_slots": tile[1]}
                                        if tile[0] == "interleaved" else
                                        {"mode": "relayout",
                                         **dict(zip(("dm_tile", "dm_per_thread",
                                                     "chan_chunk", "stages"),
                                                    tile))}),
                       "step_ms_32_beams": {str(k): v for k, v in tune.items()}},
            "batched": table(0),
            "plain_per_beam": {"value": n_plain * world, "runs": table(1)},
            "clocks": clocks}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-serving", action="store_true",
                    help="beam workload: skip the bounded serving check")
    ap.add_argument("--workload", choices=["beam", "sps", "batch", "serve",
                                           "servestep", "peaks",
                                           "cluster", "dered", "ffa",
                                           "resample", "rfi"],
                    default="beam",
                    help="beam: the full path on one 4096-channel beam block "
                         "(headline); sps: the search-only stress case; batch: "
                         "160 uneven beams in one persistent launch; serve: "
                         "real-time streaming beams (--steps blocks per beam); "
                         "servestep: device time of one serving step of "
                         "--nbeams beams (profiling); "
                         "cluster: peaks filter + DBSCAN of a candidate list; "
                         "dered: running-median de-reddening of the beam's "
                         "series; ffa: folding transform + profile search; "
                         "resample: resampling for frequency derivatives; "
                         "rfi: gptool-style RFI cleaning of a block; peaks: "
                         "microbenchmarks of the shared-memory and integer "
                         "ALU rates per SM clock")
    ap.add_argument("--nbeams", type=int, default=0,
                    help="batch: beams (0 = 160); servestep: beams (0 = 8)")
    ap.add_argument("--inflight", type=int, default=1,
                    help="serve: batched steps queued on the device at once")
    ap.add_argument("--plain-inflight", type=int, default=2,
                    help="serve: one-beam steps queued on the device at once")
    ap.add_argument("--nsamp-out", type=int, default=0,
                    help="beam: output samples per trial (0 = 262144)")
    ap.add_argument("--ndm", type=int, default=0, help="sps: DM trials (0 = 2048)")
    ap.add_argument("--nsamp", type=int, default=0,
                    help="sps: samples per trial (0 = 1048576)")
    ap.add_argument("--tile", default="",
                    help="beam: dedispersion tile 'dm_tile,dm_per_thread,"
                         "chan_chunk,stages,flags' (ddsp_plan_set_tile; "
                         "default: the library's choice)")
    ap.add_argument("--profile", action="store_true",
                    help="kernels only: no clocks, end-to-end or CPU baseline "
                         "(for profiler captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "sps":
        return run_sps(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "servestep":
        return run_servestep(args)
    if args.workload == "cluster":
        return run_cluster(args)
    if args.workload == "dered":
        return run_dered(args)
    if args.workload == "ffa":
        return run_ffa(args)
    if args.workload == "resample":
        return run_resample(args)
    if args.workload == "rfi":
        return run_rfi(args)
    if args.workload == "peaks":
        return run_peaks(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
