"""Seeded synthetic inputs: filterbanks with dispersed pulses, int32 series.

This module only *makes inputs*.  It holds none of the search method's
arithmetic (no integer delay table, no shift-and-sum, no boxcar, no median):
the same arrays feed the CUDA path and the CPU oracle.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
the i-th draw of stream ``seed`` is ``mix64(seed*0xD1B54A32D192ED03 +
(i+1)*0x9E3779B97F4A7C15)`` with the published 64-bit finaliser.  Because it
is counter based, any slice of an input can be regenerated on its own, on the
CPU (numpy) or on a GPU (torch), with identical bits.

Noise model (the 8-bit spectra of the paper's survey, Sec.2.2/2.4):
``q = clip(round_half_away(128 + 16 g), 0, 255)`` with ``g = Phi^-1(u)``
(inverse-CDF Gaussian, ``u`` the top 53 bits of a draw).  For noise-only
samples ``q`` is found exactly by comparing the 53-bit integer against the
255 quantisation thresholds, so every device produces the same bytes.

Pulses are simulated as a box of width ``W`` samples whose arrival time at
channel frequency ``f`` follows the cold-plasma dispersion sweep of Ch.1 Eq.1,
``t0 + K*DM*(f^-2 - f_ref^-2)/tsamp``, evaluated *continuously*: each sample
gets ``A`` times its fractional overlap with the box (a sky model, not the
search's rounded integer delays).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

K_DISP = 4148.808  # s MHz^2 per (pc cm^-3), Ch.1 Eq.1

_GAMMA = 0x9E3779B97F4A7C15
_SEEDMUL = 0xD1B54A32D192ED03
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_U64 = (1 << 64) - 1


def _s64(v: int) -> int:
    """Two's-complement int64 view of an unsigned 64-bit constant."""
    v &= _U64
    return v - (1 << 64) if v >= (1 << 63) else v


# ---------------------------------------------------------------- SplitMix64
def splitmix64_np(counter: np.ndarray, seed: int) -> np.ndarray:
    """uint64 draws for the given uint64 counters (numpy, wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = (np.uint64((seed * _SEEDMUL) & _U64)
             + (counter.astype(np.uint64) + np.uint64(1)) * np.uint64(_GAMMA))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def _lsr(z: torch.Tensor, s: int) -> torch.Tensor:
    return (z >> s) & ((1 << (64 - s)) - 1)


def splitmix64_torch(counter: torch.Tensor, seed: int) -> torch.Tensor:
    """Same draws as ``splitmix64_np`` as int64 bit patterns (torch)."""
    z = counter.to(torch.int64)
    z = (z + 1) * _s64(_GAMMA) + _s64(seed * _SEEDMUL)
    z = (z ^ _lsr(z, 30)) * _s64(_M1)
    z = (z ^ _lsr(z, 27)) * _s64(_M2)
    z = z ^ _lsr(z, 31)
    return z


def u53_np(counter, seed):
    return (splitmix64_np(np.asarray(counter, dtype=np.uint64), seed)
            >> np.uint64(11)).astype(np.int64)


def uniform_np(counter, seed):
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return u53_np(counter, seed).astype(np.float64) * (2.0 ** -53)


# ------------------------------------------------------------------ 8-bit noise
def _quant_thresholds(mean: float, sd: float, nlev: int) -> np.ndarray:
    """53-bit integer thresholds T_j with q >= j  <=>  u53 >= T_j.

    q = clip(round_half_away(mean + sd*g)) >= j  <=>  g >= (j - 0.5 - mean)/sd
    <=>  u >= Phi((j - 0.5 - mean)/sd).  Levels j = 1 .. nlev-1."""
    th = np.empty(nlev - 1, dtype=np.int64)
    for j in range(1, nlev):
        z = (j - 0.5 - mean) / sd
        p = 0.5 * math.erfc(-z / math.sqrt(2.0))
        th[j - 1] = min(int(math.ceil(p * 2.0 ** 53)), 1 << 53)
    return th


def noise_u8(nsamp: int, nchan: int, seed: int, device="cpu",
             mean: float = 128.0, sd: float = 16.0, chunk: int = 1 << 26,
             out: torch.Tensor | None = None) -> torch.Tensor:
    """Time-major uint8 spectra [nsamp][nchan] of quantised Gaussian noise.

    Sample (s, c) uses counter s*nchan + c of stream ``seed``."""
    th = torch.from_numpy(_quant_thresholds(mean, sd, 256)).to(device)
    n = nsamp * nchan
    if out is None:
        out = torch.empty(n, dtype=torch.uint8, device=device)
    flat = out.view(-1)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        ctr = torch.arange(lo, hi, dtype=torch.int64, device=device)
        u = _lsr(splitmix64_torch(ctr, seed), 11)
        flat[lo:hi] = torch.searchsorted(th, u, right=True).to(torch.uint8)
        del ctr, u
    return out.view(nsamp, nchan)


def noise_u8_np(nsamp, nchan, seed, mean=128.0, sd=16.0):
    """numpy twin of ``noise_u8`` (used to cross-check the torch version)."""
    th = _quant_thresholds(mean, sd, 256)
    u = u53_np(np.arange(nsamp * nchan, dtype=np.uint64), seed)
    return np.searchsorted(th, u, side="right").astype(np.uint8).reshape(nsamp, nchan)


# --------------------------------------------------------------- pulses
@dataclass
class Pulse:
    dm: float          # pc cm^-3
    t0: float          # arrival sample at the reference (highest) frequency
    width: float       # samples
    amp: float         # added per channel per fully covered sample


def channel_freqs(nchan, f_top, chan_bw):
    return f_top + np.arange(nchan, dtype=np.float64) * chan_bw


def sweep(nchan, f_top, chan_bw, tsamp, dm):
    """Continuous arrival offset (samples) of a DM-``dm`` signal per channel,
    relative to the highest channel frequency (Ch.1 Eq.1)."""
    f = channel_freqs(nchan, f_top, chan_bw)
    fr = f.max()
    return K_DISP * dm * (1.0 / f ** 2 - 1.0 / fr ** 2) / tsamp


def _round_half_away(x):
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def inject_pulses(x: torch.Tensor, pulses, f_top, chan_bw, tsamp, seed,
                  mean=128.0, sd=16.0):
    """Add dispersed box pulses to noise spectra made by ``noise_u8``.

    Only the samples a pulse touches are rewritten, each from the same draw
    as its noise value: q = clip(round(mean + sd*Phi^-1(u) + A*overlap))."""
    from scipy.special import ndtri

    nsamp, nchan = x.shape
    if not pulses:
        return x
    ss, cc, add = [], [], []
    for p in pulses:
        tau = p.t0 + sweep(nchan, f_top, chan_bw, tsamp, p.dm)
        for c in range(nchan):
            a, b = tau[c], tau[c] + p.width
            n0, n1 = int(math.floor(a)), int(math.ceil(b))
            n = np.arange(max(n0, 0), min(n1, nsamp))
            if n.size == 0:
                continue
            ov = np.minimum(n + 1, b) - np.maximum(n, a)
            ok = ov > 0
            ss.append(n[ok])
            cc.append(np.full(int(ok.sum()), c))
            add.append(p.amp * ov[ok])
    s = np.concatenate(ss)
    c = np.concatenate(cc)
    a = np.concatenate(add)
    # several pulses may touch one sample: sum their contributions
    key = s.astype(np.int64) * nchan + c
    order = np.argsort(key, kind="stable")
    key, a = key[order], a[order]
    uk, first = np.unique(key, return_index=True)
    tot = np.add.reduceat(a, first)
    g = ndtri(uniform_np(uk.astype(np.uint64), seed))
    g = np.where(np.isfinite(g), g, 0.0)
    q = np.clip(_round_half_away(mean + sd * g + tot), 0, 255).astype(np.uint8)
    flat = x.view(-1)
    idx = torch.from_numpy(uk).to(x.device)
    flat[idx] = torch.from_numpy(q).to(x.device)
    return x


# --------------------------------------------------------------- configs
@dataclass
class FilterbankConfig:
    name: str
    nchan: int
    f_top: float
    chan_bw: float
    tsamp: float
    nsamp_out: int          # output samples wanted per DM trial
    dm_lo: float
    dm_hi: float
    ndm: int
    widths: list
    threshold: float
    seed: int
    norm_window: int = 8192
    pulses: list = field(default_factory=list)

    def dm_list(self):
        """Linear grid DM_i = lo + i*(hi - lo)/(n - 1)."""
        if self.ndm == 1:
            return np.array([self.dm_lo], dtype=np.float64)
        i = np.arange(self.ndm, dtype=np.float64)
        return self.dm_lo + i * (self.dm_hi - self.dm_lo) / (self.ndm - 1)


def config1() -> FilterbankConfig:
    """256 ch over 550-750 MHz, tsamp 1.31072 ms, 16384 samples, one pulse
    at DM 100 (W = 4, +24 per channel, t0 = 8000), DMs 0..255, widths 1..32,
    threshold 7, seed 1."""
    return FilterbankConfig(
        name="c1-256ch-16384s-256dm", nchan=256, f_top=750.0, chan_bw=-0.78125,
        tsamp=1.31072e-3, nsamp_out=16384 - 1226, dm_lo=0.0, dm_hi=255.0,
        ndm=256, widths=[1, 2, 4, 8, 16, 32], threshold=7.0, seed=1,
        pulses=[Pulse(dm=100.0, t0=8000.0, width=4.0, amp=24.0)])


def config2() -> FilterbankConfig:
    """4096 ch over 300-500 MHz, tsamp 81.92 us, 262144-sample block plus
    the max-delay overlap, 1024 DMs over 0-250, widths 1..256, 20 pulses
    with DM ~ U(10, 240), W ~ U{1..64}, S/N ~ U(8, 30), seed 2."""
    cfg = FilterbankConfig(
        name="c2-4096ch-262144s-1024dm", nchan=4096, f_top=500.0,
        chan_bw=-0.048828125, tsamp=81.92e-6, nsamp_out=262144, dm_lo=0.0,
        dm_hi=250.0, ndm=1024, widths=[1 << i for i in range(9)],
        threshold=7.0, seed=2)
    cfg.pulses = random_pulses(20, cfg.nchan, 262144, seed=cfg.seed,
                               dm_range=(10.0, 240.0), wmax=64,
                               snr_range=(8.0, 30.0), spacing=12800)
    return cfg


def random_pulses(n, nchan, nsamp_out, seed, dm_range, wmax, snr_range,
                  spacing, sd=16.0):
    """n pulses, t0 spaced by ``spacing`` with a random jitter; per-channel
    amplitude A = S/N*sd/sqrt(nchan*W) so the matched boxcar reaches S/N."""
    ctr = np.arange(4 * n, dtype=np.uint64) + np.uint64(1 << 40)
    u = uniform_np(ctr, seed).reshape(n, 4)
    out = []
    for i in range(n):
        dm = dm_range[0] + u[i, 0] * (dm_range[1] - dm_range[0])
        w = 1 + int(u[i, 1] * wmax)
        snr = snr_range[0] + u[i, 2] * (snr_range[1] - snr_range[0])
        t0 = 4096 + i * spacing + int(u[i, 3] * 4096)
        if t0 + w >= nsamp_out:
            break
        amp = snr * sd / math.sqrt(nchan * w)
        out.append(Pulse(dm=dm, t0=float(t0), width=float(w), amp=amp))
    return out


def filterbank(cfg: FilterbankConfig, nsamp_in: int, device="cpu") -> torch.Tensor:
    """Noise plus the config's pulses, time-major uint8 [nsamp_in][nchan]."""
    x = noise_u8(nsamp_in, cfg.nchan, cfg.seed, device=device)
    return inject_pulses(x, cfg.pulses, cfg.f_top, cfg.chan_bw, cfg.tsamp,
                         cfg.seed)


def noise_u16(nsamp, nchan, seed, device="cpu", lo=0, hi=65536):
    """Uniform uint16 spectra (held as int32 values < 2^16, returned as a
    torch.uint16 tensor) from the same counter stream."""
    ctr = torch.arange(nsamp * nchan, dtype=torch.int64, device=device)
    u = _lsr(splitmix64_torch(ctr, seed), 11)
    v = lo + (u % (hi - lo))
    return v.to(torch.int32).to(torch.uint16).view(nsamp, nchan)


# ------------------------------------------------------- int32 series (SPS)
def gaussian_series(ndm, n, seed, mean=524288.0, sd=1024.0, device="cpu",
                    event_rate=1e-3, wmax=1024, snr_range=(6.0, 50.0),
                    row_chunk=64, out=None):
    """int32 series [ndm][n] = round(mean + sd*g) plus boxcar events.

    Events start at a fraction ``event_rate`` of positions (counter stream
    seed+1), widths log-uniform over the powers of two 1..wmax (stream
    seed+2), per-sample amplitude round(S/N*sd/sqrt(w)) with S/N uniform in
    ``snr_range`` (stream seed+3)."""
    from math import log2
    nlev = int(log2(wmax)) + 1
    if out is None:
        out = torch.empty((ndm, n), dtype=torch.int32, device=device)
    for r0 in range(0, ndm, row_chunk):
        r1 = min(ndm, r0 + row_chunk)
        ctr = (torch.arange(r0 * n, r1 * n, dtype=torch.int64, device=device))
        u = _lsr(splitmix64_torch(ctr, seed), 11).to(torch.float64) * (2.0 ** -53)
        g = torch.special.ndtri(u.clamp_min(2.0 ** -60))
        x = torch.floor(mean + sd * g + 0.5)   # values are positive here
        del u, g
        if event_rate > 0:
            ue = _lsr(splitmix64_torch(ctr, seed + 1), 11).to(torch.float64) * (2.0 ** -53)
            ev = ue < event_rate
            del ue
            idx = torch.nonzero(ev.view(-1)).view(-1)
            del ev
            if idx.numel():
                gi = idx + r0 * n
                uw = _lsr(splitmix64_torch(gi, seed + 2), 11).to(torch.float64) * (2.0 ** -53)
                w = torch.pow(2, torch.floor(uw * nlev)).to(torch.int64)
                us = _lsr(splitmix64_torch(gi, seed + 3), 11).to(torch.float64) * (2.0 ** -53)
                snr = snr_range[0] + us * (snr_range[1] - snr_range[0])
                a = torch.floor(snr * sd / torch.sqrt(w.to(torch.float64)) + 0.5)
                rows = idx // n
                cols = idx % n
                diff = torch.zeros((r1 - r0, n + 1), dtype=torch.float64, device=device)
                flatd = diff.view(-1)
                flatd.index_add_(0, rows * (n + 1) + cols, a)
                end = torch.clamp(cols + w, max=n)
                flatd.index_add_(0, rows * (n + 1) + end, -a)
                x += torch.cumsum(diff, dim=1)[:, :n].reshape(-1)
                del diff
        out[r0:r1] = x.view(r1 - r0, n).to(torch.int32)
        del x, ctr
    return out


# --------------------------------------------------------- uneven beam mix
def config3(nbeams=160, seed=3, nsamp_range=(65536, 262144),
            nchan_choices=(1024, 1024, 2048, 4096), dm_hi_choices=(100.0, 250.0, 500.0),
            ndm_choices=(256, 512, 1024, 2048)):
    """Beams of uneven shape over 300-500 MHz at 81.92 us: channel counts in
    a 2:1:1 mix of 1024/2048/4096, output blocks uniform in `nsamp_range`
    (multiples of 4096), DM ranges 0-100/0-250/0-500 with 256..2048 trials,
    0-5 dispersed pulses each (DM within the range, W ~ U{1..64}, S/N ~
    U(8, 30)); widths 1..256, threshold 7, L 8192.  Returns a list of
    FilterbankConfig, one per beam, each with its own noise seed."""
    ctr = np.arange(8 * nbeams, dtype=np.uint64) + np.uint64(1 << 41)
    u = uniform_np(ctr, seed).reshape(nbeams, 8)
    lo, hi = nsamp_range[0] // 4096, nsamp_range[1] // 4096
    beams = []
    for b in range(nbeams):
        nchan = nchan_choices[int(u[b, 0] * len(nchan_choices))]
        nout = 4096 * (lo + int(u[b, 1] * (hi - lo + 1)))
        dm_hi = dm_hi_choices[int(u[b, 2] * len(dm_hi_choices))]
        ndm = ndm_choices[int(u[b, 3] * len(ndm_choices))]
        npulse = int(u[b, 4] * 6)
        cfg = FilterbankConfig(
            name=f"c3-beam{b}", nchan=nchan, f_top=500.0, chan_bw=-200.0 / nchan,
            tsamp=81.92e-6, nsamp_out=nout, dm_lo=0.0, dm_hi=dm_hi, ndm=ndm,
            widths=[1 << i for i in range(9)], threshold=7.0,
            seed=seed * 100000 + b)
        spacing = max(4096, nout // max(npulse, 1) - 4096)
        cfg.pulses = random_pulses(npulse, nchan, nout, seed=cfg.seed,
                                   dm_range=(0.05 * dm_hi, 0.95 * dm_hi), wmax=64,
                                   snr_range=(8.0, 30.0), spacing=spacing)
        beams.append(cfg)
    return beams


# ------------------------------------------------------ streaming arrivals (c5)
BLOCK_PERIOD_S = 16384 * 81.92e-6   # one 16384-spectrum block at 81.92 us


def arrival_times(nbeams, nblocks, period=BLOCK_PERIOD_S, seed=5,
                  jitter_mean=0.05):
    """Arrival time (s) of block k of beam b: k*period + phi_b + e_bk, with
    a per-beam phase phi_b ~ U[0, period) and an exponential delay e_bk of
    mean `jitter_mean` (inverse CDF of counter-based uniforms).  Returns
    float64 [nbeams, nblocks], increasing along each beam."""
    nb, nk = int(nbeams), int(nblocks)
    ctr_phase = np.arange(nb, dtype=np.uint64) + np.uint64(1 << 44)
    phi = uniform_np(ctr_phase, seed) * period
    ctr = np.arange(nb * nk, dtype=np.uint64) + np.uint64(1 << 45)
    u = uniform_np(ctr, seed).reshape(nb, nk)
    e = -jitter_mean * np.log1p(-u)
    t = np.arange(nk, dtype=np.float64)[None, :] * period + phi[:, None] + e
    # a block cannot arrive before the one before it
    return np.maximum.accumulate(t, axis=1)


def config5(nbeams=64, seed=5):
    """Streaming beams of the 4096-channel shape of config2 (300-500 MHz,
    81.92 us, 1024 DMs over 0-250, widths 1..256, L 8192) delivering
    16384-spectrum blocks; one FilterbankConfig per beam (nsamp_out = one
    block) with its own seed."""
    base = config2()
    beams = []
    for b in range(int(nbeams)):
        cfg = FilterbankConfig(
            name=f"c5-beam{b}", nchan=base.nchan, f_top=base.f_top,
            chan_bw=base.chan_bw, tsamp=base.tsamp, nsamp_out=16384,
            dm_lo=base.dm_lo, dm_hi=base.dm_hi, ndm=base.ndm,
            widths=list(base.widths), threshold=base.threshold,
            seed=seed * 100000 + b)
        beams.append(cfg)
    return beams



def config5_stream(nblocks=10, seed=500000, block=16384):
    """One beam's continuous stream of the c5 shape for checking the serving
    path block by block: (FilterbankConfig of the c2 channel / DM shape,
    time-major uint8 [nblocks*block][4096] on the CPU).  Noise from stream
    ``seed``; dispersed pulses every ~0.6 block (DM U(20, 240), W U{1..64},
    S/N U(10, 30)), so pulses straddle block boundaries and sweep across
    several blocks of the ring."""
    base = config2()
    cfg = FilterbankConfig(
        name=f"c5-stream-{nblocks}x{block}", nchan=base.nchan, f_top=base.f_top,
        chan_bw=base.chan_bw, tsamp=base.tsamp, nsamp_out=block,
        dm_lo=base.dm_lo, dm_hi=base.dm_hi, ndm=base.ndm,
        widths=list(base.widths), threshold=base.threshold, seed=seed)
    n = nblocks * block
    cfg.pulses = random_pulses(n // 10000, cfg.nchan, n, seed=seed,
                               dm_range=(20.0, 240.0), wmax=64,
                               snr_range=(10.0, 30.0), spacing=10000)
    x = noise_u8(n, cfg.nchan, seed)
    inject_pulses(x, cfg.pulses, cfg.f_top, cfg.chan_bw, cfg.tsamp, seed)
    return cfg, x

# ------------------------------------------------- single-pulse candidate lists
CAND_DTYPE = np.dtype([("dm_idx", np.uint32), ("t", np.uint32),
                       ("w_idx", np.uint32), ("snr", np.float32)])


def candidate_list(ndm, nsamp, nwidths, n_events, seed, thr=6.5,
                   snr_range=(8.0, 50.0), dm_half=(1, 40), t_half=(1, 256),
                   noise=0, quantum=0.0):
    """Seeded single-pulse candidate records in the DM-time plane, shaped
    like a search's output for the peaks filter and the clustering stage.

    Event e (stream ``seed``, counters e*8 ..): centre (k_e, t_e) uniform on
    the plane, peak S/N S_e uniform in ``snr_range``, half extents a_e trials
    and b_e samples log-uniform in ``dm_half`` / ``t_half``, width index w_e
    uniform.  It yields a record at every (k, t) of its rectangle whose
    S/N = S_e * (1 - |dk|/(a_e+1)) * (1 - |dt|/(b_e+1)) reaches ``thr``, with
    width index w_e where |dt| <= b_e/2, else max(w_e - 1, 0).  ``quantum`` >
    0 rounds every S/N to a multiple of it (exact ties between neighbours).
    ``noise`` isolated records (stream seed+1) sit uniformly on the plane
    with S/N thr + 0.5*Exp(1).  Where records meet at one (k, t) the one
    with the largest S/N stays (then the first made).  The records come back
    in a seeded random order (stream seed+2), as an unordered search
    emits them."""
    parts_k, parts_t, parts_w, parts_s = [], [], [], []
    if n_events > 0:
        u = uniform_np(np.arange(8 * n_events, dtype=np.uint64),
                       seed).reshape(n_events, 8)
        for e in range(n_events):
            ke = int(u[e, 0] * ndm)
            te = int(u[e, 1] * nsamp)
            se = snr_range[0] + u[e, 2] * (snr_range[1] - snr_range[0])
            a = int(round(math.exp(math.log(dm_half[0]) + u[e, 3] *
                                   (math.log(dm_half[1]) - math.log(dm_half[0])))))
            b = int(round(math.exp(math.log(t_half[0]) + u[e, 4] *
                                   (math.log(t_half[1]) - math.log(t_half[0])))))
            we = min(int(u[e, 5] * nwidths), nwidths - 1)
            dk = np.arange(-a, a + 1)
            dt = np.arange(-b, b + 1)
            kk = ke + dk[:, None] + 0 * dt[None, :]
            tt = te + dt[None, :] + 0 * dk[:, None]
            sn = (se * (1.0 - np.abs(dk)[:, None] / (a + 1.0))
                  * (1.0 - np.abs(dt)[None, :] / (b + 1.0)))
            ww = np.where(np.abs(dt)[None, :] + 0 * dk[:, None] <= b // 2, we,
                          max(we - 1, 0))
            m = (kk >= 0) & (kk < ndm) & (tt >= 0) & (tt < nsamp) & (sn >= thr)
            parts_k.append(kk[m])
            parts_t.append(tt[m])
            parts_w.append(ww[m])
            parts_s.append(sn[m])
    if noise > 0:
        u = uniform_np(np.arange(4 * noise, dtype=np.uint64),
                       seed + 1).reshape(noise, 4)
        parts_k.append((u[:, 0] * ndm).astype(np.int64))
        parts_t.append((u[:, 1] * nsamp).astype(np.int64))
        parts_w.append(np.minimum((u[:, 2] * nwidths).astype(np.int64),
                                  nwidths - 1))
        parts_s.append(thr - 0.5 * np.log1p(-u[:, 3]))
    if not parts_k:
        return np.zeros(0, dtype=CAND_DTYPE)
    k = np.concatenate(parts_k).astype(np.int64)
    t = np.concatenate(parts_t).astype(np.int64)
    w = np.concatenate(parts_w).astype(np.int64)
    s = np.concatenate(parts_s)
    if quantum > 0:
        s = np.round(s / quantum) * quantum
    s32 = s.astype(np.float32)
    # one record per (k, t): the strongest, then the first made
    key = k * nsamp + t
    order = np.lexsort((np.arange(key.size), -s32.astype(np.float64), key))
    first = np.ones(order.size, dtype=bool)
    first[1:] = key[order][1:] != key[order][:-1]
    sel = order[first]
    out = np.empty(sel.size, dtype=CAND_DTYPE)
    out["dm_idx"] = k[sel]
    out["t"] = t[sel]
    out["w_idx"] = w[sel]
    out["snr"] = s32[sel]
    perm = np.argsort(splitmix64_np(np.arange(sel.size, dtype=np.uint64),
                                    seed + 2), kind="stable")
    return out[perm]


def red_series(ndm, n, seed, amp=3000.0, period=(40000, 200000), device="cpu",
               out=None):
    """``gaussian_series`` (mean 524288, sd 1024, 0.1% boxcar events) plus a
    slowly varying baseline per row, the "red noise" of Sec.3.3:
    round(amp * sin(2 pi t / P_k + phi_k)), period P_k log-uniform in
    ``period`` samples and phase phi_k uniform (stream seed+7)."""
    x = gaussian_series(ndm, n, seed, device=device, out=out)
    u = uniform_np(np.arange(2 * ndm, dtype=np.uint64), seed + 7).reshape(ndm, 2)
    lp = np.log(period[0]) + u[:, 0] * (np.log(period[1]) - np.log(period[0]))
    P = torch.from_numpy(np.exp(lp)).to(device)
    phi = torch.from_numpy(2 * np.pi * u[:, 1]).to(device)
    t = torch.arange(n, dtype=torch.float64, device=device)
    for r0 in range(0, ndm, 64):
        r1 = min(ndm, r0 + 64)
        base = amp * torch.sin(2 * np.pi * t[None, :] / P[r0:r1, None]
                               + phi[r0:r1, None])
        x[r0:r1] += torch.round(base).to(torch.int32)
    return x
