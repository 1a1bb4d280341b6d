"""GPU parity of unpack + dedispersion against the CPU oracle (bit-exact).

Covers every tile shape of the staged kernel and the direct kernel, ragged
channel / sample / DM counts, unsorted DM lists, uint16 input, the
256-channel configuration in full, and the 4096-channel 262144-sample
configuration at full size on sampled outputs plus the DM = 0 invariant."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import DdspError, Plan, build, synth
from paper_2605_03531_b300 import _lib as ddsp_lib

pytestmark = pytest.mark.gpu

# (dm_tile, dm_per_thread, chan_chunk, stages, flags); dm_tile 0 = library's
# choice, -1 = direct kernel; flags 1 = single element buffer, 4 = int32
# totals in registers (only with 1), 8 = warp-specialised kernel, 16 =
# interleaved rows staged by TMA, 48 = that with 16 consumer warps
TILES = [(0, 4, 8, 2, 0), (4, 4, 1, 2, 0), (4, 4, 8, 3, 1), (8, 4, 8, 2, 0),
         (8, 4, 6, 3, 1), (8, 4, 32, 4, 1), (16, 4, 8, 2, 0), (16, 4, 16, 3, 1),
         (8, 4, 8, 3, 5), (16, 4, 5, 2, 5), (4, 2, 8, 2, 5), (8, 4, 7, 2, 0),
         (2, 2, 8, 2, 0), (4, 2, 5, 3, 0), (8, 2, 8, 2, 1), (8, 2, 3, 4, 1),
         # flags 8 = warp-specialised producer/consumer kernel
         (8, 4, 6, 4, 8), (16, 8, 4, 2, 8), (8, 8, 5, 2, 8), (32, 8, 3, 4, 8),
         (4, 4, 8, 2, 8), (16, 4, 7, 2, 8), (16, 8, 5, 2, 8),
         # flags 16 = TMA-staged pre-interleaved rows, a ring of 2..8 stages
         (16, 8, 7, 2, 16), (16, 8, 4, 3, 16), (16, 8, 2, 8, 16),
         (8, 8, 5, 2, 16), (32, 8, 3, 4, 16), (8, 4, 4, 4, 16),
         (4, 4, 7, 2, 16), (16, 4, 1, 8, 16), (16, 4, 6, 2, 16),
         # flags 48 = the same with 16 consumer warps (one block per SM)
         (16, 8, 11, 2, 48), (8, 8, 5, 2, 48), (32, 8, 3, 5, 48),
         (16, 8, 1, 8, 48), (16, 4, 9, 2, 48), (8, 4, 6, 3, 48),
         (4, 4, 16, 2, 48),
         (-1, 4, 8, 2, 0)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _plan(nchan, f_top, bw, ts, dms, nbits=8, widths=(1, 2, 4)):
    return Plan(nchan, f_top, bw, ts, dms, list(widths), nbits=nbits,
                norm_window=8192, cand_capacity=1 << 16)


def to_dev(x):
    """numpy uint8/uint16 array -> CUDA tensor of the same bits."""
    if x.dtype == np.uint16:
        return torch.from_numpy(x.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(x).cuda()


def from_dev(t):
    if t.dtype == torch.uint16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def _set_tile(plan, t):
    try:
        plan.set_tile(*t)
        return True
    except Exception:
        return False  # shape does not fit on chip for this plan


@pytest.mark.parametrize("nchan,nin,nbits", [(256, 1000, 8), (4096, 300, 8),
                                             (37, 777, 8), (100, 129, 8),
                                             (64, 500, 16), (33, 301, 16)])
def test_unpack_byte_exact(nchan, nin, nbits):
    rng = np.random.default_rng(nchan + nin)
    dt = np.uint8 if nbits == 8 else np.uint16
    x = rng.integers(0, np.iinfo(dt).max + 1, size=(nin, nchan)).astype(dt)
    p = _plan(nchan, 500.0, -0.1, 1e-3, [0.0], nbits=nbits)
    pitch = ((nin + 127) // 128) * 128 + 128
    out = from_dev(p.unpack(to_dev(x), pitch))
    ref = oracle.unpack(x)
    assert np.array_equal(out[:, :nin], ref)
    assert not out[:, nin:].any()


def test_plan_delays_match_oracle():
    cfg = synth.config2()
    p = _plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list())
    d_ref, D = oracle.delay_table(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp,
                                  cfg.dm_list())
    assert p.max_delay == D == 89989
    assert np.array_equal(p.delays(), d_ref)


@pytest.fixture(scope="module")
def c1():
    cfg = synth.config1()
    x = synth.filterbank(cfg, 16384)
    d, D = oracle.delay_table(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp,
                              cfg.dm_list())
    ref = oracle.dedisperse(x.numpy(), d)
    return cfg, x, ref


@pytest.mark.parametrize("tile", TILES)
def test_c1_bit_exact_every_tile(c1, tile):
    cfg, x, ref = c1
    p = _plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list())
    if not _set_tile(p, tile):
        pytest.skip("tile does not fit")
    out = p.dedisperse(x.cuda())
    torch.cuda.synchronize()
    assert out.shape == ref.shape == (256, 15158)
    assert np.array_equal(out.cpu().numpy(), ref)


SHAPES = [
    # nchan, nin, dms, nbits, f_top, bw, tsamp
    (37, 3000, np.linspace(0, 40, 5), 8, 450.0, -2.0, 1e-3),
    (100, 5000, np.random.default_rng(1).uniform(0, 60, 33), 8, 500.0, -1.0, 1e-3),
    (16, 777, [17.0], 8, 400.0, -4.0, 1e-3),
    (64, 4100, np.linspace(0, 20, 20)[::-1], 16, 420.0, -1.5, 1e-3),
    (48, 2000, np.random.default_rng(2).uniform(0, 30, 17), 16, 380.0, 1.0, 1e-3),
    (300, 3333, np.linspace(3, 9, 9), 8, 700.0, -0.5, 5e-4),
    (1, 600, np.linspace(0, 100, 7), 8, 300.0, -1.0, 1e-3),
]


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("tile", [(0, 4, 8, 2, 0), (4, 4, 3, 2, 1),
                                  (8, 4, 8, 3, 0), (16, 4, 4, 2, 1),
                                  (8, 4, 7, 3, 5), (8, 2, 7, 3, 0),
                                  (8, 2, 5, 2, 1), (8, 4, 5, 4, 8),
                                  (16, 8, 3, 2, 8), (16, 8, 7, 2, 16),
                                  (8, 4, 3, 5, 16), (4, 4, 1, 2, 16),
                                  (16, 8, 11, 2, 48), (8, 4, 5, 3, 48),
                                  (-1, 4, 8, 2, 0)])
def test_ragged_shapes_bit_exact(shape, tile):
    nchan, nin, dms, nbits, f_top, bw, ts = SHAPES[shape]
    rng = np.random.default_rng(shape)
    dt = np.uint8 if nbits == 8 else np.uint16
    hi = 256 if nbits == 8 else 65536
    x = rng.integers(0, hi, size=(nin, nchan)).astype(dt)
    p = _plan(nchan, f_top, bw, ts, dms, nbits=nbits)
    if nbits == 16 and not tile[4] & 16:
        tile = tile[:4] + (tile[4] & 1,)   # uint16 totals are always in registers
    if not _set_tile(p, tile):
        pytest.skip("tile does not fit")
    d = p.delays()
    ref = oracle.dedisperse(x, d)
    out = p.dedisperse(to_dev(x))
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_impulses_land_at_their_delays():
    """I2 on the GPU: unit impulses reappear at t = s0 - d[k][c] only."""
    nchan, nin = 96, 6000
    dms = np.linspace(0, 150, 24)
    p = _plan(nchan, 450.0, -1.0, 1e-3, dms)
    d = p.delays()
    D = p.max_delay
    nout = nin - D
    x = np.zeros((nin, nchan), dtype=np.uint8)
    hits = [(0, 100), (95, nin - 1), (50, 3000), (7, D + 5)]
    for c, s0 in hits:
        x[s0, c] = 1
    out = p.dedisperse(torch.from_numpy(x).cuda()).cpu().numpy()
    expect = np.zeros((len(dms), nout), dtype=np.int64)
    for c, s0 in hits:
        for k in range(len(dms)):
            t = s0 - d[k, c]
            if 0 <= t < nout:
                expect[k, t] += 1
    assert np.array_equal(out, expect)


def test_saturated_input_no_overflow():
    """All-255 input over 4096 channels: the SWAR lanes widen correctly."""
    nchan, nin = 4096, 3000
    p = _plan(nchan, 500.0, -0.048828125, 81.92e-6, np.linspace(0, 2, 16))
    x = torch.full((nin, nchan), 255, dtype=torch.uint8, device="cuda")
    out = p.dedisperse(x)
    assert (out == 255 * 4096).all().item()


def test_full_size_4096ch_sampled():
    """4096 ch x (262144 + 89989) samples x 1024 DMs, the launch the
    benchmark times: sampled outputs against the oracle one by one, and the
    DM = 0 trial equal to the channel sum over the whole block."""
    cfg = synth.config2()
    p = _plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
              widths=cfg.widths)
    D = p.max_delay
    nin = cfg.nsamp_out + D
    x = synth.noise_u8(nin, cfg.nchan, cfg.seed, device="cuda")
    synth.inject_pulses(x, cfg.pulses, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.seed)
    out = p.dedisperse(x)
    torch.cuda.synchronize()
    nout = cfg.nsamp_out
    chan_sum = x[:nout].to(torch.int32).sum(dim=1, dtype=torch.int32)
    assert torch.equal(out[0], chan_sum)
    xh = x.cpu().numpy()
    d = p.delays()
    rng = np.random.default_rng(7)
    ks = np.concatenate([[0, cfg.ndm - 1, 511, 512], rng.integers(0, cfg.ndm, 600)])
    ts = np.concatenate([[0, nout - 1, 2047, 2048], rng.integers(0, nout, 600)])
    for pl in cfg.pulses[:5]:
        k = int(np.argmin(np.abs(cfg.dm_list() - pl.dm)))
        ks = np.append(ks, [k, k])
        ts = np.append(ts, [int(pl.t0), int(pl.t0) + 1])
    outh = out.cpu().numpy()
    for k, t in zip(ks, ts):
        assert outh[k, t] == oracle.dedisperse_at(xh, d, int(k), int(t)), (k, t)


def test_injected_pulse_found_on_gpu(c1):
    cfg, x, _ = c1
    p = _plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
              widths=cfg.widths)
    series = p.dedisperse(x.cuda())
    p.single_pulse_search(series, cfg.threshold)
    cands, n = p.fetch()
    assert n > 0
    best = cands[np.argmax(cands["snr"])]
    assert best["dm_idx"] == 100 and cfg.widths[best["w_idx"]] == 4
    assert abs(int(best["t"]) - 8000) <= 1


def test_warp_specialised_tile_needs_even_stages():
    """Each of the two producer warps owns every other chunk and half the
    raw stages, so an odd stage count is refused."""
    p = _plan(256, 750.0, -200.0 / 256, 1.31072e-3, np.arange(64.0))
    with pytest.raises(DdspError) as e:
        p.set_tile(16, 8, 4, 3, 8)
    assert e.value.code == ddsp_lib.DDSP_E_INVALID_ARG
    p.set_tile(16, 8, 4, 2, 8)
    assert p.get_tile()["stages"] == 2


@pytest.mark.parametrize("nchan,nbits", [(256, 8), (100, 8), (48, 16)])
def test_stage_then_dedisperse_staged(nchan, nbits):
    """ddsp_stage + ddsp_dedisperse_staged give ddsp_dedisperse's output for
    the interleaved tile (fused single-pass staging for uint8 with nchan % 16
    == 0, unpack + interleave otherwise) and for the relayout tile; a tile
    change drops the staged block and a wrong nsamp_out is refused."""
    rng = np.random.default_rng(nchan)
    dt = np.uint8 if nbits == 8 else np.uint16
    hi = 256 if nbits == 8 else 65536
    dms = np.linspace(0, 30, 24)
    p = _plan(nchan, 500.0, -1.0, 1e-3, dms, nbits=nbits)
    x = rng.integers(0, hi, size=(4000, nchan)).astype(dt)
    ref = oracle.dedisperse(x, p.delays())
    xd = to_dev(x)
    for tile in [(16, 4, 6, 2, 16), (16, 4, 9, 2, 48),
                 (8, 4, 5, 4, 8 if nbits == 8 else 0)]:
        p.set_tile(*tile)
        with pytest.raises(DdspError) as e:
            p.dedisperse_staged(ref.shape[1])
        assert e.value.code == ddsp_lib.DDSP_E_STATE
        nout = p.stage(xd)
        assert nout == ref.shape[1]
        with pytest.raises(DdspError) as e:
            p.dedisperse_staged(nout - 1)
        assert e.value.code == ddsp_lib.DDSP_E_SHAPE
        out = p.dedisperse_staged(nout)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref), tile


def test_interleaved_cm_path_matches_oracle():
    """dedisperse_cm with the interleaved tile rebuilds the interleaved rows
    from caller-owned channel-major rows (zeros past the valid samples)."""
    cfg_nchan, nin = 128, 6000
    dms = np.linspace(0, 50, 40)
    p = _plan(cfg_nchan, 600.0, -1.5, 1e-3, dms)
    p.set_tile(16, 8, 7, 2, 16)
    x = np.random.default_rng(9).integers(0, 256, size=(nin, cfg_nchan)).astype(np.uint8)
    ref = oracle.dedisperse(x, p.delays())
    nout = ref.shape[1]
    # the plan's smallest pitch, and a wider caller pitch (the interleave
    # reads with the caller's pitch and writes the plan's rows)
    for pitch in (p.cm_pitch(nout), p.cm_pitch(nout) + 384):
        cm = p.unpack(to_dev(x), pitch)
        out = p.dedisperse_cm(cm, pitch, nout)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref), pitch


def test_wide_flag_needs_the_interleaved_tile():
    """DDSP_TILE_WIDE (16 consumer warps) exists only for the interleaved
    kernel: alone or with the relayout kernel it is refused; with it the
    time tile doubles for the same DM tile."""
    p = _plan(256, 750.0, -200.0 / 256, 1.31072e-3, np.arange(64.0))
    for flags in (32, 32 | 8, 32 | 1):
        with pytest.raises(DdspError) as e:
            p.set_tile(16, 8, 4, 2, flags)
        assert e.value.code == ddsp_lib.DDSP_E_INVALID_ARG
    p.set_tile(16, 8, 4, 2, 16)
    narrow = p.get_tile()["time_tile"]
    p.set_tile(16, 8, 4, 2, 48)
    t = p.get_tile()
    assert t["flags"] == 48 and t["time_tile"] == 2 * narrow
    p.set_tile(16, 4, 4, 2, 48)           # 4 trials x 8 elements per thread
    assert p.get_tile()["time_tile"] == 2 * narrow


def test_stage_refuses_a_block_shorter_than_the_delays():
    """N_out = N_in - D must be positive: ddsp_stage refuses the block with
    DDSP_E_SHAPE and leaves nothing staged."""
    dms = np.linspace(0, 30, 8)
    p = _plan(64, 500.0, -1.0, 1e-3, dms)
    x = np.zeros((p.max_delay + 100, 64), np.uint8)
    assert p.stage(to_dev(x)) == 100
    short = to_dev(np.zeros((p.max_delay, 64), np.uint8))
    with pytest.raises(DdspError) as e:
        p.stage(short)
    assert e.value.code == ddsp_lib.DDSP_E_SHAPE
    with pytest.raises(DdspError) as e:
        p.dedisperse_staged(100)
    assert e.value.code == ddsp_lib.DDSP_E_STATE


def test_full_size_4096ch_whole_series_and_candidates():
    """The single full-size beam (4096 ch x (262144 + 89989) samples x 1024
    DMs, widths 1..256, L 8192, threshold 7) through stage + dedisperse +
    search in the launch configuration the benchmark times, against the
    oracle's whole result stored by tests/golden/make_golden.py (the oracle
    takes minutes on it): every dedispersed row bit-exact (row digests of
    the oracle's series), and the complete candidate list identical under
    the tolerance rule.  A different best width is checked against the
    oracle's own series row, recomputed for that DM trial."""
    from parity import (GOLDEN, compare_to_stored, read_candidates,
                        read_digests, row_digests)
    cfg = synth.config2()
    p = Plan(cfg.nchan, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.dm_list(),
             cfg.widths, nbits=8, norm_window=cfg.norm_window,
             cand_capacity=1 << 20)
    D = p.max_delay
    nin = cfg.nsamp_out + D
    x = synth.noise_u8(nin, cfg.nchan, cfg.seed, device="cuda")
    synth.inject_pulses(x, cfg.pulses, cfg.f_top, cfg.chan_bw, cfg.tsamp, cfg.seed)
    nout = p.stage(x)
    out = p.dedisperse_staged(nout)
    p.single_pulse_search(out, cfg.threshold)
    got, n = p.fetch()
    p.check()
    stored = read_digests(os.path.join(GOLDEN, "c2_series_rows.txt"))
    mine = row_digests(out.cpu().numpy())
    bad = [k for k in range(cfg.ndm) if mine[k] != stored[str(k)]]
    assert not bad, f"{len(bad)} dedispersed rows differ, first {bad[:8]}"
    ref = read_candidates(os.path.join(GOLDEN, "c2_candidates.txt"))
    assert n == got.size > 0
    xh = x.cpu().numpy()
    d = p.delays()

    def width_check(k, t, wg, s_ref):
        row = oracle.dedisperse(xh, d[k:k + 1])[0]
        w = cfg.widths[wg]
        B = int(row[t:t + w].astype(np.int64).sum())
        m2, mad4 = oracle.window_stats(row, cfg.norm_window)
        j = min(t // cfg.norm_window, m2.size - 1)
        s = oracle.snr(B, w, m2[j], mad4[j])
        assert abs(s - s_ref) <= 1e-5 * abs(s_ref), ("width", k, t)

    compare_to_stored(got, ref, cfg.threshold, width_check)
