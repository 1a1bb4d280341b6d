"""Tile autotuning of a single-beam plan: ddsp_plan_autotune times the
candidate tiles on a block, keeps the fastest and records it in a JSON
cache; a plan created afterwards with DDSP_TILE_CACHE naming that file takes
the cached tile; every tile gives the oracle's dedispersion bit for bit."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import Plan, build, tile_cache_get

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _plan():
    return Plan(512, 500.0, -200.0 / 512, 81.92e-6, np.linspace(0, 60, 96),
                [1, 2, 4, 8], nbits=8, norm_window=8192, cand_capacity=1 << 16)


def test_autotune_cache_and_plan_creation(tmp_path, monkeypatch):
    cache = str(tmp_path / "tiles.json")
    p = _plan()
    nin = p.max_delay + 20000
    x = np.random.default_rng(3).integers(0, 256, size=(nin, 512)).astype(np.uint8)
    ref = oracle.dedisperse(x, p.delays())
    xd = torch.from_numpy(x).cuda()
    ms, best = p.autotune(xd, cache=cache, reps=2)
    assert best >= 0 and ms[best] > 0
    assert all(m < 0 or m >= ms[best] for m in ms)
    t = p.get_tile()
    stored = tile_cache_get(cache, p.tile_key())
    assert stored is not None
    assert stored[0] == (t["dm_tile"], t["dm_per_thread"], t["chan_chunk"],
                         t["stages"], t["flags"])
    assert np.array_equal(p.dedisperse(xd).cpu().numpy(), ref)
    # a new plan of the same shape picks the cached tile
    monkeypatch.setenv("DDSP_TILE_CACHE", cache)
    q = _plan()
    assert q.get_tile() == t
    assert np.array_equal(q.dedisperse(xd).cpu().numpy(), ref)
    monkeypatch.delenv("DDSP_TILE_CACHE")
    # a cache entry for another shape leaves the built-in choice alone
    other = Plan(256, 500.0, -200.0 / 256, 81.92e-6, np.linspace(0, 30, 40),
                 [1, 2], nbits=8, norm_window=8192, cand_capacity=1024)
    assert other.tile_key() != p.tile_key()
