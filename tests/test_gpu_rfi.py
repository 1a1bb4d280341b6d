"""GPU parity of the gptool-style RFI mitigation (Sec.2.1) with the CPU
oracle: integer arithmetic throughout, so the cleaned block, both flag sets
and the fill level are identical."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import DdspError, Rfi, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _block(nt, nc, seed, rfi_c=(), rfi_t=(), gain=True):
    x = synth.noise_u8_np(nt, nc, seed).astype(np.int64)
    if gain:                    # a gentle bandpass slope across the band
        g = np.linspace(0.8, 1.2, nc)
        x = np.round(x * g[None, :])
    x[:, list(rfi_c)] += 60
    x[list(rfi_t), :] += 40
    return np.clip(x, 0, 255).astype(np.uint8)


def check(x, **kw):
    nt, nc = x.shape
    r = Rfi(nt, nc)
    out = r.clean(torch.from_numpy(x).cuda(), **kw).cpu().numpy()
    fc, ft, fill = r.flags()
    r.close()
    ref, rfc, rft = oracle.rfi_clean(x, kw.get("half_window", 10),
                                     kw.get("kc", 4), kw.get("kt", 3),
                                     kw.get("rounds", 2))
    assert np.array_equal(fc, rfc) and np.array_equal(ft, rft)
    assert np.array_equal(out, ref)
    return out, fc, ft, fill


@pytest.mark.parametrize("nt,nc,seed,rfi_c,rfi_t", [
    (4096, 256, 3, (17, 40, 41, 200), (100, 2000, 3001)),
    (16384, 4096, 4, (5, 1000, 1001, 4095), (0, 777, 16383)),   # the c5 block
    (1000, 37, 5, (), ()),
    (333, 1, 6, (), (7,)),                                     # one channel
])
def test_clean_matches_oracle(nt, nc, seed, rfi_c, rfi_t):
    x = _block(nt, nc, seed, rfi_c, rfi_t)
    out, fc, ft, fill = check(x)
    if nc > 1:
        assert set(rfi_c) <= set(np.nonzero(fc)[0])
    assert set(rfi_t) <= set(np.nonzero(ft)[0]) or nc == 1


@pytest.mark.parametrize("kw", [dict(half_window=0), dict(half_window=32),
                                dict(rounds=1), dict(rounds=3, kc=3, kt=2),
                                dict(kc=0, kt=0)])
def test_parameters_match_oracle(kw):
    check(_block(2048, 300, 8, (10, 150), (5, 1500)), **kw)


def test_unaligned_rows_match_oracle():
    """A view starting one byte into its buffer (no 32-bit accesses)."""
    x = _block(700, 128, 9, (3, 90), (11,))
    buf = torch.zeros(x.size + 1, dtype=torch.uint8, device="cuda")
    view = buf[1:].view(700, 128)
    view.copy_(torch.from_numpy(x))
    r = Rfi(700, 128)
    out = r.clean(view).cpu().numpy()
    fc, ft, fill = r.flags()
    ref, rfc, rft = oracle.rfi_clean(x)
    assert np.array_equal(out, ref) and np.array_equal(fc, rfc)
    r.close()


def test_in_place_and_constant_block():
    x = np.full((500, 64), 77, np.uint8)
    r = Rfi(500, 64)
    xd = torch.from_numpy(x).cuda()
    r.clean(xd, out=xd)
    fc, ft, fill = r.flags()
    assert (xd.cpu().numpy() == 77).all() and not fc.any() and not ft.any()
    assert fill == 77
    r.close()


def test_arguments():
    with pytest.raises(DdspError):
        Rfi(1 << 23, 64)
    with pytest.raises(DdspError):
        Rfi(100, 9000)
    r = Rfi(100, 64)
    x = torch.zeros((200, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(DdspError):
        r.clean(x)                                    # more samples than room
    y = torch.zeros((100, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(DdspError):
        r.clean(y, half_window=33)
    with pytest.raises(DdspError):
        r.clean(y, rounds=0)
    with pytest.raises(DdspError):
        r.flags()                                     # no clean yet
    r.close()
