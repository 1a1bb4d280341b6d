"""GPU parity of the resampling for frequency derivatives (Sec.3.4) with the
CPU oracle.

The oracle accumulates the bin edges bin by bin in FP64; the GPU takes
every 32nd edge from the closed form in FP64 (within K t_K 2^-53 of the
oracle's) and places the 31 after it by an FP32 prefix sum of the width
deviations, with every FP32 value near 1 (below 2^-20 samples more), so an output differs by at most twice the edge error times
max|x|, plus the FP32 rounding of a sum of up to three products (a few
2^-24 of |out|).  The bin count is the same for these (generic)
parameters.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_03531_b300 import DdspError, Plan, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _plan():
    return Plan(16, 500.0, -1.0, 1e-3, np.zeros(4), [1, 2], nbits=8,
                norm_window=8192, cand_capacity=1024)


@pytest.mark.parametrize("n,f0,f1,f2", [
    (5000, 7.0, 0.0, 0.0),           # identity
    (20000, 25.0, -0.01, 0.0),
    (20000, 25.0, 0.01, 0.0),        # reversed
    (50000, 3.0, -0.002, -1e-6),
    (50000, 3.0, 0.002, 1e-6),
    (777, 100.0, -1.0, 0.5),         # short, strong drift
])
def test_resample_matches_oracle(n, f0, f1, f2):
    ts = 1e-3
    rng = np.random.default_rng(n)
    x = rng.integers(-10000, 10000, size=(3, n)).astype(np.int32)
    pl = _plan()
    y = pl.resample(torch.from_numpy(x).cuda(), ts, f0, f1, f2).cpu().numpy()
    K = y.shape[1]
    assert K == Plan.resample_length(n, ts, f0, f1, f2)
    for r in range(3):
        ref = oracle.resample(x[r], f0, f1, f2, ts)
        assert ref.size == K
        edge = K * K * 2.0 ** -53 + 2.0 ** -20
        tol = 2 * edge * np.abs(x[r]).max() + 4 * 2.0 ** -24 * np.abs(ref)
        assert (np.abs(y[r] - ref) <= tol + 1e-6).all(), r
    if f1 == 0 and f2 == 0:
        assert np.array_equal(y, x.astype(np.float32))


def test_resample_invalid_laws():
    pl = _plan()
    x = torch.ones((1, 1000), dtype=torch.int32, device="cuda")
    with pytest.raises(DdspError):
        pl.resample(x, 1e-3, 0.0, 0.0, 0.0)          # f0 <= 0
    # f2 > 0 with f1 <= 0: widths 1 - 0.005 k^2 reach 0 near k = 14
    with pytest.raises(DdspError):
        pl.resample(x, 1e-3, 1.0, 0.0, 1e4)
    with pytest.raises(DdspError):
        Plan.resample_length(1000, 1e-3, 1.0, 0.0, 1e4)
    with pytest.raises(ValueError):
        oracle.resample(np.ones(1000, np.int32), 1.0, 0.0, 1e4, 1e-3)
    with pytest.raises(DdspError):
        pl.resample(x, 0.0, 1.0, 0.0, 0.0)           # tsamp <= 0
