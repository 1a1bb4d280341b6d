"""The bounds-checked build (libddsp_bounds.so, compiled with
-DDDSP_BOUNDS_CHECK): the index of every shared- and global-memory access of
the staging, interleave, dedispersion and search kernels is checked against
its buffer before the access, and the first violation is recorded in a
device word.  A child pytest runs the small-shape parity tests against that
library (DDSP_LIB) and reports the word at the end of its session
(DDSP_BOUNDS_REPORT, see conftest.py); the tests must pass and no check may
have failed.  This stands in for a memory checker, which this pool does not
offer."""
import os
import subprocess
import sys

import pytest

from paper_2605_03531_b300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SMALL = [
    "tests/test_gpu_dedisperse.py::test_unpack_byte_exact",
    "tests/test_gpu_dedisperse.py::test_c1_bit_exact_every_tile",
    "tests/test_gpu_dedisperse.py::test_ragged_shapes_bit_exact",
    "tests/test_gpu_dedisperse.py::test_impulses_land_at_their_delays",
    "tests/test_gpu_dedisperse.py::test_stage_then_dedisperse_staged",
    "tests/test_gpu_dedisperse.py::test_interleaved_cm_path_matches_oracle",
    "tests/test_gpu_sps.py::test_dense_matches_oracle",
    "tests/test_gpu_sps.py::test_candidates_match_oracle",
    "tests/test_gpu_sps.py::test_window_stats_across_spreads",
    "tests/test_gpu_sps.py::test_window_stats_misleading_estimate",
    "tests/test_gpu_sps.py::test_mad_zero_gives_no_candidates",
    "tests/test_gpu_server.py::test_server_blocks_equal_plain_path_in_any_mix",
    "tests/test_gpu_batch.py::test_batch_equals_plain_per_beam",
]


def test_small_parity_under_bounds_checks(tmp_path):
    lib = build.build_bounds()
    report = tmp_path / "bounds.txt"
    env = dict(os.environ, DDSP_LIB=lib, DDSP_BOUNDS_REPORT=str(report))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p",
                        "no:cacheprovider", "-m", "gpu", *SMALL],
                       cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    enabled, violation = report.read_text().split()
    assert enabled == "1", "the child did not load the checked build"
    assert int(violation) == 0, (
        f"bounds violation: site {int(violation) >> 32}, "
        f"index {int(violation) & 0xffffffff}")
