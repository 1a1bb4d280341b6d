import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for _p in (ROOT, HERE):
    if _p not in sys.path:
        sys.path.insert(0, _p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _has_gpu():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_sessionfinish(session, exitstatus):
    """With DDSP_BOUNDS_REPORT set (a run against the bounds-checked build,
    see test_gpu_bounds.py): write '<enabled> <first violation>' there and
    fail the session if a check failed."""
    path = os.environ.get("DDSP_BOUNDS_REPORT")
    if not path:
        return
    import ctypes as C
    from paper_2605_03531_b300 import _lib
    en, v = C.c_int(), C.c_uint64()
    rc = _lib.lib().ddsp_bounds_check_status(C.byref(en), C.byref(v))
    with open(path, "w") as f:
        f.write(f"{en.value} {v.value}\n")
    if rc != 0 or v.value:
        session.exitstatus = 1
