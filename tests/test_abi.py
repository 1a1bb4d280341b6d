"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/ddsp.h declares, computes the same delay table as the
oracle (independently written code, same definition: Ch.1 Eq.1), and
rejects bad arguments before touching the device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_2605_03531_b300 import _lib, build, delay_table, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ddsp.h")


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ddsp_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(\S+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(L, n)
    # the binding declares exactly the header's functions
    assert sorted(_lib.SIGNATURES) == names


def test_bounds_build_exports_the_same_symbols(L):
    """The bounds-checked build (tests only) has the same ABI; only it
    reports itself as checked."""
    lib = build.build_bounds()
    out = subprocess.run(["nm", "-D", "--defined-only", lib],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(\S+)", out))
    assert not [n for n in declared_functions() if n not in exported]
    en, v = C.c_int(), C.c_uint64()
    assert L.ddsp_bounds_check_status(C.byref(en), C.byref(v)) == 0
    assert en.value == 0 and v.value == 0


def test_error_strings(L):
    for code in range(0, -9, -1):
        s = L.ddsp_error_string(code).decode()
        assert s and s != "unknown error"
    assert L.ddsp_error_string(-100).decode() == "unknown error"


CASES = [
    (256, 750.0, -0.78125, 1.31072e-3, np.arange(256, dtype=np.float64)),
    (4096, 500.0, -0.048828125, 81.92e-6, np.linspace(0.0, 250.0, 1024)),
    (1024, 300.0, 0.1953125, 81.92e-6, np.linspace(0.0, 500.0, 37)),
    (37, 1460.0, -10.0, 1e-4, np.array([2000.0, 0.0, 3.3, 999.9])),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_delay_table_parity_with_oracle(L, case):
    nchan, f_top, bw, ts, dms = CASES[case]
    d, D = delay_table(nchan, f_top, bw, ts, dms)
    d_ref, D_ref = oracle.delay_table(nchan, f_top, bw, ts, dms)
    assert D == D_ref
    assert np.array_equal(d, d_ref)


def test_delay_table_reports_near_ties(L):
    """Entries within 1e-9 of a .5 tie would depend on evaluation order; list
    them (none are expected for the standard grids)."""
    nchan, f_top, bw, ts, dms = CASES[0]
    near = []
    for dm in dms[::17]:
        for c in range(0, nchan, 5):
            x = oracle.delay_exact(nchan, f_top, bw, ts, dm, c)
            if abs(x - np.floor(x) - 0.5) < 1e-9:
                near.append((dm, c, x))
    assert near == []


def _create(L, **kw):
    args = dict(nchan=64, f_top=500.0, bw=-1.0, ts=1e-3, dms=[0.0, 10.0],
                widths=[1, 2, 4], nbits=8, win=1024, cap=100)
    args.update(kw)
    h = C.c_void_p()
    dms = np.ascontiguousarray(args["dms"], dtype=np.float64)
    ws = np.ascontiguousarray(args["widths"], dtype=np.int32)
    rc = L.ddsp_plan_create(C.byref(h), args["nchan"], args["f_top"], args["bw"],
                            args["ts"], dms.ctypes.data_as(C.c_void_p), dms.size,
                            ws.ctypes.data_as(C.c_void_p), ws.size, args["nbits"],
                            args["win"], args["cap"])
    return rc, h


@pytest.mark.parametrize("bad", [
    dict(nchan=0), dict(bw=0.0), dict(ts=0.0), dict(ts=-1.0), dict(f_top=-5.0),
    dict(dms=[-1.0]), dict(dms=[float("nan")]), dict(dms=[float("inf")]),
    dict(widths=[3]), dict(widths=[2, 1]), dict(widths=[2048]), dict(widths=[0]),
    dict(nbits=12), dict(cap=0), dict(win=-1),
    dict(nchan=600, f_top=300.0, bw=-1.0),     # band crosses zero frequency
])
def test_plan_create_rejects_bad_arguments(L, bad):
    rc, h = _create(L, **bad)
    assert rc == _lib.DDSP_E_INVALID_ARG
    assert not h.value


def test_null_handles(L):
    n = C.c_int64()
    assert L.ddsp_plan_nsamp_out(None, 100, C.byref(n)) == _lib.DDSP_E_INVALID_ARG
    assert L.ddsp_dedisperse(None, None, 10, None, None) == _lib.DDSP_E_INVALID_ARG
    sz = C.c_size_t()
    assert L.ddsp_candidates_fetch(None, None, 0, C.byref(sz)) == _lib.DDSP_E_INVALID_ARG
    L.ddsp_plan_destroy(None)


def test_product_path_has_no_oracle_dependency():
    """The package and the CUDA sources never import or link the oracle."""
    pkg = os.path.join(ROOT, "paper_2605_03531_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt and "orc_" not in txt, f


def test_generator_numpy_torch_agree():
    a = synth.noise_u8(513, 48, 9).numpy()
    b = synth.noise_u8_np(513, 48, 9)
    assert np.array_equal(a, b)
    assert abs(a.mean() - 128) < 0.5 and abs(a.std() - 16) < 0.5


def test_every_source_file_is_a_build_dependency():
    """A change to any file under csrc/ (kernels, headers, device headers)
    must rebuild the library."""
    import glob
    import os
    from paper_2605_03531_b300 import build as b
    files = {os.path.abspath(f) for f in glob.glob(os.path.join(b.CSRC, "*"))
             if os.path.isfile(f)}
    deps = {os.path.abspath(d) for d in b._deps()}
    assert files and files <= deps, sorted(files - deps)
