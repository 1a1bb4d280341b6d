"""ctypes declarations of the C ABI in include/ddsp.h (libddsp.so).

There is no fallback: if the compiled library is missing, ``lib()`` raises.
Build it with ``python -m paper_2605_03531_b300.build``.
"""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# DDSP_LIB selects another build of the same ABI (the tests' bounds-checked
# libddsp_bounds.so); the default is the in-tree libddsp.so
LIB_PATH = os.environ.get("DDSP_LIB") or os.path.join(_HERE, "libddsp.so")

DDSP_OK = 0
DDSP_E_INVALID_ARG = -1
DDSP_E_SHAPE = -2
DDSP_E_CUDA = -3
DDSP_E_NOMEM = -4
DDSP_E_TIMEOUT = -5
DDSP_E_TRUNCATED = -6
DDSP_E_RANGE = -7
DDSP_E_STATE = -8


class DdspCand(C.Structure):
    _fields_ = [("dm_idx", C.c_uint32), ("t", C.c_uint32),
                ("w_idx", C.c_uint32), ("snr", C.c_float)]


class DdspUnitPeaks(C.Structure):
    _fields_ = [("sms", C.c_int), ("blocks_per_sm", C.c_int * 4),
                ("smem_bytes_per_clk", C.c_double),
                ("iadd3_per_clk", C.c_double), ("prmt_per_clk", C.c_double),
                ("swar_adds_per_clk", C.c_double)]


P = C.c_void_p
I64 = C.c_int64
I32 = C.c_int
PI64 = C.POINTER(C.c_int64)

# name -> (restype, argtypes); the same list the header declares
SIGNATURES = {
    "ddsp_plan_create": (I32, [C.POINTER(P), I32, C.c_double, C.c_double,
                               C.c_double, P, I32, P, I32, I32, I64, C.c_size_t]),
    "ddsp_delay_table": (I32, [I32, C.c_double, C.c_double, C.c_double, P,
                               I32, P, C.POINTER(C.c_int32)]),
    "ddsp_plan_nsamp_out": (I32, [P, I64, PI64]),
    "ddsp_plan_max_delay": (I32, [P, C.POINTER(C.c_int32)]),
    "ddsp_plan_get_delays": (I32, [P, P]),
    "ddsp_unpack": (I32, [P, P, I64, P, I64, P]),
    "ddsp_dedisperse": (I32, [P, P, I64, P, P]),
    "ddsp_dedisperse_cm": (I32, [P, P, I64, I64, P, P]),
    "ddsp_stage": (I32, [P, P, I64, P]),
    "ddsp_dedisperse_staged": (I32, [P, I64, P, P]),
    "ddsp_plan_cm_pitch": (I32, [P, I64, PI64]),
    "ddsp_single_pulse_search": (I32, [P, P, I64, C.c_float, P]),
    "ddsp_single_pulse_search_dense": (I32, [P, P, I64, P, P, P, P]),
    "ddsp_single_pulse_search_noalloc": (I32, [P, I32, I64, P, I32, I64,
                                               C.c_float, P, C.c_uint32, P, P]),
    "ddsp_single_pulse_search_noalloc_check": (I32, [P]),
    "ddsp_plan_get_stats": (I32, [P, P, P, I64, PI64]),
    "ddsp_candidates_fetch": (I32, [P, P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "ddsp_candidates_count": (I32, [P, C.POINTER(C.c_size_t)]),
    "ddsp_candidates_fetch_dm_range": (I32, [P, C.c_uint32, C.c_uint32, P,
                                             C.c_size_t, C.POINTER(C.c_size_t),
                                             C.POINTER(C.c_size_t)]),
    "ddsp_plan_check": (I32, [P, P]),
    "ddsp_batch_create": (I32, [C.POINTER(P), P, I32, P, P]),
    "ddsp_batch_destroy": (None, [P]),
    "ddsp_batch_input": (I32, [P, I32, C.POINTER(P), PI64, PI64]),
    "ddsp_batch_ingest": (I32, [P, I32, P, P]),
    "ddsp_batch_series": (I32, [P, I32, C.POINTER(P), PI64]),
    "ddsp_batch_run": (I32, [P, C.c_float, I32, P]),
    "ddsp_batch_check": (I32, [P, P]),
    "ddsp_batch_set_tile": (I32, [P, I32, I32, I32, I32]),
    "ddsp_batch_get_tile": (I32, [P] + [C.POINTER(C.c_int)] * 6),
    "ddsp_batch_get_beam_chunk": (I32, [P, I32, C.POINTER(C.c_int)]),
    "ddsp_batch_get_beam_tile": (I32, [P, I32] + [C.POINTER(C.c_int)] * 5),
    "ddsp_batch_autotune": (I32, [P, I32, P, C.POINTER(C.c_float), I32,
                                  C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ddsp_server_create": (I32, [C.POINTER(P), P, I64, I32, I64, I32, I32,
                                 I32, I32]),
    "ddsp_server_destroy": (None, [P]),
    "ddsp_server_info": (I32, [P] + [PI64] * 5),
    "ddsp_server_get_tile": (I32, [P] + [C.POINTER(C.c_int)] * 6),
    "ddsp_server_admit": (I32, [P, C.POINTER(C.c_int)]),
    "ddsp_server_evict": (I32, [P, I32]),
    "ddsp_server_push": (I32, [P, I32, P, P]),
    "ddsp_server_step": (I32, [P, C.c_float, I32, P, PI64, C.POINTER(C.c_int),
                               I32, C.POINTER(C.c_int)]),
    "ddsp_server_query": (I32, [P, I64]),
    "ddsp_server_fetch": (I32, [P, I32, I64, P, C.c_size_t,
                                C.POINTER(C.c_size_t), PI64]),
    "ddsp_server_series": (I32, [P, I32, C.POINTER(P), PI64]),
    "ddsp_server_check": (I32, [P, P]),
    "ddsp_plan_destroy": (None, [P]),
    "ddsp_error_string": (C.c_char_p, [I32]),
    "ddsp_last_error_detail": (C.c_char_p, []),
    "ddsp_plan_set_tile": (I32, [P, I32, I32, I32, I32, I32]),
    "ddsp_plan_get_tile": (I32, [P] + [C.POINTER(C.c_int)] * 6),
    "ddsp_plan_set_wait_limit": (I32, [P, I64]),
    "ddsp_plan_autotune": (I32, [P, P, I64, C.c_char_p, I32, P,
                                 C.POINTER(C.c_float), I32, C.POINTER(C.c_int)]),
    "ddsp_plan_tile_key": (I32, [P, C.c_char_p, C.c_size_t]),
    "ddsp_tile_cache_get": (I32, [C.c_char_p, C.c_char_p, C.POINTER(C.c_int),
                                  C.POINTER(C.c_float)]),
    "ddsp_tile_cache_put": (I32, [C.c_char_p, C.c_char_p, C.POINTER(C.c_int),
                                  C.c_float]),
    "ddsp_bounds_check_status": (I32, [C.POINTER(C.c_int),
                                       C.POINTER(C.c_uint64)]),
    "ddsp_plan_withhold_copy": (I32, [P, I32]),
    "ddsp_cluster_create": (I32, [C.POINTER(P), I32, I32, I64, I64]),
    "ddsp_cluster_destroy": (None, [P]),
    "ddsp_peaks_cluster": (I32, [P, P, P, I64, P, I32, I32, I32, I32, P]),
    "ddsp_cluster_fetch_peaks": (I32, [P, P, P, C.c_size_t,
                                       C.POINTER(C.c_size_t)]),
    "ddsp_cluster_fetch_reps": (I32, [P, P, P, C.c_size_t,
                                      C.POINTER(C.c_size_t)]),
    "ddsp_plan_candidates_device": (I32, [P, C.POINTER(P), C.POINTER(P),
                                          C.POINTER(C.c_size_t)]),
    "ddsp_downsample": (I32, [P, P, I64, I64, I64, I64, P, I64, P]),
    "ddsp_dered": (I32, [P, P, I64, I64, I64, I64, P, I64, P]),
    "ddsp_ffa": (I32, [P, P, I64, I64, I64, I32, P, C.POINTER(C.c_int), P]),
    "ddsp_ffa_search": (I32, [P, P, I64, I64, I64, I32, I32, P, I32, P, P, P,
                              P, I64, P]),
    "ddsp_resample_length": (I32, [I64, C.c_double, C.c_double, C.c_double,
                                   C.c_double, PI64]),
    "ddsp_resample": (I32, [P, P, I64, I64, I64, C.c_double, C.c_double,
                            C.c_double, C.c_double, P, I64, PI64, P]),
    "ddsp_rfi_create": (I32, [C.POINTER(P), I32, I64, I32]),
    "ddsp_rfi_destroy": (None, [P]),
    "ddsp_rfi_clean": (I32, [P, P, I64, I32, I32, I32, I32, I32, P, P]),
    "ddsp_rfi_flags": (I32, [P, P, P, PI64]),
    "ddsp_probe_unit_peaks": (I32, [I32, C.POINTER(DdspUnitPeaks)]),
    "ddsp_batch_set_mode": (I32, [P, I32]),
    "ddsp_batch_get_mode": (I32, [P, C.POINTER(C.c_int)]),
    "ddsp_server_set_mode": (I32, [P, I32, I32]),
    "ddsp_server_get_mode": (I32, [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
}

_lib = None


def lib():
    """The loaded libddsp.so with every exported signature declared."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -m paper_2605_03531_b300.build` (there is no CPU "
                "fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class DdspError(RuntimeError):
    def __init__(self, code, call):
        self.code = code
        msg = lib().ddsp_error_string(code).decode()
        detail = lib().ddsp_last_error_detail().decode() if code == DDSP_E_CUDA else ""
        super().__init__(f"{call} failed: {msg} ({code})"
                         + (f" [{detail}]" if detail else ""))


def check(code, call):
    if code != DDSP_OK:
        raise DdspError(code, call)
    return code
