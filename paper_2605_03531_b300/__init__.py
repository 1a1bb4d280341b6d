"""B300-native brute-force dedispersion and boxcar single-pulse search.

Python side of the C ABI in ``include/ddsp.h``: argument marshalling only.
Every step of the path (unpack, dedispersion, window statistics, boxcar S/N,
candidate compaction) runs in the CUDA kernels of ``libddsp.so``; PyTorch
provides device memory and streams.  Importing this package does not load
the library; the first ``Plan`` does, and fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import DdspError, DdspCand


__all__ = ["Plan", "Batch", "Server", "Cluster", "Rfi", "DdspError",
           "CAND_DTYPE", "delay_table", "probe_unit_peaks", "tile_cache_get",
           "tile_cache_put"]

CAND_DTYPE = np.dtype([("dm_idx", np.uint32), ("t", np.uint32),
                       ("w_idx", np.uint32), ("snr", np.float32)])


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class _DeviceArray:
    """A library-owned device buffer exposed through the CUDA array
    interface, so torch can view it without a copy."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {
            "data": (int(ptr), False), "shape": tuple(int(d) for d in shape),
            "typestr": typestr, "strides": None, "version": 3}


def _torch_int32():
    import torch
    return torch.int32


def _tensor_view(ptr, shape, dtype):
    import torch
    typestr = {torch.int32: "<i4", torch.uint8: "|u1"}[dtype]
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")


def _dev_ptr(t, dtype=None, what="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def tile_cache_get(path, key):
    """(tile tuple, ms) cached under `key` in the JSON file `path`, or None
    (ddsp_tile_cache_get; host only)."""
    t = (C.c_int * 5)()
    ms = C.c_float()
    rc = _lib.lib().ddsp_tile_cache_get(str(path).encode(), key.encode(), t,
                                        C.byref(ms))
    if rc == _lib.DDSP_E_STATE:
        return None
    _lib.check(rc, "ddsp_tile_cache_get")
    return tuple(t), ms.value


def tile_cache_put(path, key, tile, ms):
    """Record `tile` (dm_tile, dm_per_thread, chan_chunk, stages, flags)
    under `key` in the JSON file `path` (ddsp_tile_cache_put; host only)."""
    t = (C.c_int * 5)(*[int(v) for v in tile])
    _lib.check(_lib.lib().ddsp_tile_cache_put(str(path).encode(), key.encode(),
                                              t, float(ms)),
               "ddsp_tile_cache_put")


def delay_table(nchan, f_top, chan_bw, tsamp, dm_list):
    """(d[k][c] int32, D) from the library's host-side delay code."""
    dms = np.ascontiguousarray(dm_list, dtype=np.float64)
    d = np.empty((dms.size, int(nchan)), dtype=np.int32)
    D = C.c_int32()
    _lib.check(_lib.lib().ddsp_delay_table(
        int(nchan), float(f_top), float(chan_bw), float(tsamp),
        dms.ctypes.data_as(C.c_void_p), int(dms.size),
        d.ctypes.data_as(C.c_void_p), C.byref(D)), "ddsp_delay_table")
    return d, D.value


class Plan:
    """A dedispersion + single-pulse-search plan (``ddsp_plan_create``)."""

    def __init__(self, nchan, f_top, chan_bw, tsamp, dm_list, widths,
                 nbits=8, norm_window=8192, cand_capacity=1 << 20):
        self._h = C.c_void_p()
        L = _lib.lib()
        dms = np.ascontiguousarray(dm_list, dtype=np.float64)
        ws = np.ascontiguousarray(widths, dtype=np.int32)
        _lib.check(L.ddsp_plan_create(
            C.byref(self._h), int(nchan), float(f_top), float(chan_bw),
            float(tsamp), dms.ctypes.data_as(C.c_void_p), int(dms.size),
            ws.ctypes.data_as(C.c_void_p), int(ws.size), int(nbits),
            int(norm_window), int(cand_capacity)), "ddsp_plan_create")
        self.nchan, self.ndm, self.nbits = int(nchan), int(dms.size), int(nbits)
        self.widths = [int(w) for w in ws]
        self.norm_window = int(norm_window)
        self.cand_capacity = int(cand_capacity)

    # ---------------------------------------------------------------- info
    @property
    def max_delay(self) -> int:
        D = C.c_int32()
        _lib.check(_lib.lib().ddsp_plan_max_delay(self._h, C.byref(D)),
                   "ddsp_plan_max_delay")
        return D.value

    def nsamp_out(self, nsamp_in) -> int:
        n = C.c_int64()
        _lib.check(_lib.lib().ddsp_plan_nsamp_out(self._h, int(nsamp_in),
                                                  C.byref(n)),
                   "ddsp_plan_nsamp_out")
        return n.value

    def delays(self) -> np.ndarray:
        d = np.empty((self.ndm, self.nchan), dtype=np.int32)
        _lib.check(_lib.lib().ddsp_plan_get_delays(
            self._h, d.ctypes.data_as(C.c_void_p)), "ddsp_plan_get_delays")
        return d

    def set_tile(self, dm_tile=0, dm_per_thread=4, chan_chunk=8, stages=2,
                 flags=0):
        """Pick the dedispersion tile shape (0: library's choice, -1: the
        direct kernel); see ddsp_plan_set_tile."""
        _lib.check(_lib.lib().ddsp_plan_set_tile(
            self._h, int(dm_tile), int(dm_per_thread), int(chan_chunk),
            int(stages), int(flags)), "ddsp_plan_set_tile")

    def get_tile(self):
        """dict(dm_tile, dm_per_thread, time_tile, chan_chunk, stages, flags)."""
        v = [C.c_int() for _ in range(6)]
        _lib.check(_lib.lib().ddsp_plan_get_tile(self._h, *[C.byref(a) for a in v]),
                   "ddsp_plan_get_tile")
        keys = ("dm_tile", "dm_per_thread", "time_tile", "chan_chunk", "stages",
                "flags")
        return dict(zip(keys, (a.value for a in v)))

    # ---------------------------------------------------------------- path
    def _in_dtype(self):
        import torch
        return torch.uint8 if self.nbits == 8 else torch.uint16

    def unpack(self, x, pitch, out=None, stream=None):
        import torch
        nin = x.shape[0]
        if out is None:
            out = torch.empty((self.nchan, pitch), dtype=x.dtype, device=x.device)
        _lib.check(_lib.lib().ddsp_unpack(
            self._h, _dev_ptr(x, self._in_dtype(), "spectra"), int(nin),
            _dev_ptr(out, self._in_dtype(), "out"), int(pitch),
            _stream_handle(stream)), "ddsp_unpack")
        return out

    def dedisperse(self, x, out=None, stream=None):
        """x: CUDA tensor [nsamp_in][nchan] (uint8/uint16) -> int32
        [ndm][nsamp_out]."""
        import torch
        if x.dim() != 2 or x.shape[1] != self.nchan:
            raise ValueError("spectra must be [nsamp_in][nchan]")
        nin = x.shape[0]
        nout = self.nsamp_out(nin)
        if out is None:
            out = torch.empty((self.ndm, nout), dtype=torch.int32, device=x.device)
        elif tuple(out.shape) != (self.ndm, nout):
            raise ValueError("out must be [ndm][nsamp_out]")
        _lib.check(_lib.lib().ddsp_dedisperse(
            self._h, _dev_ptr(x, self._in_dtype(), "spectra"), int(nin),
            _dev_ptr(out, torch.int32, "out"), _stream_handle(stream)),
            "ddsp_dedisperse")
        return out

    def stage(self, x, stream=None) -> int:
        """Stage the time-major block x (CUDA [nsamp_in][nchan]) into the
        plan's rows for the current tile; returns nsamp_out."""
        if x.dim() != 2 or x.shape[1] != self.nchan:
            raise ValueError("spectra must be [nsamp_in][nchan]")
        nin = x.shape[0]
        _lib.check(_lib.lib().ddsp_stage(
            self._h, _dev_ptr(x, self._in_dtype(), "spectra"), int(nin),
            _stream_handle(stream)), "ddsp_stage")
        return self.nsamp_out(nin)

    def dedisperse_staged(self, nsamp_out, out=None, device=None, stream=None):
        """Dedisperse the block staged by stage() into int32
        [ndm][nsamp_out]."""
        import torch
        if out is None:
            out = torch.empty((self.ndm, int(nsamp_out)), dtype=torch.int32,
                              device=device or "cuda")
        elif tuple(out.shape) != (self.ndm, int(nsamp_out)):
            raise ValueError("out must be [ndm][nsamp_out]")
        _lib.check(_lib.lib().ddsp_dedisperse_staged(
            self._h, int(nsamp_out), _dev_ptr(out, torch.int32, "out"),
            _stream_handle(stream)), "ddsp_dedisperse_staged")
        return out

    def cm_pitch(self, nsamp_out) -> int:
        v = C.c_int64()
        _lib.check(_lib.lib().ddsp_plan_cm_pitch(self._h, int(nsamp_out),
                                                 C.byref(v)),
                   "ddsp_plan_cm_pitch")
        return v.value

    def dedisperse_cm(self, cm, pitch, nsamp_out, out=None, stream=None):
        """Dedisperse channel-major rows cm[nchan][pitch] already on the GPU."""
        import torch
        if out is None:
            out = torch.empty((self.ndm, nsamp_out), dtype=torch.int32,
                              device=cm.device)
        _lib.check(_lib.lib().ddsp_dedisperse_cm(
            self._h, _dev_ptr(cm, self._in_dtype(), "cm"), int(pitch),
            int(nsamp_out), _dev_ptr(out, torch.int32, "out"),
            _stream_handle(stream)), "ddsp_dedisperse_cm")
        return out

    def single_pulse_search(self, series, threshold, stream=None):
        import torch
        if series.dim() != 2 or series.shape[0] != self.ndm:
            raise ValueError("series must be [ndm][nsamp_out]")
        _lib.check(_lib.lib().ddsp_single_pulse_search(
            self._h, _dev_ptr(series, torch.int32, "series"),
            int(series.shape[1]), float(threshold), _stream_handle(stream)),
            "ddsp_single_pulse_search")

    def search_dense(self, series, stream=None):
        """Per-sample best width index, FP32 S/N and boxcar sum."""
        import torch
        n = series.shape[1]
        bw = torch.empty((self.ndm, n), dtype=torch.int32, device=series.device)
        bs = torch.empty((self.ndm, n), dtype=torch.float32, device=series.device)
        bsum = torch.empty((self.ndm, n), dtype=torch.int32, device=series.device)
        _lib.check(_lib.lib().ddsp_single_pulse_search_dense(
            self._h, _dev_ptr(series, torch.int32, "series"), int(n),
            _dev_ptr(bw), _dev_ptr(bs), _dev_ptr(bsum), _stream_handle(stream)),
            "ddsp_single_pulse_search_dense")
        return bw, bs, bsum

    def fetch(self, cap=None, allow_truncated=False):
        """(candidates sorted by (dm_idx, t), true count)."""
        if cap is None:
            cap = self.cand_capacity
        buf = np.zeros(cap, dtype=CAND_DTYPE)
        n = C.c_size_t()
        rc = _lib.lib().ddsp_candidates_fetch(
            self._h, buf.ctypes.data_as(C.c_void_p), int(cap), C.byref(n))
        if rc == _lib.DDSP_E_TRUNCATED and allow_truncated:
            return buf[:min(cap, self.cand_capacity)], n.value
        _lib.check(rc, "ddsp_candidates_fetch")
        return buf[:n.value].copy(), n.value

    def count(self):
        """Number of candidates the last search found (no records copied)."""
        n = C.c_size_t()
        _lib.check(_lib.lib().ddsp_candidates_count(self._h, C.byref(n)),
                   "ddsp_candidates_count")
        return n.value

    def candidates_device(self):
        """(int32 CUDA view [stored][4] of the last search's records, true
        count): the plan-owned device buffer as ddsp_plan_candidates_device
        gives it, unsorted; valid until the next search on this plan."""
        d_c, d_n, cap = C.c_void_p(), C.c_void_p(), C.c_size_t()
        _lib.check(_lib.lib().ddsp_plan_candidates_device(
            self._h, C.byref(d_c), C.byref(d_n), C.byref(cap)),
            "ddsp_plan_candidates_device")
        n = self.count()
        stored = min(n, cap.value)
        if stored == 0:
            import torch
            return torch.zeros((0, 4), dtype=torch.int32, device="cuda"), n
        return _tensor_view(d_c.value, (stored, 4), _torch_int32()), n

    def fetch_dm_range(self, dm_lo, dm_hi, cap=1 << 22):
        """(candidates with dm_lo <= dm_idx < dm_hi sorted, count in range,
        device count)."""
        buf = np.zeros(cap, dtype=CAND_DTYPE)
        nr, nt = C.c_size_t(), C.c_size_t()
        _lib.check(_lib.lib().ddsp_candidates_fetch_dm_range(
            self._h, int(dm_lo), int(dm_hi), buf.ctypes.data_as(C.c_void_p),
            int(cap), C.byref(nr), C.byref(nt)), "ddsp_candidates_fetch_dm_range")
        return buf[:nr.value].copy(), nr.value, nt.value

    def downsample(self, series, factor, out=None, stream=None):
        """int32 [rows][n] CUDA tensor -> [rows][n // factor], sums of
        ``factor`` consecutive samples (Sec.3.2)."""
        import torch
        rows, n = series.shape
        m = n // int(factor) if int(factor) >= 1 else 0
        if out is None:
            out = torch.empty((rows, m), dtype=torch.int32, device=series.device)
        _lib.check(_lib.lib().ddsp_downsample(
            self._h, _dev_ptr(series, torch.int32, "series"), int(rows), int(n),
            int(series.stride(0)), int(factor),
            _dev_ptr(out, torch.int32, "out") if m > 0 else None,
            int(max(m, out.stride(0))), _stream_handle(stream)), "ddsp_downsample")
        return out

    def dered(self, series, half_window, out=None, stream=None):
        """int32 [rows][n] CUDA tensor minus its running median over
        [t - h, t + h] (Sec.3.3)."""
        import torch
        rows, n = series.shape
        if out is None:
            out = torch.empty_like(series)
        _lib.check(_lib.lib().ddsp_dered(
            self._h, _dev_ptr(series, torch.int32, "series"), int(rows), int(n),
            int(series.stride(0)), int(half_window),
            _dev_ptr(out, torch.int32, "out"), int(out.stride(0)),
            _stream_handle(stream)), "ddsp_dered")
        return out

    @staticmethod
    def ffa_rows(nsamp, p):
        """m: the largest power of two with m * p <= nsamp (0 if p > nsamp)."""
        if p < 1 or nsamp < p:
            return 0
        m = 1
        while 2 * m * p <= nsamp:
            m *= 2
        return m

    def ffa(self, series, p, stream=None):
        """Folding transform (Sec.3.5) of int32 [rows][n] series at base
        period p: int32 [rows][m][p]."""
        import torch
        rows, n = series.shape
        m0 = max(self.ffa_rows(n, int(p)), 1)
        out = torch.empty((rows, m0, max(int(p), 1)), dtype=torch.int32,
                          device=series.device)
        m = C.c_int()
        _lib.check(_lib.lib().ddsp_ffa(
            self._h, _dev_ptr(series, torch.int32, "series"), int(rows), int(n),
            int(series.stride(0)), int(p), _dev_ptr(out, torch.int32, "out"),
            C.byref(m), _stream_handle(stream)), "ddsp_ffa")
        return out

    def ffa_search(self, series, p_lo, p_hi, widths, sigma, stream=None):
        """Best boxcar of every folded profile for base periods p_lo ..
        p_hi - 1 (Sec.3.5): (snr, w_idx, phase), each [rows][np][mmax]."""
        import torch
        rows, n = series.shape
        mmax = max(self.ffa_rows(n, int(p_lo)), 1)
        shape = (rows, max(int(p_hi) - int(p_lo), 1), mmax)
        snr = torch.empty(shape, dtype=torch.float32, device=series.device)
        wi = torch.empty(shape, dtype=torch.int32, device=series.device)
        ph = torch.empty(shape, dtype=torch.int32, device=series.device)
        ws = np.ascontiguousarray(widths, dtype=np.int32)
        sg = torch.as_tensor(np.broadcast_to(np.asarray(sigma, np.float32), (rows,))
                             .copy(), device=series.device)
        _lib.check(_lib.lib().ddsp_ffa_search(
            self._h, _dev_ptr(series, torch.int32, "series"), int(rows), int(n),
            int(series.stride(0)), int(p_lo), int(p_hi),
            ws.ctypes.data_as(C.c_void_p), int(ws.size),
            _dev_ptr(sg, torch.float32, "sigma"), _dev_ptr(snr), _dev_ptr(wi),
            _dev_ptr(ph), int(mmax), _stream_handle(stream)), "ddsp_ffa_search")
        return snr, wi, ph

    @staticmethod
    def resample_length(nsamp, tsamp, f0, f1, f2):
        """Output bins of ``resample`` for these parameters."""
        k = C.c_int64()
        _lib.check(_lib.lib().ddsp_resample_length(
            int(nsamp), float(tsamp), float(f0), float(f1), float(f2),
            C.byref(k)), "ddsp_resample_length")
        return k.value

    def resample(self, series, tsamp, f0, f1, f2, stream=None):
        """int32 [rows][n] CUDA tensor resampled for f = f0 + f1 t +
        f2 t^2 / 2 (Sec.3.4): float32 [rows][nout]."""
        import torch
        rows, n = series.shape
        nout = self.resample_length(n, tsamp, f0, f1, f2)
        out = torch.empty((rows, max(nout, 1)), dtype=torch.float32,
                          device=series.device)
        k = C.c_int64()
        _lib.check(_lib.lib().ddsp_resample(
            self._h, _dev_ptr(series, torch.int32, "series"), int(rows), int(n),
            int(series.stride(0)), float(tsamp), float(f0), float(f1), float(f2),
            _dev_ptr(out, torch.float32, "out"), int(out.stride(0)), C.byref(k),
            _stream_handle(stream)), "ddsp_resample")
        return out[:, :k.value]

    def stats(self):
        """Per-(DM, window) exact (2*median, 4*MAD) of the last search."""
        nwin = C.c_int64()
        L = _lib.lib()
        _lib.check(L.ddsp_plan_get_stats(self._h, None, None, 0, C.byref(nwin)),
                   "ddsp_plan_get_stats")
        m2 = np.empty((self.ndm, nwin.value), dtype=np.int64)
        mad4 = np.empty((self.ndm, nwin.value), dtype=np.int64)
        _lib.check(L.ddsp_plan_get_stats(
            self._h, m2.ctypes.data_as(C.c_void_p),
            mad4.ctypes.data_as(C.c_void_p), m2.size, C.byref(nwin)),
            "ddsp_plan_get_stats")
        return m2, mad4

    def check(self, stream=None):
        _lib.check(_lib.lib().ddsp_plan_check(self._h, _stream_handle(stream)),
                   "ddsp_plan_check")

    TUNE_CANDIDATES = 10   # tiles ddsp_plan_autotune tries

    def autotune(self, x, cache=None, reps=2, stream=None):
        """Time the candidate dedispersion tiles on block x (time-major CUDA
        tensor), keep the fastest, record it in the JSON cache file `cache`
        (if given); returns (ms per candidate, -1 where it does not fit;
        index of the winner).  See ddsp_plan_autotune."""
        ms = (C.c_float * self.TUNE_CANDIDATES)()
        best = C.c_int()
        _lib.check(_lib.lib().ddsp_plan_autotune(
            self._h, _dev_ptr(x, self._in_dtype(), "block"), int(x.shape[0]),
            cache.encode() if cache else None, int(reps), _stream_handle(stream),
            ms, self.TUNE_CANDIDATES, C.byref(best)), "ddsp_plan_autotune")
        return list(ms), best.value

    def tile_key(self):
        """The key this plan's tile is cached under (ddsp_plan_tile_key)."""
        buf = C.create_string_buffer(512)
        _lib.check(_lib.lib().ddsp_plan_tile_key(self._h, buf, 512),
                   "ddsp_plan_tile_key")
        return buf.value.decode()

    def set_wait_limit(self, cycles=0):
        """Bound (SM cycles) of the interleaved kernel's hand-off waits; 0 =
        the default (ddsp_plan_set_wait_limit)."""
        _lib.check(_lib.lib().ddsp_plan_set_wait_limit(self._h, int(cycles)),
                   "ddsp_plan_set_wait_limit")

    def withhold_copy(self, chunk=-1):
        """Failure-detection test switch: the copy warp stops before channel
        chunk `chunk` (-1 = off; ddsp_plan_withhold_copy)."""
        _lib.check(_lib.lib().ddsp_plan_withhold_copy(self._h, int(chunk)),
                   "ddsp_plan_withhold_copy")

    def close(self):
        if self._h:
            _lib.lib().ddsp_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Cluster:
    """Peaks filtering with square DM-time stencils, DBSCAN clustering of the
    peaks in the DM-time plane and the strongest member of each cluster
    (Sec.2.1), on a plane of ``ndm`` trials x ``nsamp`` samples; see
    ddsp_peaks_cluster for the exact rules."""

    def __init__(self, ndm, nsamp, capacity, device=None):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        self.ndm, self.nsamp, self.capacity = int(ndm), int(nsamp), int(capacity)
        self._h = C.c_void_p()
        _lib.check(_lib.lib().ddsp_cluster_create(
            C.byref(self._h), int(device), self.ndm, self.nsamp, self.capacity),
            "ddsp_cluster_create")

    @staticmethod
    def to_device(cands, device="cuda"):
        """Candidate records (CAND_DTYPE) as a contiguous int32 [n, 4] CUDA
        tensor with the record layout of ddsp_cand."""
        import torch
        a = np.ascontiguousarray(cands, dtype=CAND_DTYPE)
        return torch.from_numpy(a.view(np.int32).reshape(-1, 4).copy()).to(device)

    def run(self, cands, half, eps_dm, eps_t, min_pts, n=None, count=None,
            stream=None):
        """cands: int32 [>= n, 4] CUDA tensor of records (``to_device``), or
        a raw device pointer with ``n`` given; ``count``: optional device
        counter pointer (the first min(*count, n) records are used)."""
        import torch
        if isinstance(cands, torch.Tensor):
            if cands.dim() != 2 or cands.shape[1] != 4:
                raise ValueError("cands must be [n, 4] int32 records")
            ptr = _dev_ptr(cands, torch.int32, "cands")
            if n is None:
                n = cands.shape[0]
        else:
            ptr = C.c_void_p(int(cands))
        hf = np.ascontiguousarray(half, dtype=np.int32)
        _lib.check(_lib.lib().ddsp_peaks_cluster(
            self._h, ptr, C.c_void_p(int(count)) if count else None, int(n),
            hf.ctypes.data_as(C.c_void_p), int(hf.size), int(eps_dm),
            int(eps_t), int(min_pts), _stream_handle(stream)),
            "ddsp_peaks_cluster")

    def run_plan(self, plan, half, eps_dm, eps_t, min_pts, stream=None):
        """Cluster the candidates of ``plan``'s last search in place, with no
        host round trip (its device buffer and counter)."""
        d_c, d_n, cap = C.c_void_p(), C.c_void_p(), C.c_size_t()
        _lib.check(_lib.lib().ddsp_plan_candidates_device(
            plan._h, C.byref(d_c), C.byref(d_n), C.byref(cap)),
            "ddsp_plan_candidates_device")
        self.run(d_c.value, half, eps_dm, eps_t, min_pts,
                 n=min(cap.value, self.capacity), count=d_n.value, stream=stream)

    def peaks(self, cap=None):
        """(peaks sorted by (dm_idx, t), their int32 cluster labels)."""
        if cap is None:
            cap = self.capacity
        buf = np.zeros(max(cap, 1), dtype=CAND_DTYPE)
        lab = np.zeros(max(cap, 1), dtype=np.int32)
        n = C.c_size_t()
        _lib.check(_lib.lib().ddsp_cluster_fetch_peaks(
            self._h, buf.ctypes.data_as(C.c_void_p),
            lab.ctypes.data_as(C.c_void_p), int(cap), C.byref(n)),
            "ddsp_cluster_fetch_peaks")
        return buf[:n.value].copy(), lab[:n.value].copy()

    def reps(self, cap=None):
        """(strongest member of each cluster in label order, its index in
        the sorted peaks)."""
        if cap is None:
            cap = self.capacity
        buf = np.zeros(max(cap, 1), dtype=CAND_DTYPE)
        idx = np.zeros(max(cap, 1), dtype=np.uint32)
        n = C.c_size_t()
        _lib.check(_lib.lib().ddsp_cluster_fetch_reps(
            self._h, buf.ctypes.data_as(C.c_void_p),
            idx.ctypes.data_as(C.c_void_p), int(cap), C.byref(n)),
            "ddsp_cluster_fetch_reps")
        return buf[:n.value].copy(), idx[:n.value].copy()

    def close(self):
        if self._h:
            _lib.lib().ddsp_cluster_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Rfi:
    """gptool-style RFI mitigation of blocks of 8-bit spectra (Sec.2.1);
    see ddsp_rfi_clean for the exact rules."""

    def __init__(self, max_nsamp, max_nchan, device=None):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        self._h = C.c_void_p()
        self._shape = (0, 0)
        _lib.check(_lib.lib().ddsp_rfi_create(
            C.byref(self._h), int(device), int(max_nsamp), int(max_nchan)),
            "ddsp_rfi_create")

    def clean(self, x, out=None, half_window=10, kc=4, kt=3, rounds=2,
              stream=None):
        """uint8 [nsamp][nchan] CUDA tensor -> cleaned uint8 tensor."""
        import torch
        nt, nc = x.shape
        if out is None:
            out = torch.empty_like(x)
        _lib.check(_lib.lib().ddsp_rfi_clean(
            self._h, _dev_ptr(x, torch.uint8, "spectra"), int(nt), int(nc),
            int(half_window), int(kc), int(kt), int(rounds),
            _dev_ptr(out, torch.uint8, "out"), _stream_handle(stream)),
            "ddsp_rfi_clean")
        self._shape = (nt, nc)
        return out

    def flags(self):
        """(channel flags, time flags, fill level) of the last clean."""
        nt, nc = self._shape
        fc = np.zeros(nc, np.uint8)
        ft = np.zeros(nt, np.uint8)
        fill = C.c_int64()
        _lib.check(_lib.lib().ddsp_rfi_flags(
            self._h, fc.ctypes.data_as(C.c_void_p), ft.ctypes.data_as(C.c_void_p),
            C.byref(fill)), "ddsp_rfi_flags")
        return fc.astype(bool), ft.astype(bool), fill.value

    def close(self):
        if self._h:
            _lib.lib().ddsp_rfi_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many plans (beams of uneven shape) searched together: one persistent
    dedispersion launch plus one batched search launch per step, optionally
    replayed from a captured CUDA graph (``ddsp_batch_*``)."""

    def __init__(self, plans, nsamp_in, series=None):
        import torch
        self.plans = list(plans)
        self.nbeams = len(self.plans)
        self.nsamp_in = [int(n) for n in nsamp_in]
        if series is None:
            series = [torch.empty((p.ndm, p.nsamp_out(n)), dtype=torch.int32,
                                  device="cuda")
                      for p, n in zip(self.plans, self.nsamp_in)]
        self.series = series
        hs = (C.c_void_p * self.nbeams)(*[p._h.value for p in self.plans])
        ns = (C.c_int64 * self.nbeams)(*self.nsamp_in)
        outs = (C.c_void_p * self.nbeams)(
            *[_dev_ptr(t, torch.int32, "series").value for t in series])
        self._h = C.c_void_p()
        _lib.check(_lib.lib().ddsp_batch_create(
            C.byref(self._h), hs, self.nbeams, ns, outs), "ddsp_batch_create")

    def ingest(self, beam, x, stream=None):
        """Unpack beam `beam`'s time-major block (CUDA uint8 tensor)."""
        import torch
        _lib.check(_lib.lib().ddsp_batch_ingest(
            self._h, int(beam), _dev_ptr(x, torch.uint8, "spectra"),
            _stream_handle(stream)), "ddsp_batch_ingest")

    def input_rows(self, beam):
        """(device pointer, pitch, nsamp_in) of a beam's channel-major rows."""
        ptr, pitch, nin = C.c_void_p(), C.c_int64(), C.c_int64()
        _lib.check(_lib.lib().ddsp_batch_input(
            self._h, int(beam), C.byref(ptr), C.byref(pitch), C.byref(nin)),
            "ddsp_batch_input")
        return ptr.value, pitch.value, nin.value

    def run(self, threshold, use_graph=True, stream=None):
        _lib.check(_lib.lib().ddsp_batch_run(self._h, float(threshold),
                                             int(bool(use_graph)),
                                             _stream_handle(stream)),
                   "ddsp_batch_run")

    def check(self, stream=None):
        _lib.check(_lib.lib().ddsp_batch_check(self._h, _stream_handle(stream)),
                   "ddsp_batch_check")

    def set_tile(self, dm_tile, dm_per_thread, chan_chunk, stages):
        _lib.check(_lib.lib().ddsp_batch_set_tile(
            self._h, int(dm_tile), int(dm_per_thread), int(chan_chunk),
            int(stages)), "ddsp_batch_set_tile")

    def get_tile(self):
        v = [C.c_int() for _ in range(6)]
        _lib.check(_lib.lib().ddsp_batch_get_tile(self._h, *[C.byref(a) for a in v]),
                   "ddsp_batch_get_tile")
        keys = ("dm_tile", "dm_per_thread", "time_tile", "chan_chunk", "stages",
                "grid")
        return dict(zip(keys, (a.value for a in v)))

    def beam_chunk(self, beam):
        """Channels per staging chunk beam `beam` uses under the current
        tile (the tile's chan_chunk is the upper limit)."""
        v = C.c_int()
        _lib.check(_lib.lib().ddsp_batch_get_beam_chunk(self._h, int(beam),
                                                         C.byref(v)),
                   "ddsp_batch_get_beam_chunk")
        return v.value

    PERSISTENT = 0
    PER_BEAM = 1

    def set_mode(self, mode):
        """Batch.PERSISTENT (persistent relayout kernel over a work queue)
        or Batch.PER_BEAM (beam after beam through the interleaved kernel,
        one shared staging area); see ddsp_batch_set_mode."""
        _lib.check(_lib.lib().ddsp_batch_set_mode(self._h, int(mode)),
                   "ddsp_batch_set_mode")

    def get_mode(self) -> int:
        v = C.c_int()
        _lib.check(_lib.lib().ddsp_batch_get_mode(self._h, C.byref(v)),
                   "ddsp_batch_get_mode")
        return v.value

    def beam_tile(self, beam):
        """dict(dm_tile, dm_per_thread, time_tile, chan_chunk, group) of the
        shape beam `beam` is dedispersed with (group 1: the second
        persistent launch for coarse DM grids)."""
        v = [C.c_int() for _ in range(5)]
        _lib.check(_lib.lib().ddsp_batch_get_beam_tile(
            self._h, int(beam), *[C.byref(a) for a in v]), "ddsp_batch_get_beam_tile")
        keys = ("dm_tile", "dm_per_thread", "time_tile", "chan_chunk", "group")
        return dict(zip(keys, (a.value for a in v)))

    def autotune(self, reps=2, stream=None):
        """Time every candidate tile on a 1/16 sample of the work items,
        keep the fastest, then one whole pass of the per-beam interleaved
        mode (the last candidate), taken if faster; returns (list of
        estimated full-launch ms per candidate (-1 = does not fit or not
        available), chosen index)."""
        cap = 64
        ms = (C.c_float * cap)()
        nt, best = C.c_int(), C.c_int()
        _lib.check(_lib.lib().ddsp_batch_autotune(
            self._h, int(reps), _stream_handle(stream), ms, cap, C.byref(nt),
            C.byref(best)), "ddsp_batch_autotune")
        return [ms[i] for i in range(nt.value)], best.value

    def close(self):
        if self._h:
            _lib.lib().ddsp_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Streaming search of many beams of one plan's shape (``ddsp_server_*``):
    per-beam rings in device memory, admission against free device memory,
    and steps that dedisperse and search the waiting block of every ready
    beam in one persistent launch plus one batched search launch."""

    def __init__(self, plan, block_samples, max_beams, hbm_reserve_bytes=0,
                 tile=None):
        self.plan = plan
        self.block = int(block_samples)
        self.max_beams = int(max_beams)
        dm_tile, dm_per_thread, chan_chunk, stages = tile or (0, 0, 0, 0)
        self._h = C.c_void_p()
        _lib.check(_lib.lib().ddsp_server_create(
            C.byref(self._h), plan._h, self.block, self.max_beams,
            int(hbm_reserve_bytes), int(dm_tile), int(dm_per_thread),
            int(chan_chunk), int(stages)), "ddsp_server_create")
        v = [C.c_int64() for _ in range(5)]
        _lib.check(_lib.lib().ddsp_server_info(self._h, *[C.byref(a) for a in v]),
                   "ddsp_server_info")
        (self.beam_bytes, self.ring_samples, self.series_cols, self.carry,
         self.first_delay) = (a.value for a in v)
        # a beam's ring holds the B + D16 samples a step reads plus one
        # block: one block per beam may wait for a step
        self.max_waiting = 1

    RELAYOUT = 0
    INTERLEAVED = 1

    def set_mode(self, mode, staging_slots=8):
        """Server.RELAYOUT (persistent relayout kernel on the rings) or
        Server.INTERLEAVED (beam-blocks interleaved into staging_slots
        slots, one interleaved launch per group); see ddsp_server_set_mode.
        Set it before admitting beams."""
        _lib.check(_lib.lib().ddsp_server_set_mode(self._h, int(mode),
                                                   int(staging_slots)),
                   "ddsp_server_set_mode")

    def get_mode(self):
        """(mode, staging slots)."""
        m, k = C.c_int(), C.c_int()
        _lib.check(_lib.lib().ddsp_server_get_mode(self._h, C.byref(m),
                                                   C.byref(k)),
                   "ddsp_server_get_mode")
        return m.value, k.value

    def get_tile(self):
        v = [C.c_int() for _ in range(6)]
        _lib.check(_lib.lib().ddsp_server_get_tile(self._h, *[C.byref(a) for a in v]),
                   "ddsp_server_get_tile")
        keys = ("dm_tile", "dm_per_thread", "time_tile", "chan_chunk", "stages",
                "grid")
        return dict(zip(keys, (a.value for a in v)))

    def admit(self):
        """Index of a newly admitted beam; DdspError(DDSP_E_NOMEM) if its
        buffers do not fit the free device memory less the reserve."""
        b = C.c_int()
        _lib.check(_lib.lib().ddsp_server_admit(self._h, C.byref(b)),
                   "ddsp_server_admit")
        return b.value

    def evict(self, beam):
        _lib.check(_lib.lib().ddsp_server_evict(self._h, int(beam)),
                   "ddsp_server_evict")

    def push(self, beam, x, stream=None):
        """Ingest beam `beam`'s next block (CUDA uint8 [block][nchan]);
        returns False (nothing done) if the beam's previous block has not
        been taken by a step yet."""
        import torch
        rc = _lib.lib().ddsp_server_push(self._h, int(beam),
                                         _dev_ptr(x, torch.uint8, "block"),
                                         _stream_handle(stream))
        if rc == _lib.DDSP_E_STATE:
            return False
        _lib.check(rc, "ddsp_server_push")
        return True

    def step(self, threshold, max_beams_in_step=0, stream=None):
        """Launch one step; returns (step id, beams in it) or (-1, [])."""
        sid, n = C.c_int64(), C.c_int()
        beams = (C.c_int * self.max_beams)()
        _lib.check(_lib.lib().ddsp_server_step(
            self._h, float(threshold), int(max_beams_in_step),
            _stream_handle(stream), C.byref(sid), beams, self.max_beams,
            C.byref(n)), "ddsp_server_step")
        return sid.value, list(beams[:n.value])

    def done(self, step_id):
        rc = _lib.lib().ddsp_server_query(self._h, int(step_id))
        if rc < 0:
            _lib.check(rc, "ddsp_server_query")
        return rc == 1

    def fetch(self, beam, block, cap=None, allow_truncated=False):
        """(candidates sorted by (dm_idx, t), true count, global output
        sample of series column 0) of one of the beam's two most recently
        stepped blocks.  With allow_truncated, a block that found more than
        the capacity returns the stored records and the true count."""
        if cap is None:
            cap = self.plan.cand_capacity
        buf = np.zeros(cap, dtype=CAND_DTYPE)
        n, t0 = C.c_size_t(), C.c_int64()
        rc = _lib.lib().ddsp_server_fetch(
            self._h, int(beam), int(block), buf.ctypes.data_as(C.c_void_p),
            int(cap), C.byref(n), C.byref(t0))
        if rc == _lib.DDSP_E_TRUNCATED and allow_truncated:
            return buf[:min(cap, self.plan.cand_capacity)].copy(), n.value, t0.value
        _lib.check(rc, "ddsp_server_fetch")
        return buf[:n.value].copy(), n.value, t0.value

    def series(self, beam):
        """The series [ndm][carry + block] of the beam's last stepped block as
        a CUDA int32 view of its series slot (once its step completed), while
        it is still there: only blocks of the last group of the latest step
        (DdspError DDSP_E_STATE otherwise); the next step reuses the slot."""
        import torch
        ptr, ncols = C.c_void_p(), C.c_int64()
        _lib.check(_lib.lib().ddsp_server_series(self._h, int(beam), C.byref(ptr),
                                                 C.byref(ncols)),
                   "ddsp_server_series")
        return _tensor_view(ptr.value, (self.plan.ndm, ncols.value), torch.int32)

    def check(self, stream=None):
        _lib.check(_lib.lib().ddsp_server_check(self._h, _stream_handle(stream)),
                   "ddsp_server_check")

    def close(self):
        if self._h:
            _lib.lib().ddsp_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_unit_peaks(device=0) -> dict:
    """Measured per-SM rates of the units the dedispersion is bound by
    (ddsp_probe_unit_peaks): shared-memory bytes, 3-input adds, byte
    permutes and dedispersion-loop sample adds per SM clock."""
    v = _lib.DdspUnitPeaks()
    _lib.check(_lib.lib().ddsp_probe_unit_peaks(int(device), C.byref(v)),
               "ddsp_probe_unit_peaks")
    return {"sms": v.sms, "blocks_per_sm": list(v.blocks_per_sm),
            "smem_bytes_per_clk": v.smem_bytes_per_clk,
            "iadd3_per_clk": v.iadd3_per_clk, "prmt_per_clk": v.prmt_per_clk,
            "swar_adds_per_clk": v.swar_adds_per_clk}
