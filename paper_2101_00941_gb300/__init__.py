"""Python binding of the GB300 dedispersion + single-pulse-search library (``libdd.so``).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels behind the C ABI declared in ``include/dd.h``. The functions keep the C
names (``dd_plan``, ``dd_run``, ``sps_run``, ...); ``Plan`` is a thin owner of a
plan handle. There is no CPU fallback: if the library was not built, loading
it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build_lib import LIB_PATH, build  # noqa: F401

DD_OK = 0
DD_ERR_ARG = -1
DD_ERR_NOMEM = -2
DD_ERR_CUDA = -3
DD_ERR_TIMEOUT = -4
DD_KERNEL_TILED, DD_KERNEL_DIRECT, DD_KERNEL_PER_OUTPUT = 1, 2, 3
DD_ERR_CAP = -5
DD_ERR_STATE = -6
DD_FLAG_TIMING = 1
DD_FLAG_NAIVE = 2
DD_FLAG_DEVICE_INPUT = 4
DD_FLAG_TILE256 = 8
DD_FLAG_TRIALS32 = 16
DD_FLAG_AUTOTUNE = 32
DD_FLAG_WARPS32 = 64
DD_EST_WINDOW = 0
DD_EST_CLIPPED = 1
DD_FUSE_KEEP_SERIES = 1
DD_BATCH_GRAPH = 1
DD_BATCH_AUTOTUNE = 2
DD_BATCH_PERSISTENT = 4

EXPORTS = ("dd_plan", "dd_plan_info", "dd_plan_kernel", "dd_selftest_wait",
           "dd_tiled_plan_check", "dd_run", "dd_series", "sps_run", "dd_candidates", "dd_sync",
           "dd_stats", "dd_sps_static", "dd_serve_create", "dd_serve_add_beam", "dd_serve_submit",
           "dd_serve_poll", "dd_serve_pending", "dd_serve_destroy", "dd_batch_create",
           "dd_batch_run", "dd_batch_wait", "dd_batch_info", "dd_batch_candidates",
           "dd_batch_destroy", "dd_plan_destroy", "dd_last_error", "dd_moments",
           "dd_plan_model", "dd_measure_peaks", "dd_stats_range", "dd_group_candidates",
           "sps_run_ex")


class dd_range_t(ctypes.Structure):
    _fields_ = [("dm_start", ctypes.c_double), ("dm_step", ctypes.c_double),
                ("n_trials", ctypes.c_int32), ("decimation", ctypes.c_int32)]


class dd_opts_t(ctypes.Structure):
    _fields_ = [("chunk_len", ctypes.c_int64), ("n_streams", ctypes.c_int32),
                ("max_width", ctypes.c_int32), ("peak_block", ctypes.c_int32),
                ("device", ctypes.c_int32), ("max_cands", ctypes.c_int64),
                ("flags", ctypes.c_uint32), ("staging_threads", ctypes.c_int32)]


class dd_launch_model_t(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("tile_samples", ctypes.c_int32),
                ("tile_trials", ctypes.c_int32), ("cta_threads", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("fused", ctypes.c_int32),
                ("outputs", ctypes.c_int64), ("adds", ctypes.c_double),
                ("dram_bytes", ctypes.c_double), ("smem_wavefronts", ctypes.c_double),
                ("copy_bytes", ctypes.c_double)]


class dd_peaks_t(ctypes.Structure):
    _fields_ = [("sms", ctypes.c_int32), ("pad", ctypes.c_int32), ("sm_mhz", ctypes.c_double),
                ("alu_lanes_per_clk", ctypes.c_double), ("dp_lanes_per_clk", ctypes.c_double),
                ("int_lanes_per_clk", ctypes.c_double), ("add_per_clk", ctypes.c_double),
                ("lds_wavefronts_per_clk", ctypes.c_double)]


GROUP_DTYPE = np.dtype([("rep", "<i8"), ("members", "<i8"), ("dm_lo", "<f8"), ("dm_hi", "<f8"),
                        ("t_lo", "<i8"), ("t_hi", "<i8")])

MOMENTS_DTYPE = np.dtype([("s1", "<i8"), ("s2lo", "<u8"), ("s2hi", "<u8"), ("pad", "<u8")])


class dd_sps_opts_t(ctypes.Structure):
    _fields_ = [("estimator", ctypes.c_int32), ("clip_iters", ctypes.c_int32),
                ("clip_kappa", ctypes.c_double)]


class dd_batch_beam_t(ctypes.Structure):
    _fields_ = [("freqs_mhz", ctypes.c_void_p), ("nchans", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("tsamp_s", ctypes.c_double), ("nsamp", ctypes.c_int64), ("input", ctypes.c_void_p)]


class dd_serve_result_t(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("beam", ctypes.c_int32), ("status", ctypes.c_int32),
                ("seq", ctypes.c_int64), ("ncands", ctypes.c_int64), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]


CAND_DTYPE = np.dtype([("trial", "<i4"), ("range", "<i4"), ("t_start", "<i8"), ("width", "<i4"),
                       ("pad", "<i4"), ("snr", "<f8")])


class DDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dd error {code}: {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load libdd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2101_00941_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, f32, f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                  ctypes.c_double)
        P = ctypes.POINTER
        L.dd_plan.argtypes = [vp, i32, f64, vp, i32, P(dd_opts_t), P(vp)]
        L.dd_plan_info.argtypes = [vp, P(i64), P(i32), P(vp)]
        L.dd_plan_kernel.argtypes = [vp, i32, P(i32), P(i32)]
        L.dd_selftest_wait.argtypes = [i32, P(i32), P(ctypes.c_double)]
        L.dd_tiled_plan_check.argtypes = [vp, i32, i32, i32, i32, i32, P(i32), P(i64)]
        L.dd_run.argtypes = [vp, vp, i64, vp]
        L.dd_series.argtypes = [vp, i32, P(vp), P(i64), P(i64), P(i64)]
        L.sps_run.argtypes = [vp, vp, i32, f32]
        L.dd_fuse_search.argtypes = [vp, vp, i32, ctypes.c_uint32, P(i32)]
        L.sps_run_ex.argtypes = [vp, vp, i32, f32, P(dd_sps_opts_t)]
        L.dd_candidates.argtypes = [vp, i64, vp, i64, P(i64), i64]
        L.dd_sync.argtypes = [vp]
        L.dd_stats.argtypes = [vp, P(i64), P(f64), P(i64), i32]
        L.dd_moments.argtypes = [vp, i32, P(vp), P(i64)]
        L.dd_stats_range.argtypes = [vp, i32, P(f64), P(i64)]
        L.dd_group_candidates.argtypes = [vp, i64, vp, i32, f64, i64, vp, i64, P(i64), vp]
        L.dd_plan_model.argtypes = [vp, i32, i64, P(dd_launch_model_t)]
        L.dd_measure_peaks.argtypes = [i32, P(dd_peaks_t)]
        L.dd_sps_static.argtypes = [vp, i32, i64, i64, i32, i32, i64, vp, i32, f32, i32, vp, i64,
                                    vp, vp]
        L.dd_plan_destroy.argtypes = [vp]
        L.dd_plan_destroy.restype = None
        L.dd_serve_create.argtypes = [i32, i64, i32, P(vp)]
        L.dd_serve_add_beam.argtypes = [vp, vp, i32, f64, vp, i32, P(dd_opts_t), vp, i32, f32,
                                        P(i32)]
        L.dd_serve_submit.argtypes = [vp, i32, vp, i64, vp, i64, P(i64)]
        L.dd_serve_poll.argtypes = [vp, vp, i32, P(i32), i64]
        L.dd_serve_pending.argtypes = [vp, P(i64), P(i32)]
        L.dd_serve_destroy.argtypes = [vp]
        L.dd_serve_destroy.restype = None
        L.dd_batch_create.argtypes = [i32, vp, vp, i32, P(dd_opts_t), vp, i32, f32, i64,
                                      ctypes.c_uint32, P(vp)]
        L.dd_batch_run.argtypes = [vp]
        L.dd_batch_wait.argtypes = [vp, i64]
        L.dd_batch_info.argtypes = [vp, i32, P(i64), P(i64), P(i32)]
        L.dd_batch_candidates.argtypes = [vp, i32, i64, vp, i64, P(i64)]
        L.dd_batch_destroy.argtypes = [vp]
        L.dd_batch_destroy.restype = None
        L.dd_last_error.argtypes = []
        L.dd_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("dd_plan_destroy", "dd_serve_destroy", "dd_batch_destroy",
                            "dd_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def dd_last_error() -> str:
    return lib().dd_last_error().decode()


def _check(rc: int):
    if rc != DD_OK:
        raise DDError(rc, dd_last_error())
    return rc


def _ptr(a) -> int:
    """Address of a numpy array, a torch tensor (host or device) or an int."""
    if a is None:
        return 0
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def dd_plan(freqs_mhz, tsamp_s: float, ranges, chunk_len: int, n_streams: int = 1,
            max_width: int = 256, peak_block: int = 32, device: int = 0, max_cands: int = 0,
            flags: int = 0, staging_threads: int = 0) -> int:
    """Create a plan; ``ranges`` rows are (dm_start, dm_step, n_trials, decimation)."""
    f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
    rr = (dd_range_t * len(ranges))(*[dd_range_t(float(r[0]), float(r[1]), int(r[2]), int(r[3]))
                                      for r in ranges])
    o = dd_opts_t(int(chunk_len), int(n_streams), int(max_width), int(peak_block), int(device),
                  int(max_cands), int(flags), int(staging_threads))
    h = ctypes.c_void_p()
    _check(lib().dd_plan(f.ctypes.data, f.size, float(tsamp_s), ctypes.addressof(rr), len(ranges),
                         ctypes.byref(o), ctypes.byref(h)))
    return h.value


def dd_plan_info(plan: int, nchans: int):
    """(overlap, total trials, host copy of the delay table [trials][nchans])."""
    O = ctypes.c_int64()
    nt = ctypes.c_int32()
    sp = ctypes.c_void_p()
    _check(lib().dd_plan_info(plan, ctypes.byref(O), ctypes.byref(nt), ctypes.byref(sp)))
    buf = (ctypes.c_int32 * (nt.value * nchans)).from_address(sp.value)
    return O.value, nt.value, np.ctypeslib.as_array(buf).reshape(nt.value, nchans).copy()


def dd_plan_kernel(plan: int, range_idx: int):
    """(kernel kind of range `range_idx`: DD_KERNEL_TILED / _DIRECT / _PER_OUTPUT, tile or 0)."""
    t, tt = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().dd_plan_kernel(plan, int(range_idx), ctypes.byref(t), ctypes.byref(tt)))
    return t.value, tt.value


def dd_selftest_wait(device: int = 0):
    """(1 if the device-side bounded wait ran out and was reported, host ms) -- see dd.h."""
    t, ms = ctypes.c_int32(), ctypes.c_double()
    _check(lib().dd_selftest_wait(int(device), ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def dd_tiled_plan_check(shifts, decimation: int, tile_samples: int = 512, tile_trials: int = 64):
    """Host-only check of the tiled plan of one range (see dd.h): (ok, violations).
    `shifts` is int32 [n_trials][cpad] with cpad a multiple of 8."""
    a = np.ascontiguousarray(shifts, dtype=np.int32)
    ok, bad = ctypes.c_int32(), ctypes.c_int64()
    _check(lib().dd_tiled_plan_check(a.ctypes.data, a.shape[0], a.shape[1], int(decimation),
                                     int(tile_samples), int(tile_trials), ctypes.byref(ok),
                                     ctypes.byref(bad)))
    return ok.value, bad.value


def dd_run(plan: int, chunk, nsamp: int, cuda_stream: int = 0):
    _check(lib().dd_run(plan, _ptr(chunk), int(nsamp), int(cuda_stream) or None))


def dd_series(plan: int, range_idx: int):
    """(device pointer, window length, row stride, global index of sample 0)."""
    p = ctypes.c_void_p()
    n, st, j0 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().dd_series(plan, int(range_idx), ctypes.byref(p), ctypes.byref(n),
                           ctypes.byref(st), ctypes.byref(j0)))
    return p.value, n.value, st.value, j0.value


def dd_moments(plan: int, range_idx: int):
    """(device pointer to dd_moments_t [n_trials], window length n) of the latest chunk."""
    p, n = ctypes.c_void_p(), ctypes.c_int64()
    _check(lib().dd_moments(plan, int(range_idx), ctypes.byref(p), ctypes.byref(n)))
    return p.value, n.value


def dd_fuse_search(plan: int, widths, keep_series: bool = False) -> int:
    """Fuse the search's position pass into the dedispersion kernel (see dd.h); returns the
    number of fused ranges."""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    n = ctypes.c_int32()
    _check(lib().dd_fuse_search(plan, w.ctypes.data, int(w.size),
                                DD_FUSE_KEEP_SERIES if keep_series else 0, ctypes.byref(n)))
    return n.value


def dd_plan_model(plan: int, range_idx: int, nout: int) -> dict:
    """Work of one dedispersion launch of a range over nout outputs (see dd.h)."""
    m = dd_launch_model_t()
    _check(lib().dd_plan_model(plan, int(range_idx), int(nout), ctypes.byref(m)))
    return {f: getattr(m, f) for f, _ in dd_launch_model_t._fields_}


def dd_measure_peaks(device: int = 0) -> dict:
    """Measured integer and shared-memory issue rates of the device (see dd.h)."""
    p = dd_peaks_t()
    _check(lib().dd_measure_peaks(int(device), ctypes.byref(p)))
    return {f: getattr(p, f) for f, _ in dd_peaks_t._fields_ if f != "pad"}


def sps_run(plan: int, widths, threshold: float):
    w = np.ascontiguousarray(widths, dtype=np.int32)
    _check(lib().sps_run(plan, w.ctypes.data, w.size, ctypes.c_float(threshold)))


def sps_run_ex(plan: int, widths, threshold: float, estimator: int = DD_EST_WINDOW,
               clip_iters: int = 3, clip_kappa: float = 3.0):
    """sps_run with a choice of noise statistic (see dd.h)."""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    o = dd_sps_opts_t(int(estimator), int(clip_iters), float(clip_kappa))
    _check(lib().sps_run_ex(plan, w.ctypes.data, w.size, ctypes.c_float(threshold),
                            ctypes.byref(o)))


def dd_candidates(plan: int, seq: int, cap: int = 1 << 20, timeout_ms: int = 0) -> np.ndarray:
    out = np.zeros(cap, dtype=CAND_DTYPE)
    n = ctypes.c_int64()
    rc = lib().dd_candidates(plan, int(seq), out.ctypes.data, int(cap), ctypes.byref(n),
                             int(timeout_ms))
    _check(rc)
    return out[:n.value]


def dd_sync(plan: int):
    _check(lib().dd_sync(plan))


def dd_stats(plan: int, reset: bool = False):
    """(kernel launches, summed dedispersion ms, dedispersion launches timed)."""
    a, b, c = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    _check(lib().dd_stats(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), int(reset)))
    return a.value, b.value, c.value


def dd_group_candidates(cands: np.ndarray, ranges, dm_link: float, t_link: int):
    """(per-candidate group label, GROUP_DTYPE records) -- friends-of-friends; see dd.h."""
    c = np.ascontiguousarray(cands, dtype=CAND_DTYPE)
    rr = (dd_range_t * len(ranges))(*[dd_range_t(float(r[0]), float(r[1]), int(r[2]), int(r[3]))
                                      for r in ranges])
    out = np.zeros(max(1, c.size), dtype=GROUP_DTYPE)
    label = np.zeros(max(1, c.size), dtype=np.int64)
    n = ctypes.c_int64()
    _check(lib().dd_group_candidates(c.ctypes.data if c.size else None, c.size,
                                     ctypes.addressof(rr), len(ranges), float(dm_link),
                                     int(t_link), out.ctypes.data, out.size, ctypes.byref(n),
                                     label.ctypes.data))
    return label[:c.size], out[:n.value]


def dd_stats_range(plan: int, range_idx: int):
    """(dedispersion ms of one range's launches, their number) -- see dd.h."""
    b, c = ctypes.c_double(), ctypes.c_int64()
    _check(lib().dd_stats_range(plan, int(range_idx), ctypes.byref(b), ctypes.byref(c)))
    return b.value, c.value


def dd_sps_static(series_ptr: int, n_trials: int, n: int, stride: int, range_idx: int,
                  decimation: int, j0: int, widths, threshold: float, peak_block: int,
                  cands_ptr: int, cap: int, count_ptr: int, cuda_stream: int = 0):
    """Search device series with the library's fixed scratch (no allocation); see dd.h."""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    _check(lib().dd_sps_static(int(series_ptr), int(n_trials), int(n), int(stride),
                               int(range_idx), int(decimation), int(j0), w.ctypes.data, w.size,
                               ctypes.c_float(threshold), int(peak_block), int(cands_ptr),
                               int(cap), int(count_ptr), int(cuda_stream) or None))


def dd_plan_destroy(plan: int):
    if plan:
        lib().dd_plan_destroy(plan)


class Plan:
    """Owner of a plan handle (destroys it on close)."""

    def __init__(self, freqs_mhz, tsamp_s, ranges, chunk_len, **kw):
        self.nchans = int(np.asarray(freqs_mhz).size)
        self.ranges = [tuple(r) for r in ranges]
        self.h = dd_plan(freqs_mhz, tsamp_s, ranges, chunk_len, **kw)
        self.O, self.ntrials, self.shifts = dd_plan_info(self.h, self.nchans)
        self.seq = -1

    def kernel(self, range_idx):
        """(kernel kind, tile samples) of one range; see dd_plan_kernel."""
        return dd_plan_kernel(self.h, range_idx)

    def run(self, chunk, nsamp=None, cuda_stream=0) -> int:
        n = chunk.shape[0] if nsamp is None else nsamp
        dd_run(self.h, chunk, n, cuda_stream)
        self.seq += 1
        return self.seq

    def search(self, widths, threshold, estimator=None, clip_iters=3, clip_kappa=3.0):
        if estimator is None:
            sps_run(self.h, widths, threshold)
        else:
            sps_run_ex(self.h, widths, threshold, estimator, clip_iters, clip_kappa)

    def candidates(self, seq=None, cap=1 << 20, timeout_ms=0):
        return dd_candidates(self.h, self.seq if seq is None else seq, cap, timeout_ms)

    def series(self, range_idx):
        """The latest chunk's series of a range: (torch int32 [n_trials][len] copy, j0)."""
        ptr, n, stride, j0 = dd_series(self.h, range_idx)
        ntr = int(self.ranges[range_idx][2])
        dd_sync(self.h)
        return device_view(ptr, (ntr, stride), "<i4")[:, :n].clone(), j0

    def moments(self, range_idx):
        """The latest chunk's moments of a range as a numpy MOMENTS_DTYPE [n_trials] copy, and
        the window length they cover."""
        ptr, n = dd_moments(self.h, range_idx)
        ntr = int(self.ranges[range_idx][2])
        dd_sync(self.h)
        raw = device_view(ptr, (ntr, 4), "<i8").cpu().numpy()
        return raw.copy().view(MOMENTS_DTYPE).reshape(ntr), n

    def model(self, range_idx, nout):
        return dd_plan_model(self.h, range_idx, nout)

    def fuse_search(self, widths, keep_series=False) -> int:
        """dd_fuse_search: returns the number of fused ranges."""
        return dd_fuse_search(self.h, widths, keep_series)

    def sync(self):
        dd_sync(self.h)

    def stats(self, reset=False):
        return dd_stats(self.h, reset)

    def stats_range(self, range_idx):
        return dd_stats_range(self.h, range_idx)

    def close(self):
        if self.h:
            dd_plan_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop over many beams (dd_serve_*): submit chunks as they arrive, poll results."""

    def __init__(self, max_inflight: int, hbm_budget_bytes: int, device: int = 0):
        h = ctypes.c_void_p()
        _check(lib().dd_serve_create(int(max_inflight), int(hbm_budget_bytes), int(device),
                                     ctypes.byref(h)))
        self.h = h.value
        self._keep = {}  # ticket -> (chunk, out buffer) kept alive until polled

    def add_beam(self, freqs_mhz, tsamp_s, ranges, chunk_len, widths, threshold, n_streams=2,
                 max_width=None, peak_block=32, max_cands=0, flags=0, staging_threads=0) -> int:
        f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
        rr = (dd_range_t * len(ranges))(*[dd_range_t(float(r[0]), float(r[1]), int(r[2]),
                                                     int(r[3])) for r in ranges])
        w = np.ascontiguousarray(widths, dtype=np.int32)
        o = dd_opts_t(int(chunk_len), int(n_streams), int(max_width or int(w.max())),
                      int(peak_block), 0, int(max_cands), int(flags), int(staging_threads))
        b = ctypes.c_int32()
        _check(lib().dd_serve_add_beam(self.h, f.ctypes.data, f.size, float(tsamp_s),
                                       ctypes.addressof(rr), len(ranges), ctypes.byref(o),
                                       w.ctypes.data, w.size, ctypes.c_float(threshold),
                                       ctypes.byref(b)))
        return b.value

    def submit(self, beam: int, chunk, nsamp=None, cap: int = 1 << 16) -> int:
        n = chunk.shape[0] if nsamp is None else nsamp
        out = np.zeros(cap, dtype=CAND_DTYPE)
        t = ctypes.c_int64()
        _check(lib().dd_serve_submit(self.h, int(beam), _ptr(chunk), int(n), out.ctypes.data,
                                     int(cap), ctypes.byref(t)))
        self._keep[t.value] = (chunk, out)
        return t.value

    def poll(self, max_results: int = 64, timeout_ms: int = 0):
        """Finished results as (dd_serve_result_t fields dict, candidates array)."""
        buf = (dd_serve_result_t * max_results)()
        n = ctypes.c_int32()
        _check(lib().dd_serve_poll(self.h, ctypes.addressof(buf), int(max_results),
                                   ctypes.byref(n), int(timeout_ms)))
        out = []
        for k in range(n.value):
            r = buf[k]
            d = {f: getattr(r, f) for f, _ in dd_serve_result_t._fields_}
            _, cands = self._keep.pop(r.ticket, (None, None))
            out.append((d, None if cands is None else cands[:min(r.ncands, cands.size)]))
        return out

    def pending(self):
        q, i = ctypes.c_int64(), ctypes.c_int32()
        _check(lib().dd_serve_pending(self.h, ctypes.byref(q), ctypes.byref(i)))
        return q.value, i.value

    def close(self):
        if self.h:
            lib().dd_serve_destroy(self.h)
            self.h = 0
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many beams processed in one step (dd_batch_*). `beams`: list of (freqs, tsamp, device
    uint8 tensor [nsamp][nchans]); the tensors must stay alive and in place."""

    def __init__(self, beams, ranges, chunk_len, widths, threshold, n_streams=1,
                 max_width=None, peak_block=32, cap_per_chunk=1 << 14, graph=False,
                 autotune=False, persistent=False, device=0, flags=DD_FLAG_DEVICE_INPUT):
        self._freqs = [np.ascontiguousarray(f, dtype=np.float64) for f, _, _ in beams]
        self._inputs = [x for _, _, x in beams]
        arr = (dd_batch_beam_t * len(beams))()
        for k, (f, ts, x) in enumerate(beams):
            arr[k] = dd_batch_beam_t(self._freqs[k].ctypes.data, int(self._freqs[k].size), 0,
                                     float(ts), int(x.shape[0]), _ptr(x))
        rr = (dd_range_t * len(ranges))(*[dd_range_t(float(r[0]), float(r[1]), int(r[2]),
                                                     int(r[3])) for r in ranges])
        w = np.ascontiguousarray(widths, dtype=np.int32)
        o = dd_opts_t(int(chunk_len), int(n_streams), int(max_width or int(w.max())),
                      int(peak_block), int(device), 0, int(flags), 0)
        h = ctypes.c_void_p()
        bf = ((DD_BATCH_GRAPH if graph else 0) | (DD_BATCH_AUTOTUNE if autotune else 0) |
              (DD_BATCH_PERSISTENT if persistent else 0))
        _check(lib().dd_batch_create(len(beams), ctypes.addressof(arr), ctypes.addressof(rr),
                                     len(ranges), ctypes.byref(o), w.ctypes.data, w.size,
                                     ctypes.c_float(threshold), int(cap_per_chunk), bf,
                                     ctypes.byref(h)))
        self.h = h.value
        self.cap = int(cap_per_chunk)
        self.nbeams = len(beams)

    def run(self):
        _check(lib().dd_batch_run(self.h))

    def wait(self, timeout_ms=0):
        _check(lib().dd_batch_wait(self.h, int(timeout_ms)))

    def info(self, beam):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib().dd_batch_info(self.h, int(beam), ctypes.byref(a), ctypes.byref(b),
                                   ctypes.byref(c)))
        return a.value, b.value, c.value

    def candidates(self, beam, chunk):
        out = np.zeros(self.cap, dtype=CAND_DTYPE)
        n = ctypes.c_int64()
        _check(lib().dd_batch_candidates(self.h, int(beam), int(chunk), out.ctypes.data,
                                         self.cap, ctypes.byref(n)))
        return out[:n.value]

    def close(self):
        if self.h:
            lib().dd_batch_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _CudaArray:
    """Exposes a plan-owned device buffer through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_view(ptr: int, shape, typestr: str):
    """A torch tensor viewing device memory owned by the library (valid while the plan lives)."""
    import torch
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")
