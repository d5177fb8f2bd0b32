"""CPU oracle: plain, slow, obviously correct dedispersion + single-pulse search.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The GPU library
(``paper_2101_00941_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``dd_oracle.c`` (FP64 delay table and SNR, exact
integer sums), built with gcc and ``-ffp-contract=off``; this module only
marshals arrays and applies the chunk-window bookkeeping.

Problem statement followed (Novotny, Adamek & Armour, Sec. 1-2.2): 8-bit
filterbank data is split into time chunks; each chunk is dedispersed over a
DM-trial plan (brute-force incoherent sum over channels at per-channel
dispersion delays, with time decimation for high-DM ranges), then searched
for single pulses with boxcar filters. The paper prints no formulas; the
READINGs taken are stated in ``dd_oracle.c`` beside each function.

Chunk windows (READING): a plan has overlap O (original samples, a multiple
of the largest decimation). After chunk k has delivered samples [T, T+n), the
outputs of range r are the global decimated indices j with
j*d_r in [max(0, T-O), max(0, T+n-O)); whole-run output is the union.

Parity status: every function here is pinned by tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdd_oracle.so")
_lock = threading.Lock()
_lib = None

CAND_DTYPE = np.dtype([("trial", "<i4"), ("range", "<i4"), ("t_start", "<i8"), ("width", "<i4"),
                       ("pad", "<i4"), ("snr", "<f8")])


def build(force: bool = False) -> str:
    """Compile dd_oracle.c (gcc -O2 -fopenmp -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, f64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.or_shift_table.restype = ctypes.c_int
            lib.or_shift_table.argtypes = [vp, i32, f64, f64, f64, i32, i32, vp]
            lib.or_delay_seconds.restype = None
            lib.or_delay_seconds.argtypes = [vp, i32, f64, vp]
            lib.or_decimate.restype = ctypes.c_int
            lib.or_decimate.argtypes = [vp, i64, i64, i32, i32, i64, i64, vp]
            lib.or_dedisperse.restype = ctypes.c_int
            lib.or_dedisperse.argtypes = [vp, i64, i64, i32, vp, vp, i32, i64, i64, vp]
            lib.or_moments.restype = None
            lib.or_moments.argtypes = [vp, i64, vp, vp, vp]
            lib.or_sps.restype = ctypes.c_int64
            lib.or_sps.argtypes = [vp, i32, i64, vp, i32, i32, i64, vp, i32, i32, f64, vp, i64]
            lib.or_clipped_moments.restype = None
            lib.or_clipped_moments.argtypes = [vp, i64, i32, f64, i32, vp, vp, vp, vp]
            lib.or_sps_clipped.restype = ctypes.c_int64
            lib.or_sps_clipped.argtypes = [vp, i32, i64, vp, i32, i32, i64, vp, i32, i32, f64,
                                           f64, i32, vp, i64]
            lib.or_fof.restype = ctypes.c_int64
            lib.or_fof.argtypes = [vp, i64, vp, vp, f64, i64, vp]
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- plan (delay table)

def shift_table(freqs, tsamp: float, dm_start: float, dm_step: float, n_trials: int,
                decimation: int) -> np.ndarray:
    """int32 [n_trials][nchans] delays in decimated samples (dd_oracle.c: or_shift_table)."""
    lib = _load()
    f = _f64(freqs)
    out = np.empty((n_trials, f.size), dtype=np.int32)
    rc = lib.or_shift_table(f.ctypes.data, f.size, float(tsamp), float(dm_start), float(dm_step),
                            int(n_trials), int(decimation), out.ctypes.data)
    if rc != 0:
        raise ValueError("shift does not fit int32")
    return out


def shift_tables(freqs, tsamp: float, ranges) -> list:
    """One table per range; ``ranges`` rows are (dm_start, dm_step, n_trials, decimation)."""
    return [shift_table(freqs, tsamp, r[0], r[1], int(r[2]), int(r[3])) for r in ranges]


def overlap(tables, ranges) -> int:
    """Overlap O in original samples: d_max * ceil(max_r(d_r * max s_r) / d_max).

    Output j of range r reads decimated samples up to j + max s_r, i.e. original
    samples below (j + 1 + max s_r) * d_r, so a chunk must carry d_r * max s_r
    samples of history; rounding up to d_max keeps chunk windows aligned to
    every decimation.
    """
    d_max = max(int(r[3]) for r in ranges)
    need = max(int(r[3]) * int(t.max(initial=0)) for t, r in zip(tables, ranges))
    need = max(need, 0)
    return d_max * ((need + d_max - 1) // d_max)


def delay_seconds(freqs, dm: float) -> np.ndarray:
    """Per-channel dispersion delay (s) relative to the highest frequency."""
    lib = _load()
    f = _f64(freqs)
    out = np.empty(f.size, dtype=np.float64)
    lib.or_delay_seconds(f.ctypes.data, f.size, float(dm), out.ctypes.data)
    return out


def delay_samples(freqs, tsamp: float, dm: float) -> np.ndarray:
    """Per-channel delay rounded to whole samples (for placing injected pulses)."""
    return np.floor(delay_seconds(freqs, dm) / tsamp + 0.5).astype(np.int64)


# ---------------------------------------------------------------- decimation / dedispersion

def decimate(x_tm: np.ndarray, t_in0: int, d: int, j_first: int, n_out: int) -> np.ndarray:
    """Channel-major uint32 [C][n_out]: out[c][j] = sum_k x[(j_first+j)*d + k][c]."""
    lib = _load()
    x = np.ascontiguousarray(x_tm, dtype=np.uint8)
    nsamp, nch = x.shape
    out = np.empty((nch, n_out), dtype=np.uint32)
    rc = lib.or_decimate(x.ctypes.data, int(t_in0), int(nsamp), int(nch), int(d), int(j_first),
                         int(n_out), out.ctypes.data)
    if rc != 0:
        raise ValueError("decimation window outside the input")
    return out


def dedisperse(xd: np.ndarray, base: int, shifts: np.ndarray, trials, j0: int,
               nout: int) -> np.ndarray:
    """int32 [len(trials)][nout]: y[i][j] = sum_c xd[c][j0 + j + s[trial_i][c] - base]."""
    lib = _load()
    xd = np.ascontiguousarray(xd, dtype=np.uint32)
    nch, nd = xd.shape
    sh = np.ascontiguousarray(shifts, dtype=np.int32)
    assert sh.shape[1] == nch
    tr = np.ascontiguousarray(trials, dtype=np.int32)
    y = np.empty((tr.size, max(nout, 0)), dtype=np.int32)
    if tr.size == 0 or nout <= 0:
        return y
    rc = lib.or_dedisperse(xd.ctypes.data, int(base), int(nd), int(nch), sh.ctypes.data,
                           tr.ctypes.data, int(tr.size), int(j0), int(nout), y.ctypes.data)
    if rc != 0:
        raise ValueError("dedispersion index outside the decimated input")
    return y


def moments(y: np.ndarray):
    """(n, S1, S2) of one series with S2 as a Python int (exact)."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.int32)
    s1 = np.zeros(1, np.int64)
    lo = np.zeros(1, np.uint64)
    hi = np.zeros(1, np.uint64)
    lib.or_moments(y.ctypes.data, y.size, s1.ctypes.data, lo.ctypes.data, hi.ctypes.data)
    return y.size, int(s1[0]), (int(hi[0]) << 64) | int(lo[0])


def sps(y: np.ndarray, trial_ids, range_idx: int, d: int, J0: int, widths_dec, block: int,
        threshold: float, cap: int | None = None) -> np.ndarray:
    """Candidates (CAND_DTYPE) of a window of series y [ntr][n]; see or_sps in dd_oracle.c."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.int32)
    ntr, n = y.shape
    tr = np.ascontiguousarray(trial_ids, dtype=np.int32)
    w = np.ascontiguousarray(widths_dec, dtype=np.int32)
    if cap is None:
        cap = max(1, ntr * ((n + block - 1) // block))
    out = np.zeros(cap, dtype=CAND_DTYPE)
    total = lib.or_sps(y.ctypes.data, int(ntr), int(n), tr.ctypes.data, int(range_idx), int(d),
                       int(J0), w.ctypes.data, int(w.size), int(block), float(threshold),
                       out.ctypes.data, int(cap))
    return out[:min(total, cap)]


def clipped_moments(y: np.ndarray, w: int, kappa: float = 3.0, iters: int = 3):
    """(N, T1, T2) of the clipped boxcar series B_w of one series, T2 a Python int (exact);
    see or_clipped_moments in dd_oracle.c."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.int32)
    n1 = np.zeros(1, np.int64)
    t1 = np.zeros(1, np.int64)
    lo = np.zeros(1, np.uint64)
    hi = np.zeros(1, np.uint64)
    lib.or_clipped_moments(y.ctypes.data, y.size, int(w), float(kappa), int(iters),
                           n1.ctypes.data, t1.ctypes.data, lo.ctypes.data, hi.ctypes.data)
    return int(n1[0]), int(t1[0]), (int(hi[0]) << 64) | int(lo[0])


def sps_clipped(y: np.ndarray, trial_ids, range_idx: int, d: int, J0: int, widths_dec,
                block: int, threshold: float, kappa: float = 3.0, iters: int = 3,
                cap: int | None = None) -> np.ndarray:
    """Candidates (CAND_DTYPE) with per-width clipped statistics; see or_sps_clipped."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.int32)
    ntr, n = y.shape
    tr = np.ascontiguousarray(trial_ids, dtype=np.int32)
    w = np.ascontiguousarray(widths_dec, dtype=np.int32)
    if cap is None:
        cap = max(1, ntr * ((n + block - 1) // block))
    out = np.zeros(cap, dtype=CAND_DTYPE)
    total = lib.or_sps_clipped(y.ctypes.data, int(ntr), int(n), tr.ctypes.data, int(range_idx),
                               int(d), int(J0), w.ctypes.data, int(w.size), int(block),
                               float(threshold), float(kappa), int(iters), out.ctypes.data,
                               int(cap))
    return out[:min(total, cap)]


GROUP_DTYPE = np.dtype([("rep", "<i8"), ("members", "<i8"), ("dm_lo", "<f8"), ("dm_hi", "<f8"),
                        ("t_lo", "<i8"), ("t_hi", "<i8")])


def candidate_dm(cands: np.ndarray, ranges) -> np.ndarray:
    """DM of each candidate: dm_start + trial * dm_step of its range (FP64, as the delay table)."""
    start = np.array([float(r[0]) for r in ranges])
    step = np.array([float(r[1]) for r in ranges])
    r = cands["range"].astype(np.int64)
    return start[r] + cands["trial"].astype(np.float64) * step[r]


def fof(cands: np.ndarray, ranges, dm_link: float, t_link: int):
    """Friends-of-friends groups of candidates (see or_fof): per candidate the smallest index of
    its group, and one GROUP_DTYPE record per group, in order of that index: its
    representative (the largest SNR; ties to the smaller index), member count, DM extent and the
    extent [t_lo, t_hi] of its boxcars in original samples."""
    lib = _load()
    c = np.ascontiguousarray(cands, dtype=CAND_DTYPE)
    start = _f64([float(r[0]) for r in ranges])
    step = _f64([float(r[1]) for r in ranges])
    label = np.empty(c.size, dtype=np.int64)
    if c.size:
        lib.or_fof(c.ctypes.data, c.size, start.ctypes.data, step.ctypes.data, float(dm_link),
                   int(t_link), label.ctypes.data)
    dm = candidate_dm(c, ranges)
    groups = []
    for g in sorted(set(label.tolist())):
        idx = np.flatnonzero(label == g)
        rep = int(idx[0])
        for k in idx[1:]:
            if c["snr"][k] > c["snr"][rep]:
                rep = int(k)
        groups.append((rep, idx.size, dm[idx].min(), dm[idx].max(), int(c["t_start"][idx].min()),
                       int((c["t_start"][idx] + c["width"][idx] - 1).max())))
    return label, np.array(groups, dtype=GROUP_DTYPE)


def widths_for_range(widths, d: int) -> np.ndarray:
    """Decimated widths searched in a range of decimation d (READING: w >= d, w % d == 0)."""
    return np.array([w // d for w in widths if w >= d and w % d == 0], dtype=np.int32)


# ---------------------------------------------------------------- chunk bookkeeping + driver

def chunk_windows(chunk_sizes, O: int):
    """Per chunk: (T, n, lo, hi) -- samples [T, T+n) arrive; outputs cover [lo, hi) original."""
    out = []
    T = 0
    for n in chunk_sizes:
        lo, hi = max(0, T - O), max(0, T + n - O)
        out.append((T, n, lo, hi))
        T += n
    return out


def run(x_tm: np.ndarray, freqs, tsamp: float, ranges, widths, threshold: float, block: int,
        chunk_sizes, trials=None, want_series: bool = True):
    """Dedisperse + search the whole input chunk by chunk.

    ``x_tm`` is the time-major uint8 filterbank of all samples (global sample 0 first).
    ``trials``: optional list (per range) of trial indices to compute (default all).
    Returns dict(O=..., tables=..., chunks=[{range: {'J0','series','cands','moments'}}]).
    """
    tables = shift_tables(freqs, tsamp, ranges)
    O = overlap(tables, ranges)
    res = {"O": O, "tables": tables, "chunks": []}
    for (T, n, lo, hi) in chunk_windows(chunk_sizes, O):
        per = {}
        for r, (rng, tab) in enumerate(zip(ranges, tables)):
            d = int(rng[3])
            tr = np.arange(tab.shape[0]) if trials is None else np.asarray(trials[r])
            J0, J1 = lo // d, hi // d
            nout = J1 - J0
            if nout > 0:
                smax = int(tab.max(initial=0))
                xd = decimate(x_tm, 0, d, J0, nout + smax)
                y = dedisperse(xd, J0, tab, tr, J0, nout)
            else:
                y = np.zeros((tr.size, 0), dtype=np.int32)
            wd = widths_for_range(widths, d)
            cands = sps(y, tr, r, d, J0, wd, block, threshold) if nout > 0 else \
                np.zeros(0, dtype=CAND_DTYPE)
            mom = [moments(y[k]) for k in range(tr.size)] if nout > 0 else []
            per[r] = {"J0": J0, "series": y if want_series else None, "cands": cands,
                      "moments": mom, "trials": tr}
        res["chunks"].append(per)
    return res
