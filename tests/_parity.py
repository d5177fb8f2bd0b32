"""Helpers comparing the GPU library (through its C ABI) with the CPU oracle.

Series and moments must be bit-exact. Candidates must match one-to-one per
(range, trial, block) with SNR within SNR_RTOL relative; a block whose oracle
maximum lies within SNR_RTOL of the threshold may appear on either side, and
where the two pick a different (sample, width) inside a block, the GPU's pick
must score within SNR_RTOL of the block maximum (several answers are correct
when SNRs tie to that precision).
"""
from __future__ import annotations

import math

import numpy as np

import oracle

SNR_RTOL = 1e-5


def oracle_trial_snr(y: np.ndarray, j: int, w: int) -> float:
    """SNR of a trailing boxcar of w samples ending at window sample j (exact integers, FP64)."""
    n = y.size
    s1 = int(y.astype(np.int64).sum())
    s2 = int((y.astype(np.int64) ** 2).sum()) if n < 1 << 20 else sum(int(v) * int(v) for v in y)
    v = n * s2 - s1 * s1
    b = int(y[j - w + 1:j + 1].astype(np.int64).sum())
    return (n * b - w * s1) / (math.sqrt(w) * math.sqrt(float(v)))


def compare_candidates(gpu: np.ndarray, ref: np.ndarray, threshold: float, block: int,
                       series_of=None, J0_of=None, d_of=None, trial_snr=oracle_trial_snr):
    """Assert the candidate lists agree (see module doc). Returns the number of matched blocks.
    trial_snr(y, j, w) scores an alternative pick (default: the window-statistics SNR)."""
    def key(c, J0, d):
        wd = int(c["width"]) // d
        jend = int(c["t_start"]) // d + wd - 1 - J0
        return (int(c["range"]), int(c["trial"]), jend // block)

    def index(arr):
        out = {}
        for c in arr:
            r = int(c["range"])
            k = key(c, J0_of(r), d_of(r))
            assert k not in out, f"two candidates in one block: {k}"
            out[k] = c
        return out

    g, o = index(gpu), index(ref)
    tol_thr = SNR_RTOL * max(1.0, abs(threshold))
    for k in set(o) - set(g):
        assert abs(o[k]["snr"] - threshold) <= tol_thr, f"oracle candidate missing on GPU: {o[k]}"
    for k in set(g) - set(o):
        assert abs(g[k]["snr"] - threshold) <= tol_thr, f"GPU candidate not in oracle: {g[k]}"
    for k in set(g) & set(o):
        a, b = g[k], o[k]
        assert a["snr"] == np.float64(b["snr"]) or \
            abs(a["snr"] - b["snr"]) <= SNR_RTOL * abs(b["snr"]), (a, b)
        if (a["t_start"], a["width"]) != (b["t_start"], b["width"]):
            assert series_of is not None, (a, b)
            r, tr = int(a["range"]), int(a["trial"])
            d, J0 = d_of(r), J0_of(r)
            y = series_of(r, tr)
            wd = int(a["width"]) // d
            j = int(a["t_start"]) // d + wd - 1 - J0
            alt = trial_snr(y, j, wd)
            assert abs(alt - b["snr"]) <= SNR_RTOL * abs(b["snr"]), (a, b, alt)
    return len(set(g) & set(o))


def clipped_trial_snr(kappa: float, iters: int):
    """SNR of a trailing boxcar under the clipped per-width statistics (oracle.clipped_moments)."""
    def snr(y: np.ndarray, j: int, w: int) -> float:
        N, T1, T2 = oracle.clipped_moments(y, w, kappa, iters)
        b = int(y[j - w + 1:j + 1].astype(np.int64).sum())
        return (N * b - T1) / math.sqrt(float(N * T2 - T1 * T1))
    return snr


def assert_moments_equal(got, want, what=""):
    """Device moments records (MOMENTS_DTYPE rows) against the oracle's (n, S1, S2) tuples,
    bit for bit: S1 as int64 and S2 as the full 128-bit value."""
    assert len(got) == len(want), what
    for k, (g, (_, s1, s2)) in enumerate(zip(got, want)):
        g_s2 = (int(g["s2hi"]) << 64) | int(g["s2lo"])
        assert int(g["s1"]) == s1 and g_s2 == s2, (what, k, int(g["s1"]), s1, g_s2, s2)


def oracle_chunk(x_tm, freqs, tsamp, ranges, widths, threshold, block, chunk_sizes, trials=None):
    return oracle.run(x_tm, freqs, tsamp, ranges, widths, threshold, block, chunk_sizes,
                      trials=trials)
