"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names the plausible mistake it is there to catch. Sources: the
textbook dispersion law (tests/golden/dispersion_delay.txt), exact rational
arithmetic, closed forms of the boxcar SNR, invariants of a brute-force sum,
Gaussian statistics, and recovery of injected dispersed pulses.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from synth import configs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ delay table

def test_delay_matches_textbook_values():
    """Catches a wrong constant, f^-1 instead of f^-2, or a wrong reference frequency."""
    rows = np.loadtxt(os.path.join(GOLDEN, "dispersion_delay.txt"), comments="#")
    for dm, flo, fhi, want in rows:
        got = oracle.delay_seconds([fhi, flo], dm)
        assert got[0] == 0.0
        assert got[1] == pytest.approx(want, rel=1e-9)


def _exact_shift(f, fref, dm_start, dm_step, i, tsamp, d):
    # exact rational evaluation of floor(k*DM*(f^-2 - fref^-2)/(tsamp*d) + 1/2) from the same doubles
    k = Fraction(4148.808)
    dm = Fraction(dm_start) + i * Fraction(dm_step)
    tau = k * dm * (1 / Fraction(f) ** 2 - 1 / Fraction(fref) ** 2)
    x = tau / (Fraction(tsamp) * d) + Fraction(1, 2)
    return math.floor(x), x - math.floor(x)


@pytest.mark.parametrize("d", [1, 2, 8])
def test_shift_rounding_against_exact_rationals(d):
    """Catches truncation instead of round-half-up, or forgetting the decimation factor."""
    w = configs.mid(nsamp=1 << 14)
    f = w.freqs()[::97]
    tab = oracle.shift_table(f, w.tsamp, 3.0, 0.7, 40, d)
    checked = 0
    for i in range(0, 40, 3):
        for c in range(f.size):
            want, frac = _exact_shift(f[c], f.max(), 3.0, 0.7, i, w.tsamp, d)
            if min(frac, 1 - frac) < 1e-9:
                continue  # within rounding noise of a half-way point
            assert tab[i, c] == want, (i, c)
            checked += 1
    assert checked > 400


def test_shift_structure():
    """Zero at DM 0 and at the top channel, non-negative, monotone in DM and in 1/f^2."""
    w = configs.tiny()
    tab = oracle.shift_table(w.freqs(), w.tsamp, 0.0, 1.0, 401, 1)
    assert (tab[0] == 0).all()
    assert (tab[:, 0] == 0).all()  # channel 0 is the highest frequency
    assert (tab >= 0).all()
    assert (np.diff(tab, axis=0) >= 0).all()
    assert (np.diff(tab, axis=1) >= 0).all()  # frequencies descend with channel index
    # worked by hand: 4.148808e3 s MHz^2 * DM * (1/1401.5625^2 - 1/1500^2) MHz^-2 / 64 us
    #   DM 300 -> 1256.75 samples, DM 400 -> 1675.67 samples (the tiny workload's overlap)
    assert tab[300, 63] == 1257
    assert tab[400, 63] == 1676


def test_overlap_rule():
    """O covers the largest delay of every range, is a multiple of d_max, and is minimal."""
    w = configs.mid(nsamp=1 << 14)
    f = w.freqs()[::64]
    rr = w.ranges_array()
    tabs = oracle.shift_tables(f, w.tsamp, rr)
    O = oracle.overlap(tabs, rr)
    need = max(int(r[3]) * int(t.max()) for t, r in zip(tabs, rr))
    assert O % 8 == 0 and O >= need and O - 8 < need


# ------------------------------------------------------------------ decimation

def test_decimation_sum_and_cascade():
    """Catches mean instead of sum, misaligned windows, or dropped samples."""
    rng = np.random.default_rng(1)
    x = rng.integers(0, 256, size=(512, 5), dtype=np.uint8)
    for d in (1, 2, 4, 8, 16):
        full = oracle.decimate(x, 0, d, 0, 512 // d)
        ref = x.astype(np.uint32).reshape(512 // d, d, 5).sum(axis=1).T
        np.testing.assert_array_equal(full, ref)
        assert full.sum() == x.astype(np.int64).sum()
    two = oracle.decimate(x, 0, 2, 0, 256).T
    four = two.reshape(128, 2, 5).sum(axis=1).T
    np.testing.assert_array_equal(four, oracle.decimate(x, 0, 4, 0, 128))
    # sub-window with an input offset
    part = oracle.decimate(x[64:], 64, 4, 20, 50)
    np.testing.assert_array_equal(part, oracle.decimate(x, 0, 4, 0, 128)[:, 20:70])


# ------------------------------------------------------------------ dedispersion

def _tiny_problem(nch=8, nsamp=512, d=1, seed=3):
    freqs = 1500.0 - 12.5 * np.arange(nch)
    tsamp = 64e-6
    tab = oracle.shift_table(freqs, tsamp, 0.0, 3.0, 12, d)  # max delay ~120 samples
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 256, size=(nsamp, nch), dtype=np.uint8)
    return freqs, tsamp, tab, x


def test_dm_zero_is_channel_sum():
    """Trial DM=0 must be the plain sum over channels (catches channel/time transposition)."""
    freqs, tsamp, tab, x = _tiny_problem()
    xd = oracle.decimate(x, 0, 1, 0, 512)
    y = oracle.dedisperse(xd, 0, tab, [0], 0, 300)
    np.testing.assert_array_equal(y[0], x[:300].astype(np.int64).sum(axis=1))


def test_constant_input():
    """A constant k gives C*k*d in every output (catches dropped channels or samples)."""
    freqs, tsamp, tab, _ = _tiny_problem(d=4)
    x = np.full((512, 8), 7, dtype=np.uint8)
    xd = oracle.decimate(x, 0, 4, 0, 128)
    y = oracle.dedisperse(xd, 0, tab, range(12), 0, 128 - int(tab.max()))
    assert (y == 8 * 7 * 4).all()


def test_impulse_lands_once_per_trial():
    """A single sample at (c, t0) appears exactly once per trial, at j = t0/d - s[i][c]."""
    for d in (1, 2):
        freqs, tsamp, tab, _ = _tiny_problem(d=d)
        c0, t0 = 5, 300
        x = np.zeros((512, 8), dtype=np.uint8)
        x[t0, c0] = 200
        nd = 512 // d
        xd = oracle.decimate(x, 0, d, 0, nd)
        nout = nd - int(tab.max())
        y = oracle.dedisperse(xd, 0, tab, range(12), 0, nout)
        for i in range(12):
            j = t0 // d - tab[i, c0]
            assert y[i].sum() == 200
            assert y[i, j] == 200


def test_brute_force_and_linearity():
    """Second naive loop on a tiny input; dedispersion is linear in the data."""
    freqs, tsamp, tab, x = _tiny_problem(nch=4, nsamp=128, d=2)
    xd = oracle.decimate(x, 0, 2, 0, 64)
    nout = 64 - int(tab.max())
    y = oracle.dedisperse(xd, 0, tab, range(12), 0, nout)
    for i in range(12):
        for j in range(nout):
            s = 0
            for c in range(4):
                t = 2 * (j + int(tab[i, c]))
                s += int(x[t, c]) + int(x[t + 1, c])
            assert y[i, j] == s
    _, _, _, x2 = _tiny_problem(nch=4, nsamp=128, d=2, seed=9)
    x2 = x2 // 2
    xa = (x // 2)
    ya = oracle.dedisperse(oracle.decimate(xa, 0, 2, 0, 64), 0, tab, range(12), 0, nout)
    yb = oracle.dedisperse(oracle.decimate(x2, 0, 2, 0, 64), 0, tab, range(12), 0, nout)
    yab = oracle.dedisperse(oracle.decimate(xa + x2, 0, 2, 0, 64), 0, tab, range(12), 0, nout)
    np.testing.assert_array_equal(yab, ya + yb)


def test_moments_exact():
    rng = np.random.default_rng(4)
    y = rng.integers(0, 2**31 - 1, size=5000, dtype=np.int64).astype(np.int32)
    n, s1, s2 = oracle.moments(y)
    assert n == 5000
    assert s1 == sum(int(v) for v in y)
    assert s2 == sum(int(v) * int(v) for v in y)
    assert s2 >= 2**64  # exercises the 128-bit carry


# ------------------------------------------------------------------ single-pulse search

def test_sps_constant_series_has_no_candidates():
    y = np.full((1, 1000), 12345, dtype=np.int32)
    c = oracle.sps(y, [0], 0, 1, 0, [1, 2, 4], 32, -1e9)
    assert c.size == 0


def test_sps_delta_closed_form():
    """A single delta: SNR = sqrt(n-1) at width 1 (catches wrong variance normalisation)."""
    n, j0, h = 1000, 517, 40
    y = np.zeros((1, n), dtype=np.int32)
    y[0, j0] = h
    c = oracle.sps(y, [7], 2, 4, 100, [1, 2, 4, 8], 32, 5.0)
    assert c.size == 1
    assert c["snr"][0] == pytest.approx(math.sqrt(n - 1), rel=1e-12)
    assert c["width"][0] == 4  # one decimated sample of a x4 range
    assert c["t_start"][0] == (100 + j0) * 4
    assert c["trial"][0] == 7 and c["range"][0] == 2


def test_sps_boxcar_closed_form_and_width():
    """A top-hat of W ones: best width W with SNR sqrt(n-W) (catches a missing sqrt(w))."""
    n, W, start = 4096, 16, 1000
    y = np.zeros((1, n), dtype=np.int32)
    y[0, start:start + W] = 1
    c = oracle.sps(y, [0], 0, 1, 0, [1, 2, 4, 8, 16, 32], 32, 10.0)
    best = c[np.argmax(c["snr"])]
    assert best["width"] == W and best["t_start"] == start
    assert best["snr"] == pytest.approx(math.sqrt(n - W), rel=1e-12)
    # widths 8 and 32 score sqrt(n-W)/sqrt(2) at best
    assert (c["snr"] <= math.sqrt(n - W) + 1e-9).all()


def test_sps_ties_and_ragged_block():
    """Equal peaks in a block go to the earlier sample; the ragged last block is searched."""
    n = 100  # blocks [0,32) [32,64) [64,96) [96,100)
    y = np.zeros((1, n), dtype=np.int32)
    y[0, 40] = y[0, 50] = 9
    y[0, 98] = 9
    c = oracle.sps(y, [0], 0, 1, 0, [1], 32, 3.0)
    assert list(c["t_start"]) == [40, 98]
    # a trailing boxcar needs w-1 samples of history inside the window
    y2 = np.zeros((1, 64), dtype=np.int32)
    y2[0, 0] = 50
    c2 = oracle.sps(y2, [0], 0, 1, 0, [4], 32, -1e9)
    assert c2["t_start"].min() >= 0


def test_sps_gaussian_noise_statistics():
    """Boxcar SNR of white Gaussian noise is N(0,1): P(SNR > 3) = 1.35e-3 at every width."""
    rng = np.random.default_rng(11)
    n = 1 << 18
    y = np.rint(rng.normal(1e5, 300.0, size=(1, n))).astype(np.int32)
    for w in (1, 16):
        c = oracle.sps(y, [0], 0, 1, 0, [w], 1, 3.0)
        frac = c.size / (n - w + 1)
        assert frac == pytest.approx(0.00135, rel=0.25), (w, frac)


# ------------------------------------------------------------------ whole pipeline

def test_chunk_windows_tile_the_output():
    wins = oracle.chunk_windows([4096] * 5 + [1024], 1680)
    assert wins[0][2] == 0
    for a, b in zip(wins, wins[1:]):
        assert a[3] == b[2]
    assert wins[-1][3] == 5 * 4096 + 1024 - 1680


def test_injected_pulses_recovered_tiny():
    """Pulses at DM 50/150/300 (+24 per channel, 16 samples) come out at their DM and time."""
    w = configs.tiny()
    f = w.freqs()
    x = w.generate(lambda dm: oracle.delay_samples(f, w.tsamp, dm))
    res = oracle.run(x, f, w.tsamp, w.ranges_array(), w.widths, w.threshold, 32, [w.nsamp],
                     want_series=False)
    cands = res["chunks"][0][0]["cands"]
    design = 24.0 * math.sqrt(16 * 64) / 16.0
    for p in w.pulses:
        near = cands[np.abs(cands["t_start"] - p.t_ref) <= p.width + 32]
        assert near.size > 0
        top = near[np.argmax(near["snr"])]
        assert abs(top["trial"] - p.dm) <= 1.0
        assert p.width / 2 <= top["width"] <= p.width * 2
        assert top["snr"] >= 0.7 * design
    # away from the pulses the noise stays below 6 sigma
    far = np.ones(cands.size, bool)
    for p in w.pulses:
        far &= np.abs(cands["t_start"] - p.t_ref) > 2000
    assert far.sum() <= 3


def test_generator_is_chunk_consistent():
    """Any sub-range of samples is byte-identical to the same rows of a longer generation."""
    w = configs.tiny()
    f = w.freqs()
    arr = lambda dm: oracle.delay_samples(f, w.tsamp, dm)
    full = w.generate(arr, nsamp=30000)
    part = w.generate(arr, t0=8000, nsamp=20000)
    np.testing.assert_array_equal(full[8000:28000], part)
    v = full.astype(np.float64)
    assert abs(v.mean() - 128.0) < 0.2 and abs(v.std() - 16.0) < 0.3
