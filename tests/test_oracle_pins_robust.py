"""Pins of the oracle's robust search statistics and candidate grouping (Sec. 2.2 readings).

The paper names the SPDT estimators without defining them; the oracle reads them as iterative
kappa-sigma clipping of each boxcar-filtered series, and groups candidates friends-of-friends
over DM and time. These tests tie both to facts outside the oracle: closed forms of clipped
moments and SNRs, the variance of a clipped Gaussian (a textbook formula), and connected
components computed by networkx. Each names the mistake it catches.
"""
import math

import numpy as np
import pytest

import oracle

CAND = oracle.CAND_DTYPE


# ------------------------------------------------------------------ clipped moments

def _alternating(n, lo=99, hi=101):
    y = np.empty(n, dtype=np.int32)
    y[0::2], y[1::2] = lo, hi
    return y


def test_clipping_removes_an_outlier_exactly():
    """Catches no clipping step, clipping on one side only, or a bound that keeps the outlier:
    1000 samples alternating 99/101 plus a spike of 10^6. Unclipped: every value; after one or
    more steps: exactly the alternating samples (N 1000, T1 100000, T2 500 x (99^2 + 101^2))."""
    y = np.concatenate([_alternating(1000), np.array([10 ** 6], np.int32)])
    assert oracle.clipped_moments(y, 1, 3.0, 0) == (1001, 100000 + 10 ** 6,
                                                    500 * (99 ** 2 + 101 ** 2) + 10 ** 12)
    for iters in (1, 3):
        assert oracle.clipped_moments(y, 1, 3.0, iters) == (1000, 100000,
                                                            500 * (99 ** 2 + 101 ** 2))


def test_clipped_moments_of_boxcar_sums_brute_force():
    """Catches an off-by-one in the boxcar positions (j >= w - 1) or in the width: on tiny series
    with no clipping, (N, T1, T2) equal the count, sum and sum of squares of every w-sample
    window sum, computed here from slices."""
    rng = np.random.default_rng(11)
    for n in (1, 5, 17, 64):
        y = rng.integers(0, 2 ** 20, n).astype(np.int32)
        for w in (1, 2, 5, 16, 64):
            sums = [int(y[j - w + 1:j + 1].astype(np.int64).sum()) for j in range(w - 1, n)]
            want = (len(sums), sum(sums), sum(s * s for s in sums))
            assert oracle.clipped_moments(y, w, 3.0, 0) == want, (n, w)


def _truncated_sigma(kappa, iters):
    """Deviation (in units of sigma) after `iters` clipping steps of a Gaussian: a normal
    variable restricted to |x| <= a has variance 1 - 2 a phi(a) / (2 Phi(a) - 1)."""
    s = 1.0
    for _ in range(iters):
        a = kappa * s
        phi = math.exp(-a * a / 2) / math.sqrt(2 * math.pi)
        big = math.erf(a / math.sqrt(2))  # 2 Phi(a) - 1
        s = math.sqrt(1 - 2 * a * phi / big)
    return s


@pytest.mark.parametrize("kappa,iters", [(3.0, 1), (3.0, 3), (2.0, 3)])
def test_clipped_sigma_of_gaussian_noise(kappa, iters):
    """Catches a wrong kappa, a wrong number of steps or a sample (n-1) variance: 2^22 Gaussian
    samples of sigma 1000 clip to the truncated-normal deviation within 0.06% (the statistical
    error is about 0.035%), which separates one step from three at kappa 3 (0.17% apart)."""
    rng = np.random.default_rng(12)
    y = np.rint(rng.normal(0.0, 1000.0, 1 << 22)).astype(np.int32) + 10 ** 6
    N, T1, T2 = oracle.clipped_moments(y, 1, kappa, iters)
    sd = math.sqrt(N * T2 - T1 * T1) / N
    assert sd / 1000.0 == pytest.approx(_truncated_sigma(kappa, iters), rel=6e-4)
    assert T1 / N == pytest.approx(10 ** 6, abs=3.0)
    other = 0 if iters == 1 else 1
    assert abs(_truncated_sigma(kappa, iters) - _truncated_sigma(kappa, other)) > 1.5e-3


def test_clipped_search_closed_form():
    """Catches SNRs normalised by unclipped statistics: 4096 samples alternating 99/101 with a
    delta of 100 + h inserted. Clipping removes the delta, leaving N 4096, mean 100 and deviation
    exactly 1 (N T2 - T1^2 = 4096^2), so the delta's w = 1 SNR is h exactly; every 2-sample
    boxcar of the rest sums to 200 (no variance: width 2 gives nothing)."""
    h, j0 = 5000, 2001
    alt = _alternating(4096)
    y = np.concatenate([alt[:j0], np.array([100 + h], np.int32), alt[j0:]])
    c = oracle.sps_clipped(y[None, :], [7], 0, 1, 0, np.array([1, 2], np.int32), 32, 6.0)
    assert c.size == 1
    assert (int(c["trial"][0]), int(c["t_start"][0]), int(c["width"][0])) == (7, j0, 1)
    assert float(c["snr"][0]) == h
    # without clipping, the same delta scores far lower
    c0 = oracle.sps_clipped(y[None, :], [7], 0, 1, 0, np.array([1], np.int32), 32, 6.0, iters=0)
    assert c0.size == 1 and float(c0["snr"][0]) < 70


def test_clipped_search_is_shift_invariant():
    """Catches a mean term dropped from the numerator: adding a constant to every sample leaves
    every candidate and SNR unchanged (noise with pulses, values far from the clip bounds)."""
    rng = np.random.default_rng(13)
    y = rng.normal(0.0, 30.0, (3, 8192))
    y[:, 4000:4016] += 25.0
    y = np.rint(y).astype(np.int32) + 1000
    wd = np.array([1, 4, 16, 64], np.int32)
    a = oracle.sps_clipped(y, [0, 1, 2], 0, 1, 0, wd, 32, 5.0)
    b = oracle.sps_clipped(y + 12345, [0, 1, 2], 0, 1, 0, wd, 32, 5.0)
    assert a.size > 0
    np.testing.assert_array_equal(a[["trial", "t_start", "width"]], b[["trial", "t_start", "width"]])
    np.testing.assert_allclose(a["snr"], b["snr"], rtol=1e-12)


# ------------------------------------------------------------------ friends of friends

def _cands(rows):
    """rows: (range, trial, t_start, width, snr)."""
    c = np.zeros(len(rows), dtype=CAND)
    for k, (r, t, ts, w, s) in enumerate(rows):
        c[k] = (t, r, ts, w, 0, s)
    return c


RANGES = [(0.0, 0.5, 100, 1), (50.0, 1.0, 100, 2)]


def test_fof_chain_is_one_group():
    """Catches a pairwise-only grouping: a-b and b-c are friends (DM 0.5 apart, the link), a-c
    are not (DM 1.0 apart), yet all three form one group; a fourth candidate far away in time
    stays alone."""
    c = _cands([(0, 10, 1000, 4, 7.0), (0, 11, 1002, 4, 9.0), (0, 12, 1004, 4, 8.0),
                (0, 11, 50000, 4, 6.5)])
    label, g = oracle.fof(c, RANGES, dm_link=0.5, t_link=0)
    assert label.tolist() == [0, 0, 0, 3]
    assert g["rep"].tolist() == [1, 3] and g["members"].tolist() == [3, 1]
    assert (g["dm_lo"][0], g["dm_hi"][0]) == (5.0, 6.0)
    assert (int(g["t_lo"][0]), int(g["t_hi"][0])) == (1000, 1007)


def test_fof_link_lengths_are_inclusive():
    """Catches < instead of <= at the linking lengths: DM exactly dm_link apart and a later
    boxcar starting exactly t_link samples after the earlier one's last sample are friends; one
    DM step or one sample more is not."""
    # boxcars [100, 103] and [108, 111]: the second starts 5 samples after the first's last
    base = (0, 20, 100, 4, 8.0)
    near = [(0, 21, 108, 4, 7.0)]
    assert oracle.fof(_cands([base] + near), RANGES, 0.5, 5)[0].tolist() == [0, 0]
    assert oracle.fof(_cands([base] + near), RANGES, 0.5, 4)[0].tolist() == [0, 1]
    assert oracle.fof(_cands(near + [base]), RANGES, 0.5, 5)[0].tolist() == [0, 0]
    assert oracle.fof(_cands([base, (0, 22, 100, 4, 7.0)]), RANGES, 0.5, 0)[0].tolist() == [0, 1]
    assert oracle.fof(_cands([base, (0, 22, 100, 4, 7.0)]), RANGES, 1.0, 0)[0].tolist() == [0, 0]


def test_fof_across_ranges_uses_each_ranges_dm():
    """Catches DM taken from the trial index alone: range 1 trial 0 is DM 50, next to range 0's
    trial 99 (DM 49.5), not to range 0's trial 0."""
    c = _cands([(0, 99, 500, 8, 7.0), (1, 0, 502, 8, 9.0), (0, 0, 500, 8, 6.0)])
    label, g = oracle.fof(c, RANGES, 0.5, 0)
    assert label.tolist() == [0, 0, 2]
    assert g["rep"].tolist() == [1, 2]


def test_fof_matches_networkx_components():
    """Catches an incomplete relaxation: on random candidate sets the groups are the connected
    components of the friendship graph as networkx computes them, and the representative is the
    member with the largest SNR (ties: the smaller index)."""
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(14)
    for trial in range(20):
        n = int(rng.integers(1, 120))
        rows = [(int(rng.integers(0, 2)), int(rng.integers(0, 40)), int(rng.integers(0, 3000)),
                 int(2 ** rng.integers(0, 6)), float(rng.integers(60, 90)) / 10) for _ in range(n)]
        c = _cands(rows)
        label, g = oracle.fof(c, RANGES, 1.0, 16)
        dm = oracle.candidate_dm(c, RANGES)
        G = nx.Graph()
        G.add_nodes_from(range(n))
        for a in range(n):
            for b in range(a + 1, n):
                ta, wa = int(c["t_start"][a]), int(c["width"][a])
                tb, wb = int(c["t_start"][b]), int(c["width"][b])
                if abs(dm[a] - dm[b]) <= 1.0 and ta <= tb + wb - 1 + 16 and tb <= ta + wa - 1 + 16:
                    G.add_edge(a, b)
        comps = sorted(sorted(cc) for cc in nx.connected_components(G))
        assert sorted(g["members"].tolist()) == sorted(len(cc) for cc in comps)
        for cc in comps:
            assert all(label[k] == cc[0] for k in cc)
            rep = max(cc, key=lambda k: (c["snr"][k], -k))
            row = g[np.flatnonzero(g["rep"] == rep)]
            assert row.size == 1 and int(row["members"][0]) == len(cc)
