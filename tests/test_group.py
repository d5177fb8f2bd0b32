"""dd_group_candidates (host code of the library) against the oracle's friends-of-friends
grouping: labels and group records equal on random candidate sets, on candidate lists of a real
search, and at the linking lengths' edges. Runs without a GPU."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2101_00941_gb300 as dd

RANGES = [(0.0, 0.5, 100, 1), (50.0, 1.0, 100, 2), (150.0, 2.5, 60, 4)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    dd.build()
    dd.lib()


def _random_cands(rng, n):
    c = np.zeros(n, dtype=dd.CAND_DTYPE)
    c["range"] = rng.integers(0, len(RANGES), n)
    c["trial"] = [int(rng.integers(0, RANGES[r][2])) for r in c["range"]]
    c["t_start"] = rng.integers(0, 20000, n)
    c["width"] = 2 ** rng.integers(0, 8, n)
    c["snr"] = rng.integers(60, 200, n) / 10.0  # many ties
    return c[np.lexsort((c["width"], c["t_start"], c["trial"], c["range"]))]


def _same(c, dm_link, t_link):
    lab, g = dd.dd_group_candidates(c, RANGES, dm_link, t_link)
    want_lab, want_g = oracle.fof(c, RANGES, dm_link, t_link)
    np.testing.assert_array_equal(lab, want_lab)
    assert g.size == want_g.size
    for f in ("rep", "members", "t_lo", "t_hi"):
        np.testing.assert_array_equal(g[f], want_g[f])
    np.testing.assert_array_equal(g["dm_lo"], want_g["dm_lo"])
    np.testing.assert_array_equal(g["dm_hi"], want_g["dm_hi"])
    return g.size


@pytest.mark.parametrize("dm_link,t_link", [(0.0, 0), (0.5, 0), (1.0, 16), (5.0, 200)])
def test_groups_equal_the_oracles_on_random_sets(dm_link, t_link):
    rng = np.random.default_rng(21)
    for n in (0, 1, 2, 50, 400):
        _same(_random_cands(rng, n), dm_link, t_link)


def test_groups_of_a_search_result():
    """Candidates the oracle's search finds in noise with dispersed pulses, grouped alike."""
    rng = np.random.default_rng(22)
    y = rng.normal(0.0, 20.0, (40, 4096))
    for t in range(15, 25):  # a pulse seen over ten neighbouring trials
        y[t, 2000:2008] += 30.0
    y = np.rint(y).astype(np.int32) + 5000
    c = oracle.sps(y, np.arange(40), 0, 1, 0, np.array([1, 2, 4, 8], np.int32), 32, 4.0)
    c = c[np.lexsort((c["width"], c["t_start"], c["trial"], c["range"]))]
    assert _same(c, 0.5, 8) < c.size  # the pulse's candidates merge


def test_inclusive_link_edges():
    c = np.zeros(2, dtype=dd.CAND_DTYPE)
    c[0] = (20, 0, 100, 4, 0, 8.0)
    c[1] = (21, 0, 108, 4, 0, 7.0)
    assert dd.dd_group_candidates(c, RANGES, 0.5, 5)[0].tolist() == [0, 0]
    assert dd.dd_group_candidates(c, RANGES, 0.5, 4)[0].tolist() == [0, 1]
    assert dd.dd_group_candidates(c, RANGES, 0.49, 5)[0].tolist() == [0, 1]


def test_group_errors():
    c = np.zeros(3, dtype=dd.CAND_DTYPE)
    c["width"] = 1
    c["t_start"] = [0, 10000, 20000]
    with pytest.raises(dd.DDError) as e:
        dd.dd_group_candidates(c, RANGES, -1.0, 0)
    assert e.value.code == dd.DD_ERR_ARG
    bad = c.copy()
    bad["range"][1] = 7
    with pytest.raises(dd.DDError) as e:
        dd.dd_group_candidates(bad, RANGES, 0.5, 0)
    assert e.value.code == dd.DD_ERR_ARG
    # three isolated candidates, room for two groups: DD_ERR_CAP with the true count
    out = np.zeros(2, dtype=dd.GROUP_DTYPE)
    n = ctypes.c_int64()
    rr = (dd.dd_range_t * 3)(*[dd.dd_range_t(*r) for r in RANGES])
    rc = dd.lib().dd_group_candidates(c.ctypes.data, 3, ctypes.addressof(rr), 3, 0.5, 0,
                                      out.ctypes.data, 2, ctypes.byref(n), None)
    assert rc == dd.DD_ERR_CAP and n.value == 3
