"""Host logic of the tiled kernel's plan (no GPU): the plan-time delay-class tables, staging
windows and build work lists, checked against the delay tables they come from.

The delay tables are the oracle's (the GPU builds the same table bit for bit; see the parity
tests), padded to a multiple of 8 channels by repeating the last channel as the library does.
"""
import numpy as np
import pytest

import oracle
from synth import configs
import paper_2101_00941_gb300 as dd


@pytest.fixture(scope="module", autouse=True)
def _built():
    dd.build()
    dd.lib()


def _tables(w):
    tabs = oracle.shift_tables(w.freqs(), w.tsamp, w.ranges_array())
    out = []
    for t in tabs:
        cp = -(-t.shape[1] // 8) * 8
        out.append(np.pad(t, ((0, 0), (0, cp - t.shape[1])), mode="edge").astype(np.int32))
    return out


SHAPES = [(512, 64), (256, 64), (256, 32)]


@pytest.mark.parametrize("tt,trials", SHAPES)
def test_4096_channel_plan(tt, trials):
    w = configs.mid(nsamp=1 << 17)
    for tab, r in zip(_tables(w), w.ranges):
        ok, bad = dd.dd_tiled_plan_check(tab, r.decimation, tt, trials)
        assert (ok, bad) == (1, 0), r


@pytest.mark.parametrize("tt,trials", SHAPES)
def test_8192_channel_plan_edges(tt, trials):
    w = configs.out_of_core(nsamp=1 << 20)
    tabs = _tables(w)
    for k in (0, len(w.ranges) - 1):  # x1 and the widest, x16
        ok, bad = dd.dd_tiled_plan_check(tabs[k], w.ranges[k].decimation, tt, trials)
        assert bad == 0, w.ranges[k]
        # a two-CTA shape must fit half an SM's shared memory: the 64 x 256 tile of this plan's
        # x1 range does not (117 KB), the 32 x 256 tile does
        if k == 0:
            assert ok == (0 if (tt, trials) == (256, 64) else 1)


def test_ragged_channels_and_trial_tiles():
    """1001 channels (padded to 1008) and ranges of 150, 75, 130, 70, 40, 30, 20, 10 trials;
    above x16 the sum of two groups' eight channels does not fit a pair word's 16-bit lanes."""
    ranges = (configs.DMRange(0.0, 0.0625, 150, 1), configs.DMRange(9.375, 0.125, 75, 2),
              configs.DMRange(18.75, 0.15625, 130, 4), configs.DMRange(39.0625, 0.3125, 70, 8),
              configs.DMRange(60.9375, 0.625, 40, 16), configs.DMRange(85.9375, 1.25, 30, 32),
              configs.DMRange(123.4375, 2.5, 20, 64), configs.DMRange(173.4375, 5.0, 10, 128))
    w = configs.mid(nsamp=1 << 15, nchans=4096, ranges=ranges)
    w.nchans, w.foff = 1001, -300.0 / 1024
    for tab, r in zip(_tables(w), w.ranges):
        for tt, trials in SHAPES:
            ok, bad = dd.dd_tiled_plan_check(tab, r.decimation, tt, trials)
            assert bad == 0
            assert ok == (1 if r.decimation <= 16 else 0), (r, tt, trials)


def test_odd_group_count():
    """993 channels: padded to 1000, 125 eight-channel groups, so the last stage holds one."""
    ranges = (configs.DMRange(0.0, 0.0625, 100, 1), configs.DMRange(6.25, 0.125, 50, 2))
    w = configs.mid(nsamp=1 << 15, nchans=4096, ranges=ranges)
    w.nchans, w.foff = 993, -300.0 / 1024
    for tab, r in zip(_tables(w), w.ranges):
        assert tab.shape[1] == 1000
        assert dd.dd_tiled_plan_check(tab, r.decimation, 512) == (1, 0), r


def test_coarse_channels_and_bad_tables_are_refused():
    w = configs.tiny()  # 64 coarse channels: up to 63 delay classes per group
    (tab,) = _tables(w)
    assert dd.dd_tiled_plan_check(tab, 1, 512) == (0, 0)
    mid = _tables(configs.mid(nsamp=1 << 17))[0].copy()
    mid[10, 5] = mid[11, 5] + 1  # a delay that decreases with DM
    assert dd.dd_tiled_plan_check(mid, 1, 512) == (0, 0)
    with pytest.raises(dd.DDError):
        dd.dd_tiled_plan_check(np.zeros((4, 12), np.int32), 1, 512)  # 12 channels: not padded
