"""The search fused into the dedispersion kernel (dd_fuse_search) against the CPU oracle and the
plain path.

The fused form records per (trial, width, peak block) the block's largest boxcar sum and its
earliest sample while each tile is still on chip; a CTA walks a segment of time tiles and reads
the previous tile's prefix sums, and boxcars that start before a segment are completed by a
second pass. The tests cover segments of one tile (every boundary completed by that pass) and of
several tiles (the walking history), ragged windows, peak blocks 1, 8 and 32, odd widths, widths
up to 512 samples, tile prefix sums that wrap 2^32, the kept series, and the call's error paths.
With a threshold of -1e30 every block yields a candidate, so those cases compare every block's
maximum, not only the blocks above a detection threshold.
"""
import numpy as np
import pytest

import oracle
from synth import configs

torch = pytest.importorskip("torch")
import paper_2101_00941_gb300 as dd  # noqa: E402
from _gpu_check import _arrivals, oracle_candidates_match  # noqa: E402
from _parity import assert_moments_equal, compare_candidates  # noqa: E402

pytestmark = pytest.mark.gpu

EVERY_BLOCK = -1e30


@pytest.fixture(scope="module", autouse=True)
def _built():
    dd.build()
    dd.lib()


def _tiled(nchans, nsamp, ranges, index, chunk_len=1 << 16, npulses=8):
    """Channel width and DM steps in the tiled kernel's regime (as the 4096-channel workload):
    nchans channels from 1450 MHz down by 300/1024 MHz, 64 us."""
    w = configs.mid(nsamp=nsamp, chunk_len=chunk_len, n_streams=2, npulses=npulses, nchans=4096,
                    ranges=ranges, index=index)
    w.nchans = nchans
    w.foff = -300.0 / 1024
    w.pulses = tuple(configs.PulseSpec(p.dm * 0.05, min(p.t_ref, nsamp - 8000), p.width,
                                       p.amp * 3.0) for p in w.pulses)
    return w


def _workload(nsamp=1 << 17, widths=(1, 2, 3, 4, 8, 16, 31, 64, 128, 256, 512)):
    """512 channels: a x1 range of 256 trials (4 trial tiles: with 128 time tiles per
    65536-sample window the fused launch walks segments of 4 tiles), x2 and x4 ranges of 100 and
    70 trials (one or two trial tiles: segments of one tile)."""
    ranges = (configs.DMRange(0.0, 0.0625, 256, 1), configs.DMRange(16.0, 0.125, 100, 2),
              configs.DMRange(28.5, 0.15625, 70, 4))
    w = _tiled(512, nsamp, ranges, 11)
    w.widths = tuple(widths)
    return w


def _run(w, x, sizes, L, fuse, block=32, threshold=None, keep=False, streams=2, series=False):
    thr = w.threshold if threshold is None else threshold
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), L, n_streams=streams,
                   max_width=max(w.widths), peak_block=block, max_cands=1 << 23)
    out = []
    try:
        nf = plan.fuse_search(w.widths, keep_series=keep) if fuse else 0
        models = [plan.model(r, L // int(w.ranges[r].decimation)) for r in range(len(w.ranges))]
        T = 0
        for n in sizes:
            seq = plan.run(torch.from_numpy(x[T:T + n]).cuda(), n)
            plan.search(w.widths, thr)
            c = plan.candidates(seq, cap=1 << 23)
            s = [plan.series(r)[0].cpu().numpy() for r in range(len(w.ranges))] if series else None
            m = [plan.moments(r)[0] for r in range(len(w.ranges))]
            out.append((c, s, m))
            T += n
    finally:
        plan.close()
    return nf, models, out


def _oracle_every_block(w, x, sizes, got_per_chunk, block):
    """With EVERY_BLOCK the candidate sets must be equal as sets of blocks (no tolerance band
    at the threshold); within a block, tests/_parity.py's comparison."""
    ranges = w.ranges_array()
    ref = oracle.run(x[:sum(sizes)], w.freqs(), w.tsamp, ranges, w.widths, EVERY_BLOCK, block,
                     sizes)
    total = 0
    for got, per in zip(got_per_chunk, ref["chunks"]):
        want = np.concatenate([per[r]["cands"] for r in range(len(ranges))])
        assert got.size == want.size
        n = compare_candidates(got, want, EVERY_BLOCK, block, lambda r, t, per=per:
                               per[r]["series"][t], lambda r, per=per: per[r]["J0"],
                               lambda r: int(ranges[r][3]))
        assert n == want.size
        total += n
    return total


def _same_candidates(a, b):
    assert a.size == b.size
    for f in ("trial", "range", "t_start", "width"):
        np.testing.assert_array_equal(a[f], b[f])
    np.testing.assert_array_equal(a["snr"], b["snr"])  # bit-identical FP64


@pytest.mark.parametrize("block,threshold", [(32, EVERY_BLOCK), (8, 4.0), (1, 4.5)])
def test_fused_equals_plain_and_oracle(block, threshold):
    w = _workload()
    w.threshold = threshold
    x = w.generate(_arrivals(w))
    L = 1 << 16
    sizes = [L, L - 4096 - 512 - 44]  # the second window ends inside a tile (multiple of 4)
    nf, models, fused = _run(w, x, sizes, L, True, block, threshold)
    assert nf == 3 and all(m["fused"] == 1 for m in models)
    _, _, plain = _run(w, x, sizes, L, False, block, threshold)
    for (cf, _, mf), (cp, _, mp) in zip(fused, plain):
        _same_candidates(cf, cp)
        for a, b in zip(mf, mp):
            np.testing.assert_array_equal(a, b)
    if threshold == EVERY_BLOCK:  # every block of every trial, against the oracle as well
        assert _oracle_every_block(w, x, sizes, [c for c, _, _ in fused], block) > 100000
    else:
        assert oracle_candidates_match(w, x, sizes, [c for c, _, _ in fused], block) > 0


def test_kept_series_and_moments_equal_oracle():
    w = _workload(nsamp=1 << 16, widths=(1, 2, 4, 8, 16, 32, 64, 128, 256))
    x = w.generate(_arrivals(w))
    L = 1 << 15
    sizes = [L, L]
    w.threshold = 5.0
    _, _, fused = _run(w, x, sizes, L, True, 32, keep=True, series=True)
    ref = oracle.run(x[:sum(sizes)], w.freqs(), w.tsamp, w.ranges_array(), w.widths, 5.0, 32,
                     sizes)
    for (c, s, m), per in zip(fused, ref["chunks"]):
        for r in range(len(w.ranges)):
            np.testing.assert_array_equal(s[r], per[r]["series"])
            assert_moments_equal(m[r], per[r]["moments"], f"range {r}")
    assert oracle_candidates_match(w, x, sizes, [c for c, _, _ in fused], 32) > 0


def test_prefix_sums_wrapping_2_32_within_a_tile():
    """40000 channels of bytes 250..255: a tile's 512 outputs sum past 2^32 (the fused prefix
    sums wrap); every boxcar sum stays below 2^31 (widths up to 128)."""
    nch = 40000
    ranges = (configs.DMRange(0.0, 0.02, 70, 1), configs.DMRange(1.4, 0.02, 40, 2))
    w = configs.mid(nsamp=6144, chunk_len=2048, n_streams=1, npulses=0, nchans=nch,
                    ranges=ranges, index=12)
    w.widths = (1, 2, 8, 32, 128)
    rng = np.random.default_rng(5)
    x = rng.integers(250, 256, size=(6144, nch), dtype=np.uint8)
    x[3000:3010] = 255  # one bright block
    sizes = [2048, 2048, 2048]
    assert 512 * nch * 250 >= 1 << 32
    nf, _, fused = _run(w, x, sizes, 2048, True, 32, EVERY_BLOCK, streams=1)
    assert nf == 2
    _, _, plain = _run(w, x, sizes, 2048, False, 32, EVERY_BLOCK, streams=1)
    for (cf, _, _), (cp, _, _) in zip(fused, plain):
        _same_candidates(cf, cp)
        assert cf.size > 0


def test_ranges_the_fused_form_cannot_take_keep_the_plain_path():
    """Widths above 512 decimated samples leave the x1 range on the plain path (its series kept);
    the x2 range (widths / 2 <= 512) is fused. Candidates equal the plain plan's."""
    ranges = (configs.DMRange(0.0, 0.0625, 90, 1), configs.DMRange(5.625, 0.125, 60, 2))
    w = _tiled(512, 1 << 15, ranges, 13, chunk_len=1 << 14, npulses=4)
    w.widths = (2, 4, 64, 1024)
    x = w.generate(_arrivals(w))
    sizes = [1 << 14, 1 << 14]
    nf, models, fused = _run(w, x, sizes, 1 << 14, True, 32, 2.0)
    assert nf == 1 and models[0]["fused"] == 0 and models[1]["fused"] == 1
    _, _, plain = _run(w, x, sizes, 1 << 14, False, 32, 2.0)
    for (cf, _, _), (cp, _, _) in zip(fused, plain):
        _same_candidates(cf, cp)


def test_fuse_search_errors():
    w = _workload(nsamp=1 << 14)
    x = w.generate(_arrivals(w))
    L = 1 << 13
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), L, n_streams=1, max_width=512)
    try:
        with pytest.raises(dd.DDError) as e:
            plan.fuse_search([4, 2])
        assert e.value.code == dd.DD_ERR_ARG
        with pytest.raises(dd.DDError) as e:
            plan.fuse_search([1, 2048])
        assert e.value.code == dd.DD_ERR_ARG
        assert plan.fuse_search(w.widths) == 3
        with pytest.raises(dd.DDError) as e:
            plan.fuse_search(w.widths)
        assert e.value.code == dd.DD_ERR_STATE
        plan.run(torch.from_numpy(x[:L]).cuda(), L)
        with pytest.raises(dd.DDError) as e:
            plan.series(0)
        assert e.value.code == dd.DD_ERR_STATE
        with pytest.raises(dd.DDError) as e:
            plan.search([1, 2, 4], 6.0)
        assert e.value.code == dd.DD_ERR_ARG
        with pytest.raises(dd.DDError) as e:
            plan.search(w.widths, 6.0, estimator=dd.DD_EST_CLIPPED)
        assert e.value.code == dd.DD_ERR_STATE
        plan.search(w.widths, 6.0)
        plan.candidates()
    finally:
        plan.close()
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), L, n_streams=1, max_width=512)
    try:
        plan.run(torch.from_numpy(x[:L]).cuda(), L)
        with pytest.raises(dd.DDError) as e:
            plan.fuse_search(w.widths)
        assert e.value.code == dd.DD_ERR_STATE
    finally:
        plan.close()


def test_kept_series_serve_the_clipped_estimator():
    w = _workload(nsamp=1 << 15, widths=(1, 4, 16, 64))
    x = w.generate(_arrivals(w))
    L = 1 << 14
    res = []
    for fuse in (True, False):
        plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), L, n_streams=1, max_width=64)
        try:
            if fuse:
                plan.fuse_search(w.widths, keep_series=True)
            seq = plan.run(torch.from_numpy(x[:L]).cuda(), L)
            plan.search(w.widths, 4.0, estimator=dd.DD_EST_CLIPPED)
            res.append(plan.candidates(seq))
        finally:
            plan.close()
    _same_candidates(res[0], res[1])
    assert res[0].size > 0


def test_ranges_planned_on_another_tile_shape_are_replanned():
    """A plan made on 256-sample tiles (DD_FLAG_TILE256) is re-planned on the 64 x 512 tile for
    the fused form; its candidates equal the plain plan's."""
    w = _workload(nsamp=1 << 15, widths=(1, 2, 8, 32, 128))
    x = w.generate(_arrivals(w))
    L = 1 << 14
    res = []
    for fuse in (True, False):
        plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), L, n_streams=1, max_width=128,
                       flags=dd.DD_FLAG_TILE256)
        try:
            assert all(plan.kernel(r) == (dd.DD_KERNEL_TILED, 256) for r in range(3))
            if fuse:
                assert plan.fuse_search(w.widths) == 3
                assert all(plan.kernel(r) == (dd.DD_KERNEL_TILED, 512) for r in range(3))
            out = []
            for k in range(2):
                seq = plan.run(torch.from_numpy(x[k * L:(k + 1) * L]).cuda(), L)
                plan.search(w.widths, 3.0)
                out.append(plan.candidates(seq))
            res.append(out)
        finally:
            plan.close()
    for a, b in zip(*res):
        _same_candidates(a, b)
        assert a.size > 0
