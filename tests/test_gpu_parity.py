"""GPU path (through the C ABI) against the CPU oracle.

Dedispersed series and the moments the library exposes (dd_moments) bit-exact;
candidates per block with SNR within 1e-5 relative (tests/_parity.py). Covers the tiny workload whole and chunked
over 1 and 4 streams, multi-range decimated plans with ragged chunks and
ragged channel counts, every input kind (device, pinned, pageable), pipelined
streams, an empty first window, and the full-size 4096-channel workload on
sampled trials in the benchmark's launch configuration.
"""
import os

import numpy as np
import pytest

import oracle
from synth import configs

torch = pytest.importorskip("torch")
import paper_2101_00941_gb300 as dd  # noqa: E402
from _gpu_check import _arrivals, check, run_gpu  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    dd.build()
    dd.lib()


# ----------------------------------------------------------------------------- tests

def test_plan_matches_oracle_delay_table():
    w = configs.mid(nsamp=1 << 16)
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 1 << 16, n_streams=1)
    try:
        tabs = oracle.shift_tables(w.freqs(), w.tsamp, w.ranges_array())
        np.testing.assert_array_equal(plan.shifts, np.concatenate(tabs))
        assert plan.O == oracle.overlap(tabs, w.ranges_array())
    finally:
        plan.close()


def test_tiny_whole():
    w = configs.tiny()
    x = w.generate(_arrivals(w))
    assert check(w, x, [w.nsamp], 1) > 0


@pytest.mark.parametrize("n_streams", [1, 4])
def test_tiny_chunked_streams(n_streams):
    w = configs.tiny()
    x = w.generate(_arrivals(w))
    assert check(w, x, [8192] * 8, n_streams) > 0


def _small_multirange(nchans=128, nsamp=1 << 15, npulses=6):
    ranges = (configs.DMRange(0.0, 2.0, 40, 1), configs.DMRange(80.0, 4.0, 30, 2),
              configs.DMRange(200.0, 5.0, 20, 4), configs.DMRange(300.0, 10.0, 18, 8))
    w = configs.mid(nsamp=nsamp, chunk_len=4096, n_streams=3, npulses=npulses, nchans=4096,
                    ranges=ranges, index=7)
    w.nchans = nchans
    w.foff = -300.0 / nchans
    w.pulses = tuple(configs.PulseSpec(p.dm * 0.35, min(p.t_ref, nsamp - 6000), p.width,
                                       p.amp * 4.0) for p in w.pulses)
    return w


def test_multirange_decimated_ragged_chunks():
    w = _small_multirange()
    x = w.generate(_arrivals(w))
    sizes = [4096] * 7 + [2048, 2040]  # ragged tail chunks (multiples of d_max = 8)
    assert sum(sizes) <= w.nsamp
    assert check(w, x[:sum(sizes)], sizes, 3) > 0


def _tiled_regime(nchans=1001, nsamp=1 << 15):
    """Channel width and DM steps in the regime of the 4096-channel workload (8-11 delay classes
    per 8-channel group and 64-trial tile) at a size the oracle checks in full: 1001 channels
    (neither a multiple of 8 nor of 16) from 1550 MHz down by 300/1024 MHz, 64 us, and eight
    ranges x1..x128 whose trial counts leave ragged 64-trial tiles."""
    ranges = (configs.DMRange(0.0, 0.0625, 150, 1), configs.DMRange(9.375, 0.125, 75, 2),
              configs.DMRange(18.75, 0.15625, 130, 4), configs.DMRange(39.0625, 0.3125, 70, 8),
              configs.DMRange(60.9375, 0.625, 40, 16), configs.DMRange(85.9375, 1.25, 30, 32),
              configs.DMRange(123.4375, 2.5, 20, 64), configs.DMRange(173.4375, 5.0, 10, 128))
    w = configs.mid(nsamp=nsamp, chunk_len=4096, n_streams=3, npulses=6, nchans=4096,
                    ranges=ranges, index=9)
    w.nchans = nchans
    w.foff = -300.0 / 1024
    w.pulses = tuple(configs.PulseSpec(p.dm * 0.2, min(p.t_ref, nsamp - 6000), p.width,
                                       p.amp * 2.0) for p in w.pulses)
    return w


def test_kernel_choice():
    """Ranges whose delay classes fit the tiled kernel's tables run on it (512-sample tiles);
    x32 .. x128 decimation (two groups' eight channels of 255 x d do not fit a 16-bit lane)
    and the tiny workload's 64 coarse channels (up to 63 classes per group) run on the direct
    kernel, and DD_FLAG_NAIVE selects the one-thread-per-output kernel."""
    w = _tiled_regime()
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=1)
    try:
        got = [plan.kernel(r) for r in range(len(w.ranges))]
    finally:
        plan.close()
    assert got == [(dd.DD_KERNEL_TILED, 512)] * 5 + [(dd.DD_KERNEL_DIRECT, 0)] * 3
    t = configs.tiny()
    plan = dd.Plan(t.freqs(), t.tsamp, t.ranges_array(), 4096, n_streams=1)
    try:
        assert plan.kernel(0) == (dd.DD_KERNEL_DIRECT, 0)
    finally:
        plan.close()
    plan = dd.Plan(t.freqs(), t.tsamp, t.ranges_array(), 4096, n_streams=1, flags=dd.DD_FLAG_NAIVE)
    try:
        assert plan.kernel(0) == (dd.DD_KERNEL_PER_OUTPUT, 0)
    finally:
        plan.close()


@pytest.mark.parametrize("sizes,n_streams", [
    ([1 << 15], 1),                            # one chunk: the whole input
    ([4096] * 7 + [2048, 1920], 3),            # ragged chunks (multiples of d_max = 128)
])
def test_tiled_kernel_full_parity(sizes, n_streams):
    """Every series of every trial of every range bit-exact against the oracle, and every
    candidate, through the tiled kernel at the workload's channel width."""
    w = _tiled_regime()
    x = w.generate(_arrivals(w))
    assert check(w, x[:sum(sizes)], sizes, n_streams) > 0


@pytest.mark.parametrize("block", [1, 8])
def test_search_peak_blocks_and_odd_widths(block):
    """Peak blocks smaller than a warp, and boxcar widths that are not powers of two (3, 6, 12,
    24, 100 original samples: decimated widths 1 .. 100 with every residue mod 4)."""
    w = _tiled_regime(nsamp=1 << 14)
    w.widths = (1, 3, 6, 12, 24, 100)
    x = w.generate(_arrivals(w))
    assert check(w, x, [4096] * 4, 2, block=block) > 0


def test_search_widest_boxcars():
    """Boxcars up to the largest width the plan accepts (1024 original samples: a 1024-sample
    history in every search pass), in chunks of 4096 samples."""
    w = _tiled_regime(nsamp=1 << 14)
    w.widths = (1, 5, 64, 1000, 1024)
    x = w.generate(_arrivals(w))
    assert check(w, x, [4096] * 4, 2) > 0


def test_single_trial_and_ragged_tiles():
    """Ranges of 1 trial, 65 trials (a full 64-trial tile and a 1-trial tile) and 1 decimated
    trial, through the tiled kernel, with a ragged last chunk."""
    w = _tiled_regime(nsamp=1 << 14)
    w.ranges = (configs.DMRange(0.0, 0.0625, 1, 1), configs.DMRange(1.0, 0.0625, 65, 1),
                configs.DMRange(10.0, 0.125, 1, 2))
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=1)
    try:
        assert [plan.kernel(r)[0] for r in range(3)] == [dd.DD_KERNEL_TILED] * 3
    finally:
        plan.close()
    x = w.generate(_arrivals(w))
    check(w, x, [4096] * 3 + [2048], 2)


def test_direct_kernel_huge_delay_spans():
    """16 channels from 1500 down to 100 MHz at 1 ms: adjacent channels' delays differ by
    thousands of samples (overlap 49151 samples), so the range runs on the direct kernel."""
    w = configs.tiny()
    w.nchans, w.fch1, w.foff, w.tsamp = 16, 1500.0, -1400.0 / 15, 1e-3
    w.nsamp, w.widths = 1 << 17, (1, 2, 4, 8)
    w.ranges = (configs.DMRange(100.0, 1.0, 20, 1),)
    w.pulses = (configs.PulseSpec(110.0, 70000, 4, 40.0),)
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 1 << 16, n_streams=1)
    try:
        assert plan.kernel(0) == (dd.DD_KERNEL_DIRECT, 0)
    finally:
        plan.close()
    x = w.generate(_arrivals(w))
    check(w, x, [1 << 16, 1 << 16], 1)


def test_tiled_kernel_odd_group_count():
    """993 channels (padded to 1000: 125 eight-channel groups, so the last stage holds one
    group), every trial of two ranges, in ragged chunks."""
    w = _tiled_regime(nchans=993, nsamp=1 << 14)
    w.ranges = (configs.DMRange(0.0, 0.0625, 100, 1), configs.DMRange(6.25, 0.125, 50, 2))
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=1)
    try:
        assert [plan.kernel(r)[0] for r in range(2)] == [dd.DD_KERNEL_TILED] * 2
    finally:
        plan.close()
    x = w.generate(_arrivals(w))
    assert check(w, x, [4096] * 3 + [2048], 2) >= 0


def test_tiled_kernel_256_sample_tiles():
    """The 256-sample-tile instances (uint8 and uint16), forced by DD_FLAG_TILE256, on every
    trial of ranges x1 .. x8, in ragged chunks."""
    w = _tiled_regime(nsamp=1 << 14)
    w.ranges = w.ranges[:4]
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=1,
                   flags=dd.DD_FLAG_TILE256)
    try:
        assert [plan.kernel(r) for r in range(4)] == [(dd.DD_KERNEL_TILED, 256)] * 4
    finally:
        plan.close()
    x = w.generate(_arrivals(w))
    assert check(w, x, [4096] * 3 + [2048], 2, flags=dd.DD_FLAG_TILE256) >= 0


@pytest.mark.parametrize("flags,shape", [
    (dd.DD_FLAG_WARPS32, (512, 64, 1024)),          # 32 warps on the 64 x 512 tile
    (dd.DD_FLAG_TILE256, (256, 64, 512)),           # two CTAs per SM
    (dd.DD_FLAG_TILE256 | dd.DD_FLAG_TRIALS32, (256, 32, 512)),
    (dd.DD_FLAG_AUTOTUNE, None),                    # whichever shape the timing picks
])
def test_tiled_kernel_tile_shapes(flags, shape):
    """Every tile shape of the tiled kernel, forced by the testing flags or picked by the plan's
    autotuner, on every trial of ranges x1 .. x16 in ragged chunks: series, moments and
    candidates against the oracle."""
    w = _tiled_regime(nsamp=1 << 14)
    w.ranges = w.ranges[:5]
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=1, flags=flags)
    try:
        for r in range(len(w.ranges)):
            m = plan.model(r, 1)
            assert m["kind"] == dd.DD_KERNEL_TILED
            if shape is not None:
                assert (m["tile_samples"], m["tile_trials"], m["cta_threads"]) == shape
    finally:
        plan.close()
    x = w.generate(_arrivals(w))
    assert check(w, x, [4096] * 3 + [2048], 2, flags=flags) >= 0


def test_tiled_kernel_odd_output_counts():
    """Windows of odd length: x1 ranges only, so the overlap is the largest delay (63 samples),
    and chunks of 4096, 4096, 2047 and 1001 samples give windows of 4033, 4096, 2047 and 1001
    outputs. The tiled kernel writes a lane's outputs in pairs; the last output of an odd window
    is written, and counted in the moments, alone."""
    w = _tiled_regime(nsamp=1 << 14)
    w.ranges = (configs.DMRange(0.0, 0.0625, 70, 1), configs.DMRange(4.375, 0.0625, 3, 1))
    sizes = [4096, 4096, 2047, 1001]
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=1)
    try:
        assert plan.O == 63
        assert [plan.kernel(r)[0] for r in range(2)] == [dd.DD_KERNEL_TILED] * 2
    finally:
        plan.close()
    x = w.generate(_arrivals(w))
    assert check(w, x[:sum(sizes)], sizes, 2) >= 0


def test_one_thread_per_output_kernel_matches():
    """The testing-aid kernel (DD_FLAG_NAIVE) obeys the same contract as the tiled one."""
    w = _small_multirange(nsamp=1 << 14)
    x = w.generate(_arrivals(w))
    check(w, x, [4096] * 4, 2, flags=dd.DD_FLAG_NAIVE)


@pytest.mark.parametrize("kind", ["pinned", "pageable", "staged"])
def test_ragged_channels_host_input(kind):
    w = _small_multirange(nchans=98, nsamp=1 << 14, npulses=3)
    x = w.generate(_arrivals(w))
    check(w, x, [4096] * 4, 2, kind=kind)


def test_input_kinds_give_identical_results():
    """Sec. 2.1: pinned, pageable and pageable-through-pinned-staging inputs give the same
    results as device-resident input."""
    w = _small_multirange(nsamp=1 << 14)
    x = w.generate(_arrivals(w))
    res = [run_gpu(w, x, [4096] * 4, 2, kind=k)[0]
           for k in ("device", "pinned", "pageable", "staged")]
    for other in res[1:]:
        for (sa, ca), (sb, cb) in zip(res[0], other):
            np.testing.assert_array_equal(ca, cb)
            for (a, _, ma), (b, _, mb) in zip(sa, sb):
                np.testing.assert_array_equal(a, b)
                np.testing.assert_array_equal(ma, mb)


def test_pipelined_streams_match_sequential():
    """Chunks enqueued back to back on 4 streams give the same candidates as one at a time."""
    w = _small_multirange(nsamp=1 << 15)
    x = w.generate(_arrivals(w))
    sizes = [4096] * 8
    seq_res = run_gpu(w, x, sizes, 1, want_series=False)[0]
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=4,
                   max_width=max(w.widths))
    xs = torch.from_numpy(x[:sum(sizes)]).cuda()
    got = []
    try:
        for k in range(8):
            plan.run(xs[4096 * k:4096 * (k + 1)], 4096)
            plan.search(w.widths, w.threshold)
            if k >= 3:
                got.append(plan.candidates(k - 3))
        for k in range(5, 8):
            got.append(plan.candidates(k))
    finally:
        plan.close()
    for (_, want), g in zip(seq_res, got):
        np.testing.assert_array_equal(g, want)


def test_first_chunk_shorter_than_overlap():
    w = _small_multirange(nsamp=1 << 14)
    x = w.generate(_arrivals(w))
    tabs = oracle.shift_tables(w.freqs(), w.tsamp, w.ranges_array())
    O = oracle.overlap(tabs, w.ranges_array())
    first = (O // 2) // 8 * 8
    sizes = [first, 4096, 4096]
    check(w, x[:sum(sizes)], sizes, 2)


def test_full_size_sampled_trials():
    """4096 channels, 2^20 samples, 4050 trials, 8 chunks over 4 streams (the benchmark's
    launch configuration); sampled trials of every range, every chunk, bit-exact series."""
    w = configs.mid()
    x = w.generate(_arrivals(w))
    rng = np.random.default_rng(5)
    trials = []
    for r in w.ranges:
        t = {0, r.n_trials - 1} | set(int(v) for v in rng.integers(0, r.n_trials, 2))
        trials.append(sorted(t))
    # also the trials nearest each injected pulse, so candidates are exercised
    for p in w.pulses:
        for ri, r in enumerate(w.ranges):
            if r.dm_start <= p.dm < r.dm_start + r.n_trials * r.dm_step:
                trials[ri] = sorted(set(trials[ri]) | {int((p.dm - r.dm_start) / r.dm_step)})
    sizes = [w.chunk_len] * (w.nsamp // w.chunk_len)
    assert check(w, x, sizes, w.n_streams, trials=trials) > 0


def test_errors_are_reported():
    w = _small_multirange(nsamp=1 << 13)
    x = w.generate(_arrivals(w))
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=2,
                   max_width=max(w.widths))
    xs = torch.from_numpy(x).cuda()
    try:
        with pytest.raises(dd.DDError) as e:
            plan.run(xs[:100], 100)  # not a multiple of the largest decimation
        assert e.value.code == dd.DD_ERR_ARG
        with pytest.raises(dd.DDError) as e:
            dd.sps_run(plan.h, w.widths, w.threshold)  # nothing run yet
        assert e.value.code == dd.DD_ERR_STATE
        for k in range(3):
            plan.run(xs[4096 * (k % 2):4096 * (k % 2 + 1)], 4096)
            plan.search(w.widths, -1e30)  # every block is a candidate
        with pytest.raises(dd.DDError) as e:
            plan.search(w.widths, 6.0)
        assert e.value.code == dd.DD_ERR_STATE
        with pytest.raises(dd.DDError) as e:
            plan.candidates(0)  # recycled by chunk 2 (2 streams)
        assert e.value.code == dd.DD_ERR_STATE
        full = plan.candidates(2)
        assert full.size > 10
        with pytest.raises(dd.DDError) as e:
            plan.candidates(2, cap=5)
        assert e.value.code == dd.DD_ERR_CAP
        with pytest.raises(dd.DDError) as e:
            plan.search([4, 2], 6.0)
        assert e.value.code == dd.DD_ERR_ARG
    finally:
        plan.close()


def test_timing_and_launch_counters():
    w = _small_multirange(nsamp=1 << 14)
    x = w.generate(_arrivals(w))
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=2,
                   max_width=max(w.widths), flags=dd.DD_FLAG_TIMING)
    try:
        plan.stats(reset=True)
        xs = torch.from_numpy(x).cuda()
        for k in range(4):
            plan.run(xs[4096 * k:4096 * (k + 1)], 4096)
            plan.search(w.widths, w.threshold)
        plan.sync()
        launches, ms, nlaunch = plan.stats()
        # every chunk: corner turn + 3 decimation levels; every range with a non-empty
        # window: dedispersion (+ moments in the one-thread-per-output path) + search
        windows = oracle.chunk_windows([4096] * 4, plan.O)
        live = sum(1 for (_, _, lo, hi) in windows for r in w.ranges if hi // r.decimation >
                   lo // r.decimation)
        assert launches >= 4 * 4 + 2 * live
        assert ms > 0 and nlaunch == live
    finally:
        plan.close()


def test_out_of_core_shape_from_pageable_memory_through_staging():
    """8192 channels, 1000-1500 MHz, 50 us, DM 0-3000 with x1..x16 decimation (overlap ~138k
    samples), two 2^18-sample chunks from pageable memory through the pinned staging threads;
    sampled trials of every range, bit-exact series and matching candidates."""
    w = configs.out_of_core(nsamp=1 << 19)
    w.chunk_len = 1 << 18
    w.n_streams = 2
    x = w.generate(_arrivals(w))
    rng = np.random.default_rng(8)
    trials = [sorted({0, r.n_trials - 1} | set(int(v) for v in rng.integers(0, r.n_trials, 2)))
              for r in w.ranges]
    assert check(w, x, [w.chunk_len, w.chunk_len], 2, kind="staged", trials=trials) >= 0


def test_out_of_core_beam_in_the_benchmark_launch_configuration():
    """The benchmark's default workload as it is launched: 8192 channels, DM 0-3000 x1..x16,
    2^19-sample chunks over 4 streams, the plan's tile autotuner on, device-resident chunks.
    Three chunks (the first window is shorter than a chunk by the overlap; the third is a full
    window with history from both before it); two trials of every range, and the trial nearest
    each injected pulse, bit-exact series and moments against the oracle, candidates per block.
    About 10 minutes on the GPU machine, most of it the oracle's full-width decimation of 13 GB of
    input, so it runs when DD_FULL_SIZE_TESTS=1 is set."""
    if os.environ.get("DD_FULL_SIZE_TESTS") != "1":
        pytest.skip("full-size out-of-core parity: set DD_FULL_SIZE_TESTS=1")
    w = configs.out_of_core(nsamp=3 << 19)
    x = w.generate(_arrivals(w))
    trials = [sorted({0, r.n_trials - 1}) for r in w.ranges]
    for p in w.pulses:
        for ri, r in enumerate(w.ranges):
            if r.dm_start <= p.dm < r.dm_start + r.n_trials * r.dm_step and p.t_ref < 3 << 19:
                trials[ri] = sorted(set(trials[ri]) | {int((p.dm - r.dm_start) / r.dm_step)})
    L = w.chunk_len
    assert L == 1 << 19 and w.n_streams == 4
    assert check(w, x, [L, L, L], 4, kind="device", trials=trials,
                 flags=dd.DD_FLAG_AUTOTUNE) >= 0
