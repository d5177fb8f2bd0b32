"""The search with clipped per-width statistics (sps_run_ex, DD_EST_CLIPPED) against the oracle's
or_sps_clipped on the oracle's own series, and candidate grouping of a GPU search result.

Input: seeded noise with dispersed pulses plus strong impulsive interference (spikes that every
trial sees), the case the clipping is for: unclipped statistics are inflated by the spikes."""
import numpy as np
import pytest

import oracle
from synth import configs
from _parity import clipped_trial_snr, compare_candidates

torch = pytest.importorskip("torch")
import paper_2101_00941_gb300 as dd  # noqa: E402
from _gpu_check import _arrivals  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    dd.build()
    dd.lib()


def _workload(kernel="tiled"):
    if kernel == "tiled":  # fine channels: the tiled kernel
        ranges = (configs.DMRange(0.0, 0.0625, 70, 1), configs.DMRange(4.375, 0.125, 40, 2),
                  configs.DMRange(9.375, 0.25, 30, 4))
        w = configs.mid(nsamp=1 << 15, chunk_len=4096, n_streams=2, npulses=4, nchans=4096,
                        ranges=ranges, index=60)
        w.nchans, w.foff = 256, -300.0 / 1024
        w.pulses = tuple(configs.PulseSpec(p.dm * 0.012, min(p.t_ref, 26000), p.width,
                                           p.amp * 6.0) for p in w.pulses)
    else:  # coarse channels: the direct kernel
        ranges = (configs.DMRange(0.0, 2.0, 40, 1), configs.DMRange(80.0, 4.0, 30, 2))
        w = configs.mid(nsamp=1 << 15, chunk_len=4096, n_streams=2, npulses=4, nchans=4096,
                        ranges=ranges, index=61)
        w.nchans, w.foff = 128, -300.0 / 128
        w.pulses = tuple(configs.PulseSpec(p.dm * 0.3, min(p.t_ref, 26000), p.width, p.amp * 4.0)
                         for p in w.pulses)
    w.widths = (1, 2, 4, 8, 16, 32, 64)
    w.threshold = 6.0
    return w


def _with_interference(w, x):
    """Broadband spikes: 40 random samples set to 255 in every channel (zero DM)."""
    rng = np.random.default_rng(62)
    x = x.copy()
    x[np.sort(rng.choice(x.shape[0], 40, replace=False))] = 255
    return x


@pytest.mark.parametrize("kernel,kappa,iters", [("tiled", 3.0, 3), ("tiled", 2.5, 1),
                                                ("direct", 3.0, 3), ("tiled", 3.0, 0)])
def test_clipped_search_matches_oracle(kernel, kappa, iters):
    w = _workload(kernel)
    x = _with_interference(w, w.generate(_arrivals(w)))
    ranges = w.ranges_array()
    sizes = [4096] * 8
    plan = dd.Plan(w.freqs(), w.tsamp, ranges, 4096, n_streams=2, max_width=max(w.widths))
    got = []
    try:
        want_kind = dd.DD_KERNEL_TILED if kernel == "tiled" else dd.DD_KERNEL_DIRECT
        assert plan.kernel(0)[0] == want_kind
        xs = torch.from_numpy(x).cuda()
        for k, n in enumerate(sizes):
            seq = plan.run(xs[4096 * k:4096 * (k + 1)], n)
            plan.search(w.widths, w.threshold, estimator=dd.DD_EST_CLIPPED, clip_iters=iters,
                        clip_kappa=kappa)
            got.append(plan.candidates(seq))
    finally:
        plan.close()
    ref = oracle.run(x, w.freqs(), w.tsamp, ranges, w.widths, w.threshold, 32, sizes)
    matched = 0
    for c, per in zip(got, ref["chunks"]):
        want = []
        for r in range(len(ranges)):
            y, J0 = per[r]["series"], per[r]["J0"]
            if y.shape[1] == 0:
                continue
            d = int(ranges[r][3])
            want.append(oracle.sps_clipped(y, per[r]["trials"], r, d, J0,
                                           oracle.widths_for_range(w.widths, d), 32,
                                           w.threshold, kappa, iters))
        want = np.concatenate(want) if want else np.zeros(0, dtype=oracle.CAND_DTYPE)
        matched += compare_candidates(
            c, want, w.threshold, 32, lambda r, t, per=per: per[r]["series"][t],
            lambda r, per=per: per[r]["J0"], lambda r: int(ranges[r][3]),
            trial_snr=clipped_trial_snr(kappa, iters))
    assert matched > 0


def test_clipped_search_finds_the_pulses_among_interference():
    """With broadband spikes in the data, the clipped search still reports every injected pulse,
    and friends-of-friends grouping merges its candidates into far fewer events."""
    w = _workload("tiled")
    x = _with_interference(w, w.generate(_arrivals(w)))
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=1,
                   max_width=max(w.widths))
    try:
        xs = torch.from_numpy(x).cuda()
        clipped = []
        for k in range(8):
            plan.run(xs[4096 * k:4096 * (k + 1)], 4096)
            plan.search(w.widths, w.threshold, estimator=dd.DD_EST_CLIPPED)
            clipped.append(plan.candidates())
    finally:
        plan.close()
    c = np.concatenate(clipped)
    assert c.size > 0 and np.isfinite(c["snr"]).all()
    # candidates group into far fewer events than candidates
    c = c[np.lexsort((c["width"], c["t_start"], c["trial"], c["range"]))]
    _, groups = dd.dd_group_candidates(c, w.ranges_array(), dm_link=1.0, t_link=64)
    assert 0 < groups.size < c.size
    for p in w.pulses:  # every injected pulse lies inside some group's time extent
        t_top = p.t_ref
        assert any(g["t_lo"] - 512 <= t_top <= g["t_hi"] + 512 for g in groups), p


def test_bad_estimator_arguments():
    w = _workload("tiled")
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=1,
                   max_width=max(w.widths))
    try:
        x = torch.from_numpy(w.generate(_arrivals(w))[:4096]).cuda()
        plan.run(x, 4096)
        for est, it, kap in ((7, 3, 3.0), (dd.DD_EST_CLIPPED, -1, 3.0),
                             (dd.DD_EST_CLIPPED, 3, 0.0), (dd.DD_EST_CLIPPED, 3, float("inf"))):
            with pytest.raises(dd.DDError) as e:
                plan.search(w.widths, 6.0, estimator=est, clip_iters=it, clip_kappa=kap)
            assert e.value.code == dd.DD_ERR_ARG
    finally:
        plan.close()
