"""dd_sps_static: the search without library allocations, against the oracle and the plan's own
search.

Callers that cannot let a library allocate device memory at run time (a real-time pipeline
with a fixed GPU memory budget, a plug-in whose host owns all device memory) use this entry
point; its scratch is a fixed device array shared by all calls. Two chunks are searched in a
row, so the second call runs on scratch the first one left behind. This file sorts last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from synth import configs
from _parity import SNR_RTOL, compare_candidates

torch = pytest.importorskip("torch")
import paper_2101_00941_gb300 as dd  # noqa: E402

pytestmark = pytest.mark.gpu


def _workload():
    ranges = (configs.DMRange(0.0, 2.0, 40, 1), configs.DMRange(80.0, 4.0, 30, 2),
              configs.DMRange(200.0, 5.0, 20, 4))
    w = configs.mid(nsamp=1 << 14, chunk_len=4096, n_streams=2, npulses=4, nchans=4096,
                    ranges=ranges, index=9)
    w.nchans = 128
    w.foff = -300.0 / 128
    w.pulses = tuple(configs.PulseSpec(p.dm * 0.25, min(p.t_ref, 9000), p.width, p.amp * 4.0)
                     for p in w.pulses)
    w.threshold = 4.5  # low enough that noise alone gives candidates in every chunk
    return w


def _sorted(c):
    return c[np.lexsort((c["width"], c["t_start"], c["trial"], c["range"]))]


def test_static_search_matches_plan_search_twice():
    dd.build()
    w = _workload()
    f = w.freqs()
    x = w.generate(lambda dm: oracle.delay_samples(f, w.tsamp, dm))
    ranges = w.ranges_array()
    plan = dd.Plan(f, w.tsamp, ranges, 4096, n_streams=2, max_width=max(w.widths))
    cap = 1 << 16
    cands = torch.zeros(cap * dd.CAND_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    xs = torch.from_numpy(x).cuda()
    ref = oracle.run(x[:4096 * 4], f, w.tsamp, ranges, w.widths, w.threshold, 32, [4096] * 4)
    compared = 0
    try:
        for k in (2, 3):  # two chunks with full windows, searched one after the other
            if plan.seq < k - 1:
                for j in range(plan.seq + 1, k):
                    plan.run(xs[4096 * j:4096 * (j + 1)], 4096)
                    plan.search(w.widths, w.threshold)
            seq = plan.run(xs[4096 * k:4096 * (k + 1)], 4096)
            plan.search(w.widths, w.threshold)
            want = plan.candidates(seq)
            got = []
            for r, row in enumerate(ranges):
                ptr, n, stride, j0 = dd.dd_series(plan.h, r)
                dd.dd_sps_static(ptr, int(row[2]), n, stride, r, int(row[3]), j0, w.widths,
                                 w.threshold, 32, cands.data_ptr(), cap, count.data_ptr())
                torch.cuda.synchronize()
                m = int(count.item())
                assert m <= cap
                got.append(cands[:m * dd.CAND_DTYPE.itemsize].cpu().numpy().view(dd.CAND_DTYPE))
            got = _sorted(np.concatenate(got))
            assert got.size == want.size and want.size > 0
            np.testing.assert_array_equal(got[["trial", "range", "t_start", "width"]],
                                          want[["trial", "range", "t_start", "width"]])
            np.testing.assert_allclose(got["snr"], want["snr"], rtol=SNR_RTOL)
            per = ref["chunks"][k]
            assert compare_candidates(
                got, np.concatenate([per[r]["cands"] for r in range(len(ranges))]), w.threshold,
                32, lambda r, t, per=per: per[r]["series"][t], lambda r, per=per: per[r]["J0"],
                lambda r: int(ranges[r][3])) > 0
            compared += 1
    finally:
        plan.close()
    assert compared == 2


def test_static_search_rejects_more_trials_than_its_scratch():
    dd.build()
    series = torch.zeros((16385, 64), dtype=torch.int32, device="cuda")
    cands = torch.zeros(64 * dd.CAND_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(dd.DDError) as e:
        dd.dd_sps_static(series.data_ptr(), 16385, 64, 64, 0, 1, 0, [1, 2], 6.0, 32,
                         cands.data_ptr(), 64, count.data_ptr())
    assert e.value.code == dd.DD_ERR_ARG and "16384" in str(e.value)
    with pytest.raises(dd.DDError) as e:
        dd.dd_sps_static(series.data_ptr(), 16, 64, 64, 0, 1, 0, [1, 2], float("nan"), 32,
                         cands.data_ptr(), 64, count.data_ptr())
    assert e.value.code == dd.DD_ERR_ARG and "finite" in str(e.value)
