"""Failure detection on the GPU without a GPU fault.

* The device-side bounded wait (the tiled kernel's copy barriers) runs out on a barrier that
  nothing completes, reports it through a status word the host reads, and leaves the CUDA
  context usable: a plan run afterwards still matches the oracle bit for bit.
* The host-side bounded wait of dd_candidates reports DD_ERR_TIMEOUT for a chunk still on the
  GPU, and the same chunk is collected normally afterwards.
"""
import numpy as np
import pytest

import oracle
from synth import configs

torch = pytest.importorskip("torch")
import paper_2101_00941_gb300 as dd  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    dd.build()
    dd.lib()


def _small():
    ranges = (configs.DMRange(0.0, 0.0625, 70, 1), configs.DMRange(4.375, 0.125, 40, 2))
    w = configs.mid(nsamp=1 << 14, chunk_len=4096, n_streams=2, npulses=3, nchans=4096,
                    ranges=ranges, index=11)
    w.nchans = 256
    w.foff = -300.0 / 1024
    return w


def test_device_bounded_wait_times_out_and_context_survives():
    timed_out, ms = dd.dd_selftest_wait(0)
    assert timed_out == 1
    assert 1000.0 < ms < 60000.0  # the bound is 2 s of device time (or 2^26 polls)
    # the context still runs kernels and produces exact results
    w = _small()
    f = w.freqs()
    x = w.generate(lambda dm: oracle.delay_samples(f, w.tsamp, dm))
    plan = dd.Plan(f, w.tsamp, w.ranges_array(), 4096, n_streams=1, max_width=max(w.widths))
    try:
        plan.run(torch.from_numpy(x[:4096]).cuda(), 4096)
        plan.search(w.widths, w.threshold)
        plan.candidates()
        series, j0 = plan.series(0)
        got = series.cpu().numpy()
    finally:
        plan.close()
    ref = oracle.run(x[:4096], f, w.tsamp, w.ranges_array(), w.widths, w.threshold, 32, [4096])
    np.testing.assert_array_equal(got, ref["chunks"][0][0]["series"])


def test_candidate_wait_reports_timeout_then_collects():
    w = configs.mid(nsamp=1 << 17)
    f = w.freqs()
    x = torch.zeros((1 << 17, w.nchans), dtype=torch.uint8, device="cuda")
    plan = dd.Plan(f, w.tsamp, w.ranges_array(), 1 << 17, n_streams=1, max_width=max(w.widths))
    try:
        seq = plan.run(x, 1 << 17)  # tens of ms of GPU work
        plan.search(w.widths, w.threshold)
        with pytest.raises(dd.DDError) as e:
            dd.dd_candidates(plan.h, seq, timeout_ms=1)
        assert e.value.code == dd.DD_ERR_TIMEOUT
        assert plan.candidates(seq).size == 0  # all-zero input: constant series, no candidates
    finally:
        plan.close()
