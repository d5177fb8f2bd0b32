"""Serving loop (dd_serve_*): beams of different shapes submitted interleaved give, chunk by
chunk, the oracle's candidates (per block, tests/_parity.py) and exactly the candidates each beam
gives alone; admission respects the HBM budget and refuses bad search parameters."""
import time

import numpy as np
import pytest

import oracle
from synth import configs

torch = pytest.importorskip("torch")
import paper_2101_00941_gb300 as dd  # noqa: E402
from _gpu_check import oracle_candidates_match  # noqa: E402

pytestmark = pytest.mark.gpu


def _beams():
    out = []
    for k, (nch, scale) in enumerate(((128, 0.35), (64, 0.25), (96, 0.3))):
        ranges = (configs.DMRange(0.0, 2.0, 40, 1), configs.DMRange(80.0, 4.0, 30, 2))
        w = configs.mid(nsamp=1 << 14, chunk_len=4096, n_streams=2, npulses=3, nchans=4096,
                        ranges=ranges, index=20 + k)
        w.nchans = nch
        w.foff = -300.0 / nch
        w.pulses = tuple(configs.PulseSpec(p.dm * scale, min(p.t_ref, 9000), p.width, p.amp * 4)
                         for p in w.pulses)
        w.threshold = 5.0
        f = w.freqs()
        x = w.generate(lambda dm, f=f, w=w: oracle.delay_samples(f, w.tsamp, dm))
        out.append((w, x))
    return out


def _alone(w, x, sizes):
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=2,
                   max_width=max(w.widths))
    res, T = [], 0
    try:
        for n in sizes:
            seq = plan.run(torch.from_numpy(x[T:T + n]).cuda(), n)
            plan.search(w.widths, w.threshold)
            res.append(plan.candidates(seq))
            T += n
    finally:
        plan.close()
    return res


def test_each_chunk_is_the_same_alone_and_in_the_mix():
    dd.build()
    beams = _beams()
    sizes = [4096, 4096, 2048, 4096]
    want = [_alone(w, x, sizes) for w, x in beams]
    srv = dd.Server(max_inflight=4, hbm_budget_bytes=40 << 30)
    try:
        ids = [srv.add_beam(w.freqs(), w.tsamp, w.ranges_array(), 4096, w.widths, w.threshold,
                            n_streams=2) for w, _ in beams]
        dev = [torch.from_numpy(x).cuda() for _, x in beams]
        offs = [0] * len(beams)
        tickets = {}
        for k, n in enumerate(sizes):  # interleave the beams' chunks
            for b, bid in enumerate(ids):
                t = srv.submit(bid, dev[b][offs[b]:offs[b] + n], n)
                tickets[t] = (b, k)
                offs[b] += n
        got = {}
        deadline = time.time() + 120
        while len(got) < len(tickets) and time.time() < deadline:
            for r, c in srv.poll(64, timeout_ms=200):
                assert r["status"] == 0
                got[r["ticket"]] = (r, c)
        assert len(got) == len(tickets)
        per_beam = [[None] * len(sizes) for _ in beams]
        for t, (b, k) in tickets.items():
            r, c = got[t]
            assert r["beam"] == ids[b] and r["seq"] == k
            assert r["latency_ms"] >= r["queue_ms"] >= 0.0
            np.testing.assert_array_equal(c, want[b][k])
            per_beam[b][k] = c
        assert srv.pending() == (0, 0)
        matched = sum(oracle_candidates_match(w, x, sizes, per_beam[b])
                      for b, (w, x) in enumerate(beams))
        assert matched > 0
    finally:
        srv.close()


def test_beam_over_budget_is_refused():
    dd.build()
    (w, _), = _beams()[:1]
    srv = dd.Server(max_inflight=2, hbm_budget_bytes=1 << 20)  # 1 MiB: no plan fits
    try:
        with pytest.raises(dd.DDError) as e:
            srv.add_beam(w.freqs(), w.tsamp, w.ranges_array(), 4096, w.widths, w.threshold)
        assert e.value.code == dd.DD_ERR_NOMEM
    finally:
        srv.close()


def test_beam_with_bad_search_parameters_is_refused():
    """Widths above the plan's max_width, or a threshold that is not finite, are refused when the
    beam is added, so that no chunk's search can fail after its dedispersion was enqueued."""
    dd.build()
    (w, _), = _beams()[:1]
    srv = dd.Server(max_inflight=2, hbm_budget_bytes=40 << 30)
    try:
        for widths, thr, mw in (((1, 2, 64), w.threshold, 32), (w.widths, float("nan"), None)):
            with pytest.raises(dd.DDError) as e:
                srv.add_beam(w.freqs(), w.tsamp, w.ranges_array(), 4096, widths, thr,
                             max_width=mw)
            assert e.value.code == dd.DD_ERR_ARG
    finally:
        srv.close()
