"""Batched execution (dd_batch_*): beams of different channel counts and lengths processed in
one step -- directly, as a replayed CUDA graph, and with autotuned tiles -- give for every
(beam, chunk) the oracle's candidates (per block, tests/_parity.py) and exactly the candidates of
that beam processed alone."""
import numpy as np
import pytest

import oracle
from synth import configs

torch = pytest.importorskip("torch")
import paper_2101_00941_gb300 as dd  # noqa: E402
from _gpu_check import oracle_candidates_match  # noqa: E402

pytestmark = pytest.mark.gpu

RANGES = (configs.DMRange(0.0, 2.0, 40, 1), configs.DMRange(80.0, 4.0, 30, 2),
          configs.DMRange(200.0, 5.0, 20, 4))


def _beams():
    out = []
    for k, (nch, nsamp) in enumerate(((128, 12288), (64, 20480), (96, 8192), (128, 16384))):
        w = configs.mid(nsamp=nsamp, chunk_len=4096, n_streams=1, npulses=3, nchans=4096,
                        ranges=RANGES, index=30 + k)
        w.nchans = nch
        w.foff = -300.0 / nch
        w.pulses = tuple(configs.PulseSpec(p.dm * 0.3, min(p.t_ref, nsamp - 6000), p.width,
                                           p.amp * 4) for p in w.pulses)
        w.threshold = 5.0
        f = w.freqs()
        x = w.generate(lambda dm, f=f, w=w: oracle.delay_samples(f, w.tsamp, dm))
        out.append((w, x))
    return out


def _sizes(w):
    return [min(4096, w.nsamp - k) for k in range(0, w.nsamp, 4096)]


def _alone(w, x):
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, n_streams=1,
                   max_width=max(w.widths))
    xs = torch.from_numpy(x).cuda()
    res = []
    try:
        for k in range(0, x.shape[0], 4096):
            seq = plan.run(xs[k:k + 4096], min(4096, x.shape[0] - k))
            plan.search(w.widths, w.threshold)
            res.append(plan.candidates(seq))
    finally:
        plan.close()
    return res


@pytest.mark.parametrize("mode", ["direct", "graph", "autotune", "persistent"])
def test_batch_equals_each_beam_alone(mode):
    dd.build()
    beams = _beams()
    want = [_alone(w, x) for w, x in beams]
    w0 = beams[0][0]
    dev = [torch.from_numpy(x).cuda() for _, x in beams]
    b = dd.Batch([(w.freqs(), w.tsamp, d) for (w, _), d in zip(beams, dev)],
                 w0.ranges_array(), 4096, w0.widths, w0.threshold, n_streams=2,
                 graph=mode == "graph", autotune=mode == "autotune",
                 persistent=mode == "persistent")
    try:
        matched = 0
        for step in range(2):  # a second step (graph replay) gives the same results
            b.run()
            b.wait()
            for i, (w, x) in enumerate(beams):
                nchunks, outputs, tile = b.info(i)
                assert nchunks == len(want[i])
                got = [b.candidates(i, k) for k in range(nchunks)]
                for k in range(nchunks):
                    np.testing.assert_array_equal(got[k], want[i][k])
                if step == 1:
                    matched += oracle_candidates_match(w, x, _sizes(w), got)
        assert sum(c.size for ws in want for c in ws) > 0 and matched > 0
    finally:
        b.close()


def test_device_input_plans_refuse_host_chunks():
    dd.build()
    (w, x), = _beams()[:1]
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 4096, flags=dd.DD_FLAG_DEVICE_INPUT)
    try:
        with pytest.raises(dd.DDError) as e:
            plan.run(np.ascontiguousarray(x[:4096]), 4096)
        assert e.value.code == dd.DD_ERR_ARG
    finally:
        plan.close()


@pytest.mark.parametrize("graph,persistent", [(False, False), (True, False), (False, True),
                                              (True, True)])
def test_batch_of_tiled_beams(graph, persistent):
    """Beams of 256 fine channels whose ranges (x1, x2) run on the tiled kernel, whose error
    bits a batch collects in a word of its own: the step reports that word clean, and every
    (beam, chunk) has exactly the candidates of the beam alone -- also when each round's tiles
    of every beam and range are taken from one work list by a persistent launch, directly and
    as a replayed graph."""
    dd.build()
    ranges = (configs.DMRange(0.0, 0.0625, 70, 1), configs.DMRange(4.375, 0.125, 40, 2))
    beams = []
    for k, nsamp in enumerate((12288, 8192, 6144)):
        w = configs.mid(nsamp=nsamp, chunk_len=4096, n_streams=1, npulses=3, nchans=4096,
                        ranges=ranges, index=40 + k)
        w.nchans, w.foff = 256, -300.0 / 1024
        w.pulses = (configs.PulseSpec(2.5 + 3 * k, 3000, 8, 20 * 16.0 / (8 * 256) ** 0.5),
                    configs.PulseSpec(6.0, nsamp - 2500, 16, 20 * 16.0 / (16 * 256) ** 0.5))
        f = w.freqs()
        x = w.generate(lambda dm, f=f, w=w: oracle.delay_samples(f, w.tsamp, dm))
        beams.append((w, x))
    want = [_alone(w, x) for w, x in beams]
    w0 = beams[0][0]
    dev = [torch.from_numpy(x).cuda() for _, x in beams]
    b = dd.Batch([(w.freqs(), w.tsamp, d) for (w, _), d in zip(beams, dev)],
                 w0.ranges_array(), 4096, w0.widths, w0.threshold, n_streams=2, graph=graph,
                 persistent=persistent)
    try:
        matched = 0
        for step in range(2):
            b.run()
            b.wait()
            for i, (w, x) in enumerate(beams):
                nchunks, _, tile = b.info(i)
                assert tile > 0  # range 0 runs on the tiled kernel
                assert nchunks == len(want[i])
                got = [b.candidates(i, k) for k in range(nchunks)]
                for k in range(nchunks):
                    np.testing.assert_array_equal(got[k], want[i][k])
                if step == 1:
                    matched += oracle_candidates_match(w, x, _sizes(w), got)
        assert sum(c.size for ws in want for c in ws) > 0 and matched > 0
    finally:
        b.close()
