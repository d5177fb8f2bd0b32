"""Runs a workload through the GPU library's C ABI chunk by chunk and compares every chunk with
the CPU oracle: delay table and overlap equal, series and moments bit-exact, candidates per block
(tests/_parity.py). Shared by the GPU test files."""
import numpy as np
import torch

import oracle
import paper_2101_00941_gb300 as dd
from _parity import assert_moments_equal, compare_candidates


def _arrivals(w):
    f = w.freqs()
    return lambda dm: oracle.delay_samples(f, w.tsamp, dm)


def _as_input(part, kind):
    if kind == "device":
        return torch.from_numpy(part).cuda()
    if kind == "pinned":
        return torch.from_numpy(part).pin_memory()
    return np.ascontiguousarray(part)  # pageable (copied by the CUDA driver or staging threads)


def run_gpu(w, x, chunk_sizes, n_streams, kind="device", flags=0, want_series=True,
            chunk_len=None, trials=None, block=32):
    ranges = w.ranges_array()
    L = chunk_len or int(-(-max(chunk_sizes) // 256) * 256)
    staging = 4 if kind == "staged" else 0
    plan = dd.Plan(w.freqs(), w.tsamp, ranges, L, n_streams=n_streams, max_width=max(w.widths),
                   peak_block=block, flags=flags, staging_threads=staging)
    out = []
    T = 0
    try:
        for n in chunk_sizes:
            buf = _as_input(x[T:T + n], kind)
            seq = plan.run(buf, n)
            plan.search(w.widths, w.threshold)
            cands = plan.candidates(seq)
            series = []
            if want_series:
                for r in range(len(ranges)):
                    s, j0 = plan.series(r)
                    s = s.cpu().numpy()
                    m, nm = plan.moments(r)
                    assert nm == s.shape[1]
                    if trials is not None:
                        s = s[np.asarray(trials[r])]
                        m = m[np.asarray(trials[r])]
                    if nm == 0:
                        m = m[:0]  # an empty window writes no moments
                    series.append((s, j0, m))
            out.append((series, cands))
            T += n
        O = plan.O
        shifts = plan.shifts
    finally:
        plan.close()
    return out, O, shifts


def check(w, x, chunk_sizes, n_streams, kind="device", trials=None, flags=0, block=32):
    ranges = w.ranges_array()
    gpu, O, shifts = run_gpu(w, x, chunk_sizes, n_streams, kind, trials=trials, flags=flags,
                             block=block)
    ref = oracle.run(x, w.freqs(), w.tsamp, ranges, w.widths, w.threshold, block, chunk_sizes,
                     trials=trials)
    assert O == ref["O"]
    np.testing.assert_array_equal(shifts, np.concatenate(ref["tables"]))
    nmatch = 0
    for k, ((series, cands), per) in enumerate(zip(gpu, ref["chunks"])):
        for r in range(len(ranges)):
            s, j0, m = series[r]
            assert j0 == per[r]["J0"]
            np.testing.assert_array_equal(s, per[r]["series"], err_msg=f"chunk {k} range {r}")
            assert_moments_equal(m, per[r]["moments"], f"chunk {k} range {r}")
        want = np.concatenate([per[r]["cands"] for r in range(len(ranges))])
        got = cands
        if trials is not None:
            keep = np.zeros(got.size, bool)
            for r in range(len(ranges)):
                keep |= (got["range"] == r) & np.isin(got["trial"], trials[r])
            got = got[keep]
        d_of = lambda r: int(ranges[r][3])
        J0_of = lambda r, per=per: per[r]["J0"]
        tr_index = lambda r: {int(t): i for i, t in enumerate(per[r]["trials"])}
        series_of = lambda r, t, per=per: per[r]["series"][tr_index(r)[t]]
        nmatch += compare_candidates(got, want, w.threshold, block, series_of, J0_of, d_of)
    return nmatch


def oracle_candidates_match(w, x, chunk_sizes, got_per_chunk, block=32):
    """Run the oracle over the chunks and compare each chunk's candidates (sorted by the library:
    range, trial, t_start, width) with it, per block (tests/_parity.py). Returns the number of
    matched blocks."""
    ranges = w.ranges_array()
    ref = oracle.run(x[:sum(chunk_sizes)], w.freqs(), w.tsamp, ranges, w.widths, w.threshold,
                     block, chunk_sizes)
    assert len(got_per_chunk) == len(ref["chunks"])
    nmatch = 0
    for got, per in zip(got_per_chunk, ref["chunks"]):
        want = np.concatenate([per[r]["cands"] for r in range(len(ranges))])
        d_of = lambda r: int(ranges[r][3])
        J0_of = lambda r, per=per: per[r]["J0"]
        series_of = lambda r, t, per=per: per[r]["series"][t]
        nmatch += compare_candidates(got, want, w.threshold, block, series_of, J0_of, d_of)
    return nmatch
