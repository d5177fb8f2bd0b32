"""bench.py prints one JSON line with the fields its consumers read.

The reference arm (the CPU oracle on the host cores) runs here without a GPU; the GPU arm runs
on a short 2-chunk beam of the 4096-channel workload.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--workload", "mid", "--steps", "1", "--warmup", "0"],
             timeout=900)
    assert d["impl"] == "reference"
    assert d["metric"] == "DM-trial·samples/s dedispersed" and d["unit"] == "DM-trial·samples/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["config"]["workload"] == "mid_4096ch_1048576"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "trials per range" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_gpu_arm_line():
    """The default (out-of-core) workload on a 2-chunk beam: every key of the contract, a
    roofline against the measured peaks with per-range shared-memory fractions, clocks."""
    pytest.importorskip("torch")
    d = _run(["--steps", "3", "--warmup", "3", "--nsamp", str(2 << 19), "--streams", "2",
              "--no-cpu-baseline"], timeout=1200)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "gpu_launches", "roofline", "clocks"):
        assert k in d, k
    assert d["config"]["workload"] == "ooc_8192ch_1048576" and d["config"]["nchans"] == 8192
    assert d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 3 and d["gpu_launches"] > 0
    assert d["e2e"]["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == (2 << 19) * 8192
    assert "exposed_copy_ms_per_chunk" in d["e2e"] and "chunk_latency_ms" in d["e2e"]
    assert d["input_equivalent"]["value"] > d["value"]  # decimated ranges count d_r samples
    r = d["roofline"]
    assert r["bound"] == "alu" and 0 < r["frac"] < 2 and r["peak"] > 0
    assert 0 < r["frac_smem"] < 1.5
    assert len(r["per_range"]) == 5 and all(p["frac_smem"] for p in r["per_range"])
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_metric_counts_the_outputs_of_the_chunk_windows():
    """The benchmark's DM-trial·samples (outputs_of_chunks) equal the outputs of the chunk
    windows as the oracle lays them out, from the first sample and for a stream that continues
    past its warm-up steps (full windows)."""
    import oracle
    from synth import configs
    bench = _bench_module()
    w = configs.mid()
    ranges = w.ranges_array()
    O = oracle.overlap(oracle.shift_tables(w.freqs(), w.tsamp, ranges), ranges)
    assert O == 14496
    sizes = [w.chunk_len] * (w.nsamp // w.chunk_len)
    for steps_before in (0, 3):
        all_sizes = sizes * (steps_before + 1)
        wins = oracle.chunk_windows(all_sizes, O)[len(sizes) * steps_before:]
        produced = sum(int(r[2]) * (hi // int(r[3]) - lo // int(r[3]))
                       for (_, _, lo, hi) in wins for r in ranges)
        assert bench.outputs_of_chunks(w, O, steps_before * w.nsamp, sizes) == produced
    # a continuing stream's step produces every range's full N / d_r outputs per trial
    assert bench.outputs_of_chunks(w, O, 3 * w.nsamp, sizes) == \
        sum(r.n_trials * (w.nsamp // r.decimation) for r in w.ranges)
    # counted at the original sampling, every trial covers the whole N samples
    assert bench.outputs_of_chunks(w, O, 3 * w.nsamp, sizes, input_equivalent=True) == \
        w.n_trials * w.nsamp
