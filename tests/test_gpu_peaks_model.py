"""The measured roofline denominators (dd_measure_peaks) and the launch model (dd_plan_model).

The peaks are measured on the device, so this checks that they are physically plausible for one
SM: at most 4 warp-instructions (128 lanes) issued per clock, and at most a few 128-byte
shared-memory wavefronts per clock. The model's counts are checked for their invariants: adds are
one per channel per output, the tiled kernel's shared-memory work grows with whole time tiles, and
kernels that stage nothing in shared memory report none.
"""
import pytest

from synth import configs

torch = pytest.importorskip("torch")
import paper_2101_00941_gb300 as dd  # noqa: E402

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    dd.build()
    p = dd.dd_measure_peaks(0)
    assert p["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 300.0 < p["sm_mhz"] < 4000.0
    for k in ("alu_lanes_per_clk", "dp_lanes_per_clk", "int_lanes_per_clk", "add_per_clk"):
        assert 8.0 <= p[k] <= 260.0, (k, p[k])
    assert p["int_lanes_per_clk"] <= 128.0 * 1.02  # issue: 4 warp-instructions per SM-clock
    assert p["int_lanes_per_clk"] >= 0.9 * max(p["alu_lanes_per_clk"], p["dp_lanes_per_clk"])
    assert 0.2 <= p["lds_wavefronts_per_clk"] <= 4.0


def test_launch_model_invariants():
    dd.build()
    w = configs.mid(nsamp=1 << 16)
    ranges = w.ranges_array()
    plan = dd.Plan(w.freqs(), w.tsamp, ranges, 1 << 16, n_streams=1, max_width=max(w.widths))
    try:
        for r in range(len(ranges)):
            kind, tt = plan.kernel(r)
            m1 = plan.model(r, tt)
            assert m1["kind"] == kind and m1["tile_samples"] == tt
            assert m1["outputs"] == int(ranges[r][2]) * tt
            assert m1["adds"] == m1["outputs"] * w.nchans
            assert m1["dram_bytes"] >= 4 * m1["outputs"]
            if kind == dd.DD_KERNEL_TILED:
                assert m1["smem_wavefronts"] > 0 and m1["copy_bytes"] > 0
                # a partial time tile costs a whole one; 3 tiles cost 3 times one
                m_part = plan.model(r, tt + 1)
                m3 = plan.model(r, 3 * tt)
                assert m_part["smem_wavefronts"] == 2 * m1["smem_wavefronts"]
                assert m3["smem_wavefronts"] == 3 * m1["smem_wavefronts"]
                # the accumulation alone: 16 warps x 4 trials x tt/64 words x 2 groups per stage
                stages = (w.nchans // 8 + 1) // 2
                tiles = -(-int(ranges[r][2]) // 64)
                assert m1["smem_wavefronts"] >= tiles * stages * 16 * 4 * (tt // 64) * 2
            assert plan.model(r, 0)["smem_wavefronts"] == 0
    finally:
        plan.close()
    t = configs.tiny()
    plan = dd.Plan(t.freqs(), t.tsamp, t.ranges_array(), 4096, n_streams=1)
    try:
        m = plan.model(0, 4096)
        assert m["kind"] == dd.DD_KERNEL_DIRECT and m["smem_wavefronts"] == 0
    finally:
        plan.close()
