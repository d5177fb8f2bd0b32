"""The GPU path at the arithmetic limits of its packed and fixed-width sums, against the oracle.

The seeded noise generator stays near 128 +- 6 sigma, so these tests build their inputs here:
all-255 (saturated) bytes and uniform 0..255 bytes, which drive every packed lane to its bound.
Each test names the limit it reaches:
  - the tiled kernel adds two groups' eight-channel sums in 16-bit lanes: 16 x 255 x d, which at
    decimation x16 is 65,280 (the largest value below 2^16 the plan admits);
  - the direct kernel adds uint8 samples in 16-bit lanes flushed every 256 channels:
    256 x 255 = 65,280 per lane before each flush (600 channels: two flushes and a ragged third);
  - the search's uint32 prefix sums wrap, and boxcar sums are exact only below 2^31: with 8192
    channels and 1024-sample boxcars a saturated stretch gives 8192 x 255 x 1024 = 2,139,095,040,
    the largest sum dd_plan admits (nchans x 255 x max(width, decimation) < 2^31);
  - S2 is a 128-bit sum: series near 65,532 x 255 x 16 (tiled, x16) and 8192 x 255 x 256 (direct,
    x256) make S2 pass 2^64 within a few hundred samples, through one CTA and through the
    carries of the tiled kernel's atomics across time tiles.
Series and moments bit-exact, candidates per block (tests/_parity.py).
"""
import numpy as np
import pytest

from synth import configs

torch = pytest.importorskip("torch")
import paper_2101_00941_gb300 as dd  # noqa: E402
from _gpu_check import check, run_gpu  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    dd.build()
    dd.lib()


def _workload(nchans, fch1, foff, tsamp, ranges, widths, nsamp, threshold=6.0):
    w = configs.mid(nsamp=nsamp, chunk_len=4096, n_streams=2, npulses=0, nchans=4096,
                    ranges=ranges, index=50)
    w.nchans, w.fch1, w.foff, w.tsamp = nchans, fch1, foff, tsamp
    w.widths, w.threshold = tuple(widths), threshold
    return w


def _kernels(w, flags=0, chunk_len=4096):
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), chunk_len, n_streams=1,
                   max_width=max(w.widths), flags=flags)
    try:
        return [plan.kernel(r) for r in range(len(w.ranges))], plan.O
    finally:
        plan.close()


def _saturated(nsamp, nchans):
    return np.full((nsamp, nchans), 255, dtype=np.uint8)


def _uniform(nsamp, nchans, seed):
    return np.random.default_rng(seed).integers(0, 256, (nsamp, nchans), dtype=np.uint8)


def _mostly_saturated(nsamp, nchans, seed, frac=0.02):
    """255 everywhere except a random `frac` of the samples, which take a value in 0..254."""
    rng = np.random.default_rng(seed)
    x = _saturated(nsamp, nchans)
    idx = rng.integers(0, x.size, int(x.size * frac))
    x.reshape(-1)[idx] = rng.integers(0, 255, idx.size, dtype=np.uint8)
    return x


# ---------------------------------------------------------------- tiled kernel, 16-bit lanes

def _tiled_x1_x16():
    # 512 channels of 300/1024 MHz from 1550 MHz, 64 us: the tiled kernel's regime for x1 and x16
    return _workload(512, 1550.0, -300.0 / 1024, 64e-6,
                     (configs.DMRange(0.0, 0.0625, 70, 1), configs.DMRange(60.9375, 0.625, 40, 16)),
                     (1, 2, 16, 32, 64), 1 << 14)


@pytest.mark.parametrize("fill", ["saturated", "uniform"])
def test_tiled_kernel_lane_bound_at_x16(fill):
    """Limit: 16 x 255 x 16 = 65,280 in a 16-bit lane (two groups of eight x16-decimated channels
    of 255), and 8 x 255 x 2 per lane of the x1 pair words."""
    w = _tiled_x1_x16()
    kinds, _ = _kernels(w)
    assert [k for k, _ in kinds] == [dd.DD_KERNEL_TILED] * 2
    x = _saturated(w.nsamp, w.nchans) if fill == "saturated" else _uniform(w.nsamp, w.nchans, 1)
    sizes = [4096] * 3 + [2048]
    check(w, x[:sum(sizes)], sizes, 2)
    if fill == "saturated":
        # a constant input dedisperses to C x 255 x d in every output: no variance, no candidates
        out, _, _ = run_gpu(w, x[:sum(sizes)], sizes, 1)
        for series, cands in out[1:]:
            assert cands.size == 0
            for r, (s, _, _) in enumerate(series):
                assert (s == w.nchans * 255 * int(w.ranges[r].decimation)).all()


# ---------------------------------------------------------------- direct kernel, SWAR flush

def _direct_coarse():
    # 600 coarse channels of 1 MHz (1500 -> 901 MHz): too many delay classes for the tiled kernel
    return _workload(600, 1500.0, -1.0, 64e-6,
                     (configs.DMRange(0.0, 1.0, 20, 1), configs.DMRange(20.0, 2.0, 10, 32)),
                     (1, 2, 32, 64), 1 << 15)


@pytest.mark.parametrize("fill", ["saturated", "uniform"])
def test_direct_kernel_swar_flush(fill):
    """Limit: 256 x 255 = 65,280 in a 16-bit SWAR lane before each 256-channel flush (uint8, x1),
    and 600 x 255 x 32 = 4,896,000 in the 32-bit sums of x32 (uint16) data."""
    w = _direct_coarse()
    kinds, O = _kernels(w, chunk_len=8192)
    assert [k for k, _ in kinds] == [dd.DD_KERNEL_DIRECT] * 2
    x = _saturated(w.nsamp, w.nchans) if fill == "saturated" else _uniform(w.nsamp, w.nchans, 2)
    sizes = [8192] * 3
    assert O < 8192
    check(w, x[:sum(sizes)], sizes, 2)


# ---------------------------------------------------------------- search: sums just under 2^31

def test_search_boxcar_sums_at_the_int32_limit():
    """Limit: a saturated stretch of 2048 samples in 8192 channels gives 1024-sample boxcar sums of
    8192 x 255 x 1024 = 2,139,095,040, the largest dd_plan admits (< 2^31); the search's uint32
    prefix sums wrap every ~2000 samples of 2.09e6 each."""
    w = _workload(8192, 1500.0, -500.0 / 8192, 50e-6, (configs.DMRange(0.0, 0.5, 3, 1),),
                  (1, 4, 64, 1024), 1 << 14, threshold=6.0)
    x = _mostly_saturated(w.nsamp, w.nchans, 3, frac=0.2)
    x[11000:13048] = 255  # every channel, every trial's delays (<= 46 samples) inside it
    sizes = [8192, 8192]
    _, O = _kernels(w, chunk_len=8192)
    assert O < 64
    assert check(w, x, sizes, 1) > 0


# ---------------------------------------------------------------- 128-bit S2

def test_moments_pass_2_to_the_64_in_the_tiled_kernel():
    """Limit: y up to 65,532 x 255 x 16 = 267,370,560 (x16 on the tiled kernel), so S2 over a
    320-sample window exceeds 2^64; 256-sample time tiles (DD_FLAG_TILE256) split the window over
    two CTAs, whose partial S2 sums (the first just below 2^64) carry into s2hi through the
    atomics."""
    w = _workload(65532, 1500.0, -500.0 / 65532, 50e-6, (configs.DMRange(0.0, 0.02, 3, 16),),
                  (16, 32), 5120)
    kinds, O = _kernels(w, flags=dd.DD_FLAG_TILE256, chunk_len=5120)
    assert kinds == [(dd.DD_KERNEL_TILED, 256)]
    assert O == 0
    x = _mostly_saturated(w.nsamp, w.nchans, 4, frac=0.01)
    out, _, _ = run_gpu(w, x, [5120], 1, flags=dd.DD_FLAG_TILE256, chunk_len=5120)
    (s, _, m), = out[0][0]
    assert s.shape[1] == 320
    assert all(int(v["s2hi"]) > 0 for v in m)  # past 2^64
    check(w, x, [5120], 1, flags=dd.DD_FLAG_TILE256)


def test_moments_pass_2_to_the_64_in_the_direct_kernel():
    """Limit: y up to 8192 x 255 x 256 = 534,773,760 (x256 on the direct kernel), S2 over a
    96-sample window beyond 2^64 (k_moments' 128-bit sums)."""
    w = _workload(8192, 1500.0, -500.0 / 8192, 50e-6, (configs.DMRange(0.0, 0.05, 3, 256),),
                  (256,), 24576)
    kinds, O = _kernels(w, chunk_len=24576)
    assert kinds == [(dd.DD_KERNEL_DIRECT, 0)]
    assert O == 0
    x = _mostly_saturated(w.nsamp, w.nchans, 5, frac=0.01)
    out, _, _ = run_gpu(w, x, [24576], 1, chunk_len=24576)
    (s, _, m), = out[0][0]
    assert s.shape[1] == 96
    assert all(int(v["s2hi"]) > 0 for v in m)
    check(w, x, [24576], 1)
