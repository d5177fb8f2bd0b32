"""The C-ABI library builds, loads and exports every entry point include/dd.h declares.

Runs without a GPU: only argument validation that precedes any CUDA call is
exercised here; everything that computes is in the -m gpu tests.
"""
import ctypes
import os
import re

import pytest

import paper_2101_00941_gb300 as dd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_\w+|sps_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    dd.build()
    return dd.lib()


def test_exports_every_declared_function(lib):
    names = _declared()
    assert {"dd_plan", "dd_run", "sps_run", "dd_candidates", "dd_last_error"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    assert set(dd.EXPORTS) <= set(names)


def test_header_structs_match_binding():
    src = open(os.path.join(ROOT, "include", "dd.h")).read()
    assert ctypes.sizeof(dd.dd_range_t) == 24
    assert ctypes.sizeof(dd.dd_opts_t) == 40
    assert dd.CAND_DTYPE.itemsize == 32
    for k in ("DD_ERR_ARG (-1)", "DD_ERR_STATE (-6)", "DD_FLAG_TIMING 1u"):
        assert k in src


def _opts(**kw):
    o = dict(chunk_len=4096, n_streams=2, max_width=32, peak_block=32, device=0, max_cands=0,
             flags=0, staging_threads=0)
    o.update(kw)
    return dd.dd_opts_t(**o)


def _plan(lib, nchans=16, freqs=None, ranges=((0.0, 1.0, 8, 1),), **kw):
    f = (ctypes.c_double * nchans)(*(freqs or [1500.0 - i for i in range(nchans)]))
    rr = (dd.dd_range_t * len(ranges))(*[dd.dd_range_t(*r) for r in ranges])
    h = ctypes.c_void_p()
    o = _opts(**kw)
    return lib.dd_plan(f, nchans, ctypes.c_double(64e-6), rr, len(ranges), ctypes.byref(o),
                       ctypes.byref(h))


@pytest.mark.parametrize("kw", [
    dict(nchans=0), dict(chunk_len=1000), dict(n_streams=0), dict(n_streams=17),
    dict(max_width=0), dict(peak_block=3), dict(peak_block=64),
    dict(ranges=((0.0, 1.0, 8, 3),)), dict(ranges=((0.0, 1.0, 0, 1),)),
    dict(ranges=((-1.0, 1.0, 8, 1),)), dict(freqs=[1500.0, -1.0] + [1400.0] * 14),
    dict(nchans=8192, max_width=1024), dict(staging_threads=-1), dict(staging_threads=65),
    dict(chunk_len=1 << 24), dict(ranges=((0.0, 1.0, 65536, 1),)),
])
def test_invalid_plans_are_rejected_before_any_gpu_work(lib, kw):
    assert _plan(lib, **kw) == dd.DD_ERR_ARG
    assert len(lib.dd_last_error()) > 0


def test_null_handles(lib):
    assert lib.dd_run(None, None, 0, None) == dd.DD_ERR_ARG
    assert lib.sps_run(None, None, 0, ctypes.c_float(6.0)) == dd.DD_ERR_ARG
    assert lib.dd_sync(None) == dd.DD_ERR_ARG
    assert lib.dd_plan_kernel(None, 0, None, None) == dd.DD_ERR_ARG
    assert lib.dd_selftest_wait(0, None, None) == dd.DD_ERR_ARG
    lib.dd_plan_destroy(None)


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(dd, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(dd, "_lib", None)
    with pytest.raises(RuntimeError):
        dd.lib()
