"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package makes input data only: 8-bit time-major filterbanks with
Gaussian-like noise and boxcar pulses whose per-channel arrival samples the
caller supplies. It contains none of the dedispersion or search arithmetic.
The C kernel in ``synth.c`` is built with gcc on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``_build/libsynth.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_filterbank.restype = None
            lib.synth_filterbank.argtypes = [
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            _lib = lib
    return _lib


class Pulse:
    """A boxcar pulse: first sample per channel, width in samples, amplitude per channel.

    ``amp`` is in LSB of the 8-bit data and may be fractional (it is carried in
    1/4096 LSB, so sub-LSB amplitudes are dithered by the noise).
    """

    def __init__(self, arrival, width: int, amp: float):
        self.arrival = np.ascontiguousarray(arrival, dtype=np.int64)
        self.width = int(width)
        self.amp = float(amp)

    @property
    def amp_q12(self) -> int:
        return int(round(self.amp * 4096.0))


def filterbank(nsamp: int, nchans: int, seed: int, beam: int = 0, pulses=(), t0: int = 0,
               out: np.ndarray | None = None) -> np.ndarray:
    """Return (or fill) a uint8 array [nsamp][nchans] covering samples [t0, t0+nsamp).

    ``out`` may be any C-contiguous uint8 buffer of that size (for example a
    pinned host tensor's numpy view); it is filled in place.
    """
    lib = _load()
    if out is None:
        out = np.empty((nsamp, nchans), dtype=np.uint8)
    assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size == nsamp * nchans
    pulses = list(pulses)
    npul = len(pulses)
    if npul:
        arr = np.ascontiguousarray(np.stack([p.arrival for p in pulses]), dtype=np.int64)
        assert arr.shape == (npul, nchans)
        wid = np.array([p.width for p in pulses], dtype=np.int32)
        amp = np.array([p.amp_q12 for p in pulses], dtype=np.int32)
        pa, pw, pq = arr.ctypes.data, wid.ctypes.data, amp.ctypes.data
    else:
        pa = pw = pq = None
    lib.synth_filterbank(out.ctypes.data, int(t0), int(nsamp), int(nchans), int(seed), int(beam),
                         npul, pa, pw, pq)
    return out
