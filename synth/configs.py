"""Workload definitions (sizes, frequency setup, DM-trial plans, pulse draws).

These describe synthetic inputs shaped like an SKA-like survey beam: 8-bit
data, 64 us sampling, 1024-8192 channels over 200-500 MHz of band. Pulses are
drawn here as (DM, reference arrival sample, width, amplitude); turning a DM
into per-channel arrival samples is left to the caller, so this module holds
none of the dedispersion arithmetic.

Seeds are 210100941 + the workload's index (+ the beam index for multi-beam
workloads).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Sequence

import numpy as np

from . import Pulse, filterbank

SEED_BASE = 210100941


@dataclasses.dataclass(frozen=True)
class DMRange:
    dm_start: float
    dm_step: float
    n_trials: int
    decimation: int


@dataclasses.dataclass(frozen=True)
class PulseSpec:
    dm: float          # pc cm^-3
    t_ref: int         # first sample at the highest channel frequency
    width: int         # samples
    amp: float         # LSB per channel per sample


@dataclasses.dataclass
class Workload:
    name: str
    index: int
    nchans: int
    fch1: float        # MHz, frequency of channel 0 (the highest)
    foff: float        # MHz per channel (negative: descending)
    tsamp: float       # s
    nsamp: int
    ranges: Sequence[DMRange]
    widths: Sequence[int]   # boxcar widths in original samples
    threshold: float
    chunk_len: int
    n_streams: int
    pulses: Sequence[PulseSpec] = ()
    beam: int = 0

    @property
    def seed(self) -> int:
        return SEED_BASE + self.index

    def freqs(self) -> np.ndarray:
        """Channel-centre frequencies in MHz, f_c = fch1 + c * foff."""
        return self.fch1 + np.arange(self.nchans, dtype=np.float64) * self.foff

    def ranges_array(self) -> np.ndarray:
        return np.array([(r.dm_start, r.dm_step, r.n_trials, r.decimation) for r in self.ranges],
                        dtype=np.float64)

    @property
    def n_trials(self) -> int:
        return sum(r.n_trials for r in self.ranges)

    @property
    def d_max(self) -> int:
        return max(r.decimation for r in self.ranges)

    def make_pulses(self, arrival_offsets: Callable[[float], np.ndarray]) -> List[Pulse]:
        """Pulses for the generator; ``arrival_offsets(dm)`` gives per-channel delays in samples."""
        out = []
        for p in self.pulses:
            off = np.asarray(arrival_offsets(p.dm), dtype=np.int64)
            out.append(Pulse(p.t_ref + off, p.width, p.amp))
        return out

    def generate(self, arrival_offsets: Callable[[float], np.ndarray] | None = None, t0: int = 0,
                 nsamp: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
        """Time-major uint8 filterbank [nsamp][nchans] for samples [t0, t0+nsamp)."""
        n = self.nsamp - t0 if nsamp is None else nsamp
        pulses = self.make_pulses(arrival_offsets) if (arrival_offsets and self.pulses) else ()
        return filterbank(n, self.nchans, self.seed, self.beam, pulses, t0=t0, out=out)


def _snr_amp(snr: float, width: int, nchans: int) -> float:
    # A boxcar of `width` samples at amplitude a in every channel sums to a*width*nchans against
    # noise of sd 16*sqrt(width*nchans) in the same sum.
    return snr * 16.0 / math.sqrt(width * nchans)


MID_RANGES = (DMRange(0.0, 0.1, 1500, 1), DMRange(150.0, 0.2, 750, 2),
              DMRange(300.0, 0.25, 800, 4), DMRange(500.0, 0.5, 1000, 8))


def tiny() -> Workload:
    """64 channels, 1500 MHz down by 1.5625 MHz, 64 us, 65536 samples, DM 0-400 step 1."""
    w = 16  # 1 ms at 64 us
    pulses = (PulseSpec(50.0, 8192, w, 24.0), PulseSpec(150.0, 24576, w, 24.0),
              PulseSpec(300.0, 40960, w, 24.0))
    return Workload("tiny_64ch_65536", 0, 64, 1500.0, -1.5625, 64e-6, 65536,
                    (DMRange(0.0, 1.0, 401, 1),), (1, 2, 4, 8, 16, 32), 6.0, 65536, 1, pulses)


def mid(nsamp: int = 1 << 20, chunk_len: int = 1 << 17, n_streams: int = 4, npulses: int = 20,
        nchans: int = 4096, ranges: Sequence[DMRange] = MID_RANGES, index: int = 1,
        beam: int = 0) -> Workload:
    """4096 channels over 1250-1550 MHz, 64 us, 2^20 samples, DM 0-1000 with x1..x8 decimation."""
    rng = np.random.default_rng(SEED_BASE + index + 1000 * beam)
    pulses = []
    for _ in range(npulses):
        dm = float(rng.uniform(0.0, 1000.0))
        width = int(round(math.exp(rng.uniform(0.0, math.log(256.0)))))
        snr = float(rng.uniform(8.0, 30.0))
        t_ref = int(rng.integers(0, max(1, nsamp - 20000)))
        pulses.append(PulseSpec(dm, t_ref, width, _snr_amp(snr, width, nchans)))
    foff = -300.0 / 4096 if nchans == 4096 else -200.0 / nchans
    fch1 = 1550.0 if nchans == 4096 else 1450.0
    return Workload(f"mid_{nchans}ch_{nsamp}", index, nchans, fch1, foff, 64e-6, nsamp, tuple(ranges),
                    (1, 2, 4, 8, 16, 32, 64, 128, 256), 6.0, chunk_len, n_streams, tuple(pulses), beam)


def batched_beams(nbeams: int = 48, seed_index: int = 2) -> List[Workload]:
    """Beams of log-uniform length 2^18-2^21 (multiples of 128), 1024 or 4096 channels, DM 0-500."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    out = []
    for b in range(nbeams):
        n = int(2 ** rng.uniform(18, 21)) // 128 * 128
        nch = 4096 if rng.integers(0, 2) else 1024
        out.append(mid(nsamp=n, chunk_len=n, n_streams=1, npulses=5, nchans=nch,
                       ranges=MID_RANGES[:3], index=seed_index, beam=b))
    return out


def out_of_core(nsamp: int = 1 << 25) -> Workload:
    """8192 channels over 1000-1500 MHz, 50 us, 2^25 samples, DM 0-3000 with x1..x16 decimation."""
    ranges = MID_RANGES + (DMRange(1000.0, 1.0, 2000, 16),)
    w = mid(nsamp=nsamp, chunk_len=1 << 19, n_streams=4, npulses=20, nchans=8192, ranges=ranges, index=4)
    w.name = f"ooc_8192ch_{nsamp}"
    w.fch1, w.foff, w.tsamp = 1500.0, -500.0 / 8192, 50e-6
    w.widths = (1, 2, 4, 8, 16, 32, 64, 128, 256, 512)
    return w
