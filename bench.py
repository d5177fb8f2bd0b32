#!/usr/bin/env python3
"""Benchmark: streamed brute-force dedispersion + boxcar single-pulse search on GB300.

Default workload (the out-of-core beam): 8192 channels over 1000-1500 MHz, 50 us sampling,
2^25 uint8 samples (275 GB, more than the GPU's memory), 6050 DM trials over 0-3000 pc cm^-3
with x1/x2/x4/x8/x16 decimation, boxcars 1..512 at 6 sigma. One step = the whole beam: 64 chunks
of 2^19 samples over 4 CUDA streams, each chunk corner-turned, decimated, dedispersed, searched
and its candidates copied to the host. The input is a ring of 8 distinct seeded 2^19-sample
chunks (4.3 GB each), reused cyclically to make up the 2^25 samples.

  value : DM-trial*samples/s with the ring resident in HBM
  e2e   : the same through the C ABI from the ring in pinned HOST memory (H2D inside the step)

`--workload mid` is the 4096-channel, 2^20-sample beam (4050 trials over 0-1000, x1..x8, 8 chunks
of 2^17 over 4 streams); serve, batch, transfer and peaks are the other workloads.
Timing: CUDA events around the timed steps with a device synchronize on both sides, W warm-up
steps; every chunk (4.3 GB) is larger than L2, so no flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torchrun: one independent beam per rank (weak scaling), max of the
per-rank step times.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import configs  # noqa: E402

METRIC = "DM-trial·samples/s dedispersed"
UNIT = "DM-trial·samples/s"
# DRAM bytes over algorithmic bytes of the dedispersion launches, from one ncu capture; valid only
# for the kernel source it was taken on (its SHA-256 is stored beside the figures)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dedisp_dram_traffic.json")
TRAFFIC_FILE_FUSED = os.path.join(ROOT, "profiles", "dedisp_fused_dram_traffic.json")
DEDISP_SOURCE = os.path.join(ROOT, "paper_2101_00941_gb300", "csrc", "dd_dedisp.cu")


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_max(values, device):
    """Element-wise max over ranks of per-rank timings (a multi-GPU step lasts as long as its
    slowest rank); the values unchanged with one process."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if tdist.is_available() and tdist.is_initialized() and tdist.get_world_size() > 1:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def pulse_offsets(w):
    """Per-channel arrival offsets (samples) of a pulse at a given DM, for input synthesis."""
    f = w.freqs()
    fref = f.max()

    def off(dm):
        return np.floor(4.148808e3 * dm * (1.0 / f ** 2 - 1.0 / fref ** 2) / w.tsamp + 0.5
                        ).astype(np.int64)
    return off


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def run_step(plan, chunks, w, lat=None):
    """Enqueue every chunk (4-deep pipeline over the plan's streams) and collect candidates."""
    import paper_2101_00941_gb300 as dd
    S = w.n_streams
    ncand = 0
    t_sub = {}
    for k, c in enumerate(chunks):
        t_sub[k] = time.perf_counter()
        seq = plan.run(c, c.shape[0])
        plan.search(w.widths, w.threshold)
        if k >= S - 1:
            j = seq - (S - 1)
            ncand += dd.dd_candidates(plan.h, j).size
            if lat is not None:
                lat.append(time.perf_counter() - t_sub[k - (S - 1)])
    for j in range(max(0, len(chunks) - (S - 1)), len(chunks)):
        seq = plan.seq - (len(chunks) - 1 - j)
        ncand += dd.dd_candidates(plan.h, seq).size
        if lat is not None:
            lat.append(time.perf_counter() - t_sub[j])
    return ncand


def time_steps(plan, chunks, w, steps, warmup, barrier, lat=None):
    import torch
    for _ in range(warmup):
        run_step(plan, chunks, w)
    plan.sync()
    plan.stats(reset=True)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ncand = 0
    for _ in range(steps):
        ncand += run_step(plan, chunks, w, lat)
    plan.sync()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    launches, dd_ms, dd_n = plan.stats()
    return ms, ncand, launches, dd_ms, dd_n


def stream_workload(name: str, nsamp: int | None = None, beam: int = 0, streams: int = 4):
    """(workload, chunks in the input ring) of a streamed workload: the out-of-core beam (8192
    channels, DM 0-3000) or the 4096-channel beam (DM 0-1000)."""
    if name == "ooc":
        L = 1 << 19
        ring = 8
        # pulses are drawn over the ring's samples so that they land in it
        w = configs.out_of_core(nsamp=ring * L)
        w.beam = beam
        w.nsamp = nsamp or (1 << 25)
        w.name = f"ooc_8192ch_{w.nsamp}"
        w.chunk_len, w.n_streams = L, streams
        return w, min(ring, w.nsamp // L)
    w = configs.mid(beam=beam, nsamp=nsamp or (1 << 20), n_streams=streams)
    return w, w.nsamp // w.chunk_len


def baseline_window(w, O):
    """(first global sample, samples) of the CPU baseline's input: one window of up to 65536
    outputs starting where the second chunk's window starts (L - O), with the O samples of
    history its outputs read."""
    L = w.chunk_len
    win = min(L, 1 << 16)
    return L - O, O + win


def cpu_baseline(w, x_win, t_in0, O, target_s: float = 15.0):
    """The oracle, as it stands, on a bounded sample of the same workload: every range, a few
    trials spread over the range, over one window of up to 65536 samples with full history.
    x_win holds global samples [t_in0, t_in0 + len); t_in0 = L - O. Returns DM-trial*samples/s."""
    import oracle
    oracle.build()
    f = w.freqs()
    ranges = w.ranges_array()
    tabs = oracle.shift_tables(f, w.tsamp, ranges)
    lo = t_in0
    hi = t_in0 + x_win.shape[0] - O
    ntr = 8
    done_out, elapsed = 0, 0.0
    while elapsed < target_s and ntr <= 4096:
        t0 = time.perf_counter()
        outs = 0
        for r, tab in enumerate(tabs):
            d = int(ranges[r][3])
            tr = np.linspace(0, tab.shape[0] - 1, min(ntr, tab.shape[0])).astype(np.int32)
            J0, J1 = lo // d, hi // d
            xd = oracle.decimate(x_win, t_in0, d, J0, J1 - J0 + int(tab.max()))
            y = oracle.dedisperse(xd, J0, tab, tr, J0, J1 - J0)
            oracle.sps(y, tr, r, d, J0, oracle.widths_for_range(w.widths, d), 32, w.threshold)
            outs += tr.size * (J1 - J0)
        dt = time.perf_counter() - t0
        done_out, elapsed = outs, dt
        if dt * 4 > target_s:
            break
        ntr *= 4
    per_range = "/".join(str(r.n_trials) for r in w.ranges)
    return {"value": done_out / elapsed, "unit": UNIT, "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{done_out} DM-trial*samples: {ntr} trials per range (of {per_range}) over "
                      f"a {hi - lo}-sample window with full history, dedispersion + search, "
                      f"{elapsed:.1f} s"}


def main_reference(args):
    """The reference arm: the CPU oracle timed on the host cores on this arm's workload, each
    step a bounded sample of it (rank 0 only)."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    w, nring = stream_workload(args.workload if args.workload in ("mid", "ooc") else "ooc")
    import oracle
    f = w.freqs()
    O = oracle.overlap(oracle.shift_tables(f, w.tsamp, w.ranges_array()), w.ranges_array())
    t_in0, n = baseline_window(w, O)
    x = w.generate(pulse_offsets(w), t0=t_in0, nsamp=n)
    for _ in range(args.warmup):
        cpu_baseline(w, x, t_in0, O, target_s=2.0)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, x, t_in0, O, target_s=8.0))
    wall = time.perf_counter() - t0
    value = float(np.mean([v["value"] for v in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/i32",
            "data": "synthetic", "config": {"workload": w.name, "nchans": w.nchans,
                                           "nsamp": w.nsamp, "trials": w.n_trials},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": vals[-1]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def serve_workload(args):
    """16 beams, 4096 channels, the full DM 0-1000 plan, chunks of 2^16 samples (10% 2^17)
    arriving as Poisson streams; the served loop against the plain per-chunk loop."""
    import torch

    import paper_2101_00941_gb300 as dd
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    dd.build()
    nbeams, cadence_s = args.beams, (1 << 16) * 64e-6
    rng = np.random.default_rng(configs.SEED_BASE + 3)
    beams, pools = [], []
    for b in range(nbeams):
        w = configs.mid(nsamp=(1 << 17) * 2, chunk_len=1 << 17, n_streams=2, npulses=5,
                        index=3, beam=b)
        beams.append(w)
        # a pool of two distinct seeded 2^17-sample chunks per beam, reused cyclically
        x = torch.empty(((1 << 17) * 2, w.nchans), dtype=torch.uint8, pin_memory=True)
        w.generate(pulse_offsets(w), out=x.numpy())
        pools.append(x)
    # arrivals: per beam a Poisson stream at cadence/speedup; 10% of chunks are 2^17 long
    arr = []
    for b in range(nbeams):
        t = 0.0
        for k in range(args.chunks_per_beam):
            t += rng.exponential(cadence_s / args.speedup)
            n = (1 << 17) if rng.random() < 0.1 else (1 << 16)
            arr.append((t, b, k, n))
    arr.sort()
    outs = {b: 0 for b in range(nbeams)}

    def view(b, k, n):
        base = (k % 2) * (1 << 17)
        return pools[b][base:base + n]

    def outputs(w, n, O, T):
        lo, hi = max(0, T - O), max(0, T + n - O)
        return sum(r.n_trials * ((hi // r.decimation) - (lo // r.decimation)) for r in w.ranges)

    # ---- served loop
    srv = dd.Server(max_inflight=args.inflight, hbm_budget_bytes=200 << 30, device=dev)
    ids = [srv.add_beam(w.freqs(), w.tsamp, w.ranges_array(), 1 << 17, w.widths, w.threshold,
                        n_streams=2) for w in beams]
    O = dd.Plan(beams[0].freqs(), beams[0].tsamp, beams[0].ranges_array(), 1 << 17).O
    lat, done_outputs, T = [], 0, {b: 0 for b in range(nbeams)}
    torch.cuda.synchronize()
    clk = ClockSampler(dev).__enter__()
    t0 = time.perf_counter()
    pending = 0
    for (ta, b, k, n) in arr:
        while time.perf_counter() - t0 < ta:
            for r, _ in srv.poll(64, timeout_ms=0):
                lat.append(r["latency_ms"])
                pending -= 1
            time.sleep(0.0005)
        srv.submit(ids[b], view(b, k, n), n)
        done_outputs += outputs(beams[b], n, O, T[b])
        T[b] += n
        pending += 1
    while pending > 0:
        for r, _ in srv.poll(64, timeout_ms=1000):
            lat.append(r["latency_ms"])
            pending -= 1
    served_s = time.perf_counter() - t0
    clk.__exit__()
    srv.close()
    # ---- plain per-chunk loop: one stream per beam, each chunk copied, dedispersed,
    #      searched and synchronised before the next one starts
    plans = [dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 1 << 17, n_streams=1,
                     max_width=max(w.widths)) for w in beams]
    plain_lat = []
    torch.cuda.synchronize()
    clk_plain = ClockSampler(dev).__enter__()
    t0 = time.perf_counter()
    for (ta, b, k, n) in arr:
        while time.perf_counter() - t0 < ta:
            time.sleep(0.0005)
        t_arr = t0 + ta
        p = plans[b]
        p.run(view(b, k, n), n)
        p.search(beams[b].widths, beams[b].threshold)
        p.candidates()
        plain_lat.append(1e3 * (time.perf_counter() - t_arr))
    plain_s = time.perf_counter() - t0
    clk_plain.__exit__()
    for p in plans:
        p.close()
    obs = sum(n for (_, _, _, n) in arr) * 64e-6
    line = {
        "metric": METRIC, "value": done_outputs / served_s, "unit": UNIT, "n_gpus": 1,
        "steps": 1, "warmup": 0, "ms_per_step": 1e3 * served_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/i32", "data": "synthetic",
        "config": {"workload": f"serve_{nbeams}beams_4096ch_2e16", "beams": nbeams,
                   "chunks": len(arr), "arrival_speedup": args.speedup,
                   "max_inflight": args.inflight, "input": "pinned host, 2 chunks per beam reused"},
        "real_time_factor": obs / served_s,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "plain_loop": {"value": done_outputs / plain_s, "real_time_factor": obs / plain_s,
                       "latency_ms": {"p50": float(np.percentile(plain_lat, 50)),
                                      "p99": float(np.percentile(plain_lat, 99))},
                       "clocks": clk_plain.summary()},
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    return 0


def batch_workload(args):
    """48 beams of log-uniform length 2^18-2^21 with 1024 or 4096 channels, DM 0-500: one
    captured, autotuned batch step, in persistent form (one dedispersion launch per round and
    data type over a device work list of every beam's tiles) and in stream form (every beam's
    launches on its own stream), against the plain per-chunk loop over the same beams."""
    import torch

    import paper_2101_00941_gb300 as dd
    torch.cuda.set_device(0)
    dev_idx = torch.cuda.current_device()
    dd.build()
    ws = configs.batched_beams()
    if args.batch_scale > 1:
        for w in ws:
            w.nsamp = max(1 << 17, w.nsamp // args.batch_scale // 128 * 128)
    big = max(w.nsamp * w.nchans for w in ws)
    pinned = torch.empty(big, dtype=torch.uint8, pin_memory=True)
    dev = []
    for w in ws:
        h = pinned[:w.nsamp * w.nchans].view(w.nsamp, w.nchans)
        w.generate(pulse_offsets(w), out=h.numpy())
        dev.append(h.cuda())
    del pinned
    L = 1 << 17
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_batch(persistent):
        t_build = time.perf_counter()
        b = dd.Batch([(w.freqs(), w.tsamp, d) for w, d in zip(ws, dev)], ws[0].ranges_array(),
                     L, ws[0].widths, ws[0].threshold, n_streams=1, graph=True, autotune=True,
                     persistent=persistent, cap_per_chunk=1 << 16)
        t_build = time.perf_counter() - t_build
        outs = sum(b.info(i)[1] for i in range(len(ws)))
        tiles = sorted({b.info(i)[2] for i in range(len(ws))})
        for _ in range(args.warmup):
            b.run()
            b.wait()
        torch.cuda.synchronize()
        with ClockSampler(dev_idx) as clk:
            e0.record()
            for _ in range(args.steps):
                b.run()
                b.wait()
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        ncand = sum(b.candidates(i, k).size for i in range(len(ws))
                    for k in range(b.info(i)[0]))
        b.close()
        return ms, outs, tiles, t_build, ncand, clk.summary()

    ms_p, outs, tiles, tb_p, ncand_p, clk_p = timed_batch(True)
    ms_s, _, _, tb_s, ncand_s, clk_s = timed_batch(False)
    # plain per-chunk loop: each beam alone, one stream, every chunk synchronised
    torch.cuda.synchronize()
    with ClockSampler(dev_idx) as clk_plain:
        e0.record()
        for w, d in zip(ws, dev):
            p = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), L, n_streams=1,
                        max_width=max(w.widths), flags=dd.DD_FLAG_DEVICE_INPUT)
            for k in range(0, w.nsamp, L):
                p.run(d[k:k + L], min(L, w.nsamp - k))
                p.search(w.widths, w.threshold)
                p.candidates()
            p.close()
        e1.record()
        torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    obs = sum(w.nsamp for w in ws) * 64e-6
    line = {
        "metric": METRIC, "value": outs / (ms_p * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_p,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/i32",
        "data": "synthetic",
        "config": {"workload": f"batch_{len(ws)}beams_1024-4096ch", "beams": len(ws),
                   "samples": int(sum(w.nsamp for w in ws)), "input_gb":
                   sum(w.nsamp * w.nchans for w in ws) / 1e9, "graph": True,
                   "form": "persistent: one dedispersion launch per round and data type over "
                           "a device work list of every beam's (range, trial tile, time tile)",
                   "autotuned_tiles": tiles, "plan_and_capture_s": tb_p, "candidates": ncand_p,
                   "input": "device-resident beams (no host copies in the step)"},
        "real_time_factor": obs / (ms_p * 1e-3),
        "clocks": clk_p,
        "stream_form": {"value": outs / (ms_s * 1e-3), "ms_per_step": ms_s,
                        "plan_and_capture_s": tb_s, "candidates": ncand_s, "clocks": clk_s},
        "plain_loop": {"value": outs / (plain_ms * 1e-3), "ms": plain_ms,
                       "real_time_factor": obs / (plain_ms * 1e-3),
                       "clocks": clk_plain.summary()},
    }
    print(json.dumps(line))
    return 0


def transfer_workload(args):
    """The paper's transfer micro-experiment (Sec. 2, Sec. 2.1) on this machine: host-to-device
    throughput from pageable and from pinned memory, and the cost of allocating pinned memory
    (first allocation of each size), for 1 MiB .. 4 GiB. Each copy is timed with CUDA events,
    best of 5 after one warm-up."""
    import torch
    torch.cuda.set_device(0)
    sizes = [1 << 20, 16 << 20, 256 << 20, 1 << 30, 4 << 30]
    rows = []
    dst = torch.empty(max(sizes), dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def h2d_gbs(src, nbytes):
        best = None
        for k in range(6):
            torch.cuda.synchronize()
            e0.record()
            dst[:nbytes].copy_(src, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if k > 0:
                best = ms if best is None else min(best, ms)
        return nbytes / (best * 1e-3) / 1e9

    for nb in sizes:
        pageable = torch.from_numpy(np.ones(nb, dtype=np.uint8))
        t0 = time.perf_counter()
        pinned = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
        alloc_ms = 1e3 * (time.perf_counter() - t0)
        pinned.fill_(1)
        rows.append({"bytes": nb, "pageable_gbs": h2d_gbs(pageable, nb),
                     "pinned_gbs": h2d_gbs(pinned, nb), "pinned_alloc_ms": alloc_ms})
        del pinned, pageable
    big = rows[-1]
    line = {
        "metric": "H2D GB/s from pinned host memory", "value": big["pinned_gbs"], "unit": "GB/s",
        "n_gpus": 1, "steps": 5, "warmup": 1, "higher_is_better": True, "vs_baseline": None,
        "dtype": "u8", "data": "synthetic",
        "config": {"workload": "transfer_1MiB-4GiB", "timing": "CUDA events, best of 5",
                   "allocator": "torch pin_memory (cudaHostAlloc)"},
        "sizes": rows,
    }
    print(json.dumps(line))
    return 0


def shapes_workload(args):
    """Every tile shape of the tiled dedispersion kernel (forced by the plan's testing flags) and
    the autotuned plan, on the 4096-channel and the out-of-core plans: each range's launch over a
    full chunk window alone on one stream (best of three), in ms."""
    import torch

    import paper_2101_00941_gb300 as dd
    torch.cuda.set_device(0)
    dd.build()
    shapes = (("64x512x512", 0), ("64x512x1024", dd.DD_FLAG_WARPS32),
              ("64x256x512", dd.DD_FLAG_TILE256),
              ("32x256x512", dd.DD_FLAG_TILE256 | dd.DD_FLAG_TRIALS32),
              ("autotune", dd.DD_FLAG_AUTOTUNE))
    res = {}
    for name in ("mid", "ooc"):
        w, _ = stream_workload(name, streams=1)
        L = w.chunk_len
        x = torch.empty((2, L, w.nchans), dtype=torch.uint8)
        off = pulse_offsets(w)
        for k in range(2):
            w.generate(off, t0=k * L, nsamp=L, out=x[k].numpy())
        xd = x.cuda()
        st = torch.cuda.Stream()
        for label, fl in shapes:
            plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), L, n_streams=1,
                           max_width=max(w.widths),
                           flags=fl | dd.DD_FLAG_TIMING | dd.DD_FLAG_DEVICE_INPUT)
            chosen = []
            for r in range(len(w.ranges)):
                m = plan.model(r, 1)
                chosen.append([m["tile_trials"], m["tile_samples"], m["cta_threads"]]
                              if m["kind"] == dd.DD_KERNEL_TILED else "direct")
            plan.run(xd[0], L, cuda_stream=st.cuda_stream)
            plan.search(w.widths, w.threshold)
            plan.sync()
            best = None
            for rep in range(3):
                plan.stats(reset=True)
                plan.run(xd[1], L, cuda_stream=st.cuda_stream)
                plan.search(w.widths, w.threshold)
                plan.sync()
                ms = [plan.stats_range(r)[0] for r in range(len(w.ranges))]
                best = ms if best is None else [min(a, b) for a, b in zip(best, ms)]
            plan.close()
            res[f"{w.name}/{label}"] = {"tiles": chosen, "ms": [round(v, 3) for v in best],
                                         "total_ms": round(sum(best), 3)}
        del xd
    line = {"metric": "dedispersion ms per chunk window and range, by tile shape",
            "value": res[next(k for k in res if k.endswith("/autotune"))]["total_ms"],
            "unit": "ms", "n_gpus": 1, "higher_is_better": False, "vs_baseline": None,
            "dtype": "u8/i32", "data": "synthetic", "config": {"workload": "shapes"},
            "shapes": res}
    print(json.dumps(line))
    return 0


def peaks_workload(args):
    """The measured integer and shared-memory issue rates (dd_measure_peaks), three runs."""
    import torch

    import paper_2101_00941_gb300 as dd
    torch.cuda.set_device(0)
    dd.build()
    runs = [dd.dd_measure_peaks(0) for _ in range(3)]
    best = {k: max(r[k] for r in runs) for k in runs[0] if k != "sms"}
    best["sms"] = runs[0]["sms"]
    line = {"metric": "integer lane-instructions per SM-clock (LOP3 + DP2A)",
            "value": best["int_lanes_per_clk"], "unit": "lanes/clk/SM", "n_gpus": 1,
            "higher_is_better": True, "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": "peaks"}, "runs": runs, "best": best}
    print(json.dumps(line))
    return 0


def outputs_of_chunks(w, O: int, T0: int, sizes, input_equivalent: bool = False) -> int:
    """DM-trial*samples the library produces for chunks of `sizes` samples delivered from stream
    position T0 on: range r outputs the decimated indices j with j*d_r in [T - O, T + n - O).
    With input_equivalent, each decimated output counts the d_r original samples it covers."""
    out, T = 0, T0
    for n in sizes:
        lo, hi = max(0, T - O), max(0, T + n - O)
        out += sum(r.n_trials * (hi // r.decimation - lo // r.decimation) *
                   (r.decimation if input_equivalent else 1) for r in w.ranges)
        T += n
    return out


def launch_model(plan, w, O: int, T0: int, sizes):
    """Summed dd_plan_model of the dedispersion launches of these chunks, in total and per range:
    {adds, dram_bytes, smem_wavefronts, copy_bytes, outputs, launches}."""
    keys = ("adds", "dram_bytes", "smem_wavefronts", "copy_bytes", "outputs")
    tot = {k: 0.0 for k in keys + ("launches",)}
    per = [dict(tot) for _ in w.ranges]
    T = T0
    for n in sizes:
        lo, hi = max(0, T - O), max(0, T + n - O)
        for r, rg in enumerate(w.ranges):
            nout = hi // rg.decimation - lo // rg.decimation
            if nout <= 0:
                continue
            m = plan.model(r, nout)
            for k in keys:
                per[r][k] += m[k]
                tot[k] += m[k]
            per[r]["launches"] += 1
            tot["launches"] += 1
        T += n
    return tot, per


def dram_traffic_ratio(path=TRAFFIC_FILE):
    """DRAM bytes (read + write) of the dedispersion launches over their algorithmic bytes, from
    the committed ncu capture, or None when the capture was taken on another revision of the
    kernel source (its SHA-256 is stored beside the figures)."""
    try:
        with open(path) as fh:
            rec = json.load(fh)
        with open(DEDISP_SOURCE, "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha256") != sha:
        return None
    return float(rec["dram_bytes"]) / float(rec["algorithmic_bytes"])


def main(args):
    import torch

    import paper_2101_00941_gb300 as dd

    rank, world, local = dist_info()
    if args.gpus > 1 or world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")

        def barrier():
            tdist.barrier()
    else:
        torch.cuda.set_device(0)

        def barrier():
            pass
    dev = torch.cuda.current_device()
    dd.build()
    w, nring = stream_workload(args.workload, args.nsamp, beam=rank, streams=args.streams)
    L = w.chunk_len
    nchunks = w.nsamp // L
    # the input ring: nring distinct seeded chunks in pinned host memory, and a copy in HBM
    xh = torch.empty((nring, L, w.nchans), dtype=torch.uint8, pin_memory=True)
    off = pulse_offsets(w)
    for k in range(nring):
        w.generate(off, t0=k * L, nsamp=L, out=xh[k].numpy())
    xd = xh.cuda()
    dchunks = [xd[k % nring] for k in range(nchunks)]
    hchunks = [xh[k % nring] for k in range(nchunks)]
    t_plan = time.perf_counter()
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), L, n_streams=w.n_streams,
                   max_width=max(w.widths), peak_block=32, device=dev,
                   flags=dd.DD_FLAG_TIMING | (0 if args.no_autotune else dd.DD_FLAG_AUTOTUNE))
    nfused = plan.fuse_search(w.widths) if args.fused else 0
    t_plan = time.perf_counter() - t_plan
    O = plan.O
    shapes = [plan.model(r, 1) for r in range(len(w.ranges))]
    peaks = dd.dd_measure_peaks(dev)
    with ClockSampler(dev) as clk:
        ms, ncand, launches, dd_ms, dd_n = time_steps(plan, dchunks, w, args.steps, args.warmup,
                                                      barrier)
    T0 = args.warmup * w.nsamp  # stream position of the timed steps
    sizes = [L] * nchunks * args.steps
    outs = outputs_of_chunks(w, O, T0, sizes)
    outs_in = outputs_of_chunks(w, O, T0, sizes, input_equivalent=True)
    tot, per = launch_model(plan, w, O, T0, sizes)
    lat = []
    ms_e2e, ncand_e2e, _, _, _ = time_steps(plan, hchunks, w, args.steps, args.warmup, barrier,
                                            lat)
    # each range's launches alone: two chunks (full windows) on one stream, so no launch of
    # another range or chunk overlaps them
    solo = torch.cuda.Stream()
    plan.sync()
    plan.stats(reset=True)
    T_solo = (2 * args.warmup + 2 * args.steps) * w.nsamp
    for k in range(2):
        plan.run(dchunks[k % len(dchunks)], L, cuda_stream=solo.cuda_stream)
        plan.search(w.widths, w.threshold)
    plan.sync()
    range_ms = [plan.stats_range(r) for r in range(len(w.ranges))]
    _, per_solo = launch_model(plan, w, O, T_solo, [L, L])
    plan.close()
    if world > 1:
        ms, ms_e2e = rank_max([ms, ms_e2e], "cuda")
    total_outs = outs * world
    value = total_outs / (ms * 1e-3)
    e2e = total_outs / (ms_e2e * 1e-3)
    clocks = clk.summary()
    sm_hz = (clocks["sm_mhz"] or peaks["sm_mhz"]) * 1e6
    peak_int = peaks["int_lanes_per_clk"] * peaks["sms"] * sm_hz
    peak_wf = peaks["lds_wavefronts_per_clk"] * peaks["sms"] * sm_hz
    dd_s = dd_ms * 1e-3
    achieved = tot["adds"] / dd_s if dd_s > 0 else None
    smem_wf = tot["smem_wavefronts"] + tot["copy_bytes"] / 128.0
    ratio = dram_traffic_ratio(TRAFFIC_FILE_FUSED if nfused else TRAFFIC_FILE)
    per_range = []
    for r, (rms, rn) in enumerate(range_ms):
        p = per_solo[r]
        rs = rms * 1e-3
        m = shapes[r]
        per_range.append({
            "decimation": w.ranges[r].decimation, "launches": rn, "ms": rms,
            "tile": [m["tile_trials"], m["tile_samples"], m["cta_threads"], m["ctas_per_sm"]],
            "adds_per_s": p["adds"] / rs if rs > 0 else None,
            "frac": p["adds"] / rs / peak_int if rs > 0 else None,
            "frac_smem": (p["smem_wavefronts"] + p["copy_bytes"] / 128.0) / rs / peak_wf
            if rs > 0 and p["smem_wavefronts"] > 0 else None,
            "dram_gbs_algorithmic": p["dram_bytes"] / rs / 1e9 if rs > 0 else None})
    obs = w.nsamp * w.tsamp
    if rank != 0:
        return 0
    ring_note = (f"ring of {nring} distinct seeded {L}-sample chunks "
                 f"({L * w.nchans / 1e9:.1f} GB each) reused cyclically to make up the "
                 f"{w.nsamp}-sample beam; resident in HBM for value, pinned host memory for e2e")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/i32", "data": "synthetic",
        "config": {"workload": w.name, "nchans": w.nchans, "nsamp": w.nsamp,
                   "tsamp_us": w.tsamp * 1e6, "trials": w.n_trials,
                   "ranges": [[r.dm_start, r.dm_step, r.n_trials, r.decimation] for r in w.ranges],
                   "chunk_len": L, "chunks": nchunks, "n_streams": w.n_streams,
                   "widths": list(w.widths), "threshold": w.threshold, "overlap": O,
                   "input": ring_note,
                   "l2": f"every chunk {L * w.nchans / 1e9:.1f} GB > L2 (no flush)",
                   "fused_search_ranges": nfused},
        "real_time_factor": obs / (ms * 1e-3 / args.steps),
        "input_equivalent": {"value": outs_in * world / (ms * 1e-3), "unit": UNIT,
                             "note": "the same steps counting each decimated output as the d_r "
                                     "original samples it covers (sum over ranges of n_r x the "
                                     "chunk window at the original sampling)"},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": w.nsamp * w.nchans,
                "d2h_bytes_per_step": int(ncand_e2e / args.steps * 32 + nchunks * 16),
                "real_time_factor": obs / (ms_e2e * 1e-3 / args.steps),
                # host-to-device time the streams did not hide: e2e step minus resident step
                "exposed_copy_ms_per_chunk": max(0.0, (ms_e2e - ms) / args.steps / nchunks),
                "chunk_latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                     "p99": 1e3 * float(np.percentile(lat, 99))}},
        "gpu_launches": launches,
        "candidates_per_step": ncand / args.steps,
        "roofline": {
            "bound": "alu", "achieved": achieved, "peak": peak_int, "unit": "adds/s",
            "frac": achieved / peak_int if achieved else None,
            "traffic": ratio * tot["dram_bytes"] / dd_n if (ratio and dd_n) else None,
            "traffic_unit": "bytes per launch",
            "traffic_note": "measured DRAM bytes / algorithmic bytes of a committed ncu capture "
                            "of the same kernel source (profiles/dedisp_dram_traffic.json, or "
                            "dedisp_fused_dram_traffic.json for the fused search) x the "
                            "algorithmic bytes of the timed launches (dd_plan_model); null when "
                            "the kernel source has changed since the capture",
            "algorithmic_dram_bytes_per_launch": tot["dram_bytes"] / dd_n if dd_n else None,
            "kernel": ("k_dedisp_fused + k_fused_edges (the search's position pass fused; "
                       f"{nfused} ranges)") if nfused else "k_dedisp_tiled (all ranges)",
            "launches_timed": dd_n, "dedisp_ms": dd_ms,
            "peak_note": "measured: integer lane-instructions per SM-clock with LOP3 and DP2A "
                         "interleaved (dd_measure_peaks) x SMs x median SM clock of the timed "
                         "region; achieved counts algorithmic channel-adds (one per channel per "
                         "output), which packed lanes let one instruction carry several of",
            "frac_smem": smem_wf / dd_s / peak_wf if dd_s > 0 else None,
            "smem_note": "dd_plan_model's shared-memory wavefronts (+ copy bytes / 128) of the "
                         "timed launches over their union time, against measured conflict-free "
                         "32-bit load wavefronts per SM-clock x SMs x clock",
            "per_range": per_range,
            "per_range_note": "each range's launches timed alone (two chunks on one stream); "
                              "tile = [trials, outputs, threads per CTA, CTAs per SM] chosen by "
                              "the plan's autotuner",
            "plan_s": t_plan,
            "measured_peaks": peaks},
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        t_in0, n = baseline_window(w, O)
        x0 = xh[0].numpy()
        x1 = xh[1 % nring].numpy()
        xw = np.concatenate([x0[t_in0:], x1[:n - (L - t_in0)]])
        line["cpu_baseline"] = cpu_baseline(w, xw, t_in0, O)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 2 for the out-of-core beam, 5 otherwise)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fused", action="store_true",
                    help="ooc/mid: fuse the search's position pass into dedispersion "
                         "(dd_fuse_search); the series are not written")
    ap.add_argument("--no-autotune", action="store_true",
                    help="plan without timing the tile shapes (profiler captures count launches)")
    ap.add_argument("--nsamp", type=int, default=None,
                    help="samples per beam (a multiple of the chunk length; smaller only for "
                         "tests and profiler captures)")
    ap.add_argument("--streams", type=int, default=4, help="CUDA streams the chunks rotate over")
    ap.add_argument("--workload", choices=["ooc", "mid", "serve", "batch", "transfer", "peaks",
                                           "shapes"],
                    default="ooc")
    ap.add_argument("--batch-scale", type=int, default=1,
                    help="batch: divide every beam's length by this (profiling only)")
    ap.add_argument("--beams", type=int, default=16, help="serve: beams")
    ap.add_argument("--chunks-per-beam", type=int, default=6, help="serve: chunks per beam")
    ap.add_argument("--speedup", type=float, default=8.0,
                    help="serve: arrival rate relative to real time (1 = 4.19 s cadence)")
    ap.add_argument("--inflight", type=int, default=8,
                    help="serve: most chunks on the GPU at once (the admission limit's cap)")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = 2 if a.workload == "ooc" else 5
    if a.impl == "reference":
        sys.exit(main_reference(a))
    if a.workload == "serve":
        sys.exit(serve_workload(a))
    if a.workload == "transfer":
        sys.exit(transfer_workload(a))
    if a.workload == "peaks":
        sys.exit(peaks_workload(a))
    if a.workload == "shapes":
        sys.exit(shapes_workload(a))
    sys.exit(batch_workload(a) if a.workload == "batch" else main(a))
