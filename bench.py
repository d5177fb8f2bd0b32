#!/usr/bin/env python3
"""Benchmark: streamed brute-force dedispersion + boxcar single-pulse search on GB300.

One step = the whole hot path over one synthetic beam of the 4096-channel
workload (1250-1550 MHz, 64 us, 2^20 uint8 samples = 4.3 GB, 4050 DM trials
over 0-1000 pc cm^-3 with x1/x2/x4/x8 decimation, boxcars 1..256, 6 sigma):
eight 2^17-sample chunks over four CUDA streams, each chunk corner-turned,
decimated, dedispersed, searched, and its candidates copied to the host.

  value : DM-trial*samples/s with the input already resident in HBM
  e2e   : the same through the C ABI from pinned HOST memory (H2D inside the step)
Timing: CUDA events around each step with a device synchronize on both sides;
W warm-up steps; the 4.3 GB input is larger than L2 (no flush needed).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torchrun: one independent beam per rank (weak scaling),
max of the per-rank step times.
"""
from __future__ import annotations

import argparse
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
# Integer ALU roofline: 152 SMs x 128 int32 lanes per clock (ALU + FMA pipes) x 2070 MHz.
ALU_PEAK_ADDS = 152 * 128 * 2070e6
# DRAM bytes (read + write) of the four dedispersion launches of one full 131072-sample chunk
# window of the 4096-channel workload, from one ncu capture of the current kernel
# (dram__bytes_read.sum + dram__bytes_write.sum; profiles/k_dedisp_tiled_mid_4096ch.md).
DEDISP_DRAM_BYTES_PER_FULL_CHUNK = 1.312e9 + 0.791e9 + 0.386e9 + 0.196e9


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


def outputs_per_pass(w, O: int) -> int:
    """DM-trial*samples produced from one beam: sum_r n_r * (N - O) / d_r."""
    return sum(r.n_trials * ((w.nsamp - O) // r.decimation) for r in w.ranges)


def adds_per_pass(w, O: int) -> int:
    """Algorithmic adds of brute-force dedispersion: one per channel per output sample."""
    return outputs_per_pass(w, O) * w.nchans


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


def make_input(w, pinned: bool):
    import torch
    x = torch.empty((w.nsamp, w.nchans), dtype=torch.uint8, pin_memory=pinned)
    w.generate(pulse_offsets(w), out=x.numpy())
    return x


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


def cpu_baseline(w, x_np, O, target_s: float = 15.0):
    """The oracle, as it stands, on a bounded sample of the same workload: every range, a few
    trials spread over the range, over one full chunk window. Returns DM-trial*samples/s."""
    import oracle
    oracle.build()
    f = w.freqs()
    ranges = w.ranges_array()
    tabs = oracle.shift_tables(f, w.tsamp, ranges)
    k = 1  # second chunk: a full window with history
    T = k * w.chunk_len
    lo, hi = T - O, T + w.chunk_len - O
    ntr = 16  # at least one trial per host thread in the oracle's parallel loops
    done_out, elapsed = 0, 0.0
    while elapsed < target_s and ntr <= 4096:
        t0 = time.perf_counter()
        outs = 0
        for r, tab in enumerate(tabs):
            d = int(ranges[r][3])
            tr = np.linspace(0, tab.shape[0] - 1, min(ntr, tab.shape[0])).astype(np.int32)
            J0, J1 = lo // d, hi // d
            xd = oracle.decimate(x_np, 0, d, J0, J1 - J0 + int(tab.max()))
            y = oracle.dedisperse(xd, J0, tab, tr, J0, J1 - J0)
            oracle.sps(y, tr, r, d, J0, oracle.widths_for_range(w.widths, d), 32, w.threshold)
            outs += tr.size * (J1 - J0)
        dt = time.perf_counter() - t0
        done_out, elapsed = outs, dt
        if dt * 4 > target_s:
            break
        ntr *= 4
    return {"value": done_out / elapsed, "unit": UNIT, "cores": min(os.cpu_count(), ntr),
            "kind": "oracle",
            "sample": f"{done_out} DM-trial*samples: {ntr} trials per range (of 1500/750/800/1000) "
                      f"over one full {w.chunk_len}-sample chunk window, dedispersion + search, "
                      f"{elapsed:.1f} s"}


def main_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    w = configs.mid()
    import oracle
    f = w.freqs()
    O = oracle.overlap(oracle.shift_tables(f, w.tsamp, w.ranges_array()), w.ranges_array())
    # host input only: two chunks of samples are enough for a one-chunk-window sample
    n = 2 * w.chunk_len + w.chunk_len
    x = w.generate(pulse_offsets(w), nsamp=n)
    for _ in range(args.warmup):
        cpu_baseline(w, x, O, target_s=2.0)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, x, O, target_s=8.0))
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
    srv.close()
    # ---- plain per-chunk loop: one stream per beam, each chunk copied, dedispersed,
    #      searched and synchronised before the next one starts
    plans = [dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), 1 << 17, n_streams=1,
                     max_width=max(w.widths)) for w in beams]
    plain_lat = []
    torch.cuda.synchronize()
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
                                      "p99": float(np.percentile(plain_lat, 99))}},
    }
    print(json.dumps(line))
    return 0


def batch_workload(args):
    """48 beams of log-uniform length 2^18-2^21 with 1024 or 4096 channels, DM 0-500: one
    captured, autotuned batch step against the plain per-chunk loop over the same beams."""
    import torch

    import paper_2101_00941_gb300 as dd
    torch.cuda.set_device(0)
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
    outs = 0
    t_build = time.perf_counter()
    b = dd.Batch([(w.freqs(), w.tsamp, d) for w, d in zip(ws, dev)], ws[0].ranges_array(), L,
                 ws[0].widths, ws[0].threshold, n_streams=1, graph=True, autotune=True,
                 cap_per_chunk=1 << 16)
    t_build = time.perf_counter() - t_build
    for i in range(len(ws)):
        outs += b.info(i)[1]
    tiles = sorted({b.info(i)[2] for i in range(len(ws))})
    for _ in range(args.warmup):
        b.run()
        b.wait()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        b.run()
        b.wait()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ncand = sum(b.candidates(i, k).size for i in range(len(ws)) for k in range(b.info(i)[0]))
    b.close()
    # plain per-chunk loop: each beam alone, one stream, every chunk synchronised
    torch.cuda.synchronize()
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
        "metric": METRIC, "value": outs / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/i32",
        "data": "synthetic",
        "config": {"workload": f"batch_{len(ws)}beams_1024-4096ch", "beams": len(ws),
                   "samples": int(sum(w.nsamp for w in ws)), "input_gb":
                   sum(w.nsamp * w.nchans for w in ws) / 1e9, "graph": True, "autotuned_tiles":
                   tiles, "plan_and_capture_s": t_build, "candidates": ncand},
        "real_time_factor": obs / (ms * 1e-3),
        "plain_loop": {"value": outs / (plain_ms * 1e-3), "ms": plain_ms,
                       "real_time_factor": obs / (plain_ms * 1e-3)},
    }
    print(json.dumps(line))
    return 0


def ooc_workload(args):
    """The out-of-core shape: 8192 channels over 1000-1500 MHz, 50 us, DM 0-3000 with x1..x16
    decimation (6050 trials, overlap ~138k samples), 2^19-sample chunks over 4 streams, input in
    pageable host memory. One step = --ooc-chunks chunks of one continuing stream (a pool of two
    distinct seeded chunks, reused). Three ways in: pageable through the pinned staging threads
    (Sec. 2.1; the headline), pageable through the CUDA driver, and pinned host memory."""
    import torch

    import paper_2101_00941_gb300 as dd
    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    dd.build()
    L = 1 << 19
    w = configs.out_of_core(nsamp=2 * L)
    w.chunk_len, w.n_streams = L, 4
    x = np.empty((2 * L, w.nchans), dtype=np.uint8)  # pageable
    w.generate(pulse_offsets(w), out=x)
    pool = [x[:L], x[L:]]
    nchunks = args.ooc_chunks
    per_chunk = sum(r.n_trials * (L // r.decimation) for r in w.ranges)  # full windows
    res = {}
    for mode in ("staged", "driver", "pinned"):
        plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), L, n_streams=w.n_streams,
                       max_width=max(w.widths), device=dev,
                       staging_threads=4 if mode == "staged" else 0)
        src = [torch.from_numpy(c).pin_memory() for c in pool] if mode == "pinned" else pool
        chunks = [src[k % 2] for k in range(nchunks)]
        # the first chunk of the stream fills the overlap; it runs before the timed steps
        plan.run(chunks[0], L)
        plan.search(w.widths, w.threshold)
        plan.sync()
        with ClockSampler(dev) as clk:
            ms, ncand, launches, _, _ = time_steps(plan, chunks, w, args.steps, args.warmup,
                                                   lambda: None)
        plan.close()
        del src
        res[mode] = {"value": per_chunk * nchunks * args.steps / (ms * 1e-3),
                     "ms_per_step": ms / args.steps, "candidates_per_step": ncand / args.steps,
                     "real_time_factor": nchunks * L * w.tsamp / (ms * 1e-3 / args.steps),
                     "gpu_launches": launches, "clocks": clk.summary()}
    head = res["staged"]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/i32",
        "data": "synthetic",
        "config": {"workload": "ooc_8192ch_2e19_chunks", "nchans": w.nchans, "tsamp_us": 50.0,
                   "trials": w.n_trials, "chunk_len": L, "chunks_per_step": nchunks,
                   "n_streams": w.n_streams, "staging_threads": 4,
                   "ranges": [[r.dm_start, r.dm_step, r.n_trials, r.decimation] for r in w.ranges],
                   "input": "pageable host memory, two 4.3 GB chunks reused",
                   "h2d_bytes_per_step": nchunks * L * w.nchans},
        "real_time_factor": head["real_time_factor"],
        "gpu_launches": head["gpu_launches"],
        "candidates_per_step": head["candidates_per_step"],
        "clocks": head["clocks"],
        "pageable_through_driver": {k: res["driver"][k] for k in ("value", "ms_per_step",
                                                                  "real_time_factor")},
        "pinned_host": {k: res["pinned"][k] for k in ("value", "ms_per_step", "real_time_factor")},
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
    w = configs.mid(beam=rank, nsamp=args.nsamp, n_streams=args.streams)
    xh = make_input(w, pinned=True)
    xd = xh.cuda()
    L = w.chunk_len
    nchunks = w.nsamp // L
    dchunks = [xd[L * k:L * (k + 1)] for k in range(nchunks)]
    hchunks = [xh[L * k:L * (k + 1)] for k in range(nchunks)]
    plan = dd.Plan(w.freqs(), w.tsamp, w.ranges_array(), L, n_streams=w.n_streams,
                   max_width=max(w.widths), peak_block=32, device=dev, flags=dd.DD_FLAG_TIMING)
    O = plan.O
    outs = outputs_per_pass(w, O)
    with ClockSampler(dev) as clk:
        ms, ncand, launches, dd_ms, dd_n = time_steps(plan, dchunks, w, args.steps, args.warmup,
                                                      barrier)
    lat = []
    ms_e2e, ncand_e2e, _, _, _ = time_steps(plan, hchunks, w, args.steps, args.warmup, barrier,
                                            lat)
    plan.close()
    if world > 1:
        ms, ms_e2e = rank_max([ms, ms_e2e], "cuda")
    total_outs = outs * args.steps * world
    value = total_outs / (ms * 1e-3)
    e2e = total_outs / (ms_e2e * 1e-3)
    adds_per_launch = adds_per_pass(w, O) * args.steps / max(dd_n, 1)
    achieved = adds_per_launch / (dd_ms * 1e-3 / max(dd_n, 1)) if dd_ms > 0 else None
    # DRAM traffic per launch, averaged like `achieved`: the captured per-chunk bytes scaled by
    # the step's summed chunk windows (N - O samples); only for the captured configuration
    traffic = None
    if (w.nchans, L, tuple(w.ranges)) == (4096, 1 << 17, tuple(configs.MID_RANGES)) and dd_n:
        traffic = (DEDISP_DRAM_BYTES_PER_FULL_CHUNK * (w.nsamp - O) / L * args.steps / dd_n)
    obs = w.nsamp * w.tsamp
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/i32", "data": "synthetic",
        "config": {"workload": w.name, "nchans": w.nchans, "nsamp": w.nsamp,
                   "tsamp_us": w.tsamp * 1e6, "trials": w.n_trials,
                   "ranges": [[r.dm_start, r.dm_step, r.n_trials, r.decimation] for r in w.ranges],
                   "chunk_len": L, "chunks": nchunks, "n_streams": w.n_streams,
                   "widths": list(w.widths), "threshold": w.threshold, "overlap": O,
                   "l2": f"input {w.nsamp * w.nchans / 1e9:.1f} GB per step > L2 (no flush)"},
        "real_time_factor": obs / (ms * 1e-3 / args.steps),
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": w.nsamp * w.nchans,
                "d2h_bytes_per_step": int(ncand_e2e / args.steps * 32 + nchunks * 8),
                "real_time_factor": obs / (ms_e2e * 1e-3 / args.steps),
                # host-to-device time the streams did not hide: e2e step minus resident step
                "exposed_copy_ms_per_chunk": max(0.0, (ms_e2e - ms) / args.steps / nchunks),
                "chunk_latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                     "p99": 1e3 * float(np.percentile(lat, 99))}},
        "gpu_launches": launches,
        "candidates_per_step": ncand / args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_ADDS, "unit": "adds/s",
                     "frac": (achieved / ALU_PEAK_ADDS) if achieved else None,
                     "traffic": traffic, "traffic_unit": "bytes per launch",
                     "kernel": "dedispersion", "launches_timed": dd_n,
                     "peak_note": "152 SMs x 128 int32 lanes/clk x 2070 MHz (derived)"},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, xh.numpy(), O)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nsamp", type=int, default=1 << 20,
                    help="samples per beam (a multiple of 2^17; smaller only for profiler captures)")
    ap.add_argument("--streams", type=int, default=4, help="CUDA streams the chunks rotate over")
    ap.add_argument("--workload", choices=["mid", "serve", "batch", "ooc", "transfer"],
                    default="mid")
    ap.add_argument("--ooc-chunks", type=int, default=6,
                    help="ooc: 2^19-sample chunks per step")
    ap.add_argument("--batch-scale", type=int, default=1,
                    help="batch: divide every beam's length by this (profiling only)")
    ap.add_argument("--beams", type=int, default=16, help="serve: beams")
    ap.add_argument("--chunks-per-beam", type=int, default=6, help="serve: chunks per beam")
    ap.add_argument("--speedup", type=float, default=8.0,
                    help="serve: arrival rate relative to real time (1 = 4.19 s cadence)")
    ap.add_argument("--inflight", type=int, default=8, help="serve: chunks on the GPU at once")
    a = ap.parse_args()
    if a.impl == "reference":
        sys.exit(main_reference(a))
    if a.workload == "serve":
        sys.exit(serve_workload(a))
    if a.workload == "ooc":
        sys.exit(ooc_workload(a))
    if a.workload == "transfer":
        sys.exit(transfer_workload(a))
    sys.exit(batch_workload(a) if a.workload == "batch" else main(a))
