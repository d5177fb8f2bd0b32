"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2): each rank runs its
own beam (seeded by rank), and the job's step time is the max over ranks."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    from synth import configs
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, wsize, local = bench.dist_info()
        times = bench.rank_max([10.0 + rank, 20.0 - rank], "cpu")
        # each rank's beam: same workload shape, its own seed
        w = configs.mid(beam=r, nsamp=1 << 12, nchans=64, npulses=0)
        x = w.generate(lambda dm: np.zeros(w.nchans, dtype=np.int64), nsamp=256)
        q.put((rank, r, wsize, local, times, int(x.astype(np.int64).sum())))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, wsize, local, times, _ in out:
        assert (r, wsize, local) == (rank, 2, rank)
        assert times == [11.0, 20.0]  # max over the two ranks, element-wise
    assert out[0][5] != out[1][5]  # the ranks' beams differ
