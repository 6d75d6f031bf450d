"""The N-GPU path of bench.py on CPU: two gloo ranks (no GPU).

Queries are independent, so N GPUs run N replicas with no data-path collective; the only
cross-rank steps are the barrier around the timed region and the max over ranks of the
timed seconds.  Checked here with world_size 2: each rank draws its own stream of
sources (disjoint from the other rank's), the slowest rank's time is what every rank
sees, the whole-job rate counts both ranks' queries, and the reference arm runs on rank
0 only (rank 1 returns without work or output).
"""
import io
import os
import socket
import sys
import contextlib

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


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                             world_size=world)
    try:
        n, B = 1 << 14, 64
        mine = [bench.replica_sources(n, B, rank, step) for step in range(3)]
        gathered = [None] * world
        tdist.all_gather_object(gathered, [m.tolist() for m in mine])
        tdist.barrier()
        local_seconds = 0.100 + 0.050 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(local_seconds, tdist, "cpu")
        rate = bench.whole_job_rate(B * 3, world, slowest)
        # the reference arm: rank 0 alone works; the others return without output
        buf = io.StringIO()
        if rank != 0:
            with contextlib.redirect_stdout(buf):
                bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1",
                                                      "--warmup", "0"]))
        out.put((rank, gathered, slowest, rate, buf.getvalue()))
    finally:
        tdist.destroy_process_group()


def test_two_replicas_disjoint_sources_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    results = {}
    for _ in procs:
        rank, gathered, slowest, rate, printed = out.get(timeout=120)
        results[rank] = (gathered, slowest, rate, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        gathered, slowest, rate, printed = results[rank]
        assert slowest == pytest.approx(0.150)
        assert rate == pytest.approx(64 * 3 * 2 / 0.150)
        r0 = [np.array(x) for x in gathered[0]]
        r1 = [np.array(x) for x in gathered[1]]
        for a, b in zip(r0, r1):
            assert a.shape == b.shape == (64,)
            assert not np.array_equal(a, b)  # the replicas work on different sources
        assert not np.array_equal(r0[0], r0[1])  # and each step draws new ones
    assert results[1][3] == ""  # rank 1 of the reference arm printed nothing
