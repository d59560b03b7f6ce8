"""The multi-GPU path is replicas only: every rank zooms its own frames and
the ranks meet only in a barrier and a max-over-ranks of the timed region.
This drives that host logic of bench.py with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse
    import contextlib
    import io

    import torch.distributed as dist

    import bench
    w, r, local = bench.dist_setup(world, backend="gloo")
    bench.barrier(w)
    t_local = 1.0 + rank  # rank 1 is the slower one
    t_max = bench.max_over_ranks(w, t_local, "cpu")
    value = bench.replica_value(w, 10, bench.OUT_PX, t_max)
    # the reference arm runs on rank 0 only; other ranks leave without work
    printed = ""
    if rank != 0:
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(argparse.Namespace(steps=1, warmup=1, gpus=world))
        printed = buf.getvalue()
    bench.barrier(w)
    dist.destroy_process_group()
    out_q.put((rank, w, r, local, t_max, value, printed))


def test_two_replicas_agree_on_time_and_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import bench
    for rank, (r_, w, r, local, t_max, value, printed) in enumerate(results):
        assert (w, r, local) == (world, rank, rank)
        assert t_max == pytest.approx(2.0)  # the slowest rank's time
        assert value == pytest.approx(world * 10 * bench.OUT_PX / 2.0 / 1e9)
    assert results[1][6] == ""  # rank 1 printed no reference line
