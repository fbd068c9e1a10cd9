"""The N > 1 path of bench.py on CPU: replicas on two gloo ranks (world size
2, rendezvous on 127.0.0.1).  The whole-job value is the objects of all
ranks over the largest rank time; every rank runs its own seed; the
reference arm runs on rank 0 only."""
import argparse
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        b = load_bench()
        assert b.dist_setup() == (ws, rank, rank)
        t, objs, af = b.reduce_over_ranks(0.5 + rank, 1000 * (rank + 1), 10 + rank, "cpu")
        args = argparse.Namespace(warmup=0, steps=1, gpus=ws)
        ref_rc = b.run_reference(args, ws, rank) if rank == 1 else None
        q.put((rank, t, objs, af, b.replica_seed(rank), ref_rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_sum_objects():
    ws, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = {}
    while not q.empty():
        r = q.get()
        res[r[0]] = r
    assert set(res) == {0, 1}
    for r in (0, 1):
        assert res[r][1] == 1.5          # the slowest rank's time
        assert res[r][2] == 3000         # objects of both ranks
        assert res[r][3] == 21
    assert res[0][4] != res[1][4]        # independent replicas
    assert res[1][5] == 0                # the reference arm: rank 1 exits without work
