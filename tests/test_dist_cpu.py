"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Templates are independent, so each rank searches its own shard of the bank with no
data-path collective; gloo carries only the barrier and the max-over-ranks time.
This checks the shards are disjoint, cover the bank, share one series, and that the
timing reduction returns the slowest rank's time on every rank."""
import os
import socket
import sys
import types

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    args = types.SimpleNamespace(logn=12, templates=6)
    ws2, r2, _ = bench.dist_init(args)
    assert (ws2, r2) == (ws, rank)
    w, bank = bench.workload(args, ws, rank)
    bench.barrier(ws)
    slowest = bench.allmax(ws, 1.0 + rank)
    q.put((rank, bank.copy(), w.bank.copy(), float(w.series[:64].sum()), slowest))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_template_shards_and_max_time():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort(key=lambda t: t[0])
    full = out[0][2]
    assert full.shape == (12, 5)
    assert np.array_equal(out[0][2], out[1][2])
    assert np.array_equal(np.concatenate([out[0][1], out[1][1]]), full)
    assert out[0][3] == out[1][3]  # same series on every rank
    assert out[0][4] == out[1][4] == 2.0
