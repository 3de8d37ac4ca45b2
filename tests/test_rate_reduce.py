"""The cross-rank dt reduction of one-shard-per-process meshes
(reduce_rate_max) on CPU over gloo, world size 2: the max of the ranks'
signal rates, and a NaN rate on one rank reaching every rank as +inf (so
that dt = 0 marks the state non-finite everywhere) instead of being dropped
or kept by one backend and not another."""
import math
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2202_12309_gb300 import reduce_rate_max
    out = []
    for vals in ((0.5, 2.0), (3.0, 1.0), (float("nan"), 1.0), (1.0, float("nan")), (float("inf"), 1.0)):
        r = torch.tensor([vals[rank]], dtype=torch.float64)
        reduce_rate_max(r, dist)
        out.append(float(r[0]))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_rate_max_over_two_gloo_ranks_keeps_nan_as_inf():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [2.0, 3.0, math.inf, math.inf, math.inf]
    assert res == [(0, want), (1, want)]
