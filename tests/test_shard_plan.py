"""Host logic of the domain decomposition (no GPU): the partition of the
Z-ordered root grid into contiguous shards (Sec. 2.1) and the per-cell halo
plan of the exchange between them (Sec. 3.7), through ph_shard_plan.

* what shard s plans to send to p is exactly what p plans to receive from s,
  key for key and in the same order (the message layout has no handshake);
* on periodic meshes, the ghost cells a shard receives are exactly the ones
  an independent re-derivation here (its own Morton order, partition and
  periodic neighbour rule) finds with a source on another shard;
* every ghost cell is received at most once, and never from its own shard;
* the same checks across two processes talking over gloo: each rank computes
  only its own plan and the ranks compare what they exchange."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NG = 2


def _ph():
    sys.path.insert(0, ROOT)
    import paper_2202_12309_gb300 as ph
    return ph


def morton(i, j, k):
    key = 0
    for b in range(21):
        key |= ((i >> b) & 1) << (3 * b) | ((j >> b) & 1) << (3 * b + 1) | ((k >> b) & 1) << (3 * b + 2)
    return key


def expected_recv(nx, nb, nshards, shard):
    """Keys (global leaf x padded cells + padded cell) of the ghost cells of
    `shard`'s leaves whose periodic source leaf lies on another shard."""
    locs = sorted(((morton(i, j, k), (i, j, k)) for k in range(nb[2]) for j in range(nb[1])
                   for i in range(nb[0])))
    locs = [l for _, l in locs]
    index = {l: g for g, l in enumerate(locs)}
    N = len(locs)
    first = [s * N // nshards for s in range(nshards + 1)]
    owner = np.zeros(N, dtype=int)
    for s in range(nshards):
        owner[first[s]:first[s + 1]] = s
    S = [n + 2 * NG for n in nx]
    cells = S[0] * S[1] * S[2]
    keys = {}
    for g in range(first[shard], first[shard + 1]):
        l = locs[g]
        for k in range(S[2]):
            for j in range(S[1]):
                for i in range(S[0]):
                    o = [(-1 if x < NG else (1 if x >= NG + n else 0)) for x, n in zip((i, j, k), nx)]
                    if o == [0, 0, 0]:
                        continue
                    src = index[tuple((l[d] + o[d]) % nb[d] for d in range(3))]
                    if owner[src] != shard:
                        keys[g * cells + (k * S[1] + j) * S[0] + i] = owner[src]
    return keys


CASES = [((8, 8, 8), (4, 2, 2), None), ((8, 4, 6), (3, 3, 2), None),
         ((8, 8, 8), (4, 2, 2), ("reflect", "outflow", "periodic", "periodic", "outflow", "reflect"))]


@pytest.mark.parametrize("nx,nb,bc", CASES)
@pytest.mark.parametrize("nshards", [2, 3, 5])
def test_send_and_receive_lists_agree(nx, nb, bc, nshards):
    ph = _ph()
    cfg = ph.make_config(nx, nb, bc=bc)
    plans = {(s, p): ph.shard_plan(cfg, nshards, s, p) for s in range(nshards) for p in range(nshards)}
    ranges = [plans[(s, 0)][2] for s in range(nshards)]
    assert ranges[0][0] == 0 and ranges[-1][1] == nb[0] * nb[1] * nb[2]
    assert all(ranges[s][1] == ranges[s + 1][0] for s in range(nshards - 1))
    for s in range(nshards):
        send, recv, _ = plans[(s, s)]
        assert send.size == 0 and recv.size == 0
        for p in range(nshards):
            if p == s:
                continue
            assert np.array_equal(plans[(s, p)][0], plans[(p, s)][1]), (s, p)
            keys = plans[(s, p)][1]
            assert np.all(np.diff(keys) > 0)  # message order, each cell once
        allrecv = np.concatenate([plans[(s, p)][1] for p in range(nshards)])
        assert np.unique(allrecv).size == allrecv.size


@pytest.mark.parametrize("nx,nb", [((8, 8, 8), (4, 2, 2)), ((8, 4, 6), (3, 3, 2))])
@pytest.mark.parametrize("nshards", [2, 3])
def test_periodic_receive_lists_match_an_independent_derivation(nx, nb, nshards):
    ph = _ph()
    cfg = ph.make_config(nx, nb)
    for s in range(nshards):
        want = expected_recv(nx, nb, nshards, s)
        got = {}
        for p in range(nshards):
            for key in ph.shard_plan(cfg, nshards, s, p)[1]:
                got[int(key)] = p
        assert got == want, s


def test_bad_shard_arguments_rejected():
    ph = _ph()
    cfg = ph.make_config((8, 8, 8), (2, 1, 1))
    for args in [(0, 0, 0), (3, 0, 0), (2, 2, 0), (2, 0, 2)]:   # 3 shards > 2 blocks
        with pytest.raises(ph.PhError):
            ph.shard_plan(cfg, *args)
    with pytest.raises(ph.PhError):
        ph.shard_plan(ph.make_config((8, 8, 8), (2, 2, 2), max_level=1), 2, 0, 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import paper_2202_12309_gb300 as ph
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = ph.make_config((8, 8, 8), (4, 4, 2), bc=("outflow", "outflow") + ("periodic",) * 4)
    peer = 1 - rank
    send, recv, rng = ph.shard_plan(cfg, world, rank, peer)
    # exchange the send lists; each rank checks the peer's against its own
    # receive list
    n = torch.tensor([send.size], dtype=torch.int64)
    nn = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(nn, n)
    peer_send = torch.zeros(int(nn[peer].item()), dtype=torch.int64)
    ops = [dist.P2POp(dist.isend, torch.from_numpy(send), peer),
           dist.P2POp(dist.irecv, peer_send, peer)]
    for w in dist.batch_isend_irecv(ops):
        w.wait()
    ok = bool(np.array_equal(peer_send.numpy(), recv)) and recv.size > 0
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ok, rng))


def test_plans_agree_across_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [True, True]
    assert res[0][2] == (0, 16) and res[1][2] == (16, 32)
