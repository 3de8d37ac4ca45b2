"""Domain decomposition on the GPU: a uniform mesh split into shards (Sec.
2.1: contiguous ranges of the Z-ordered blocks) whose ghost zones across
shard boundaries are filled by the pack / exchange / unpack of Sec. 3.7 and
whose dt is the max-reduction over shards (Sec. 3.10) must advance exactly
as the same mesh in one piece: state, dt and time bit for bit every cycle.

* shards of one process (ph_shards_sync / ph_shards_step): periodic FP64
  with 2 and 3 shards, FP32 on the paired kernel, reflecting and outflow
  walls (the exchange carries mirrored momenta across shard boundaries);
* one shard per process: two processes on this GPU talking over gloo
  (host-staged messages, the dt all-reduced), against the same mesh in one
  process.  No kernel waits on another process: every wait is on the host."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_12309_gb300 as ph
    return ph


def _compare_runs(ph, nx, nb, nshards, cycles, precision="fp64", bc=None):
    cfg = ph.make_config(nx, nb, precision=precision, bc=bc)
    whole = ph.Mesh(cfg)
    sm = ph.ShardedMesh(cfg, nshards)
    assert np.array_equal(sm.tree(), whole.tree())
    geo = W.Geometry(nx, nb)
    dtype = np.float32 if precision == "fp32" else np.float64
    U = W.blast(geo, whole.tree(), seed=11, center=(0.2, -0.15, 0.1), radius=0.2, p_in=40.0).astype(dtype)
    whole.set_state(U)
    sm.set_state(U)
    assert sm.dt() == whole.dt()
    for c in range(cycles):
        whole.step(1)
        sm.step(1)
        assert np.array_equal(sm.get_state(), whole.get_state()), "cycle %d" % c
        assert sm.dt() == whole.dt() and sm.time() == whole.time(), "cycle %d" % c
    for sh in sm.shards:
        assert sh.status()[0] == 0
    # per-shard totals add up to the mesh's (momentum totals are round-off
    # around zero: compare on the scale of the largest total)
    tot = sum(sh.totals() for sh in sm.shards)
    ref = whole.totals()
    assert np.all(np.abs(tot - ref) <= 1e-13 * np.abs(ref).max())
    sm.close()
    whole.close()


@pytest.mark.parametrize("nshards", [2, 3])
def test_shards_match_one_mesh_periodic_fp64(nshards):
    ph = _ph()
    _compare_runs(ph, (16, 16, 16), (4, 2, 2), nshards, 10)


def test_shards_match_one_mesh_fp32_paired_kernel():
    ph = _ph()
    cfg = ph.make_config((32, 32, 32), (2, 2, 2), precision="fp32")
    assert tuple(ph.Shard(cfg, 2, 0).tile())[:2] == (32, 16)
    _compare_runs(ph, (32, 32, 32), (2, 2, 2), 2, 6, precision="fp32")


def test_shards_match_one_mesh_fp32_16_wide_paired_kernel():
    ph = _ph()
    cfg = ph.make_config((16, 16, 16), (4, 2, 2), precision="fp32")
    assert tuple(ph.Shard(cfg, 3, 0).tile())[:2] == (16, 16)
    _compare_runs(ph, (16, 16, 16), (4, 2, 2), 3, 6, precision="fp32")


def test_shards_match_one_mesh_with_walls():
    ph = _ph()
    bc = ("reflect", "outflow", "periodic", "periodic", "outflow", "reflect")
    _compare_runs(ph, (16, 16, 16), (4, 2, 2), 3, 8, bc=bc)


def test_shard_refuses_whole_mesh_calls():
    ph = _ph()
    cfg = ph.make_config((16, 16, 16), (2, 1, 1))
    sh = ph.Shard(cfg, 2, 0)
    sh.set_state(np.ones(sh.state_shape()) * np.array([1.0, 0, 0, 0, 2.0])[None, :, None, None, None])
    with pytest.raises(ph.PhError):
        sh.step(1)
    with pytest.raises(ph.PhError):
        ph.Shard(ph.make_config((16, 16, 16), (2, 1, 1), max_level=1), 2, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


NX, NB, CYCLES = (16, 16, 16), (4, 2, 2), 5


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import paper_2202_12309_gb300 as ph
    import workloads as W
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = ph.make_config(NX, NB)
    ds = ph.DistShard(cfg)
    a, b = ds.range
    geo = W.Geometry(NX, NB)
    # this shard's blocks only (the generator is keyed by global cell index)
    U = W.blast(geo, ds.m.tree(), seed=11, center=(0.2, -0.15, 0.1), radius=0.2, p_in=40.0)
    ds.set_state(U)
    ds.step(CYCLES)
    out = ds.get_state()
    t = ds.m.time()
    dt = ds.m.dt()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, a, b, out, t, dt))


def test_one_shard_per_process_over_gloo():
    ph = _ph()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    cfg = ph.make_config(NX, NB)
    whole = ph.Mesh(cfg)
    geo = W.Geometry(NX, NB)
    U = W.blast(geo, whole.tree(), seed=11, center=(0.2, -0.15, 0.1), radius=0.2, p_in=40.0)
    whole.set_state(U)
    whole.step(CYCLES)
    G = whole.get_state()
    for rank, a, b, out, t, dt in res:
        assert np.array_equal(out, G[a:b]), rank
        assert t == whole.time() and dt == whole.dt()
    assert res[0][2] == res[1][1] and res[1][2] == G.shape[0]
