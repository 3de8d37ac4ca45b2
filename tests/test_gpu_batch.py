"""Batched persistent launch: many independent meshes with uneven sizes in
one cooperative kernel per cycle.  Each member must match the same mesh run
alone through ph_mesh bit for bit (the per-tile arithmetic is shared, and a
face's flux does not depend on which tile computes it), and the FP64 oracle
within 1e-12.  The bounded grid barrier gives up and reports instead of
hanging."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from parity import describe, field_errors

pytestmark = pytest.mark.gpu


def _ph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_12309_gb300 as ph
    return ph


MEMBERS = [  # (cells per dim, block edge, centre, p_in)
    (32, 16, (0.1, -0.05, 0.0), 30.0),
    (64, 32, (-0.2, 0.1, 0.15), 80.0),
    (48, 16, (0.0, 0.0, 0.0), 10.0),
    (32, 32, (0.25, 0.2, -0.1), 55.0),
    (64, 16, (-0.1, -0.25, 0.05), 20.0),
]


def build(ph, precision, members=MEMBERS):
    cfgs, states = [], []
    for n, bk, c, pin in members:
        nb = n // bk
        cfg = ph.make_config((bk,) * 3, (nb,) * 3, precision=precision)
        cfgs.append(cfg)
        geo = W.Geometry((bk,) * 3, (nb,) * 3)
        leaves = ph.Mesh(cfg).tree()
        states.append(W.blast(geo, leaves, seed=n + bk, center=c, p_in=pin))
    return cfgs, states


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_single_meshes_bit_exact(precision):
    ph = _ph()
    cfgs, states = build(ph, precision)
    dtype = np.float32 if precision == "fp32" else np.float64
    B = ph.Batch(cfgs)
    for s, U in enumerate(states):
        B.set_state(s, U.astype(dtype))
    B.step(4)
    dts = B.dt()
    t, cyc = B.time()
    assert np.all(cyc == 4)
    launch = B.launch()
    for s, (cfg, U) in enumerate(zip(cfgs, states)):
        # FP32 batches whose blocks are 16 wide run the 16 x 16 paired tile on
        # every member (pair mode); FP64 batches the one-cell tile of the
        # launch choice.  The single mesh is pinned to the same kernel (the
        # paired and one-cell kernels round differently).
        if precision == "fp32":
            assert tuple(launch[:2]) == (16, 16)
        cfg.tile[:] = [16, 16, cfg.nx[2]]
        m = ph.Mesh(cfg)
        m.set_state(U.astype(dtype))
        m.step(4)
        assert np.array_equal(B.get_state(s), m.get_state()), "member %d" % s
        assert dts[s] == m.dt()
    rc, floors, nonfinite = B.status()
    assert rc == 0 and floors == 0 and nonfinite == 0


def test_batch_32_wide_paired_tiles_match_single_meshes():
    """Members whose blocks are all 32 wide take the 32 x 16 paired tile by
    default; a batch with 16-wide blocks refuses it."""
    ph = _ph()
    members = [m for m in MEMBERS if m[1] == 32]
    cfgs, states = build(ph, "fp32", members)
    B = ph.Batch(cfgs)
    assert tuple(B.launch()[:2]) == (32, 16)
    for s, U in enumerate(states):
        B.set_state(s, U.astype(np.float32))
    B.step(3)
    for s, (cfg, U) in enumerate(zip(cfgs, states)):
        for tile in ([32, 16, cfg.nx[2]], [16, 16, cfg.nx[2]]):   # both widths: the same bits
            cfg.tile[:] = tile
            m = ph.Mesh(cfg)
            m.set_state(U.astype(np.float32))
            m.step(3)
            assert np.array_equal(B.get_state(s), m.get_state()), (s, tile)
            m.close()
    mixed, _ = build(ph, "fp32")
    Bm = ph.Batch(mixed)
    with pytest.raises(ph.PhError):
        Bm.set_launch([32, 16, 16, 0])


def test_batch_members_match_oracle():
    ph = _ph()
    members = MEMBERS[:3]
    cfgs, states = build(ph, "fp64", members)
    B = ph.Batch(cfgs)
    for s, U in enumerate(states):
        B.set_state(s, U)
    B.step(3)
    for s, ((n, bk, c, pin), U) in enumerate(zip(members, states)):
        om = O.OracleMesh(O.make_config((bk,) * 3, (n // bk,) * 3))
        om.set_state(U)
        om.step(3)
        err = field_errors(B.get_state(s), om.get_state())
        assert err.max() <= 1e-12, "member %d: %s" % (s, describe(err))


def test_batch_autotune_keeps_results():
    ph = _ph()
    cfgs, states = build(ph, "fp32")
    B = ph.Batch(cfgs)
    for s, U in enumerate(states):
        B.set_state(s, U.astype(np.float32))
    B.step(2)
    before = [B.get_state(s).copy() for s in range(len(cfgs))]
    t0, c0 = B.time()
    choice = B.autotune(1)
    assert B.launch() == choice
    # the state and clocks are restored after tuning
    t1, c1 = B.time()
    assert np.array_equal(c0, c1) and np.array_equal(t0, t1)
    for s in range(len(cfgs)):
        assert np.array_equal(B.get_state(s), before[s])
    B.step(2)
    # the same launch choice from the start gives the same bits (the paired
    # and one-cell FP32 tiles round differently, so the choice matters)
    ref = ph.Batch(cfgs)
    ref.set_launch(choice)
    for s, U in enumerate(states):
        ref.set_state(s, U.astype(np.float32))
    ref.step(4)
    for s in range(len(cfgs)):
        assert np.array_equal(B.get_state(s), ref.get_state(s))


def test_barrier_timeout_is_reported_not_hung():
    ph = _ph()
    rc, gave_up = ph.debug_barrier_timeout(nctas=4, spin_limit=1 << 14)
    assert rc == -4 and gave_up == 4
    # the context is still usable afterwards
    cfgs, states = build(ph, "fp64", MEMBERS[:1])
    B = ph.Batch(cfgs)
    B.set_state(0, states[0])
    B.step(1)
    assert B.status()[0] == 0


def test_batch_benchmark_set_runs():
    """The 64-member workload (seeded sizes 32..128, blocks 16 or 32) runs and
    conserves mass per member."""
    ph = _ph()
    mem = W.batch_members(seed=0, nsim=64)
    cfgs, states = [], []
    for m in mem:
        nb = m.n // m.block
        cfg = ph.make_config((m.block,) * 3, (nb,) * 3, precision="fp32")
        cfgs.append(cfg)
        geo = W.Geometry((m.block,) * 3, (nb,) * 3)
        states.append(W.blast(geo, ph.Mesh(cfg).tree(), seed=m.seed, center=m.center,
                              p_in=m.p_in).astype(np.float32))
    B = ph.Batch(cfgs)
    for s, U in enumerate(states):
        B.set_state(s, U)
    B.step(3)
    rc, floors, nonfinite = B.status()
    assert rc == 0 and floors == 0 and nonfinite == 0
    for s in (0, 17, 63):
        m0 = states[s][:, 0].astype(np.float64).sum()
        m1 = B.get_state(s)[:, 0].astype(np.float64).sum()
        assert abs(m1 - m0) <= 1e-6 * m0
