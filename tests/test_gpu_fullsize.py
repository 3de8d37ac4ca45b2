"""Parity at the workloads' full sizes, in the launch configurations the
benchmark times.

* uniform 256^3 zones in 512 blocks of 32^3 (the benchmark mesh, default
  tile): one full cycle against the FP64 oracle, FP64 and FP32;
* two-level blast, root 128^3 zones in 16^3 blocks with the static cube and
  adaptive refinement (960 leaves): all 50 cycles against the oracle (tree,
  refinement indicator and flags bit for bit, state within 1e-12 per field
  every cycle), then conservation and tiling.  The blast stays inside the
  pinned static cube, so the tree does not change in these 50 cycles;
* derefinement on the same 960-leaf mesh: 64 refined parents carrying a
  smooth state merge as soon as their children reach the derefinement age,
  against the oracle every cycle;
* the 256^3 wave in 4096 blocks of 16^3, FP32 on the 16-wide paired tile:
  one cycle against the oracle, cell by cell over the domain;
* the 64-member batch as the benchmark autotunes it, FP64 and FP32: a member
  of every size matches its own single-mesh run bit for bit (single meshes
  are pinned to the oracle above and in test_gpu_uniform)."""
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


@pytest.fixture(scope="module")
def oracle_256():
    nx, nb = (32, 32, 32), (8, 8, 8)
    om = O.OracleMesh(O.make_config(nx, nb))
    geo = W.Geometry(nx, nb)
    U0 = W.linear_wave(geo, om.tree(), seed=0, amp=1e-4, kvec=(1, 1, 1))
    om.set_state(U0)
    dt = om.step(1)[0]
    return U0, om.get_state(), dt, om.tree()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_uniform_256cube_one_cycle(oracle_256, precision):
    ph = _ph()
    U0, ref, odt, tree = oracle_256
    m = ph.Mesh(ph.make_config((32, 32, 32), (8, 8, 8), precision=precision))
    assert np.array_equal(m.tree(), tree)
    dtype = np.float32 if precision == "fp32" else np.float64
    m.set_state(U0.astype(dtype))
    m.step(1)
    err = field_errors(m.get_state(), ref)
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert err.max() <= tol, describe(err)
    assert abs(m.dt() - odt) <= (1e-12 if precision == "fp64" else 1e-6) * odt
    assert m.status()[0] == 0


def _global(U, tree, n):
    """Blocks U[b][v][k][j][i] of a uniform tree (rows: level, l1, l2, l3)
    assembled into one array [v][k][j][i]."""
    nb = [int(tree[:, 1 + d].max()) + 1 for d in range(3)]
    G = np.zeros((U.shape[1], nb[2] * n, nb[1] * n, nb[0] * n), dtype=np.float64)
    for b, (lev, l1, l2, l3) in enumerate(tree[:, :4]):
        G[:, l3 * n:(l3 + 1) * n, l2 * n:(l2 + 1) * n, l1 * n:(l1 + 1) * n] = U[b]
    return G


def test_uniform_256cube_16blocks_fp32_paired_16_wide(oracle_256):
    """The 256^3 benchmark wave in 4096 blocks of 16^3, FP32: the default
    tile is the 16-wide paired kernel; one cycle against the oracle's (run
    on 32^3 blocks: on a periodic uniform mesh the blocking does not change
    the method), compared cell by cell on the whole domain."""
    ph = _ph()
    U0, ref, odt, tree = oracle_256
    m = ph.Mesh(ph.make_config((16, 16, 16), (16, 16, 16), precision="fp32"))
    assert m.tile()[:2] == (16, 16)
    geo = W.Geometry((16, 16, 16), (16, 16, 16))
    U16 = W.linear_wave(geo, m.tree(), seed=0, amp=1e-4, kvec=(1, 1, 1))
    assert np.array_equal(_global(U16, m.tree(), 16), _global(U0, tree, 32))
    m.set_state(U16.astype(np.float32))
    m.step(1)
    G = _global(m.get_state().astype(np.float64), m.tree(), 16)
    R = _global(ref, tree, 32)
    err = field_errors(G[None], R[None])
    assert err.max() <= 2e-6, describe(err)
    assert abs(m.dt() - odt) <= 1e-6 * odt
    assert m.status()[0] == 0


def _cycle_against_oracle(m, om, c):
    """Tree and refinement flags bit for bit, state within 1e-12 per field.
    The indicator, |rho_{+1} - rho_{-1}| / (2 rho), is computed from each
    side's own state; with densities of order 1 that agree to ~1e-15 the
    indicators agree to ~1e-15 absolute, whatever their size (a difference
    quotient of nearly equal densities, ~5e-6 for the sound wave), so the
    check is absolute: 1e-11.  A flag decided that close to a tolerance would
    be a near-threshold event, reported as such."""
    assert np.array_equal(m.tree(), om.tree()), "cycle %d: tree" % c
    gf, gmb = m.tag()
    of, omb = om.tag()
    near = np.min(np.abs(omb - 0.05)), np.min(np.abs(omb - 0.0125))
    assert np.array_equal(gf, of), "cycle %d: flags (closest to a tolerance: %.3g, %.3g)" % ((c,) + near)
    assert np.abs(gmb - omb).max() <= 1e-11, "cycle %d: indicator %.3g" % (c, np.abs(gmb - omb).max())
    err, plain = field_errors(m.get_state(), om.get_state(), with_plain=True)
    assert err.max() <= 1e-12, "cycle %d: %s" % (c, describe(err, plain))


def _indicator_on_oracle_state(m, om):
    """The GPU indicator of the oracle's own state is the oracle's, bit for bit."""
    m.set_state(om.get_state())
    gf, gmb = m.tag()
    of, omb = om.tag()
    assert np.array_equal(gmb, omb) and np.array_equal(gf, of)


@pytest.mark.slow
def test_two_level_blast_full_size():
    ph = _ph()
    nx, nb = (16, 16, 16), (8, 8, 8)
    kw = dict(max_level=1, static_region=1, adaptive=1)
    om = O.OracleMesh(O.make_config(nx, nb, **kw))
    m = ph.Mesh(ph.make_config(nx, nb, **kw))
    tree = m.tree()
    assert np.array_equal(tree, om.tree())
    assert len(tree) == 512 - 64 + 512
    geo = W.Geometry(nx, nb)
    U0 = W.blast(geo, tree, seed=0)
    om.set_state(U0)
    m.set_state(U0)
    t0 = m.totals()
    for c in range(50):
        odt = om.step(1)[0]
        m.step(1)
        assert abs(m.dt() - odt) <= 1e-12 * odt, "cycle %d: dt" % c
        _cycle_against_oracle(m, om, c)
    t1 = m.totals()
    assert np.all(np.abs(t1 - t0) <= 1e-12 * np.abs(t0).max()), t1 - t0
    rc, floors, nonfinite = m.status()
    assert rc == 0 and floors == 0 and nonfinite == 0
    t, cyc = m.time()
    assert cyc == 50
    _indicator_on_oracle_state(m, om)
    tree = m.tree()
    cover = np.zeros((16, 16, 16), dtype=int)
    for l, a, b, c in tree:
        s = 2 if l == 0 else 1
        a, b, c = (int(v) * s for v in (a, b, c))
        cover[c:c + s, b:b + s, a:a + s] += 1
    assert np.all(cover == 1)


@pytest.mark.slow
def test_derefinement_full_size():
    """The 960-leaf mesh of the two-level blast built by explicit refinement
    of the central 4^3 root blocks (no static region), carrying the 1e-4
    sound wave: every indicator is below the derefinement tolerance, so all
    64 parents merge at the cycle their children reach derefine_count (10)
    cycles of age."""
    ph = _ph()
    nx, nb = (16, 16, 16), (8, 8, 8)
    kw = dict(max_level=1, adaptive=1, derefine_count=10)
    om = O.OracleMesh(O.make_config(nx, nb, **kw))
    m = ph.Mesh(ph.make_config(nx, nb, **kw))
    flags = np.zeros(512, dtype=np.int8)
    for b, (l, a, j, k) in enumerate(om.tree()):
        if 2 <= a < 6 and 2 <= j < 6 and 2 <= k < 6:
            flags[b] = 1
    assert om.remesh(flags, check_age=False)
    assert m.refine_where(flags, check_age=False)
    assert np.array_equal(m.tree(), om.tree()) and m.nblocks == 960
    geo = W.Geometry(nx, nb)
    U0 = W.linear_wave(geo, om.tree(), seed=1, amp=1e-4, kvec=(1, 1, 1))
    om.set_state(U0)
    m.set_state(U0)
    merged_at = None
    for c in range(12):
        om.step(1)
        m.step(1)
        _cycle_against_oracle(m, om, c)
        if merged_at is None and m.nblocks == 512:
            merged_at = c
    assert merged_at is not None and 8 <= merged_at <= 10, merged_at
    _indicator_on_oracle_state(m, om)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_full_members_match_single_meshes(precision):
    """FP32: the autotuned launch is the paired tile on every member; single
    meshes pinned to the same tile shape run the same kernel arithmetic."""
    ph = _ph()
    mem = W.batch_members(seed=0, nsim=64)
    dtype = np.float32 if precision == "fp32" else np.float64
    cfgs, states = [], []
    for mb in mem:
        nb = mb.n // mb.block
        cfg = ph.make_config((mb.block,) * 3, (nb,) * 3, precision=precision)
        cfgs.append(cfg)
        geo = W.Geometry((mb.block,) * 3, (nb,) * 3)
        states.append(W.blast(geo, ph.Mesh(cfg).tree(), seed=mb.seed, center=mb.center,
                              p_in=mb.p_in).astype(dtype))
    B = ph.Batch(cfgs)
    for s, U in enumerate(states):
        B.set_state(s, U)
    launch = B.autotune(1)
    B.step(3)
    seen = set()
    for s, mb in enumerate(mem):
        key = (mb.n, mb.block)
        if key in seen:
            continue
        seen.add(key)
        if precision == "fp32":
            cfgs[s].tile[:] = [launch[0], launch[1], cfgs[s].nx[2]]
        m = ph.Mesh(cfgs[s])
        m.set_state(states[s])
        m.step(3)
        assert np.array_equal(B.get_state(s), m.get_state()), key
        m.close()
    assert len(seen) >= 4
