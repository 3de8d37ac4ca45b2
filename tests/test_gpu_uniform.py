"""GPU parity of the uniform-mesh hot path (ghost exchange K1, fused stage K3,
dt reduction K5) against the FP64 oracle, cycle by cycle, through the C ABI.

Bar: FP64 within 1e-12 relative L-inf per field per cycle (and dt within
1e-12); block tree bit-exact; FP32 within the stated per-field tolerance."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from parity import describe, field_errors

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def run_pair(nx, nb, init, cycles, precision="fp64", tile=(0, 0, 0), **cfgkw):
    _torch()
    import paper_2202_12309_gb300 as ph
    ocfg = O.make_config(nx, nb, **cfgkw)
    om = O.OracleMesh(ocfg)
    gm = ph.Mesh(ph.make_config(nx, nb, precision=precision, tile=tile, **cfgkw))
    assert np.array_equal(gm.tree(), om.tree())
    geo = W.Geometry(tuple(nx), tuple(nb), tuple(ocfg.xmin), tuple(ocfg.xmax))
    U0 = init(geo, om.tree())
    om.set_state(U0)
    gm.set_state(U0)
    dt_tol = TOL64 if precision == "fp64" else 1e-5
    assert abs(gm.dt() - om.compute_dt()) <= dt_tol * om.compute_dt()
    errs, dterr = [], []
    gamma = cfgkw.get("gamma", 5.0 / 3.0)
    for c in range(cycles):
        odt = om.step(1)[0]
        gm.step(1)
        gdt = gm.dt()
        dterr.append(abs(gdt - odt) / odt)
        errs.append(field_errors(gm.get_state(), om.get_state(), gamma))
    t, cyc = gm.time()
    assert cyc == cycles
    ot, _, _ = om.time()
    assert abs(t - ot) <= dt_tol * ot
    rc, floors, nonfinite = gm.status()
    assert floors == 0 and nonfinite == 0 and rc == 0
    return np.array(errs), np.array(dterr), gm, om


def blast(geo, leaves):
    return W.blast(geo, leaves, seed=0)


def test_blast_32cube_8blocks_10cycles_fp64():
    """32^3 zones as 8 blocks of 16^3, blast wave, 10 cycles (the correctness workload)."""
    errs, dterr, gm, om = run_pair((16, 16, 16), (2, 2, 2), blast, 10)
    assert errs.max() <= TOL64, describe(errs.max(axis=0))
    assert dterr.max() <= TOL64
    assert gm.launches_per_cycle() == 3   # periodic: the stages fill the ghost zones


@pytest.mark.parametrize("nx,nb,tile", [
    ((12, 12, 12), (2, 2, 2), (8, 8, 12)),     # ragged tiles in x1 and x2
    ((24, 16, 8), (1, 2, 3), (16, 8, 8)),       # non-cubic blocks, ragged x1
    ((16, 16, 32), (2, 1, 1), (16, 16, 8)),     # 4 chunks along x3
    ((16, 16, 16), (1, 1, 1), (32, 8, 16)),     # one block, periodic onto itself
    ((4, 4, 4), (3, 3, 3), (8, 8, 4)),          # smallest block (2 ghost widths)
    ((32, 32, 32), (2, 1, 1), (32, 8, 13)),     # ragged x3 chunks
])
def test_blast_shapes_fp64(nx, nb, tile):
    errs, dterr, gm, om = run_pair(nx, nb, blast, 3, tile=tile)
    assert gm.tile() == tuple(tile)
    assert errs.max() <= TOL64, describe(errs.max(axis=0))
    assert dterr.max() <= TOL64


def test_linear_wave_fp64():
    """The sound-wave workload (amplitude 1e-4): momentum errors are measured
    against the flow's momentum unit rho c_s (see tests/parity.py)."""
    init = lambda geo, leaves: W.linear_wave(geo, leaves, seed=1, kvec=(1, 1, 0))
    errs, dterr, gm, om = run_pair((16, 16, 16), (2, 2, 2), init, 10)
    assert errs.max() <= TOL64, describe(errs.max(axis=0))
    assert dterr.max() <= TOL64


def test_ghosts_match_oracle_bit_exact():
    _torch()
    import paper_2202_12309_gb300 as ph
    nx, nb = (8, 12, 16), (3, 2, 2)
    om = O.OracleMesh(O.make_config(nx, nb))
    gm = ph.Mesh(ph.make_config(nx, nb))
    rng = np.random.default_rng(4)
    U = rng.uniform(0.5, 2.0, size=om.state_shape())
    om.set_state(U)
    gm.set_state(U)
    assert np.array_equal(gm.get_full(), om.get_full())


def test_uniform_state_bit_exact():
    _torch()
    import paper_2202_12309_gb300 as ph
    gm = ph.Mesh(ph.make_config((16, 16, 16), (2, 2, 2)))
    U = np.zeros(gm.state_shape())
    U[:, 0], U[:, 1], U[:, 2], U[:, 3], U[:, 4] = 1.3, 0.2, -0.7, 0.05, 2.5
    gm.set_state(U)
    gm.step(3)
    assert np.array_equal(gm.get_state(), U)


def test_conservation_gpu():
    _torch()
    import paper_2202_12309_gb300 as ph
    nx, nb = (16, 16, 16), (2, 2, 2)
    gm = ph.Mesh(ph.make_config(nx, nb))
    geo = W.Geometry(nx, nb)
    gm.set_state(W.blast(geo, gm.tree(), seed=2))
    t0 = gm.totals()
    gm.step(10)
    t1 = gm.totals()
    assert np.all(np.abs(t1 - t0) <= 1e-13 * np.abs(t0).max())


# FP32 state and fluxes against the FP64 oracle: stated per-field bound after
# 10 cycles of the blast workload (round-off of ~1e-7 per operation, carried
# through the nonlinear update; momenta are relative to their own max).
TOL32 = {"rho": 2e-5, "m1": 1e-4, "m2": 1e-4, "m3": 1e-4, "E": 2e-5}


def test_blast_fp32_against_fp64_oracle():
    errs, dterr, gm, om = run_pair((16, 16, 16), (2, 2, 2), blast, 10, precision="fp32")
    worst = errs.max(axis=0)
    for v, name in enumerate(("rho", "m1", "m2", "m3", "E")):
        assert worst[v] <= TOL32[name], describe(worst)
    assert dterr.max() <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,nb,tile", [
    ((16, 16, 16), (2, 2, 2), (16, 16, 16)),
    ((32, 32, 32), (2, 1, 1), (32, 8, 32)),
    ((12, 12, 12), (2, 2, 2), (8, 8, 12)),     # ragged tiles: TMA boxes reach past the block
    ((24, 16, 8), (1, 2, 3), (16, 8, 8)),
])
def test_tma_and_plain_loads_bit_identical(precision, nx, nb, tile, monkeypatch):
    """Planes staged by TMA tensor copies or by per-thread loads feed the same
    arithmetic: results must agree bit for bit."""
    _torch()
    import paper_2202_12309_gb300 as ph
    if precision == "fp32" and tuple(tile[:2]) == (16, 16):
        tile = (16, 8, tile[2])  # FP32 16 x 16 tiles with TMA staging run the paired kernel
    geo = W.Geometry(nx, nb)
    out = {}
    for mode in ("tma", "plain"):
        monkeypatch.setenv("PH_STAGE_LOADS", mode)
        m = ph.Mesh(ph.make_config(nx, nb, precision=precision, tile=tile))
        U = W.blast(geo, m.tree(), seed=3).astype(np.float32 if precision == "fp32" else np.float64)
        m.set_state(U)
        m.step(3)
        out[mode] = (m.get_state(), m.dt())
        assert m.status()[0] == 0
        m.close()
    assert np.array_equal(out["tma"][0], out["plain"][0])
    assert out["tma"][1] == out["plain"][1]


def test_default_chunks_fill_the_gpu_on_small_meshes():
    """Default tiles march 16 planes; where shorter chunks (8 or 4 planes)
    need fewer whole waves of resident CTAs for the planes they march, as on a
    mesh too small to fill the GPU, they are taken; the result does not
    depend on the chunk length."""
    _torch()
    import paper_2202_12309_gb300 as ph
    big = ph.Mesh(ph.make_config((32, 32, 32), (4, 4, 4)))
    assert big.tile() == (16, 16, 16)
    small = ph.Mesh(ph.make_config((32, 32, 32), (2, 2, 2)))
    assert small.tile() == (16, 16, 4)
    nx, nb = (32, 32, 32), (2, 2, 2)
    geo = W.Geometry(nx, nb)
    U = W.blast(geo, small.tree(), seed=8, radius=0.2)
    fixed = ph.Mesh(ph.make_config(nx, nb, tile=(16, 16, 16)))
    small.set_state(U)
    fixed.set_state(U)
    small.step(2)
    fixed.step(2)
    assert np.array_equal(small.get_state(), fixed.get_state())


def test_multilevel_chunk_follows_the_leaf_count():
    """On a multi-level mesh with default tiles the chunk depth is chosen for
    the current leaf count and chosen again after a remesh; the cycles agree
    bit for bit with a mesh whose chunks are fixed."""
    _torch()
    import paper_2202_12309_gb300 as ph
    nx, nb = (16, 16, 16), (8, 8, 8)
    kw = dict(max_level=1, static_region=1, adaptive=1)
    auto = ph.Mesh(ph.make_config(nx, nb, **kw))
    fixed = ph.Mesh(ph.make_config(nx, nb, tile=(16, 16, 16), **kw))
    assert auto.tile()[:2] == (16, 16) and auto.tile()[2] in (8, 16)
    if auto.nblocks == 960:   # 1920 CTAs: 7 waves of 8 planes beat 4 waves of 16
        assert auto.tile()[2] == 8
    geo = W.Geometry(nx, nb)
    U = W.blast(geo, auto.tree(), seed=0)
    auto.set_state(U)
    fixed.set_state(U)
    for _ in range(3):
        auto.step(1)
        fixed.step(1)
        assert np.array_equal(auto.tree(), fixed.tree())
        assert np.array_equal(auto.get_state(), fixed.get_state())
