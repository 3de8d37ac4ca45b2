"""GPU parity of the physical boundaries (outflow, reflecting) against the
FP64 oracle: ghost values bit-exact on uniform and two-level meshes, the
evolved state within 1e-12 per field per cycle, the block tree bit-exact,
FP32 within the stated per-field bound, and a closed box conserving mass and
energy; batched meshes and the adjoint refuse non-periodic meshes."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from parity import describe, field_errors

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
MIXED = ("outflow", "reflect", "periodic", "periodic", "reflect", "outflow")


def _ph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_12309_gb300 as ph
    return ph


def pair(nx, nb, precision="fp64", **kw):
    ph = _ph()
    ocfg = O.make_config(nx, nb, **kw)
    om = O.OracleMesh(ocfg)
    gm = ph.Mesh(ph.make_config(nx, nb, precision=precision, **kw))
    geo = W.Geometry(tuple(nx), tuple(nb), tuple(ocfg.xmin), tuple(ocfg.xmax))
    assert np.array_equal(gm.tree(), om.tree())
    return om, gm, geo


def test_uniform_ghosts_bit_exact():
    om, gm, geo = pair((8, 8, 8), (2, 3, 2), bc=MIXED)
    rng = np.random.default_rng(1)
    U = rng.uniform(0.5, 2.0, size=om.state_shape())
    om.set_state(U)
    gm.set_state(U)
    assert np.array_equal(gm.get_full(), om.get_full())


@pytest.mark.parametrize("bc", [MIXED, ("reflect",) * 6, ("outflow",) * 6])
def test_uniform_blast_matches_oracle(bc):
    om, gm, geo = pair((16, 16, 16), (2, 2, 2), bc=bc)
    U = W.blast(geo, om.tree(), seed=3, center=(0.3, -0.35, 0.25), radius=0.15)
    om.set_state(U)
    gm.set_state(U)
    for c in range(8):
        odt = om.step(1)[0]
        gm.step(1)
        err = field_errors(gm.get_state(), om.get_state())
        assert err.max() <= TOL64, "cycle %d: %s" % (c, describe(err))
        assert abs(gm.dt() - odt) <= TOL64 * odt


def test_two_level_with_boundaries_matches_oracle():
    kw = dict(max_level=1, static_region=1, adaptive=1, derefine_count=2, bc=MIXED,
              static_lo=(-0.45, -0.2, 0.1), static_hi=(-0.1, 0.2, 0.45))
    om, gm, geo = pair((8, 8, 8), (4, 4, 4), **kw)
    U = W.blast(geo, om.tree(), seed=6, center=(-0.35, 0.0, 0.35), radius=0.15)
    om.set_state(U)
    gm.set_state(U)
    assert np.array_equal(gm.get_full(), om.get_full())
    for c in range(5):
        om.step(1)
        gm.step(1)
        assert np.array_equal(gm.tree(), om.tree()), "tree differs at cycle %d" % c
        err = field_errors(gm.get_state(), om.get_state())
        assert err.max() <= TOL64, "cycle %d: %s" % (c, describe(err))
    # ghosts of the evolved state: the images of interiors that agree to 1e-12
    assert field_errors(gm.get_full(), om.get_full()).max() <= TOL64


def test_fp32_with_boundaries_against_fp64_oracle():
    om, gm, geo = pair((16, 16, 16), (2, 2, 2), precision="fp32", bc=MIXED)
    U = W.blast(geo, om.tree(), seed=3, center=(0.3, -0.35, 0.25), radius=0.15)
    om.set_state(U)
    gm.set_state(U.astype(np.float32))
    om.step(10)
    gm.step(10)
    err = field_errors(gm.get_state(), om.get_state())
    bound = np.array([2e-5, 1e-4, 1e-4, 1e-4, 2e-5])
    assert np.all(err <= bound), describe(err)


def test_closed_box_conserves_mass_and_energy_on_gpu():
    ph = _ph()
    nx, nb = (16, 16, 16), (2, 2, 2)
    gm = ph.Mesh(ph.make_config(nx, nb, bc=("reflect",) * 6))
    geo = W.Geometry(nx, nb)
    gm.set_state(W.blast(geo, gm.tree(), seed=2, center=(0.2, 0.1, -0.15), radius=0.2, p_in=10.0))
    t0 = gm.totals()
    gm.step(12)
    t1 = gm.totals()
    for v in (0, 4):
        assert abs(t1[v] - t0[v]) <= 1e-13 * abs(t0[v]), (v, t0[v], t1[v])


def test_batch_and_adjoint_refuse_non_periodic_meshes():
    ph = _ph()
    cfg = ph.make_config((8, 8, 8), (1, 1, 1), bc=("outflow",) * 6)
    with pytest.raises(ph.PhError, match="PH_ERR_INVALID"):
        ph.Batch([cfg])
    m = ph.Mesh(cfg)
    U = np.zeros(m.state_shape())
    U[:, 0] = 1.0
    U[:, 4] = 1.0
    m.set_state(U)
    with pytest.raises(ph.PhError, match="PH_ERR_INVALID"):
        m.adjoint(U, U, 2, 1)
