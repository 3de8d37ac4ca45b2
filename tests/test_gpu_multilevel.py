"""GPU parity of trees deeper than two levels against the FP64 oracle: the
tree (bit-exact, including refinement cascades), the composite-field ghosts
(bit-exact), the evolved state (1e-12 per field per cycle) on static and
adaptive meshes with three and four levels, the Kelvin-Helmholtz problem,
physical boundaries, conservation, and a bitwise restart."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from parity import describe, field_errors

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _ph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_12309_gb300 as ph
    return ph


def pair(nx, nb, **kw):
    ph = _ph()
    ocfg = O.make_config(nx, nb, **kw)
    om = O.OracleMesh(ocfg)
    gm = ph.Mesh(ph.make_config(nx, nb, **kw))
    geo = W.Geometry(tuple(nx), tuple(nb), tuple(ocfg.xmin), tuple(ocfg.xmax))
    assert np.array_equal(gm.tree(), om.tree())
    return om, gm, geo


STATIC3 = dict(max_level=2, static_region=1, static_lo=(0.05, -0.1, 0.05), static_hi=(0.1, 0.1, 0.1))
STATIC4 = dict(max_level=3, static_region=1, static_lo=(-0.3, -0.3, -0.3), static_hi=(-0.28, -0.28, -0.28))


@pytest.mark.parametrize("kw", [STATIC3, STATIC4])
def test_static_multilevel_ghosts_bit_exact(kw):
    om, gm, geo = pair((8, 8, 8), (2, 2, 2), **kw)
    assert om.tree()[:, 0].max() == kw["max_level"]
    rng = np.random.default_rng(2)
    U = rng.uniform(0.5, 2.0, size=om.state_shape())
    om.set_state(U)
    gm.set_state(U)
    assert np.array_equal(gm.get_full(), om.get_full())


@pytest.mark.parametrize("kw", [STATIC3, STATIC4])
def test_static_multilevel_blast_matches_oracle(kw):
    om, gm, geo = pair((8, 8, 8), (2, 2, 2), **kw)
    U = W.blast(geo, om.tree(), seed=4, center=(0.08, 0.0, 0.08), radius=0.12, p_in=10.0)
    om.set_state(U)
    gm.set_state(U)
    t0 = gm.totals()
    for c in range(4):
        odt = om.step(1)[0]
        gm.step(1)
        err = field_errors(gm.get_state(), om.get_state())
        assert err.max() <= TOL64, "cycle %d: %s" % (c, describe(err))
        assert abs(gm.dt() - odt) <= TOL64 * odt
    t1 = gm.totals()
    assert np.all(np.abs(t1 - t0) <= 2e-14 * np.abs(t0).max()), t1 - t0


def test_refinement_cascade_matches_oracle():
    om, gm, geo = pair((8, 8, 8), (4, 4, 4), max_level=2)
    U = np.zeros(om.state_shape())
    U[:, 0] = 1.0
    U[:, 4] = 1.5
    om.set_state(U)
    gm.set_state(U)
    for target in ((0, 1, 1, 1), (1, 2, 2, 2)):
        tree = om.tree()
        flags = np.array([1 if tuple(t) == target else 0 for t in tree], dtype=np.int8)
        assert om.remesh(flags)
        assert gm.refine_where(flags)
        assert np.array_equal(gm.tree(), om.tree())
    assert np.array_equal(gm.get_full(), om.get_full())


@pytest.mark.parametrize("max_level", [2, 3])
def test_adaptive_kelvin_helmholtz_matches_oracle(max_level):
    kw = dict(max_level=max_level, adaptive=1, gamma=1.4, derefine_count=3,
              xmin=(-0.5, -0.5, -0.125), xmax=(0.5, 0.5, 0.125))
    om, gm, geo = pair((8, 8, 8), (4, 4, 1), **kw)
    U = W.kelvin_helmholtz(geo, om.tree(), seed=1)
    om.set_state(U)
    gm.set_state(U)
    for c in range(5):
        om.step(1)
        gm.step(1)
        ot, gt = om.tree(), gm.tree()
        if not np.array_equal(ot, gt):
            _, mb = om.tag()
            pytest.fail("tree differs at cycle %d (min |m_b - tol| = %.3g)"
                        % (c, np.min(np.abs(mb - 0.05))))
        err = field_errors(gm.get_state(), om.get_state(), gamma=1.4)
        assert err.max() <= TOL64, "cycle %d: %s" % (c, describe(err))
    assert gm.tree()[:, 0].max() == max_level
    rc, floors, nonfinite = gm.status()
    assert rc == 0 and floors == 0 and nonfinite == 0


def test_multilevel_with_reflecting_walls_matches_oracle():
    kw = dict(max_level=2, static_region=1, static_lo=(-0.5, -0.1, -0.1), static_hi=(-0.45, 0.1, 0.1),
              bc=("reflect", "reflect", "outflow", "outflow", "periodic", "periodic"))
    om, gm, geo = pair((8, 8, 8), (2, 2, 2), **kw)
    U = W.blast(geo, om.tree(), seed=8, center=(-0.4, 0.0, 0.0), radius=0.15, p_in=10.0)
    om.set_state(U)
    gm.set_state(U)
    assert np.array_equal(gm.get_full(), om.get_full())
    for c in range(3):
        om.step(1)
        gm.step(1)
        err = field_errors(gm.get_state(), om.get_state())
        assert err.max() <= TOL64, "cycle %d: %s" % (c, describe(err))


def test_multilevel_restart_is_bitwise(tmp_path):
    ph = _ph()
    nx, nb = (8, 8, 8), (4, 4, 1)
    cfg = ph.make_config(nx, nb, max_level=2, adaptive=1, gamma=1.4, derefine_count=2,
                         xmin=(-0.5, -0.5, -0.125), xmax=(0.5, 0.5, 0.125))
    m = ph.Mesh(cfg)
    geo = W.Geometry(nx, nb, tuple(cfg.xmin), tuple(cfg.xmax))
    m.set_state(W.kelvin_helmholtz(geo, m.tree(), seed=3))
    m.step(2)
    path = str(tmp_path / "ml.phr")
    m.save(path)
    m.step(3)
    r = ph.Mesh.load(path)
    r.step(3)
    assert np.array_equal(r.tree(), m.tree())
    assert np.array_equal(r.get_state(), m.get_state())
    assert r.dt() == m.dt()
