"""GPU parity of the two-level path against the FP64 oracle: composite ghost
exchange (copy / restriction / prolongation, bit-exact), flux correction at
fine-coarse faces, refinement indicator and flags (bit-exact), remesh data
movement (bit-exact), the block tree (bit-exact) and the evolved state
(1e-12 per field per cycle)."""
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


def pair(nx=(8, 8, 8), nb=(4, 4, 4), **kw):
    ph = _ph()
    args = dict(max_level=1, static_region=1)
    args.update(kw)
    ocfg = O.make_config(nx, nb, **args)
    om = O.OracleMesh(ocfg)
    gm = ph.Mesh(ph.make_config(nx, nb, **args))
    geo = W.Geometry(tuple(nx), tuple(nb), tuple(ocfg.xmin), tuple(ocfg.xmax))
    assert np.array_equal(gm.tree(), om.tree())
    return om, gm, geo


def smooth_flow(geo, leaves, seed=4):
    U = W.smooth_random_density(geo, leaves, seed=seed)
    U[:, 1] = 0.3 * U[:, 0]
    U[:, 2] = -0.2 * U[:, 0]
    U[:, 4] += 0.5 * (0.09 + 0.04) * U[:, 0]
    return U


def test_two_level_ghosts_bit_exact():
    om, gm, geo = pair()
    rng = np.random.default_rng(3)
    U = rng.uniform(0.5, 1.5, size=om.state_shape())
    om.set_state(U)
    gm.set_state(U)
    assert np.array_equal(gm.get_full(), om.get_full())


def test_two_level_cycles_match_oracle():
    om, gm, geo = pair()
    U = smooth_flow(geo, om.tree())
    om.set_state(U)
    gm.set_state(U)
    for c in range(4):
        odt = om.step(1)[0]
        gm.step(1)
        assert abs(gm.dt() - odt) <= TOL64 * odt
        err = field_errors(gm.get_state(), om.get_state())
        assert err.max() <= TOL64, "cycle %d: %s" % (c, describe(err))
    t0 = gm.totals()
    gm.step(3)
    t1 = gm.totals()
    assert np.all(np.abs(t1 - t0) <= 1e-13 * np.abs(t0).max()), t1 - t0


def test_two_level_blast_static_region():
    om, gm, geo = pair()
    U = W.blast(geo, om.tree(), seed=1)
    om.set_state(U)
    gm.set_state(U)
    for c in range(3):
        om.step(1)
        gm.step(1)
        err = field_errors(gm.get_state(), om.get_state())
        assert err.max() <= TOL64, "cycle %d: %s" % (c, describe(err))


def test_indicator_and_flags_bit_exact():
    om, gm, geo = pair(static_region=0, nb=(4, 4, 4))
    U = W.blast(geo, om.tree(), seed=2, radius=0.2, noise=0.02)
    om.set_state(U)
    gm.set_state(U)
    of, omb = om.tag()
    gf, gmb = gm.tag()
    assert np.array_equal(gmb, omb)
    assert np.array_equal(gf, of)


def test_explicit_remesh_bit_exact():
    om, gm, geo = pair(static_region=0)
    U = smooth_flow(geo, om.tree(), seed=9)
    om.set_state(U)
    gm.set_state(U)
    flags = np.zeros(om.nblocks, dtype=np.int8)
    flags[[1, 6, 20, 33, 47]] = 1
    assert om.remesh(flags, check_age=False)
    assert gm.refine_where(flags, check_age=False)
    assert np.array_equal(gm.tree(), om.tree())
    assert np.array_equal(gm.get_full(), om.get_full())
    # merge two of them back
    tree = om.tree()
    flags = np.zeros(len(tree), dtype=np.int8)
    fine = np.where(tree[:, 0] == 1)[0]
    flags[fine[:16]] = -1
    assert om.remesh(flags, check_age=False)
    assert gm.refine_where(flags, check_age=False)
    assert np.array_equal(gm.tree(), om.tree())
    assert np.array_equal(gm.get_full(), om.get_full())


def test_adaptive_refinement_follows_oracle():
    om, gm, geo = pair(static_region=0, adaptive=1, derefine_count=2)
    U = W.blast(geo, om.tree(), seed=5, radius=0.15)
    om.set_state(U)
    gm.set_state(U)
    n0 = om.nblocks
    for c in range(6):
        om.step(1)
        gm.step(1)
        ot, gt = om.tree(), gm.tree()
        if not np.array_equal(ot, gt):
            # a flag decided within round-off of a tolerance: report the margin
            _, mb = om.tag()
            pytest.fail("tree differs at cycle %d (min |m_b - tol| = %.3g)"
                        % (c, np.min(np.abs(mb - 0.05))))
        err = field_errors(gm.get_state(), om.get_state())
        assert err.max() <= TOL64, "cycle %d: %s" % (c, describe(err))
    assert om.nblocks > n0   # the blast refined the mesh
