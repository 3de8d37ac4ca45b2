"""Pins of the oracle's trees deeper than two levels (more levels with the
one-level rule between touching leaves, and the Kelvin-Helmholtz problem of
Sec. 4.1): the tree tiles the domain and touching leaves
differ by one level at most (brute force), refinement cascades and blocked
merges follow that rule, a uniform state is preserved bit for bit, mass,
momentum and energy are conserved to round-off across every level jump,
linear data are prolonged exactly through two levels, restriction undoes
prolongation, and the shear layers of the Kelvin-Helmholtz problem refine to
the finest level.  CPU only."""
import itertools

import numpy as np

import oracle as O
import workloads as W


def make(nx, nb, **kw):
    cfg = O.make_config(nx, nb, **kw)
    m = O.OracleMesh(cfg)
    geo = W.Geometry(tuple(nx), tuple(nb), tuple(cfg.xmin), tuple(cfg.xmax))
    return m, geo, cfg


def extents(tree, nb, max_level):
    """Leaf boxes in units of finest-level blocks: (lo[3], hi[3], level)."""
    out = []
    for lev, l1, l2, l3 in tree:
        f = 1 << (max_level - lev)
        lo = np.array([l1, l2, l3]) * f
        out.append((lo, lo + f, lev))
    return out


def check_tiling_and_balance(tree, nb, max_level, periodic=(True, True, True)):
    """Every finest-level block covered once; touching leaves (faces, edges,
    corners, periodic images included) differ by at most one level."""
    N = np.array(nb) << max_level
    owner = -np.ones(tuple(N[::-1]), dtype=np.int64)
    boxes = extents(tree, nb, max_level)
    for b, (lo, hi, lev) in enumerate(boxes):
        sl = owner[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        assert np.all(sl == -1), "overlap"
        sl[...] = b
    assert np.all(owner >= 0), "gap"
    level = np.array([lv for _, _, lv in boxes])
    # touching = some finest block of A is adjacent (26-neighbourhood) to one of B
    for off in itertools.product((-1, 0, 1), repeat=3):
        if off == (0, 0, 0):
            continue
        sh = owner
        for ax, o in zip((2, 1, 0), off):
            if o == 0:
                continue
            sh = np.roll(sh, -o, axis=ax)
        a, b = owner, sh
        if not all(periodic):
            mask = np.ones_like(owner, dtype=bool)
            for ax, o, per in zip((2, 1, 0), off, periodic):
                if o and not per:
                    idx = [slice(None)] * 3
                    idx[ax] = slice(-1, None) if o > 0 else slice(0, 1)
                    mask[tuple(idx)] = False
            a, b = a[mask], b[mask]
        diff = np.abs(level[a] - level[b])
        assert diff.max() <= 1, "leaves two levels apart touch (offset %s)" % (off,)


def test_static_three_and_four_level_trees_tile_and_balance():
    for ml in (2, 3):
        m, geo, cfg = make((8, 8, 8), (2, 2, 2), max_level=ml, static_region=1,
                           static_lo=(0.05, 0.05, 0.05), static_hi=(0.1, 0.1, 0.1))
        tree = m.tree()
        assert tree[:, 0].max() == ml
        check_tiling_and_balance(tree, (2, 2, 2), ml)
        # Z-order: keys strictly increase
        keys = [O.morton(int(l), int(a), int(b), int(c), ml) for l, a, b, c in tree]
        assert all(k1 < k2 for k1, k2 in zip(keys, keys[1:]))


def test_refinement_cascades_to_keep_one_level_jumps():
    """Refining the level-1 leaf in the corner of a refined root block makes
    the 7 root blocks around that corner refine as well."""
    m, geo, cfg = make((8, 8, 8), (4, 4, 4), max_level=2)
    U = np.zeros(m.state_shape())
    U[:, 0] = 1.0
    U[:, 4] = 1.5
    m.set_state(U)
    flags = np.zeros(m.nblocks, dtype=np.int8)
    tree = m.tree()
    flags[[i for i, t in enumerate(tree) if tuple(t) == (0, 1, 1, 1)][0]] = 1
    assert m.remesh(flags)
    tree = m.tree()
    assert len(tree) == 64 - 1 + 8
    flags = np.zeros(m.nblocks, dtype=np.int8)
    flags[[i for i, t in enumerate(tree) if tuple(t) == (1, 2, 2, 2)][0]] = 1   # the (0,0,0) corner
    assert m.remesh(flags)
    tree = m.tree()
    check_tiling_and_balance(tree, (4, 4, 4), 2)
    roots = {tuple(t[1:]) for t in tree if t[0] == 0}
    for c in itertools.product((0, 1), repeat=3):
        assert c not in roots, "root block %s touching the level-2 leaves was not refined" % (c,)
    assert (2, 4, 4, 4) in {tuple(t) for t in tree}


def test_merge_refused_next_to_two_levels_finer():
    m, geo, cfg = make((8, 8, 8), (2, 2, 2), max_level=2, adaptive=0)
    U = np.zeros(m.state_shape())
    U[:, 0] = 1.0
    U[:, 4] = 1.5
    m.set_state(U)
    assert m.remesh(np.ones(m.nblocks, dtype=np.int8))           # all level 1
    tree = m.tree()
    flags = np.array([1 if tuple(t) == (1, 1, 1, 1) else 0 for t in tree], dtype=np.int8)
    assert m.remesh(flags)                                         # one corner at level 2
    tree = m.tree()
    # every level-1 leaf asks to merge; the siblings of root block (1,1,1)'s
    # neighbours... every root block touches (1,1,1)'s children, so no merge
    flags = np.array([-1 if t[0] == 1 else 0 for t in tree], dtype=np.int8)
    changed = m.remesh(flags, check_age=False)
    assert not changed
    check_tiling_and_balance(m.tree(), (2, 2, 2), 2)
    # without the level-2 leaves the level-1 leaves merge back
    flags = np.array([-1 if t[0] == 2 else 0 for t in m.tree()], dtype=np.int8)
    assert m.remesh(flags, check_age=False)
    flags = np.array([-1 if t[0] == 1 else 0 for t in m.tree()], dtype=np.int8)
    assert m.remesh(flags, check_age=False)
    assert m.nblocks == 8


def test_three_level_uniform_state_bit_exact():
    m, geo, cfg = make((8, 8, 8), (2, 2, 2), max_level=2, static_region=1,
                       static_lo=(0.05, 0.05, 0.05), static_hi=(0.1, 0.1, 0.1))
    U = np.zeros(m.state_shape())
    U[:, 0] = 1.3
    U[:, 1], U[:, 2], U[:, 3] = 0.2, -0.7, 0.05
    U[:, 4] = 2.5
    m.set_state(U)
    m.step(3)
    assert np.array_equal(m.get_state(), U)


def test_three_level_conservation_with_flux_correction():
    m, geo, cfg = make((8, 8, 8), (2, 2, 2), max_level=2, static_region=1,
                       static_lo=(0.05, -0.1, 0.05), static_hi=(0.1, 0.1, 0.1))
    leaves = m.tree()
    U = W.smooth_random_density(geo, leaves, seed=4)
    U[:, 1] = 0.3 * U[:, 0]
    U[:, 2] = -0.2 * U[:, 0]
    U[:, 4] += 0.5 * (0.09 + 0.04) * U[:, 0]
    m.set_state(U)
    t0 = m.totals()
    m.step(4)
    t1 = m.totals()
    assert np.all(np.abs(t1 - t0) <= 2e-14 * np.abs(t0).max()), t1 - t0


def test_linear_data_prolonged_exactly_through_two_levels():
    m, geo, cfg = make((8, 8, 8), (2, 2, 2), max_level=2)
    # level-0 leaves hold a linear field; evaluate the composite field at level 2
    leaves = m.tree()
    U = np.zeros(m.state_shape())
    a = np.array([0.3, -0.2, 0.1])
    for b, leaf in enumerate(leaves):
        _, _, (x, y, z) = W._block_cells(geo, leaf)
        for v in range(5):
            U[b, v] = 1.0 + (v + 1) * (a[0] * x + a[1] * y + a[2] * z)
    m.set_state(U)
    h = geo.dx(0, 2)
    # level 2 has 64 cells per axis; stay two level-0 cells away from the
    # periodic seam, where the linear field jumps
    for I, J, K in ((20, 30, 40), (33, 17, 45), (10, 50, 25), (9, 9, 54)):
        val = m.composite(2, I, J, K)
        x = -0.5 + (np.array([I, J, K]) + 0.5) * h
        expect = np.array([1.0 + (v + 1) * a.dot(x) for v in range(5)])
        assert np.allclose(val, expect, rtol=0, atol=1e-14), (I, J, K, val - expect)


def test_restriction_of_two_level_prolongation_is_identity():
    m, geo, cfg = make((8, 8, 8), (2, 2, 2), max_level=2)
    rng = np.random.default_rng(5)
    U = rng.uniform(0.5, 1.5, size=m.state_shape())
    m.set_state(U)
    # a level-0 cell equals the mean of its 64 level-2 descendants (restriction
    # undoes prolongation, exactly up to the order of the additions)
    for I, J, K in ((2, 3, 4), (9, 12, 15)):
        val0 = m.composite(0, I, J, K)
        acc = np.zeros(5)
        for c in itertools.product(range(4), repeat=3):
            acc += m.composite(2, 4 * I + c[0], 4 * J + c[1], 4 * K + c[2])
        assert np.allclose(acc / 64.0, val0, rtol=1e-14, atol=0)


def test_kelvin_helmholtz_refines_the_shear_layers():
    m, geo, cfg = make((8, 8, 8), (4, 4, 1), max_level=2, adaptive=1, gamma=1.4,
                       xmin=(-0.5, -0.5, -0.125), xmax=(0.5, 0.5, 0.125))
    m.set_state(W.kelvin_helmholtz(geo, m.tree(), seed=1))
    n0 = m.nblocks
    m.step(2)
    tree = m.tree()
    assert m.nblocks > n0 and tree[:, 0].max() == 2
    check_tiling_and_balance(tree, (4, 4, 1), 2)
    # finest leaves sit on the layers |x2| = 1/4
    h = 1.0 / (4 << 2)
    for lev, l1, l2, l3 in tree:
        if lev == 2:
            y0, y1 = -0.5 + l2 * h, -0.5 + (l2 + 1) * h
            assert min(abs(y0 - 0.25), abs(y1 - 0.25), abs(y0 + 0.25), abs(y1 + 0.25)) < 2 * h
    t0 = m.totals()
    m.step(2)
    assert np.all(np.abs(m.totals() - t0) <= 2e-14 * np.abs(t0).max())
