"""Pins of the oracle's physical boundaries (outflow and reflecting; the
paper's reflective boundaries mirror the normal vector component, Sec. 3.4),
each against something other than the oracle's own boundary code: a
reflecting wall against the mirrored problem on a doubled periodic domain
(bit-exact), ghost values against images computed by brute force, a uniform
flow through outflow faces, the Sod shock tube with outflow ends against the
exact Riemann solution, and conservation of mass and energy in a closed box.
CPU only."""
import math

import numpy as np

import exact_riemann as ER
import oracle as O
import workloads as W
from test_oracle_mesh import to_global


def from_global(G, leaves, nx):
    U = np.zeros((len(leaves), 5, nx[2], nx[1], nx[0]))
    for b, (lev, l1, l2, l3) in enumerate(leaves):
        U[b] = G[:, l3 * nx[2]:(l3 + 1) * nx[2], l2 * nx[1]:(l2 + 1) * nx[1], l1 * nx[0]:(l1 + 1) * nx[0]]
    return U


def make(nx, nb, **kw):
    cfg = O.make_config(nx, nb, **kw)
    m = O.OracleMesh(cfg)
    geo = W.Geometry(tuple(nx), tuple(nb), tuple(cfg.xmin), tuple(cfg.xmax))
    return m, geo


def test_reflecting_wall_equals_mirrored_doubled_domain_bit_exact():
    """A box with reflecting walls on both faces of axis d evolves exactly as
    the left half of a periodic domain twice as long holding the state and its
    mirror image (normal momentum negated)."""
    nx, nb = (8, 8, 8), (2, 2, 2)
    for d in range(3):
        bc = ["periodic"] * 6
        bc[2 * d] = bc[2 * d + 1] = "reflect"
        half, geo = make(nx, nb, bc=bc)
        leaves = half.tree()
        U = W.blast(geo, leaves, seed=7, center=(0.13, -0.21, 0.07), radius=0.2, p_in=10.0)
        half.set_state(U)
        nb2 = list(nb)
        nb2[d] *= 2
        xmax2 = [0.5, 0.5, 0.5]
        xmax2[d] = 1.5
        dbl, _ = make(nx, tuple(nb2), xmax=tuple(xmax2))
        G = to_global(U, leaves, nx, nb)
        ax = 3 - d
        M = np.flip(G, axis=ax).copy()
        M[1 + d] = -M[1 + d]
        G2 = np.concatenate([G, M], axis=ax)
        dbl.set_state(from_global(G2, dbl.tree(), nx))
        assert half.compute_dt() == dbl.compute_dt()
        half.step(4)
        dbl.step(4)
        Gh = to_global(half.get_state(), leaves, nx, nb)
        Gd = to_global(dbl.get_state(), dbl.tree(), nx, tuple(nb2))
        n = nx[d] * nb[d]
        sl = [slice(None)] * 4
        sl[ax] = slice(0, n)
        assert np.array_equal(Gh, Gd[tuple(sl)]), "axis x%d" % (d + 1)
        assert half.time() == dbl.time()


def test_ghost_values_are_the_boundary_images():
    """Every ghost cell against its image computed by brute force: periodic
    shift, outflow clamp to the first interior layer, or mirror with the normal
    momentum negated, applied axis by axis."""
    nx, nb = (6, 4, 8), (2, 3, 1)
    bc = ["outflow", "reflect", "periodic", "periodic", "reflect", "outflow"]
    m, geo = make(nx, nb, bc=bc)
    rng = np.random.default_rng(3)
    U = rng.uniform(0.5, 2.0, size=m.state_shape())
    m.set_state(U)
    full = m.get_full()
    leaves = m.tree()
    G = to_global(U, leaves, nx, nb)
    N = [nx[d] * nb[d] for d in range(3)]

    def image(g, d):
        n = N[d]
        if 0 <= g < n:
            return g, False
        side = 0 if g < 0 else 1
        kind = bc[2 * d + side]
        if kind == "periodic":
            return g % n, False
        if kind == "outflow":
            return (0 if side == 0 else n - 1), False
        return (-1 - g if side == 0 else 2 * n - 1 - g), True

    for b, (_, l1, l2, l3) in enumerate(leaves):
        lo = (l1 * nx[0], l2 * nx[1], l3 * nx[2])
        for k in range(nx[2] + 4):
            for j in range(nx[1] + 4):
                for i in range(nx[0] + 4):
                    g = (lo[0] + i - 2, lo[1] + j - 2, lo[2] + k - 2)
                    im = [image(g[d], d) for d in range(3)]
                    val = G[:, im[2][0], im[1][0], im[0][0]].copy()
                    for d in range(3):
                        if im[d][1]:
                            val[1 + d] = -val[1 + d]
                    assert np.array_equal(full[b][:, k, j, i], val), (b, i, j, k)


def test_uniform_flow_through_outflow_faces_is_preserved():
    m, geo = make((8, 8, 8), (2, 2, 2), bc=["outflow"] * 6)
    U = np.zeros(m.state_shape())
    U[:, 0] = 1.3
    U[:, 1], U[:, 2], U[:, 3] = 0.4, -0.9, 0.15
    U[:, 4] = 2.5
    m.set_state(U)
    m.step(3)
    assert np.array_equal(m.get_state(), U)


def sod_run(N, t_end=0.1):
    nx, nb = (16, 4, 4), (N // 16, 1, 1)
    h = 1.0 / N
    m, geo = make(nx, nb, xmin=(-0.5, 0.0, 0.0), xmax=(0.5, 4 * h, 4 * h), gamma=1.4,
                  bc=["outflow", "outflow", "periodic", "periodic", "periodic", "periodic"])
    leaves = m.tree()
    m.set_state(W.sod(geo, leaves, gamma=1.4, x_if=0.0))
    dt_cfl = m.compute_dt()
    n = int(math.ceil(t_end / (0.5 * dt_cfl)))
    m.step_dt(np.full(n, t_end / n))
    G = to_global(m.get_state(), leaves, nx, nb)
    x = -0.5 + (np.arange(N) + 0.5) * h
    re_, ue, pe = ER.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, x / t_end)
    return x, G[0, 1, 1, :], re_


def test_sod_with_outflow_ends_against_exact_solution():
    """One interface in a closed-off tube with zero-gradient ends: before the
    waves reach the ends the solution is the textbook one."""
    errs = []
    for N in (64, 128, 256):
        x, rho, rex = sod_run(N)
        errs.append(np.mean(np.abs(rho - rex)))
        # the ends stay at the initial states (no wave has reached them)
        assert abs(rho[0] - 1.0) < 1e-12 and abs(rho[-1] - 0.125) < 1e-12
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(r >= 0.7 for r in rates), (errs, rates)
    assert errs[-1] < 6e-3


def test_closed_box_conserves_mass_and_energy():
    """Reflecting walls on every face: no mass or energy crosses a wall (the
    HLLE mass and energy fluxes of mirror states vanish); momentum is not
    conserved (the walls push back)."""
    m, geo = make((8, 8, 8), (2, 2, 2), bc=["reflect"] * 6)
    U = W.blast(geo, m.tree(), seed=2, center=(0.2, 0.1, -0.15), radius=0.2, p_in=10.0)
    m.set_state(U)
    t0 = m.totals()
    m.step(12)
    t1 = m.totals()
    for v in (0, 4):
        assert abs(t1[v] - t0[v]) <= 1e-13 * abs(t0[v]), (v, t0[v], t1[v])
    assert np.abs(t1[1:4] - t0[1:4]).max() > 1e-6
    assert m.floor_hits() == 0


def test_two_level_reflecting_wall_matches_mirrored_domain():
    """Two levels: static refinement touching the wall; the mirrored doubled
    domain refines the mirror image.  Equal up to the order of the 8-term
    restriction sums, which mirroring reverses."""
    nx, nb = (8, 8, 8), (2, 2, 2)
    bc = ["reflect", "reflect"] + ["periodic"] * 4
    half, geo = make(nx, nb, bc=bc, max_level=1, static_region=1,
                     static_lo=(0.3, -0.2, -0.2), static_hi=(0.7, 0.2, 0.2))
    dbl, geo2 = make(nx, (4, 2, 2), xmax=(1.5, 0.5, 0.5), max_level=1, static_region=1,
                     static_lo=(0.3, -0.2, -0.2), static_hi=(0.7, 0.2, 0.2))
    assert half.nblocks > 8 and dbl.nblocks == 2 * half.nblocks

    def field(geo_, leaves):
        U = np.zeros((len(leaves), 5) + tuple(reversed(nx)))
        # reflect the doubled field about x1 = 1/2 cell by cell
        for b, (lev, l1, l2, l3) in enumerate(leaves):
            _, _, (x, y, z) = W._block_cells(geo_, (lev, l1, l2, l3))
            xm = np.where(x > 0.5, 1.0 - x, x)
            s = np.where(x > 0.5, -1.0, 1.0)
            U[b, 0] = 1.0 + 0.2 * np.cos(2 * np.pi * xm) * np.cos(2 * np.pi * y) + 0.1 * np.sin(2 * np.pi * z)
            U[b, 1] = s * 0.3 * np.sin(2 * np.pi * xm) * U[b, 0]
            U[b, 2] = 0.1 * U[b, 0]
            U[b, 3] = 0.0
            U[b, 4] = 0.9 + 0.5 * (U[b, 1] ** 2 + U[b, 2] ** 2) / U[b, 0]
        return U

    half.set_state(field(geo, half.tree()))
    dbl.set_state(field(geo2, dbl.tree()))
    half.step(3)
    dbl.step(3)
    th, td = half.tree(), dbl.tree()
    Uh, Ud = half.get_state(), dbl.get_state()
    index = {tuple(t): b for b, t in enumerate(td)}
    scale = np.abs(Ud).max(axis=(0, 2, 3, 4))
    for b, t in enumerate(th):
        db = index[tuple(t)]
        err = np.abs(Uh[b] - Ud[db]).max(axis=(1, 2, 3)) / scale
        assert err.max() <= 1e-13, (t, err)
