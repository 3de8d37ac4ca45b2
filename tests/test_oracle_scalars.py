"""Pins of the oracle's passive scalars (Sec. 3.4: the hydro package advects
every variable flagged as advected): a scalar is one more conserved
variable rho r whose flux is the HLLE formula with the hydro wave speeds.
Pinned by a uniform concentration staying uniform (uniform and two-level
meshes, through prolongation and restriction), a zero scalar staying exactly
zero, conservation, a reflecting wall leaving scalars unflipped, and linear
advection of a smooth profile converging to the shifted exact solution.
CPU only."""
import math

import numpy as np

import oracle as O
import workloads as W
from test_oracle_mesh import to_global


def make(nx, nb, **kw):
    cfg = O.make_config(nx, nb, **kw)
    m = O.OracleMesh(cfg)
    geo = W.Geometry(tuple(nx), tuple(nb), tuple(cfg.xmin), tuple(cfg.xmax))
    return m, geo


def with_scalars(U, conc):
    """Append scalars rho * r_s (r_s arrays broadcastable to the density)."""
    rho = U[:, 0:1]
    return np.concatenate([U] + [rho * c for c in conc], axis=1)


def test_uniform_concentration_stays_uniform():
    for kw in (dict(), dict(max_level=1, static_region=1)):
        m, geo = make((8, 8, 8), (2, 2, 2), nscalars=2, **kw)
        U = W.blast(geo, m.tree(), seed=4, radius=0.2, p_in=10.0)
        m.set_state(with_scalars(U, [np.full_like(U[:, 0:1], 0.3), np.zeros_like(U[:, 0:1])]))
        m.step(5)
        V = m.get_state()
        r = V[:, 5] / V[:, 0]
        assert np.abs(r - 0.3).max() <= 1e-13, np.abs(r - 0.3).max()
        assert np.all(V[:, 6] == 0.0)           # a zero scalar stays exactly zero


def test_scalars_are_conserved():
    m, geo = make((8, 8, 8), (2, 2, 2), nscalars=1, max_level=1, static_region=1)
    leaves = m.tree()
    U = W.blast(geo, leaves, seed=5, radius=0.2, p_in=10.0)
    conc = W.smooth_random_density(geo, leaves, seed=7)[:, 0:1] - 0.5
    m.set_state(with_scalars(U, [conc]))
    t0 = m.totals()
    assert t0.shape == (6,)
    m.step(5)
    t1 = m.totals()
    assert abs(t1[5] - t0[5]) <= 1e-14 * np.abs(t0).max()


def test_reflecting_wall_leaves_scalars_unflipped():
    nx, nb = (6, 4, 4), (2, 2, 1)
    m, geo = make(nx, nb, nscalars=1, bc=["reflect"] * 6)
    rng = np.random.default_rng(3)
    U = rng.uniform(0.5, 2.0, size=m.state_shape())
    m.set_state(U)
    full = m.get_full()
    leaves = m.tree()
    G = to_global(U[:, :5], leaves, nx, nb)
    S = to_global(U[:, 5:6].repeat(5, axis=1), leaves, nx, nb)[0]
    # the ghost at x1 = -1 of the first block mirrors interior x1 = 0
    b0 = [b for b, t in enumerate(leaves) if tuple(t) == (0, 0, 0, 0)][0]
    assert np.array_equal(full[b0][5, 2:-2, 2:-2, 1], S[0:4, 0:4, 0])
    assert np.array_equal(full[b0][1, 2:-2, 2:-2, 1], -G[1, 0:4, 0:4, 0])


def advect(N, t_end=1.0):
    """A smooth concentration carried by a uniform flow along x1 through a
    periodic thin box: after one crossing it returns to its start."""
    nx, nb = (16, 4, 4), (N // 16, 1, 1)
    h = 1.0 / N
    m, geo = make(nx, nb, xmin=(-0.5, 0.0, 0.0), xmax=(0.5, 4 * h, 4 * h), nscalars=1)
    leaves = m.tree()
    U = np.zeros(m.state_shape())
    U[:, 0] = 1.0
    U[:, 1] = 1.0
    U[:, 4] = 0.6 / (2.0 / 3.0) + 0.5
    for b, leaf in enumerate(leaves):
        _, _, (x, _, _) = W._block_cells(geo, leaf)
        U[b, 5] = 0.5 + 0.4 * np.sin(2 * np.pi * x)
    r0 = to_global(np.repeat(U[:, 5:6], 5, axis=1), leaves, nx, nb)[0, 1, 1, :].copy()
    m.set_state(U)
    n = int(math.ceil(t_end / (0.3 * h / 2.0)))
    m.step_dt(np.full(n, t_end / n))
    V = m.get_state()
    hydro = to_global(V[:, :5], leaves, nx, nb)
    r = to_global(np.repeat(V[:, 5:6] / V[:, 0:1], 5, axis=1), leaves, nx, nb)[0, 1, 1, :]
    return np.mean(np.abs(r - r0)), hydro


def test_advected_scalar_converges_to_the_shifted_profile():
    errs = []
    for N in (32, 64, 128):
        e, hydro = advect(N)
        errs.append(e)
        assert np.all(hydro[0] == 1.0) and np.all(hydro[1] == 1.0)   # the flow stays uniform
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(r >= 1.6 for r in rates), (errs, rates)
    assert errs[-1] < 2e-3
