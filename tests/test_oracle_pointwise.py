"""Pins of the oracle's pointwise pieces (EOS, van Leer slope, HLLE flux,
minmod, Morton key) against closed forms, textbook identities and symmetries.
CPU only."""
import math
import os

import numpy as np
import pytest

import exact_riemann as ER
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def euler_flux(w, d, gamma):
    """Physical flux of the Euler equations along d for primitive w (textbook)."""
    rho, v, p = w[0], np.array(w[1:4]), w[4]
    E = p / (gamma - 1.0) + 0.5 * rho * float(v @ v)
    f = np.zeros(5)
    f[0] = rho * v[d]
    f[1:4] = rho * v[d] * v
    f[1 + d] += p
    f[4] = (E + p) * v[d]
    return f


def test_toro_table_pins_exact_solver():
    rows = np.loadtxt(os.path.join(HERE, "golden", "toro_star_states.txt"))
    for r in rows:
        ps, us = ER.star_state(tuple(r[0:3]), tuple(r[3:6]), 1.4)
        assert abs(ps - r[6]) <= 5e-5 * max(1.0, abs(r[6])) + 1e-5
        assert abs(us - r[7]) <= 5e-5 * max(1.0, abs(r[7])) + 1e-5


def test_cons_to_prim_closed_form():
    # gamma = 1.5 keeps every step exact in binary.
    w = O.cons_to_prim([2.0, 2.0, -4.0, 1.0, 10.0], 1.5)
    # v = (1, -2, 0.5); ke = 0.5 * 2 * (1 + 4 + 0.25) = 5.25; p = 0.5 * (10 - 5.25)
    assert list(w) == [2.0, 1.0, -2.0, 0.5, 2.375]


def test_cons_to_prim_floors():
    w = O.cons_to_prim([1e-20, 0.0, 0.0, 0.0, 1e-30], 5.0 / 3.0, dfloor=1e-12, pfloor=1e-10)
    assert w[0] == 1e-12 and w[4] == 1e-10


def test_vanleer_linear_and_extrema():
    assert O.vanleer(1.0, 2.0, 3.0) == 1.0          # linear data: exact slope
    assert O.vanleer(3.0, 2.0, 1.0) == -1.0
    assert O.vanleer(1.0, 3.0, 2.0) == 0.0          # local maximum
    assert O.vanleer(2.0, 1.0, 2.0) == 0.0          # local minimum
    assert O.vanleer(1.0, 1.0, 5.0) == 0.0          # one-sided flat
    assert O.vanleer(0.0, 1.0, 3.0) == 4.0 / 3.0    # harmonic mean 2*1*2/(1+2)


def test_vanleer_tvd_bounds():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a, b, c = rng.normal(size=3)
        d = O.vanleer(a, b, c)
        dl, dr = b - a, c - b
        if dl * dr <= 0:
            assert d == 0.0
        else:
            assert np.sign(d) == np.sign(dl)
            assert abs(d) <= 2.0 * min(abs(dl), abs(dr)) * (1 + 1e-15)
            # face values stay within the neighbouring cell averages
            assert min(b, c) - 1e-15 <= b + 0.5 * d <= max(b, c) + 1e-15


def test_minmod():
    assert O.minmod(1.0, 2.0) == 1.0
    assert O.minmod(-3.0, -1.5) == -1.5
    assert O.minmod(1.0, -1.0) == 0.0
    assert O.minmod(0.0, 4.0) == 0.0


def random_state(rng):
    return np.array([rng.uniform(0.1, 3.0), *rng.normal(size=3), rng.uniform(0.05, 5.0)])


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hlle_consistency(d):
    """F(W, W) is the physical flux (consistency of the Riemann solver)."""
    rng = np.random.default_rng(10 + d)
    for _ in range(200):
        w = random_state(rng)
        f = O.hlle(w, w, d, 5.0 / 3.0)
        fe = euler_flux(w, d, 5.0 / 3.0)
        assert np.allclose(f, fe, rtol=1e-14, atol=1e-14 * np.abs(fe).max())


def test_hlle_supersonic_upwind():
    """Both states supersonic to the right: b- = 0 and F = F_L."""
    g = 1.4
    wl = np.array([1.0, 5.0, 0.3, -0.2, 1.0])
    wr = np.array([0.5, 4.0, -0.1, 0.4, 0.7])
    f = O.hlle(wl, wr, 0, g)
    assert np.allclose(f, euler_flux(wl, 0, g), rtol=4e-16, atol=0)
    # and supersonic to the left: F = F_R
    wl2 = wl.copy(); wl2[1] = -5.0
    wr2 = wr.copy(); wr2[1] = -4.0
    f2 = O.hlle(wl2, wr2, 0, g)
    assert np.allclose(f2, euler_flux(wr2, 0, g), rtol=4e-16, atol=0)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hlle_mirror_antisymmetry(d):
    """Reflecting x_d -> -x_d swaps the states and flips v_d: the flux of the
    reflected problem is the reflected flux with its sign flipped, bit for bit."""
    rng = np.random.default_rng(20 + d)
    for _ in range(200):
        wl, wr = random_state(rng), random_state(rng)
        ml, mr = wr.copy(), wl.copy()
        ml[1 + d] = -ml[1 + d]
        mr[1 + d] = -mr[1 + d]
        f = O.hlle(wl, wr, d, 5.0 / 3.0)
        g = O.hlle(ml, mr, d, 5.0 / 3.0)
        expect = -f
        expect[1 + d] = f[1 + d]
        assert np.array_equal(g, expect)


def test_hlle_rotation():
    """The y-flux of a rotated state is the rotated x-flux."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        wl, wr = random_state(rng), random_state(rng)
        f = O.hlle(wl, wr, 0, 1.4)
        perm = [0, 2, 3, 1, 4]  # (v1,v2,v3) -> (v3?,...) cyclic: new v2 = old v1
        rl = np.empty(5); rr = np.empty(5)
        # rotated frame: new v2 = old v1, new v3 = old v2, new v1 = old v3
        for src, dst in ((0, 0), (1, 2), (2, 3), (3, 1), (4, 4)):
            rl[dst] = wl[src]; rr[dst] = wr[src]
        g = O.hlle(rl, rr, 1, 1.4)
        fr = np.empty(5)
        for src, dst in ((0, 0), (1, 2), (2, 3), (3, 1), (4, 4)):
            fr[dst] = f[src]
        assert np.allclose(g, fr, rtol=1e-14, atol=1e-14 * np.abs(f).max()), perm


def test_hlle_bounds_exact_riemann_speeds():
    """Einfeldt's bounds enclose the exact wave fan of the Sod problem: the
    HLLE flux lies between the fluxes it mixes and reduces to the exact
    Godunov flux when the exact fan is entirely supersonic."""
    g = 1.4
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    wl = np.array([left[0], left[1], 0, 0, left[2]])
    wr = np.array([right[0], right[1], 0, 0, right[2]])
    f = O.hlle(wl, wr, 0, g)
    # mass flux is positive (flow to the right) and bounded by the star mass flux
    rho, u, p = ER.sample(left, right, g, np.array([0.0]))
    f_godunov = rho[0] * u[0]
    assert 0.0 < f[0] < 2.0 * f_godunov


def test_morton_order_small():
    # level-0 2x2x2 root grid: Z-order is x fastest, then y, then z
    keys = [O.morton(0, i, j, k, 0) for k in range(2) for j in range(2) for i in range(2)]
    assert keys == list(range(8))
    # level 1 inside a max_level=1 tree: (1,1,0,0) sits between (1,0,0,0) and (1,0,1,0)
    assert O.morton(1, 1, 0, 0, 1) == 1 and O.morton(1, 0, 1, 0, 1) == 2
    assert O.morton(0, 1, 0, 0, 1) == 8  # parent-level block scaled by 2
