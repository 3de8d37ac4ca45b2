"""Pins of the oracle's complex-step derivatives (the FP64 reference for the
adjoint): closed forms on a uniform state and central finite differences of
the real oracle under the same frozen dt schedule.  CPU only."""
import numpy as np

import oracle as O
import workloads as W


def small():
    cfg = O.make_config((8, 8, 8), (2, 2, 1))
    m = O.OracleMesh(cfg)
    geo = W.Geometry((8, 8, 8), (2, 2, 1))
    return cfg, m, geo


def test_uniform_state_tangent_closed_form():
    cfg, m, geo = small()
    U0 = np.zeros(m.state_shape())
    U0[:, 0], U0[:, 1], U0[:, 4] = 1.2, 0.3, 2.0
    V = np.zeros_like(U0)
    V[:, 0], V[:, 2], V[:, 4] = 0.5, -0.25, 1.0   # a uniform perturbation stays uniform
    dts = np.full(3, 2e-3)
    Uf, JV = O.jvp_state(cfg, U0, V, 0.0, dts)
    assert np.array_equal(Uf, U0)
    assert np.allclose(JV, V, rtol=0, atol=1e-14)
    # gamma does not move a uniform state
    _, JG = O.jvp_state(cfg, U0, np.zeros_like(U0), 1.0, dts)
    assert np.abs(JG).max() <= 1e-14


def generic_state(geo, leaves):
    """Every primitive field varies smoothly, so no slope sits on the limiter's
    kink (dL dR = 0), where finite differences see one-sided derivatives."""
    rho = W.smooth_random_density(geo, leaves, seed=3)[:, 0]
    f = [W.smooth_random_density(geo, leaves, seed=s)[:, 0] - 1.0 for s in (5, 6, 7, 8)]
    v = [0.2 + f[0], f[1], f[2]]
    p = 0.6 * (1.0 + f[3])
    U = np.zeros((len(leaves), 5) + rho.shape[1:])
    U[:, 0] = rho
    for d in range(3):
        U[:, 1 + d] = rho * v[d]
    U[:, 4] = p / (2.0 / 3.0) + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    return U


def test_tangent_matches_central_differences():
    cfg, m, geo = small()
    U0 = generic_state(geo, m.tree())
    rng = np.random.default_rng(1)
    V = rng.normal(size=U0.shape) * 1e-2
    m.set_state(U0)
    dts = m.step(3)
    Uf, JV = O.jvp_state(cfg, U0, V, 0.3, dts)
    # eps x V = 1e-8 absolute: larger steps flip limiter branches in cells
    # whose one-sided differences are ~1e-6, smaller ones drown in round-off;
    # per-cell FD is good to ~2e-6 of max |J V| here, the scalar loss to 1e-8.
    eps = 1e-6

    def run(U, g):
        c = O.make_config((8, 8, 8), (2, 2, 1), gamma=g)
        mm = O.OracleMesh(c)
        mm.set_state(U)
        mm.step_dt(dts)
        return mm.get_state()

    fd = (run(U0 + eps * V, cfg.gamma + eps * 0.3) - run(U0 - eps * V, cfg.gamma - eps * 0.3)) / (2 * eps)
    assert np.abs(fd - JV).max() <= 1e-5 * np.abs(JV).max()
    target = U0[:, 0] * 0.9
    J, dJ = O.jvp(cfg, U0, V, 0.3, target, dts)
    assert np.isclose(dJ, np.sum(2 * (Uf[:, 0] - target) * JV[:, 0]), rtol=1e-12)
    Jp = np.sum((run(U0 + eps * V, cfg.gamma + eps * 0.3)[:, 0] - target) ** 2)
    Jm = np.sum((run(U0 - eps * V, cfg.gamma - eps * 0.3)[:, 0] - target) ** 2)
    assert abs((Jp - Jm) / (2 * eps) - dJ) <= 1e-6 * abs(dJ)
