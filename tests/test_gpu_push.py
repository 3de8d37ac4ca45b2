"""Ghost exchange inside the stage kernels (push form, periodic uniform meshes):
every stage writes the new interior values into the ghost zones of its output
that they fill.  It must leave exactly the state, ghost zones included, that
the separate pull-exchange launch leaves (PH_GHOSTS=launch at creation), for
every stage kernel (FP64 and FP32 one-cell, FP32 paired), ragged tiles,
blocks that are their own periodic neighbour, and passive scalars."""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _ph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_12309_gb300 as ph
    return ph


def _mesh(ph, cfg, launch):
    if launch:
        os.environ["PH_GHOSTS"] = "launch"
    try:
        return ph.Mesh(cfg)
    finally:
        os.environ.pop("PH_GHOSTS", None)


CASES = [
    # nx, nb, precision, tile (None: default), nscalars
    ((16, 16, 16), (2, 2, 2), "fp64", None, 0),
    ((32, 32, 32), (2, 1, 2), "fp32", None, 0),          # paired kernel
    ((32, 32, 32), (2, 2, 1), "fp32", (16, 16, 16), 0),  # one-cell FP32 kernel
    ((24, 16, 8), (1, 2, 3), "fp64", (16, 8, 8), 0),     # ragged x1 tiles, non-cubic
    ((16, 16, 16), (1, 1, 1), "fp64", None, 0),          # its own neighbour on every side
    ((32, 16, 16), (1, 1, 1), "fp32", None, 0),          # paired kernel, own neighbour
    ((4, 4, 4), (3, 3, 3), "fp64", (8, 8, 4), 0),        # smallest block
    ((16, 16, 16), (2, 1, 2), "fp64", None, 2),          # passive scalars
    ((16, 16, 16), (2, 2, 1), "fp32", None, 1),
]


@pytest.mark.parametrize("nx,nb,prec,tile,ns", CASES)
def test_push_exchange_matches_the_exchange_launch(nx, nb, prec, tile, ns):
    ph = _ph()
    cfg = ph.make_config(nx, nb, precision=prec, tile=tile or (0, 0, 0), nscalars=ns)
    pull = _mesh(ph, cfg, launch=True)
    push = _mesh(ph, cfg, launch=False)
    assert pull.launches_per_cycle() == 5 and push.launches_per_cycle() == 3
    assert pull.tile() == push.tile()
    geo = W.Geometry(nx, nb)
    U = W.blast(geo, pull.tree(), seed=5, center=(0.3, -0.25, 0.4), radius=0.3)
    if ns:
        rng = np.random.default_rng(11)
        r = rng.uniform(0.1, 1.0, size=(U.shape[0], ns) + U.shape[2:])
        U = np.concatenate([U, U[:, :1] * r], axis=1)
    dt = np.float32 if prec == "fp32" else np.float64
    pull.set_state(U.astype(dt))
    push.set_state(U.astype(dt))
    for c in range(3):
        pull.step(1)
        push.step(1)
        a, b = pull.get_full(), push.get_full()
        assert np.array_equal(a, b), "cycle %d: %d cells differ" % (c, int((a != b).sum()))
        assert pull.dt() == push.dt()
    assert pull.status() == push.status() == (0, 0, 0)


def test_physical_boundaries_keep_the_exchange_launch():
    ph = _ph()
    cfg = ph.make_config((16, 16, 16), (2, 1, 1), bc=("outflow",) * 2 + ("periodic",) * 4)
    assert ph.Mesh(cfg).launches_per_cycle() == 5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_push_exchange_matches_its_ghost_phases(precision):
    """The persistent batch kernel without its two ghost phases (the stages
    push) against the same batch with them."""
    ph = _ph()
    members = [((16,) * 3, (2,) * 3, (0.1, -0.05, 0.0)), ((32,) * 3, (2, 1, 2), (-0.2, 0.1, 0.15)),
               ((16,) * 3, (1, 1, 1), (0.2, 0.2, -0.1))]
    cfgs = [ph.make_config(nx, nb, precision=precision) for nx, nb, _ in members]
    dtype = np.float32 if precision == "fp32" else np.float64

    def batch(launch):
        if launch:
            os.environ["PH_GHOSTS"] = "launch"
        try:
            B = ph.Batch(cfgs)
        finally:
            os.environ.pop("PH_GHOSTS", None)
        for s, (nx, nb, c) in enumerate(members):
            geo = W.Geometry(nx, nb)
            U = W.blast(geo, ph.Mesh(cfgs[s]).tree(), seed=s, center=c)
            B.set_state(s, U.astype(dtype))
        return B

    pull, push = batch(True), batch(False)
    pull.step(3)
    push.step(3)
    assert np.array_equal(pull.dt(), push.dt())
    for s in range(len(members)):
        assert np.array_equal(pull.get_state(s), push.get_state(s)), s
