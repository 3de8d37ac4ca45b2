"""Restart files (Sec. 3.9): a run resumed from a restart file continues bit
for bit (state, dt, time, cycle, block tree); outputs of lower precision hold
each value rounded to nearest."""
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


def _same_run(a, b):
    assert np.array_equal(a.tree(), b.tree())
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.dt() == b.dt()
    ta, ca = a.time()
    tb, cb = b.time()
    assert ta == tb and ca == cb


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_uniform_restart_is_bitwise(tmp_path, precision):
    ph = _ph()
    nx, nb = (16, 16, 16), (2, 2, 2)
    cfg = ph.make_config(nx, nb, precision=precision)
    m = ph.Mesh(cfg)
    geo = W.Geometry(nx, nb)
    U = W.blast(geo, m.tree(), seed=11)
    m.set_state(U.astype(m.dtype))
    m.step(3)
    path = str(tmp_path / "r.phr")
    m.save(path)
    m.step(4)
    r = ph.Mesh.load(path)
    assert r.cfg.precision == cfg.precision and tuple(r.cfg.nx) == nx
    t, c = r.time()
    assert c == 3
    r.step(4)
    _same_run(m, r)


def test_two_level_adaptive_restart_is_bitwise(tmp_path):
    """A blast that keeps refining after the restart point."""
    ph = _ph()
    nx, nb = (8, 8, 8), (4, 4, 4)
    cfg = ph.make_config(nx, nb, max_level=1, static_region=0, adaptive=1, derefine_count=2)
    m = ph.Mesh(cfg)
    geo = W.Geometry(nx, nb, tuple(cfg.xmin), tuple(cfg.xmax))
    m.set_state(W.blast(geo, m.tree(), seed=5, radius=0.2))
    m.step(2)
    path = str(tmp_path / "amr.phr")
    m.save(path)
    trees = []
    for _ in range(6):
        m.step(1)
        trees.append(m.tree().copy())
    r = ph.Mesh.load(path)
    for c in range(6):
        r.step(1)
        assert np.array_equal(r.tree(), trees[c]), "tree differs %d cycles after the restart" % (c + 1)
    _same_run(m, r)
    assert len({t.shape[0] for t in trees}) > 1  # the tree changed after the restart


def test_restart_keeps_the_derefinement_cadence(tmp_path):
    """Leaves refined at cycle 0 merge back once they are derefine_count
    cycles old; a restart after one cycle must merge them on the same cycle
    (the per-leaf ages travel with the tree)."""
    ph = _ph()
    nx, nb = (8, 8, 8), (2, 2, 2)
    cfg = ph.make_config(nx, nb, max_level=1, static_region=0, adaptive=1, derefine_count=3)
    m = ph.Mesh(cfg)
    U = np.zeros(m.state_shape())
    U[:, 0] = 1.0
    U[:, 4] = 0.9   # uniform state at rest: every indicator is 0, every fine leaf flags -1
    m.set_state(U)
    flags = np.zeros(m.nblocks, dtype=np.int8)
    flags[[0, 5]] = 1
    assert m.refine_where(flags)
    assert m.nblocks == 8 - 2 + 16
    m.step(1)
    path = str(tmp_path / "age.phr")
    m.save(path)
    counts = []
    for _ in range(4):
        m.step(1)
        counts.append(m.nblocks)
    assert counts[0] == 22 and counts[-1] == 8   # merged once old enough
    r = ph.Mesh.load(path)
    for c in range(4):
        r.step(1)
        assert r.nblocks == counts[c], (c, r.nblocks, counts)
    _same_run(m, r)


def test_fp32_mesh_restart_through_fp64_file(tmp_path):
    ph = _ph()
    nx, nb = (16, 16, 16), (2, 2, 1)
    m = ph.Mesh(ph.make_config(nx, nb, precision="fp32"))
    geo = W.Geometry(nx, nb)
    m.set_state(W.blast(geo, m.tree(), seed=12).astype(np.float32))
    m.step(2)
    path = str(tmp_path / "w.phr")
    m.save(path, precision="fp64")  # widening is exact
    m.step(3)
    r = ph.Mesh.load(path)
    r.step(3)
    _same_run(m, r)


def test_fp32_output_of_fp64_mesh(tmp_path):
    ph = _ph()
    nx, nb = (16, 16, 16), (1, 2, 2)
    m = ph.Mesh(ph.make_config(nx, nb))
    geo = W.Geometry(nx, nb)
    m.set_state(W.blast(geo, m.tree(), seed=13))
    m.step(2)
    path = str(tmp_path / "o.phr")
    m.save(path, precision="fp32")
    full = str(tmp_path / "f.phr")
    m.save(full)
    assert os.path.getsize(full) - os.path.getsize(path) == 4 * m.count()
    o = ph.Mesh.load(path)  # an FP64 mesh holding the rounded values
    assert np.array_equal(o.get_state(), m.get_state().astype(np.float32).astype(np.float64))
    assert o.time() == m.time()


def test_load_rejects_bad_files(tmp_path):
    ph = _ph()
    m = ph.Mesh(ph.make_config((8, 8, 8), (1, 1, 1)))
    with pytest.raises(ph.PhError):
        m.save(str(tmp_path / "x.phr"))  # no state yet: PH_ERR_STATE
    m.set_state(np.ones(m.state_shape()) * np.array([1, 0, 0, 0, 1.5]).reshape(1, 5, 1, 1, 1))
    good = str(tmp_path / "g.phr")
    m.save(good)
    raw = open(good, "rb").read()
    bad = str(tmp_path / "t.phr")
    open(bad, "wb").write(raw[:-8])  # truncated state
    with pytest.raises(ph.PhError, match="PH_ERR_IO"):
        ph.Mesh.load(bad)
    with pytest.raises(ph.PhError, match="PH_ERR_IO"):
        m.save(str(tmp_path / "no_such_dir" / "x.phr"))
