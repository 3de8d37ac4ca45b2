"""Edge and degenerate cases of the GPU path: no-op and out-of-order calls,
wrong sizes, a non-finite state planted on the host, a vacuum region that
trips the floors, a maximum-size mesh, and the torch allocator hook."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _ph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_12309_gb300 as ph
    return torch, ph


def test_call_order_and_sizes():
    torch, ph = _ph()
    m = ph.Mesh(ph.make_config((8, 8, 8), (2, 2, 2)))
    with pytest.raises(ph.PhError) as e:
        m.step(1)                                   # no state yet
    assert e.value.code == -6
    # a buffer of the wrong size: the binding passes its real element count
    # and the ABI rejects it before touching it
    with pytest.raises(ph.PhError) as e:
        m.set_state(np.zeros((8, 5, 8, 8, 7)))
    assert e.value.code == -1
    with pytest.raises(ph.PhError) as e:
        m.get_state(np.zeros((8, 5, 8, 8, 7)))
    assert e.value.code == -1
    geo = W.Geometry((8, 8, 8), (2, 2, 2))
    U = W.blast(geo, m.tree(), seed=0)
    m.set_state(U)
    m.step(0)                                       # no-op
    assert m.time() == (0.0, 0)
    assert np.array_equal(m.get_state(), U)
    with pytest.raises(ph.PhError):
        m.step(-1)


def test_non_finite_state_is_reported():
    torch, ph = _ph()
    m = ph.Mesh(ph.make_config((8, 8, 8), (2, 2, 2)))
    geo = W.Geometry((8, 8, 8), (2, 2, 2))
    U = W.blast(geo, m.tree(), seed=0)
    U[3, 4, 2, 2, 2] = np.nan                      # planted on the host
    m.set_state(U)
    m.step(2)
    rc, floors, nonfinite = m.status()
    assert rc == -3 and nonfinite == 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_one_nan_cell_makes_the_first_dt_non_finite(precision):
    """A NaN density in one cell, in the middle of the cells one thread of
    the dt reduction visits (32^3 block: 1024-cell planes, 4 cells a thread),
    must survive the running max: the first dt is not finite and the status
    says so before any cycle."""
    torch, ph = _ph()
    m = ph.Mesh(ph.make_config((32, 32, 32), (1, 1, 1), precision=precision))
    geo = W.Geometry((32, 32, 32), (1, 1, 1))
    U = W.blast(geo, m.tree(), seed=0).astype(np.float32 if precision == "fp32" else np.float64)
    U[0, 0, 5, 0, 0] = np.nan   # plane 5, the first cell a thread visits there
    m.set_state(U)
    rc, floors, nonfinite = m.status()
    assert nonfinite == 1 and rc == -3
    assert not np.isfinite(m.dt())


@pytest.mark.parametrize("precision,nx,nb,kw", [
    ("fp64", (16, 16, 16), (2, 2, 2), {}),                      # cubic cells
    ("fp64", (24, 16, 8), (1, 2, 3), {}),                       # dx1 = dx3 != dx2
    ("fp32", (32, 32, 32), (2, 2, 2), {}),                      # 32x16 paired tiles
    ("fp32", (16, 16, 16), (2, 2, 2), {}),                      # 16x16 paired tiles
    ("fp64", (8, 8, 8), (2, 2, 2),                              # two levels: flux correction
     dict(max_level=1, static_region=1, static_lo=(-0.3, -0.3, -0.3), static_hi=(-0.1, -0.1, -0.1))),
])
def test_rate_kernel_gives_the_dt_the_stage_epilogue_folded(precision, nx, nb, kw):
    """The dt a cycle's stage 2 folds into its epilogue (and, on two levels,
    the flux correction for the cells it changes) is the dt the rate kernel
    computes from the same state, bit for bit."""
    torch, ph = _ph()
    cfg = ph.make_config(nx, nb, precision=precision, **kw)
    m = ph.Mesh(cfg)
    geo = W.Geometry(nx, nb)
    U = W.blast(geo, m.tree(), seed=3).astype(np.float32 if precision == "fp32" else np.float64)
    m.set_state(U)
    m.step(2)
    folded = m.next_dt()
    state = m.get_state()
    m2 = ph.Mesh(cfg)
    assert np.array_equal(m2.tree(), m.tree())
    m2.set_state(state)
    assert m2.dt() == folded and m2.next_dt() == folded
    assert m.status()[0] == 0 and m2.status()[0] == 0


def test_vacuum_region_hits_floors_and_is_counted():
    torch, ph = _ph()
    m = ph.Mesh(ph.make_config((8, 8, 8), (2, 2, 2)))
    geo = W.Geometry((8, 8, 8), (2, 2, 2))
    U = W.blast(geo, m.tree(), seed=0)
    U[0, 0, 3:5, 3:5, 3:5] = 1e-14                 # density below the 1e-12 floor
    m.set_state(U)
    m.step(1)
    rc, floors, nonfinite = m.status()
    assert rc == -3 and floors > 0 and nonfinite == 0
    assert np.all(np.isfinite(m.get_state()))


def test_maximum_size_mesh_conserves():
    """512^3 zones in 512 blocks of 64^3 (FP64, ~14 GB of state pools)."""
    torch, ph = _ph()
    nx, nb = (64, 64, 64), (8, 8, 8)
    m = ph.Mesh(ph.make_config(nx, nb))
    geo = W.Geometry(nx, nb)
    U = W.linear_wave(geo, m.tree(), seed=2, kvec=(1, 2, 3))
    m.set_state(U)
    t0 = m.totals()
    m.step(2)
    t1 = m.totals()
    assert np.all(np.abs(t1 - t0) <= 1e-13 * np.abs(t0).max())
    assert m.status()[0] == 0
    del U
    m.close()


def test_torch_allocator_hook():
    torch, ph = _ph()
    ph.use_torch_allocator()
    try:
        before = torch.cuda.memory_allocated()
        m = ph.Mesh(ph.make_config((16, 16, 16), (2, 2, 2)))
        assert torch.cuda.memory_allocated() > before + 2 * 8 * 5 * 20 ** 3 * 8
        geo = W.Geometry((16, 16, 16), (2, 2, 2))
        m.set_state(W.blast(geo, m.tree(), seed=1))
        m.step(2)
        assert m.status()[0] == 0
        m.close()
        assert torch.cuda.memory_allocated() <= before + 1024
    finally:
        ph.lib().ph_set_allocator(None, None, None)
