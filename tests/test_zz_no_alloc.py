"""ph_totals_noalloc: conserved totals for callers that may not allocate
device memory (their host application owns it all, or their loop must not
enter the CUDA allocator).  The entry point takes a caller-owned state and
output and keeps its scratch in a fixed device array, so it is compared here
with ph_totals, which uses scratch its mesh allocated: on two calls in a row
on uniform meshes, on a mesh with passive scalars (a wider block stride and
more totals) and on a three-level mesh (a cell volume per level).

This file is named to be collected last."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

# the tolerance the conservation tests use for totals
RTOL = 1e-13


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_12309_gb300 as ph
    return torch, ph


def _device_state(torch, m, precision):
    U = torch.empty(m.state_shape(), dtype=torch.float32 if precision == "fp32" else torch.float64,
                    device="cuda")
    m.get_state(U)
    return U


def _level_volumes(geo, nlevels):
    return [geo.dx(0, l) * geo.dx(1, l) * geo.dx(2, l) for l in range(nlevels)]


def _assert_close(got, ref):
    scale = np.abs(ref).max()
    assert got.shape == ref.shape
    assert np.all(np.abs(got - ref) <= RTOL * scale), (got, ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_totals_noalloc_matches_totals_two_calls(precision):
    torch, ph = _setup()
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    # call 1: 27 blocks of 8^3; call 2: 8 blocks of 16^3 (fewer blocks than
    # the first call left in the shared scratch array)
    cases = [((8, 8, 8), (3, 3, 3), 3, 1), ((16, 16, 16), (2, 2, 2), 2, 2)]
    for nx, nb, cycles, seed in cases:
        m = ph.Mesh(ph.make_config(nx, nb, precision=precision))
        geo = W.Geometry(nx, nb)
        dtype = np.float32 if precision == "fp32" else np.float64
        m.set_state(W.blast(geo, m.tree(), seed=seed).astype(dtype))
        m.step(cycles)
        ref = m.totals()
        U = _device_state(torch, m, precision)
        ph.totals_noalloc(U, nx, m.nblocks, out, precision=precision, vol=_level_volumes(geo, 1))
        torch.cuda.synchronize()
        _assert_close(out.cpu().numpy(), ref)
        m.close()


def test_totals_noalloc_passive_scalars():
    """7 variables per cell: every block after the first starts 7 fields on."""
    torch, ph = _setup()
    nx, nb = (8, 8, 8), (2, 2, 2)
    m = ph.Mesh(ph.make_config(nx, nb, nscalars=2))
    geo = W.Geometry(nx, nb)
    leaves = m.tree()
    U = W.blast(geo, leaves, seed=5, center=(0.15, -0.1, 0.05), radius=0.2, p_in=10.0)
    conc = [W.smooth_random_density(geo, leaves, seed=6 + s)[:, 0:1] - 0.6 for s in range(2)]
    U0 = np.concatenate([U] + [U[:, 0:1] * c for c in conc], axis=1)
    m.set_state(U0)
    m.step(2)
    ref = m.totals()
    assert ref.shape == (7,)
    U = _device_state(torch, m, "fp64")
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    ph.totals_noalloc(U, nx, m.nblocks, out, nvar=7, vol=_level_volumes(geo, 1))
    torch.cuda.synchronize()
    _assert_close(out.cpu().numpy(), ref)


def test_totals_noalloc_three_levels():
    """Leaves on levels 0, 1 and 2, each summed with its own cell volume."""
    torch, ph = _setup()
    nx, nb = (8, 8, 8), (4, 4, 4)
    kw = dict(max_level=2, static_region=1, static_lo=(-0.1, -0.1, -0.1), static_hi=(0.1, 0.1, 0.1))
    m = ph.Mesh(ph.make_config(nx, nb, **kw))
    tree = m.tree()
    assert set(tree[:, 0].tolist()) == {0, 1, 2}
    geo = W.Geometry(nx, nb)
    m.set_state(W.blast(geo, tree, seed=7))
    m.step(2)
    ref = m.totals()
    U = _device_state(torch, m, "fp64")
    level = torch.tensor(tree[:, 0].astype(np.int8), device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    ph.totals_noalloc(U, nx, m.nblocks, out, level=level, vol=_level_volumes(geo, 3))
    torch.cuda.synchronize()
    _assert_close(out.cpu().numpy(), ref)
    # a level with no volume given makes the totals NaN instead of using a
    # wrong volume
    ph.totals_noalloc(U, nx, m.nblocks, out, level=level, vol=_level_volumes(geo, 2))
    torch.cuda.synchronize()
    assert np.all(np.isnan(out.cpu().numpy()))


def test_totals_noalloc_rejects_bad_arguments():
    torch, ph = _setup()
    U = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(ph.PhError) as ei:
        ph.totals_noalloc(U, (1, 1, 1), ph_max_blocks() + 1, out)
    assert "PH_TOTALS_NOALLOC_MAX_BLOCKS" in str(ei.value)
    with pytest.raises(ph.PhError) as ei:
        ph.totals_noalloc(U, (1, 1, 1), 1, out, nvar=8)
    assert "nvar" in str(ei.value)
    with pytest.raises(ph.PhError) as ei:
        ph.totals_noalloc(U[:5], (1, 1, 1), 1, out, vol=(1.0, 0.125))
    assert "nlevels" in str(ei.value)


def ph_max_blocks():
    import os
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "ph_hydro.h")).read()
    for line in hdr.splitlines():
        if line.startswith("#define PH_TOTALS_NOALLOC_MAX_BLOCKS"):
            return int(line.split()[-1])
    raise AssertionError("limit not declared")
