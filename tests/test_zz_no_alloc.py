"""ph_totals_noalloc: conserved totals for callers that may not allocate
device memory (their host application owns it all, or their loop must not
enter the CUDA allocator).  The entry point takes a caller-owned state and
output and keeps its scratch in a fixed device array, so it is compared here
with ph_totals, which uses scratch its mesh allocated, on two calls in a row.

This file is named to be collected last."""
import ctypes

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


def _mesh_state(ph, torch, nx, nb, precision, cycles, seed):
    cfg = ph.make_config(nx, nb, precision=precision)
    m = ph.Mesh(cfg)
    geo = W.Geometry(nx, nb)
    dtype = np.float32 if precision == "fp32" else np.float64
    m.set_state(W.blast(geo, m.tree(), seed=seed).astype(dtype))
    m.step(cycles)
    ref = m.totals()
    U = torch.empty(m.state_shape(), dtype=torch.float32 if precision == "fp32" else torch.float64,
                    device="cuda")
    m.get_state(U)
    vol = geo.dx(0, 0) * geo.dx(1, 0) * geo.dx(2, 0)
    return m, U, ref, vol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_totals_noalloc_matches_totals_two_calls(precision):
    torch, ph = _setup()
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    # call 1: 27 blocks of 8^3; call 2: 8 blocks of 16^3 (fewer blocks than
    # the first call left in the shared scratch array)
    cases = [((8, 8, 8), (3, 3, 3), 3, 1), ((16, 16, 16), (2, 2, 2), 2, 2)]
    for nx, nb, cycles, seed in cases:
        m, U, ref, vol = _mesh_state(ph, torch, nx, nb, precision, cycles, seed)
        ph.totals_noalloc(U, nx, m.nblocks, out, precision=precision, vol=(vol, vol / 8))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = np.abs(ref).max()
        assert np.all(np.abs(got - ref) <= RTOL * scale), (got, ref)
        m.close()


def test_totals_noalloc_rejects_too_many_blocks():
    torch, ph = _setup()
    U = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(ph.PhError) as ei:
        ph.totals_noalloc(U, (1, 1, 1), ph_max_blocks() + 1, out)
    assert "PH_TOTALS_NOALLOC_MAX_BLOCKS" in str(ei.value)


def ph_max_blocks():
    import os
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "ph_hydro.h")).read()
    for line in hdr.splitlines():
        if line.startswith("#define PH_TOTALS_NOALLOC_MAX_BLOCKS"):
            return int(line.split()[-1])
    raise AssertionError("limit not declared")
