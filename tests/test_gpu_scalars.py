"""GPU parity of passive scalars against the FP64 oracle: uniform and
two-level meshes, one and two scalars, FP64 (1e-12 per field per cycle) and
FP32 (stated bound), ghosts bit-exact, physical boundaries, a uniform
concentration staying uniform, conservation, and a restart; batched meshes
and the adjoint refuse meshes with scalars."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from parity import describe, field_errors

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _ph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_12309_gb300 as ph
    return ph


def pair(nx, nb, precision="fp64", **kw):
    ph = _ph()
    ocfg = O.make_config(nx, nb, **kw)
    om = O.OracleMesh(ocfg)
    gm = ph.Mesh(ph.make_config(nx, nb, precision=precision, **kw))
    geo = W.Geometry(tuple(nx), tuple(nb), tuple(ocfg.xmin), tuple(ocfg.xmax))
    assert np.array_equal(gm.tree(), om.tree())
    return om, gm, geo


def state(geo, leaves, ns, seed=3):
    U = W.blast(geo, leaves, seed=seed, center=(0.15, -0.1, 0.05), radius=0.2, p_in=10.0)
    conc = [W.smooth_random_density(geo, leaves, seed=seed + 10 + s)[:, 0:1] - 0.6 for s in range(ns)]
    return np.concatenate([U] + [U[:, 0:1] * c for c in conc], axis=1)


def scalar_errors(g, o):
    """max |a - b| / max |b| of every scalar field."""
    return np.array([np.abs(g[:, v] - o[:, v]).max() / np.abs(o[:, v]).max() for v in range(5, g.shape[1])])


@pytest.mark.parametrize("ns", [1, 2])
@pytest.mark.parametrize("kw", [dict(), dict(max_level=1, static_region=1),
                                dict(bc=("reflect", "outflow", "periodic", "periodic", "outflow", "reflect"))])
def test_scalars_match_oracle_fp64(ns, kw):
    om, gm, geo = pair((16, 16, 16), (2, 2, 2), nscalars=ns, **kw)
    U = state(geo, om.tree(), ns)
    om.set_state(U)
    gm.set_state(U)
    assert gm.state_shape()[1] == 5 + ns
    assert np.array_equal(gm.get_full(), om.get_full())
    for c in range(5):
        odt = om.step(1)[0]
        gm.step(1)
        G, R = gm.get_state(), om.get_state()
        err = field_errors(G[:, :5], R[:, :5])
        assert err.max() <= TOL64, "cycle %d: %s" % (c, describe(err))
        es = scalar_errors(G, R)
        assert es.max() <= TOL64, (c, es)
        assert abs(gm.dt() - odt) <= TOL64 * odt
    t = gm.totals()
    assert t.shape == (5 + ns,)


def test_scalars_fp32_against_fp64_oracle():
    om, gm, geo = pair((16, 16, 16), (2, 2, 2), precision="fp32", nscalars=2)
    U = state(geo, om.tree(), 2)
    om.set_state(U)
    gm.set_state(U.astype(np.float32))
    om.step(8)
    gm.step(8)
    G, R = gm.get_state(), om.get_state()
    err = field_errors(G[:, :5], R[:, :5])
    assert np.all(err <= np.array([2e-5, 1e-4, 1e-4, 1e-4, 2e-5])), describe(err)
    assert scalar_errors(G, R).max() <= 1e-4


def test_uniform_concentration_and_conservation_on_gpu():
    ph = _ph()
    nx, nb = (16, 16, 16), (2, 2, 2)
    cfg = ph.make_config(nx, nb, nscalars=1, max_level=1, static_region=1)
    m = ph.Mesh(cfg)
    geo = W.Geometry(nx, nb)
    U = W.blast(geo, m.tree(), seed=4, radius=0.2, p_in=10.0)
    m.set_state(np.concatenate([U, 0.3 * U[:, 0:1]], axis=1))
    t0 = m.totals()
    m.step(6)
    V = m.get_state()
    assert np.abs(V[:, 5] / V[:, 0] - 0.3).max() <= 1e-13
    t1 = m.totals()
    assert abs(t1[5] - t0[5]) <= 1e-14 * np.abs(t0).max()


def test_scalar_mesh_restart_and_refusals(tmp_path):
    ph = _ph()
    nx, nb = (16, 16, 16), (1, 1, 2)
    cfg = ph.make_config(nx, nb, nscalars=2)
    m = ph.Mesh(cfg)
    geo = W.Geometry(nx, nb)
    m.set_state(state(geo, m.tree(), 2))
    m.step(2)
    path = str(tmp_path / "s.phr")
    m.save(path)
    m.step(2)
    r = ph.Mesh.load(path)
    assert r.state_shape() == m.state_shape()
    r.step(2)
    assert np.array_equal(r.get_state(), m.get_state())
    with pytest.raises(ph.PhError, match="PH_ERR_INVALID"):
        ph.Batch([cfg])
    U = m.get_state()
    with pytest.raises(ph.PhError, match="PH_ERR_INVALID"):
        m.adjoint(U, U, 1, 1)
