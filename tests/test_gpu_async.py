"""Stream-ordered state copies (ph_set_state_async / ph_get_state_async):
the same results as the synchronous calls, also with two meshes on two
streams whose transfers and cycles interleave."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _ph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_12309_gb300 as ph
    return ph, torch


def test_async_copies_match_sync_on_two_streams():
    ph, torch = _ph()
    nx, nb = (16, 16, 16), (2, 2, 2)
    cfg = ph.make_config(nx, nb)
    geo = W.Geometry(nx, nb)
    ref = ph.Mesh(cfg)
    states = [W.blast(geo, ref.tree(), seed=s) for s in (1, 2, 3, 4)]
    expect = []
    for U in states:
        ref.set_state(U)
        ref.step(2)
        expect.append((ref.get_state(), ref.dt()))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    meshes = [ph.Mesh(cfg, stream=st.cuda_stream) for st in streams]
    host_in = [torch.from_numpy(U).pin_memory() for U in states]
    host_out = [torch.zeros_like(h).pin_memory() for h in host_in]
    for k in range(4):
        m = meshes[k % 2]
        m.set_state(host_in[k].numpy(), sync=False)
        m.step(2)
        m.get_state(host_out[k].numpy(), sync=False)
    for st in streams:
        st.synchronize()
    for k in range(4):
        assert np.array_equal(host_out[k].numpy(), expect[k][0]), k
    # the last state of each mesh reports the same dt as the synchronous run
    assert meshes[0].dt() == expect[2][1] and meshes[1].dt() == expect[3][1]


def test_async_get_needs_a_state():
    ph, torch = _ph()
    m = ph.Mesh(ph.make_config((8, 8, 8), (1, 1, 1)))
    out = np.zeros(m.state_shape())
    with pytest.raises(ph.PhError, match="PH_ERR_STATE"):
        m.get_state(out, sync=False)
