"""Device-allocation failure, injected on the host: an allocator installed
through ph_set_allocator that passes requests to PyTorch's caching allocator
and refuses its k-th one.

* ph_create with the k-th request refused, for every k a creation makes:
  PH_ERR_OOM, and every byte the failed creation took is given back;
* an explicit refinement whose remesh cannot get its memory (each of the
  requests a remesh makes refused in turn): PH_ERR_OOM, the mesh keeps its
  old tree and state and keeps stepping, bit for bit as a mesh that never
  tried; the same refinement then succeeds once memory is available;
* a mesh made with the ordinary allocator, and the GPU context, stay usable
  throughout.
No GPU fault is involved: the failure is a NULL returned on the host."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_12309_gb300 as ph
    return torch, ph


class FailingAllocator:
    """Counts requests; refuses request number `fail_at` (0: none)."""

    def __init__(self, torch):
        self.calls = 0
        self.fail_at = 0
        self.live = {}

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                       int(stream or 0)))
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, stream, ctx):
            self.live.pop(int(ptr))
            torch.cuda.caching_allocator_delete(int(ptr))

        self._a, self._f = ALLOC(_alloc), FREE(_free)

    def install(self, ph):
        ph.check(ph.lib().ph_set_allocator(ctypes.cast(self._a, ctypes.c_void_p),
                                           ctypes.cast(self._f, ctypes.c_void_p), None))

    def arm(self, k):
        """Refuse the k-th request from now on (k >= 1)."""
        self.fail_at = self.calls + k


def _restore_default(ph):
    ph.check(ph.lib().ph_set_allocator(None, None, None))


CONFIGS = [dict(nx=(16, 16, 16), nb=(2, 2, 2)),
           dict(nx=(8, 8, 8), nb=(4, 4, 4), max_level=1, static_region=1)]


@pytest.mark.parametrize("kw", CONFIGS)
def test_create_fails_cleanly_at_every_allocation(kw):
    torch, ph = _setup()
    kw = dict(kw)
    nx, nb = kw.pop("nx"), kw.pop("nb")
    cfg = ph.make_config(nx, nb, **kw)
    geo = W.Geometry(nx, nb)
    bystander = ph.Mesh(ph.make_config(nx, nb, **kw))   # ordinary allocator
    U = W.blast(geo, bystander.tree(), seed=3)
    bystander.set_state(U)
    bystander.step(1)
    fa = FailingAllocator(torch)
    fa.install(ph)
    try:
        m = ph.Mesh(cfg)      # count the requests of a successful creation
        n_req = fa.calls
        m.close()
        assert n_req >= 3 and not fa.live
        for k in range(1, n_req + 1):
            fa.arm(k)
            with pytest.raises(ph.PhError) as ei:
                ph.Mesh(cfg)
            assert ei.value.code == -2, str(ei.value)      # PH_ERR_OOM
            assert "allocation" in str(ei.value)
            assert not fa.live, "a failed creation kept %d allocations" % len(fa.live)
        fa.fail_at = 0
        m = ph.Mesh(cfg)       # memory available again
        m.set_state(U)
        m.step(1)
        bystander.step(1)
        ref = ph.Mesh(ph.make_config(nx, nb, **kw))
        ref.set_state(U)
        ref.step(2)
        assert np.array_equal(bystander.get_state(), ref.get_state())
        m.step(1)
        assert np.array_equal(m.get_state(), ref.get_state())
        m.close()
        ref.close()
    finally:
        _restore_default(ph)
    bystander.close()


def test_remesh_failure_keeps_the_old_tree():
    torch, ph = _setup()
    nx, nb = (8, 8, 8), (4, 4, 4)
    kw = dict(max_level=1, static_region=1)
    geo = W.Geometry(nx, nb)
    fa = FailingAllocator(torch)
    fa.install(ph)
    try:
        m = ph.Mesh(ph.make_config(nx, nb, **kw))
        ref = ph.Mesh(ph.make_config(nx, nb, **kw))
        tree0 = m.tree()
        U = W.blast(geo, tree0, seed=4, radius=0.15)
        m.set_state(U)
        ref.set_state(U)
        flags = np.zeros(m.nblocks, dtype=np.int8)
        flags[np.where(tree0[:, 0] == 0)[0][:3]] = 1
        # count the requests of a successful remesh on a scratch mesh
        probe = ph.Mesh(ph.make_config(nx, nb, **kw))
        probe.set_state(U)
        c0 = fa.calls
        assert probe.refine_where(flags, check_age=False)
        n_req = fa.calls - c0
        probe.close()
        assert n_req >= 3
        for k in range(1, n_req + 1):
            fa.arm(k)
            with pytest.raises(ph.PhError) as ei:
                m.refine_where(flags, check_age=False)
            assert ei.value.code == -2, str(ei.value)
            assert np.array_equal(m.tree(), tree0)
            assert np.array_equal(m.get_full(), ref.get_full())
        fa.fail_at = 0
        # still steps exactly like the mesh that never tried
        m.step(2)
        ref.step(2)
        assert np.array_equal(m.tree(), ref.tree())
        assert np.array_equal(m.get_state(), ref.get_state())
        # and the refinement goes through once memory is there
        assert m.refine_where(flags, check_age=False)
        assert ref.refine_where(flags, check_age=False)
        assert np.array_equal(m.tree(), ref.tree())
        assert np.array_equal(m.get_full(), ref.get_full())
        m.step(1)
        ref.step(1)
        assert np.array_equal(m.get_state(), ref.get_state())
        m.close()
        ref.close()
        assert not fa.live
    finally:
        _restore_default(ph)
