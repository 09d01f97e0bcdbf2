"""Failure handling on the GPU without a GPU fault: device allocations that the
host allocator refuses, and pools over their memory limit, end the call with
HBX_ERR_OOM, and the context keeps working with the same results as before."""
import ctypes

import numpy as np
import pytest

import paper_2208_00613_gb300 as hbx
import synth

pytestmark = pytest.mark.gpu

HBX_ERR_OOM = -2


@pytest.fixture(scope="module")
def small_graph():
    w = synth.WORKLOADS["ic_rmat4k"]
    return w, w.graph()


class BudgetAllocator:
    """Allocates through torch's caching allocator until a byte budget is used
    up, then refuses (returns NULL), as an exhausted device would."""

    def __init__(self, tc, budget):
        import torch
        self.torch, self.tc, self.left, self.sizes = torch, tc, budget, {}
        self.refused = 0

        def _alloc(size, user):
            if size > self.left:
                self.refused += 1
                return None
            ptr = torch.cuda.caching_allocator_alloc(int(size), tc.device, tc.stream)
            self.left -= size
            self.sizes[ptr] = size
            return ptr

        def _free(ptr, user):
            self.left += self.sizes.pop(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self._a = hbx._ALLOC_T(_alloc)
        self._f = hbx._FREE_T(_free)
        hbx.hbx_set_allocator(tc.ctx, ctypes.cast(self._a, ctypes.c_void_p), ctypes.cast(self._f, ctypes.c_void_p))


def test_refused_allocation_reports_oom_and_context_survives(small_graph):
    w, g = small_graph
    with hbx.torch_context(0) as tc:
        ref = hbx.hbx_imm(tc.ctx, hbx.hbx_graph_create(tc.ctx, g), w.model, w.k, w.eps, w.ell, w.rr_seed)
    with hbx.torch_context(0) as tc:
        alloc = BudgetAllocator(tc, 1 << 30)
        G = hbx.hbx_graph_create(tc.ctx, g)
        alloc.left = 16 << 10  # the graph is resident; the pool will not fit
        with pytest.raises(hbx.HbxError) as e:
            hbx.hbx_imm(tc.ctx, G, w.model, w.k, w.eps, w.ell, w.rr_seed)
        assert e.value.code == HBX_ERR_OOM
        assert alloc.refused > 0
        held = sum(alloc.sizes.values())
        alloc.left += 1 << 30  # memory comes back
        r = hbx.hbx_imm(tc.ctx, G, w.model, w.k, w.eps, w.ell, w.rr_seed)
        assert np.array_equal(r["seeds"], ref["seeds"])
        assert r["influence"] == ref["influence"]
        hbx.hbx_graph_destroy(G)
        assert sum(alloc.sizes.values()) <= held  # the failed call left nothing behind


def test_pool_memory_limit(small_graph):
    w, g = small_graph
    with hbx.torch_context(0) as tc:
        G = hbx.hbx_graph_create(tc.ctx, g)
        p = hbx.hbx_pool_create(tc.ctx, G, "IC", w.rr_seed, hbx.hbx_default_options(encode=0, max_device_bytes=1 << 16))
        with pytest.raises(hbx.HbxError) as e:
            hbx.hbx_pool_extend(tc.ctx, p, 1000)
        assert e.value.code == HBX_ERR_OOM
        hbx.hbx_pool_destroy(p)
        p = hbx.hbx_pool_create(tc.ctx, G, "IC", w.rr_seed, hbx.hbx_default_options(encode=0))
        hbx.hbx_pool_extend(tc.ctx, p, 1000)
        assert hbx.hbx_pool_size(p) == 1000
        hbx.hbx_pool_destroy(p)
        hbx.hbx_graph_destroy(G)


def test_selection_wait_that_runs_out_reports_timeout(small_graph):
    """The batched form's selection waits at grid barriers; each wait is
    bounded.  With a budget of one clock cycle the first block to arrive gives
    up at once: the call must end with TIMEOUT (not hang), and the context must
    then give the same results as before."""
    w, g = small_graph
    with hbx.torch_context(0) as tc:
        G = hbx.hbx_graph_create(tc.ctx, g)
        ref = hbx.hbx_imm(tc.ctx, G, w.model, w.k, w.eps, w.ell, w.rr_seed)
        with pytest.raises(hbx.HbxError) as e:
            hbx.hbx_imm(tc.ctx, G, w.model, w.k, w.eps, w.ell, w.rr_seed, hbx.hbx_default_options(wait_cycles=1))
        assert e.value.code == -4  # HBX_ERR_TIMEOUT
        r = hbx.hbx_imm(tc.ctx, G, w.model, w.k, w.eps, w.ell, w.rr_seed)
        assert np.array_equal(r["seeds"], ref["seeds"])
        assert r["influence"] == ref["influence"]
        hbx.hbx_graph_destroy(G)
