"""The allocation-free argmax entry point against the selection's own argmax.

hbx_argmax_noalloc serves callers that cannot allocate device memory where
they need an argmax: a service that reserves all of its GPU memory up front and
must stay within that fixed budget, or code running inside a memory allocator's
hook, where allocating again would re-enter the allocator.  Its scratch lives
in a static device array instead of library allocations.

The check: through the C ABI, it must pick the same vertex as the existing
selection path (the first seed of hbx_pool_select is the argmax of the initial
counts, lowest id on ties) -- exactly, since this is integer work -- on two
calls in a row with different inputs.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

hbx = pytest.importorskip("paper_2208_00613_gb300")


def test_noalloc_argmax_matches_selection():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hbx.build()
    tc = hbx.torch_context(0)
    try:
        w = synth.WORKLOADS["ic_rmat4k"]
        g = w.graph()
        G = hbx.hbx_graph_create(tc.ctx, g)
        p = hbx.hbx_pool_create(tc.ctx, G, "IC", w.rr_seed, hbx.hbx_default_options(encode=1, warmup_sets=500))
        hbx.hbx_pool_extend(tc.ctx, p, 6000)
        off, verts = hbx.hbx_pool_decode_sets(tc.ctx, p, 0, 6000)
        out = torch.full((1,), -1, dtype=torch.int32, device="cuda:0")
        stream = torch.cuda.current_stream().cuda_stream
        for T in (6000, 1234):  # two calls in a row, different inputs
            counts = np.bincount(verts[:int(off[T])].astype(np.int64), minlength=g.n).astype(np.int32)
            d = torch.from_numpy(counts).to("cuda:0")
            rc = hbx.hbx_argmax_noalloc(d.data_ptr(), g.n, out.data_ptr(), stream)
            torch.cuda.synchronize()
            assert rc == 0, hbx.hbx_strerror(rc)
            seeds, _, _ = hbx.hbx_pool_select(tc.ctx, p, T, 1)
            assert int(out.item()) == int(seeds[0])
            assert int(out.item()) == int(np.argmax(counts))
        # sizes above the static scratch's capacity are rejected before any launch
        rc = hbx.hbx_argmax_noalloc(d.data_ptr(), 16777216 + 1, out.data_ptr(), stream)
        assert rc == -1
        hbx.hbx_pool_destroy(p)
        hbx.hbx_graph_destroy(G)
    finally:
        tc.close()
