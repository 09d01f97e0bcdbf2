"""The allocation-free argmax entry point against the selection's own argmax.

hbx_argmax_noalloc serves callers that cannot allocate device memory where
they need an argmax: a service that reserves all of its GPU memory up front and
must stay within that fixed budget, or code running inside a memory allocator's
hook, where allocating again would re-enter the allocator.  Its scratch lives
in a static device array instead of library allocations.

The checks, through the C ABI: it must pick the same vertex as the existing
selection path (the first seed of hbx_pool_select is the argmax of the initial
counts, lowest id on ties) -- exactly, since this is integer work -- on two
calls in a row with different inputs; and, over many blocks, the same index as
numpy's argmax (first index of the largest value) for any int32 counts:
negative values and the int32 extremes, ties whose copies sit in different
blocks, a partial last block, and the largest accepted size, with two launches
queued back to back on one stream before either is read.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

hbx = pytest.importorskip("paper_2208_00613_gb300")

NMAX = 16777216  # HBX_ARGMAX_NOALLOC_MAX
PER_BLOCK = 256 * 16  # counts reduced by one block of the kernel


@pytest.fixture(scope="module")
def tc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hbx.build()
    t = hbx.torch_context(0)
    # the one-time set-up alone: loads the kernel and resolves the scratch address
    assert hbx.hbx_argmax_noalloc(0, 0, 0, torch.cuda.current_stream().cuda_stream) == 0
    yield t
    t.close()


def test_noalloc_argmax_matches_selection(tc):
    import torch
    w = synth.WORKLOADS["ic_rmat4k"]
    g = w.graph()
    G = hbx.hbx_graph_create(tc.ctx, g)
    p = hbx.hbx_pool_create(tc.ctx, G, "IC", w.rr_seed, hbx.hbx_default_options(encode=1, warmup_sets=500))
    try:
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
        # sizes above the static scratch's capacity, and empty input, are
        # rejected before any launch
        assert hbx.hbx_argmax_noalloc(d.data_ptr(), NMAX + 1, out.data_ptr(), stream) == -1
        assert hbx.hbx_argmax_noalloc(d.data_ptr(), 0, out.data_ptr(), stream) == -1
    finally:
        hbx.hbx_pool_destroy(p)
        hbx.hbx_graph_destroy(G)


def _cases():
    rng = np.random.default_rng(2208)
    lo, hi = np.iinfo(np.int32).min, np.iinfo(np.int32).max
    # random int32 over the whole range, the maximum (INT_MAX) in the partial last block
    n = (1 << 20) + 3
    a = rng.integers(lo, hi, size=n, dtype=np.int32, endpoint=False)
    a[a == hi] = hi - 1
    a[n - 2] = hi
    a[5] = lo
    yield "full range, max in the last block", a
    # a tie whose copies sit in different blocks: the lower index wins
    b = rng.integers(-1000, 1000, size=n, dtype=np.int32)
    b[3 * PER_BLOCK + 17] = 5000
    b[200 * PER_BLOCK + 1] = 5000
    b[n - 1] = 5000
    yield "tie across blocks", b
    # every count negative; the largest value is INT_MIN + 7 at two places
    c = np.full(n, lo, dtype=np.int32)
    c[PER_BLOCK * 100 + 9] = lo + 7
    c[PER_BLOCK * 7 + 3] = lo + 7
    yield "all negative", c
    # the largest accepted size (exactly 4096 blocks), the maximum tied between
    # the first block's end and the last block
    d = rng.integers(0, 1 << 20, size=NMAX, dtype=np.int32)
    d[PER_BLOCK - 1] = 1 << 24
    d[NMAX - 1] = 1 << 24
    yield "n = maximum", d
    e = rng.integers(-5, 5, size=NMAX, dtype=np.int32)
    e[NMAX - 1] = 99
    yield "n = maximum, max at the very end", e


def test_noalloc_argmax_many_blocks(tc):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    cases = list(_cases())
    outs = torch.full((len(cases),), -1, dtype=torch.int32, device="cuda:0")
    devs = [torch.from_numpy(a).to("cuda:0") for _, a in cases]
    torch.cuda.synchronize()
    # queue pairs of launches back to back on one stream, read both afterwards
    for i in range(0, len(cases), 2):
        for k in range(i, min(i + 2, len(cases))):
            rc = hbx.hbx_argmax_noalloc(devs[k].data_ptr(), int(devs[k].numel()), outs[k:k + 1].data_ptr(), stream)
            assert rc == 0, hbx.hbx_strerror(rc)
        torch.cuda.synchronize()
    got = outs.cpu().numpy()
    for (name, a), gi in zip(cases, got):
        assert int(gi) == int(np.argmax(a)), name
