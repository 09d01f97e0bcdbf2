"""GPU parity of the paper-literal modes against the oracle.

- Algorithm 1's per-graph scheme (Characterize on the warm-up block): the
  decision equals the oracle's; Huffmax codes every set (density cut off) and
  Bitmax stores every set as a column of the vertex-major 32-set tiles of
  Section 4.2.3 / Eq. (3).  Sets, encodings, seeds and IMM results equal the
  oracle's.
- Recount-from-scratch selection (Algorithms 2 and 3 as printed) and the
  adaptive choice between recounting and decrementing on Huffman, bitmap-row,
  tile and uncompressed pools: seeds, marginal gains and coverage equal the
  oracle's greedy, its per-iteration recount and, for tiles, its BitmaxQuery
  (POPCOUNT / SUBTRACT).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

hbx = pytest.importorskip("paper_2208_00613_gb300")


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hbx.build()
    c = hbx.torch_context(0)
    yield c.ctx
    c.close()


def gpu_sets(ctx, p, j0, j1):
    off, verts = hbx.hbx_pool_decode_sets(ctx, p, j0, j1)
    return [verts[off[i]:off[i + 1]] for i in range(j1 - j0)]


def same_sets(ctx, p, op, T):
    off, verts = op.concat(0, T)
    got = gpu_sets(ctx, p, 0, T)
    for j in range(T):
        assert np.array_equal(got[j], verts[off[j]:off[j + 1]]), j


def dense_graph():
    # uniform R-MAT (a = b = c = d = 1/4), mean live in-degree 2: about 80% of
    # the sets reach most of the graph, so the sizes skew negative (Bitmax)
    g = synth.rmat(1 << 13, 1 << 17, 41, 0.25, 0.25, 0.25)
    g.prob = synth.ic_uniform(g, 41, 0.25)
    return g


def skewed_graph():
    g = synth.rmat(1 << 14, 1 << 17, 5)
    g.prob = synth.weighted_cascade(g)
    return g


def test_scheme_bitmax_tiles(ctx):
    g = dense_graph()
    G = hbx.hbx_graph_create(ctx, g)
    T, W = 1000, 160
    p = hbx.hbx_pool_create(ctx, G, "IC", 13, hbx.hbx_default_options(encode=1, warmup_sets=W, scheme=1))
    try:
        hbx.hbx_pool_extend(ctx, p, 300)  # a partial tile, completed by the next extension
        hbx.hbx_pool_extend(ctx, p, T)
        op = oracle.Pool(g, oracle.IC, 13)
        op.extend(T)
        bitmax, skew = op.scheme(W)
        st = hbx.hbx_pool_stats(ctx, p)
        assert bitmax and st["scheme"] == 3 and st["scheme_skewness"] == skew
        assert st["sets_bitmap"] == T and st["sets_huffman"] == 0
        same_sets(ctx, p, op, T)
        sc, lv = op.edge_counts()
        assert st["edges_scanned"] == sc and 0 < st["edges_live"] <= lv
        # each set's bitmap equals the oracle encoder's with every set a bitmap
        cb = oracle.Codebook(g.n, op.warmup_freq(W, 0))
        for j in list(range(0, T, 37)) + [31, 32, 299, 300, T - 1]:
            got = hbx.hbx_pool_export_set(ctx, p, j)
            ref = oracle.encode_set(cb, g.n + 1, op.set(j))
            assert got["kind"] == 1 and np.array_equal(got["bitmap"], ref["bitmap"]), j
        # greedy on the tiles, by decrement and by recount, equals the oracle's
        # greedy and its BitmaxQuery on the same tiles
        ref = op.greedy(T, 20)
        bq = oracle.bitmax_query(op.bitmax_tiles(T), T, 20)
        assert bq[0].tolist() == ref[0].tolist() and bq[1].tolist() == ref[1].tolist()
        for T2 in (T, 517):
            s, m, c = hbx.hbx_pool_select(ctx, p, T2, 20)
            so, mo, co = op.greedy(T2, 20)
            assert s.tolist() == so.tolist() and m.tolist() == mo.tolist() and c == co
    finally:
        hbx.hbx_pool_destroy(p)
    for mode in (1, 2):  # recount, adaptive (the first seeds cover most sets here)
        p = hbx.hbx_pool_create(ctx, G, "IC", 13, hbx.hbx_default_options(encode=1, warmup_sets=W, scheme=1,
                                                                          select_mode=mode))
        try:
            hbx.hbx_pool_extend(ctx, p, T)
            s, m, c = hbx.hbx_pool_select(ctx, p, T, 20)
            so, mo, co = op.greedy_recount(T, 20)
            assert s.tolist() == so.tolist() and m.tolist() == mo.tolist() and c == co, mode
        finally:
            hbx.hbx_pool_destroy(p)
    # the whole IMM under the per-graph scheme, against the oracle's IMM
    r = hbx.hbx_imm(ctx, G, "IC", 10, 0.5, 1.0, 13, hbx.hbx_default_options(scheme=1))
    ro = oracle.Pool(g, oracle.IC, 13).imm(10, 0.5, 1.0)
    assert np.array_equal(r["seeds"], ro["seeds"]) and r["influence"] == ro["influence"]
    assert r["stats"]["scheme"] == 3
    hbx.hbx_graph_destroy(G)


def test_scheme_huffmax(ctx):
    g = skewed_graph()
    G = hbx.hbx_graph_create(ctx, g)
    T, W = 3000, 400
    p = hbx.hbx_pool_create(ctx, G, "IC", 9, hbx.hbx_default_options(encode=1, warmup_sets=W, scheme=1))
    try:
        hbx.hbx_pool_extend(ctx, p, T)
        op = oracle.Pool(g, oracle.IC, 9)
        op.extend(T)
        bitmax, skew = op.scheme(W)
        st = hbx.hbx_pool_stats(ctx, p)
        assert not bitmax and st["scheme"] == 1 and st["scheme_skewness"] == skew
        assert st["sets_bitmap"] == 0 and st["sets_huffman"] == T
        same_sets(ctx, p, op, T)
        # every set Huffman-coded: codebook from all warm-up sets (cut 0)
        f = op.warmup_freq(W, 0)
        cbg = hbx.hbx_pool_export_codebook(ctx, p, g.n)
        assert np.array_equal(cbg["freq"], f)
        cb = oracle.Codebook(g.n, f)
        for j in range(0, T, 11):
            got = hbx.hbx_pool_export_set(ctx, p, j)
            ref = oracle.encode_set(cb, 0, op.set(j))
            assert got["kind"] == 0 and got["bytes"] == ref["bytes"], j
            assert np.array_equal(got["raw"], ref["raw"]), j
        # Algorithm 2 over the oracle's encodings gives the same seeds
        encs = [oracle.encode_set(cb, 0, op.set(j)) for j in range(T)]
        hq = oracle.huffmax_query(cb, encs, 15)
        s, m, c = hbx.hbx_pool_select(ctx, p, T, 15)
        assert s.tolist() == hq[0].tolist() and m.tolist() == hq[1].tolist() and c == hq[2]
    finally:
        hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)


@pytest.mark.parametrize("kind", ["huffman", "rows", "raw"])
def test_recount_selection(ctx, kind):
    if kind == "rows":
        g = dense_graph()  # sets over n/32 vertices are bitmap rows under the per-set cut
        o = dict(encode=1, warmup_sets=150)
    elif kind == "huffman":
        g = skewed_graph()
        o = dict(encode=1, warmup_sets=300)
    else:
        g = skewed_graph()
        o = dict(encode=0)
    G = hbx.hbx_graph_create(ctx, g)
    T, k = 1200, 25
    op = oracle.Pool(g, oracle.IC, 21)
    op.extend(T)
    ref = op.greedy(T, k)
    assert [x.tolist() if hasattr(x, "tolist") else x for x in op.greedy_recount(T, k)] == \
        [x.tolist() if hasattr(x, "tolist") else x for x in ref]
    for mode in (0, 1, 2):  # decrement, recount, adaptive
        p = hbx.hbx_pool_create(ctx, G, "IC", 21, hbx.hbx_default_options(select_mode=mode, **o))
        try:
            hbx.hbx_pool_extend(ctx, p, T)
            st = hbx.hbx_pool_stats(ctx, p)
            if kind == "rows":
                assert st["sets_bitmap"] > 0 and st["sets_huffman"] > 0
            for T2 in (T, 700):
                s, m, c = hbx.hbx_pool_select(ctx, p, T2, k)
                so, mo, co = op.greedy(T2, k)
                assert s.tolist() == so.tolist() and m.tolist() == mo.tolist() and c == co, (mode, T2)
        finally:
            hbx.hbx_pool_destroy(p)
    # IMM with recount selection equals the oracle's IMM
    r = hbx.hbx_imm(ctx, G, "IC", 12, 0.5, 1.0, 21, hbx.hbx_default_options(select_mode=1, **{
        kk: v for kk, v in o.items() if kk == "encode"}))
    ro = oracle.Pool(g, oracle.IC, 21).imm(12, 0.5, 1.0)
    assert np.array_equal(r["seeds"], ro["seeds"]) and r["influence"] == ro["influence"]
    hbx.hbx_graph_destroy(G)


@pytest.mark.parametrize("encode", [0, 1])
def test_imm_fresh_final_phase(ctx, encode):
    """IMM whose final phase draws theta new sets [T_i, T_i + theta): seeds,
    influence and theta equal the oracle's.  A second IMM (different k) on the
    same pool, whose T_i falls inside a batch the first one sampled, selects on
    a range that starts mid-batch."""
    w = synth.WORKLOADS["ic_rmat4k"]
    g = w.graph()
    G = hbx.hbx_graph_create(ctx, g)
    o = hbx.hbx_default_options(encode=encode, fresh_final=1, warmup_sets=300)
    p = hbx.hbx_pool_create(ctx, G, "IC", w.rr_seed, o)
    try:
        op = oracle.Pool(g, oracle.IC, w.rr_seed)
        for k, eps in ((w.k, w.eps), (3, 0.35)):
            r = hbx.hbx_imm_pool(ctx, p, k, eps, w.ell)
            ro = op.imm(k, eps, w.ell, fresh_final=True)
            assert np.array_equal(r["seeds"], ro["seeds"]), k
            assert np.array_equal(r["marginal"], ro["marginal"]), k
            assert r["influence"] == ro["influence"] and r["stats"]["theta"] == ro["theta"], k
    finally:
        hbx.hbx_pool_destroy(p)
    r = hbx.hbx_imm(ctx, G, "IC", w.k, w.eps, w.ell, w.rr_seed, hbx.hbx_default_options(fresh_final=1))
    ro = oracle.Pool(g, oracle.IC, w.rr_seed).imm(w.k, w.eps, w.ell, fresh_final=True)
    assert np.array_equal(r["seeds"], ro["seeds"]) and r["influence"] == ro["influence"]
    hbx.hbx_graph_destroy(G)
