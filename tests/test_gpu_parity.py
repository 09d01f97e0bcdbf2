"""GPU parity: the CUDA path, called through the C ABI, against the oracle.

Integer work (RR sets, codebooks, encoded bytes, seeds, coverage) must match
bit for bit; the FP64 IMM outputs (theta, LB, influence) must match exactly,
since both sides evaluate the same expressions in the same order.
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


_GRAPHS = {}


def workload_graph(name):
    if name not in _GRAPHS:
        _GRAPHS[name] = synth.WORKLOADS[name].graph()
    return _GRAPHS[name]


def oracle_sets(pool, j0, j1):
    off, verts = pool.concat(j0, j1)
    return [verts[off[i]:off[i + 1]] for i in range(j1 - j0)]


def gpu_sets(ctx, p, j0, j1):
    off, verts = hbx.hbx_pool_decode_sets(ctx, p, j0, j1)
    return [verts[off[i]:off[i + 1]] for i in range(j1 - j0)]


def assert_same_sets(a, b, j0=0):
    assert len(a) == len(b)
    for i, (x, y) in enumerate(zip(a, b)):
        if not np.array_equal(x, y):
            raise AssertionError(f"set {j0 + i}: gpu {x[:20]}... ({len(x)}) vs oracle {y[:20]}... ({len(y)})")


def opts(**kw):
    return hbx.hbx_default_options(**kw)


# ---------------------------------------------------------------------------
# sampling
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("qw", [64, 256])
def test_raw_sets_ic_tiny(ctx, form, qw):
    w = synth.WORKLOADS["ic_rmat4k"]
    g = workload_graph("ic_rmat4k")
    G = hbx.hbx_graph_create(ctx, g)
    T = 5003  # several tiles and a ragged tail
    p = hbx.hbx_pool_create(ctx, G, "IC", w.rr_seed, opts(encode=0, form=form, warp_capacity=qw))
    hbx.hbx_pool_extend(ctx, p, T)
    op = oracle.Pool(g, oracle.IC, w.rr_seed)
    op.extend(T)
    assert_same_sets(gpu_sets(ctx, p, 0, T), oracle_sets(op, 0, T))
    st = hbx.hbx_pool_stats(ctx, p)
    sc, lv = op.edge_counts()
    assert st["edges_scanned"] == sc and st["edges_live"] == lv
    assert st["rr_vertices"] == int(op.sizes().sum())
    if qw == 64:
        assert st["sets_big"] > 0  # the block path ran
    hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)


def _check_encoded(ctx, p, op, g, W, cut, T, sample=None):
    n = g.n
    cb_gpu = hbx.hbx_pool_export_codebook(ctx, p, n)
    f = op.warmup_freq(W, cut)
    assert np.array_equal(cb_gpu["freq"], f)
    cb = oracle.Codebook(n, f)
    assert np.array_equal(cb_gpu["len"], cb.len)
    assert np.array_equal(cb_gpu["code"], cb.code)
    assert np.array_equal(cb_gpu["rank"], cb.rank)
    ids = range(T) if sample is None else sample
    for j in ids:
        s = op.set(j)
        ref = oracle.encode_set(cb, cut, s)
        got = hbx.hbx_pool_export_set(ctx, p, j)
        assert got["kind"] == ref["kind"], j
        assert got["size"] == ref["size"], j
        if ref["kind"] == 0:
            assert got["n_coded"] == ref["n_coded"] and got["code_bits"] == ref["code_bits"], j
            assert got["bytes"] == ref["bytes"], j
            assert np.array_equal(got["raw"], ref["raw"]), j
        else:
            assert np.array_equal(got["bitmap"], ref["bitmap"]), j


@pytest.mark.parametrize("qw", [64, 512])
@pytest.mark.parametrize("cut", [32, 4])
def test_encoded_sets_ic_tiny(ctx, qw, cut):
    w = synth.WORKLOADS["ic_rmat4k"]
    g = workload_graph("ic_rmat4k")
    G = hbx.hbx_graph_create(ctx, g)
    T, W = 3001, 400
    p = hbx.hbx_pool_create(ctx, G, "IC", w.rr_seed, opts(encode=1, warmup_sets=W, density_cut=cut,
                                                          warp_capacity=qw))
    hbx.hbx_pool_extend(ctx, p, T)
    op = oracle.Pool(g, oracle.IC, w.rr_seed)
    op.extend(T)
    _check_encoded(ctx, p, op, g, W, cut, T)
    assert_same_sets(gpu_sets(ctx, p, 0, T), oracle_sets(op, 0, T))
    st = hbx.hbx_pool_stats(ctx, p)
    sizes = op.sizes()
    assert st["sets_bitmap"] == int((cut * sizes > g.n).sum())
    assert st["sets_huffman"] == T - st["sets_bitmap"]
    if cut == 32:
        assert st["sets_bitmap"] > 0
    hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)


def test_encoded_sets_plain_form(ctx):
    # the plain form samples and encodes every set with the HBM-scratch block kernel
    w = synth.WORKLOADS["ic_rmat4k"]
    g = workload_graph("ic_rmat4k")
    G = hbx.hbx_graph_create(ctx, g)
    T, W, cut = 2500, 300, 32
    p = hbx.hbx_pool_create(ctx, G, "IC", w.rr_seed, opts(encode=1, warmup_sets=W, density_cut=cut, form=0))
    hbx.hbx_pool_extend(ctx, p, T)
    op = oracle.Pool(g, oracle.IC, w.rr_seed)
    op.extend(T)
    _check_encoded(ctx, p, op, g, W, cut, T)
    st = hbx.hbx_pool_stats(ctx, p)
    assert st["sets_big"] == T
    sc, lv = op.edge_counts()
    assert st["edges_scanned"] == sc and st["edges_live"] == lv
    hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)


def test_encoded_sets_wc_1m(ctx):
    """Weighted cascade on the 2^20-vertex graph: Huffman and bitmap sets, every
    set checked byte for byte on a prefix, decoded sets compared on the rest."""
    w = synth.WORKLOADS["wc_rmat1m"]
    g = workload_graph("wc_rmat1m")
    G = hbx.hbx_graph_create(ctx, g)
    T, W = 20000, 2000
    p = hbx.hbx_pool_create(ctx, G, "IC", w.rr_seed, opts(encode=1, warmup_sets=W))
    hbx.hbx_pool_extend(ctx, p, T)
    op = oracle.Pool(g, oracle.IC, w.rr_seed)
    op.extend(T)
    _check_encoded(ctx, p, op, g, W, 32, T, sample=range(0, T, 7))
    assert_same_sets(gpu_sets(ctx, p, 0, T), oracle_sets(op, 0, T))
    hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)


@pytest.mark.parametrize("cut", [32, 2])
def test_giant_ic_sets_bit_parallel(ctx, cut):
    """Supercritical IC (mean live in-degree 2): many sets outgrow shared memory
    and are searched 32 at a time.  cut 32 makes them bitmaps; with cut 2 the
    ones under n/2 vertices are Huffman-coded from their membership rows.  Sets,
    their encodings, the warm-up frequencies and the edge counts equal the
    oracle's."""
    g = synth.rmat(1 << 15, 1 << 19, 41)
    g.prob = synth.ic_uniform(g, 41, 0.25)
    G = hbx.hbx_graph_create(ctx, g)
    T, W = 700, 150
    p = hbx.hbx_pool_create(ctx, G, "IC", 13, opts(encode=1, warmup_sets=W, density_cut=cut))
    hbx.hbx_pool_extend(ctx, p, T)
    op = oracle.Pool(g, oracle.IC, 13)
    op.extend(T)
    sizes = op.sizes()
    assert (sizes > 4096).sum() > 64  # several batches of the bit-parallel search
    assert_same_sets(gpu_sets(ctx, p, 0, T), oracle_sets(op, 0, T))
    _check_encoded(ctx, p, op, g, W, cut, T, sample=range(0, T, 5))
    st = hbx.hbx_pool_stats(ctx, p)
    sc, lv = op.edge_counts()
    # the bit-parallel search skips the coins of edges into sources a set has
    # already visited: scanned edges are exact, live edges a subset
    assert st["edges_scanned"] == sc and 0 < st["edges_live"] <= lv
    assert st["rr_vertices"] == int(sizes.sum())
    assert st["sets_bitmap"] == int((cut * sizes > g.n).sum())
    # hubs of over 512 in-edges had their expansion deferred (same sets)
    assert st["ms_deferrals"] > 0 and st["ms_group_visits"] > 0
    if cut == 2:
        assert ((sizes > 4096) & (cut * sizes <= g.n)).sum() > 0  # some were Huffman-coded
    s, m, c = hbx.hbx_pool_select(ctx, p, T, 20)
    so, mo, co = op.greedy(T, 20)
    assert s.tolist() == so.tolist() and m.tolist() == mo.tolist() and c == co
    hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)


@pytest.mark.parametrize("qw", [64, 256])
def test_lt_sets(ctx, qw):
    g = synth.rmat(1 << 16, 1 << 20, 33)
    g.lt_weight = synth.lt_weights(g, 33)
    G = hbx.hbx_graph_create(ctx, g)
    T, W = 20011, 2500
    p = hbx.hbx_pool_create(ctx, G, "LT", 9, opts(encode=1, warmup_sets=W, warp_capacity=qw))
    hbx.hbx_pool_extend(ctx, p, T)
    op = oracle.Pool(g, oracle.LT, 9)
    op.extend(T)
    assert_same_sets(gpu_sets(ctx, p, 0, T), oracle_sets(op, 0, T))
    _check_encoded(ctx, p, op, g, W, 32, T, sample=range(0, T, 3))
    st = hbx.hbx_pool_stats(ctx, p)
    sc, lv = op.edge_counts()
    assert st["edges_scanned"] == sc and st["edges_live"] == lv
    hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)


def test_degenerate_graphs(ctx):
    # p = 1 chain (and LT weight 1): every set is a prefix path of up to 6000
    # vertices, so sets go through the warp, shared-memory block (<= 4096) and
    # global-bitmap block (> 4096) tiers
    P = 6000
    edges = [(i, i + 1) for i in range(P - 1)]
    g = synth.from_edges(P, edges, prob=[1.0] * (P - 1), lt_weight=[1.0] * (P - 1))
    G = hbx.hbx_graph_create(ctx, g)
    for model, om in (("IC", oracle.IC), ("LT", oracle.LT)):
        for enc in (0, 1):
            p = hbx.hbx_pool_create(ctx, G, model, 5, opts(encode=enc, warmup_sets=50, warp_capacity=128))
            hbx.hbx_pool_extend(ctx, p, 300)
            op = oracle.Pool(g, om, 5)
            op.extend(300)
            assert_same_sets(gpu_sets(ctx, p, 0, 300), oracle_sets(op, 0, 300))
            assert int(op.sizes().max()) > 4096
            hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)
    # no edges at all: every set is its root; greedy takes the most frequent roots
    g = synth.from_edges(50, [], prob=[])
    G = hbx.hbx_graph_create(ctx, g)
    p = hbx.hbx_pool_create(ctx, G, "IC", 6, opts(encode=1, warmup_sets=100))
    hbx.hbx_pool_extend(ctx, p, 1000)
    op = oracle.Pool(g, oracle.IC, 6)
    op.extend(1000)
    assert_same_sets(gpu_sets(ctx, p, 0, 1000), oracle_sets(op, 0, 1000))
    s, m, c = hbx.hbx_pool_select(ctx, p, 1000, 50)
    so, mo, co = op.greedy(1000, 50)
    assert s.tolist() == so.tolist() and m.tolist() == mo.tolist() and c == co
    hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)


# ---------------------------------------------------------------------------
# selection and IMM
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("enc,form", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_select_tiny(ctx, enc, form):
    w = synth.WORKLOADS["ic_rmat4k"]
    g = workload_graph("ic_rmat4k")
    G = hbx.hbx_graph_create(ctx, g)
    T = 6007
    p = hbx.hbx_pool_create(ctx, G, "IC", w.rr_seed, opts(encode=enc, form=form, warmup_sets=700))
    hbx.hbx_pool_extend(ctx, p, T)
    op = oracle.Pool(g, oracle.IC, w.rr_seed)
    op.extend(T)
    for TT, k in [(T, 10), (T - 1000, 40), (17, 30)]:
        s, m, c = hbx.hbx_pool_select(ctx, p, TT, k)
        so, mo, co = op.greedy(TT, k)
        assert s.tolist() == so.tolist()
        assert m.tolist() == mo.tolist()
        assert c == co
    hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)


@pytest.mark.parametrize("enc", [0, 1])
def test_select_incremental_counts(ctx, enc):
    # selections on growing prefixes of one pool restore the previous prefix's
    # counts and count only the new sets; each must equal the oracle's greedy
    w = synth.WORKLOADS["ic_rmat4k"]
    g = workload_graph("ic_rmat4k")
    G = hbx.hbx_graph_create(ctx, g)
    p = hbx.hbx_pool_create(ctx, G, "IC", w.rr_seed, opts(encode=enc, form=1, warmup_sets=300, density_cut=8))
    op = oracle.Pool(g, oracle.IC, w.rr_seed)
    op.extend(6000)
    for T, TT, k in [(1000, 1000, 12), (2500, 2500, 12), (2500, 1700, 5), (6000, 6000, 25), (6000, 3001, 7)]:
        hbx.hbx_pool_extend(ctx, p, T)
        s, m, c = hbx.hbx_pool_select(ctx, p, TT, k)
        so, mo, co = op.greedy(TT, k)
        assert s.tolist() == so.tolist(), (T, TT)
        assert m.tolist() == mo.tolist(), (T, TT)
        assert c == co
    if enc:
        assert hbx.hbx_pool_stats(ctx, p)["sets_bitmap"] > 0
    hbx.hbx_pool_destroy(p)
    hbx.hbx_graph_destroy(G)


@pytest.mark.parametrize("enc,form", [(0, 0), (1, 1)])
def test_imm_tiny(ctx, enc, form):
    w = synth.WORKLOADS["ic_rmat4k"]
    g = workload_graph("ic_rmat4k")
    G = hbx.hbx_graph_create(ctx, g)
    r = hbx.hbx_imm(ctx, G, "IC", w.k, w.eps, w.ell, w.rr_seed, opts(encode=enc, form=form))
    op = oracle.Pool(g, oracle.IC, w.rr_seed)
    ro = op.imm(w.k, w.eps, w.ell)
    assert r["seeds"].tolist() == ro["seeds"].tolist()
    assert r["marginal"].tolist() == ro["marginal"].tolist()
    assert r["stats"]["theta"] == ro["theta"]
    assert r["stats"]["covered"] == ro["covered"]
    assert r["stats"]["rounds"] == ro["rounds"]
    assert r["stats"]["lb"] == ro["lb"]
    assert r["influence"] == ro["influence"]
    hbx.hbx_graph_destroy(G)


def test_imm_wc_1m(ctx):
    w = synth.WORKLOADS["wc_rmat1m"]
    g = workload_graph("wc_rmat1m")
    G = hbx.hbx_graph_create(ctx, g)
    r = hbx.hbx_imm(ctx, G, "IC", w.k, w.eps, w.ell, w.rr_seed, opts(encode=1, form=1))
    op = oracle.Pool(g, oracle.IC, w.rr_seed)
    ro = op.imm(w.k, w.eps, w.ell)
    assert r["stats"]["theta"] == ro["theta"]
    assert r["seeds"].tolist() == ro["seeds"].tolist()
    assert r["marginal"].tolist() == ro["marginal"].tolist()
    assert r["influence"] == ro["influence"]
    # the warm-up block is ceil(T_1 / 8) sets, T_1 being IMM's first sampling
    # target (the reading of Algorithm 1's "first block" when theta is not
    # known up front); its copy-array share is reported
    T1 = int(ro["round_T"][0])
    assert r["stats"]["warmup_sets"] == (T1 + 7) // 8
    assert 0 < r["stats"]["uncoded_vertices"] < r["stats"]["rr_vertices"]
    hbx.hbx_graph_destroy(G)


def test_imm_lt_4m(ctx):
    w = synth.WORKLOADS["lt_rmat4m"]
    g = workload_graph("lt_rmat4m")
    G = hbx.hbx_graph_create(ctx, g)
    r = hbx.hbx_imm(ctx, G, "LT", w.k, w.eps, w.ell, w.rr_seed, opts(encode=1, form=1))
    op = oracle.Pool(g, oracle.LT, w.rr_seed)
    ro = op.imm(w.k, w.eps, w.ell)
    assert r["stats"]["theta"] == ro["theta"]
    assert r["seeds"].tolist() == ro["seeds"].tolist()
    assert r["marginal"].tolist() == ro["marginal"].tolist()
    assert r["influence"] == ro["influence"]
    hbx.hbx_graph_destroy(G)


def test_invalid_arguments(ctx):
    g = synth.from_edges(3, [(0, 1), (2, 1)], lt_weight=[0.75, 0.5])
    with pytest.raises(hbx.HbxError) as e:
        hbx.hbx_graph_create(ctx, g)
    assert e.value.code == -5
    g = synth.from_edges(3, [(0, 1), (2, 1)], prob=[0.5, 1.5])
    with pytest.raises(hbx.HbxError) as e:
        hbx.hbx_graph_create(ctx, g)
    assert e.value.code == -1
    g = synth.from_edges(3, [(0, 1), (2, 1)], prob=[0.5, 0.5])
    G = hbx.hbx_graph_create(ctx, g)
    with pytest.raises(hbx.HbxError):
        hbx.hbx_imm(ctx, G, "IC", 4, 0.5, 1.0, 1)  # k > n
    with pytest.raises(hbx.HbxError):
        hbx.hbx_imm(ctx, G, "LT", 1, 0.5, 1.0, 1)  # no LT weights
    with pytest.raises(hbx.HbxError):
        hbx.hbx_imm(ctx, G, "IC", 1, 1.5, 1.0, 1)  # eps out of range
    hbx.hbx_graph_destroy(G)
