"""The synthetic inputs: the stand-ins for the paper's Table 4 graphs and the
serving query stream are deterministic, well formed, and have the shapes the
workloads state (R-MAT skew, exact edge counts, IC / weighted-cascade / LT
weights in range, Poisson arrivals at the stated rate)."""
import numpy as np
import pytest

import synth


def csr_ok(g):
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    assert rp[0] == 0 and rp[-1] == g.m and len(rp) == g.n + 1
    assert np.all(np.diff(rp) >= 0)
    col = np.asarray(g.col)
    assert col.shape == (g.m,) and col.min() >= 0 and col.max() < g.n


def test_rmat_deterministic_exact_and_well_formed():
    a = synth.rmat(1 << 12, 1 << 15, 1)
    b = synth.rmat(1 << 12, 1 << 15, 1)
    c = synth.rmat(1 << 12, 1 << 15, 2)
    csr_ok(a)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert not np.array_equal(a.col, c.col)
    # a non-power-of-two vertex count keeps every id in range (pairs out of range are redrawn)
    d = synth.rmat(3000, 20000, 3)
    csr_ok(d)
    assert d.m == 20000


def test_rmat_is_skewed_and_relabelled():
    g = synth.rmat(1 << 14, 1 << 18, 5)
    indeg = np.diff(np.asarray(g.row_ptr, dtype=np.int64))
    # power-law-like in-degrees: the top 1% of vertices hold far more than 1% of edges
    top = np.sort(indeg)[::-1][: g.n // 100].sum()
    assert top > 0.1 * g.m
    # the seeded relabelling spreads heavy vertices over the id range
    heavy = np.nonzero(indeg > np.percentile(indeg, 99))[0]
    assert heavy.min() < g.n // 4 and heavy.max() > 3 * g.n // 4


def test_ic_wc_lt_weights():
    g = synth.rmat(1 << 12, 1 << 15, 7)
    p = synth.ic_uniform(g, 7, 0.1)
    assert p.dtype == np.float32 and p.shape == (g.m,)
    assert p.min() >= 0.0 and p.max() < 0.1
    assert abs(float(p.mean()) - 0.05) < 0.002
    wc = synth.weighted_cascade(g)
    indeg = np.diff(np.asarray(g.row_ptr, dtype=np.int64))
    per_edge_deg = np.repeat(indeg, indeg)
    assert np.array_equal(wc, (1.0 / per_edge_deg.astype(np.float32)).astype(np.float32))
    w = synth.lt_weights(g, 7)
    assert w.min() > 0.0
    # fixed-point weights of every vertex sum to at most 2^32 (the LT validation rule)
    q = np.floor(w.astype(np.float64) * 2.0 ** 32)
    sums = np.add.reduceat(q, np.asarray(g.row_ptr[:-1], dtype=np.int64)[indeg > 0])
    assert sums.max() <= 2.0 ** 32


def test_workloads_shapes():
    W = synth.WORKLOADS
    assert (W["ic_rmat4k"].n, W["ic_rmat4k"].m) == (4096, 32768)
    assert (W["wc_rmat1m"].n, W["wc_rmat1m"].m) == (1 << 20, 1 << 24)
    assert (W["lt_rmat4m"].n, W["lt_rmat4m"].m) == (1 << 22, 1 << 26)
    assert (W["ic_rmat42m"].n, W["ic_rmat42m"].m) == (41652230, 1468365182)
    for w in W.values():
        assert w.model in ("IC", "LT") and 0 < w.eps < 1 and w.k >= 1


def test_poisson_queries():
    qs = synth.poisson_queries(seed=3, count=4000, rate_per_s=20.0, graphs=[0, 1, 2])
    assert qs == synth.poisson_queries(seed=3, count=4000, rate_per_s=20.0, graphs=[0, 1, 2])
    t = np.array([q["t"] for q in qs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 20.0) < 0.005  # exponential gaps at rate 20/s
    assert abs(np.std(gaps) - 1 / 20.0) < 0.006
    assert {q["graph"] for q in qs} == {0, 1, 2}
    assert {q["model"] for q in qs} == {"IC", "LT"}
    ks = np.array([q["k"] for q in qs])
    assert ks.min() >= 10 and ks.max() <= 200
    assert {q["eps"] for q in qs} == {0.13, 0.2, 0.3, 0.5}


@pytest.mark.parametrize("edges", [[(0, 1), (1, 2), (0, 2)], [(2, 0), (2, 0), (1, 1)]])
def test_from_edges_transposed(edges):
    g = synth.from_edges(3, edges, prob=[0.5] * len(edges))
    csr_ok(g)
    # row v lists the sources u of the edges u -> v
    for v in range(3):
        srcs = sorted(int(u) for u in g.col[g.row_ptr[v]:g.row_ptr[v + 1]])
        assert srcs == sorted(u for (u, x) in edges if x == v)
