"""Pins the oracle's RR-set sampler to the diffusion models themselves.

- Exact distributions by brute force over every live-edge world of tiny graphs
  (IC: each edge live with its probability, Section 2.1; LT: each vertex keeps
  at most one in-edge, edge e with probability w_e) against the sampler's
  empirical frequencies (chi-square).
- The RR-set identity sigma(S) = n Pr[R meets S] (Section 2.2, Borgs et al.),
  with sigma(S) computed by brute force over worlds, against the sampler.
- Closed forms on stars and paths with p in {0, 1}.
"""
import itertools
from collections import Counter

import numpy as np
import pytest
from scipy import stats

import oracle
import synth

IC, LT = oracle.IC, oracle.LT


def _reverse_reach(n, live_in, root):
    """live_in[v] = list of sources u of live edges u -> v."""
    seen = {root}
    stack = [root]
    while stack:
        v = stack.pop()
        for u in live_in[v]:
            if u not in seen:
                seen.add(u)
                stack.append(u)
    return frozenset(seen)


def _forward_reach(n, live_out, S):
    seen = set(S)
    stack = list(S)
    while stack:
        u = stack.pop()
        for v in live_out[u]:
            if v not in seen:
                seen.add(v)
                stack.append(v)
    return len(seen)


def _ic_worlds(n, edges, probs):
    """Yield (probability, live edge list) for all 2^m IC worlds."""
    m = len(edges)
    for mask in range(1 << m):
        pr = 1.0
        live = []
        for i in range(m):
            if mask >> i & 1:
                pr *= probs[i]
                live.append(edges[i])
            else:
                pr *= 1.0 - probs[i]
        if pr > 0:
            yield pr, live


def _lt_worlds(n, edges, q):
    """LT live-edge worlds: each vertex picks in-edge e with prob q_e / 2^32 or none."""
    in_edges = [[i for i, (u, v) in enumerate(edges) if v == t] for t in range(n)]
    choices = []
    for t in range(n):
        opts = [(None, 1.0 - sum(q[i] for i in in_edges[t]) / 2**32)]
        opts += [(i, q[i] / 2**32) for i in in_edges[t]]
        choices.append(opts)
    for combo in itertools.product(*choices):
        pr = 1.0
        live = []
        for c, p in combo:
            pr *= p
            if c is not None:
                live.append(edges[c])
        if pr > 0:
            yield pr, live


def _exact_set_dist(n, worlds):
    dist = Counter()
    for pr, live in worlds:
        live_in = [[] for _ in range(n)]
        for (u, v) in live:
            live_in[v].append(u)
        for r in range(n):
            dist[_reverse_reach(n, live_in, r)] += pr / n
    return dist


def _empirical(g, model, seed, N):
    pool = oracle.Pool(g, model, seed)
    pool.extend(N)
    off, verts = pool.concat()
    c = Counter()
    for j in range(N):
        c[frozenset(verts[off[j]:off[j + 1]].tolist())] += 1
    return c


def _chi2_pvalue(exact, emp, N):
    keys = sorted(exact, key=lambda s: -exact[s])
    assert set(emp) <= set(exact), "sampler produced a set that no world produces"
    obs, exp = [], []
    rest_o, rest_e = 0, 0.0
    for s in keys:
        e = exact[s] * N
        if e >= 5:
            obs.append(emp.get(s, 0))
            exp.append(e)
        else:
            rest_o += emp.get(s, 0)
            rest_e += e
    if rest_e > 0:
        obs.append(rest_o)
        exp.append(rest_e)
    exp = np.array(exp)
    exp *= N / exp.sum()
    return stats.chisquare(obs, exp).pvalue


TINY_EDGES = [(1, 0), (2, 0), (2, 1), (3, 1), (0, 2), (4, 2), (3, 4), (0, 4), (5, 3), (1, 5), (4, 5), (5, 0)]


def test_ic_distribution_matches_all_worlds():
    n = 6
    rng = np.random.default_rng(3)
    probs = rng.uniform(0.1, 0.9, size=len(TINY_EDGES)).astype(np.float32)
    g = synth.from_edges(n, TINY_EDGES, prob=probs)
    # the sampler's coin is u24(x) < p, so the exact live probability of an edge
    # is ceil(p * 2^24) / 2^24
    order = sorted(range(len(TINY_EDGES)), key=lambda i: (TINY_EDGES[i][1], i))
    p_exact = [np.ceil(float(probs[i]) * 2**24) / 2**24 for i in range(len(TINY_EDGES))]
    exact = _exact_set_dist(n, _ic_worlds(n, TINY_EDGES, p_exact))
    assert abs(sum(exact.values()) - 1.0) < 1e-9
    N = 200_000
    emp = _empirical(g, IC, 11, N)
    assert _chi2_pvalue(exact, emp, N) > 1e-4
    del order


def test_lt_distribution_matches_all_worlds():
    n = 6
    rng = np.random.default_rng(5)
    raw = rng.uniform(0.05, 1.0, size=len(TINY_EDGES))
    w = np.zeros(len(TINY_EDGES), dtype=np.float32)
    for t in range(n):
        idx = [i for i, (u, v) in enumerate(TINY_EDGES) if v == t]
        tot = raw[idx].sum() * 1.25  # leave some probability of no activation
        for i in idx:
            w[i] = np.float32(raw[i] / tot)
    g = synth.from_edges(n, TINY_EDGES, lt_weight=w)
    q = [int(np.floor(float(w[i]) * 2**32)) for i in range(len(TINY_EDGES))]
    exact = _exact_set_dist(n, _lt_worlds(n, TINY_EDGES, q))
    assert abs(sum(exact.values()) - 1.0) < 1e-9
    N = 200_000
    emp = _empirical(g, LT, 13, N)
    assert _chi2_pvalue(exact, emp, N) > 1e-4


@pytest.mark.parametrize("model", [IC, LT])
def test_rr_identity_sigma(model):
    """n * Pr[R meets S] = sigma(S) = E_world |reach(S)|."""
    n = 6
    rng = np.random.default_rng(7)
    if model == IC:
        probs = rng.uniform(0.2, 0.8, size=len(TINY_EDGES)).astype(np.float32)
        g = synth.from_edges(n, TINY_EDGES, prob=probs)
        p_exact = [np.ceil(float(probs[i]) * 2**24) / 2**24 for i in range(len(TINY_EDGES))]
        worlds = list(_ic_worlds(n, TINY_EDGES, p_exact))
    else:
        w = np.full(len(TINY_EDGES), 0.3, dtype=np.float32)
        g = synth.from_edges(n, TINY_EDGES, lt_weight=w)
        q = [int(np.floor(float(x) * 2**32)) for x in w]
        worlds = list(_lt_worlds(n, TINY_EDGES, q))
    N = 100_000
    pool = oracle.Pool(g, model, 21)
    pool.extend(N)
    off, verts = pool.concat()
    for S in [(0,), (2,), (1, 4), (3, 5)]:
        sigma = 0.0
        for pr, live in worlds:
            out = [[] for _ in range(n)]
            for (u, v) in live:
                out[u].append(v)
            sigma += pr * _forward_reach(n, out, S)
        hits = np.array([bool(set(verts[off[j]:off[j + 1]].tolist()) & set(S)) for j in range(N)])
        est = n * hits.mean()
        se = n * np.sqrt(hits.mean() * (1 - hits.mean()) / N)
        assert abs(est - sigma) <= 4 * se + 1e-9, (S, est, sigma)


def test_star_and_path_closed_forms():
    # star centre 0 -> leaves 1..L, p = 1: R(leaf) = {leaf, 0}, R(0) = {0}
    L = 9
    g = synth.from_edges(L + 1, [(0, i) for i in range(1, L + 1)], prob=[1.0] * L)
    pool = oracle.Pool(g, IC, 3)
    pool.extend(2000)
    for j in range(2000):
        s = pool.set(j).tolist()
        assert s == [0] or (len(s) == 2 and s[0] == 0)
    # path v0 -> v1 -> ... -> v_{L-1}, p = 1: R(v_i) = {v_0..v_i}
    P = 12
    g = synth.from_edges(P, [(i, i + 1) for i in range(P - 1)], prob=[1.0] * (P - 1))
    pool = oracle.Pool(g, IC, 4)
    pool.extend(2000)
    for j in range(2000):
        s = pool.set(j).tolist()
        assert s == list(range(len(s)))
    # LT with weight 1 on the path gives the same sets as IC with p = 1 (the
    # fixed-point weight is 1 - 2^-32, so this holds unless a draw is 2^32 - 1)
    gl = synth.from_edges(P, [(i, i + 1) for i in range(P - 1)], lt_weight=[1.0] * (P - 1))
    pl = oracle.Pool(gl, LT, 4)
    pl.extend(2000)
    for j in range(2000):
        assert pl.set(j).tolist() == pool.set(j).tolist()
    # p = 0: R = {root}
    g0 = synth.from_edges(P, [(i, i + 1) for i in range(P - 1)], prob=[0.0] * (P - 1))
    p0 = oracle.Pool(g0, IC, 5)
    p0.extend(3000)
    assert all(len(p0.set(j)) == 1 for j in range(3000))


def test_roots_uniform():
    n = 37
    g = synth.from_edges(n, [], prob=[])
    pool = oracle.Pool(g, IC, 99)
    N = 100_000
    pool.extend(N)
    off, verts = pool.concat()
    assert np.all(np.diff(off) == 1)
    counts = np.bincount(verts, minlength=n)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_sets_sorted_unique_and_contain_root():
    g = synth.WORKLOADS["ic_rmat4k"].graph()
    pool = oracle.Pool(g, IC, 7)
    pool.extend(3000)
    off, verts = pool.concat()
    for j in range(3000):
        s = verts[off[j]:off[j + 1]]
        assert len(s) >= 1
        assert np.all(np.diff(s.astype(np.int64)) > 0)
        assert oracle.rr_set(g, IC, 7, 0, j).tolist() == s.tolist()


def test_validation():
    g = synth.from_edges(3, [(0, 1), (2, 1)], prob=[0.5, 1.5])
    assert oracle.validate(g, IC) == -1
    g = synth.from_edges(3, [(0, 1), (2, 1)], lt_weight=[0.75, 0.5])
    assert oracle.validate(g, LT) == -2
    g = synth.from_edges(3, [(0, 1), (2, 1)], lt_weight=[0.5, 0.5])
    assert oracle.validate(g, LT) == 0
