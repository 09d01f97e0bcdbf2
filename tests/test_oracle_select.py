"""Pins the oracle's greedy max coverage and IMM bounds.

- The paper's worked Bitmax example (Section 4.3.2, Eq. (3)) fixes counts, the
  first two choices of u* and the coverage.
- Brute force: greedy by recounting marginal gains from scratch (the per-
  iteration recount of Algorithms 2 and 3) on random small instances, and the
  (1 - 1/e) guarantee against the best k-subset found by enumeration.
- IMM's theta_i (Eq. (1), Section 2.2) against hand-worked values, and against
  the paper's printed form of Eq. (1) evaluated with scipy's log-gamma.
- The paper-literal selection modes -- Algorithm 3's POPCOUNT / SUBTRACT query
  over vertex-major tiles, Algorithm 2's decode query over encoded sets, the
  per-iteration recount -- against Eq. (3)'s worked example and the greedy;
  Algorithm 1's scheme switch against closed-form size distributions.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle
import synth
from conftest import read_golden


def _golden_bitmax():
    rows = read_golden("bitmax_example.txt")
    d = {}
    for r in rows:
        key, val = r.split(maxsplit=1)
        d.setdefault(key, []).append(val)
    return d


def test_bitmax_worked_example():
    d = _golden_bitmax()
    mat = np.array([[int(c) for c in row] for row in d["matrix"]])
    n, T = mat.shape
    sets = [np.nonzero(mat[:, j])[0].tolist() for j in range(T)]
    counts = [int(x) for x in d["counts"][0].split()]
    assert mat.sum(axis=1).tolist() == counts
    seeds, marg, cov = oracle.greedy_lists(n, sets, 2)
    assert seeds.tolist() == [int(x) for x in d["seeds"][0].split()]
    assert marg.tolist() == [int(x) for x in d["marginal"][0].split()]
    assert cov == T
    # the rows after subtracting u* = v1 (SUBTRACT = v AND NOT u*)
    after = np.array([[int(c) for c in row] for row in d["after"]])
    u = mat[seeds[0]]
    assert np.array_equal(mat & (1 - u)[None, :], after)
    # the paper's own form of SUBTRACT, v AND (v XOR u*), is the same
    assert np.array_equal(mat & (mat ^ u[None, :]), after)
    # greedy over the remaining sets picks the row with the most ones
    assert int(np.argmax(after.sum(axis=1))) == seeds[1]


def _greedy_recount(n, sets, k):
    chosen, alive, marg = [], [True] * len(sets), []
    for _ in range(k):
        best, best_gain = None, -1
        for v in range(n):
            if v in chosen:
                continue
            gain = sum(1 for j, s in enumerate(sets) if alive[j] and v in s)
            if gain > best_gain:
                best, best_gain = v, gain
        chosen.append(best)
        marg.append(best_gain)
        for j, s in enumerate(sets):
            if alive[j] and best in s:
                alive[j] = False
    return chosen, marg


@pytest.mark.parametrize("seed", range(40))
def test_greedy_matches_recount_and_bound(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    T = int(rng.integers(1, 13))
    k = int(rng.integers(1, n + 1))
    sets = [sorted(set(rng.integers(0, n, size=int(rng.integers(1, n + 1))).tolist())) for _ in range(T)]
    seeds, marg, cov = oracle.greedy_lists(n, sets, k)
    ref_seeds, ref_marg = _greedy_recount(n, [set(s) for s in sets], k)
    assert seeds.tolist() == ref_seeds
    assert marg.tolist() == ref_marg
    assert cov == sum(ref_marg)
    opt = max(sum(1 for s in sets if set(s) & set(S)) for S in itertools.combinations(range(n), k))
    assert cov >= (1 - 1 / math.e) * opt - 1e-9


def test_greedy_zero_counts_take_lowest_unselected():
    # one set {3}: after it is covered, every count is zero, so the lowest ids
    # not yet chosen follow
    seeds, marg, cov = oracle.greedy_lists(6, [[3]], 4)
    assert seeds.tolist() == [3, 0, 1, 2]
    assert marg.tolist() == [1, 0, 0, 0]


def test_theta_hand_values():
    d = {r.split()[0]: r.split()[1:] for r in read_golden("imm_theta_rmat4k.txt")}
    T = [int(x) for x in d["T"]]
    prm = oracle.imm_params(4096, 10, 0.5, 1.0)
    got = [math.ceil(prm["lambda_p"] / (4096 / 2 ** i)) for i in range(1, 6)]
    assert got == T
    assert abs(prm["lambda_star"] / 4096 - float(d["lambda_star_over_n"][0])) < 0.1


@pytest.mark.parametrize("n,k,eps,ell", [(4096, 10, 0.5, 1.0), (1 << 20, 50, 0.5, 1.0),
                                         (1 << 22, 100, 0.3, 1.0), (41652230, 100, 0.5, 1.0),
                                         (1000, 1, 0.1, 2.0)])
def test_theta_paper_form(n, k, eps, ell):
    """Eq. (1) as printed, in eps (not eps'), with log C(n,k) from log-gamma."""
    prm = oracle.imm_params(n, k, eps, ell)
    ellp = ell * (1 + math.log(2) / math.log(n))
    lnc = special.gammaln(n + 1) - special.gammaln(k + 1) - special.gammaln(n - k + 1)
    for i in range(1, 6):
        th = (2 + 2 * math.sqrt(2) / 3 * eps) * (lnc + ellp * math.log(n) + math.log(math.log2(n))) * 2 ** i / (
            2 * eps * eps)
        assert abs(prm["lambda_p"] / (n / 2 ** i) - th) <= 1e-9 * th
    # lambda* of IMM with (1 - 1/e) alpha + beta
    a = math.sqrt(ellp * math.log(n) + math.log(2))
    b = math.sqrt((1 - 1 / math.e) * (lnc + ellp * math.log(n) + math.log(2)))
    lam = 2 * n * ((1 - 1 / math.e) * a + b) ** 2 / eps ** 2
    assert abs(prm["lambda_star"] - lam) <= 1e-9 * lam


def test_imm_invariants_tiny():
    w = synth.WORKLOADS["ic_rmat4k"]
    g = w.graph()
    pool = oracle.Pool(g, oracle.IC, w.rr_seed)
    r = pool.imm(w.k, w.eps, w.ell)
    n = g.n
    prm = oracle.imm_params(n, w.k, w.eps, w.ell)
    # the estimation rounds double, the final theta covers lambda*/LB
    rT = r["round_T"].tolist()
    golden_T = [int(x) for x in dict((l.split()[0], l.split()[1:]) for l in read_golden("imm_theta_rmat4k.txt"))["T"]]
    assert rT[:-1] == golden_T[:r["rounds"]]
    assert r["theta"] == max(rT[-2], math.ceil(prm["lambda_star"] / r["lb"]))
    assert r["covered"] == int(r["marginal"].sum())
    assert r["influence"] == n * r["covered"] / r["theta"]
    # the greedy on the same prefix gives the same answer
    s2, m2, c2 = pool.greedy(r["theta"], w.k)
    assert s2.tolist() == r["seeds"].tolist() and c2 == r["covered"]
    # marginal gains never increase (submodularity of coverage)
    assert np.all(np.diff(r["marginal"].astype(np.int64)) <= 0)


def test_imm_estimate_close_to_brute_force_sigma():
    """On a tiny graph the IMM influence estimate of the chosen seeds is within
    eps of sigma(S) computed over all live-edge worlds."""
    n = 8
    edges = [(0, 1), (0, 2), (1, 3), (2, 3), (3, 4), (4, 5), (5, 6), (6, 7), (7, 0), (2, 6), (1, 5), (3, 7)]
    probs = np.array([0.7, 0.6, 0.5, 0.4, 0.8, 0.3, 0.6, 0.5, 0.2, 0.4, 0.3, 0.5], dtype=np.float32)
    g = synth.from_edges(n, edges, prob=probs)
    pool = oracle.Pool(g, oracle.IC, 5)
    r = pool.imm(2, 0.3, 1.0)
    S = r["seeds"].tolist()
    p_exact = [np.ceil(float(p) * 2**24) / 2**24 for p in probs]
    sigma = 0.0
    for mask in range(1 << len(edges)):
        pr = 1.0
        out = [[] for _ in range(n)]
        for i, (u, v) in enumerate(edges):
            if mask >> i & 1:
                pr *= p_exact[i]
                out[u].append(v)
            else:
                pr *= 1 - p_exact[i]
        seen, stack = set(S), list(S)
        while stack:
            u = stack.pop()
            for v in out[u]:
                if v not in seen:
                    seen.add(v)
                    stack.append(v)
        sigma += pr * len(seen)
    assert abs(r["influence"] - sigma) <= 0.3 * sigma


# ---------------------------------------------------------------------------
# paper-literal selection modes: Algorithm 3 over vertex-major tiles, Algorithm
# 2 over encoded sets, and the per-iteration recount, against the worked
# example of Eq. (3) and against the plain greedy
# ---------------------------------------------------------------------------
def _tiles_from_matrix(mat):
    n, T = mat.shape
    tiles = np.zeros(((T + 31) // 32, n), dtype=np.uint32)
    for v in range(n):
        for s in range(T):
            if mat[v, s]:
                tiles[s // 32, v] |= np.uint32(1 << (s % 32))
    return tiles


def test_bitmax_query_worked_example():
    d = _golden_bitmax()
    mat = np.array([[int(c) for c in row] for row in d["matrix"]])
    n, T = mat.shape
    seeds, marg, cov = oracle.bitmax_query(_tiles_from_matrix(mat), T, 2)
    assert seeds.tolist() == [int(x) for x in d["seeds"][0].split()]
    assert marg.tolist() == [int(x) for x in d["marginal"][0].split()]
    assert cov == T
    # k = 1 leaves exactly the SUBTRACT rows of Eq. (3): their popcounts pick v5
    after = np.array([[int(c) for c in row] for row in d["after"]])
    s1, m1, _ = oracle.bitmax_query(_tiles_from_matrix(mat), T, 1)
    assert s1.tolist() == [0] and m1.tolist() == [int(mat[0].sum())]
    assert int(np.argmax(after.sum(axis=1))) == int(seeds[1])


def _small_pool(seed, T, p=0.1):
    g = synth.rmat(512, 4096, seed)
    g.prob = synth.ic_uniform(g, seed, p)
    pool = oracle.Pool(g, oracle.IC, seed)
    pool.extend(T)
    return g, pool


@pytest.mark.parametrize("seed,T,k", [(3, 100, 8), (4, 257, 20), (5, 64, 64)])
def test_bitmax_tiles_layout(seed, T, k):
    g, pool = _small_pool(seed, T)
    tiles = pool.bitmax_tiles(T)
    assert tiles.shape == ((T + 31) // 32, g.n)
    for j in range(T):
        members = set(pool.set(j).tolist())
        col = (tiles[j // 32] >> np.uint32(j % 32)) & np.uint32(1)
        assert set(np.nonzero(col)[0].tolist()) == members
    # columns past T are zero
    if T % 32:
        assert not np.any(tiles[-1] >> np.uint32(T % 32))


@pytest.mark.parametrize("seed,T,k,p", [(3, 100, 8, 0.1), (4, 257, 20, 0.1), (5, 64, 64, 0.1), (6, 300, 12, 0.3)])
def test_literal_modes_equal_greedy(seed, T, k, p):
    g, pool = _small_pool(seed, T, p)
    ref = pool.greedy(T, k)
    for got in (pool.greedy_recount(T, k), oracle.bitmax_query(pool.bitmax_tiles(T), T, k)):
        assert got[0].tolist() == ref[0].tolist()
        assert got[1].tolist() == ref[1].tolist() and got[2] == ref[2]
    # Algorithm 2 over the encoded sets (codebook from the first quarter), for
    # the per-set cut and for Huffmax (every set coded)
    cb = oracle.Codebook(g.n, pool.warmup_freq(T // 4, 0))
    for cut in (32, 0):
        encs = [oracle.encode_set(cb, cut, pool.set(j)) for j in range(T)]
        got = oracle.huffmax_query(cb, encs, k)
        assert got[0].tolist() == ref[0].tolist()
        assert got[1].tolist() == ref[1].tolist() and got[2] == ref[2]


def test_scheme_switch_closed_forms():
    """Algorithm 1's Characterize: Bitmax iff the warm-up sizes' skewness is
    negative.  Star centre -> leaves with p = 1: a leaf's RR set is {leaf,
    centre} (size 2) and the centre's is {centre} (size 1), so the sizes have
    a long left tail (negative skew): Bitmax.  p = 0: every set is its root,
    the sizes have no spread (skewness 0): Huffmax."""
    n = 64
    star = synth.from_edges(n, [(0, v) for v in range(1, n)], prob=[1.0] * (n - 1))
    pool = oracle.Pool(star, oracle.IC, 3)
    pool.extend(400)
    sizes = pool.sizes(0, 400)
    assert set(sizes.tolist()) == {1, 2} and (sizes == 1).any()
    bitmax, sk = pool.scheme(400)
    assert bitmax and sk < 0
    assert abs(sk - stats.skew(sizes.astype(np.float64), bias=True)) < 1e-12
    none = synth.from_edges(n, [(0, v) for v in range(1, n)], prob=[0.0] * (n - 1))
    pool0 = oracle.Pool(none, oracle.IC, 3)
    pool0.extend(100)
    assert pool0.scheme(100) == (False, 0.0)
    # a skewed pool (small sets with a few large ones) keeps Huffmax
    g, pool2 = _small_pool(7, 400, 0.1)
    bm2, sk2 = pool2.scheme(400)
    s2 = pool2.sizes(0, 400).astype(np.float64)
    assert abs(sk2 - stats.skew(s2, bias=True)) < 1e-9 * max(1.0, abs(sk2))
    assert bm2 == (sk2 < 0)


def test_imm_fresh_final_phase():
    """IMM with fresh final-phase sets: the estimation rounds and LB are those
    of the reusing form, the final phase takes theta = ceil(lambda*/LB) new sets
    (ids from T_i on), and greedy on exactly those sets gives the seeds."""
    w = synth.WORKLOADS["ic_rmat4k"]
    g = w.graph()
    reuse = oracle.Pool(g, oracle.IC, w.rr_seed).imm(w.k, w.eps, w.ell)
    pool = oracle.Pool(g, oracle.IC, w.rr_seed)
    fresh = pool.imm(w.k, w.eps, w.ell, fresh_final=True)
    prm = oracle.imm_params(g.n, w.k, w.eps, w.ell)
    assert fresh["rounds"] == reuse["rounds"] and fresh["lb"] == reuse["lb"]
    Ti = int(fresh["round_T"][fresh["rounds"] - 1])
    theta = math.ceil(prm["lambda_star"] / fresh["lb"])
    assert fresh["theta"] == theta and int(fresh["round_T"][fresh["rounds"]]) == Ti + theta
    assert fresh["influence"] == g.n * fresh["covered"] / theta
    # greedy over the fresh sets only (written out with the list greedy)
    sets = [pool.set(j) for j in range(Ti, Ti + theta)]
    s2, m2, c2 = oracle.greedy_lists(g.n, sets, w.k)
    assert s2.tolist() == fresh["seeds"].tolist() and m2.tolist() == fresh["marginal"].tolist()
    assert c2 == fresh["covered"]


def test_imm_fresh_estimate_close_to_brute_force_sigma():
    n = 8
    edges = [(0, 1), (0, 2), (1, 3), (2, 3), (3, 4), (4, 5), (5, 6), (6, 7), (7, 0), (2, 6), (1, 5), (3, 7)]
    probs = np.array([0.7, 0.6, 0.5, 0.4, 0.8, 0.3, 0.6, 0.5, 0.2, 0.4, 0.3, 0.5], dtype=np.float32)
    g = synth.from_edges(n, edges, prob=probs)
    r = oracle.Pool(g, oracle.IC, 5).imm(2, 0.3, 1.0, fresh_final=True)
    S = r["seeds"].tolist()
    p_exact = [np.ceil(float(p) * 2**24) / 2**24 for p in probs]
    sigma = 0.0
    for mask in range(1 << len(edges)):
        pr = 1.0
        out = [[] for _ in range(n)]
        for i, (u, v) in enumerate(edges):
            if mask >> i & 1:
                pr *= p_exact[i]
                out[u].append(v)
            else:
                pr *= 1 - p_exact[i]
        seen, stack = set(S), list(S)
        while stack:
            u = stack.pop()
            for v in out[u]:
                if v not in seen:
                    seen.add(v)
                    stack.append(v)
        sigma += pr * len(seen)
    assert abs(r["influence"] - sigma) <= 0.3 * sigma
