"""Pins the oracle's greedy max coverage and IMM bounds.

- The paper's worked Bitmax example (Section 4.3.2, Eq. (3)) fixes counts, the
  first two choices of u* and the coverage.
- Brute force: greedy by recounting marginal gains from scratch (the per-
  iteration recount of Algorithms 2 and 3) on random small instances, and the
  (1 - 1/e) guarantee against the best k-subset found by enumeration.
- IMM's theta_i (Eq. (1), Section 2.2) against hand-worked values, and against
  the paper's printed form of Eq. (1) evaluated with scipy's log-gamma.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import special

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
