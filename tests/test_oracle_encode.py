"""Pins the oracle's codebook, encoder and decoder.

- Huffman (1952) optimality: Kraft equality, the entropy bounds, and minimum
  total cost against every admissible length vector on small alphabets.
- Canonical assignment against RFC 1951 Section 3.2.2's worked example.
- Byte layout of one encoded set worked by hand from that codebook.
- Lossless round trips (Section 4.2.2: the copy array keeps uncoded vertices,
  so the encoding "preserves the exact information"), for Huffman and bitmap
  (Section 4.2.3) sets, including the density cut of Section 3.2.
- Skewness and density (Eq. (2)) against scipy.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import synth
from conftest import read_golden


def _kraft(lens):
    return sum(2.0 ** -int(l) for l in lens)


@pytest.mark.parametrize("seed", range(20))
def test_huffman_kraft_and_entropy(seed):
    rng = np.random.default_rng(seed)
    ns = int(rng.integers(2, 300))
    f = rng.integers(1, 1000, size=ns).astype(np.uint64)
    lens = oracle.huffman_lengths(f)
    assert abs(_kraft(lens) - 1.0) < 1e-12
    p = f / f.sum()
    H = -(p * np.log2(p)).sum()
    avg = (p * lens).sum()
    assert H - 1e-12 <= avg < H + 1


def _min_cost_bruteforce(f):
    """Minimum sum f_i l_i over length vectors with Kraft sum exactly 1."""
    ns = len(f)
    best = None
    for lens in itertools.product(range(1, ns), repeat=ns):
        if sum(2.0 ** -l for l in lens) != 1.0:
            continue
        c = sum(a * b for a, b in zip(f, lens))
        best = c if best is None else min(best, c)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_huffman_optimal_small(seed):
    rng = np.random.default_rng(100 + seed)
    ns = int(rng.integers(2, 7))
    f = rng.integers(1, 20, size=ns).tolist()
    lens = oracle.huffman_lengths(f)
    assert sum(a * int(b) for a, b in zip(f, lens)) == _min_cost_bruteforce(f)


def test_huffman_single_symbol_and_length_limit():
    assert oracle.huffman_lengths([5]).tolist() == [1]
    # Fibonacci weights give a maximally deep tree: 40 symbols -> depth 39 > 32
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    lens = oracle.huffman_lengths(fib)
    assert lens.max() <= 32
    assert abs(_kraft(lens) - 1.0) < 1e-12
    # heavier symbols never get longer codes
    order = np.argsort(fib, kind="stable")
    assert np.all(np.diff(lens[order].astype(np.int64)) <= 0)


def test_huffman_tie_rules_and_rescale_worked_cases():
    """Cases worked by hand under the codebook reading (Section 4.2.2): the
    leaf-first tie rule, the (f, id) symbol order and the ceil(f/2) rescale
    each decide one of them, so changing any of the three fails here."""
    rows = read_golden("huffman_ties.txt")
    assert len(rows) == 6
    for fr, lr in zip(rows[0::2], rows[1::2]):
        f = [int(x) for x in fr.split()[1:]]
        want = [int(x) for x in lr.split()[1:]]
        assert oracle.huffman_lengths(f).tolist() == want, f[:4]
    # the Fibonacci weights need the rescale: the partial sums stay below the
    # next-but-one leaf (F1 + ... + Fi = F(i+2) - 1), so the first build is a
    # chain in which v0 and v1 sit 33 deep
    fib = [int(x) for x in rows[4].split()[1:]]
    assert all(sum(fib[:i + 1]) == fib[i + 2] - 1 for i in range(32))
    assert abs(_kraft([int(x) for x in rows[5].split()[1:]]) - 1.0) < 1e-12


def test_canonical_rfc1951():
    d = {r.split()[0]: r.split()[1:] for r in read_golden("rfc1951_canonical.txt")}
    lengths = [int(x) for x in d["lengths"]]
    codes, ranks = oracle.canonical(lengths)
    for L, c, want in zip(lengths, codes, d["codes"]):
        assert format(int(c), f"0{L}b") == want
    # rank order is (length, symbol)
    assert sorted(range(8), key=lambda i: ranks[i]) == sorted(range(8), key=lambda i: (lengths[i], i))


def test_encode_bytes_by_hand():
    """Codebook of RFC 1951's example over 10 vertices (8 and 9 uncoded).
    Set {0 (A), 5 (F), 7 (H), 9} with cut 2 (2*4 <= 10, so Huffman): rank order
    F, A, H -> bits 00 010 1111 = 000101111 -> bytes 0x17 0x80 (MSB first, zero
    pad); copy array [9]."""
    lengths = [3, 3, 3, 3, 3, 2, 4, 4, 0, 0]
    cb = oracle.Codebook.from_lengths(lengths)
    enc = oracle.encode_set(cb, 2, [0, 5, 7, 9])
    assert enc["kind"] == 0 and enc["n_coded"] == 3 and enc["n_raw"] == 1
    assert enc["code_bits"] == 9
    assert enc["bytes"] == bytes([0x17, 0x80])
    assert enc["raw"].tolist() == [9]
    assert oracle.decode_set(cb, enc).tolist() == [0, 5, 7, 9]
    # a 32-bit-aligned bitmap: set {1, 3, 33} over n=40 with cut 32 (32*3 > 40)
    cb2 = oracle.Codebook.from_lengths([0] * 40)
    enc = oracle.encode_set(cb2, 32, [1, 3, 33])
    assert enc["kind"] == 1
    assert enc["bitmap"].tolist() == [0b1010, 0b10]


def test_density_cut_equality_stays_huffman():
    n = 64
    cb = oracle.Codebook.from_lengths([6] * n)
    assert oracle.encode_set(cb, 32, [1, 2])["kind"] == 0       # 32*2 = 64 = n
    assert oracle.encode_set(cb, 32, [1, 2, 3])["kind"] == 1    # 96 > 64


@pytest.mark.parametrize("seed", range(10))
def test_round_trip_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(50, 3000))
    freq = rng.integers(0, 50, size=n).astype(np.uint32)
    freq[rng.random(n) < 0.3] = 0  # uncoded vertices
    cb = oracle.Codebook(n, freq)
    assert cb.n_coded == int((freq > 0).sum())
    for _ in range(50):
        size = int(rng.integers(1, n // 10 + 3))
        s = np.unique(rng.integers(0, n, size=size)).astype(np.uint32)
        for cut in (1, 32, 10**9):
            enc = oracle.encode_set(cb, cut, s)
            assert enc["kind"] == (1 if cut * len(s) > n else 0)
            assert oracle.decode_set(cb, enc).tolist() == s.tolist()


def test_round_trip_pool_and_warmup():
    w = synth.WORKLOADS["ic_rmat4k"]
    g = w.graph()
    pool = oracle.Pool(g, oracle.IC, w.rr_seed)
    pool.extend(4000)
    W = 500
    f = pool.warmup_freq(W, 32)
    sizes = pool.sizes(0, W)
    elig = sizes[32 * sizes <= g.n]
    assert int(f.sum()) == int(elig.sum())
    cb = oracle.Codebook(g.n, f)
    nbits = 0
    nverts = 0
    for j in range(4000):
        s = pool.set(j)
        enc = oracle.encode_set(cb, 32, s)
        assert oracle.decode_set(cb, enc).tolist() == s.tolist()
        nverts += len(s)
        nbits += enc["code_bits"]
    assert nbits > 0


def test_size_stats_against_scipy():
    rng = np.random.default_rng(1)
    sizes = (rng.pareto(1.5, size=5000) * 10 + 1).astype(np.uint64)
    sk, de = oracle.size_stats(sizes, 100000)
    assert abs(sk - stats.skew(sizes.astype(np.float64), bias=True)) < 1e-9 * max(1, abs(sk))
    assert abs(de - sizes.sum() / (5000 * 100000)) < 1e-15
