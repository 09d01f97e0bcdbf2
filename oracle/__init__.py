"""ORACLE -- test infrastructure only.

Python wrapper over ``oracle.cpp``: a plain CPU statement of the RR-set IMM
method (uncompressed sorted sets, greedy max coverage, IMM bounds in FP64) and a
separate Huffman/bitmap encoder and decoder.  Only ``tests/``, the smoke check
and the benchmark's CPU-baseline leg may import this package; the product path
never does, and the two share no code.

The library is compiled on first use with the host's g++ into
``oracle/_build/liboracle.so`` (``-O2 -fopenmp -ffp-contract=off``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

IC, LT = 0, 1
NONE = 0xFFFFFFFF


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("m", ctypes.c_uint64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("prob", ctypes.c_void_p), ("lt_weight", ctypes.c_void_p)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P, U32, U64, D, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
    sig = {
        "orc_philox": (None, [P, P, P]),
        "orc_philox_batch": (None, [U64, P, P, P]),
        "orc_validate": (I, [P, I]),
        "orc_rr_set": (U64, [P, I, U64, U32, U64, P, U64]),
        "orc_pool_new": (P, [P, I, U64, U32]),
        "orc_pool_free": (None, [P]),
        "orc_pool_extend": (I, [P, U64, I]),
        "orc_pool_count": (U64, [P]),
        "orc_pool_set_size": (U64, [P, U64]),
        "orc_pool_get_set": (None, [P, U64, P]),
        "orc_pool_sizes": (None, [P, U64, U64, P]),
        "orc_pool_concat": (None, [P, U64, U64, P]),
        "orc_pool_edge_counts": (None, [P, P, P]),
        "orc_pool_greedy": (I, [P, U64, U32, P, P, P]),
        "orc_greedy_lists": (I, [U32, U64, P, P, U32, P, P, P]),
        "orc_imm_params": (I, [U32, U32, D, D, P]),
        "orc_imm_pool": (I, [P, U32, D, D, I, P, P, P, P, P, P, P, P]),
        "orc_imm_pool_fresh": (I, [P, U32, D, D, I, I, P, P, P, P, P, P, P, P]),
        "orc_size_stats": (None, [P, U64, U32, P, P]),
        "orc_pool_warmup_freq": (I, [P, U64, U32, P]),
        "orc_huffman_lengths": (I, [U64, P, P]),
        "orc_codebook": (U32, [U32, P, P, P, P]),
        "orc_canonical": (U32, [U64, P, P, P]),
        "orc_encode_set": (I, [U32, U32, P, P, P, P, U64, P, P, P, P, U64, P, P, P, U64]),
        "orc_decode_set": (ctypes.c_int64, [U32, P, P, U32, U32, U64, P, P, U32, P, P]),
        "orc_pool_greedy_recount": (I, [P, U64, U32, P, P, P]),
        "orc_pool_scheme": (I, [P, U64, P]),
        "orc_pool_bitmax_tiles": (I, [P, U64, P]),
        "orc_bitmax_query": (I, [U32, U64, P, U32, P, P, P]),
        "orc_huffmax_query": (I, [U32, P, P, U64, P, P, P, P, P, P, P, P, P, P, U32, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


# ---------------------------------------------------------------------------
def philox(ctr, key):
    """Philox4x32-10 of counters ctr (shape [N,4] or [4]) under key (k0, k1)."""
    c = _u32(np.atleast_2d(ctr))
    k = _u32(key)
    out = np.empty_like(c)
    _load().orc_philox_batch(c.shape[0], _p(c), _p(k), _p(out))
    return out if np.ndim(ctr) == 2 else out[0]


class OGraph:
    """Keeps the numpy arrays alive behind the C struct."""

    def __init__(self, g):
        self.n, self.m = int(g.n), int(g.m)
        self._rp = _u32(g.row_ptr)
        self._col = _u32(g.col) if g.m else np.zeros(1, np.uint32)
        self._prob = None if g.prob is None else np.ascontiguousarray(g.prob, dtype=np.float32)
        self._w = None if g.lt_weight is None else np.ascontiguousarray(g.lt_weight, dtype=np.float32)
        self.s = _Graph(self.n, self.m, self._rp.ctypes.data, self._col.ctypes.data,
                        None if self._prob is None else self._prob.ctypes.data,
                        None if self._w is None else self._w.ctypes.data)

    @property
    def ref(self):
        return ctypes.byref(self.s)


def validate(g, model: int) -> int:
    og = OGraph(g)
    return _load().orc_validate(og.ref, model)


def rr_set(g, model: int, seed: int, epoch: int, j: int) -> np.ndarray:
    og = OGraph(g)
    cap = og.n
    out = np.empty(cap, dtype=np.uint32)
    sz = _load().orc_rr_set(og.ref, model, seed, epoch, j, _p(out), cap)
    return out[:sz].copy()


class Pool:
    """RR sets [0, T) of one (graph, model, seed, epoch), sorted, uncompressed."""

    def __init__(self, g, model: int, seed: int, epoch: int = 0):
        self.g = OGraph(g)
        self.n = self.g.n
        self.h = _load().orc_pool_new(self.g.ref, model, seed, epoch)

    def __del__(self):
        if getattr(self, "h", None):
            _load().orc_pool_free(self.h)
            self.h = None

    def extend(self, T: int, nthreads: int = 0):
        _load().orc_pool_extend(self.h, T, nthreads)

    @property
    def T(self) -> int:
        return int(_load().orc_pool_count(self.h))

    def set(self, j: int) -> np.ndarray:
        sz = _load().orc_pool_set_size(self.h, j)
        out = np.empty(max(sz, 1), dtype=np.uint32)
        _load().orc_pool_get_set(self.h, j, _p(out))
        return out[:sz]

    def sizes(self, j0: int = 0, j1: int | None = None) -> np.ndarray:
        j1 = self.T if j1 is None else j1
        out = np.empty(max(j1 - j0, 1), dtype=np.uint64)
        _load().orc_pool_sizes(self.h, j0, j1, _p(out))
        return out[:j1 - j0]

    def concat(self, j0: int = 0, j1: int | None = None):
        """(offsets[T+1], verts) of sets [j0, j1)."""
        j1 = self.T if j1 is None else j1
        sz = self.sizes(j0, j1)
        off = np.zeros(len(sz) + 1, dtype=np.uint64)
        np.cumsum(sz, out=off[1:])
        verts = np.empty(max(int(off[-1]), 1), dtype=np.uint32)
        _load().orc_pool_concat(self.h, j0, j1, _p(verts))
        return off, verts[:int(off[-1])]

    def edge_counts(self):
        s, l = ctypes.c_uint64(), ctypes.c_uint64()
        _load().orc_pool_edge_counts(self.h, ctypes.byref(s), ctypes.byref(l))
        return s.value, l.value

    def greedy(self, T: int, k: int):
        seeds = np.empty(k, dtype=np.uint32)
        marg = np.empty(k, dtype=np.uint64)
        cov = ctypes.c_uint64()
        rc = _load().orc_pool_greedy(self.h, T, k, _p(seeds), _p(marg), ctypes.byref(cov))
        if rc != 0:
            raise ValueError("orc_pool_greedy: bad arguments")
        return seeds, marg, cov.value

    def imm(self, k: int, eps: float, ell: float, nthreads: int = 0, fresh_final: bool = False) -> dict:
        """IMM on this pool's sets; fresh_final draws the final phase's sets
        anew (ids [T_i, T_i + theta)) instead of reusing [0, theta)."""
        seeds = np.empty(k, dtype=np.uint32)
        marg = np.empty(k, dtype=np.uint64)
        infl, lb = ctypes.c_double(), ctypes.c_double()
        theta, cov = ctypes.c_uint64(), ctypes.c_uint64()
        rounds = ctypes.c_uint32()
        rT = np.zeros(64, dtype=np.uint64)
        rc = _load().orc_imm_pool_fresh(self.h, k, eps, ell, nthreads, int(bool(fresh_final)), _p(seeds), _p(marg),
                                        ctypes.byref(infl), ctypes.byref(theta), ctypes.byref(cov), ctypes.byref(lb),
                                        ctypes.byref(rounds), _p(rT))
        if rc != 0:
            raise ValueError("orc_imm_pool: bad arguments")
        return dict(seeds=seeds, marginal=marg, influence=infl.value, theta=theta.value,
                    covered=cov.value, lb=lb.value, rounds=rounds.value,
                    round_T=rT[:rounds.value + 1].copy())

    def greedy_recount(self, T: int, k: int):
        """Greedy with the table rebuilt every iteration (Algorithms 2 and 3)."""
        seeds = np.empty(k, dtype=np.uint32)
        marg = np.empty(k, dtype=np.uint64)
        cov = ctypes.c_uint64()
        if _load().orc_pool_greedy_recount(self.h, T, k, _p(seeds), _p(marg), ctypes.byref(cov)) != 0:
            raise ValueError("orc_pool_greedy_recount: bad arguments")
        return seeds, marg, cov.value

    def scheme(self, W: int):
        """(True for Bitmax / False for Huffmax, skewness of the warm-up sizes):
        Algorithm 1's Characterize over sets [0, W)."""
        sk = ctypes.c_double()
        r = _load().orc_pool_scheme(self.h, W, ctypes.byref(sk))
        if r < 0:
            raise ValueError("warm-up block larger than the pool")
        return bool(r), sk.value

    def bitmax_tiles(self, T: int) -> np.ndarray:
        """Vertex-major Bitmax tiles of sets [0, T): shape (ceil(T/32), n)."""
        nt = (T + 31) // 32
        out = np.empty(max(nt * self.n, 1), dtype=np.uint32)
        if _load().orc_pool_bitmax_tiles(self.h, T, _p(out)) != 0:
            raise ValueError("orc_pool_bitmax_tiles: bad arguments")
        return out[:nt * self.n].reshape(nt, self.n)

    def warmup_freq(self, W: int, cut: int = 32) -> np.ndarray:
        f = np.empty(self.n, dtype=np.uint32)
        if _load().orc_pool_warmup_freq(self.h, W, cut, _p(f)) != 0:
            raise ValueError("warm-up block larger than the pool")
        return f


def bitmax_query(tiles: np.ndarray, T: int, k: int):
    """Algorithm 3 (POPCOUNT, argmax, SUBTRACT) over vertex-major tiles of
    shape (ceil(T/32), n); the tiles are not modified."""
    t = np.ascontiguousarray(tiles, dtype=np.uint32).copy()
    n = t.shape[1]
    seeds = np.empty(k, dtype=np.uint32)
    marg = np.empty(k, dtype=np.uint64)
    cov = ctypes.c_uint64()
    if _load().orc_bitmax_query(n, T, _p(t), k, _p(seeds), _p(marg), ctypes.byref(cov)) != 0:
        raise ValueError("orc_bitmax_query: bad arguments")
    return seeds, marg, cov.value


def huffmax_query(cb: "Codebook", encs, k: int):
    """Algorithm 2 over encoded sets (dicts from encode_set)."""
    T = len(encs)
    kind = np.array([e["kind"] for e in encs], dtype=np.uint32)
    ncod = np.array([e["n_coded"] for e in encs], dtype=np.uint32)
    bits = np.array([e["code_bits"] for e in encs], dtype=np.uint64)
    nraw = np.array([e["n_raw"] for e in encs], dtype=np.uint32)
    blen = [len(e["bytes"]) for e in encs]
    boff = np.concatenate([[0], np.cumsum(blen)]).astype(np.uint64)
    roff = np.concatenate([[0], np.cumsum(nraw.astype(np.uint64))]).astype(np.uint64)
    words = (cb.n + 31) // 32
    bmoff = np.zeros(T, dtype=np.uint64)
    bms = []
    for j, e in enumerate(encs):
        bmoff[j] = words * len(bms)
        if e["kind"] == 1:
            bms.append(_u32(e["bitmap"]))
    by = np.frombuffer(b"".join(e["bytes"] for e in encs) + b"\0", dtype=np.uint8).copy()
    raw = np.concatenate([_u32(e["raw"]) for e in encs] + [np.zeros(1, np.uint32)])
    bm = np.concatenate(bms + [np.zeros(words, np.uint32)])
    seeds = np.empty(k, dtype=np.uint32)
    marg = np.empty(k, dtype=np.uint64)
    cov = ctypes.c_uint64()
    rc = _load().orc_huffmax_query(cb.n, _p(cb.len), _p(cb.code), T, _p(kind), _p(ncod), _p(bits), _p(boff[:T]),
                                   _p(by), _p(nraw), _p(roff[:T]), _p(raw), _p(bmoff), _p(bm), k, _p(seeds),
                                   _p(marg), ctypes.byref(cov))
    if rc != 0:
        raise ValueError("orc_huffmax_query: bad arguments or stream")
    return seeds, marg, cov.value


def greedy_lists(n: int, sets, k: int):
    off = np.zeros(len(sets) + 1, dtype=np.uint64)
    for i, s in enumerate(sets):
        off[i + 1] = off[i] + len(s)
    verts = _u32(np.concatenate([np.asarray(s, dtype=np.uint32) for s in sets]) if sets else np.zeros(1))
    if verts.size == 0:
        verts = np.zeros(1, np.uint32)
    seeds = np.empty(k, dtype=np.uint32)
    marg = np.empty(k, dtype=np.uint64)
    cov = ctypes.c_uint64()
    if _load().orc_greedy_lists(n, len(sets), _p(off), _p(verts), k, _p(seeds), _p(marg), ctypes.byref(cov)):
        raise ValueError("orc_greedy_lists: bad arguments")
    return seeds, marg, cov.value


def imm_params(n: int, k: int, eps: float, ell: float) -> dict:
    out = np.empty(7, dtype=np.float64)
    if _load().orc_imm_params(n, k, eps, ell, _p(out)) != 0:
        raise ValueError("bad IMM parameters")
    return dict(zip(["eps_p", "ell_p", "lnC", "lambda_p", "lambda_star", "alpha", "beta"], out.tolist()))


def size_stats(sizes, n: int):
    s = np.ascontiguousarray(sizes, dtype=np.uint64)
    sk, de = ctypes.c_double(), ctypes.c_double()
    _load().orc_size_stats(_p(s), len(s), n, ctypes.byref(sk), ctypes.byref(de))
    return sk.value, de.value


def huffman_lengths(f) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.uint64)
    out = np.empty(max(len(f), 1), dtype=np.uint32)
    _load().orc_huffman_lengths(len(f), _p(f), _p(out))
    return out[:len(f)]


def canonical(lengths):
    """Canonical codes and ranks for symbols 0..ns-1 with the given lengths."""
    ln = _u32(lengths)
    code = np.empty(max(len(ln), 1), dtype=np.uint32)
    rank = np.empty(max(len(ln), 1), dtype=np.uint32)
    _load().orc_canonical(len(ln), _p(ln), _p(code), _p(rank))
    return code[:len(ln)], rank[:len(ln)]


class Codebook:
    """Per-vertex (len, code, rank); built from warm-up frequencies, or given
    lengths directly (``Codebook.from_lengths``)."""

    def __init__(self, n: int, freq=None):
        self.n = n
        self.len = np.zeros(n, dtype=np.uint32)
        self.code = np.zeros(n, dtype=np.uint32)
        self.rank = np.full(n, NONE, dtype=np.uint32)
        self.n_coded = 0
        if freq is not None:
            freq = _u32(freq)
            self.n_coded = int(_load().orc_codebook(n, _p(freq), _p(self.len), _p(self.code), _p(self.rank)))

    @classmethod
    def from_lengths(cls, lengths):
        cb = cls(len(lengths))
        cb.len = _u32(lengths).copy()
        cb.code, cb.rank = canonical(cb.len)
        cb.n_coded = int((cb.len > 0).sum())
        return cb


def encode_set(cb: Codebook, cut: int, s) -> dict:
    s = _u32(s)
    n = cb.n
    kind, ncod, nraw = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    bits = ctypes.c_uint64()
    cap_bytes = 4 * len(s) + 8
    by = np.zeros(cap_bytes, dtype=np.uint8)
    raw = np.zeros(max(len(s), 1), dtype=np.uint32)
    words = (n + 31) // 32
    bm = np.zeros(words, dtype=np.uint32)
    rc = _load().orc_encode_set(n, cut, _p(cb.len), _p(cb.code), _p(cb.rank), _p(s), len(s), ctypes.byref(kind),
                                ctypes.byref(ncod), ctypes.byref(bits), _p(by), cap_bytes, _p(raw),
                                ctypes.byref(nraw), _p(bm), words)
    if rc != 0:
        raise ValueError("encode buffer too small")
    if kind.value == 1:
        return dict(kind=1, size=len(s), n_coded=0, n_raw=0, code_bits=0, bytes=b"", raw=np.zeros(0, np.uint32),
                    bitmap=bm)
    nb = (bits.value + 7) // 8
    return dict(kind=0, size=len(s), n_coded=ncod.value, n_raw=nraw.value, code_bits=bits.value,
                bytes=by[:nb].tobytes(), raw=raw[:nraw.value].copy(), bitmap=None)


def decode_set(cb: Codebook, enc: dict) -> np.ndarray:
    n = cb.n
    out = np.empty(n, dtype=np.uint32)
    by = np.frombuffer(enc["bytes"], dtype=np.uint8).copy() if enc["bytes"] else np.zeros(1, np.uint8)
    raw = _u32(enc["raw"]) if len(enc["raw"]) else np.zeros(1, np.uint32)
    bm = _u32(enc["bitmap"]) if enc["bitmap"] is not None else np.zeros(1, np.uint32)
    sz = _load().orc_decode_set(n, _p(cb.len), _p(cb.code), enc["kind"], enc["n_coded"], enc["code_bits"],
                                _p(by), _p(raw), enc["n_raw"], _p(bm), _p(out))
    if sz < 0:
        raise ValueError("malformed stream")
    return out[:sz].copy()
