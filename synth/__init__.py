"""Seeded synthetic workloads for RR-set influence maximization.

The paper's graphs (Table 4) are not available, so the workloads are directed
R-MAT graphs of matching size and skew, plus edge parameters for the two
diffusion models of Section 2.1 (IC probabilities, LT in-weights).  Nothing
here computes any part of the method: both the CPU oracle and the CUDA path
take their inputs from this module, and from nowhere else.

The C helpers are compiled on first use with the host's gcc into
``synth/_build/libsynth.so``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library (portable C, no target-specific flags)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.synth_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, P, P]
        lib.synth_rmat.restype = ctypes.c_int
        lib.synth_ic_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_float, P]
        lib.synth_weighted_cascade.argtypes = [ctypes.c_uint32, P, P]
        lib.synth_lt_weights.argtypes = [ctypes.c_uint32, P, ctypes.c_uint64, P]
        lib.synth_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


@dataclasses.dataclass
class Graph:
    """Transposed CSR: in-edges of v are col[row_ptr[v]:row_ptr[v+1]]."""
    n: int
    m: int
    row_ptr: np.ndarray  # uint32 [n+1]
    col: np.ndarray      # uint32 [m]
    prob: np.ndarray | None = None       # float32 [m], IC activation probability of each edge
    lt_weight: np.ndarray | None = None  # float32 [m], LT in-weight of each edge

    @property
    def indeg(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


def rmat(n: int, m: int, seed: int, a: float = 0.57, b: float = 0.19, c: float = 0.19) -> Graph:
    lib = _load()
    row_ptr = np.empty(n + 1, dtype=np.uint32)
    col = np.empty(max(m, 1), dtype=np.uint32)
    rc = lib.synth_rmat(n, m, seed, a, b, c, _ptr(row_ptr), _ptr(col))
    if rc != 0:
        raise ValueError("synth_rmat: bad arguments or out of memory")
    return Graph(n, m, row_ptr, col[:m])


def ic_uniform(g: Graph, seed: int, pmax: float = 0.1) -> np.ndarray:
    p = np.empty(max(g.m, 1), dtype=np.float32)
    _load().synth_ic_uniform(g.m, seed, ctypes.c_float(pmax), _ptr(p))
    return p[:g.m]


def weighted_cascade(g: Graph) -> np.ndarray:
    p = np.zeros(max(g.m, 1), dtype=np.float32)
    _load().synth_weighted_cascade(g.n, _ptr(g.row_ptr), _ptr(p))
    return p[:g.m]


def lt_weights(g: Graph, seed: int) -> np.ndarray:
    w = np.zeros(max(g.m, 1), dtype=np.float32)
    _load().synth_lt_weights(g.n, _ptr(g.row_ptr), seed, _ptr(w))
    return w[:g.m]


def draws(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.empty(max(count, 1), dtype=np.uint64)
    _load().synth_draws(seed, stream, count, _ptr(out))
    return out[:count]


def from_edges(n: int, edges, prob=None, lt_weight=None) -> Graph:
    """Small hand-made graphs: `edges` is a list of (u, v) meaning u -> v.

    Row v of the transposed CSR lists the sources in the given edge order, so
    per-edge parameters are given in the same order as `edges`."""
    edges = list(edges)
    order = sorted(range(len(edges)), key=lambda i: (edges[i][1], i))
    row_ptr = np.zeros(n + 1, dtype=np.uint32)
    for (_, v) in edges:
        row_ptr[v + 1] += 1
    row_ptr = np.cumsum(row_ptr, dtype=np.uint64).astype(np.uint32)
    col = np.array([edges[i][0] for i in order], dtype=np.uint32)
    g = Graph(n, len(edges), row_ptr, col)
    if prob is not None:
        g.prob = np.array([prob[i] for i in order], dtype=np.float32)
    if lt_weight is not None:
        g.lt_weight = np.array([lt_weight[i] for i in order], dtype=np.float32)
    return g


# ---------------------------------------------------------------------------
# Named workloads.  Sizes follow the paper's graph shapes (Table 4); the IC
# probabilities are not stated in the paper, so they are chosen here.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    n: int
    m: int
    graph_seed: int
    model: str          # "IC" or "LT"
    weights: str        # "uniform0.1", "wc" or "lt"
    k: int
    eps: float
    ell: float
    rr_seed: int
    encode: int         # 0 = uncompressed int32 sets, 1 = Huffman + bitmap
    density_cut: int = 32

    def graph(self) -> Graph:
        g = rmat(self.n, self.m, self.graph_seed)
        if self.weights == "uniform0.1":
            g.prob = ic_uniform(g, self.graph_seed, 0.1)
        elif self.weights == "wc":
            g.prob = weighted_cascade(g)
        elif self.weights == "lt":
            g.lt_weight = lt_weights(g, self.graph_seed)
            # the LT-shaped graph of the serving mix also carries IC probabilities
            g.prob = ic_uniform(g, self.graph_seed, 0.1)
        else:
            raise ValueError(self.weights)
        return g


WORKLOADS = {
    # tiny IC, uniform probabilities, uncompressed sets
    "ic_rmat4k": Workload("ic_rmat4k", 4096, 32768, 1, "IC", "uniform0.1", 10, 0.5, 1.0, 7, 0),
    # weighted-cascade IC on a Skitter-sized skewed graph, Huffman + bitmap pool
    "wc_rmat1m": Workload("wc_rmat1m", 1 << 20, 1 << 24, 2, "IC", "wc", 50, 0.5, 1.0, 7, 1),
    # LT on a LiveJournal-sized graph
    "lt_rmat4m": Workload("lt_rmat4m", 1 << 22, 1 << 26, 3, "LT", "lt", 100, 0.3, 1.0, 7, 1),
    # the same kind of graph at 2^23 vertices, 2^28 edges: a profiling-size case
    # of the full-size kernels (a few GB on the device)
    "ic_rmat8m": Workload("ic_rmat8m", 1 << 23, 1 << 28, 78, "IC", "uniform0.1", 100, 0.5, 1.0, 7, 1),
    # IC on a twitter7-sized graph (41.65M vertices, 1.468B edges)
    "ic_rmat42m": Workload("ic_rmat42m", 41652230, 1468365182, 4, "IC", "uniform0.1", 100, 0.5, 1.0, 7, 1),
}


def poisson_queries(seed: int, count: int, rate_per_s: float, graphs, k_range=(10, 200),
                    eps_choices=(0.13, 0.2, 0.3, 0.5)):
    """Query stream for the serving workload: Poisson arrivals at `rate_per_s`,
    graph uniform over `graphs`, model IC or LT with probability 1/2 each,
    k uniform on k_range (inclusive), eps uniform over eps_choices."""
    d = draws(seed, 1, 5 * count).reshape(count, 5)
    u = ((d[:, 0] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    gaps = -np.log(u) / rate_per_s
    t = np.cumsum(gaps)
    out = []
    for i in range(count):
        out.append(dict(
            t=float(t[i]),
            graph=graphs[int(d[i, 1] % np.uint64(len(graphs)))],
            model="IC" if int(d[i, 2] & np.uint64(1)) == 0 else "LT",
            k=int(k_range[0] + int(d[i, 3] % np.uint64(k_range[1] - k_range[0] + 1))),
            eps=float(eps_choices[int(d[i, 4] % np.uint64(len(eps_choices)))]),
        ))
    return out


def scale_log2(n: int) -> int:
    return max(1, math.ceil(math.log2(n)))
