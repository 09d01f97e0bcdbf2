"""Python binding of the GB300 RR-set influence-maximization library.

Thin ctypes marshalling over the C ABI in ``include/hbx.h``: every function
here has the name of the C entry point it calls, converts numpy arrays to
pointers and raises :class:`HbxError` on a negative return code.  All work runs
in the CUDA library ``_build/libhbx.so`` (built by :func:`build`); there is no
fallback, and importing the binding fails loudly if the library is missing.

PyTorch is used for plumbing only: :func:`torch_context` creates a context on a
``torch.cuda.Stream`` whose device memory comes from torch's caching allocator.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build_mod

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build_mod.LIB

HBX_IC, HBX_LT = 0, 1
KIND_HUFFMAN, KIND_BITMAP, KIND_RAW = 0, 1, 2
ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "WEIGHTS_GT_1",
          -6: "ADMISSION", -7: "CANCELLED", -8: "INTERNAL"}


class HbxError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")


class hbx_options(ctypes.Structure):
    _fields_ = [("density_cut", ctypes.c_uint32), ("warmup_sets", ctypes.c_uint32), ("encode", ctypes.c_uint32),
                ("form", ctypes.c_uint32), ("pool_epoch", ctypes.c_uint32), ("warp_capacity", ctypes.c_uint32),
                ("warp_group_budget", ctypes.c_uint32), ("block_cluster", ctypes.c_uint32),
                ("max_device_bytes", ctypes.c_uint64), ("wait_cycles", ctypes.c_uint64),
                ("scheme", ctypes.c_uint32), ("select_mode", ctypes.c_uint32),
                ("fresh_final", ctypes.c_uint32), ("reserved_opt", ctypes.c_uint32)]


class hbx_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in
                ["theta", "covered", "sets_huffman", "sets_bitmap", "sets_raw", "sets_big", "rr_vertices",
                 "edges_scanned", "edges_live", "pool_bytes", "raw_int32_bytes", "code_bits", "warmup_sets"]] + \
               [("rounds", ctypes.c_uint32), ("warp_capacity", ctypes.c_uint32),
                ("warp_group_budget", ctypes.c_uint32), ("block_cluster", ctypes.c_uint32)] + \
               [(f, ctypes.c_double) for f in ["lb", "sample_s", "select_s", "total_s", "skewness", "density",
                                                "sample_kernel_s"]] + \
               [("sample_kernel_launches", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("count_kernel_s", ctypes.c_double), ("count_bytes", ctypes.c_uint64),
                ("ms_kernel_s", ctypes.c_double), ("ms_sets", ctypes.c_uint64), ("ms_philox_blocks", ctypes.c_uint64),
                ("select_kernel_s", ctypes.c_double), ("select_iterations", ctypes.c_uint64),
                ("dec_s", ctypes.c_double), ("dec_bytes", ctypes.c_uint64), ("uncoded_vertices", ctypes.c_uint64),
                ("scheme", ctypes.c_uint32), ("second_warp_capacity", ctypes.c_uint32), ("scheme_skewness", ctypes.c_double),
                ("argmax_s", ctypes.c_double), ("ms_group_visits", ctypes.c_uint64), ("ms_deferrals", ctypes.c_uint64)]

    def to_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (nvcc) into the package tree."""
    return _build_mod.build(force=force)


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run paper_2208_00613_gb300.build())")
    L = ctypes.CDLL(LIB_PATH)
    P, U32, U64, D, I, I64 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                              ctypes.c_int64)
    sig = {
        "hbx_strerror": (ctypes.c_char_p, [I]),
        "hbx_last_error": (ctypes.c_char_p, [P]),
        "hbx_default_options": (None, [P]),
        "hbx_create": (I, [P, I, P]),
        "hbx_set_allocator": (I, [P, P, P, P]),
        "hbx_destroy": (None, [P]),
        "hbx_graph_create": (I, [P, U32, U64, P, P, P, P, P]),
        "hbx_graph_destroy": (None, [P]),
        "hbx_imm": (I, [P, P, I, U32, D, D, U64, P, P, P, P, P]),
        "hbx_pool_create": (I, [P, P, I, U64, P, P]),
        "hbx_pool_destroy": (None, [P]),
        "hbx_pool_extend": (I, [P, U64]),
        "hbx_pool_size": (U64, [P]),
        "hbx_pool_select": (I, [P, U64, U32, P, P, P]),
        "hbx_imm_pool": (I, [P, U32, D, D, P, P, P, P]),
        "hbx_pool_export_set": (I, [P, U64, P, P, P, P, P, P, U64, P]),
        "hbx_pool_decode_sets": (I, [P, U64, U64, P, P, U64, P]),
        "hbx_pool_export_codebook": (I, [P, P, P, P, P]),
        "hbx_pool_stats": (I, [P, P]),
        "hbx_server_create": (I, [P, U32, U64, P]),
        "hbx_server_destroy": (None, [P]),
        "hbx_submit": (I, [P, P, I, U32, D, D, U64, P, P]),
        "hbx_wait": (I, [P, P, P, P, P, I64]),
        "hbx_cancel": (I, [P]),
        "hbx_ticket_destroy": (None, [P]),
        "hbx_argmax_noalloc": (I, [P, U32, P, P]),
        "hbx_philox_ceiling": (I, [P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _check(rc, ctx=None):
    if rc != 0:
        msg = lib().hbx_last_error(ctx).decode() if ctx else lib().hbx_strerror(rc).decode()
        raise HbxError(rc, msg)


def model_id(model) -> int:
    if isinstance(model, str):
        return {"IC": HBX_IC, "LT": HBX_LT}[model.upper()]
    return int(model)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def hbx_strerror(code: int) -> str:
    return lib().hbx_strerror(code).decode()


def hbx_last_error(ctx) -> str:
    return lib().hbx_last_error(ctx).decode()


def hbx_default_options(**overrides) -> hbx_options:
    o = hbx_options()
    lib().hbx_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def hbx_create(device: int = 0, stream: int | None = None):
    h = ctypes.c_void_p()
    _check(lib().hbx_create(ctypes.byref(h), device, ctypes.c_void_p(stream) if stream else None))
    return h


def hbx_set_allocator(ctx, alloc_fn, free_fn, user=None):
    _check(lib().hbx_set_allocator(ctx, alloc_fn, free_fn, user), ctx)


def hbx_destroy(ctx):
    lib().hbx_destroy(ctx)


def hbx_graph_create(ctx, g):
    """g: object with n, m, row_ptr (uint32), col (uint32), prob / lt_weight (float32 or None)."""
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint32)
    col = np.ascontiguousarray(g.col, dtype=np.uint32) if g.m else np.zeros(1, np.uint32)
    pr = None if getattr(g, "prob", None) is None else np.ascontiguousarray(g.prob, dtype=np.float32)
    lw = None if getattr(g, "lt_weight", None) is None else np.ascontiguousarray(g.lt_weight, dtype=np.float32)
    h = ctypes.c_void_p()
    _check(lib().hbx_graph_create(ctx, g.n, g.m, _p(rp), _p(col), _p(pr), _p(lw), ctypes.byref(h)), ctx)
    return h


def hbx_graph_destroy(g):
    lib().hbx_graph_destroy(g)


def hbx_imm(ctx, graph, model, k, eps, ell, seed, opts=None):
    seeds = np.empty(k, dtype=np.uint32)
    marg = np.empty(k, dtype=np.uint64)
    infl = ctypes.c_double()
    st = hbx_stats()
    _check(lib().hbx_imm(ctx, graph, model_id(model), k, eps, ell, seed, ctypes.byref(opts) if opts else None,
                         _p(seeds), ctypes.byref(infl), _p(marg), ctypes.byref(st)), ctx)
    return dict(seeds=seeds, influence=infl.value, marginal=marg, stats=st.to_dict())


def hbx_pool_create(ctx, graph, model, seed, opts=None):
    h = ctypes.c_void_p()
    _check(lib().hbx_pool_create(ctx, graph, model_id(model), seed, ctypes.byref(opts) if opts else None,
                                 ctypes.byref(h)), ctx)
    return h


def hbx_pool_destroy(pool):
    lib().hbx_pool_destroy(pool)


def hbx_pool_extend(ctx, pool, T):
    _check(lib().hbx_pool_extend(pool, T), ctx)


def hbx_pool_size(pool) -> int:
    return int(lib().hbx_pool_size(pool))


def hbx_pool_select(ctx, pool, T, k):
    seeds = np.empty(k, dtype=np.uint32)
    marg = np.empty(k, dtype=np.uint64)
    cov = ctypes.c_uint64()
    _check(lib().hbx_pool_select(pool, T, k, _p(seeds), _p(marg), ctypes.byref(cov)), ctx)
    return seeds, marg, cov.value


def hbx_imm_pool(ctx, pool, k, eps, ell):
    seeds = np.empty(k, dtype=np.uint32)
    marg = np.empty(k, dtype=np.uint64)
    infl = ctypes.c_double()
    st = hbx_stats()
    _check(lib().hbx_imm_pool(pool, k, eps, ell, _p(seeds), ctypes.byref(infl), _p(marg), ctypes.byref(st)), ctx)
    return dict(seeds=seeds, influence=infl.value, marginal=marg, stats=st.to_dict())


def hbx_pool_export_set(ctx, pool, j, cap=1 << 16):
    kind, size, ncod, nraw = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    bits, nbytes = ctypes.c_uint64(), ctypes.c_uint64()
    while True:
        buf = np.zeros(max(cap, 1), dtype=np.uint8)
        rc = lib().hbx_pool_export_set(pool, j, ctypes.byref(kind), ctypes.byref(size), ctypes.byref(ncod),
                                       ctypes.byref(nraw), ctypes.byref(bits), _p(buf), cap, ctypes.byref(nbytes))
        if rc == -1 and nbytes.value > cap:
            cap = nbytes.value
            continue
        _check(rc, ctx)
        break
    payload = buf[:nbytes.value]
    d = dict(kind=kind.value, size=size.value, n_coded=ncod.value, n_raw=nraw.value, code_bits=bits.value)
    if kind.value == KIND_HUFFMAN:
        nb = (bits.value + 7) // 8
        at = (nb + 3) & ~3
        d["bytes"] = payload[:nb].tobytes()
        d["raw"] = payload[at:at + 4 * nraw.value].view(np.uint32).copy()
    elif kind.value == KIND_BITMAP:
        d["bitmap"] = payload.view(np.uint32).copy()
    else:
        d["verts"] = payload.view(np.uint32).copy()
    return d


def hbx_pool_decode_sets(ctx, pool, j0, j1):
    off = np.zeros(j1 - j0 + 1, dtype=np.uint64)
    need = ctypes.c_uint64()
    rc = lib().hbx_pool_decode_sets(pool, j0, j1, _p(off), None, 0, ctypes.byref(need))
    if rc not in (0, -1):
        _check(rc, ctx)
    verts = np.empty(max(need.value, 1), dtype=np.uint32)
    _check(lib().hbx_pool_decode_sets(pool, j0, j1, _p(off), _p(verts), need.value, ctypes.byref(need)), ctx)
    return off, verts[:need.value]


def hbx_pool_export_codebook(ctx, pool, n):
    ln, code, rank, freq = (np.empty(n, dtype=np.uint32) for _ in range(4))
    _check(lib().hbx_pool_export_codebook(pool, _p(ln), _p(code), _p(rank), _p(freq)), ctx)
    return dict(len=ln, code=code, rank=rank, freq=freq)


def hbx_pool_stats(ctx, pool):
    st = hbx_stats()
    _check(lib().hbx_pool_stats(pool, ctypes.byref(st)), ctx)
    return st.to_dict()


def hbx_server_create(ctx, max_inflight=4, memory_budget=0):
    h = ctypes.c_void_p()
    _check(lib().hbx_server_create(ctx, max_inflight, memory_budget, ctypes.byref(h)), ctx)
    return h


def hbx_server_destroy(server):
    lib().hbx_server_destroy(server)


def hbx_submit(ctx, server, graph, model, k, eps, ell, seed, opts=None):
    h = ctypes.c_void_p()
    _check(lib().hbx_submit(server, graph, model_id(model), k, eps, ell, seed, ctypes.byref(opts) if opts else None,
                            ctypes.byref(h)), ctx)
    return h


def hbx_wait(ticket, k, timeout_us=-1):
    """Returns (rc, result-dict-or-None); rc is the raw code (TIMEOUT keeps the ticket)."""
    seeds = np.empty(k, dtype=np.uint32)
    infl, lat = ctypes.c_double(), ctypes.c_double()
    st = hbx_stats()
    rc = lib().hbx_wait(ticket, _p(seeds), ctypes.byref(infl), ctypes.byref(st), ctypes.byref(lat), timeout_us)
    if rc != 0:
        return rc, None
    return 0, dict(seeds=seeds, influence=infl.value, stats=st.to_dict(), latency_s=lat.value)


def hbx_cancel(ticket) -> int:
    return lib().hbx_cancel(ticket)


def hbx_ticket_destroy(ticket):
    lib().hbx_ticket_destroy(ticket)


def hbx_philox_ceiling(ctx) -> float:
    """Philox4x32-10 blocks per second of the device (see include/hbx.h)."""
    out = ctypes.c_double()
    _check(lib().hbx_philox_ceiling(ctx, ctypes.byref(out)), ctx)
    return out.value


def hbx_argmax_noalloc(d_counts: int, n: int, d_out: int, stream: int | None = None) -> int:
    """Allocation-free argmax (see include/hbx.h): device pointers in, the
    winning index written to d_out on `stream`.  Returns the raw code."""
    return lib().hbx_argmax_noalloc(ctypes.c_void_p(d_counts), n, ctypes.c_void_p(d_out),
                                    ctypes.c_void_p(stream) if stream else None)


# ---------------------------------------------------------------------------
# torch plumbing
# ---------------------------------------------------------------------------
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class TorchContext:
    """A library context on a torch CUDA stream, allocating through torch's
    caching allocator.  Keeps the callbacks alive; call close() (or use as a
    context manager) to destroy."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        self.stream = torch.cuda.Stream(device=device)
        self.ctx = hbx_create(device, self.stream.cuda_stream)

        def _alloc(size, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(size), device, self.stream)
            except Exception:
                return None

        def _free(ptr, user):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc = _ALLOC_T(_alloc)
        self._free = _FREE_T(_free)
        hbx_set_allocator(self.ctx, ctypes.cast(self._alloc, ctypes.c_void_p), ctypes.cast(self._free, ctypes.c_void_p))

    def close(self):
        if self.ctx:
            hbx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def torch_context(device: int = 0) -> TorchContext:
    return TorchContext(device)
