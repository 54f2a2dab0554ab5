"""B300-native sieved multi-way join (SieveJoin, arXiv 2308.16370).

Thin Python binding over the C ABI of ``libsievejoin.so`` (``include/sievejoin.h``):
argument marshalling only, every step runs in the CUDA kernels.  PyTorch
provides device memory, streams and zero-copy views of result columns.

The library must be built first (``python -m paper_2308_16370_b300.build``);
there is no CPU fallback, and every entry point raises if the CUDA library or
a GPU is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Context", "Relation", "Filter", "SieveJoinError", "load_library", "LIB_PATH",
           "REGBLOCKED32", "BLOCKED256", "CLASSIC", "FWD_BWD", "BWD_ONLY", "NO_SIEVE", "COUNT_SUM",
           "MATERIALIZE", "KERNEL_KINDS", "INSERT_GATED", "INSERT_CONTAINED", "INSERT_NEW"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsievejoin.so")

REGBLOCKED32, BLOCKED256, CLASSIC = 0, 1, 2
FWD_BWD, BWD_ONLY, NO_SIEVE = 0, 1, 2
COUNT_SUM, MATERIALIZE = 0, 1
INSERT_GATED, INSERT_CONTAINED, INSERT_NEW = 0, 1, 2
DEVICE_BORROW, DEVICE_COPY, HOST_COPY, HOST_MAPPED = 0, 1, 2, 3
MAX_COLS, MAX_REL, MAX_PROBES, MAX_TERMS, MAX_STEPS = 8, 8, 4, 8, 32
KERNEL_KINDS = {"bloom_build": 0, "sieve": 1, "ht_build": 2, "ht_probe": 3, "ht_expand": 4,
                "agg": 5, "other": 6}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "hash table full",
          4: "device wait timed out", 5: "COUNT overflow", 6: "CUDA error"}

# exported symbols of the C ABI (checked by the CPU tests against the header)
EXPORTS = ["sj_create", "sj_destroy", "sj_sync", "sj_last_error", "sj_status_str", "sj_version",
           "sj_load_relation", "sj_rel_info", "sj_free_rel", "sj_build_filter", "sj_filter_info",
           "sj_filter_probe", "sj_free_filter", "sj_sieve", "sj_sieve_path", "sj_sieve_path_batch", "sj_join",
           "sj_prof_enable", "sj_prof_kinds", "sj_prof_reset", "sj_prof_read", "sj_counters", "sj_graph_stats", "sj_graphs_enable", "sj_sieve_noalloc",
           "sj_server_create", "sj_server_add_relation", "sj_server_submit", "sj_server_poll",
           "sj_server_stats_get", "sj_server_destroy", "sj_triangles", "sj_sieve_join", "sj_prof_gaps",
           "sj_selftest_wait_timeout", "sj_filter_insert"]


class SieveJoinError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


# ----------------------------------------------------------------------------- ctypes mirror
class FilterParams(ctypes.Structure):
    _fields_ = [("bits_per_key", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("layout", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("seed", ctypes.c_uint64)]


class Pred(ctypes.Structure):
    _fields_ = [("col", ctypes.c_int32), ("lo", ctypes.c_int32), ("hi", ctypes.c_int32)]


class Edge(ctypes.Structure):
    _fields_ = [("rel_a", ctypes.c_int32), ("col_a", ctypes.c_int32),
                ("rel_b", ctypes.c_int32), ("col_b", ctypes.c_int32)]


class Path(ctypes.Structure):
    _fields_ = [("nrel", ctypes.c_int32), ("root", ctypes.c_int32),
                ("rels", ctypes.POINTER(ctypes.c_void_p)), ("edges", ctypes.POINTER(Edge)),
                ("preds", ctypes.POINTER(Pred))]


class SieveOpts(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("filter", FilterParams), ("leaf_filters", ctypes.POINTER(ctypes.c_void_p))]


class StepStat(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("rel", ctypes.c_int32),
                ("rows_in", ctypes.c_int64), ("rows_out", ctypes.c_int64)]


class SieveStats(ctypes.Structure):
    _fields_ = [("nsteps", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("step", StepStat * MAX_STEPS), ("rows_final", ctypes.c_int64 * MAX_REL),
                ("filter_bytes", ctypes.c_uint64)]


class ColRef(ctypes.Structure):
    _fields_ = [("rel", ctypes.c_int32), ("col", ctypes.c_int32), ("wide", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("nslots", ctypes.c_int32),
                ("hbm_budget", ctypes.c_uint64), ("passes", ctypes.c_int32),
                ("cache_filters", ctypes.c_int32), ("filter", FilterParams),
                ("batch", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("batch_max_rows", ctypes.c_uint64)]


class Query(ctypes.Structure):
    _fields_ = [("nrel", ctypes.c_int32), ("root", ctypes.c_int32),
                ("rel", ctypes.c_int32 * MAX_REL), ("edges", Edge * (MAX_REL - 1)),
                ("preds", Pred * MAX_REL), ("nterms", ctypes.c_int32),
                ("terms", ColRef * MAX_TERMS)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("cache_hits", ctypes.c_int32), ("count", ctypes.c_uint64),
                ("sum", ctypes.c_uint64), ("submit_ms", ctypes.c_double),
                ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("cache_hits", ctypes.c_uint64),
                ("cache_misses", ctypes.c_uint64), ("cached_filters", ctypes.c_uint64),
                ("peak_inflight_bytes", ctypes.c_uint64), ("peak_concurrency", ctypes.c_int32),
                ("peak_batch", ctypes.c_int32), ("batches", ctypes.c_uint64)]


class TriStats(ctypes.Structure):
    _fields_ = [("edges_in", ctypes.c_int64), ("edges_sieved", ctypes.c_int64),
                ("candidates", ctypes.c_uint64), ("filter_passed", ctypes.c_uint64),
                ("triangles", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("sum", ctypes.c_uint64),
                ("intermediate", ctypes.c_uint64), ("rows", ctypes.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load ``libsievejoin.so``; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2308_16370_b300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "sj_create": [PP, I, P, P, P, P],
        "sj_destroy": [P], "sj_sync": [P],
        "sj_load_relation": [P, I, PP, I64, I, PP],
        "sj_rel_info": [P, ctypes.POINTER(I64), ctypes.POINTER(I), PP],
        "sj_free_rel": [P, P],
        "sj_build_filter": [P, P, I, ctypes.POINTER(Pred), ctypes.POINTER(FilterParams), PP],
        "sj_filter_info": [P, P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), PP],
        "sj_filter_probe": [P, P, P, I64, P],
        "sj_filter_insert": [P, P, P, I, I, ctypes.POINTER(ctypes.c_int), PP, P, ctypes.POINTER(I64)],
        "sj_free_filter": [P, P],
        "sj_sieve": [P, P, I, ctypes.POINTER(ctypes.c_int), PP, ctypes.POINTER(Pred), PP,
                     ctypes.POINTER(I64)],
        "sj_sieve_path": [P, ctypes.POINTER(Path), ctypes.POINTER(SieveOpts), PP,
                          ctypes.POINTER(SieveStats)],
        "sj_sieve_path_batch": [P, I, ctypes.POINTER(Path), ctypes.POINTER(SieveOpts), PP,
                                ctypes.POINTER(SieveStats)],
        "sj_join": [P, ctypes.POINTER(Path), PP, I, I, ctypes.POINTER(ColRef), ctypes.POINTER(Result)],
        "sj_prof_enable": [P, I], "sj_prof_kinds": [P, ctypes.c_uint32], "sj_prof_reset": [P],
        "sj_prof_read": [P, I, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_double)],
        "sj_counters": [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)],
        "sj_graphs_enable": [P, I],
        "sj_graph_stats": [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.c_char_p, I],
        "sj_prof_gaps": [P, ctypes.POINTER(ctypes.c_double)],
        "sj_selftest_wait_timeout": [P],
        "sj_sieve_noalloc": [P, I, PP, I64, I, P, ctypes.c_uint64, ctypes.POINTER(FilterParams),
                             PP, P, P, ctypes.POINTER(ctypes.c_char_p)],
        "sj_server_create": [PP, ctypes.POINTER(ServerOpts)],
        "sj_server_add_relation": [P, I, PP, I64, ctypes.POINTER(ctypes.c_int32)],
        "sj_server_submit": [P, ctypes.POINTER(Query), ctypes.POINTER(ctypes.c_uint64)],
        "sj_server_poll": [P, ctypes.POINTER(Completion), I, ctypes.POINTER(I), I],
        "sj_server_stats_get": [P, ctypes.POINTER(ServerStats)],
        "sj_server_destroy": [P],
        "sj_triangles": [P, P, I, P, I, ctypes.POINTER(FilterParams), P, ctypes.POINTER(TriStats)],
        "sj_sieve_join": [P, ctypes.POINTER(Path), ctypes.POINTER(SieveOpts), I, I,
                          ctypes.POINTER(ColRef), ctypes.POINTER(Result), ctypes.POINTER(SieveStats)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.sj_last_error.argtypes = [P]
    lib.sj_last_error.restype = ctypes.c_char_p
    lib.sj_status_str.argtypes = [ctypes.c_int]
    lib.sj_status_str.restype = ctypes.c_char_p
    lib.sj_version.argtypes = []
    lib.sj_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


class _CudaArray:
    """Zero-copy ``__cuda_array_interface__`` view of library-owned memory."""

    def __init__(self, ptr: int, n: int, typestr: str = "<i4"):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _torch():
    import torch
    return torch


# ----------------------------------------------------------------------------- handles
class Relation:
    """A columnar int32 relation on the device (library handle)."""

    def __init__(self, ctx: "Context", handle: int, keep=None):
        self.ctx = ctx
        self.handle = ctypes.c_void_p(handle)
        self._keep = keep  # borrowed tensors must outlive the handle
        n = ctypes.c_int64()
        nc = ctypes.c_int()
        ptrs = (ctypes.c_void_p * MAX_COLS)()
        ctx._check(ctx.lib.sj_rel_info(self.handle, ctypes.byref(n), ctypes.byref(nc), ptrs))
        self.nrows = int(n.value)
        self.ncols = int(nc.value)
        self.col_ptrs = [int(ptrs[j] or 0) for j in range(self.ncols)]

    def column(self, j: int):
        """Zero-copy torch view of column j (valid while this handle lives)."""
        torch = _torch()
        if self.nrows == 0:
            return torch.empty(0, dtype=torch.int32, device=f"cuda:{self.ctx.device}")
        return torch.as_tensor(_CudaArray(self.col_ptrs[j], self.nrows),
                               device=f"cuda:{self.ctx.device}")

    def to_numpy(self):
        self.ctx.sync()
        return [self.column(j).cpu().numpy().copy() for j in range(self.ncols)]

    def free(self):
        if self.handle and self.ctx.ctx:
            self.ctx.lib.sj_free_rel(self.ctx.ctx, self.handle)
        self.handle = None
        self._keep = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Filter:
    def __init__(self, ctx: "Context", handle: int, params: FilterParams):
        self.ctx = ctx
        self.handle = ctypes.c_void_p(handle)
        self.params = params

    def info(self):
        nb = ctypes.c_uint64()
        ni = ctypes.c_uint64()
        w = ctypes.c_void_p()
        self.ctx._check(self.ctx.lib.sj_filter_info(self.ctx.ctx, self.handle, ctypes.byref(nb),
                                                    ctypes.byref(ni), ctypes.byref(w)))
        return int(nb.value), int(ni.value), int(w.value)

    def words(self) -> np.ndarray:
        """Copy of the filter words (nblocks * 8 uint32)."""
        nb, _, ptr = self.info()
        t = _torch().as_tensor(_CudaArray(ptr, nb * 8, "<i4"), device=f"cuda:{self.ctx.device}")
        return t.cpu().numpy().view(np.uint32).copy()

    def free(self):
        if self.handle and self.ctx.ctx:
            self.ctx.lib.sj_free_filter(self.ctx.ctx, self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _params(bits_per_key=8, k=3, layout=REGBLOCKED32, seed=0) -> FilterParams:
    return FilterParams(int(bits_per_key), int(k), int(layout), 0, int(seed) & ((1 << 64) - 1))


def _pred(p):
    if p is None:
        return None
    c, lo, hi = p
    return Pred(int(c), int(lo), int(hi))


class Context:
    """One device + one stream.  ``stream`` is a torch.cuda.Stream (default:
    the current stream).  With ``torch_allocator`` the library allocates
    through PyTorch's caching allocator, else through cudaMallocAsync."""

    def __init__(self, device: int = 0, stream=None, torch_allocator: bool = False):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("sievejoin needs a CUDA GPU; none is visible")
        self.lib = load_library()
        self.device = int(device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._cbs = None
        alloc = free = None
        if torch_allocator:
            dev, st = self.device, self.stream

            @ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:
                    return None

            @ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
            def _free(ptr, nbytes, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cbs = (_alloc, _free)
            alloc = ctypes.cast(_alloc, ctypes.c_void_p)
            free = ctypes.cast(_free, ctypes.c_void_p)
        h = ctypes.c_void_p()
        st = self.lib.sj_create(ctypes.byref(h), self.device, ctypes.c_void_p(self.stream.cuda_stream),
                                alloc, free, None)
        if st != 0:
            raise SieveJoinError(st, "sj_create failed")
        self.ctx = h

    # --------------------------------------------------------------- plumbing
    def _check(self, st: int):
        if st != 0:
            msg = self.lib.sj_last_error(self.ctx).decode() if self.ctx else ""
            raise SieveJoinError(st, msg)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.sj_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sync(self):
        self._check(self.lib.sj_sync(self.ctx))

    # --------------------------------------------------------------- relations
    def load_relation(self, cols, where: str = "borrow") -> Relation:
        """``cols``: torch int32 CUDA tensors (``borrow``/``copy``), numpy /
        CPU tensors (``host``; copied on the context stream), or pinned CPU
        tensors (``mapped``; not copied: kernels read them over the host link,
        and they are kept alive with the handle)."""
        torch = _torch()
        mode = {"borrow": DEVICE_BORROW, "copy": DEVICE_COPY, "host": HOST_COPY,
                "mapped": HOST_MAPPED}[where]
        keep = []
        ptrs = (ctypes.c_void_p * len(cols))()
        n = None
        for j, c in enumerate(cols):
            if mode == HOST_COPY:
                if isinstance(c, np.ndarray):
                    c = np.ascontiguousarray(c, dtype=np.int32)
                    ptrs[j] = c.ctypes.data
                else:
                    c = c.contiguous()
                    assert c.dtype == torch.int32 and not c.is_cuda
                    ptrs[j] = c.data_ptr()
            elif mode == HOST_MAPPED:
                if not (c.dtype == torch.int32 and not c.is_cuda and c.is_contiguous() and c.is_pinned()):
                    raise ValueError("'mapped' columns must be contiguous pinned int32 CPU tensors")
                ptrs[j] = c.data_ptr()
            else:
                assert c.dtype == torch.int32 and c.is_cuda and c.is_contiguous()
                ptrs[j] = c.data_ptr()
            keep.append(c)
            n = len(c) if n is None else n
            if len(c) != n:
                raise ValueError("columns differ in length")
        h = ctypes.c_void_p()
        self._check(self.lib.sj_load_relation(self.ctx, len(cols), ptrs, int(n or 0), mode,
                                              ctypes.byref(h)))
        if mode == HOST_COPY:
            self.sync()  # host buffers may be released after this
            keep = None
        elif mode == DEVICE_COPY:
            keep = None
        return Relation(self, h.value, keep)

    # --------------------------------------------------------------- filters
    def build_filter(self, rel: Relation, key_col: int, pred=None, bits_per_key=8, k=3,
                     layout=REGBLOCKED32, seed=0) -> Filter:
        p = _params(bits_per_key, k, layout, seed)
        pr = _pred(pred)
        h = ctypes.c_void_p()
        self._check(self.lib.sj_build_filter(self.ctx, rel.handle, int(key_col),
                                             ctypes.byref(pr) if pr else None, ctypes.byref(p),
                                             ctypes.byref(h)))
        return Filter(self, h.value, p)

    def filter_probe(self, f: Filter, keys):
        torch = _torch()
        out = torch.empty(len(keys), dtype=torch.uint8, device=keys.device)
        self._check(self.lib.sj_filter_probe(self.ctx, f.handle, ctypes.c_void_p(keys.data_ptr()),
                                             len(keys), ctypes.c_void_p(out.data_ptr())))
        return out

    def filter_insert(self, f: Filter, rel: Relation, key_col: int, gates=()):
        """Insert maintenance (Sec. 2.4): the rows of ``rel`` are new tuples of
        the relation ``f`` was built over (key in column ``key_col``); ``gates``
        are (column, filter) pairs of the neighbours' filters.  Returns (per-row
        outcome as a uint8 tensor: INSERT_GATED / INSERT_CONTAINED / INSERT_NEW,
        counts of the three)."""
        torch = _torch()
        status = torch.empty(max(rel.nrows, 1), dtype=torch.uint8, device=f"cuda:{self.device}")
        gc = (ctypes.c_int * max(1, len(gates)))(*[int(g[0]) for g in gates])
        gf = (ctypes.c_void_p * max(1, len(gates)))(*[g[1].handle.value for g in gates])
        counts = (ctypes.c_int64 * 3)()
        self._check(self.lib.sj_filter_insert(self.ctx, f.handle, rel.handle, int(key_col), len(gates),
                                              gc, gf, ctypes.c_void_p(status.data_ptr()), counts))
        return status[:rel.nrows], [int(x) for x in counts]

    def sieve(self, rel: Relation, key_cols=(), filters=(), pred=None) -> Relation:
        kc = (ctypes.c_int * max(1, len(key_cols)))(*key_cols)
        fs = (ctypes.c_void_p * max(1, len(filters)))(*[f.handle.value for f in filters])
        pr = _pred(pred)
        h = ctypes.c_void_p()
        n = ctypes.c_int64()
        self._check(self.lib.sj_sieve(self.ctx, rel.handle, len(key_cols), kc, fs,
                                      ctypes.byref(pr) if pr else None, ctypes.byref(h),
                                      ctypes.byref(n)))
        return Relation(self, h.value)

    # --------------------------------------------------------------- paths
    def _path(self, rels, edges, preds, root):
        n = len(rels)
        hs = (ctypes.c_void_p * n)(*[r.handle.value for r in rels])
        es = (Edge * max(1, len(edges)))(*[Edge(*map(int, e)) for e in edges])
        ps = None
        if preds is not None and any(p is not None for p in preds):
            ps = (Pred * n)(*[_pred(p) if p is not None else Pred(-1, 0, 0) for p in preds])
        path = Path(n, int(root), ctypes.cast(hs, ctypes.POINTER(ctypes.c_void_p)),
                    ctypes.cast(es, ctypes.POINTER(Edge)),
                    ctypes.cast(ps, ctypes.POINTER(Pred)) if ps is not None else None)
        return path, (hs, es, ps)

    def sieve_path(self, rels, edges, preds=None, root=-1, passes=FWD_BWD, bits_per_key=8, k=3,
                   layout=REGBLOCKED32, seed=0, leaf_filters=None):
        """Pruning phase over a join tree.  Returns (sieved relations, stats).

        ``leaf_filters``: None or one Filter / None per relation, reused for
        leaves in pass 1 instead of being rebuilt (Sec. 2.3)."""
        path, keep = self._path(rels, edges, preds, root)
        lf = None
        if leaf_filters is not None:
            lf = (ctypes.c_void_p * len(rels))(*[(f.handle.value if f is not None else None)
                                                 for f in leaf_filters])
        opts = SieveOpts(int(passes), 0, _params(bits_per_key, k, layout, seed),
                         ctypes.cast(lf, ctypes.POINTER(ctypes.c_void_p)) if lf is not None else None)
        outs = (ctypes.c_void_p * len(rels))()
        stats = SieveStats()
        self._check(self.lib.sj_sieve_path(self.ctx, ctypes.byref(path), ctypes.byref(opts), outs,
                                           ctypes.byref(stats)))
        sieved = [Relation(self, outs[i]) for i in range(len(rels))]
        steps = [(("select", "fwd", "bwd")[stats.step[s].kind], stats.step[s].rel,
                  stats.step[s].rows_in, stats.step[s].rows_out) for s in range(stats.nsteps)]
        return sieved, {"steps": steps, "rows_final": [stats.rows_final[i] for i in range(len(rels))],
                        "filter_bytes": int(stats.filter_bytes)}

    def sieve_path_batch(self, queries, passes=FWD_BWD, bits_per_key=8, k=3, layout=REGBLOCKED32,
                         seed=0):
        """Pruning phases of several queries in one call (lock-step launches).

        ``queries``: dicts with ``rels``, ``edges`` and optionally ``preds``,
        ``root`` and ``leaf_filters`` (as for sieve_path).  Returns one
        (sieved relations, stats) pair per query, equal to sieve_path's."""
        nq = len(queries)
        paths = (Path * max(1, nq))()
        opts = (SieveOpts * max(1, nq))()
        keep = []
        for i, q in enumerate(queries):
            path, kp = self._path(q["rels"], q["edges"], q.get("preds"), q.get("root", -1))
            paths[i] = path
            keep.append(kp)
            lf = None
            if q.get("leaf_filters") is not None:
                lf = (ctypes.c_void_p * len(q["rels"]))(*[(f.handle.value if f is not None else None)
                                                          for f in q["leaf_filters"]])
                keep.append(lf)
            opts[i] = SieveOpts(int(passes), 0, _params(bits_per_key, k, layout, seed),
                                ctypes.cast(lf, ctypes.POINTER(ctypes.c_void_p)) if lf is not None else None)
        outs = (ctypes.c_void_p * (MAX_REL * max(1, nq)))()
        stats = (SieveStats * max(1, nq))()
        self._check(self.lib.sj_sieve_path_batch(self.ctx, nq, paths, opts, outs, stats))
        res = []
        for i, q in enumerate(queries):
            n = len(q["rels"])
            st = stats[i]
            sieved = [Relation(self, outs[i * MAX_REL + j]) for j in range(n)]
            steps = [(("select", "fwd", "bwd")[st.step[s].kind], st.step[s].rel,
                      st.step[s].rows_in, st.step[s].rows_out) for s in range(st.nsteps)]
            res.append((sieved, {"steps": steps, "rows_final": [st.rows_final[j] for j in range(n)],
                                 "filter_bytes": int(st.filter_bytes)}))
        return res

    def join(self, rels, edges, preds=None, root=-1, inputs=None, mode=COUNT_SUM, refs=()):
        """Left-deep hash join.  ``refs`` = [(rel, col, wide), ...]: SUM terms
        (COUNT_SUM) or projected columns (MATERIALIZE)."""
        path, keep = self._path(rels, edges, preds, root)
        ins = None
        if inputs is not None:
            ins = (ctypes.c_void_p * len(inputs))(*[r.handle.value for r in inputs])
        rs = (ColRef * max(1, len(refs)))(*[ColRef(int(r[0]), int(r[1]), int(r[2]) if len(r) > 2 else 0, 0)
                                            for r in refs])
        res = Result()
        self._check(self.lib.sj_join(self.ctx, ctypes.byref(path), ins, int(mode), len(refs), rs,
                                     ctypes.byref(res)))
        out = {"count": int(res.count), "sum": int(res.sum), "intermediate": int(res.intermediate),
               "rows": None}
        if res.rows:
            out["rows"] = Relation(self, res.rows)
        return out

    def sieve_join(self, rels, edges, preds=None, root=-1, mode=COUNT_SUM, refs=(), passes=FWD_BWD,
                   bits_per_key=8, k=3, layout=REGBLOCKED32, seed=0, stats=False):
        """Pruning phase then enumeration phase in one library call."""
        path, keep = self._path(rels, edges, preds, root)
        opts = SieveOpts(int(passes), 0, _params(bits_per_key, k, layout, seed), None)
        rs = (ColRef * max(1, len(refs)))(*[ColRef(int(r[0]), int(r[1]), int(r[2]) if len(r) > 2 else 0, 0)
                                            for r in refs])
        res = Result()
        st = SieveStats() if stats else None
        self._check(self.lib.sj_sieve_join(self.ctx, ctypes.byref(path), ctypes.byref(opts), int(mode),
                                           len(refs), rs, ctypes.byref(res),
                                           ctypes.byref(st) if st is not None else None))
        out = {"count": int(res.count), "sum": int(res.sum), "intermediate": int(res.intermediate),
               "rows": Relation(self, res.rows) if res.rows else None}
        if st is not None:
            out["steps"] = [(("select", "fwd", "bwd")[st.step[s].kind], st.step[s].rel,
                             st.step[s].rows_in, st.step[s].rows_out) for s in range(st.nsteps)]
        return out

    # --------------------------------------------------------------- cyclic query
    def triangles(self, edges: Relation, cuts, sieve_rounds: int = -1, bits_per_key=8, k=3, seed=0):
        """Per-subquery ordered triangle counts of the directed edge relation
        (cols: source, target) for a in [cuts[i], cuts[i+1]).  Returns
        (counts as a numpy uint64 array, stats dict)."""
        cuts = np.ascontiguousarray(cuts, dtype=np.int32)
        nsub = len(cuts) - 1
        counts = np.zeros(nsub, dtype=np.uint64)
        st = TriStats()
        p = _params(bits_per_key, k, REGBLOCKED32, seed)
        self._check(self.lib.sj_triangles(self.ctx, edges.handle, nsub, cuts.ctypes.data,
                                          int(sieve_rounds), ctypes.byref(p), counts.ctypes.data,
                                          ctypes.byref(st)))
        return counts, {f: int(getattr(st, f)) for f, _ in TriStats._fields_}

    # --------------------------------------------------------------- profiling
    def prof_enable(self, on: bool = True):
        self._check(self.lib.sj_prof_enable(self.ctx, 1 if on else 0))

    def prof_kinds(self, kinds=None):
        """Profile only these kernel classes (names of KERNEL_KINDS; None = all)."""
        mask = 0xFFFFFFFF if kinds is None else sum(1 << KERNEL_KINDS[k] for k in kinds)
        self._check(self.lib.sj_prof_kinds(self.ctx, ctypes.c_uint32(mask)))

    def prof_reset(self):
        self._check(self.lib.sj_prof_reset(self.ctx))

    def prof_read(self, kind: str):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        b = ctypes.c_double()
        self._check(self.lib.sj_prof_read(self.ctx, KERNEL_KINDS[kind], ctypes.byref(n),
                                          ctypes.byref(ms), ctypes.byref(b)))
        return {"launches": int(n.value), "ms": float(ms.value), "bytes": float(b.value)}

    def prof_gaps(self):
        """Device idle ms after launches of each kernel class (see KERNEL_KINDS)."""
        g = (ctypes.c_double * 7)()
        self._check(self.lib.sj_prof_gaps(self.ctx, g))
        return {k: float(g[v]) for k, v in KERNEL_KINDS.items()}

    def selftest_wait_timeout(self) -> int:
        """Make one bounded device wait run out; returns the status (4 = timeout)."""
        return int(self.lib.sj_selftest_wait_timeout(self.ctx))

    def graphs_enable(self, on: bool = True):
        """Capture (and replay) CUDA graphs of repeated sieve_join shapes."""
        self._check(self.lib.sj_graphs_enable(self.ctx, 1 if on else 0))

    def graph_stats(self):
        """sj_sieve_join CUDA-graph replays, captures, failed captures and the
        reason of the last failure."""
        r, c_, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        why = ctypes.create_string_buffer(512)
        self._check(self.lib.sj_graph_stats(self.ctx, ctypes.byref(r), ctypes.byref(c_), ctypes.byref(f),
                                            why, 512))
        return {"replays": int(r.value), "captures": int(c_.value), "failures": int(f.value),
                "last_failure": why.value.decode()}

    def counters(self):
        """Kernel launches, host-to-device and device-to-host bytes since the
        last prof_reset."""
        n, h2d, d2h = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.sj_counters(self.ctx, ctypes.byref(n), ctypes.byref(h2d),
                                         ctypes.byref(d2h)))
        return {"launches": int(n.value), "h2d_bytes": int(h2d.value), "d2h_bytes": int(d2h.value)}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Query server with continuous batching over `nslots` workers (one CUDA
    stream each) and a device cache of reusable leaf filters (Sec. 2.3).
    ``batch`` > 1: a worker takes up to that many queued queries at once and
    prunes them in one batched call (lock-step launches), then joins each;
    queries over more than ``batch_max_rows`` rows (0 = no limit) run alone."""

    def __init__(self, device: int = 0, nslots: int = 4, hbm_budget: int = 0, passes=FWD_BWD,
                 cache_filters: bool = True, bits_per_key=8, k=3, layout=REGBLOCKED32, seed=0,
                 batch: int = 0, batch_max_rows: int = 0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("sievejoin needs a CUDA GPU; none is visible")
        self.lib = load_library()
        self.device = int(device)
        self._keep = []
        opts = ServerOpts(self.device, int(nslots), int(hbm_budget), int(passes),
                          1 if cache_filters else 0, _params(bits_per_key, k, layout, seed),
                          int(batch), 0, int(batch_max_rows))
        h = ctypes.c_void_p()
        st = self.lib.sj_server_create(ctypes.byref(h), ctypes.byref(opts))
        if st != 0:
            raise SieveJoinError(st, "sj_server_create failed")
        self.srv = h

    def add_relation(self, cols) -> int:
        """Register device int32 columns (torch CUDA tensors, kept alive here)."""
        ptrs = (ctypes.c_void_p * len(cols))(*[c.data_ptr() for c in cols])
        rid = ctypes.c_int32()
        st = self.lib.sj_server_add_relation(self.srv, len(cols), ptrs, len(cols[0]), ctypes.byref(rid))
        if st != 0:
            raise SieveJoinError(st, "sj_server_add_relation failed")
        self._keep.append(cols)
        return int(rid.value)

    @staticmethod
    def make_query(rel_ids, edges, preds=None, terms=(), root=-1) -> Query:
        q = Query()
        q.nrel = len(rel_ids)
        q.root = int(root)
        for i, r in enumerate(rel_ids):
            q.rel[i] = int(r)
            p = preds[i] if preds is not None else None
            q.preds[i] = _pred(p) if p is not None else Pred(-1, 0, 0)
        for e, ed in enumerate(edges):
            q.edges[e] = Edge(*map(int, ed))
        q.nterms = len(terms)
        for t, tr in enumerate(terms):
            q.terms[t] = ColRef(int(tr[0]), int(tr[1]), int(tr[2]) if len(tr) > 2 else 0, 0)
        return q

    def submit(self, rel_ids, edges, preds=None, terms=(), root=-1) -> int:
        q = self.make_query(rel_ids, edges, preds, terms, root)
        t = ctypes.c_uint64()
        st = self.lib.sj_server_submit(self.srv, ctypes.byref(q), ctypes.byref(t))
        if st != 0:
            raise SieveJoinError(st, "sj_server_submit rejected the query")
        return int(t.value)

    def poll(self, max_n: int = 4096, wait_ms: int = 0):
        buf = (Completion * max_n)()
        n = ctypes.c_int()
        self.lib.sj_server_poll(self.srv, buf, max_n, ctypes.byref(n), int(wait_ms))
        return [{"ticket": int(c.ticket), "status": int(c.status), "count": int(c.count),
                 "sum": int(c.sum), "cache_hits": int(c.cache_hits), "submit_ms": c.submit_ms,
                 "start_ms": c.start_ms, "done_ms": c.done_ms} for c in buf[:n.value]]

    def stats(self):
        s = ServerStats()
        self.lib.sj_server_stats_get(self.srv, ctypes.byref(s))
        return {f: int(getattr(s, f)) for f, _ in ServerStats._fields_ if f != "reserved"}

    def close(self):
        if getattr(self, "srv", None):
            self.lib.sj_server_destroy(self.srv)
            self.srv = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workload_path(ctx: Context, w: dict, where: str = "host"):
    """Load a workload dict (see ``inputs``) into device relations."""
    return [ctx.load_relation(r, where=where) for r in w["rels"]]
