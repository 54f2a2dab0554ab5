"""CPU oracle for the sieved multi-way join -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library never does,
and the two share no code: the oracle is plain numpy plus a small plain-C
library (``sj_oracle.c``) for the join loops.

Contents, each following the passage named in its docstring:

* ``fmix64``, ``bloom_*``   -- the Bloom filter (Sec. 1; Sec. 2.1 step 1 and 3)
  under this project's reading of the unspecified hash family and layout.
* ``filter_insert``         -- insert maintenance of a built filter (Sec. 2.4).
* ``sieve``, ``sieve_path`` -- the pruning phase (Sec. 2.2): filters are built
  along the join tree and each relation keeps the tuples whose join keys pass
  the incoming filters; first toward the root, then back.
* ``hash_join``             -- the enumeration phase (Sec. 2.2): an ordinary
  left-deep binary hash join; COUNT / SUM(int64) / materialised tuples.
* ``nested_loop``           -- brute-force enumeration of the same join.
* ``agg_propagation``       -- a second exact method: per-key (count, sum)
  messages pushed toward the root of the join tree (Yannakakis-style counting).
* ``chain_agg``             -- the same counting for many chain queries over one
  relation pool, with dense per-key messages in C (checks served results).

Parity status: every function here is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (brute force, closed forms, invariants and
statistical bounds); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from collections import deque

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC_PATH = os.path.join(_HERE, "sj_oracle.c")
_lib = None

REG32 = 0
BLOCKED256 = 1
CLASSIC = 2
COUNT_SUM = 0
MATERIALIZE = 1
FWD_BWD = 0
BWD_ONLY = 1
NO_SIEVE = 2

_U64 = np.uint64
_MASK64 = (1 << 64) - 1


# ----------------------------------------------------------------------------- build
def build_lib(force: bool = False) -> str:
    """Compile ``sj_oracle.c`` into ``liboracle.so`` with gcc (plain -O2)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC_PATH):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC_PATH])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.orc_join_pairs_count.restype = i64
        lib.orc_join_pairs_count.argtypes = [P, i64, P, i64]
        lib.orc_join_pairs_fill.restype = ctypes.c_int
        lib.orc_join_pairs_fill.argtypes = [P, i64, P, i64, P, P]
        lib.orc_join_agg.restype = ctypes.c_int
        lib.orc_join_agg.argtypes = [P, i64, P, P, i64, P, P]
        lib.orc_set_threads.restype = None
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_get_threads.restype = ctypes.c_int
        lib.orc_nested_loop.restype = ctypes.c_int
        lib.orc_nested_loop.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, P, P,
                                        ctypes.c_int, P, P]
        lib.orc_chain_agg.restype = ctypes.c_int
        lib.orc_chain_agg.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, i64, P, P]
        _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Probe threads of the C join levels (1 = serial; the build stays
    serial).  Results do not depend on it."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


# ----------------------------------------------------------------------------- hashing
def fmix64(x) -> np.ndarray:
    """MurmurHash3's 64-bit finaliser (public domain), elementwise on uint64.

    The paper leaves the Bloom filter's hash family open (it cites Kirsch and
    Mitzenmacher, Sec. 1); this project reads it as one 64-bit mix per key
    from which all bit positions are sliced.
    """
    x = np.asarray(x, dtype=np.uint64).copy()
    x ^= x >> _U64(33)
    x *= _U64(0xFF51AFD7ED558CCD)
    x ^= x >> _U64(33)
    x *= _U64(0xC4CEB9FE1A85EC53)
    x ^= x >> _U64(33)
    return x


def key_hash(keys: np.ndarray, seed: int) -> np.ndarray:
    """h = fmix64(uint32(key) xor seed) -- the per-key hash of every filter."""
    k = np.asarray(keys, dtype=np.int32).view(np.uint32).astype(np.uint64)
    return fmix64(k ^ _U64(seed & _MASK64))


# ----------------------------------------------------------------------------- Bloom filter
def bloom_nblocks(n_inserted: int, bits_per_key: int) -> int:
    """Number of 256-bit blocks: ceil(bits_per_key * n / 256), at least one.

    The paper sizes Bloomjoin's filter at one bit per tuple (Sec. 2.1 step 2);
    the bits per key are a parameter here, n counts the rows inserted.
    """
    return max(1, -(-(int(bits_per_key) * int(n_inserted)) // 256))


def bloom_positions(h: np.ndarray, nblocks: int, k: int, layout: int):
    """(word index, bit mask) arrays, one pair per hash function i < k.

    REG32 (register-blocked): all k bits of a key fall in one 32-bit word,
    word = ((h >> 32) * nwords) >> 32 with nwords = 8 * nblocks, and bit
    i = (h >> 5i) & 31.
    BLOCKED256: the key's block is ((h >> 32) * nblocks) >> 32 and its bits are
    the bytes (h >> 8i) & 255 inside that 256-bit block (eight uint32 words).
    CLASSIC: bit g_i = (h1 + i*h2) mod m over the whole m = 256*nblocks bits,
    with h1 = low 32 bits of h and h2 = high 32 bits of h forced odd (double
    hashing of Kirsch and Mitzenmacher, cited in Sec. 1).
    """
    out = []
    if layout == REG32:
        word = ((h >> _U64(32)) * _U64(8 * nblocks)) >> _U64(32)
        for i in range(k):
            bit = (h >> _U64(5 * i)) & _U64(31)
            out.append((word.astype(np.int64), (_U64(1) << bit).astype(np.uint32)))
    elif layout == BLOCKED256:
        blk = ((h >> _U64(32)) * _U64(nblocks)) >> _U64(32)
        for i in range(k):
            bit = (h >> _U64(8 * i)) & _U64(255)
            word = blk * _U64(8) + (bit >> _U64(5))
            out.append((word.astype(np.int64), (_U64(1) << (bit & _U64(31))).astype(np.uint32)))
    elif layout == CLASSIC:
        m = _U64(256 * nblocks)
        h1 = h & _U64(0xFFFFFFFF)
        h2 = (h >> _U64(32)) | _U64(1)
        for i in range(k):
            g = (h1 + _U64(i) * h2) % m
            out.append(((g >> _U64(5)).astype(np.int64), (_U64(1) << (g & _U64(31))).astype(np.uint32)))
    else:
        raise ValueError("unknown layout")
    return out


def bloom_build(keys: np.ndarray, bits_per_key: int = 8, k: int = 3,
                layout: int = REG32, seed: int = 0, nblocks: int = None) -> dict:
    """Build a filter: set every hash position of every key (Sec. 2.1 step 1).
    ``nblocks`` fixes the size instead of deriving it from the key count."""
    keys = np.asarray(keys, dtype=np.int32)
    if nblocks is None:
        nblocks = bloom_nblocks(len(keys), bits_per_key)
    words = np.zeros(nblocks * 8, dtype=np.uint32)
    h = key_hash(keys, seed)
    for word, mask in bloom_positions(h, nblocks, k, layout):
        np.bitwise_or.at(words, word, mask)
    return {"words": words, "nblocks": nblocks, "k": int(k), "layout": int(layout),
            "seed": int(seed), "n_inserted": int(len(keys)), "bits_per_key": int(bits_per_key)}


def bloom_contains(f: dict, keys: np.ndarray) -> np.ndarray:
    """Membership test: a key passes iff all of its k bits are set (Sec. 2.1 step 3)."""
    keys = np.asarray(keys, dtype=np.int32)
    h = key_hash(keys, f["seed"])
    ok = np.ones(len(keys), dtype=bool)
    for word, mask in bloom_positions(h, f["nblocks"], f["k"], f["layout"]):
        ok &= (f["words"][word] & mask) != 0
    return ok


INSERT_GATED, INSERT_CONTAINED, INSERT_NEW = 0, 1, 2


def filter_insert(f: dict, cols, key_col: int, gates=()):
    """Insert maintenance (Sec. 2.4): new tuples of the relation whose filter
    ``f`` was built.  A tuple first meets the filters the relation receives
    from its other neighbours (``gates``: (column, filter) pairs): one that
    fails any of them cannot join and is dropped (INSERT_GATED).  A tuple
    whose key the filter already contains needs no update (INSERT_CONTAINED).
    Any other tuple's key bits are set (INSERT_NEW): the filter changed, and
    that tuple is the one to follow to the adjacent relations.  Containment is
    judged against the filter as it was before the call, so the outcome does
    not depend on the order of the new tuples.  The filter keeps its size.
    Returns (new filter dict, status array of int8)."""
    n = len(cols[0]) if cols else 0
    passes = np.ones(n, dtype=bool)
    for col, g in gates:
        passes &= bloom_contains(g, cols[col])
    keys = np.asarray(cols[key_col], dtype=np.int32)
    contained = bloom_contains(f, keys)
    status = np.full(n, INSERT_GATED, dtype=np.int8)
    status[passes & contained] = INSERT_CONTAINED
    new = passes & ~contained
    status[new] = INSERT_NEW
    words = f["words"].copy()
    h = key_hash(keys[new], f["seed"])
    for word, mask in bloom_positions(h, f["nblocks"], f["k"], f["layout"]):
        np.bitwise_or.at(words, word, mask)
    out = dict(f, words=words, n_inserted=f["n_inserted"] + int(new.sum()))
    return out, status


# ----------------------------------------------------------------------------- selection / sieve
def select(cols, pred):
    """Rows with lo <= cols[col] < hi, in input order (the query's range predicate)."""
    if pred is None:
        return [np.asarray(c, dtype=np.int32) for c in cols]
    c, lo, hi = pred
    keep = (cols[c] >= lo) & (cols[c] < hi)
    return [np.asarray(x, dtype=np.int32)[keep] for x in cols]


def sieve(cols, probes):
    """Keep, in input order, the rows whose probed keys pass every filter.

    ``probes`` is a list of (column, filter).  This is one pruning step of
    Sec. 2.2: a relation receives Bloom filters from its neighbours and keeps
    only the tuples that can still join (no false negatives).
    """
    n = len(cols[0]) if cols else 0
    keep = np.ones(n, dtype=bool)
    for col, f in probes:
        keep &= bloom_contains(f, cols[col])
    return [np.asarray(x, dtype=np.int32)[keep] for x in cols]


def tree_of(nrel, edges, root):
    """Parent / children / post-order / pre-order of the join tree rooted at ``root``.

    Children are visited in edge order; the sieve result does not depend on it.
    """
    adj = [[] for _ in range(nrel)]
    for e, (a, ca, b, cb) in enumerate(edges):
        adj[a].append((b, e))
        adj[b].append((a, e))
    parent = [None] * nrel
    pedge = [None] * nrel
    children = [[] for _ in range(nrel)]
    seen = [False] * nrel
    seen[root] = True
    pre = []
    dq = deque([root])
    order_bfs = []
    while dq:
        v = dq.popleft()
        order_bfs.append(v)
        for (u, e) in adj[v]:
            if not seen[u]:
                seen[u] = True
                parent[u] = v
                pedge[u] = e
                children[v].append(u)
                dq.append(u)
    if not all(seen) or len(edges) != nrel - 1:
        raise ValueError("join graph is not a tree")

    def _pre(v):
        pre.append(v)
        for c in children[v]:
            _pre(c)
    _pre(root)
    post = []

    def _post(v):
        for c in children[v]:
            _post(c)
        post.append(v)
    _post(root)
    return parent, pedge, children, post, pre


def edge_col(edges, e, rel):
    a, ca, b, cb = edges[e]
    return ca if a == rel else cb


def sieve_path(w: dict, passes: int = FWD_BWD, bits_per_key: int = 8, k: int = 3,
               layout: int = REG32, seed: int = 0):
    """The pruning phase of Sec. 2.2 over a tree-shaped join.

    Predicates are applied first.  Pass 1 ("forward", R1 -> Rn for a chain
    whose root is its last relation) walks the tree from the leaves to the
    root: a relation is sieved by the filters of all its children and then
    builds, from its surviving tuples only, the filter it sends to its parent.
    Pass 2 ("backward", Rn -> R1, the paper's one-pass backward pruning) walks
    from the root to the leaves: each relation is sieved by its parent's
    filter, built from the parent's surviving tuples.  ``BWD_ONLY`` runs pass 2
    alone; ``NO_SIEVE`` applies the predicates only.

    Returns (sieved relations, steps) where steps lists
    (kind, rel, rows_in, rows_out) for every select / sieve step.
    """
    nrel = len(w["rels"])
    edges = w["edges"]
    cur = [select(w["rels"][i], w["preds"][i]) for i in range(nrel)]
    steps = []
    for i in range(nrel):
        if w["preds"][i] is not None:
            steps.append(("select", i, len(w["rels"][i][0]), len(cur[i][0])))
    if passes == NO_SIEVE or nrel == 1:
        return cur, steps
    parent, pedge, children, post, pre = tree_of(nrel, edges, w["root"])
    fp = dict(bits_per_key=bits_per_key, k=k, layout=layout, seed=seed)

    def step(v, probes, tag):
        n0 = len(cur[v][0])
        cur[v] = sieve(cur[v], probes)
        steps.append((tag, v, n0, len(cur[v][0])))

    if passes == FWD_BWD:
        up = {}
        for v in post:
            if children[v]:
                step(v, [(edge_col(edges, pedge[c], v), up[c]) for c in children[v]], "fwd")
            if parent[v] is not None:
                up[v] = bloom_build(cur[v][edge_col(edges, pedge[v], v)], **fp)
    down = {}
    for v in pre:
        if parent[v] is not None:
            step(v, [(edge_col(edges, pedge[v], v), down[v])], "bwd")
        for c in children[v]:
            down[c] = bloom_build(cur[v][edge_col(edges, pedge[c], v)], **fp)
    return cur, steps


# ----------------------------------------------------------------------------- joins
def join_order(nrel, edges):
    """Left-deep order: start at relation 0, then repeatedly the lowest-index
    relation adjacent to the joined set, with the edge that connects it."""
    joined = [0]
    inset = {0}
    plan = []
    while len(joined) < nrel:
        best = None
        for e, (a, ca, b, cb) in enumerate(edges):
            for (x, cx, y, cy) in ((a, ca, b, cb), (b, cb, a, ca)):
                if x in inset and y not in inset and (best is None or y < best[0]):
                    best = (y, cy, x, cx)
        if best is None:
            raise ValueError("join graph is not connected")
        plan.append(best)  # (new rel, its key col, joined rel, its key col)
        joined.append(best[0])
        inset.add(best[0])
    return plan


def _term_values(cols, col, wide):
    if wide:
        lo = cols[col].view(np.uint32).astype(np.uint64)
        hi = cols[col + 1].view(np.uint32).astype(np.uint64)
        return lo | (hi << _U64(32))
    return cols[col].astype(np.int64).view(np.uint64)


def _rel_sum(cols, rel, terms):
    n = len(cols[0]) if cols else 0
    v = np.zeros(n, dtype=np.uint64)
    for (r, c, wide) in terms:
        if r == rel:
            v += _term_values(cols, c, wide)
    return v


def _u128(lo, hi):
    return int(lo) | (int(hi) << 64)


def hash_join(w: dict, rels=None, mode: int = COUNT_SUM, refs=None, presieved: bool = False):
    """The enumeration phase (Sec. 2.2): a left-deep binary hash join.

    ``rels`` defaults to the workload's relations; unless ``presieved`` the
    range predicates are applied first.  COUNT_SUM returns
    {"count": int (exact), "sum": int in [0, 2^64), "overflow": bool};
    MATERIALIZE returns {"count": n, "cols": [np.int32 ...]} with one output
    column per (rel, col) in ``refs`` (default: every column of every
    relation, relation by relation).
    """
    lib = _load()
    nrel = len(w["rels"])
    if rels is None:
        rels = w["rels"]
    if not presieved:
        rels = [select(rels[i], w["preds"][i]) for i in range(nrel)]
    rels = [[np.ascontiguousarray(c, dtype=np.int32) for c in r] for r in rels]
    terms = list(w["sum"]) if refs is None and mode == COUNT_SUM else (refs or [])
    if mode == MATERIALIZE and refs is None:
        terms = [(r, c, 0) for r in range(nrel) for c in range(len(rels[r]))]
    plan = join_order(nrel, w["edges"])
    # columns each later level still needs
    inter = {(0, c): rels[0][c] for c in range(len(rels[0]))}
    psum = _rel_sum(rels[0], 0, terms) if mode == COUNT_SUM else None
    for L, (i, ci, j, cj) in enumerate(plan):
        pk = np.ascontiguousarray(inter[(j, cj)])
        bk = rels[i][ci]
        last = (L == len(plan) - 1)
        if last and mode == COUNT_SUM:
            bval = _rel_sum(rels[i], i, terms)
            out = np.zeros(3, dtype=np.uint64)
            psum_c = np.ascontiguousarray(psum)
            if lib.orc_join_agg(_ptr(pk), len(pk), _ptr(psum_c), _ptr(bk), len(bk),
                                _ptr(bval), _ptr(out)):
                raise MemoryError("oracle join")
            cnt = _u128(out[0], out[1])
            return {"count": cnt, "sum": int(out[2]), "overflow": cnt >= (1 << 63)}
        total = lib.orc_join_pairs_count(_ptr(pk), len(pk), _ptr(bk), len(bk))
        if total < 0:
            raise MemoryError("oracle join")
        pi = np.empty(total, dtype=np.int64)
        pj = np.empty(total, dtype=np.int64)
        if lib.orc_join_pairs_fill(_ptr(pk), len(pk), _ptr(bk), len(bk), _ptr(pi), _ptr(pj)):
            raise MemoryError("oracle join")
        new = {key: col[pi] for key, col in inter.items()}
        for c in range(len(rels[i])):
            new[(i, c)] = rels[i][c][pj]
        if psum is not None:
            psum = psum[pi] + _rel_sum(rels[i], i, terms)[pj]
        inter = new
    if mode == COUNT_SUM:  # a single relation
        cnt = len(rels[0][0]) if rels[0] else 0
        return {"count": cnt, "sum": int(np.sum(psum, dtype=np.uint64)) if cnt else 0,
                "overflow": False}
    cols = [inter[(r, c)] for (r, c, _w) in terms]
    n = len(cols[0]) if cols else 0
    return {"count": n, "cols": cols}


def nested_loop(w: dict, terms=None):
    """Brute-force COUNT / SUM: every combination of rows, every predicate and
    edge checked (tiny inputs only).  Returns {"count", "sum", "overflow"}."""
    lib = _load()
    nrel = len(w["rels"])
    rels = [[np.ascontiguousarray(c, dtype=np.int32) for c in r] for r in w["rels"]]
    terms = w["sum"] if terms is None else terms
    nrows = np.array([len(r[0]) for r in rels], dtype=np.int64)
    coloff = np.zeros(nrel, dtype=np.int32)
    ptrs = []
    for i, r in enumerate(rels):
        coloff[i] = len(ptrs)
        ptrs.extend(c.ctypes.data for c in r)
    colptrs = np.array(ptrs, dtype=np.uint64)
    edges = np.array([x for e in w["edges"] for x in e] or [0], dtype=np.int32)
    preds = np.array([x for p in w["preds"] for x in (p if p is not None else (-1, 0, 0))],
                     dtype=np.int32)
    agg = np.array([x for t in terms for x in t] or [0], dtype=np.int32)
    out = np.zeros(3, dtype=np.uint64)
    if lib.orc_nested_loop(nrel, _ptr(nrows), _ptr(colptrs), _ptr(coloff), len(w["edges"]),
                           _ptr(edges), _ptr(preds), len(terms), _ptr(agg), _ptr(out)):
        raise MemoryError("oracle nested loop")
    cnt = _u128(out[0], out[1])
    return {"count": cnt, "sum": int(out[2]), "overflow": cnt >= (1 << 63)}


def agg_propagation(w: dict, rels=None, presieved: bool = False):
    """Exact COUNT / SUM by pushing per-key (count, sum) pairs to relation 0.

    For a row with value v and child messages (c_j, s_j) at its join keys,
    the row's pair is the product (1, v) (x) (c_1, s_1) (x) ... with
    (c, s) (x) (c', s') = (c c', s c' + s' c); a relation's message to its
    parent adds the pairs of its rows per parent-join key.  Counts and sums
    are kept mod 2^64 with a float64 shadow of the count for overflow.
    """
    nrel = len(w["rels"])
    if rels is None:
        rels = w["rels"]
    if not presieved:
        rels = [select(rels[i], w["preds"][i]) for i in range(nrel)]
    terms = w["sum"]
    parent, pedge, children, post, pre = tree_of(nrel, w["edges"], 0)
    msgs = {}
    for v in post:
        cols = rels[v]
        n = len(cols[0]) if cols else 0
        c = np.ones(n, dtype=np.uint64)
        s = _rel_sum(cols, v, terms)
        cf = np.ones(n, dtype=np.float64)
        for ch in children[v]:
            K, C, S, CF = msgs.pop(ch)
            keys = cols[edge_col(w["edges"], pedge[ch], v)]
            idx = np.searchsorted(K, keys)
            idx_c = np.minimum(idx, max(len(K) - 1, 0))
            found = (len(K) > 0) & (K[idx_c] == keys) if len(K) else np.zeros(n, dtype=bool)
            c2 = np.where(found, C[idx_c] if len(K) else 0, 0).astype(np.uint64)
            s2 = np.where(found, S[idx_c] if len(K) else 0, 0).astype(np.uint64)
            cf2 = np.where(found, CF[idx_c] if len(K) else 0.0, 0.0)
            c, s = c * c2, s * c2 + s2 * c
            cf = cf * cf2
        if parent[v] is None:
            cnt = int(np.sum(c, dtype=np.uint64))
            tot = int(np.sum(s, dtype=np.uint64))
            cntf = float(np.sum(cf))
            return {"count": cnt, "sum": tot, "overflow": cntf >= 2.0 ** 63,
                    "count_approx": cntf}
        keys = cols[edge_col(w["edges"], pedge[v], v)]
        K, inv = np.unique(keys, return_inverse=True)
        C = np.zeros(len(K), dtype=np.uint64)
        S = np.zeros(len(K), dtype=np.uint64)
        CF = np.zeros(len(K), dtype=np.float64)
        np.add.at(C, inv, c)
        np.add.at(S, inv, s)
        np.add.at(CF, inv, cf)
        msgs[v] = (K, C, S, CF)
    raise AssertionError("unreachable")


class ChainPool:
    """A relation pool checked once for ``chain_agg``: two int32 columns per
    relation, every key in [0, domain)."""

    def __init__(self, pool, domain: int):
        if not 0 < domain < (1 << 31):
            raise ValueError("domain must be in 1 .. 2^31 - 1")
        self.domain = int(domain)
        self.x = [np.ascontiguousarray(r[0], dtype=np.int32) for r in pool]
        self.y = [np.ascontiguousarray(r[1], dtype=np.int32) for r in pool]
        for x, y in zip(self.x, self.y):
            if len(x) != len(y):
                raise ValueError("pool relations need two columns of equal length")
            for c in (x, y):
                if len(c) and (int(c.min()) < 0 or int(c.max()) >= domain):
                    raise ValueError("pool key outside [0, domain)")
        self.n = np.asarray([len(x) for x in self.x], dtype=np.int64)
        self.px = np.asarray([x.ctypes.data for x in self.x], dtype=np.uint64)
        self.py = np.asarray([y.ctypes.data for y in self.y], dtype=np.uint64)

    def __len__(self):
        return len(self.x)


def chain_agg(pool, queries, domain: int = None):
    """COUNT(*) and SUM(first.x + last.y) of chain queries over a pool of
    two-column relations (x, y), the same counting as ``agg_propagation``
    with per-key messages held densely over the keys [0, domain) (C, over the
    oracle's threads, one query per thread at a time).

    ``pool``: a ``ChainPool`` or a list of relations (checked here against
    ``domain``).  A query is a dict with ``rels`` (pool indices r_0 .. r_k,
    joined on r_i.y = r_{i+1}.x as ``edges`` (i, 1, i + 1, 0) say), ``preds``
    (a range (0, lo, hi) on r_0.x, or None; nothing on the others) and
    ``sum`` = [(0, 0, 0), (k, 1, 0)].  Anything else raises ValueError.
    Returns one {"count", "sum"} per query, both modulo 2^64."""
    if not isinstance(pool, ChainPool):
        pool = ChainPool(pool, domain)
    qoff, qrel, qlo, qhi = [0], [], [], []
    for q in queries:
        rels = list(q["rels"])
        k = len(rels) - 1
        if k < 0 or any(r < 0 or r >= len(pool) for r in rels):
            raise ValueError("bad relation index")
        if [tuple(e) for e in q["edges"]] != [(i, 1, i + 1, 0) for i in range(k)]:
            raise ValueError("not a chain on r_i.y = r_{i+1}.x")
        preds = q.get("preds") or [None] * (k + 1)
        if any(p is not None for p in preds[1:]):
            raise ValueError("predicates only on r_0")
        p0 = preds[0]
        if p0 is not None and p0[0] != 0:
            raise ValueError("predicate only on r_0.x")
        if [tuple(t) for t in q["sum"]] != [(0, 0, 0), (k, 1, 0)]:
            raise ValueError("SUM terms must be r_0.x and r_k.y")
        # no predicate: [0, domain) lies inside [-2^31, 2^31 - 1)
        lo, hi = (int(p0[1]), int(p0[2])) if p0 is not None else (-(1 << 31), (1 << 31) - 1)
        qrel += rels
        qoff.append(len(qrel))
        qlo.append(lo)
        qhi.append(hi)
    nq = len(queries)
    if nq == 0:
        return []
    lib = _load()
    qoff = np.asarray(qoff, dtype=np.int32)
    qrel = np.asarray(qrel, dtype=np.int32)
    qlo = np.asarray(qlo, dtype=np.int32)
    qhi = np.asarray(qhi, dtype=np.int32)
    cnt = np.zeros(nq, dtype=np.uint64)
    tot = np.zeros(nq, dtype=np.uint64)
    if lib.orc_chain_agg(nq, _ptr(qoff), _ptr(qrel), _ptr(qlo), _ptr(qhi), _ptr(pool.n),
                         _ptr(pool.px), _ptr(pool.py), pool.domain, _ptr(cnt), _ptr(tot)):
        raise MemoryError("orc_chain_agg: message buffers")
    return [{"count": int(c), "sum": int(t)} for c, t in zip(cnt, tot)]


def semijoin_reduction(w: dict, rels=None):
    """Exact full reduction: the rows of each relation that occur in at least
    one result tuple (computed by materialising row ids through the join)."""
    nrel = len(w["rels"])
    if rels is None:
        rels = [select(w["rels"][i], w["preds"][i]) for i in range(nrel)]
    ids = []
    ext = []
    for i, r in enumerate(rels):
        n = len(r[0]) if r else 0
        ids.append(np.arange(n, dtype=np.int32))
        ext.append(list(r) + [ids[-1]])
    ww = dict(w, rels=ext, preds=[None] * nrel)
    refs = [(i, len(ext[i]) - 1, 0) for i in range(nrel)]
    res = hash_join(ww, rels=ext, mode=MATERIALIZE, refs=refs, presieved=True)
    keep = []
    for i in range(nrel):
        rows = np.unique(res["cols"][i]) if res["count"] else np.zeros(0, dtype=np.int32)
        keep.append([np.asarray(c)[rows] for c in rels[i]])
    return keep


def triangle_counts(src, dst, cuts):
    """Cyclic triangle query E(a,b) |x| E(b,c) |x| E(c,a) (Sec. 2.3 cyclic joins):
    ordered (a, b, c) with edges a->b, b->c and c->a, counted per subquery
    cuts[i] <= a < cuts[i+1].  Plain definition: a binary hash join E |x| E on
    b gives every wedge (a, b, c); a wedge closes when (c, a) is an edge.
    Returns an int array of per-subquery counts."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    total = lib.orc_join_pairs_count(_ptr(dst), len(dst), _ptr(src), len(src))
    if total < 0:
        raise MemoryError("oracle join")
    pi = np.empty(total, dtype=np.int64)  # wedge: edge pi = (a, b), edge pj = (b, c)
    pj = np.empty(total, dtype=np.int64)
    if lib.orc_join_pairs_fill(_ptr(dst), len(dst), _ptr(src), len(src), _ptr(pi), _ptr(pj)):
        raise MemoryError("oracle join")
    a = src[pi].astype(np.int64)
    c = dst[pj].astype(np.int64)
    edges = np.sort(_pair_key(src, dst))
    probe = _pair_key(c, a)
    pos = np.minimum(np.searchsorted(edges, probe), max(len(edges) - 1, 0))
    closes = edges[pos] == probe if len(edges) else np.zeros(len(probe), dtype=bool)
    return np.bincount(_subquery(cuts, a[closes]), minlength=len(cuts) - 1).astype(np.int64)


def _pair_key(s, d):
    """One int64 per vertex pair (s, d), distinct for distinct pairs of int32
    ids: s in the high word, d's 32-bit pattern in the low word."""
    s = np.asarray(s, dtype=np.int64)
    d = np.asarray(d, dtype=np.int64)
    return (s << 32) | (d & 0xFFFFFFFF)


def _subquery(cuts, a):
    """Subquery of each vertex a: the i with cuts[i] <= a < cuts[i+1]; a below
    cuts[0] belongs to subquery 0 and a at or above cuts[-1] to the last."""
    sub = np.searchsorted(np.asarray(cuts, dtype=np.int64), a, side="right") - 1
    return np.clip(sub, 0, len(cuts) - 2)


def triangle_counts_for(src, dst, verts):
    """Ordered triangle counts restricted to a in `verts` (one count per vertex),
    by the same plain definition as triangle_counts: the wedges (a, b, c) from
    the edges leaving a, closed when (c, a) is an edge (membership by binary
    search in the sorted edge keys)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    edges = np.sort(_pair_key(src, dst))
    order = np.argsort(src, kind="stable")
    s_sorted = src[order]

    def is_edge(keys):
        i = np.minimum(np.searchsorted(edges, keys), len(edges) - 1)
        return edges[i] == keys

    out = []
    for a in verts:
        lo, hi = np.searchsorted(s_sorted, [a, a + 1])
        bs = dst[order[lo:hi]]
        total = 0
        for b in bs:
            l2, h2 = np.searchsorted(s_sorted, [b, b + 1])
            cs = dst[order[l2:h2]]
            total += int(is_edge(_pair_key(cs, a)).sum())
        out.append(total)
    return np.array(out, dtype=np.int64)
