"""Seeded synthetic workloads for the sieved multi-way join.

This module only draws numbers: it holds none of the join, Bloom-filter or
sieve arithmetic, so both the CUDA path and the CPU oracle can take their
inputs from here without sharing any of the method's code.

A workload is a dict::

    {"name": str,
     "rels":  [ [np.int32 column, ...], ... ],       # columnar relations
     "edges": [ (rel_a, col_a, rel_b, col_b), ... ], # equality predicates
     "preds": [ None | (col, lo, hi), ... ],          # lo <= v < hi per relation
     "root":  int,                                   # sieve root (tree root)
     "sum":   [ (rel, col, wide), ... ]}             # SUM(int64) expression

``wide=1`` means the int64 value is stored as two int32 columns ``col``
(low word) and ``col+1`` (high word).

The join graphs are trees (chains and stars), as in the paper's acyclic
queries (Sec. 2.2, Sec. 3.1.1 and Sec. 3.1.2).
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


def chain_edges(nrel: int):
    """R_i.col1 = R_{i+1}.col0 for a chain of two-column relations."""
    return [(i, 1, i + 1, 0) for i in range(nrel - 1)]


def uniform_chain(nrel: int = 3, nrows: int = 100_000, domain: int = 50_000,
                  seed: int = 1, nrows_list=None) -> dict:
    """Chain R1(a,b) |x| R2(b,c) |x| ... with every column uniform in [0, domain).

    Default: the 3-way chain R(a,b) S(b,c) T(c,d) of 100k rows per relation
    over [0, 50000), SUM(a + d) over the result.
    """
    rels = []
    for i in range(nrel):
        n = int(nrows_list[i]) if nrows_list is not None else int(nrows)
        g = _rng(seed, i)
        rels.append([g.integers(0, domain, n, dtype=np.int32) for _ in range(2)])
    return {"name": f"chain{nrel}_uniform_n{nrows}_d{domain}", "rels": rels,
            "edges": chain_edges(nrel), "preds": [None] * nrel, "root": nrel - 1,
            "sum": [(0, 0, 0), (nrel - 1, 1, 0)]}


def zipf_ranks(g: np.random.Generator, n: int, domain: int, s: float) -> np.ndarray:
    """Ranks in [0, domain) with P(rank r) proportional to 1/(r+1)^s (inverse CDF)."""
    w = 1.0 / np.power(np.arange(1, domain + 1, dtype=np.float64), s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = g.random(n)
    r = np.searchsorted(cdf, u, side="right")
    return np.minimum(r, domain - 1).astype(np.int64)


def zipf_chain(nrel: int = 4, nrows: int = 10_000_000, domain: int = 5_000_000,
               s: float = 1.0, last_subset_frac: float = 0.01, payload_domain=None,
               seed: int = 2) -> dict:
    """4-way chain R1(a,k1) R2(k1,k2) R3(k2,k3) R4(k3,d) with Zipf(s) join keys.

    Every join column draws Zipf ranks that go through an independent seeded
    permutation of the key domain per (relation, column), so hot keys of
    different columns do not line up.  The last relation's join key is drawn
    from a seeded random subset of ``last_subset_frac`` of the domain, so most
    intermediate tuples of a plain binary plan die at the last level.  The
    payload columns a and d are uniform in [0, payload_domain).
    """
    pdom = domain if payload_domain is None else payload_domain
    rels = []
    for i in range(nrel):
        cols = []
        for c in range(2):
            g = _rng(seed, i, c)
            is_left_payload = (i == 0 and c == 0)
            is_right_payload = (i == nrel - 1 and c == 1)
            if is_left_payload or is_right_payload:
                cols.append(g.integers(0, pdom, nrows, dtype=np.int32))
                continue
            if i == nrel - 1 and c == 0:
                nsub = max(1, int(round(domain * last_subset_frac)))
                subset = g.permutation(domain)[:nsub]
                cols.append(subset[zipf_ranks(g, nrows, nsub, s)].astype(np.int32))
            else:
                perm = g.permutation(domain)
                cols.append(perm[zipf_ranks(g, nrows, domain, s)].astype(np.int32))
        rels.append(cols)
    return {"name": f"chain{nrel}_zipf{s}_n{nrows}_d{domain}", "rels": rels,
            "edges": chain_edges(nrel), "preds": [None] * nrel, "root": nrel - 1,
            "sum": [(0, 0, 0), (nrel - 1, 1, 0)]}


def freitag_rst(r: int, d: int, top: int = 10_000_000) -> dict:
    """The synthetic R, S, T benchmark of Sec. 3.1.1 (unary relations).

    R holds 1..top, S holds 1..(top+r)/2 and T holds (top-r)/2+1..top, every
    value repeated d times; R |x| S |x| T then has r distinct values, each
    repeated d^3 times.  (The printed lower end of T is read as exclusive, so
    that S and T share exactly r values.)
    """
    hi_s = (top + r) // 2
    lo_t = (top - r) // 2 + 1
    R = np.repeat(np.arange(1, top + 1, dtype=np.int32), d)
    S = np.repeat(np.arange(1, hi_s + 1, dtype=np.int32), d)
    T = np.repeat(np.arange(lo_t, top + 1, dtype=np.int32), d)
    return {"name": f"freitag_r{r}_d{d}_top{top}", "rels": [[R], [S], [T]],
            "edges": [(0, 0, 1, 0), (1, 0, 2, 0)], "preds": [None] * 3, "root": 2,
            "sum": [(0, 0, 0)]}


def star(nfact: int = 100_000_000, ndim: int = 4, dim_rows: int = 1_000_000,
         sel: float = 0.1, measure_hi: int = 1_000_000, seed: int = 3) -> dict:
    """Star join: fact(fk_1..fk_ndim, measure as int64 lo/hi words) and ndim dimensions.

    Dimension i is (pk, attr) with pk = row index 0..dim_rows-1 and attr
    uniform in [0, 1e6); its predicate keeps attr in [lo, lo + sel*1e6) with a
    seeded lo.  Foreign keys are uniform over [0, dim_rows); the measure is
    uniform in [0, measure_hi).  Relation 0 is the fact table and the root.
    """
    g = _rng(seed, 0)
    fact = [g.integers(0, dim_rows, nfact, dtype=np.int32) for _ in range(ndim)]
    meas = g.integers(0, measure_hi, nfact, dtype=np.int64)
    fact.append((meas & 0xFFFFFFFF).astype(np.uint32).view(np.int32))
    fact.append((meas >> 32).astype(np.int32))
    rels = [fact]
    preds = [None]
    edges = []
    attr_dom = 1_000_000
    width = int(round(sel * attr_dom))
    for i in range(ndim):
        gd = _rng(seed, 1 + i)
        pk = np.arange(dim_rows, dtype=np.int32)
        attr = gd.integers(0, attr_dom, dim_rows, dtype=np.int32)
        lo = int(gd.integers(0, attr_dom - width + 1))
        rels.append([pk, attr])
        preds.append((1, lo, lo + width))
        edges.append((0, i, 1 + i, 0))
    return {"name": f"star_f{nfact}_d{ndim}x{dim_rows}_sel{sel}", "rels": rels,
            "edges": edges, "preds": preds, "root": 0, "sum": [(0, ndim, 1)]}


def random_tree_join(g: np.random.Generator, nrel: int, nrows, domain: int,
                     ncols: int = 3, pred_prob: float = 0.3, star_like: bool = False) -> dict:
    """Small random tree-shaped join over int32 columns (for brute-force tests)."""
    rels = []
    for i in range(nrel):
        n = int(nrows[i]) if hasattr(nrows, "__len__") else int(nrows)
        rels.append([g.integers(0, domain, n, dtype=np.int32) for _ in range(ncols)])
    edges = []
    for i in range(1, nrel):
        j = 0 if star_like else int(g.integers(0, i))
        edges.append((j, int(g.integers(0, ncols)), i, int(g.integers(0, ncols))))
    preds = []
    for i in range(nrel):
        if g.random() < pred_prob:
            lo = int(g.integers(0, domain // 2 + 1))
            preds.append((int(g.integers(0, ncols)), lo, lo + max(1, domain // 2)))
        else:
            preds.append(None)
    sums = [(int(g.integers(0, nrel)), int(g.integers(0, ncols)), 0) for _ in range(2)]
    return {"name": "random_tree", "rels": rels, "edges": edges, "preds": preds,
            "root": int(g.integers(0, nrel)), "sum": sums}


def serving_pool_sizes(nrel: int = 40, min_rows: int = 10_000, max_rows: int = 50_000_000,
                       seed: int = 5) -> np.ndarray:
    """Row counts of the serving pool's relations (log-uniform in [min_rows, max_rows])."""
    g = _rng(seed, 0)
    return np.exp(g.uniform(np.log(min_rows), np.log(max_rows), nrel)).astype(np.int64)


def serving_pool(nrel: int = 40, min_rows: int = 10_000, max_rows: int = 50_000_000,
                 domain: int = 1 << 22, s: float = 0.8, seed: int = 5, device=None, only=None):
    """Resident relation pool for the serving workload: relations R_j(x, y)
    with log-uniform sizes in [min_rows, max_rows] and Zipf(s) keys over the
    domain, each column through its own seeded permutation.  ``device`` (a
    torch device) runs the inverse-CDF lookup and the permutation there: the
    same comparisons on the same float64 values, so the same columns, faster
    for pools of hundreds of millions of rows.  ``only`` (relation indices)
    generates just those relations, each as in the full pool (every relation
    draws from its own seeded stream); the others are None.  Returns numpy
    columns."""
    sizes = serving_pool_sizes(nrel, min_rows, max_rows, seed)
    w = 1.0 / np.power(np.arange(1, domain + 1, dtype=np.float64), s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cdf_t = None
    if device is not None:
        import torch
        cdf_t = torch.from_numpy(cdf).to(device)
    pool = []
    for j in range(nrel):
        if only is not None and j not in only:
            pool.append(None)
            continue
        cols = []
        for c in range(2):
            gj = _rng(seed, 1 + j, c)
            perm = gj.permutation(domain)
            u = gj.random(int(sizes[j]))
            if cdf_t is None:
                r = np.minimum(np.searchsorted(cdf, u, side="right"), domain - 1)
                cols.append(perm[r].astype(np.int32))
            else:
                import torch
                r = torch.searchsorted(cdf_t, torch.from_numpy(u).to(device), right=True)
                r.clamp_(max=domain - 1)
                col = torch.from_numpy(perm).to(device)[r].to(torch.int32)
                cols.append(col.cpu().numpy())
        pool.append(cols)
    return pool


def serving_queries(pool_sizes, nq: int, domain: int = 1 << 22, min_len: int = 2,
                    max_len: int = 6, ntemplates: int = 8, seed: int = 6):
    """Chain queries over a pool: R_{i}.y = R_{i+1}.x for 2..6 distinct relations,
    a range predicate on the first relation's x taken from `ntemplates` fixed
    ranges (so filters of repeated (relation, column, predicate) are reusable),
    COUNT(*) and SUM(first.x + last.y)."""
    g = _rng(seed, 0)
    npool = len(pool_sizes)
    width = domain // 4
    templates = [(int(t * (domain - width) // max(1, ntemplates - 1)),) for t in range(ntemplates)]
    qs = []
    for _ in range(nq):
        n = int(g.integers(min_len, min(max_len, npool) + 1))
        rels = [int(x) for x in g.choice(npool, n, replace=False)]
        lo = templates[int(g.integers(0, ntemplates))][0]
        preds = [(0, lo, lo + width)] + [None] * (n - 1)
        qs.append({"rels": rels, "edges": chain_edges(n), "preds": preds, "root": n - 1,
                   "sum": [(0, 0, 0), (n - 1, 1, 0)]})
    return qs


def rmat_edges(scale: int = 22, nedges: int = 50_000_000, a: float = 0.57, b: float = 0.19,
               c: float = 0.19, seed: int = 4):
    """Directed R-MAT graph on 2^scale vertices with exactly `nedges` distinct
    edges and no self-loops (edges drawn until that many distinct ones exist;
    the first distinct ones in draw order are kept).  Returns (src, dst) int32."""
    g = _rng(seed, 0)
    keys_seen = np.zeros(0, np.int64)
    order_seen = np.zeros(0, np.int64)
    drawn = 0
    while len(keys_seen) < nedges:
        m = int((nedges - len(keys_seen)) * 1.25) + 1024
        s = np.zeros(m, np.int64)
        d = np.zeros(m, np.int64)
        for lvl in range(scale):
            u = g.random(m)
            right = (u >= a) & (u < a + b) | (u >= a + b + c)
            down = u >= a + b
            s |= down.astype(np.int64) << lvl
            d |= right.astype(np.int64) << lvl
        keep = s != d
        k = (s[keep] << 32) | d[keep]
        allk = np.concatenate([keys_seen, k])
        allo = np.concatenate([order_seen, drawn + np.arange(len(k))])
        drawn += len(k)
        # distinct keys with the draw index of their first occurrence (stable sort)
        srt = np.argsort(allk, kind="stable")
        ks = allk[srt]
        first = np.ones(len(ks), dtype=bool)
        first[1:] = ks[1:] != ks[:-1]
        keys_seen, order_seen = ks[first], allo[srt][first]
    take = np.argsort(order_seen, kind="stable")[:nedges]
    k = keys_seen[take]
    return (k >> 32).astype(np.int32), (k & 0xFFFFFFFF).astype(np.int32)


def uneven_cuts(nvert: int, nsub: int = 64, seed: int = 4):
    """nsub + 1 increasing vertex cut points 0 = c_0 < ... < c_nsub = nvert,
    uneven: subquery sizes drawn log-uniform before normalising."""
    g = _rng(seed, 99)
    w = np.exp(g.uniform(0.0, 3.0, nsub))
    c = np.concatenate([[0.0], np.cumsum(w) / w.sum()]) * nvert
    cuts = np.unique(np.round(c).astype(np.int64))
    cuts[0], cuts[-1] = 0, nvert
    while len(cuts) < nsub + 1:  # tiny graphs: pad with distinct points
        extra = np.setdiff1d(np.arange(nvert + 1), cuts)[: nsub + 1 - len(cuts)]
        cuts = np.unique(np.concatenate([cuts, extra]))
    return cuts.astype(np.int32)
