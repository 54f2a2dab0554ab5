"""Batched pruning: sj_sieve_path_batch runs the pruning phases (Sec. 2.2) of
several queries in lock-step launches.  Every query's sieved relations (rows
and order) and step statistics must equal its own sj_sieve_path and the
oracle's sieve_path, whatever else is in the batch: trees of 1-5 relations,
empty relations, relations spanning many sieve chunks, predicates, handed-in
leaf filters (Sec. 2.3) and every filter layout.
"""
import numpy as np
import pytest

import oracle
import paper_2308_16370_b300 as sj
from paper_2308_16370_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    sj.load_library()
    c = sj.Context(0)
    yield c
    c.close()


def make_queries(seed, nq, max_rows=12_000):
    g = np.random.default_rng(seed)
    ws = []
    for q in range(nq):
        nrel = int(g.integers(1, 6))  # a star of 5: four children, the most a step probes
        sizes = g.integers(0, max_rows, nrel)
        if q % 5 == 1:
            sizes[int(g.integers(0, nrel))] = 0
        if q % 7 == 3:
            sizes[0] = 150_000  # many chunks
        w = inputs.random_tree_join(g, nrel, sizes, domain=int(g.integers(50, 6000)),
                                    star_like=bool(q % 3 == 0))
        ws.append(w)
    return ws


def check_batch(ctx, ws, passes, bpk, k, layout, seed, leaf=False):
    rels = [[ctx.load_relation(r, where="host") for r in w["rels"]] for w in ws]
    qs = []
    leaf_fs = []
    for w, rs in zip(ws, rels):
        q = {"rels": rs, "edges": w["edges"], "preds": w["preds"], "root": w["root"]}
        lf = None
        if leaf and len(rs) > 1:
            # leaves of the tree rooted at `root`: degree-1 positions other than it
            n = len(rs)
            root = w["root"] if w["root"] >= 0 else n - 1
            deg = np.zeros(n, dtype=int)
            col = {}
            for (a, ca, b, cb) in w["edges"]:
                deg[a] += 1
                deg[b] += 1
                col.setdefault(a, ca)
                col.setdefault(b, cb)
            lf = [None] * n
            for v in range(n):
                if deg[v] == 1 and v != root:
                    p = w["preds"][v]
                    lf[v] = ctx.build_filter(rs[v], col[v], pred=p, bits_per_key=bpk, k=k,
                                             layout=layout, seed=seed)
            q["leaf_filters"] = lf
        leaf_fs.append(lf)
        qs.append(q)
    out = ctx.sieve_path_batch(qs, passes=passes, bits_per_key=bpk, k=k, layout=layout, seed=seed)
    assert len(out) == len(ws)
    for w, rs, q, (sv, st) in zip(ws, rels, qs, out):
        alone, st1 = ctx.sieve_path(rs, w["edges"], w["preds"], w["root"], passes=passes,
                                    bits_per_key=bpk, k=k, layout=layout, seed=seed,
                                    leaf_filters=q.get("leaf_filters"))
        assert st["steps"] == st1["steps"]
        assert st["rows_final"] == st1["rows_final"]
        assert st["filter_bytes"] == st1["filter_bytes"]
        for a, b in zip(sv, alone):
            ga, gb = a.to_numpy(), b.to_numpy()
            assert all(np.array_equal(x, y) for x, y in zip(ga, gb))
        if not leaf:
            osv, osteps = oracle.sieve_path(w, passes=passes, bits_per_key=bpk, k=k, layout=layout,
                                            seed=seed)
            assert st["steps"] == [tuple(s) for s in osteps]
            for a, e in zip(sv, osv):
                got = a.to_numpy()
                assert all(np.array_equal(x, np.asarray(y, dtype=np.int32)) for x, y in zip(got, e))
    return out


@pytest.mark.parametrize("layout,k", [(sj.REGBLOCKED32, 3), (sj.REGBLOCKED32, 2), (sj.BLOCKED256, 4),
                                      (sj.CLASSIC, 5)])
@pytest.mark.parametrize("passes", [sj.FWD_BWD, sj.BWD_ONLY])
def test_batch_equals_alone_and_oracle(ctx, layout, k, passes):
    ws = make_queries(300 + layout * 10 + k, 12)
    check_batch(ctx, ws, passes, bpk=8, k=k, layout=layout, seed=layout + 1)


def test_batch_no_sieve_and_single_query(ctx):
    ws = make_queries(41, 5)
    check_batch(ctx, ws, sj.NO_SIEVE, bpk=8, k=3, layout=0, seed=0)
    check_batch(ctx, ws[:1], sj.FWD_BWD, bpk=8, k=3, layout=0, seed=0)


def test_batch_with_handed_in_leaf_filters(ctx):
    ws = make_queries(77, 10)
    check_batch(ctx, ws, sj.FWD_BWD, bpk=10, k=3, layout=0, seed=5, leaf=True)


def test_batch_of_serving_chains(ctx):
    """Chains of 2-6 relations over a shared pool, as the serving runtime
    batches them (the same relation in several queries of one batch)."""
    pool = inputs.serving_pool(nrel=8, min_rows=1_000, max_rows=300_000, domain=1 << 14, seed=12)
    qs = inputs.serving_queries([len(r[0]) for r in pool], 24, domain=1 << 14, seed=13)
    ws = [{"rels": [pool[r] for r in q["rels"]], "edges": q["edges"], "preds": q["preds"],
           "root": q["root"], "sum": q["sum"]} for q in qs]
    out = check_batch(ctx, ws, sj.FWD_BWD, bpk=8, k=3, layout=0, seed=0)
    # the join over the batch's sieved relations gives the oracle's COUNT and SUM
    for w, (sv, _) in zip(ws[:6], out[:6]):
        rels = [ctx.load_relation(r, where="host") for r in w["rels"]]
        res = ctx.join(rels, w["edges"], w["preds"], w["root"], inputs=sv, refs=w["sum"])
        exp = oracle.agg_propagation(w)
        assert (res["count"], res["sum"]) == (exp["count"], exp["sum"])


def test_batch_rejects_invalid_query_and_accepts_empty(ctx):
    ws = make_queries(5, 2)
    rels = [[ctx.load_relation(r, where="host") for r in w["rels"]] for w in ws]
    qs = [{"rels": rs, "edges": w["edges"], "preds": w["preds"], "root": w["root"]}
          for w, rs in zip(ws, rels)]
    assert ctx.sieve_path_batch([]) == []
    bad = dict(qs[0])
    bad["root"] = 17
    with pytest.raises(sj.SieveJoinError):
        ctx.sieve_path_batch([qs[1], bad])
    # the context stays usable
    out = ctx.sieve_path_batch(qs)
    assert len(out) == 2
