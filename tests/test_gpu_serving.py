"""Serving: continuous batching over worker slots with a leaf-filter cache.

Every query's COUNT and SUM served in a mix of concurrent queries must equal
the same query run alone, and the CPU oracle; the filter cache must be hit for
repeated (relation, column, predicate) templates; a tiny memory budget must
serialise admission without changing any result.
"""
import numpy as np
import pytest

import oracle
import paper_2308_16370_b300 as sj
from paper_2308_16370_b300 import inputs

pytestmark = pytest.mark.gpu

DOMAIN = 1 << 14


@pytest.fixture(scope="module")
def pool():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    p = inputs.serving_pool(nrel=10, min_rows=2_000, max_rows=200_000, domain=DOMAIN, seed=11)
    return p, [[torch.from_numpy(c).cuda() for c in r] for r in p]


def workload_of(pool_np, q):
    return {"rels": [pool_np[r] for r in q["rels"]], "edges": q["edges"], "preds": q["preds"],
            "root": q["root"], "sum": q["sum"]}


def serve(dev_pool, queries, nslots, budget=0, cache=True, sequential=False, batch=0, batch_max_rows=0):
    with sj.Server(nslots=nslots, hbm_budget=budget, cache_filters=cache, batch=batch,
                   batch_max_rows=batch_max_rows) as srv:
        ids = [srv.add_relation(cols) for cols in dev_pool]
        out = {}
        if sequential:
            for q in queries:
                t = srv.submit([ids[r] for r in q["rels"]], q["edges"], q["preds"], q["sum"], q["root"])
                (c,) = srv.poll(1, wait_ms=60_000)
                assert c["ticket"] == t
                out[t] = c
        else:
            tickets = [srv.submit([ids[r] for r in q["rels"]], q["edges"], q["preds"], q["sum"], q["root"])
                       for q in queries]
            while len(out) < len(tickets):
                for c in srv.poll(256, wait_ms=60_000):
                    out[c["ticket"]] = c
        stats = srv.stats()
    ordered = [out[t] for t in sorted(out)]
    return ordered, stats


def test_mix_equals_alone_and_oracle(pool):
    pool_np, dev = pool
    qs = inputs.serving_queries([len(r[0]) for r in pool_np], 60, domain=DOMAIN, max_len=5,
                                ntemplates=3, seed=21)
    mixed, st = serve(dev, qs, nslots=4)
    alone, _ = serve(dev, qs, nslots=1, cache=False, sequential=True)
    assert st["completed"] == len(qs) and st["failed"] == 0
    assert st["cache_hits"] > 0 and st["cache_misses"] <= 3 * len(pool_np)
    for q, m, a in zip(qs, mixed, alone):
        assert m["status"] == 0 and a["status"] == 0
        assert (m["count"], m["sum"]) == (a["count"], a["sum"])
        exp = oracle.agg_propagation(workload_of(pool_np, q))
        assert (m["count"], m["sum"]) == (exp["count"], exp["sum"])
        assert m["submit_ms"] <= m["start_ms"] <= m["done_ms"]


@pytest.mark.parametrize("cache,max_rows", [(True, 0), (False, 0), (True, 150_000)])
def test_batch_mode_mix_equals_alone_and_oracle(pool, cache, max_rows):
    """Batch mode (pruning of up to 8 queued queries in one batched call;
    with a row limit, larger queries run alone): every result equals the
    query run alone and the oracle."""
    pool_np, dev = pool
    qs = inputs.serving_queries([len(r[0]) for r in pool_np], 80, domain=DOMAIN, max_len=6,
                                ntemplates=3, seed=23)
    mixed, st = serve(dev, qs, nslots=2, cache=cache, batch=8, batch_max_rows=max_rows)
    alone, _ = serve(dev, qs, nslots=1, cache=False, sequential=True)
    assert st["completed"] == len(qs) and st["failed"] == 0
    assert st["batches"] > 0 and st["peak_batch"] > 1
    for q, m, a in zip(qs, mixed, alone):
        assert m["status"] == 0
        assert (m["count"], m["sum"]) == (a["count"], a["sum"])
        exp = oracle.agg_propagation(workload_of(pool_np, q))
        assert (m["count"], m["sum"]) == (exp["count"], exp["sum"])
        assert m["submit_ms"] <= m["start_ms"] <= m["done_ms"]


def test_batch_mode_tiny_budget_takes_one_query_per_batch(pool):
    pool_np, dev = pool
    qs = inputs.serving_queries([len(r[0]) for r in pool_np], 10, domain=DOMAIN, max_len=4,
                                ntemplates=2, seed=24)
    res, st = serve(dev, qs, nslots=2, budget=1, batch=8)
    assert st["peak_concurrency"] == 1 and st["peak_batch"] <= 1
    for q, r in zip(qs, res):
        exp = oracle.agg_propagation(workload_of(pool_np, q))
        assert (r["count"], r["sum"]) == (exp["count"], exp["sum"])


def test_tiny_budget_admits_one_at_a_time(pool):
    pool_np, dev = pool
    qs = inputs.serving_queries([len(r[0]) for r in pool_np], 12, domain=DOMAIN, max_len=4,
                                ntemplates=2, seed=22)
    res, st = serve(dev, qs, nslots=4, budget=1)
    assert st["peak_concurrency"] == 1
    for q, r in zip(qs, res):
        exp = oracle.agg_propagation(workload_of(pool_np, q))
        assert (r["count"], r["sum"]) == (exp["count"], exp["sum"])


def test_bad_query_is_rejected(pool):
    pool_np, dev = pool
    with sj.Server(nslots=2) as srv:
        rid = srv.add_relation(dev[0])
        with pytest.raises(sj.SieveJoinError):
            srv.submit([rid, 99], [(0, 1, 1, 0)])
        with pytest.raises(sj.SieveJoinError):
            srv.submit([rid, rid], [(0, 5, 1, 0)])
