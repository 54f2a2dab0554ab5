"""The stored oracle results of the serving workload.

``tests/golden/serving_expected.txt`` holds, for each of the 10,000 chain
queries of the serving benchmark (40 relations of 1e4..5e7 rows, Zipf(0.8)
keys over 2^22, a range predicate on the first relation), the COUNT and SUM
that ``oracle.chain_agg`` computes; ``make_serving_expected.py`` writes it from the
seeded generators and the oracle only, and ``bench.py`` checks every served
result against it.  Here the file is checked for shape and parameters, and a
sample of its entries against a second oracle method: for queries whose
relations are all small, the relations are regenerated and
``oracle.agg_propagation`` (sorted per-key messages pushed toward relation 0,
a different algorithm from chain_agg's dense per-key arrays in C) must give
the stored COUNT and SUM (Sec. 2.2: the join result is the same whatever the
evaluation order).
"""
import os

import numpy as np

import oracle
from paper_2308_16370_b300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "golden", "serving_expected.txt")
NREL, MIN_ROWS, MAX_ROWS, DOMAIN, POOL_SEED, NQ, QUERY_SEED = 40, 10_000, 50_000_000, 1 << 22, 5, 10_000, 6


def load():
    head, rows = [], []
    with open(PATH) as f:
        for line in f:
            if line.startswith("#"):
                head.append(line[1:].strip())
            elif line.strip():
                i, c, s = line.split()
                rows.append((int(i), int(c), int(s)))
    return head, rows


def test_file_shape_and_parameters():
    head, rows = load()
    assert (f"serving_pool(nrel={NREL}, min_rows={MIN_ROWS}, max_rows={MAX_ROWS}, "
            f"domain={DOMAIN}, seed={POOL_SEED}); serving_queries(nq={NQ}, seed={QUERY_SEED})") in head
    sizes = inputs.serving_pool_sizes(NREL, MIN_ROWS, MAX_ROWS, POOL_SEED)
    assert f"pool rows {int(sizes.sum())}" in head
    assert [r[0] for r in rows] == list(range(NQ))
    assert all(0 <= c < 2 ** 64 and 0 <= s < 2 ** 64 for _, c, s in rows)
    # the workload is not degenerate: most queries have results, some have none
    nonzero = sum(c > 0 for _, c, _ in rows)
    assert NQ // 10 < nonzero < NQ


def test_sample_equals_agg_propagation():
    _, rows = load()
    sizes = inputs.serving_pool_sizes(NREL, MIN_ROWS, MAX_ROWS, POOL_SEED)
    qs = inputs.serving_queries(sizes, NQ, domain=DOMAIN, seed=QUERY_SEED)
    pick = [i for i, q in enumerate(qs) if sum(int(sizes[r]) for r in q["rels"]) <= 1_500_000][:24]
    assert len(pick) == 24
    assert len({len(qs[i]["rels"]) for i in pick}) >= 2  # chains of several lengths
    need = {r for i in pick for r in qs[i]["rels"]}
    pool = inputs.serving_pool(nrel=NREL, min_rows=MIN_ROWS, max_rows=MAX_ROWS, domain=DOMAIN,
                               seed=POOL_SEED, only=need)
    for r in need:
        assert len(pool[r][0]) == int(sizes[r])
    seen_nonzero = 0
    for i in pick:
        q = qs[i]
        w = {"rels": [pool[r] for r in q["rels"]], "edges": q["edges"], "preds": q["preds"],
             "root": q["root"], "sum": q["sum"]}
        exp = oracle.agg_propagation(w)
        assert rows[i] == (i, exp["count"], exp["sum"]), i
        seen_nonzero += exp["count"] > 0
    assert seen_nonzero > 0


def test_subset_pool_equals_full_pool_relations():
    """A relation generated alone equals the same relation of the full pool."""
    full = inputs.serving_pool(nrel=5, min_rows=100, max_rows=5000, domain=1 << 12, seed=9)
    part = inputs.serving_pool(nrel=5, min_rows=100, max_rows=5000, domain=1 << 12, seed=9, only={1, 3})
    assert part[0] is None and part[2] is None and part[4] is None
    for j in (1, 3):
        for a, b in zip(full[j], part[j]):
            assert np.array_equal(a, b)


def test_bench_reads_the_stored_results_for_its_workload_only():
    """bench.py checks every served result against the stored values only
    when they are for the workload it ran."""
    import bench
    rows = bench.stored_serving_results(MAX_ROWS, DOMAIN, NQ)
    _, stored = load()
    assert rows is not None and len(rows) == NQ
    assert all(rows[i] == (0, c, s) for i, c, s in stored)
    assert bench.stored_serving_results(5_000_000, DOMAIN, NQ) is None
    assert bench.stored_serving_results(MAX_ROWS, DOMAIN, 2000) is None


def test_writer_on_a_small_workload(tmp_path):
    """The script that writes the stored values, run on a small pool of the
    same shape: its entries equal the oracle's second counting method."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_serving_expected",
                                                  os.path.join(HERE, "golden", "make_serving_expected.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    out = tmp_path / "small.txt"
    nrel, lo, hi, dom, nq = 6, 1_000, 20_000, 1 << 12, 40
    mod.write(out=str(out), nrel=nrel, min_rows=lo, max_rows=hi, domain=dom, nq=nq, log=lambda m: None)
    rows = [tuple(int(x) for x in ln.split()) for ln in out.read_text().splitlines()
            if ln and not ln.startswith("#")]
    assert [r[0] for r in rows] == list(range(nq))
    pool = inputs.serving_pool(nrel=nrel, min_rows=lo, max_rows=hi, domain=dom, seed=POOL_SEED)
    qs = inputs.serving_queries([len(r[0]) for r in pool], nq, domain=dom, seed=QUERY_SEED)
    nonzero = 0
    for (i, c, s), q in zip(rows, qs):
        w = {"rels": [pool[r] for r in q["rels"]], "edges": q["edges"], "preds": q["preds"],
             "root": q["root"], "sum": q["sum"]}
        exp = oracle.agg_propagation(w)
        assert (c, s) == (exp["count"], exp["sum"]), i
        nonzero += c > 0
    assert nonzero > 0
