"""Write serving_expected.txt: the oracle's COUNT and SUM for every query
of the serving workload (10,000 chain queries of 2-6 relations over
a pool of 40 relations with log-uniform sizes from 1e4 to 5e7 rows, Zipf(0.8)
keys over 2^22, a range predicate on the first relation from 8 fixed ranges),
so that the benchmark can check every served result.

Only the seeded input generators and the oracle are called: the chain
counting of ``oracle.chain_agg`` (per-key (count, sum) messages, the same
counting as ``oracle.agg_propagation``).  Usage:
``python tests/golden/make_serving_expected.py`` (about ten minutes on 8 cores).
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2308_16370_b300 import inputs  # noqa: E402

NREL, MIN_ROWS, MAX_ROWS, DOMAIN, POOL_SEED = 40, 10_000, 50_000_000, 1 << 22, 5
NQ, QUERY_SEED = 10_000, 6
OUT = os.path.join(HERE, "serving_expected.txt")


def write(out=OUT, nrel=NREL, min_rows=MIN_ROWS, max_rows=MAX_ROWS, domain=DOMAIN, nq=NQ, log=print):
    """The oracle's COUNT and SUM of every query of the workload, written to `out`."""
    t0 = time.time()
    pool = inputs.serving_pool(nrel=nrel, min_rows=min_rows, max_rows=max_rows, domain=domain,
                               seed=POOL_SEED)
    sizes = [len(r[0]) for r in pool]
    qs = inputs.serving_queries(sizes, nq, domain=domain, seed=QUERY_SEED)
    log(f"pool and queries in {time.time() - t0:.0f} s")
    oracle.set_threads(os.cpu_count() or 1)
    cp = oracle.ChainPool(pool, domain)
    res = []
    for i in range(0, nq, 500):
        res += oracle.chain_agg(cp, qs[i:i + 500])
        log(f"{len(res)} queries, {time.time() - t0:.0f} s")
    with open(out, "w") as f:
        f.write("# Serving workload: the oracle's COUNT and SUM (mod 2^64) per query\n")
        f.write(f"# serving_pool(nrel={nrel}, min_rows={min_rows}, max_rows={max_rows}, "
                f"domain={domain}, seed={POOL_SEED}); serving_queries(nq={nq}, seed={QUERY_SEED})\n")
        f.write(f"# pool rows {sum(sizes)}\n")
        f.write("# query count sum\n")
        for i, r in enumerate(res):
            f.write(f"{i} {r['count']} {r['sum']}\n")
    log(f"wrote {out} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    write(log=lambda m: print(m, flush=True))
