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


def main():
    t0 = time.time()
    pool = inputs.serving_pool(nrel=NREL, min_rows=MIN_ROWS, max_rows=MAX_ROWS, domain=DOMAIN,
                               seed=POOL_SEED)
    sizes = [len(r[0]) for r in pool]
    qs = inputs.serving_queries(sizes, NQ, domain=DOMAIN, seed=QUERY_SEED)
    print(f"pool and queries in {time.time() - t0:.0f} s", flush=True)
    oracle.set_threads(os.cpu_count() or 1)
    cp = oracle.ChainPool(pool, DOMAIN)
    res = []
    for i in range(0, NQ, 500):
        res += oracle.chain_agg(cp, qs[i:i + 500])
        print(f"{len(res)} queries, {time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as f:
        f.write("# Serving workload: the oracle's COUNT and SUM (mod 2^64) per query\n")
        f.write(f"# serving_pool(nrel={NREL}, min_rows={MIN_ROWS}, max_rows={MAX_ROWS}, "
                f"domain={DOMAIN}, seed={POOL_SEED}); serving_queries(nq={NQ}, seed={QUERY_SEED})\n")
        f.write(f"# pool rows {sum(sizes)}\n")
        f.write("# query count sum\n")
        for i, r in enumerate(res):
            f.write(f"{i} {r['count']} {r['sum']}\n")
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
