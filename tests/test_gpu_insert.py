"""GPU parity of filter insert maintenance (Sec. 2.4) against the oracle.

New tuples of a relation whose filter exists: every row's outcome (dropped by
a neighbour's filter, key already contained, key newly inserted), the counts
and the filter words afterwards, bit for bit, for the three layouts, with 0,
1 and 2 gates, on empty and ragged inputs; and the filter after the call
equals a same-size build over the union of the old and the admitted keys.
"""
import numpy as np
import pytest

import oracle
import paper_2308_16370_b300 as sj

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = sj.Context(0)
    yield c
    c.close()


def words_of(ctx, f):
    import torch
    nb, ni, ptr = f.info()
    t = torch.as_tensor(sj._CudaArray(ptr, nb * 8, "<u4"), device="cuda:0")
    return t.cpu().numpy().copy(), nb, ni


@pytest.mark.parametrize("layout,k", [(sj.REGBLOCKED32, 3), (sj.BLOCKED256, 4), (sj.CLASSIC, 5)])
@pytest.mark.parametrize("ngate", [0, 1, 2])
@pytest.mark.parametrize("n", [0, 1, 1023, 200_003])
def test_filter_insert_matches_oracle(ctx, layout, k, ngate, n):
    g = np.random.default_rng(n + 7 * ngate + layout)
    old = g.integers(-50_000, 50_000, 30_000, dtype=np.int32)
    f = ctx.build_filter(ctx.load_relation([old], where="host"), 0, bits_per_key=10, k=k,
                         layout=layout, seed=17)
    fo = oracle.bloom_build(old, 10, k, layout, seed=17)
    gates_gpu, gates_or = [], []
    for j in range(ngate):
        gk = g.integers(-50_000, 50_000, 20_000, dtype=np.int32)
        gates_gpu.append((1 + j, ctx.build_filter(ctx.load_relation([gk], where="host"), 0,
                                                  layout=layout, seed=3 + j)))
        gates_or.append((1 + j, oracle.bloom_build(gk, 8, 3, layout, seed=3 + j)))
    cols = [np.concatenate([old[: min(n, 300)], g.integers(-80_000, 80_000, max(0, n - 300),
                                                           dtype=np.int32)])[:n]]
    cols += [g.integers(-50_000, 50_000, n, dtype=np.int32) for _ in range(2)]
    rel = ctx.load_relation(cols, where="host")
    status, counts = ctx.filter_insert(f, rel, 0, gates_gpu)
    exp_f, exp_st = oracle.filter_insert(fo, cols, 0, gates_or)
    got_st = status.cpu().numpy().astype(np.int8)
    assert np.array_equal(got_st, exp_st)
    assert counts == [int((exp_st == v).sum()) for v in (0, 1, 2)]
    w, nb, ni = words_of(ctx, f)
    assert nb == fo["nblocks"] and np.array_equal(w, exp_f["words"])
    assert ni == exp_f["n_inserted"]
    admitted = exp_st != oracle.INSERT_GATED
    union = np.concatenate([old, cols[0][admitted]])
    assert np.array_equal(w, oracle.bloom_build(union, 10, k, layout, seed=17, nblocks=nb)["words"])
    # a second insert of the same rows changes nothing: all admitted keys are contained
    status2, counts2 = ctx.filter_insert(f, rel, 0, gates_gpu)
    assert counts2[2] == 0 and counts2[0] == counts[0]
    w2, _, _ = words_of(ctx, f)
    assert np.array_equal(w2, w)
