"""GPU parity of the cyclic triangle query (Sec. 2.3) against the oracle.

Exact per-subquery counts on small R-MAT graphs, closed forms (complete
digraph, acyclic graph, empty graph), and at the full 2^22-vertex / 50M-edge
size: invariants that hold at any size (the total is a multiple of 3, the
subqueries add up) plus per-vertex counts of sampled vertices computed one by
one by the oracle.
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
    c = sj.Context(0)
    yield c
    c.close()


def gpu_counts(ctx, src, dst, cuts, rounds=-1):
    rel = ctx.load_relation([src, dst], where="host")
    return ctx.triangles(rel, cuts, sieve_rounds=rounds)


@pytest.mark.parametrize("scale,ne,nsub", [(8, 2_000, 8), (10, 12_000, 64), (12, 45_000, 64),
                                           (13, 90_000, 17)])
@pytest.mark.parametrize("rounds", [0, 1, 2])
def test_rmat_exact(ctx, scale, ne, nsub, rounds):
    src, dst = inputs.rmat_edges(scale=scale, nedges=ne, seed=scale + 1)
    cuts = inputs.uneven_cuts(1 << scale, nsub, seed=scale)
    got, st = gpu_counts(ctx, src, dst, cuts, rounds)
    exp = oracle.triangle_counts(src, dst, cuts)
    assert np.array_equal(got.astype(np.int64), exp)
    assert st["triangles"] == int(exp.sum()) and st["edges_in"] == ne
    assert st["edges_sieved"] <= ne and st["filter_passed"] <= st["candidates"]


def test_complete_digraph(ctx):
    n = 40
    s, d = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    keep = s != d
    got, _ = gpu_counts(ctx, s[keep].astype(np.int32), d[keep].astype(np.int32),
                        np.array([0, 13, n], dtype=np.int32))
    assert int(got.sum()) == n * (n - 1) * (n - 2)
    assert list(got) == [13 * (n - 1) * (n - 2), 27 * (n - 1) * (n - 2)]


def test_acyclic_and_empty(ctx):
    g = np.random.default_rng(1)
    s = g.integers(0, 1000, 20000)
    d = g.integers(0, 1000, 20000)
    keep = s < d  # every edge goes up: no directed cycle
    k = np.unique((s[keep] << 32) | d[keep])
    got, st = gpu_counts(ctx, (k >> 32).astype(np.int32), (k & 0xFFFFFFFF).astype(np.int32),
                         np.array([0, 500, 1000], dtype=np.int32))
    assert int(got.sum()) == 0
    got, st = gpu_counts(ctx, np.zeros(0, np.int32), np.zeros(0, np.int32),
                         np.array([0, 10], dtype=np.int32))
    assert int(got.sum()) == 0 and st["edges_sieved"] == 0


def test_full_size_rmat_sampled(ctx):
    """2^22 vertices, 50M distinct edges, 64 uneven subqueries in one launch."""
    scale, ne = 22, 50_000_000
    src, dst = inputs.rmat_edges(scale=scale, nedges=ne, seed=4)
    n = 1 << scale
    cuts = inputs.uneven_cuts(n, 64, seed=4)
    rel = ctx.load_relation([src, dst], where="host")
    got, st = ctx.triangles(rel, cuts)
    total = int(got.sum())
    assert total % 3 == 0 and total == st["triangles"] and total > 0
    # isolate sampled vertices as single-vertex subqueries and check them one by one
    outd = np.bincount(src, minlength=n)
    g = np.random.default_rng(9)
    cand = np.nonzero((outd >= 5) & (outd <= 200))[0]
    verts = sorted(int(v) for v in g.choice(cand, 3, replace=False))
    vc = np.unique(np.concatenate([[0, n], verts, np.array(verts) + 1])).astype(np.int32)
    got2, st2 = ctx.triangles(rel, vc)
    assert int(got2.sum()) == total
    exp = oracle.triangle_counts_for(src, dst, verts)
    for v, e in zip(verts, exp):
        assert int(got2[np.searchsorted(vc, v, side="right") - 1]) == int(e)


def test_negative_ids_and_two_cycles_through_minus_one(ctx):
    """Vertex ids anywhere in int32, 2-cycles through -1 (whose closing pair
    (-1, -1) packs to the pair set's empty code) and ids beyond both ends of
    the cuts: exact against the oracle."""
    g = np.random.default_rng(5)
    ids = np.concatenate([np.array([-2**31, -1, 0, 2**31 - 1]), g.integers(-60, 60, 40)]).astype(np.int64)
    ids = np.unique(ids)
    s = g.choice(ids, 3000)
    d = g.choice(ids, 3000)
    extra_s = np.array([-1, 0, -1, 7, -2, -1, -1, 2**31 - 1])
    extra_d = np.array([0, -1, 7, -1, -1, -2, 2**31 - 1, -1])
    s = np.concatenate([s, extra_s])
    d = np.concatenate([d, extra_d])
    keep = s != d
    pairs = np.unique(np.stack([s[keep], d[keep]], 1), axis=0)
    src = pairs[:, 0].astype(np.int32)
    dst = pairs[:, 1].astype(np.int32)
    cuts = np.array([-30, -1, 0, 25], dtype=np.int32)
    for rounds in (0, 2):
        got, st = gpu_counts(ctx, src, dst, cuts, rounds)
        exp = oracle.triangle_counts(src, dst, cuts)
        assert np.array_equal(got.astype(np.int64), exp)
        assert st["triangles"] == int(exp.sum())
