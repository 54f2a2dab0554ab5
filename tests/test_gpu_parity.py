"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Integer work throughout, so every comparison is exact: filter words bit for
bit, sieved relations row for row in input order, COUNT and SUM (int64 mod
2^64) exactly, materialised tuples as sorted multisets (their order is
unspecified).  Sizes span several tiles (4096 rows per sieve tile) with ragged
tails, plus the full-size workloads on exact or sampled checks.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2308_16370_b300 as sj
from paper_2308_16370_b300 import inputs

pytestmark = pytest.mark.gpu

I32MIN, I32MAX = np.iinfo(np.int32).min, np.iinfo(np.int32).max


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    sj.load_library()
    c = sj.Context(0)
    yield c
    c.close()


def load(ctx, w):
    return [ctx.load_relation(r, where="host") for r in w["rels"]]


def rel_np(rel):
    return rel.to_numpy()


def assert_rel_equal(got, exp):
    assert len(got) == len(exp)
    for g, e in zip(got, exp):
        assert g.dtype == np.int32
        assert np.array_equal(g, np.asarray(e, dtype=np.int32))


def keyset(g, n, kind):
    if kind == "uniform":
        k = g.integers(I32MIN, I32MAX, n, dtype=np.int64).astype(np.int32)
    elif kind == "small":
        k = g.integers(0, 1000, n, dtype=np.int32)
    elif kind == "equal":
        k = np.full(n, 7, dtype=np.int32)
    else:  # zipf
        k = inputs.zipf_ranks(g, n, 50000, 1.0).astype(np.int32) * 7919
    if n >= 2:
        k[0], k[-1] = I32MIN, I32MAX
    return k


# ------------------------------------------------------------------ filters
FILTER_CASES = [  # (rows, layout, k, bits per key); layouts 0 REG32, 1 BLOCKED256, 2 CLASSIC
    (0, 0, 3, 8), (1, 0, 3, 8), (5, 0, 3, 8), (4097, 0, 3, 8), (100_003, 0, 3, 8),
    (100_003, 0, 1, 8), (100_003, 0, 6, 12), (1_000_001, 0, 3, 8),
    (0, 1, 3, 8), (5, 1, 3, 8), (100_003, 1, 3, 8), (100_003, 1, 1, 8), (100_003, 1, 2, 4),
    (100_003, 1, 4, 16), (1_000_001, 1, 3, 8),
    (33_333, 2, 3, 8), (33_333, 2, 1, 8), (33_335, 2, 7, 10),
]


@pytest.mark.parametrize("kind", ["uniform", "zipf", "equal"])
@pytest.mark.parametrize("n,layout,k,bpk", FILTER_CASES)
def test_bloom_build_bit_exact(ctx, n, layout, k, bpk, kind):
    g = np.random.default_rng(n + 17 * k + bpk)
    keys = keyset(g, n, kind)
    seed = int(g.integers(0, 1 << 62))
    rel = ctx.load_relation([keys], where="host")
    f = ctx.build_filter(rel, 0, bits_per_key=bpk, k=k, layout=layout, seed=seed)
    exp = oracle.bloom_build(keys, bpk, k, layout, seed)
    nb, ni, _ = f.info()
    assert (nb, ni) == (exp["nblocks"], n)
    assert np.array_equal(f.words(), exp["words"])
    # membership of inserted and fresh keys
    import torch
    probe = np.concatenate([keys, keyset(g, 5000, "uniform")])
    got = ctx.filter_probe(f, torch.from_numpy(probe).cuda()).cpu().numpy().astype(bool)
    assert np.array_equal(got, oracle.bloom_contains(exp, probe))
    assert got[:n].all()


def test_bloom_build_with_predicate(ctx):
    g = np.random.default_rng(3)
    keys = g.integers(0, 1 << 20, 300_001, dtype=np.int32)
    attr = g.integers(0, 1000, 300_001, dtype=np.int32)
    rel = ctx.load_relation([keys, attr], where="host")
    f = ctx.build_filter(rel, 0, pred=(1, 100, 200), seed=9)
    exp = oracle.bloom_build(oracle.select([keys, attr], (1, 100, 200))[0], 8, 3, 0, 9)
    assert f.info()[1] == exp["n_inserted"]
    assert np.array_equal(f.words(), exp["words"])


# ------------------------------------------------------------------ single sieve step
@pytest.mark.parametrize("n", [0, 1, 3, 4095, 4096, 4097, 65_539, 1_000_003])
@pytest.mark.parametrize("nprobe,use_pred", [(0, True), (1, False), (2, True), (4, False)])
def test_sieve_step_exact(ctx, n, nprobe, use_pred):
    g = np.random.default_rng(n + nprobe)
    cols = [g.integers(0, 20000, n, dtype=np.int32) for _ in range(5)]
    if n > 2:
        cols[1][:2] = [I32MIN, I32MAX]
    rel = ctx.load_relation(cols, where="host")
    filters, ofilters, kcols = [], [], []
    for j in range(nprobe):
        src = g.integers(0, 20000, 5000, dtype=np.int32)
        frel = ctx.load_relation([src], where="host")
        filters.append(ctx.build_filter(frel, 0, bits_per_key=4, seed=j))
        ofilters.append(oracle.bloom_build(src, 4, 3, 0, j))
        kcols.append(j + 1)
    pred = (0, 2000, 15000) if use_pred else None
    out = ctx.sieve(rel, kcols, filters, pred)
    exp = oracle.sieve(oracle.select(cols, pred), list(zip(kcols, ofilters)))
    assert out.nrows == len(exp[0])
    assert_rel_equal(rel_np(out), exp)


@pytest.mark.parametrize("generic", [False, True])
def test_sieve_step_more_chunks_than_one_wave(ctx, generic):
    """13M rows: more 16,384-row chunks (794) than one wave of CTAs holds on a
    148-SM GPU (740), so later chunks take their offsets from the groups of
    chunks that have already finished; the register-blocked k = 4 probe and
    the generic path (a predicate plus a filter)."""
    n = 13_000_013
    g = np.random.default_rng(77 + generic)
    cols = [g.integers(0, 1 << 22, n, dtype=np.int32) for _ in range(2)]
    src = g.integers(0, 1 << 22, 40_000, dtype=np.int32)
    rel = ctx.load_relation(cols, where="host")
    f = ctx.build_filter(ctx.load_relation([src], where="host"), 0, bits_per_key=8, k=4, seed=3)
    of = oracle.bloom_build(src, 8, 4, 0, 3)
    pred = (0, 1 << 20, 3 << 20) if generic else None
    out = ctx.sieve(rel, [1], [f], pred)
    exp = oracle.sieve(oracle.select(cols, pred), [(1, of)])
    assert out.nrows == len(exp[0]) > 0
    assert_rel_equal(rel_np(out), exp)


# ------------------------------------------------------------------ sieve path
def check_path(ctx, w, passes=sj.FWD_BWD, bpk=8, k=3, layout=0, seed=0):
    rels = load(ctx, w)
    sv, st = ctx.sieve_path(rels, w["edges"], w["preds"], w["root"], passes=passes,
                            bits_per_key=bpk, k=k, layout=layout, seed=seed)
    osv, osteps = oracle.sieve_path(w, passes=passes, bits_per_key=bpk, k=k, layout=layout, seed=seed)
    for i in range(len(rels)):
        assert_rel_equal(rel_np(sv[i]), osv[i])
    assert st["steps"] == [tuple(s) for s in osteps]
    return rels, sv, osv


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("passes", [sj.FWD_BWD, sj.BWD_ONLY, sj.NO_SIEVE])
def test_sieve_path_random_trees(ctx, seed, passes):
    g = np.random.default_rng(1000 + seed)
    nrel = int(g.integers(2, 6))
    sizes = g.integers(0, 9000, nrel)
    if seed == 3:
        sizes[1] = 0
    w = inputs.random_tree_join(g, nrel, sizes, domain=int(g.integers(50, 5000)),
                                star_like=bool(seed % 3 == 0))
    check_path(ctx, w, passes=passes, bpk=int(g.integers(2, 12)), k=int(g.integers(1, 5)),
               layout=int(seed % 3) if passes != sj.NO_SIEVE else 0, seed=seed)


def test_sieve_path_chain3_100k(ctx):
    """3-way chain R(a,b) S(b,c) T(c,d), 100k rows each, keys in [0, 50000)."""
    w = inputs.uniform_chain()
    rels, sv, osv = check_path(ctx, w)
    # no false negatives: the sieved relations hold the exact full reduction
    red = oracle.semijoin_reduction(w)
    for i in range(3):
        got = set(zip(*[c.tolist() for c in osv[i]]))
        assert set(zip(*[c.tolist() for c in red[i]])) <= got


# ------------------------------------------------------------------ joins
def join_both(ctx, w, rels, inputs_=None, mode=sj.COUNT_SUM, refs=None):
    refs = w["sum"] if refs is None else refs
    return ctx.join(rels, w["edges"], w["preds"], w["root"], inputs=inputs_, mode=mode, refs=refs)


@pytest.mark.parametrize("seed", range(14))
def test_join_count_sum_random_trees(ctx, seed):
    g = np.random.default_rng(2000 + seed)
    nrel = int(g.integers(1, 6))
    w = inputs.random_tree_join(g, nrel, g.integers(0, 3000, nrel), domain=int(g.integers(20, 800)),
                                star_like=bool(seed % 2))
    exp = oracle.agg_propagation(w)
    assert exp["count"] == oracle.hash_join(w)["count"]
    rels = load(ctx, w)
    plain = join_both(ctx, w, rels)
    assert (plain["count"], plain["sum"]) == (exp["count"], exp["sum"])
    sv, _ = ctx.sieve_path(rels, w["edges"], w["preds"], w["root"])
    sieved = join_both(ctx, w, rels, inputs_=sv)
    assert (sieved["count"], sieved["sum"]) == (exp["count"], exp["sum"])


@pytest.mark.parametrize("seed", range(8))
def test_join_materialize_random_trees(ctx, seed):
    g = np.random.default_rng(3000 + seed)
    nrel = int(g.integers(1, 5))
    w = inputs.random_tree_join(g, nrel, g.integers(1, 1500, nrel), domain=int(g.integers(30, 400)))
    refs = [(r, c, 0) for r in range(nrel) for c in range(len(w["rels"][r]))][:8]
    exp = oracle.hash_join(w, mode=oracle.MATERIALIZE, refs=refs)
    rels = load(ctx, w)
    for inp in (None, ctx.sieve_path(rels, w["edges"], w["preds"], w["root"])[0]):
        got = join_both(ctx, w, rels, inputs_=inp, mode=sj.MATERIALIZE, refs=refs)
        assert got["count"] == exp["count"]
        cols = rel_np(got["rows"])
        got_t = np.stack(cols, 1) if exp["count"] else np.zeros((0, len(refs)), np.int32)
        exp_t = np.stack(exp["cols"], 1) if exp["count"] else np.zeros((0, len(refs)), np.int32)
        assert np.array_equal(got_t[np.lexsort(got_t.T[::-1])], exp_t[np.lexsort(exp_t.T[::-1])])


def test_chain3_100k_full(ctx):
    """The 3-way chain at 100k rows: COUNT, SUM(a + d) and the materialised result."""
    w = inputs.uniform_chain()
    exp = oracle.hash_join(w)
    refs = [(0, 0, 0), (0, 1, 0), (1, 1, 0), (2, 1, 0)]
    expm = oracle.hash_join(w, mode=oracle.MATERIALIZE, refs=refs)
    rels = load(ctx, w)
    sv, st = ctx.sieve_path(rels, w["edges"], w["preds"], w["root"])
    for inp in (None, sv):
        r = join_both(ctx, w, rels, inputs_=inp)
        assert (r["count"], r["sum"]) == (exp["count"], exp["sum"])
        m = join_both(ctx, w, rels, inputs_=inp, mode=sj.MATERIALIZE, refs=refs)
        got_t = np.stack(rel_np(m["rows"]), 1)
        exp_t = np.stack(expm["cols"], 1)
        assert np.array_equal(got_t[np.lexsort(got_t.T[::-1])], exp_t[np.lexsort(exp_t.T[::-1])])


def test_freitag_closed_form(ctx):
    """R, S, T of Sec. 3.1.1: COUNT = r d^3 exactly."""
    r, d, top = 10_000, 3, 1_000_000
    w = inputs.freitag_rst(r, d, top=top)
    rels = load(ctx, w)
    common = np.arange((top - r) // 2 + 1, (top + r) // 2 + 1, dtype=np.int64)
    for inp in (None, ctx.sieve_path(rels, w["edges"], w["preds"], w["root"])[0]):
        res = join_both(ctx, w, rels, inputs_=inp)
        assert res["count"] == r * d ** 3
        assert res["sum"] == d ** 3 * int(common.sum())


def test_skewed_all_equal_keys(ctx):
    n = 3000
    R = [np.arange(n, dtype=np.int32), np.zeros(n, np.int32)]
    S = [np.zeros(n, np.int32), np.arange(n, dtype=np.int32) % 7]
    T = [np.arange(50, dtype=np.int32) % 7, np.arange(50, dtype=np.int32)]
    w = {"rels": [R, S, T], "edges": inputs.chain_edges(3), "preds": [None] * 3, "root": 2,
         "sum": [(0, 0, 0), (2, 1, 0)]}
    exp = oracle.agg_propagation(w)
    rels = load(ctx, w)
    for inp in (None, ctx.sieve_path(rels, w["edges"], None, 2)[0]):
        res = join_both(ctx, w, rels, inputs_=inp)
        assert (res["count"], res["sum"]) == (exp["count"], exp["sum"])
        assert res["intermediate"] in (0, n * n)


def test_wide_sum_and_negative_values(ctx):
    g = np.random.default_rng(5)
    big = g.integers(-(1 << 62), 1 << 62, 20000, dtype=np.int64)
    R = [g.integers(-50, 50, 30000, dtype=np.int32), g.integers(0, 500, 30000, dtype=np.int32)]
    S = [g.integers(0, 500, 20000, dtype=np.int32),
         (big & 0xFFFFFFFF).astype(np.uint32).view(np.int32), (big >> 32).astype(np.int32)]
    w = {"rels": [R, S], "edges": [(0, 1, 1, 0)], "preds": [None, None], "root": 1,
         "sum": [(0, 0, 0), (1, 1, 1)]}
    exp = oracle.hash_join(w)
    rels = load(ctx, w)
    res = join_both(ctx, w, rels)
    assert (res["count"], res["sum"]) == (exp["count"], exp["sum"])


def test_star_scaled(ctx):
    """Star join (fact 4 FKs + int64 measure, 4 filtered dimensions) at 1/10 of
    the fact size: sieve exact, COUNT/SUM against direct lookup."""
    w = inputs.star(nfact=10_000_000, dim_rows=1_000_000, seed=3)
    rels = load(ctx, w)
    sv, st = ctx.sieve_path(rels, w["edges"], w["preds"], w["root"])
    osv, osteps = oracle.sieve_path(w)
    assert st["steps"] == [tuple(s) for s in osteps]
    for i in range(5):
        assert_rel_equal(rel_np(sv[i]), osv[i])
    fact = w["rels"][0]
    ok = np.ones(len(fact[0]), dtype=bool)
    for i in range(4):
        _, lo, hi = w["preds"][1 + i]
        a = w["rels"][1 + i][1][fact[i]]
        ok &= (a >= lo) & (a < hi)
    meas = fact[4].view(np.uint32).astype(np.int64) | (fact[5].astype(np.int64) << 32)
    res = join_both(ctx, w, rels, inputs_=sv)
    assert (res["count"], res["sum"]) == (int(ok.sum()), int(meas[ok].sum()) % (1 << 64))


def test_chain4_zipf_full_size(ctx):
    """4-way Zipf chain at the full 10M rows per relation: every sieved relation
    exact against the oracle's pruning phase, COUNT/SUM against the oracle's
    aggregate propagation, with and without the sieve."""
    w = inputs.zipf_chain()
    rels = load(ctx, w)
    sv, st = ctx.sieve_path(rels, w["edges"], w["preds"], w["root"])
    osv, osteps = oracle.sieve_path(w)
    assert st["steps"] == [tuple(s) for s in osteps]
    for i in range(4):
        assert_rel_equal(rel_np(sv[i]), osv[i])
    exp = oracle.agg_propagation(w, rels=osv, presieved=True)
    res = join_both(ctx, w, rels, inputs_=sv)
    assert (res["count"], res["sum"]) == (exp["count"], exp["sum"])
    plain = join_both(ctx, w, rels)
    assert (plain["count"], plain["sum"]) == (exp["count"], exp["sum"])
    assert plain["intermediate"] > 10 * max(1, res["intermediate"])


@pytest.mark.parametrize("params", [
    dict(bits_per_key=12, k=3, layout=sj.REGBLOCKED32, passes=sj.BWD_ONLY),
    dict(bits_per_key=12, k=4, layout=sj.REGBLOCKED32, passes=sj.BWD_ONLY),
    dict(bits_per_key=12, k=3, layout=sj.REGBLOCKED32, passes=sj.FWD_BWD),
])
def test_headline_path_full_size(ctx, params):
    """The benchmark's exact call at its full size: sj_sieve_join on the 4-way
    Zipf chain (10M rows per relation) with the tuned filter parameters, on
    calls 1 to 6 (exact, device-sized, captured as a CUDA graph, then graph
    replays), against the oracle's aggregate propagation; the per-step row
    counts of the first call against the oracle's pruning phase with the same
    parameters."""
    w = inputs.zipf_chain()
    rels = load(ctx, w)
    exp = oracle.agg_propagation(w)
    _, osteps = oracle.sieve_path(w, passes=params["passes"], bits_per_key=params["bits_per_key"],
                                  k=params["k"], layout=params["layout"])
    got = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"], stats=True, **params)
    assert (got["count"], got["sum"]) == (exp["count"], exp["sum"])
    assert got["steps"] == [tuple(s) for s in osteps]
    g0 = ctx.graph_stats()
    for call in range(6):
        got = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"], **params)
        assert (got["count"], got["sum"]) == (exp["count"], exp["sum"]), call
    g1 = ctx.graph_stats()
    assert g1["replays"] - g0["replays"] >= 3 and g1["failures"] == g0["failures"], g1


def test_repeat_is_bit_identical(ctx):
    w = inputs.zipf_chain(nrows=500_000, domain=250_000, seed=8)
    rels = load(ctx, w)
    a = [rel_np(r) for r in ctx.sieve_path(rels, w["edges"], None, 3)[0]]
    b = [rel_np(r) for r in ctx.sieve_path(rels, w["edges"], None, 3)[0]]
    for x, y in zip(a, b):
        assert_rel_equal(x, y)
    r1 = join_both(ctx, w, rels)
    r2 = join_both(ctx, w, rels)
    assert r1 == {**r2, "rows": r1["rows"]}


def test_invalid_arguments(ctx):
    w = inputs.uniform_chain(nrows=100)
    rels = load(ctx, w)
    with pytest.raises(sj.SieveJoinError) as e:
        ctx.sieve_path(rels, [(0, 1, 1, 0), (0, 1, 1, 0)])  # not a tree
    assert e.value.status == 1
    with pytest.raises(sj.SieveJoinError):
        ctx.sieve_path(rels, [(0, 5, 1, 0), (1, 1, 2, 0)])  # column out of range
    with pytest.raises(sj.SieveJoinError):
        ctx.build_filter(rels[0], 0, k=5, layout=sj.BLOCKED256)
    with pytest.raises(sj.SieveJoinError):
        ctx.join(rels, w["edges"], mode=sj.MATERIALIZE, refs=[])
    # the context stays usable after rejected calls
    r = ctx.join(rels, w["edges"], refs=w["sum"])
    assert r["count"] == oracle.hash_join(w)["count"]


def test_sieve_join_one_call(ctx):
    """sj_sieve_join equals sj_sieve_path followed by sj_join, and the oracle."""
    w = inputs.zipf_chain(nrows=300_000, domain=150_000, seed=12)
    rels = load(ctx, w)
    one = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"], stats=True)
    sv, st = ctx.sieve_path(rels, w["edges"], w["preds"], w["root"])
    two = join_both(ctx, w, rels, inputs_=sv)
    exp = oracle.agg_propagation(w)
    assert (one["count"], one["sum"]) == (two["count"], two["sum"]) == (exp["count"], exp["sum"])
    assert one["steps"] == st["steps"]


# ------------------------------------------- device-sized (one-sync) sieve_join
DEVICE_SIZED_CASES = [
    ("zipf", sj.FWD_BWD), ("zipf", sj.BWD_ONLY), ("uniform", sj.NO_SIEVE),
    ("star", sj.FWD_BWD), ("tree", sj.FWD_BWD), ("tree", sj.BWD_ONLY),
]


@pytest.mark.parametrize("kind,passes", DEVICE_SIZED_CASES)
def test_sieve_join_device_sized_repeat(ctx, kind, passes):
    """A repeated query shape runs with every size kept on the device (buffers
    sized from the previous run): the result stays exact every time."""
    if kind == "zipf":
        w = inputs.zipf_chain(nrows=200_000, domain=100_000, seed=21)
    elif kind == "uniform":
        w = inputs.uniform_chain(nrel=4, nrows=50_001, domain=20_000, seed=22)
    elif kind == "star":
        w = inputs.star(nfact=300_001, ndim=3, dim_rows=20_000, seed=23)
    else:
        g = np.random.default_rng(24)
        w = inputs.random_tree_join(g, 6, g.integers(3000, 40_000, 6), 5000)
    rels = load(ctx, w)
    exp = oracle.agg_propagation(w)
    g0 = ctx.graph_stats()
    # call 1 exact, 2 device-sized, 3 device-sized and captured, then replays
    for _ in range(6):
        got = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"], passes=passes)
        assert (got["count"], got["sum"]) == (exp["count"], exp["sum"])
    g1 = ctx.graph_stats()
    assert g1["replays"] - g0["replays"] == 3, g1
    assert g1["failures"] == g0["failures"], g1


def test_sieve_join_device_sized_overflow_falls_back(ctx):
    """Relations borrowed from device tensors are rewritten in place so the
    intermediate result grows far beyond the buffers sized by the earlier run:
    the device-sized join records the overflow and the call reruns exactly."""
    import torch
    g = np.random.default_rng(31)
    n = 40_000
    cols = [[g.integers(0, 1 << 20, n, dtype=np.int32) for _ in range(2)] for _ in range(3)]
    dev = [[torch.from_numpy(c).cuda() for c in r] for r in cols]
    rels = [ctx.load_relation(r, where="borrow") for r in dev]
    w = {"rels": cols, "edges": inputs.chain_edges(3), "preds": [None] * 3, "root": 2,
         "sum": [(0, 0, 0), (2, 1, 0)]}
    for _ in range(2):
        got = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"])
        exp = oracle.agg_propagation(w)
        assert (got["count"], got["sum"]) == (exp["count"], exp["sum"])
    # every join key collapses to 64 values: the first level's output grows
    # from ~n^2/2^20 to ~n^2/64 tuples
    for r in range(3):
        for j in range(2):
            cols[r][j] = (cols[r][j] % 64).astype(np.int32)
            dev[r][j].copy_(torch.from_numpy(cols[r][j]))
    torch.cuda.synchronize()
    exp = oracle.agg_propagation(w)
    for _ in range(4):
        got = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"])
        assert (got["count"], got["sum"]) == (exp["count"], exp["sum"])


def test_sieve_join_reloaded_relations_not_replayed(ctx):
    """Relations freed and reloaded with the same sizes but other data: the
    query shape cache must not replay work that read the old buffers."""
    for seed in (41, 42, 43):
        w = inputs.uniform_chain(nrel=3, nrows=30_000, domain=5_000, seed=seed)
        rels = load(ctx, w)
        exp = oracle.agg_propagation(w)
        for _ in range(3):
            got = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"])
            assert (got["count"], got["sum"]) == (exp["count"], exp["sum"])
        for r in rels:
            r.free()


def test_profiled_graph_replays_report_kernel_times(ctx):
    """With profiling on, replays of a captured query still report every
    kernel class with positive device time."""
    w = inputs.zipf_chain(nrows=100_000, domain=50_000, seed=51)
    rels = load(ctx, w)
    ctx.prof_enable(True)
    try:
        for _ in range(4):  # exact, device-sized, device-sized + capture, replay
            ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"], passes=sj.BWD_ONLY)
        ctx.prof_reset()
        g0 = ctx.graph_stats()["replays"]
        for _ in range(2):
            ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"], passes=sj.BWD_ONLY)
        assert ctx.graph_stats()["replays"] - g0 == 2
        sv = ctx.prof_read("sieve")
        assert sv["launches"] == 2 * 3 and sv["ms"] > 0 and sv["bytes"] > 0
        ag = ctx.prof_read("agg")
        assert ag["launches"] > 0 and ag["ms"] > 0
    finally:
        ctx.prof_enable(False)


def test_graphs_disabled_still_exact(ctx):
    """With graph capture turned off, repeated calls stay on the device-sized
    path, capture nothing and stay exact; turning it back on restores replay."""
    w = inputs.uniform_chain(nrel=4, nrows=40_000, domain=10_000, seed=61)
    rels = load(ctx, w)
    exp = oracle.agg_propagation(w)
    ctx.graphs_enable(False)
    try:
        g0 = ctx.graph_stats()
        for _ in range(5):
            got = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"])
            assert (got["count"], got["sum"]) == (exp["count"], exp["sum"])
        g1 = ctx.graph_stats()
        assert (g1["replays"], g1["captures"]) == (g0["replays"], g0["captures"])
    finally:
        ctx.graphs_enable(True)
    for _ in range(3):  # device-sized + capture, then replays
        got = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"])
        assert (got["count"], got["sum"]) == (exp["count"], exp["sum"])
    assert ctx.graph_stats()["replays"] - g1["replays"] == 2


def test_host_mapped_relations_equal_device_and_oracle(ctx):
    """Relations left in pinned host memory (SJ_HOST_MAPPED), read by the
    kernels over the host link: new handles over the same buffers on every
    call (exact, device-sized, then graph-replay paths) give the oracle's
    COUNT and SUM; the pruning over them equals the oracle's row for row;
    pageable memory is rejected."""
    import torch
    w = inputs.zipf_chain(nrows=1_000_000, domain=500_000)
    host = [[torch.from_numpy(c).pin_memory() for c in r] for r in w["rels"]]
    exp = oracle.agg_propagation(w)
    for params in (dict(bits_per_key=8, k=4, layout=sj.REGBLOCKED32, passes=sj.BWD_ONLY), dict()):
        for _ in range(4):
            rels = [ctx.load_relation(cols, where="mapped") for cols in host]
            r = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"], **params)
            assert (r["count"], r["sum"]) == (exp["count"], exp["sum"])
            for x in rels:
                x.free()
    rels = [ctx.load_relation(cols, where="mapped") for cols in host]
    sv, st = ctx.sieve_path(rels, w["edges"], w["preds"], w["root"])
    osv, osteps = oracle.sieve_path(w)
    assert st["steps"] == [tuple(s) for s in osteps]
    for i in range(len(rels)):
        assert_rel_equal(rel_np(sv[i]), osv[i])
    with pytest.raises(ValueError):
        ctx.load_relation([torch.zeros(1024, dtype=torch.int32)], where="mapped")
    lib = sj.load_library()
    pageable = np.zeros(1024, dtype=np.int32)
    ptrs = (ctypes.c_void_p * 1)(pageable.ctypes.data)
    h = ctypes.c_void_p()
    assert lib.sj_load_relation(ctx.ctx, 1, ptrs, 1024, sj.HOST_MAPPED, ctypes.byref(h)) == 1
