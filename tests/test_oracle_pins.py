"""Pins of the CPU oracle against things other than itself.

Every oracle function is checked here against what the paper or the
mathematics fixes: hand-worked examples (tests/golden), the closed form of the
synthetic R, S, T benchmark (Sec. 3.1.1), brute-force enumeration on tiny
inputs, direct-lookup evaluation of star joins, the Bloom filter's
no-false-negative property, Eq. 3's expected number of set bits, the
false-positive rate of the layout, the Bloomjoin cardinality of Eq. 1 (read as
survivors = semijoin + non-matching x FPR), and the exact inverse of the hash
mixer.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_16370_b300 import inputs
from conftest import load_golden, workload_from_golden


# ------------------------------------------------------------------ joins: hand-worked
def test_hand_chain3_count_sum_tuples():
    g = load_golden("hand_chain3.json")
    w = workload_from_golden(g)
    for fn in (oracle.hash_join, oracle.nested_loop, oracle.agg_propagation):
        r = fn(w)
        assert r["count"] == g["expected_count"]
        assert r["sum"] == g["expected_sum_a_plus_d"]
    m = oracle.hash_join(w, mode=oracle.MATERIALIZE,
                         refs=[(0, 0, 0), (0, 1, 0), (1, 1, 0), (2, 1, 0)])
    got = sorted(zip(*[c.tolist() for c in m["cols"]]))
    assert got == sorted(tuple(t) for t in g["expected_tuples_abcd"])


def test_hand_chain3_full_reduction_and_sieve_superset():
    g = load_golden("hand_chain3.json")
    w = workload_from_golden(g)
    red = oracle.semijoin_reduction(w)
    for i, exp in enumerate(g["expected_full_reduction"]):
        assert [c.tolist() for c in red[i]] == exp
    sv, _ = oracle.sieve_path(w)
    for i in range(3):
        got = set(zip(*[c.tolist() for c in sv[i]]))
        assert set(zip(*g["expected_full_reduction"][i])) <= got


def test_hand_star():
    g = load_golden("hand_star.json")
    w = workload_from_golden(g)
    w["root"] = 0
    for fn in (oracle.hash_join, oracle.nested_loop, oracle.agg_propagation):
        r = fn(w)
        assert (r["count"], r["sum"]) == (g["expected_count"], g["expected_sum"])


# ------------------------------------------------------------------ joins: closed form
@pytest.mark.parametrize("r,d", [(10, 1), (10, 3), (40, 2)])
def test_freitag_closed_form(r, d):
    """|R |x| S |x| T| = r d^3 and SUM(R.x) = d^3 * sum of the r common values."""
    top = 200
    w = inputs.freitag_rst(r, d, top=top)
    common = np.arange((top - r) // 2 + 1, (top + r) // 2 + 1)
    assert len(common) == r
    exp_sum = d ** 3 * int(common.sum())
    for fn in (oracle.hash_join, oracle.agg_propagation):
        res = fn(w)
        assert res["count"] == r * d ** 3
        assert res["sum"] == exp_sum
    if r * d <= 40:
        res = oracle.nested_loop(w)
        assert (res["count"], res["sum"]) == (r * d ** 3, exp_sum)


# ------------------------------------------------------------------ joins: brute force
@pytest.mark.parametrize("seed", range(12))
def test_hash_join_and_propagation_vs_nested_loop(seed):
    g = np.random.default_rng(100 + seed)
    nrel = int(g.integers(1, 5))
    w = inputs.random_tree_join(g, nrel, g.integers(0, 14, nrel), domain=6,
                                star_like=bool(seed % 3 == 0))
    bf = oracle.nested_loop(w)
    hj = oracle.hash_join(w)
    ap = oracle.agg_propagation(w)
    assert (hj["count"], hj["sum"]) == (bf["count"], bf["sum"])
    assert (ap["count"], ap["sum"]) == (bf["count"], bf["sum"])
    m = oracle.hash_join(w, mode=oracle.MATERIALIZE)
    assert m["count"] == bf["count"]


def test_negative_values_and_wide_sum():
    """SUM is int64 modulo 2^64: negative values and 64-bit (two-word) terms."""
    g = np.random.default_rng(7)
    R = [g.integers(-5, 5, 30, dtype=np.int32), g.integers(0, 4, 30, dtype=np.int32)]
    big = g.integers(-(1 << 62), 1 << 62, 25, dtype=np.int64)
    S = [g.integers(0, 4, 25, dtype=np.int32),
         (big & 0xFFFFFFFF).astype(np.uint32).view(np.int32), (big >> 32).astype(np.int32)]
    w = {"rels": [R, S], "edges": [(0, 1, 1, 0)], "preds": [None, None], "root": 1,
         "sum": [(0, 0, 0), (1, 1, 1)]}
    exp_c, exp_s = 0, 0
    for i in range(30):
        for j in range(25):
            if R[1][i] == S[0][j]:
                exp_c += 1
                exp_s += int(R[0][i]) + int(big[j])
    exp_s %= 1 << 64
    for fn in (oracle.hash_join, oracle.nested_loop, oracle.agg_propagation):
        r = fn(w)
        assert (r["count"], r["sum"]) == (exp_c, exp_s)


def test_star_direct_lookup():
    """Dense-key dimensions: COUNT/SUM by direct indexing of the dimension rows."""
    w = inputs.star(nfact=20000, ndim=3, dim_rows=500, sel=0.3, seed=11)
    fact = w["rels"][0]
    ok = np.ones(len(fact[0]), dtype=bool)
    for i in range(3):
        pk, attr = w["rels"][1 + i]
        _, lo, hi = w["preds"][1 + i]
        assert np.array_equal(pk, np.arange(500))
        a = attr[fact[i]]
        ok &= (a >= lo) & (a < hi)
    meas = fact[3].view(np.uint32).astype(np.int64) | (fact[4].astype(np.int64) << 32)
    exp = (int(ok.sum()), int(meas[ok].sum()) % (1 << 64))
    for fn in (oracle.hash_join, oracle.agg_propagation):
        r = fn(w)
        assert (r["count"], r["sum"]) == exp


def test_agg_propagation_overflow_flag():
    """COUNT >= 2^63 is reported: 4 relations of 2^16 rows all on key 0 give 2^64."""
    n = 1 << 16
    z = np.zeros(n, dtype=np.int32)
    w = {"rels": [[z, z]] * 4, "edges": inputs.chain_edges(4), "preds": [None] * 4,
         "root": 3, "sum": []}
    r = oracle.agg_propagation(w)
    assert r["overflow"] and r["count"] == 0 and r["count_approx"] == 2.0 ** 64


# ------------------------------------------------------------------ hash mixer
def test_fmix64_inverse_and_fixed_point():
    """fmix64 is a bijection: undo it with the modular inverses of its
    multipliers (derived here, not typed in) and inverse xor-shifts."""
    C1, C2 = 0xFF51AFD7ED558CCD, 0xC4CEB9FE1A85EC53
    M = (1 << 64) - 1
    i1, i2 = pow(C1, -1, 1 << 64), pow(C2, -1, 1 << 64)

    def unshift33(y):
        return y ^ (y >> 33)  # 33 >= 64/2, so one step inverts x ^= x >> 33

    g = np.random.default_rng(3)
    xs = [int(v) for v in g.integers(0, 1 << 63, 200, dtype=np.int64)] + [0, 1, M, 1 << 63]
    hs = oracle.fmix64(np.array(xs, dtype=np.uint64))
    for x, h in zip(xs, hs.tolist()):
        y = unshift33(int(h))
        y = (y * i2) & M
        y = unshift33(y)
        y = (y * i1) & M
        y = unshift33(y)
        assert y == x
    assert int(oracle.fmix64(np.array([0], dtype=np.uint64))[0]) == 0


def test_fmix64_avalanche():
    g = np.random.default_rng(5)
    x = g.integers(0, 1 << 63, 20000, dtype=np.int64).astype(np.uint64)
    h0 = oracle.fmix64(x)
    for b in (0, 7, 31, 32, 63):
        h1 = oracle.fmix64(x ^ np.uint64(1 << b))
        d = np.unpackbits((h0 ^ h1).view(np.uint8)).reshape(-1, 64).sum(1)
        assert abs(d.mean() - 32) < 0.3


# ------------------------------------------------------------------ Bloom filter
@pytest.mark.parametrize("layout", [oracle.REG32, oracle.BLOCKED256, oracle.CLASSIC])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_bloom_no_false_negatives(layout, k):
    g = np.random.default_rng(k)
    keys = g.integers(-(1 << 31), (1 << 31) - 1, 5000, dtype=np.int64).astype(np.int32)
    keys[:3] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, 0]
    f = oracle.bloom_build(keys, 8, k, layout, seed=123)
    assert f["words"].size == 8 * oracle.bloom_nblocks(5000, 8)
    assert oracle.bloom_contains(f, keys).all()


def test_bloom_classic_k1_is_a_hashed_bitset():
    """k = 1 CLASSIC reduces to a bitset indexed by (low 32 bits of h) mod m."""
    g = np.random.default_rng(9)
    keys = g.integers(0, 1 << 30, 3000, dtype=np.int64).astype(np.int32)
    probe = g.integers(0, 1 << 30, 20000, dtype=np.int64).astype(np.int32)
    f = oracle.bloom_build(keys, 8, 1, oracle.CLASSIC, seed=5)
    m = 256 * f["nblocks"]
    slot = lambda ks: set((oracle.key_hash(ks, 5) & np.uint64(0xFFFFFFFF)) % np.uint64(m))
    ins = slot(keys)
    exp = np.array([int(s) in ins for s in
                    ((oracle.key_hash(probe, 5) & np.uint64(0xFFFFFFFF)) % np.uint64(m))])
    assert np.array_equal(oracle.bloom_contains(f, probe), exp)
    bits = np.unpackbits(f["words"].view(np.uint8), bitorder="little")
    assert bits.sum() == len(ins)


def test_bloom_blocked_bits_stay_in_one_block():
    """Each key sets 1..k bits, all inside one aligned 256-bit block
    (BLOCKED256) or one 32-bit word (REG32); the block / word index is
    spread evenly (chi-square over 64 bins)."""
    g = np.random.default_rng(10)
    for layout, span in ((oracle.BLOCKED256, 8), (oracle.REG32, 1)):
        for key in g.integers(-(1 << 31), (1 << 31) - 1, 50, dtype=np.int64).astype(np.int32):
            f = oracle.bloom_build(np.array([key], dtype=np.int32), 8 * 256 * 4, 3, layout, seed=1)
            nz = np.nonzero(f["words"])[0]
            assert len(set(nz // span)) == 1
            bits = np.unpackbits(f["words"].view(np.uint8)).sum()
            assert 1 <= bits <= 3
        keys = g.integers(-(1 << 31), (1 << 31) - 1, 64_000, dtype=np.int64).astype(np.int32)
        nblocks = 64 if layout == oracle.BLOCKED256 else 8  # 64 blocks or 64 words
        word, _ = oracle.bloom_positions(oracle.key_hash(keys, 3), nblocks, 1, layout)[0]
        bins = np.bincount(word // span, minlength=64)
        assert len(bins) == 64
        chi2 = ((bins - 1000.0) ** 2 / 1000.0).sum()
        assert chi2 < 120, chi2  # 63 degrees of freedom


def _poisson_mix(lam, fn, jmax=None):
    jmax = jmax or int(lam + 12 * math.sqrt(lam) + 30)
    p = math.exp(-lam)
    tot = 0.0
    for j in range(jmax):
        tot += p * fn(j)
        p *= lam / (j + 1)
    return tot


@pytest.mark.parametrize("k", [1, 3])
def test_eq3_expected_set_bits(k):
    """Eq. 3: F(1 - e^{-D/F}) bits are set (k = 1), generalised to
    m(1 - e^{-kD/m}) for k hashes; BLOCKED256 follows the Poisson mixture over
    block loads of 256(1 - (1 - 1/256)^{kj})."""
    g = np.random.default_rng(20 + k)
    D = 200_000
    keys = g.choice(1 << 30, D, replace=False).astype(np.int32)
    for layout in (oracle.CLASSIC, oracle.BLOCKED256, oracle.REG32):
        f = oracle.bloom_build(keys, 8, k, layout, seed=77)
        m = 256 * f["nblocks"]
        got = int(np.unpackbits(f["words"].view(np.uint8)).sum())
        if layout == oracle.CLASSIC:
            exp = m * (1 - math.exp(-k * D / m))
        else:
            w = 256 if layout == oracle.BLOCKED256 else 32
            nb = m // w
            exp = nb * _poisson_mix(D / nb, lambda j: w * (1 - (1 - 1 / w) ** (k * j)))
        assert abs(got - exp) / exp < 0.01, (layout, got, exp)


@pytest.mark.parametrize("bpk,k", [(8, 3), (4, 2), (16, 4)])
def test_false_positive_rate(bpk, k):
    """FPR of CLASSIC against (1 - e^{-kn/m})^k, of BLOCKED256 against the
    Poisson mixture sum_j P(j) (1 - (1 - 1/256)^{kj})^k, within a 4-sigma
    binomial band plus a 4% model allowance."""
    g = np.random.default_rng(bpk * 10 + k)
    n = 100_000
    keys = g.choice(1 << 29, n, replace=False).astype(np.int32)
    neg = (g.choice(1 << 29, 1_000_000, replace=False) + (1 << 29)).astype(np.int32)
    for layout in (oracle.CLASSIC, oracle.BLOCKED256, oracle.REG32):
        f = oracle.bloom_build(keys, bpk, k, layout, seed=99)
        m = 256 * f["nblocks"]
        fpr = oracle.bloom_contains(f, neg).mean()
        if layout == oracle.CLASSIC:
            exp = (1 - math.exp(-k * n / m)) ** k
        else:
            w = 256 if layout == oracle.BLOCKED256 else 32
            exp = _poisson_mix(n * w / m, lambda j: (1 - (1 - 1 / w) ** (k * j)) ** k)
        sig = math.sqrt(exp * (1 - exp) / len(neg))
        assert abs(fpr - exp) <= 4 * sig + 0.04 * exp, (layout, fpr, exp)


def test_bloomjoin_cardinality_eq1():
    """Eq. 1 as read here: survivors of T = SC_T + (C_T - SC_T) * FPR."""
    g = np.random.default_rng(31)
    S = g.integers(0, 400_000, 50_000, dtype=np.int32)
    T = g.integers(0, 400_000, 300_000, dtype=np.int32)
    f = oracle.bloom_build(S, 8, 3, oracle.CLASSIC, seed=4)
    kept = oracle.sieve([T], [(0, f)])[0]
    sc = int(np.isin(T, S).sum())
    D = len(np.unique(S))
    m = 256 * f["nblocks"]
    fpr = (1 - math.exp(-3 * D / m)) ** 3
    exp = sc + (len(T) - sc) * fpr
    sig = math.sqrt((len(T) - sc) * fpr)
    assert abs(len(kept) - exp) <= 4 * sig + 0.04 * (len(T) - sc) * fpr


# ------------------------------------------------------------------ sieve path
@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("passes", [oracle.FWD_BWD, oracle.BWD_ONLY])
def test_sieve_path_superset_and_same_join(seed, passes):
    """No false negatives: every sieved relation contains its exact full
    reduction, keeps input order, and the join over it is unchanged."""
    g = np.random.default_rng(200 + seed)
    nrel = int(g.integers(2, 5))
    w = inputs.random_tree_join(g, nrel, g.integers(0, 60, nrel), domain=20,
                                star_like=bool(seed % 2))
    # tag rows with their index to check order and containment
    tagged = dict(w, rels=[r + [np.arange(len(r[0]), dtype=np.int32)] for r in w["rels"]])
    sv, steps = oracle.sieve_path(tagged, passes=passes, bits_per_key=2, k=1, seed=seed)
    red = oracle.semijoin_reduction(tagged)
    for i in range(nrel):
        ids = sv[i][-1]
        assert np.all(np.diff(ids) > 0)
        assert set(red[i][-1].tolist()) <= set(ids.tolist())
        sel = oracle.select(tagged["rels"][i], w["preds"][i])
        assert set(ids.tolist()) <= set(sel[-1].tolist())
    base = oracle.hash_join(w)
    sj = oracle.hash_join(w, rels=[r[:-1] for r in sv], presieved=True)
    assert (sj["count"], sj["sum"]) == (base["count"], base["sum"])
    nsieve = sum(1 for s in steps if s[0] in ("fwd", "bwd"))
    exp_steps = 2 * (nrel - 1) if passes == oracle.FWD_BWD else nrel - 1
    # in pass 1 a node with several children is sieved once by all of them
    assert nsieve <= exp_steps


def test_sieve_path_chain_step_count():
    """Forward then backward over an n-way chain: 2(n-1) sieve steps."""
    w = inputs.uniform_chain(nrel=4, nrows=1000, domain=3000, seed=3)
    _, steps = oracle.sieve_path(w)
    assert [s[0] for s in steps] == ["fwd"] * 3 + ["bwd"] * 3
    assert [s[1] for s in steps] == [1, 2, 3, 2, 1, 0]


def test_sieve_shrinks_skewed_chain():
    """The sieve drops most tuples of a chain whose last relation covers 1% of
    the key domain, and the join result is unchanged."""
    w = inputs.zipf_chain(nrows=20000, domain=10000, seed=4)
    sv, steps = oracle.sieve_path(w)
    assert sum(len(r[0]) for r in sv) < 0.5 * sum(len(r[0]) for r in w["rels"])
    a = oracle.agg_propagation(w)
    b = oracle.agg_propagation(w, rels=sv, presieved=True)
    assert (a["count"], a["sum"]) == (b["count"], b["sum"])


# ------------------------------------------------------------------ cyclic query (triangles)
def _dense_trace_counts(src, dst, n, cuts):
    A = np.zeros((n, n))
    A[src, dst] = 1.0
    d = np.diag(A @ A @ A)  # closed walks of length 3; exact integers in float64
    return np.array([int(round(d[cuts[i]:cuts[i + 1]].sum())) for i in range(len(cuts) - 1)])


@pytest.mark.parametrize("scale,ne", [(6, 300), (8, 2500), (9, 4000)])
def test_triangles_vs_trace_of_a_cubed(scale, ne):
    """Ordered directed 3-cycles per a-range equal diag(A^3) summed over the
    range (no self-loops, so every closed 3-walk is a triangle)."""
    src, dst = inputs.rmat_edges(scale=scale, nedges=ne, seed=scale)
    assert len(set(zip(src.tolist(), dst.tolist()))) == ne and not np.any(src == dst)
    n = 1 << scale
    cuts = inputs.uneven_cuts(n, 8, seed=scale)
    got = oracle.triangle_counts(src, dst, cuts)
    assert np.array_equal(got, _dense_trace_counts(src, dst, n, cuts))
    assert got.sum() % 3 == 0


def test_triangles_complete_digraph():
    """Complete directed graph on n vertices: n(n-1)(n-2) ordered triangles."""
    n = 12
    s, d = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    keep = s != d
    src, dst = s[keep].astype(np.int32), d[keep].astype(np.int32)
    got = oracle.triangle_counts(src, dst, np.array([0, 5, n], dtype=np.int32))
    assert got.sum() == n * (n - 1) * (n - 2)
    assert list(got) == [5 * (n - 1) * (n - 2), 7 * (n - 1) * (n - 2)]


def test_triangles_single_cycle():
    src = np.array([3, 7, 9, 3], dtype=np.int32)
    dst = np.array([7, 9, 3, 9], dtype=np.int32)  # 3->7->9->3 plus a chord 3->9
    got = oracle.triangle_counts(src, dst, np.array([0, 4, 8, 16], dtype=np.int32))
    assert list(got) == [1, 1, 1]


def test_triangle_counts_for_matches_full():
    src, dst = inputs.rmat_edges(scale=9, nedges=4000, seed=3)
    n = 1 << 9
    verts = [int(v) for v in np.unique(src)[:: 37]]
    cuts = np.unique(np.concatenate([[0, n], verts, np.array(verts) + 1])).astype(np.int32)
    full = oracle.triangle_counts(src, dst, cuts)
    got = oracle.triangle_counts_for(src, dst, verts)
    for v, c in zip(verts, got):
        assert full[np.searchsorted(cuts, v, side="right") - 1] == c


def _brute_triangles(src, dst, cuts):
    """Ordered (a, b, c) with a->b, b->c, c->a by three nested loops over the
    edge list (tiny inputs only); a below cuts[0] in subquery 0, at or above
    cuts[-1] in the last."""
    edges = set(zip(src.tolist(), dst.tolist()))
    out = [0] * (len(cuts) - 1)
    for a, b in edges:
        for b2, c in edges:
            if b2 == b and (c, a) in edges:
                i = 0
                while i + 1 < len(cuts) - 1 and cuts[i + 1] <= a:
                    i += 1
                out[i] += 1
    return out


def test_triangles_negative_ids_and_two_cycles_brute_force():
    """Negative vertex ids (including -1 and INT32_MIN) and 2-cycles through -1:
    a pair of int32 ids must map to one key only, and a closing pair (c, a)
    with c == a is never an edge (no self-loops)."""
    g = np.random.default_rng(11)
    vs = np.array([-2**31, -7, -2, -1, 0, 1, 5, 2**31 - 1], dtype=np.int64)
    pairs = {(int(a), int(b)) for a in vs for b in vs if a != b and g.random() < 0.55}
    pairs |= {(-1, 0), (0, -1), (-1, 5), (5, -1), (-2, -1), (-1, -2)}  # 2-cycles through -1
    src = np.array([p[0] for p in pairs], dtype=np.int32)
    dst = np.array([p[1] for p in pairs], dtype=np.int32)
    cuts = np.array([-5, 0, 3], dtype=np.int32)  # ids below -5 and at or above 3 clamp
    got = oracle.triangle_counts(src, dst, cuts)
    assert list(got) == _brute_triangles(src, dst, cuts)
    assert got.sum() % 3 == 0
    verts = [-1, 0, 5, -2**31]
    per = oracle.triangle_counts_for(src, dst, verts)
    e = set(zip(src.tolist(), dst.tolist()))
    for v, cnt in zip(verts, per):
        # per-vertex count by brute force over the full edge set
        brute = sum(1 for a, b in e if a == v for b2, c in e if b2 == b and (c, a) in e)
        assert cnt == brute


def test_threaded_probe_gives_the_same_results():
    """The probe of the oracle's join levels split over threads returns the
    same COUNT / SUM, the same materialised rows in the same order, and the
    same triangle counts as the serial probe."""
    w = inputs.zipf_chain(nrows=60_000, domain=30_000, seed=4)
    src, dst = inputs.rmat_edges(scale=9, nedges=3000, seed=6)
    cuts = inputs.uneven_cuts(1 << 9, 5, seed=6)
    try:
        oracle.set_threads(1)
        a = oracle.hash_join(w)
        am = oracle.hash_join(w, mode=oracle.MATERIALIZE, refs=[(0, 0, 0), (3, 1, 0)])
        at = oracle.triangle_counts(src, dst, cuts)
        for t in (2, 7):
            oracle.set_threads(t)
            assert oracle.get_threads() == t
            assert oracle.hash_join(w) == a
            bm = oracle.hash_join(w, mode=oracle.MATERIALIZE, refs=[(0, 0, 0), (3, 1, 0)])
            assert bm["count"] == am["count"]
            assert all(np.array_equal(x, y) for x, y in zip(bm["cols"], am["cols"]))
            assert np.array_equal(oracle.triangle_counts(src, dst, cuts), at)
    finally:
        oracle.set_threads(1)


@pytest.mark.parametrize("layout", [oracle.REG32, oracle.BLOCKED256, oracle.CLASSIC])
def test_filter_insert_equals_build_over_union(layout):
    """Sec. 2.4 insert maintenance: after inserting new tuples, the filter is
    the one built over the old keys and the admitted new keys at the old size
    (OR is order-free); every admitted key is contained (no false negatives);
    a tuple is CONTAINED exactly when all its bits were set before the call,
    and GATED exactly when it fails a neighbour's filter."""
    g = np.random.default_rng(3)
    old = g.integers(0, 40_000, 20_000, dtype=np.int32)
    f = oracle.bloom_build(old, 8, 3, layout, seed=5)
    other = g.integers(0, 40_000, 6_000, dtype=np.int32)
    gate = oracle.bloom_build(g.integers(0, 40_000, 15_000, dtype=np.int32), 8, 3, layout, seed=6)
    new_keys = np.concatenate([old[:500], g.integers(0, 60_000, 5_500, dtype=np.int32)])
    cols = [new_keys, other]
    f2, st = oracle.filter_insert(f, cols, 0, [(1, gate)])
    admitted = oracle.bloom_contains(gate, other)
    assert np.array_equal(st == oracle.INSERT_GATED, ~admitted)
    before = oracle.bloom_contains(f, new_keys)
    assert np.array_equal(st == oracle.INSERT_CONTAINED, admitted & before)
    assert np.array_equal(st == oracle.INSERT_NEW, admitted & ~before)
    union = np.concatenate([old, new_keys[admitted]])
    rebuilt = oracle.bloom_build(union, 8, 3, layout, seed=5, nblocks=f["nblocks"])
    assert np.array_equal(f2["words"], rebuilt["words"])
    assert oracle.bloom_contains(f2, new_keys[admitted]).all()
    assert oracle.bloom_contains(f2, old).all()
    # order does not matter
    perm = g.permutation(len(new_keys))
    f3, st3 = oracle.filter_insert(f, [c[perm] for c in cols], 0, [(1, gate)])
    assert np.array_equal(f3["words"], f2["words"]) and np.array_equal(st3, st[perm])
    # no gates: every new key is admitted
    f4, st4 = oracle.filter_insert(f, [new_keys], 0)
    assert (st4 != oracle.INSERT_GATED).all()
    assert oracle.bloom_contains(f4, new_keys).all()


def _chain_pool(g, nrel, domain, max_rows):
    pool = []
    for j in range(nrel):
        n = 0 if j == 4 else int(g.integers(1, max_rows))  # relation 4 is empty
        pool.append([g.integers(0, domain, n, dtype=np.int32) for _ in range(2)])
    return pool


@pytest.mark.parametrize("seed", range(4))
def test_chain_agg_equals_propagation_and_brute_force(seed):
    """The dense chain counting used to check served results: every query's
    COUNT and SUM equal agg_propagation's (mod 2^64) on random chains of 1-6
    relations with and without a predicate (some relations empty), and the
    nested loop's on tiny ones; the thread count changes nothing."""
    g = np.random.default_rng(600 + seed)
    # small domains clear whole message buffers, large ones clear the keys used
    domain = [37, 300, 5000, 20000][seed]
    pool = _chain_pool(g, 9, domain, 400)
    qs = []
    for i in range(40):
        n = int(g.integers(1, 7))
        rels = [int(x) for x in g.choice(len(pool), n, replace=False)]
        lo = int(g.integers(-5, domain))
        pred = None if i % 5 == 0 else (0, lo, lo + int(g.integers(0, domain)))
        qs.append({"rels": rels, "edges": [(j, 1, j + 1, 0) for j in range(n - 1)],
                   "preds": [pred] + [None] * (n - 1), "root": n - 1,
                   "sum": [(0, 0, 0), (n - 1, 1, 0)]})
    oracle.set_threads(1)
    got1 = oracle.chain_agg(pool, qs, domain)
    oracle.set_threads(4)
    got4 = oracle.chain_agg(pool, qs, domain)
    oracle.set_threads(1)
    assert got1 == got4
    for q, r in zip(qs, got1):
        w = {"rels": [pool[j] for j in q["rels"]], "edges": q["edges"], "preds": q["preds"],
             "root": q["root"], "sum": q["sum"]}
        e = oracle.agg_propagation(w)
        assert (r["count"], r["sum"]) == (e["count"] & oracle._MASK64, e["sum"] & oracle._MASK64)
    # tiny relations: brute force
    tiny = []
    for n in g.integers(0, 7, 5):
        tiny.append([g.integers(0, 6, int(n), dtype=np.int32) for _ in range(2)])
    for n in range(1, 5):
        q = {"rels": list(range(n)), "edges": [(j, 1, j + 1, 0) for j in range(n - 1)],
             "preds": [(0, 1, 5)] + [None] * (n - 1), "root": n - 1, "sum": [(0, 0, 0), (n - 1, 1, 0)]}
        (r,) = oracle.chain_agg(tiny, [q], 6)
        w = {"rels": tiny[:n], "edges": q["edges"], "preds": q["preds"], "root": q["root"], "sum": q["sum"]}
        e = oracle.nested_loop(w)
        assert (r["count"], r["sum"]) == (e["count"], e["sum"] & oracle._MASK64)


def test_chain_agg_hand_example_and_rejections():
    """R0 = {(1, 2), (3, 2), (7, 4)}, R1 = {(2, 5), (2, 6), (4, 9)}: with 0 <= x < 5
    on R0 the join is (1,2,2,5), (1,2,2,6), (3,2,2,5), (3,2,2,6): COUNT 4 and
    SUM(R0.x + R1.y) = (1+5) + (1+6) + (3+5) + (3+6) = 30."""
    pool = [[np.array([1, 3, 7], np.int32), np.array([2, 2, 4], np.int32)],
            [np.array([2, 2, 4], np.int32), np.array([5, 6, 9], np.int32)]]
    q = {"rels": [0, 1], "edges": [(0, 1, 1, 0)], "preds": [(0, 0, 5), None], "sum": [(0, 0, 0), (1, 1, 0)]}
    assert oracle.chain_agg(pool, [q], 10) == [{"count": 4, "sum": 30}]
    q2 = dict(q, preds=[None, None])  # adds (7,4,4,9): 5 rows, 30 + 16
    assert oracle.chain_agg(pool, [q2], 10) == [{"count": 5, "sum": 46}]
    with pytest.raises(ValueError):
        oracle.chain_agg(pool, [dict(q, edges=[(0, 0, 1, 0)])], 10)
    with pytest.raises(ValueError):
        oracle.chain_agg(pool, [q], 8)  # key 9 outside the domain
