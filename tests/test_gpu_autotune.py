"""The autotuner: every candidate (bits per key, k, layout, schedule) returns
the identical exact result, the choice is one of the candidates, and a second
call is served from the cache."""
import pytest

import oracle
import paper_2308_16370_b300 as sj
from paper_2308_16370_b300 import autotune, inputs

pytestmark = pytest.mark.gpu


def test_autotune_chain(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    w = inputs.zipf_chain(nrows=200_000, domain=100_000, seed=13)
    exp = oracle.agg_propagation(w)
    with sj.Context(0) as ctx:
        rels = [ctx.load_relation(r, where="host") for r in w["rels"]]
        cand = {"bits_per_key": (4, 8), "k": (1, 3), "layout": (sj.REGBLOCKED32, sj.BLOCKED256),
                "root": (w["root"],)}
        path = str(tmp_path / "tune.json")
        first = autotune.tune(ctx, rels, w["edges"], w["preds"], w["root"], w["sum"],
                              candidates=cand, reps=2, path=path)
        assert not first["cached"] and len(first["timings"]) == 16
        p = first["params"]
        assert p["bits_per_key"] in (4, 8) and p["k"] in (1, 3)
        res = ctx.sieve_join(rels, w["edges"], w["preds"], w["root"], refs=w["sum"], **p)
        assert (res["count"], res["sum"]) == (exp["count"], exp["sum"])
        again = autotune.tune(ctx, rels, w["edges"], w["preds"], w["root"], w["sum"],
                              candidates=cand, reps=2, path=path)
        assert again["cached"] and again["params"] == p and again["root"] == first["root"]


def test_autotune_sieve_order(tmp_path):
    """With every relation as a candidate root (the sieve order), every
    candidate gives the oracle's result and the pick is one of them."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    w = inputs.zipf_chain(nrows=100_000, domain=50_000, seed=17)
    exp = oracle.agg_propagation(w)
    with sj.Context(0) as ctx:
        rels = [ctx.load_relation(r, where="host") for r in w["rels"]]
        cand = {"bits_per_key": (8,), "k": (3,), "layout": (sj.REGBLOCKED32,)}
        out = autotune.tune(ctx, rels, w["edges"], w["preds"], w["root"], w["sum"], candidates=cand,
                            reps=2, path=str(tmp_path / "tune.json"))
        assert sorted({t["root"] for t in out["timings"]}) == list(range(len(rels)))
        assert len(out["timings"]) == 2 * len(rels) and 0 <= out["root"] < len(rels)
        res = ctx.sieve_join(rels, w["edges"], w["preds"], out["root"], refs=w["sum"], **out["params"])
        assert (res["count"], res["sum"]) == (exp["count"], exp["sum"])
