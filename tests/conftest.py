import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


@pytest.fixture(scope="session", autouse=True)
def _oracle_built():
    import oracle
    oracle.build_lib()
    yield


def load_golden(name):
    import json
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        return json.load(f)


def workload_from_golden(g):
    import numpy as np
    rels = [[np.array(c, dtype=np.int32) for c in r] for r in g["rels"]]
    preds = [tuple(p) if p is not None else None for p in g.get("preds", [None] * len(rels))]
    return {"name": "golden", "rels": rels, "edges": [tuple(e) for e in g["edges"]],
            "preds": preds, "root": g.get("root", len(rels) - 1),
            "sum": [tuple(t) for t in g["sum"]]}
