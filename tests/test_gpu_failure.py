"""Failure detection without a GPU fault: a bounded device wait that runs out
is reported as SJ_ETIMEOUT through the status word, and the context stays
usable; host-side failures (allocator returning NULL, bad arguments) come back
as error codes."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2308_16370_b300 as sj
from paper_2308_16370_b300 import inputs

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_context_survives():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with sj.Context(0) as ctx:
        assert ctx.selftest_wait_timeout() == 4  # SJ_ETIMEOUT
        w = inputs.uniform_chain(nrows=20_000, domain=10_000, seed=3)
        rels = [ctx.load_relation(r, where="host") for r in w["rels"]]
        res = ctx.sieve_join(rels, w["edges"], refs=w["sum"])
        exp = oracle.hash_join(w)
        assert (res["count"], res["sum"]) == (exp["count"], exp["sum"])


def test_allocator_failure_is_enomem():
    """An allocator callback that returns NULL surfaces as SJ_ENOMEM."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lib = sj.load_library()
    budget = {"left": 4}  # the context's own status block, then refuse

    @ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    def alloc(nbytes, user):
        if budget["left"] <= 0:
            return None
        budget["left"] -= 1
        return torch.cuda.caching_allocator_alloc(int(nbytes), 0, torch.cuda.current_stream())

    @ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    def free(ptr, nbytes, user):
        torch.cuda.caching_allocator_delete(ptr)

    h = ctypes.c_void_p()
    assert lib.sj_create(ctypes.byref(h), 0, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                         ctypes.cast(alloc, ctypes.c_void_p), ctypes.cast(free, ctypes.c_void_p), None) == 0
    g = np.random.default_rng(1)
    cols = [g.integers(0, 100, 50_000, dtype=np.int32) for _ in range(2)]
    ptrs = (ctypes.c_void_p * 2)(*[c.ctypes.data for c in cols])
    budget["left"] = 0
    rel = ctypes.c_void_p()
    assert lib.sj_load_relation(h, 2, ptrs, 50_000, 2, ctypes.byref(rel)) == 2  # SJ_ENOMEM
    assert b"allocation" in lib.sj_last_error(h)
    budget["left"] = 1000
    assert lib.sj_load_relation(h, 2, ptrs, 50_000, 2, ctypes.byref(rel)) == 0
    assert lib.sj_free_rel(h, rel) == 0
    assert lib.sj_destroy(h) == 0
