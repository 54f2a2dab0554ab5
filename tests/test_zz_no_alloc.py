"""The allocation-free sieve step, sj_sieve_noalloc.

It is for callers that cannot allocate device memory where they sieve (code
inside a custom allocator or memory manager, runtimes that forbid cudaMalloc
on their hot path): they pass inputs and outputs, and the step's scratch is a
fixed array inside the library.  Here it is called through the C ABI and its
output is compared, exactly, with the regular sj_sieve on the same inputs, on
two calls in a row (a large call, then a smaller one, so state left in the
shared scratch by the first call must not leak into the second), and with
the oracle's sieve step; also without a status word and on an empty input.

This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2308_16370_b300 as sj

pytestmark = pytest.mark.gpu


def _ptrs(tensors):
    return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])


def _noalloc(lib, stream, cols_dev, outs, n, key_col, words, nblocks, params, count, status):
    err = ctypes.c_char_p()
    rc = lib.sj_sieve_noalloc(ctypes.c_void_p(stream.cuda_stream), len(cols_dev), _ptrs(cols_dev), n,
                              key_col, ctypes.c_void_p(words), nblocks, ctypes.byref(params),
                              _ptrs(outs), ctypes.c_void_p(count.data_ptr()),
                              ctypes.c_void_p(status.data_ptr()) if status is not None else None,
                              ctypes.byref(err))
    return rc, err.value


@pytest.mark.parametrize("layout", [sj.REGBLOCKED32, sj.BLOCKED256, sj.CLASSIC])
def test_noalloc_matches_sieve_on_two_calls_in_a_row(layout):
    """Two calls in a row (a large one, then a smaller one, so that state left
    in the shared scratch by the first must not leak into the second): the
    output equals the regular sj_sieve and the oracle's sieve step exactly."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lib = sj.load_library()
    with sj.Context(0) as ctx:
        stream = torch.cuda.current_stream()
        for n, seed in ((1_000_003, 1), (70_001, 2)):
            g = np.random.default_rng(seed)
            cols = [g.integers(0, 200_000, n, dtype=np.int32) for _ in range(3)]
            cols[1][:2] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max]
            src = g.integers(0, 200_000, 40_000, dtype=np.int32)
            f = ctx.build_filter(ctx.load_relation([src], where="host"), 0, layout=layout, seed=seed)
            rel = ctx.load_relation(cols, where="host")
            exp = ctx.sieve(rel, [1], [f]).to_numpy()
            ref = oracle.sieve(cols, [(1, oracle.bloom_build(src, 8, 3, layout, seed))])
            nblocks, _, words = f.info()

            ins = [torch.from_numpy(c).cuda() for c in cols]
            outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in cols]
            count = torch.zeros(1, dtype=torch.int64, device="cuda")
            status = torch.zeros(1, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            rc, msg = _noalloc(lib, stream, ins, outs, n, 1, words, nblocks, f.params, count, status)
            assert rc == 0, msg
            torch.cuda.synchronize()
            k = int(count.item())
            assert k == len(exp[0]) == len(ref[0]) and 0 < k < n
            assert int(status.item()) == 0
            for j in range(3):
                got = outs[j][:k].cpu().numpy()
                assert np.array_equal(got, exp[j]) and np.array_equal(got, ref[j])


def test_noalloc_without_status_word_and_empty_input():
    """status NULL (the library keeps its own word) and an input of 0 rows,
    which must report 0 kept rows."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lib = sj.load_library()
    with sj.Context(0) as ctx:
        stream = torch.cuda.current_stream()
        g = np.random.default_rng(9)
        src = g.integers(0, 5000, 3000, dtype=np.int32)
        f = ctx.build_filter(ctx.load_relation([src], where="host"), 0)
        nblocks, _, words = f.info()
        cols = [g.integers(0, 10_000, 50_000, dtype=np.int32) for _ in range(2)]
        ref = oracle.sieve(cols, [(0, oracle.bloom_build(src))])
        ins = [torch.from_numpy(c).cuda() for c in cols]
        outs = [torch.empty(50_000, dtype=torch.int32, device="cuda") for _ in cols]
        count = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        rc, msg = _noalloc(lib, stream, ins, outs, 50_000, 0, words, nblocks, f.params, count, None)
        assert rc == 0, msg
        torch.cuda.synchronize()
        k = int(count.item())
        assert k == len(ref[0])
        for j in range(2):
            assert np.array_equal(outs[j][:k].cpu().numpy(), ref[j])
        count.fill_(-1)
        rc, msg = _noalloc(lib, stream, ins, outs, 0, 0, words, nblocks, f.params, count, None)
        assert rc == 0, msg
        torch.cuda.synchronize()
        assert int(count.item()) == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lib = sj.load_library()
    a = torch.zeros(16, dtype=torch.int32, device="cuda")
    words = torch.zeros(8, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    params = sj.FilterParams(8, 3, sj.BLOCKED256, 0, 0)
    err = ctypes.c_char_p()
    rc = lib.sj_sieve_noalloc(None, 1, _ptrs([a]), (1 << 27) + 1, 0, ctypes.c_void_p(words.data_ptr()),
                              1, ctypes.byref(params), _ptrs([a]), ctypes.c_void_p(count.data_ptr()),
                              None, ctypes.byref(err))
    assert rc == 1
    assert b"SJ_NOALLOC_MAX_ROWS" in err.value
