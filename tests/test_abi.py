"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads,
and exports every entry point that include/sievejoin.h declares."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2308_16370_b300 as sj
from paper_2308_16370_b300 import build as sjbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sievejoin.h")


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^SJ_API\s+[\w\s\*]*?\b(sj_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    return sjbuild.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("sj_load_relation", "sj_build_filter", "sj_sieve_path", "sj_join"):
        assert s in syms
    assert sorted(sj.EXPORTS) == syms


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib_path], text=True)
    exported = set(re.findall(r"\bT (sj_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_library_is_built_for_sm_103a(lib_path):
    out = subprocess.check_output(["/usr/local/cuda/bin/cuobjdump", "--list-elf", lib_path], text=True)
    assert "sm_103a" in out


def test_binding_loads_and_reports_version(lib_path):
    lib = sj.load_library()
    assert lib.sj_version().decode().count(".") == 2
    assert lib.sj_status_str(3).decode() == "hash table full"


def test_no_cpu_fallback_without_gpu(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(RuntimeError):
        sj.Context(0)


def test_create_rejects_mismatched_allocator(lib_path):
    lib = sj.load_library()
    h = ctypes.c_void_p()
    # alloc given without free: rejected before any device call
    cb = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)(lambda n, u: None)
    assert lib.sj_create(ctypes.byref(h), 0, None, ctypes.cast(cb, ctypes.c_void_p), None, None) == 1


def test_serving_pool_same_columns_through_torch():
    """The pool generator's torch path (used for full-size pools on the GPU)
    gives the numpy path's columns exactly."""
    from paper_2308_16370_b300 import inputs
    a = inputs.serving_pool(nrel=4, min_rows=100, max_rows=50_000, domain=1 << 12, seed=3)
    b = inputs.serving_pool(nrel=4, min_rows=100, max_rows=50_000, domain=1 << 12, seed=3, device="cpu")
    for ra, rb in zip(a, b):
        for ca, cb in zip(ra, rb):
            assert ca.dtype == cb.dtype == np.int32 and np.array_equal(ca, cb)
