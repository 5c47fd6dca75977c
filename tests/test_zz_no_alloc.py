"""The allocation-free FP64 multiply, cht_multiply_f64_noalloc.

Some callers cannot allocate device memory while they run the product (a
serving process that reserves its whole memory budget up front, or code
whose device memory belongs to another framework's allocator).  This entry
point keeps its scratch -- the kernel's work counter -- in a static device
array instead of allocating it.  The test calls it through the C ABI twice in
a row (the second call must clear the counter left by the first) and checks
each result against cht_multiply's within the FP64 tolerance of the other
tests.  While it runs, the library's allocator is replaced by one that
counts calls and refuses them, so any allocation would show up.

This file is collected last so that a failure here does not hide the rest.
"""

from __future__ import annotations

import ctypes
import gc

import numpy as np
import pytest

import workloads as w
from tests import gpu_util as gu
from tests import setref

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-13

_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                         ctypes.c_void_p)


@pytest.mark.parametrize("case", ["banded_b32", "locality_b64"])
def test_noalloc_multiply_matches_cht_multiply(case):
    import torch
    cht = gu.cht()
    lib = cht.load()
    if case == "banded_b32":
        a, b = w.config1(2048, 32, 4)
    else:
        a, b = w.config2(8192)
    A, B = cht.from_block_matrix(a), cht.from_block_matrix(b)
    plan = cht.cht_symbolic_multiply(A, B)
    ref, _ = cht.cht_multiply(plan, A, B, sync=True)
    out = ref.like()          # the caller's output, allocated beforehand
    ref_vals = ref.values().cpu().numpy()
    out_vals = out.values()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    calls = {"alloc": 0, "free": 0}

    def refuse(nbytes, s, ctx):
        calls["alloc"] += 1
        return None

    def count_free(p, nbytes, s, ctx):
        calls["free"] += 1

    alloc_cb, free_cb = _ALLOC(refuse), _FREE(count_free)
    for _ in range(2):
        out_vals.fill_(float("nan"))
        torch.cuda.synchronize()
        gc.disable()
        assert lib.cht_set_allocator(alloc_cb, free_cb, None) == 0
        try:
            rc = lib.cht_multiply_f64_noalloc(plan.handle, A.handle, B.handle, out.handle, stream)
        finally:
            assert lib.cht_set_allocator(None, None, None) == 0
            gc.enable()
        assert rc == 0, lib.cht_last_error().decode()
        cht.sync_status()
        assert calls == {"alloc": 0, "free": 0}
        got = out_vals.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert setref.rel_fro(got, ref_vals) <= FP64_TOL


def test_noalloc_rejects_foreign_output():
    cht = gu.cht()
    lib = cht.load()
    a, b = w.config1(1024, 32, 2)
    A, B = cht.from_block_matrix(a), cht.from_block_matrix(b)
    plan = cht.cht_symbolic_multiply(A, B)
    rc = lib.cht_multiply_f64_noalloc(plan.handle, A.handle, B.handle, A.handle, None)
    assert rc == cht.CHT_ERR_INVALID


def test_noalloc_checks_operands_without_allocating():
    # The operand check compares patterns on the device with its flag in the
    # static array: a rebuilt operand (same leaves, another pattern object)
    # is accepted and gives cht_multiply's result, an operand with as many
    # leaves on another pattern is refused -- with the allocator refusing.
    import torch
    cht = gu.cht()
    lib = cht.load()
    a, b = w.config1(2048, 32, 4)
    A, B = cht.from_block_matrix(a), cht.from_block_matrix(b)
    plan = cht.cht_symbolic_multiply(A, B)
    ref, _ = cht.cht_multiply(plan, A, B, sync=True)
    ref_vals = ref.values().cpu().numpy()
    out = ref.like()
    A2 = cht.from_block_matrix(a)
    shifted = w.BlockMatrix(a.n, a.b, ((a.brow + 1) % a.grid).astype(np.int32), a.bcol.copy(),
                            a.vals.copy())
    As = cht.from_block_matrix(shifted)
    assert As.nblocks == A.nblocks
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    calls = {"alloc": 0, "free": 0}

    def refuse(nbytes, s, ctx):
        calls["alloc"] += 1
        return None

    def count_free(p, nbytes, s, ctx):
        calls["free"] += 1

    alloc_cb, free_cb = _ALLOC(refuse), _FREE(count_free)
    torch.cuda.synchronize()
    gc.disable()
    assert lib.cht_set_allocator(alloc_cb, free_cb, None) == 0
    try:
        rc_same = lib.cht_multiply_f64_noalloc(plan.handle, A2.handle, B.handle, out.handle,
                                               stream)
        rc_other = lib.cht_multiply_f64_noalloc(plan.handle, As.handle, B.handle, out.handle,
                                                stream)
    finally:
        assert lib.cht_set_allocator(None, None, None) == 0
        gc.enable()
    assert calls == {"alloc": 0, "free": 0}
    assert rc_same == 0, lib.cht_last_error().decode()
    assert rc_other == cht.CHT_ERR_SHAPE
    cht.sync_status()
    assert setref.rel_fro(out.values().cpu().numpy(), ref_vals) <= FP64_TOL
