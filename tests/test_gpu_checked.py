"""The bounds-checked debug build on valid plans.

Compiled with -DCHT_BOUNDS_CHECK, every kernel tests each leaf, pair and unit
index it follows against the length of its array before using it, and a bad
one is recorded in the device status word instead of being read.  A child
process loads that build (CHT_BOUNDS_CHECK=1) and runs every numeric path on
valid plans -- FP64 and split form at 32- and 64-leaves (the split form's
one-pair kernel included), backward, batch, host output and the
allocation-free call -- each followed by a status check that must come back
clean, and each result against the oracle.  No invalid index is planted on
the GPU: the checks are exercised for their cost and their silence.
"""

from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import ctypes
import numpy as np
import torch
import oracle
import paper_2011_11762_gb300 as cht
import workloads as w
from tests import gpu_util as gu

assert cht.library_path().endswith("libcht_checked.so"), cht.library_path()
cht.load()


def check(M, Om, tol):
    cht.sync_status()
    gu.assert_same_pattern(M, Om)
    gu.assert_values_close(M, Om, tol, leaf_tol=None if tol > 1e-13 else tol)


cases = {
    "banded_b32": w.config1(1024, 32, 4),
    "random_b32": (w.random_blocks(4096, 32, 0.02, 71), w.random_blocks(4096, 32, 0.02, 72)),
    "locality_b64": w.config2(8192),
}
for name, (a, b) in cases.items():
    A, B = cht.from_block_matrix(a), cht.from_block_matrix(b)
    plan = cht.cht_symbolic_multiply(A, B)
    Co, _ = gu.oracle_product(a, b)
    C, _ = cht.cht_multiply(plan, A, B, sync=True)
    check(C, Co, 1e-13)
    Cs, _ = cht.cht_multiply(plan, A, B, mode=cht.CHT_SPLIT_BF16, sync=True)
    check(Cs, Co, 1e-11)
    out = torch.empty((plan.nnzb_C, a.b, a.b), dtype=torch.float64, pin_memory=True)
    cht.cht_multiply_to_host(plan, A, B, out, nchunks=3)
    torch.cuda.current_stream().synchronize()
    cht.sync_status()
    assert torch.equal(out, C.values().cpu())
    lib = cht.load()
    D = C.like()
    rc = lib.cht_multiply_f64_noalloc(plan.handle, A.handle, B.handle, D.handle,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    cht.sync_status()
    assert torch.equal(D.values(), C.values())
    dA, dB = cht.cht_multiply_backward(plan, A, B, C)
    dA2, dB2 = cht.cht_multiply_backward(plan, A, B, C, recompute_pairs=True)
    cht.sync_status()
    assert torch.equal(dA.values(), dA2.values()) and torch.equal(dB.values(), dB2.values())
    print(name, "ok", flush=True)

prods = w.batched_products(count=6, scale=0.12)
mats = []
for i, (_, a, b) in enumerate(prods):
    if i % 2 == 0:
        a, b = w.reblock(a, 64), w.reblock(b, 64)
    mats.append((cht.from_block_matrix(a), cht.from_block_matrix(b), a, b))
plans = [cht.cht_symbolic_multiply(A, B) for A, B, _, _ in mats]
for mode, tol in ((cht.CHT_FP64, 1e-13), (cht.CHT_SPLIT_BF16, 1e-11)):
    bt = cht.Batch(plans, [m[0] for m in mats], [m[1] for m in mats], mode=mode)
    bt.run()
    cht.sync_status()
    for i, (_, _, a, b) in enumerate(mats):
        Co, _ = gu.oracle_product(a, b)
        check(bt.output(i), Co, tol)
print("CHECKED BUILD OK", flush=True)
"""


def test_checked_build_runs_valid_plans_cleanly():
    pytest.importorskip("torch")
    env = dict(os.environ, CHT_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "CHECKED BUILD OK" in r.stdout
