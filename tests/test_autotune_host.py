"""Host-side logic of the batch autotuner, on the CPU: the leaf reblocking
(merging f x f leaves with zero fill) against the element-level matrix and
against the numpy reblocking of the input generators; the pattern signature
that keys the decision cache; the cache file round trip."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as w
from paper_2011_11762_gb300 import autotune


def _dense(n, b, brow, bcol, vals):
    d = np.zeros((n, n))
    for r, c, v in zip(np.asarray(brow), np.asarray(bcol), np.asarray(vals)):
        d[r * b:(r + 1) * b, c * b:(c + 1) * b] = v
    return d


@pytest.mark.parametrize("n,b,b_new,p", [(512, 32, 64, 0.1), (512, 32, 128, 0.05),
                                          (384, 32, 64, 0.2), (256, 16, 64, 0.3)])
def test_reblock_keeps_the_element_matrix(n, b, b_new, p):
    a = w.random_blocks(n, b, p, 11)
    r, c, v = autotune.reblock(n, b, torch.from_numpy(a.brow), torch.from_numpy(a.bcol),
                               torch.from_numpy(a.vals), b_new, device="cpu")
    assert v.shape[1:] == (b_new, b_new) and v.dtype == torch.float64
    assert np.array_equal(_dense(n, b_new, r, c, v), a.to_dense())
    # one merged leaf per occupied b_new x b_new block, row-major order
    f = b_new // b
    occupied = sorted({(int(i) // f, int(j) // f) for i, j in zip(a.brow, a.bcol)})
    assert list(zip(r.tolist(), c.tolist())) == occupied
    ref = w.reblock(a, b_new)
    assert np.array_equal(r.numpy(), ref.brow) and np.array_equal(c.numpy(), ref.bcol)
    assert np.array_equal(v.numpy(), ref.vals)


def test_reblock_same_size_and_invalid_sizes():
    a = w.random_blocks(256, 32, 0.2, 3)
    out = autotune.reblock(256, 32, a.brow, a.bcol, a.vals, 32, device="cpu")
    assert out[0] is a.brow and out[1] is a.bcol and out[2] is a.vals
    with pytest.raises(ValueError):
        autotune.reblock(256, 32, a.brow, a.bcol, a.vals, 48, device="cpu")
    with pytest.raises(ValueError):
        autotune.reblock(384, 32, a.brow, a.bcol, a.vals, 256, device="cpu")


def test_signature_depends_on_pattern_and_mode_only():
    a = w.random_blocks(512, 32, 0.1, 5)
    b = w.random_blocks(512, 32, 0.1, 6)
    sa, sb = (a.brow, a.bcol, a.vals), (b.brow, b.bcol, b.vals)
    s0 = autotune._signature(512, sa, sb, 0)
    # other values on the same pattern: same signature
    assert autotune._signature(512, (a.brow, a.bcol, 2 * a.vals), sb, 0) == s0
    assert autotune._signature(512, sa, sb, 1) != s0
    assert autotune._signature(1024, sa, sb, 0) != s0
    assert autotune._signature(512, sb, sa, 0) != s0
    moved = (a.brow, (a.bcol + 1) % 16, a.vals)
    assert autotune._signature(512, moved, sb, 0) != s0


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "autotune.json")
    assert autotune._load_cache(path) == {}
    cache = {"abc": {"leaf": 64, "ms": [1.5, 2.0]}, "def": {"leaf": 32, "ms": [0.5]}}
    autotune._save_cache(path, cache)
    assert autotune._load_cache(path) == cache
    with open(path, "w") as f:
        f.write("{not json")
    assert autotune._load_cache(path) == {}
