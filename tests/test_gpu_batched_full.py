"""The batched workload at its stated size against the oracle.

64 independent products, N_i log-uniform in [2048, 32768] (rounded down to a
multiple of 64), structures cycling banded (+-4 leaves) / 3D locality
(cutoff 6) / random leaves (p = 0.02), leaf size 32 or 64 chosen per product
by the autotuner, all products in ONE batched launch, in FP64 and in the
split form.  For every product:

* the C pattern, in Morton order, equals the boolean block product bit for
  bit, and every C leaf's pair segment has exactly as many pairs as that
  product has inner indices K (sparse product of the 0/1 leaf patterns);
* sampled C leaves -- the one with the longest pair segment, the first, the
  last and three random ones -- equal the oracle's single-leaf product
  (the definition C_IJ = sum_K A_IK B_KJ, K ascending): FP64 within 1e-13
  relative Frobenius per leaf; the split form elementwise within its
  a-priori bound K (s + 3) 2^(-s w) 2^(e_r + f_c), with e_r and f_c the
  exponents of the largest |a| in row r of A and |b| in column c of B;
* products of at most 2 GFLOP are also compared whole with the oracle's
  product (pattern and every leaf).
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as w
from tests import gpu_util as gu
from tests import setref

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-13
S, W = 6, 8                 # split form: slices and bits per slice
FULL_ORACLE_FLOPS = 2e9     # compare whole products up to this size


@pytest.fixture(scope="module")
def lib():
    return gu.cht()


@pytest.fixture(scope="module")
def products():
    return w.batched_products()


def _line_exponents(m, axis):
    """frexp exponent of the largest |value| of every global row (axis 1) or
    column (axis 0) of m; lines without a stored value get 0."""
    b = m.b
    vmax = np.abs(m.vals).max(axis=2 if axis == 1 else 1)  # [nblk, b]
    lead = m.brow if axis == 1 else m.bcol
    lines = (lead.astype(np.int64)[:, None] * b + np.arange(b)[None, :]).ravel()
    out = np.zeros(m.n)
    np.maximum.at(out, lines, vmax.ravel())
    _, e = np.frexp(out)
    return np.where(out > 0, e, 0).astype(np.int64)


def _check_pattern(out, plan, a, b):
    crow, ccol = (t.cpu().numpy().astype(np.int64) for t in out.coords())
    seg = np.diff(plan.arrays()["cseg"].numpy())
    assert np.all(np.diff(oracle.morton_key(crow, ccol)) > 0)  # Morton order
    I, J, cnt = setref.product_pattern_counts(a.brow, a.bcol, b.brow, b.bcol, a.grid)
    rm = np.lexsort((ccol, crow))
    assert np.array_equal(crow[rm], I) and np.array_equal(ccol[rm], J)
    assert np.array_equal(seg[rm], cnt)
    return crow, ccol, seg


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_full_batch_matches_oracle(lib, products, mode):
    import torch

    from paper_2011_11762_gb300 import autotune
    m = lib.CHT_FP64 if mode == "fp64" else lib.CHT_SPLIT_BF16
    spec = [(a.n, (torch.from_numpy(a.brow), torch.from_numpy(a.bcol), torch.from_numpy(a.vals)),
             (torch.from_numpy(b.brow), torch.from_numpy(b.bcol), torch.from_numpy(b.vals)))
            for _, a, b in products]
    tuned = autotune.tune(spec, mode=m, reps=1, cache_path=None)
    bt = tuned.batch
    for i in range(bt.count):
        bt.output(i).values().fill_(float("nan"))
    bt.run()
    lib.sync_status()
    assert len(products) == 64 and set(tuned.leaf_sizes) <= {32, 64}
    rng = np.random.default_rng(404)
    whole = 0
    for i, (kind, a32, b32) in enumerate(products):
        bs = tuned.leaf_sizes[i]
        a = a32 if bs == 32 else w.reblock(a32, bs)
        b = b32 if bs == 32 else w.reblock(b32, bs)
        plan, out = tuned.plans[i], bt.output(i)
        crow, ccol, seg = _check_pattern(out, plan, a, b)
        got = out.values().cpu().numpy()
        assert np.all(np.isfinite(got)), i
        if mode == "split":
            e, f = _line_exponents(a, 1), _line_exponents(b, 0)
        OA, OB = oracle.OMatrix.from_block_matrix(a), oracle.OMatrix.from_block_matrix(b)
        nC = crow.shape[0]
        picks = {int(np.argmax(seg)), 0, nC - 1,
                 *rng.choice(nC, min(3, nC), replace=False).tolist()}
        for c in sorted(picks):
            ref, present = oracle.leaf_product(OA, OB, int(crow[c]), int(ccol[c]))
            assert present, (i, c)
            if mode == "fp64":
                assert setref.rel_fro(got[c], ref) <= FP64_TOL, (i, kind, c)
            else:
                r0, c0 = int(crow[c]) * bs, int(ccol[c]) * bs
                scale = np.ldexp(1.0, e[r0:r0 + bs, None] + f[None, c0:c0 + bs])
                K = bs * int(seg[c])
                tol = scale * (K * (S + 3) * 2.0 ** (-S * W) + 2.0 ** -50 + K * 2.0 ** -52)
                assert np.all(np.abs(got[c] - ref) <= tol), (i, kind, c)
        if plan.useful_flops <= FULL_ORACLE_FLOPS:
            whole += 1
            Co, npairs = OA.multiply(OB)
            assert plan.npairs == npairs
            gu.assert_same_pattern(out, Co)
            if mode == "fp64":
                gu.assert_values_close(out, Co, FP64_TOL)
            else:
                _, _, ov = Co.leaves()
                for c in range(nC):
                    r0, c0 = int(crow[c]) * bs, int(ccol[c]) * bs
                    scale = np.ldexp(1.0, e[r0:r0 + bs, None] + f[None, c0:c0 + bs])
                    K = bs * int(seg[c])
                    tol = scale * (K * (S + 3) * 2.0 ** (-S * W) + 2.0 ** -50 + K * 2.0 ** -52)
                    assert np.all(np.abs(got[c] - ov[c]) <= tol), (i, kind, c)
    print(f"{mode}: leaf sizes {tuned.leaf_sizes.count(32)} x 32, "
          f"{tuned.leaf_sizes.count(64)} x 64; {whole} products compared whole")
    assert whole >= 16
