"""GPU backward of C = A*B: dA = (dC B^T) on A's pattern and dB = (A^T dC) on
B's pattern, checked against the oracle, a dense FP64 torch gradient and
central finite differences of L = ||A B - T||_F^2."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as w
from tests import gpu_util as gu
from tests import setref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return gu.cht()


def _problem(lib, n=8192):
    a = w.banded(n, 64, 8, 1005)
    b = w.locality_matrix(w.lattice_points(n, 4005), 64, 6.0, 2005)
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    C, _ = lib.cht_multiply(plan, A, B, sync=True)
    crow, ccol = (t.cpu().numpy() for t in C.coords())
    t = w.values_on_pattern(n, 64, crow, ccol, 3005)
    T = gu.upload(lib, t)
    assert T.nblocks == C.nblocks
    tr, tc = (x.cpu().numpy() for x in T.coords())
    assert np.array_equal(tr, crow) and np.array_equal(tc, ccol)
    return a, b, A, B, plan, C, T


def _dc(lib, C, T):
    dC = C.like()
    dC.values().copy_(2.0 * (C.values() - T.values()))
    return dC


def _oracle_matrix(M):
    r, c, v = gu.host_leaves(M)
    return oracle.OMatrix.from_blocks(M.n, M.b, r, c, v)


def test_backward_matches_oracle(lib):
    a, b, A, B, plan, C, T = _problem(lib)
    dC = _dc(lib, C, T)
    dA, dB = lib.cht_multiply_backward(plan, A, B, dC)
    lib.sync_status()
    OdA, OdB = oracle.backward(oracle.OMatrix.from_block_matrix(a),
                               oracle.OMatrix.from_block_matrix(b), _oracle_matrix(dC))
    gu.assert_same_pattern(dA, OdA)
    gu.assert_same_pattern(dB, OdB)
    gu.assert_values_close(dA, OdA, 1e-13)
    gu.assert_values_close(dB, OdB, 1e-13)


def test_recomputed_pairs_give_identical_gradients(lib):
    _, _, A, B, plan, C, T = _problem(lib)
    dC = _dc(lib, C, T)
    dA1, dB1 = lib.cht_multiply_backward(plan, A, B, dC)
    dA2, dB2 = lib.cht_multiply_backward(None, A, B, dC, recompute_pairs=True)
    dA3, dB3 = lib.cht_multiply_backward(plan, A, B, dC, dA=dA1, dB=dB1)  # cached lists
    lib.sync_status()
    assert bool((dA1.values() == dA2.values()).all())
    assert bool((dB1.values() == dB2.values()).all())
    assert dA3 is dA1 and dB3 is dB1


def test_backward_matches_dense_torch(lib):
    import torch
    a, b, A, B, plan, C, T = _problem(lib)
    dC = _dc(lib, C, T)
    dA, dB = lib.cht_multiply_backward(plan, A, B, dC)
    lib.sync_status()
    dcd, ad, bd = dC.to_dense(), A.to_dense(), B.to_dense()
    g = a.n // a.b
    mask_a = torch.zeros(g, g, dtype=torch.float64, device="cuda")
    mask_a[torch.from_numpy(a.brow).long(), torch.from_numpy(a.bcol).long()] = 1.0
    mask_b = torch.zeros(g, g, dtype=torch.float64, device="cuda")
    mask_b[torch.from_numpy(b.brow).long(), torch.from_numpy(b.bcol).long()] = 1.0
    ones = torch.ones(a.b, a.b, dtype=torch.float64, device="cuda")
    ref_a = (dcd @ bd.T) * torch.kron(mask_a, ones)
    ref_b = (ad.T @ dcd) * torch.kron(mask_b, ones)
    got_a, got_b = dA.to_dense(), dB.to_dense()
    ea = float(torch.linalg.norm(got_a - ref_a) / torch.linalg.norm(ref_a))
    eb = float(torch.linalg.norm(got_b - ref_b) / torch.linalg.norm(ref_b))
    assert ea <= 1e-12 and eb <= 1e-12, (ea, eb)


def test_finite_differences(lib):
    # L is quadratic in each entry: central differences have no truncation
    # error.  Only the C row (for an A entry) or C column (for a B entry) that
    # the entry reaches changes, so L is summed over those leaves only.
    import torch
    a, b, A, B, plan, C, T = _problem(lib, n=4096)
    dC = _dc(lib, C, T)
    dA, dB = lib.cht_multiply_backward(plan, A, B, dC)
    lib.sync_status()
    crow, ccol = (x.long() for x in C.coords())
    tv = T.values()
    bs = a.b
    h = 1e-6
    rng = np.random.default_rng(11)

    def partial_loss(row=None, col=None):
        Cn, _ = lib.cht_multiply(plan, A, B, sync=True)
        diff = Cn.values() - tv
        if row is not None:
            sel = crow == row // bs
            return float((diff[sel][:, row % bs, :] ** 2).sum())
        sel = ccol == col // bs
        return float((diff[sel][:, :, col % bs] ** 2).sum())

    for which, M, G in (("A", A, dA), ("B", B, dB)):
        vals = M.values()
        br, bc = (x.cpu().numpy() for x in M.coords())
        gv = G.values()
        for _ in range(8):
            leaf = int(rng.integers(M.nblocks))
            r, c = int(rng.integers(bs)), int(rng.integers(bs))
            gi, gj = int(br[leaf]) * bs + r, int(bc[leaf]) * bs + c
            orig = float(vals[leaf, r, c])
            kw = {"row": gi} if which == "A" else {"col": gj}
            vals[leaf, r, c] = orig + h
            lp = partial_loss(**kw)
            vals[leaf, r, c] = orig - h
            lm = partial_loss(**kw)
            vals[leaf, r, c] = orig
            fd = (lp - lm) / (2 * h)
            an = float(gv[leaf, r, c])
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (which, fd, an)
    torch.cuda.synchronize()


def test_autograd_function(lib):
    import torch

    from paper_2011_11762_gb300 import autograd as cag
    a, b, A, B, plan, C, T = _problem(lib, n=4096)
    a_vals = A.values().requires_grad_()
    b_vals = B.values().requires_grad_()
    c, _ = cag.matmul(A, B, a_vals, b_vals, plan=plan)
    loss = ((c - T.values()) ** 2).sum()
    loss.backward()
    dC = _dc(lib, C, T)
    dA, dB = lib.cht_multiply_backward(plan, A, B, dC)
    lib.sync_status()
    assert torch.equal(a_vals.grad, dA.values())
    assert torch.equal(b_vals.grad, dB.values())
    # recompute mode (no stored pair lists) gives the same gradients
    a2 = A.values().detach().requires_grad_()
    b2 = B.values().detach().requires_grad_()
    c2, _ = cag.matmul(A, B, a2, b2, plan=plan, recompute_pairs=True)
    ((c2 - T.values()) ** 2).sum().backward()
    assert torch.equal(a2.grad, a_vals.grad) and torch.equal(b2.grad, b_vals.grad)


def test_backward_with_foreign_dc_pattern(lib):
    # dC with a pattern other than C's: only triples whose (I, J) dC stores
    a = w.banded(2048, 32, 3, 91)
    b = w.banded(2048, 32, 2, 92)
    d = w.random_blocks(2048, 32, 0.05, 93, dist="uniform")
    A, B, D = (gu.upload(lib, m) for m in (a, b, d))
    dA, dB = lib.cht_multiply_backward(None, A, B, D)
    lib.sync_status()
    OdA, OdB = oracle.backward(oracle.OMatrix.from_block_matrix(a),
                               oracle.OMatrix.from_block_matrix(b),
                               oracle.OMatrix.from_block_matrix(d))
    gu.assert_same_pattern(dA, OdA)
    gu.assert_values_close(dA, OdA, 1e-13)
    gu.assert_values_close(dB, OdB, 1e-13)
    _ = setref


def test_full_size_backward_sampled(lib):
    # the differentiation workload at its full size (N = 32768, 64x64 leaves,
    # A banded +-8, B 3D locality): sampled gradient leaves against the
    # oracle's single-leaf products dA(I,K) = (dC B^T)(I,K), dB(K,J) = (A^T dC)(K,J)
    a, b = w.config5()
    A, B = gu.upload(lib, a), gu.upload(lib, b)
    plan = lib.cht_symbolic_multiply(A, B)
    C, _ = lib.cht_multiply(plan, A, B, sync=True)
    crow, ccol = (t.cpu().numpy() for t in C.coords())
    T = gu.upload(lib, w.values_on_pattern(a.n, a.b, crow, ccol, w.SEED_T + 5))
    dC = _dc(lib, C, T)
    dA, dB = lib.cht_multiply_backward(plan, A, B, dC)
    lib.sync_status()
    OdC = _oracle_matrix(dC)
    OA, OB = oracle.OMatrix.from_block_matrix(a), oracle.OMatrix.from_block_matrix(b)
    OBt, OAt = OB.transpose(), OA.transpose()
    rng = np.random.default_rng(10)
    for M, left, right in ((dA, OdC, OBt), (dB, OAt, OdC)):
        r, c, v = gu.host_leaves(M)
        for i in list(rng.choice(r.shape[0], 8, replace=False)) + [0, r.shape[0] - 1]:
            ref, _ = oracle.leaf_product(left, right, int(r[i]), int(c[i]))
            assert setref.rel_fro(v[i], ref) <= 1e-13, (int(r[i]), int(c[i]))
