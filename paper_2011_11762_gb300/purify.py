"""McWeeny purification step X <- 3X^2 - 2X^3 with truncation, composed from
the library's calls (paper, Section 1 names density-matrix purification as
the application; Section 2.2 lists the symmetric square, symmetric
multiplication, addition and truncation it is built from).

Symmetric matrices stay as their upper-triangle leaves between the calls:
the two products are planned on I <= J only, and the truncation works on the
upper triangle with Frobenius tolerance eps / sqrt(2), so that the mirrored
full matrix loses at most eps.  Every arithmetic step runs in libcht's
kernels; this module only sequences the calls.
"""

from __future__ import annotations

import math

from . import (CHT_FP64, CHT_TRUNC_FRO, cht_add, cht_mat_mirror_upper, cht_multiply,
               cht_symbolic_multiply_symsquare, cht_symbolic_multiply_upper, cht_truncate)


def mcweeny_step(X, eps: float, mode: int = CHT_FP64, stream=None):
    """(X_next, info) for the full symmetric matrix X (a ``Matrix``); info
    holds the removed Frobenius norm, the leaf pairs of the two products and
    the leaves before and after truncation."""
    p1 = cht_symbolic_multiply_symsquare(X, stream=stream)
    x2u, _ = cht_multiply(p1, X, X, mode=mode, stream=stream)
    x2 = cht_mat_mirror_upper(x2u, stream=stream)
    p2 = cht_symbolic_multiply_upper(x2, X, stream=stream)
    x3u, _ = cht_multiply(p2, x2, X, mode=mode, stream=stream)
    yu = cht_add(3.0, x2u, -2.0, x3u, stream=stream)
    tu, removed = cht_truncate(yu, eps / math.sqrt(2.0), CHT_TRUNC_FRO, stream=stream)
    xn = cht_mat_mirror_upper(tu, stream=stream)
    info = {"removed": removed, "pairs": p1.npairs + p2.npairs,
            "flops": p1.useful_flops + p2.useful_flops,
            "leaves_upper": yu.nblocks, "leaves_upper_kept": tu.nblocks}
    return xn, info
