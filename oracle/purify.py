"""CPU oracle of one step of McWeeny purification with truncation.

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU-baseline
leg, nothing else.

Density-matrix purification (paper, Section 1) iterates a matrix polynomial
that pushes every eigenvalue of a symmetric X, with spectrum in [0, 1],
towards 0 or 1.  The McWeeny step is X <- 3X^2 - 2X^3, built from the
library operations of Section 2.2: the symmetric square, a symmetric product
(X^2 commutes with X, so X^2 X is symmetric), matrix addition and
truncation.  Symmetric matrices are kept as their upper-triangle leaves
(I <= J) between the products, and the step truncates that upper triangle
with Frobenius control eps / sqrt(2): a removed leaf off the diagonal stands
for two leaves of the full matrix, so the full matrix loses at most eps.
"""

from __future__ import annotations

import math


def mcweeny_step(X, eps: float):
    """(X_next, removed, pairs) for the full symmetric oracle matrix X.

    X2 = upper(X X) mirrored; X3u = upper(X2 X); Yu = 3 X2u - 2 X3u;
    X_next = mirror(truncate(Yu, eps / sqrt 2)); removed = Frobenius norm of
    what the truncation took from the upper triangle; pairs = leaf products
    of the two upper-triangle products."""
    x2u, p1 = X.multiply_upper(X)
    x2 = x2u.mirror_upper()
    x3u, p2 = x2.multiply_upper(X)
    yu = x2u.add(3.0, x3u, -2.0)
    tu, removed = yu.truncate(eps / math.sqrt(2.0), 0)
    return tu.mirror_upper(), removed, p1 + p2
