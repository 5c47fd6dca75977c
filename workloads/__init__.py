"""Seeded synthetic inputs for the block-sparse quadtree product C = A·B.

This package is shared by the CPU oracle's tests and by the GPU path's tests
and benchmark.  It only *draws* inputs (block patterns and leaf values); it
holds none of the product's arithmetic.

Structures follow the workloads of the paper's illustrative examples
(Section 3: banded matrices, plus structures with locality) and the five
GB300 workloads:

1. banded leaves, |I - J| <= 4, N = 4096, 32x32 leaves, U[-1, 1] entries;
2. 3D-locality ("electronic-structure-like"): jittered cubic lattice,
   Morton-ordered points grouped into 64-point leaves, leaf (I, J) present iff
   the minimum distance between the two point groups is < 6, entries
   exp(-0.5 r) * U[-1, 1];
3. random leaves present with probability 0.01, N(0, 1) entries;
4. a batch of 64 products of log-uniform size with cycling structures;
5. a banded-times-3D product with a dense-on-pattern target for
   L = ||A·B - T||_F^2.
"""

from .structures import (  # noqa: F401
    BlockMatrix,
    banded,
    lattice_dims_for,
    lattice_points,
    locality_pattern,
    locality_matrix,
    random_blocks,
    values_on_pattern,
    dense_line_pair,
    reblock,
    symmetrize,
    structure_column_counts,
    structure_flops,
    growing_block_size,
    random_blocks_layout,
    band_with_blocks,
    table1_structure,
    gershgorin_bounds,
    config2_symmetric,
    batched_products,
    config1,
    config2,
    config3,
    config5,
    SEED_A,
    SEED_B,
    SEED_T,
    SEED_GEOM,
)
