/*
 * CPU oracle for the block-sparse quadtree product C = A*B.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the GPU library: only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * build, load or call it.  It shares no code with the GPU path.
 *
 * Representation (paper, Section 2): a matrix is a sparse quadtree; a node is
 * either nil (the identically zero submatrix, a NULL pointer here), a dense
 * leaf of b x b doubles (row-major), or four quadrants [[11, 12], [21, 22]],
 * each again a sparse quadtree.  A grid of G x G leaves is padded virtually to
 * 2^D x 2^D with nil leaves (D = ceil(log2 G)).
 *
 * Every function returns 0 on success and a negative code on error:
 *   -1 invalid argument / out-of-range leaf coordinate,
 *   -2 shape mismatch, -3 duplicate leaf coordinate, -4 out of memory.
 */
#ifndef CHT_ORACLE_H
#define CHT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_mat orc_mat;

/* Build a quadtree from a list of leaves (any order): the paper's assignment
 * from matrix elements (Section 2.2: construction from row and column
 * indices and values), at leaf granularity.  Leaf i sits at leaf
 * coordinates (brow[i], bcol[i]) and holds vals[i*b*b .. (i+1)*b*b) in
 * row-major order.  Leaves whose values are all zero are identically zero
 * and are not stored (nil, Section 2).  n must be a positive multiple of b. */
int orc_build(int64_t n, int32_t b, int64_t nblk, const int32_t *brow,
              const int32_t *bcol, const double *vals, orc_mat **out);

/* C = A*B by the recursive quadtree algorithm (paper, Section 2: operations
 * recurse over the non-nil branches, a nil operand gives a nil product;
 * Section 2.2 lists the matrix-matrix multiplication); *npairs (may be
 * NULL) gets the number of leaf-times-leaf products performed. */
int orc_multiply(const orc_mat *A, const orc_mat *B, orc_mat **C,
                 int64_t *npairs);

/* Sparse approximate product (SpAMM; paper, Sections 1 and 2.2: the sparse
 * approximate multiplication for matrices with decay): the multiply
 * recursion in which a quadrant product is skipped (nil) whenever
 * ||A_sub||_F * ||B_sub||_F < tau, tested at every level including the
 * leaves.  tau = 0 is orc_multiply. */
int orc_multiply_spamm(const orc_mat *A, const orc_mat *B, double tau,
                       orc_mat **C, int64_t *npairs);

/* The upper triangle of C = A*B: its leaves (I, J) with I <= J, by the
 * multiply recursion in which a quadrant of C that lies wholly below the
 * diagonal is not formed.  For symmetric A and B = A this is the symmetric
 * square (paper, Section 2.2), whose lower leaves are the transposes. */
int orc_multiply_upper(const orc_mat *A, const orc_mat *B, orc_mat **C,
                       int64_t *npairs);

/* alpha*A + beta*B on the union of the patterns (paper, Section 2.2).  A leaf
 * on both sides is alpha*a + beta*b elementwise (two products, one sum,
 * no fused multiply-add); a leaf on one side only is alpha*a or beta*b.
 * Every leaf of the union is kept, even if it cancels to zero. */
int orc_add(double alpha, const orc_mat *A, double beta, const orc_mat *B, orc_mat **out);

/* alpha*A + beta*I (paper, Section 2.2, addition of a scaled identity): as
 * orc_add with B the identity, whose leaves are the diagonal leaves (I, I). */
int orc_add_identity(double alpha, const orc_mat *A, double beta, orc_mat **out);

/* Truncation (paper, Section 2.2: removal of small elements with error
 * control), at leaf granularity.  kind 0 (Frobenius): sort the leaves by
 * squared Frobenius norm, ascending (ties in Morton order), and remove them
 * in that order while the running sum of removed squared norms stays
 * <= eps^2; *removed = sqrt of that sum, so ||M - out||_F = *removed <= eps.
 * kind 1 (max norm): remove every leaf whose largest magnitude is <= eps;
 * *removed = the largest removed magnitude.  removed may be NULL. */
int orc_truncate(const orc_mat *M, double eps, int kind, orc_mat **out, double *removed);

/* The symmetric matrix whose upper triangle (element level) is U's: leaf
 * (J, I), I < J, is U's leaf (I, J) transposed; a diagonal leaf keeps its
 * entries on and above its diagonal and mirrors them below (paper, Section
 * 2.2: the symmetric operations, whose results are determined by one
 * triangle).  Every leaf of U is kept, all-zero or not.  -1 if U has a leaf
 * below the diagonal. */
int orc_mirror_upper(const orc_mat *U, orc_mat **out);

/* Transpose (a new matrix); a helper of the backward products below. */
int orc_transpose(const orc_mat *A, orc_mat **out);

/* The matrix with exactly M's pattern whose leaves are X's leaves where X has
 * one and zero leaves elsewhere; the pattern restriction of the backward
 * products below. */
int orc_restrict(const orc_mat *X, const orc_mat *M, orc_mat **out);

/* Gradients of L = f(C), C = A*B, given dC = dL/dC (the chain rule for the
 * product with the operands' patterns fixed; differentiation is not among
 * the paper's operations):
 * dA = (dC * B^T) on A's pattern, dB = (A^T * dC) on B's pattern. */
int orc_backward(const orc_mat *A, const orc_mat *B, const orc_mat *dC,
                 orc_mat **dA, orc_mat **dB);

/* One leaf of C = A*B straight from the definition of the block product,
 * C(I,J) = sum_K A(I,K) B(K,J), K ascending.  out: b*b doubles.
 * *present (may be NULL) is 1 when at least one K contributes. */
int orc_leaf_product(const orc_mat *A, const orc_mat *B, int64_t I, int64_t J,
                     double *out, int *present);

/* Number of stored leaves. */
int64_t orc_nleaves(const orc_mat *M);

/* Stored leaves in quadtree depth-first order (quadrants 11, 12, 21, 22),
 * which is the Morton (Z) order of the leaf coordinates.  Arrays sized by
 * orc_nleaves(); vals may be NULL to get the pattern only. */
int orc_extract(const orc_mat *M, int32_t *brow, int32_t *bcol, double *vals);

int64_t orc_dim(const orc_mat *M);
int32_t orc_leafsize(const orc_mat *M);
void orc_free(orc_mat *M);

/* Threads used by the parallel top levels of the recursion. */
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
