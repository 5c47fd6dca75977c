/*
 * libcht -- block-sparse quadtree matrix product C = A*B on one GB300 GPU.
 *
 * The paper (Chunks and Tasks Matrix Library 2.0, Section 2) represents a
 * matrix as a sparse quadtree: a node is identically zero (nil), a small dense
 * leaf matrix, or four quadrants that are again sparse quadtrees.  Its
 * functionality list (Section 2.2) starts with construction from index and
 * value vectors, extraction, and matrix-matrix multiplication; Section 3
 * demonstrates the multiplication on block-sparse matrices.
 *
 * This library keeps that contract on one GPU.  The quadtree is flattened:
 * the stored (non-nil) leaves of a matrix are kept in Morton (Z) order of
 * their leaf coordinates -- the order of a depth-first walk over quadrants
 * 11, 12, 21, 22 -- as one array of dense b x b FP64 leaves, row-major inside
 * each leaf.  The product runs in two phases:
 *   symbolic: the (A-leaf, B-leaf) pairs that meet on a shared inner index K
 *             and the product's leaf pattern (the boolean product of the two
 *             patterns), exact integer work;
 *   numeric:  one persistent kernel that sums, for every leaf (I, J) of C,
 *             the leaf products A(I,K) B(K,J) in ascending K.
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers; all others are host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls return without waiting for the
 *    GPU unless stated otherwise.
 *  - Inputs are copied: the caller keeps ownership of its buffers and may
 *    reuse them once the call's work on `stream` has completed.
 *  - Handles returned through out-parameters are owned by the caller and are
 *    released with cht_mat_free / cht_plan_free / cht_batch_free, in any
 *    order.  A handle's device memory is returned in the order of the stream
 *    that created it, which must outlive the handle; work on other streams
 *    that uses the handle must be complete (or ordered before) the free.
 *  - Every call returns a cht_status; on error no output handle is created
 *    and *out is left unchanged.  cht_last_error() gives a one-line reason.
 *  - Kernels never trap.  A device-side failure (a bounded wait that ran
 *    out) is recorded in a library-wide status word; calls that synchronise
 *    report it, and cht_sync_status() reads and clears it.
 */
#ifndef CHT_H
#define CHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cht_mat *cht_mat_t;     /* a block-sparse matrix on the GPU  */
typedef struct cht_plan *cht_plan_t;   /* symbolic result of A*B            */
typedef struct cht_batch *cht_batch_t; /* many products in one launch       */

typedef enum {
  CHT_OK = 0,
  CHT_ERR_INVALID = -1,     /* bad argument, leaf coordinate out of range */
  CHT_ERR_SHAPE = -2,       /* dimensions or leaf sizes do not match      */
  CHT_ERR_DUPLICATE = -3,   /* the same leaf coordinate given twice       */
  CHT_ERR_OOM = -4,         /* an allocation failed                       */
  CHT_ERR_CUDA = -5,        /* a CUDA runtime call failed                 */
  CHT_ERR_TIMEOUT = -6,     /* a bounded device-side wait ran out         */
  CHT_ERR_UNSUPPORTED = -7  /* valid request the library does not handle */
} cht_status;

typedef enum {
  CHT_FP64 = 0,       /* FP64 leaf products, FP64 accumulation             */
  CHT_SPLIT_BF16 = 1  /* FP64 operands split into BF16 slices, tcgen05 MMA  */
} cht_mode;

/* Leaf sizes the numeric kernels support. */
#define CHT_MIN_LEAF 32
#define CHT_MAX_LEAF 64

/* ------------------------------------------------------------------------
 * Memory.  By default the library allocates device memory with
 * cudaMallocAsync / cudaFreeAsync on the stream of the call.  A caller may
 * install its own allocator instead (e.g. a framework's caching allocator).
 * alloc returns NULL on failure (reported as CHT_ERR_OOM).  Passing NULL
 * for both restores the default.  Not thread-safe; call before other calls.
 * ---------------------------------------------------------------------- */
typedef void *(*cht_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*cht_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int cht_set_allocator(cht_alloc_fn alloc, cht_free_fn free_fn, void *ctx);

/* ------------------------------------------------------------------------
 * Construction (paper, Section 2.2, "Assignment from ... matrix elements":
 * construct a matrix from index vectors and values), at leaf granularity.
 *
 * n        matrix dimension; a positive multiple of b.
 * b        leaf size; CHT_MIN_LEAF <= b <= CHT_MAX_LEAF, a multiple of 8
 *          (the numeric kernels take b = 32 or b = 64).
 * nblocks  number of leaves given (0 is a valid, empty matrix).
 * d_brow, d_bcol  int32 leaf coordinates, 0 <= coordinate < n / b.
 * d_vals   nblocks * b * b doubles, 16-byte aligned; leaf i is
 *          d_vals[i*b*b ...], row-major.
 * All three arrays are device memory owned by the caller and copied; they
 * may be freed once the call returns.
 * Leaves may come in any order.  A leaf whose values are all zero is
 * identically zero (nil, Section 2) and is not stored.
 * Errors: CHT_ERR_INVALID (range, sizes, alignment, nblocks >= 2^31),
 * CHT_ERR_DUPLICATE (a coordinate given twice, zero leaves included),
 * CHT_ERR_UNSUPPORTED (more than 2^21 leaves per grid side: the pair keys
 * of the symbolic phase are 64-bit), CHT_ERR_OOM, CHT_ERR_CUDA.
 * Synchronises `stream` once, to validate the input and size the handle.
 * ---------------------------------------------------------------------- */
int cht_mat_from_blocks(int64_t n, int32_t b, int64_t nblocks,
                        const int32_t *d_brow, const int32_t *d_bcol,
                        const double *d_vals, void *stream, cht_mat_t *out);

/* Shape of a matrix: dimension, leaf size, number of stored leaves. */
int cht_mat_info(cht_mat_t M, int64_t *n, int32_t *b, int64_t *nblocks);

/* Device arrays of a matrix (owned by the handle, valid until it is freed):
 * leaf values [nblocks][b][b] in Morton order, and each leaf's (row, col).
 * Any out-pointer may be NULL.  The values may be written in place. */
int cht_mat_leaves(cht_mat_t M, double **d_vals, const int32_t **d_brow,
                   const int32_t **d_bcol);

/* Extraction (paper, Section 2.2): write M densely into the caller's
 * n x n row-major buffer d_out with leading dimension ld >= n (doubles).
 * The whole n x n region is overwritten (zeros outside stored leaves). */
int cht_to_dense(cht_mat_t M, double *d_out, int64_t ld, void *stream);

/* A new matrix with M's pattern (shared, not copied) and uninitialised
 * values, e.g. to hold a gradient dL/dM or a target on M's pattern. */
int cht_mat_like(cht_mat_t M, void *stream, cht_mat_t *out);

int cht_mat_free(cht_mat_t M);

/* ------------------------------------------------------------------------
 * Symbolic multiply (paper, Section 2: the multiply recursion visits only
 * non-nil quadrant pairs, and a nil operand gives a nil product).  Flattened:
 * every triple (I, K, J) with A(I,K) and B(K,J) stored is a pair; C's
 * pattern is the set of (I, J) with at least one pair (the boolean product of
 * the patterns; a leaf whose values later cancel to zero stays stored).
 * The plan holds C's pattern (Morton order), each C leaf's pair segment in
 * ascending K, and a longest-first work schedule.
 * A and B must have equal n and b (else CHT_ERR_SHAPE).
 * *nnzb_C and *npairs (either may be NULL) get the number of C leaves and of
 * pairs; the useful work of the numeric phase is 2 * b^3 * npairs flops.
 * Synchronises `stream` once, to read C's leaf count, the longest pair
 * segment and C's leaf counts per row and column: the pair list is sized
 * from the leaf counts per row and column that every pattern keeps on the
 * host (read when the pattern was made).  Grids of more than 65536 leaves
 * per side keep no such counts and cost one more synchronisation, as do
 * the filters of the _spamm, _symsquare and _upper variants.
 * ---------------------------------------------------------------------- */
int cht_symbolic_multiply(cht_mat_t A, cht_mat_t B, void *stream,
                          cht_plan_t *out, int64_t *nnzb_C, int64_t *npairs);

/* Sparse approximate symbolic multiply (paper, Section 2.2: "sparse
 * approximate multiplication", for matrices with decay): as
 * cht_symbolic_multiply, but a pair (A(I,K), B(K,J)) is kept only if
 * ||A(I,K)||_F * ||B(K,J)||_F >= tau (FP64 Frobenius norms of the current
 * leaf values).  This is the leaf-level form of the SpAMM recursion, which
 * skips a quadrant product whenever the product of the quadrants' norms is
 * below tau: an ancestor's norms bound its leaves', so the pairs the
 * recursion keeps are exactly those passing the leaf test.  The numeric
 * phase (either mode) runs unchanged on the plan.  C's pattern holds the
 * leaves with at least one kept pair.  The dropped pairs bound the error:
 * ||C - A*B||_F <= sum over dropped pairs of ||A(I,K)||_F ||B(K,J)||_F.
 * tau = 0 keeps every pair.  Synchronises `stream` four times. */
int cht_symbolic_multiply_spamm(cht_mat_t A, cht_mat_t B, double tau, void *stream,
                                cht_plan_t *out, int64_t *nnzb_C, int64_t *npairs);

/* Symmetric square (paper, Section 2.2: "symmetric matrix square"): the plan
 * of C = A*A for a symmetric A (A = A^T; not checked) restricted to the
 * upper triangle, the C leaves (I, J) with I <= J -- C is symmetric, so they
 * determine it, at about half the work.  Run the numeric phase with
 * cht_multiply(plan, A, A, ...); cht_mat_mirror_upper then gives the full C.
 * Synchronises `stream` four times. */
int cht_symbolic_multiply_symsquare(cht_mat_t A, void *stream, cht_plan_t *out,
                                    int64_t *nnzb_C, int64_t *npairs);

/* The plan of the upper-triangle leaves (I <= J) of C = A*B, for products
 * known to be symmetric though A and B differ (paper, Section 2.2 lists
 * symmetric multiplication; e.g. X^2 * X in a purification step, where the
 * factors are commuting symmetric matrices).  Nothing about symmetry is
 * checked.  cht_symbolic_multiply_symsquare(A) is this call with B = A.
 * Synchronises `stream` four times. */
int cht_symbolic_multiply_upper(cht_mat_t A, cht_mat_t B, void *stream, cht_plan_t *out,
                                int64_t *nnzb_C, int64_t *npairs);

/* The full symmetric matrix whose upper triangle is that of U, at element
 * level: leaf (J, I), I < J, of the result is leaf (I, J) of U transposed,
 * and a diagonal leaf (I, I) keeps the entries (r, c), r <= c, of U's and
 * takes its entries r > c from (c, r), so the result is exactly symmetric
 * even where U's diagonal leaves are not (rounding in a product).  Every
 * leaf of U is kept, all-zero or not.  U must hold no leaf below the diagonal
 * (CHT_ERR_INVALID otherwise, nothing created).  Synchronises `stream`
 * twice. */
int cht_mat_mirror_upper(cht_mat_t U, void *stream, cht_mat_t *out);

/* ------------------------------------------------------------------------
 * Matrix addition and truncation (paper, Section 2.2: "matrix addition",
 * including the addition of a scaled identity, and "truncation", the
 * removal of small elements with error control).  These are the building
 * blocks, with the product, of purification-style iterations such as
 * X <- 3X^2 - 2X^3.
 * ---------------------------------------------------------------------- */

/* *out = alpha*A + beta*B on the union of the two leaf patterns (Morton
 * order).  A leaf stored in both is alpha*a + beta*b elementwise, each
 * product and the sum rounded separately (no fused multiply-add), so results
 * are reproducible bit for bit; a leaf stored in one operand only is that
 * operand's scaled leaf.  Every union leaf is stored, even one that cancels
 * to zero (truncation is a separate call).  CHT_ERR_SHAPE if n or b differ.
 * Synchronises `stream` once. */
int cht_add(double alpha, cht_mat_t A, double beta, cht_mat_t B, void *stream,
            cht_mat_t *out);

/* *out = alpha*A + beta*I: cht_add with B the identity, whose stored leaves
 * are the G diagonal leaves (I, I) (1 on their diagonal, 0 elsewhere).
 * Synchronises `stream` once. */
int cht_add_identity(double alpha, cht_mat_t A, double beta, void *stream, cht_mat_t *out);

typedef enum {
  CHT_TRUNC_FRO = 0, /* removed part has Frobenius norm <= eps (greedy,     */
                     /* smallest leaves first)                               */
  CHT_TRUNC_MAX = 1  /* removed leaves have every |entry| <= eps            */
} cht_trunc_kind;

/* Truncation at leaf granularity: *out holds the leaves of M that are kept,
 * values unchanged, in Morton order; a removed leaf becomes nil.
 *  CHT_TRUNC_FRO: leaves sorted by squared Frobenius norm, ascending, ties
 *    in Morton order; with S_r the prefix sums of the sorted squared norms,
 *    the leaves before the first rank r with S_r > eps^2 are removed.
 *    *removed (may be NULL) = sqrt(S) of the removed leaves, <= eps.
 *  CHT_TRUNC_MAX: a leaf is removed iff its largest magnitude is <= eps;
 *    *removed = the largest removed magnitude (max-norm error).
 * eps = 0 removes exactly the all-zero leaves.  CHT_ERR_INVALID for eps < 0,
 * NaN eps or an unknown kind.  Synchronises `stream` once. */
int cht_truncate(cht_mat_t M, double eps, int kind, void *stream, cht_mat_t *out,
                 double *removed);

/* Plan counts; any out-pointer may be NULL. */
int cht_plan_info(cht_plan_t P, int64_t *nnzb_C, int64_t *npairs);

/* Plan arrays (device, owned by the plan): pair segments cseg[nnzb_C + 1]
 * (int64), for each pair the A leaf and B leaf (Morton indices, int32),
 * each C leaf's (row, col), and the schedule order[nnzb_C].  Any
 * out-pointer may be NULL. */
int cht_plan_arrays(cht_plan_t P, const int64_t **d_cseg,
                    const int32_t **d_pair_a, const int32_t **d_pair_b,
                    const int32_t **d_crow, const int32_t **d_ccol,
                    const int32_t **d_order);

int cht_plan_free(cht_plan_t P);

/* ------------------------------------------------------------------------
 * Numeric multiply C = A*B on a plan from cht_symbolic_multiply(A, B).
 * mode     CHT_FP64, or CHT_SPLIT_BF16 with `nslices` BF16 slices per
 *          operand (ignored for CHT_FP64).
 * *C       in/out.  If *C is NULL a new matrix on the plan's pattern is
 *          created.  If *C is a matrix previously produced from this plan,
 *          its values are overwritten in place (no allocation).
 * max_rel_err_est  may be NULL.  If given, the call synchronises `stream`,
 *          returns any device-side failure (e.g. CHT_ERR_TIMEOUT), and
 *          stores an a-priori bound on |C - A*B| / (|A| |B|) elementwise.
 * Each C leaf is summed in ascending K by one CTA: results are bitwise
 * reproducible run to run.  No atomics touch C.
 * CHT_SPLIT_BF16: nslices = 0 or 6 (6 digits of 8 bits per operand, 48
 * bits); inputs must be finite; b = 32 or 64.  At b = 32 the pairs of the
 * C leaves with at most 4 leaf pairs are computed by a kernel that stacks
 * four of them sharing a B leaf in one MMA (slice pairs i + j <= 7; a C
 * leaf of several pairs has its pairs' exact integer results summed and
 * rounded once, with one int64 scratch leaf per such pair); the other C
 * leaves by the general kernel (8 A digits, 4 stacked A slices).  The first
 * such multiply on a plan groups those pairs (from counts the symbolic phase
 * took, without a synchronisation) and keeps the groups in the plan.  The
 * B operand's pre-kernels run on a second stream of the calling thread,
 * joined to `stream` before the numeric kernels.  One work unit sums at most
 * 1016 (b = 64) or 4000 (b = 32) leaf pairs exactly; a C leaf with more is
 * cut into equal pieces whose sums are added in FP64 in piece order (still
 * reproducible; scratch of one leaf per piece).  The bound returned is
 * relative to 2^(e_r + f_c), the powers of two just above the largest |A|
 * in row r and |B| in column c.
 * Operand check: A and B must store the leaves of the plan's operands, since
 * the plan's pair lists index their leaves.  The matrices the plan was made
 * from pass at once; other matrices (e.g. rebuilt from the same blocks) are
 * compared leaf key by leaf key on the device, which synchronises `stream`
 * once.  Operands with another pattern -- even one with the same leaf count,
 * such as plan(A, B) given (B, A) -- are refused with CHT_ERR_SHAPE before
 * any work is queued.
 * ---------------------------------------------------------------------- */
int cht_multiply(cht_plan_t plan, cht_mat_t A, cht_mat_t B, int mode,
                 int32_t nslices, void *stream, cht_mat_t *C,
                 double *max_rel_err_est);

/* ------------------------------------------------------------------------
 * FP64 numeric multiply straight to host memory: the leaf values of C
 * (Morton order, the layout of cht_mat_leaves on the plan's pattern, nnzb_C
 * x b x b doubles) are written to h_C, which the caller owns and should have
 * allocated page-locked (cudaHostAlloc / pinned) for the copies to overlap.
 * The C leaves are cut into `nchunks` contiguous ranges; each range is one
 * launch of the FP64 kernel (longest pair segment first inside the range)
 * and is copied to h_C on an internal stream while the next range computes,
 * so the device-to-host transfer hides behind the arithmetic.  Values equal
 * those of cht_multiply(..., CHT_FP64, ...) bit for bit.  Returns after
 * enqueuing; `stream` is ordered after the last copy (synchronise it before
 * reading h_C).  Device scratch: C itself, freed in stream order.
 * CHT_ERR_INVALID for a NULL h_C or nchunks < 1; operands checked against
 * the plan as in cht_multiply (CHT_ERR_SHAPE).
 * ---------------------------------------------------------------------- */
int cht_multiply_to_host(cht_plan_t plan, cht_mat_t A, cht_mat_t B, void *stream,
                         double *h_C, int32_t nchunks);

/* ------------------------------------------------------------------------
 * Allocation-free FP64 numeric multiply.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory on the
 * call path -- for example a serving process that reserves its whole device
 * memory budget at start-up and may not grow it per request, or code whose
 * device memory belongs to another framework's allocator.  cht_multiply
 * takes an 8-byte work counter from the stream-ordered pool on every call
 * (and allocates C when *C is NULL); this call allocates nothing.
 *
 * Computes the same C = A*B as cht_multiply(plan, A, B, CHT_FP64, ...) with
 * the same kernel, writing into C, which must already exist on the plan's
 * product pattern (a matrix returned by cht_multiply for this plan, or
 * cht_mat_like of one).  Returns without waiting for the GPU.
 * Scratch: a file-scope device array of 256 bytes (held by every GPU that
 * loads the library until the process exits); this call uses its first
 * 8 bytes as the work counter and clears them at every call, and the next
 * 4 bytes as the flag of the operand check (cleared before each use).
 * Operands are checked against the plan as in cht_multiply: when they are
 * not the matrices the plan was made from, that check synchronises `stream`
 * once and refuses another pattern with CHT_ERR_SHAPE.  The array is
 * shared by all calls on a device: calls whose kernels overlap on the GPU
 * (e.g. on two streams) race on it and give wrong results -- order them.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.
 * Limits: at most 2^31 - 1 output leaves per call (else
 * CHT_ERR_UNSUPPORTED); b = 32 or 64.  Errors as for cht_multiply, plus
 * CHT_ERR_INVALID when C is not on the plan's pattern.
 * ---------------------------------------------------------------------- */
int cht_multiply_f64_noalloc(cht_plan_t plan, cht_mat_t A, cht_mat_t B,
                             cht_mat_t C, void *stream);

/* ------------------------------------------------------------------------
 * Backward of C = A*B for a loss L(C), given dC = dL/dC (differentiation
 * is not among the paper's operations: this is the chain rule of the
 * product with the operands' patterns held fixed):
 *   dA = (dC * B^T) restricted to A's pattern,
 *   dB = (A^T * dC) restricted to B's pattern
 * (sampled block products: only the stored leaves of A and B are outputs;
 * a stored leaf that no triple reaches gets zeros).
 * plan             the forward plan, or NULL.
 * recompute_pairs  nonzero (or plan == NULL): rebuild the triples from the
 *                  patterns of A, B and dC instead of reading the plan's
 *                  pair list (for when the plan's lists were not kept).
 *                  With a plan and dC produced from that plan, the plan's
 *                  pairs are regrouped (cached in the plan).
 * *dA, *dB         in/out as for cht_multiply (NULL = create; a matrix with
 *                  A's / B's pattern from an earlier call = overwrite).
 *                  Either pointer may be NULL to skip that gradient.
 * ---------------------------------------------------------------------- */
int cht_multiply_backward(cht_plan_t plan, cht_mat_t A, cht_mat_t B,
                          cht_mat_t dC, int recompute_pairs, void *stream,
                          cht_mat_t *dA, cht_mat_t *dB);

/* ------------------------------------------------------------------------
 * Batched products (not an operation of the paper, whose task templates
 * leave the scheduling of independent tasks to the runtime, Section 2.1;
 * here many products share one launch): `count` independent products
 * C_i = A_i * B_i, each with its own plan (own n and leaf size), computed
 * by ONE persistent kernel
 * launch whose work list concatenates all products' C leaves in
 * longest-first order.  cht_batch_create allocates every output and all
 * launch tables (and may synchronise); cht_batch_run only launches (no
 * allocation, no synchronisation), so it may be captured in a CUDA graph.
 * cht_batch_output gives a non-owning view of C_i (valid while the batch
 * lives; do not free it).  In CHT_SPLIT_BF16 mode a C leaf with more leaf
 * pairs than one unit sums (1016 at b = 64, 4000 at b = 32) is cut into
 * pieces as in cht_multiply; cht_batch_create prepares them (scratch of one
 * leaf per piece) and cht_batch_run adds them after the launch.
 * cht_batch_create checks every product's operands against its plan as
 * cht_multiply does (CHT_ERR_SHAPE).
 * ---------------------------------------------------------------------- */
int cht_batch_create(int32_t count, const cht_plan_t *plans,
                     const cht_mat_t *As, const cht_mat_t *Bs, int mode,
                     int32_t nslices, void *stream, cht_batch_t *out);
int cht_batch_run(cht_batch_t batch, void *stream);
int cht_batch_output(cht_batch_t batch, int32_t i, cht_mat_t *C);
int cht_batch_free(cht_batch_t batch);

/* ------------------------------------------------------------------------
 * Options (library-wide, not thread-safe).
 * ---------------------------------------------------------------------- */
typedef enum {
  CHT_OPT_SCHEDULE = 0,       /* 0 = longest-first (default), 1 = Morton   */
  CHT_OPT_WAIT_BUDGET_NS = 1, /* bound of each device-side wait, ns
                                 (default 2e9; 0 makes every wait expire:
                                 a test hook for the timeout path)         */
  CHT_OPT_CTAS_PER_SM = 2,    /* persistent grid = SMs * this (0 = auto)   */
  CHT_OPT_FP64_ENGINE = 3,    /* 0 = DMMA (mma.sync f64); 1 = DFMA (default:
                                 faster than DMMA on GB300; 256-thread CTAs
                                 with 4 x 4 register tiles at b = 64, 128
                                 threads at b = 32); 2 = DFMA with 128-thread
                                 CTAs (4 x 8 tiles) at b = 64 as well      */
  CHT_OPT_SPLIT_SINGLE = 4    /* split form, 32-leaves: 1 (default) = the
                                 pairs of C leaves with at most 4 leaf pairs
                                 go to the kernel that groups them by B leaf
                                 (see cht_multiply); 0 = every C leaf to the
                                 general kernel                            */
} cht_option;
int cht_set_option(int option, int64_t value);
int cht_get_option(int option, int64_t *value);

/* Synchronise `stream`, then read and clear the device status word:
 * CHT_OK or the first recorded device-side failure (CHT_ERR_TIMEOUT). */
int cht_sync_status(void *stream);

/* Kernels launched by this library since load (counted on the host). */
int64_t cht_launch_count(void);

/* Human-readable name of a status code, and the last error's detail. */
const char *cht_status_str(int status);
const char *cht_last_error(void);

/* Measure the FP64 arithmetic peak of this GPU (the denominator of the FP64
 * kernels' roofline; no passage of the paper): register-resident kernels on
 * every SM, timed with CUDA events on `stream`, which is synchronised.
 * engine 1: `chains` independent FP64 FMA chains per thread; engine 2: a
 * 4 x 8 register tile of FMAs from 12 operand registers (the leaf GEMM's
 * inner loop without its loads; `chains` ignored); engine 3: the leaf
 * GEMM's own inner loop (DFMA register tile fed from shared memory) over one
 * pair of b x b leaves held in shared memory, b = `chains` (32 or 64), 128
 * threads; engine 0: `chains` independent mma.sync m8n8k4 f64 chains per
 * warp.  `threads` per CTA (a multiple of 32, at most 1024 and at most what
 * the kernel's registers allow), `ctas_per_sm` CTAs on each SM (1..32);
 * chains 4, 8, 16 or 32.  *tflops gets FLOP/s / 1e12 of one ~40 ms launch
 * after a warm-up launch.  CHT_ERR_INVALID for other arguments.
 * cht_measure_fp64_peak returns the best of chains {8, 16, 32} (engine 3:
 * b = 32, 64) x {1, 2, 4} CTAs per SM for the engine (256 threads; engine 3:
 * 128). */
int cht_measure_fp64_peak(int engine, void *stream, double *tflops);
int cht_measure_fp64_peak_cfg(int engine, int chains, int threads, int ctas_per_sm,
                              void *stream, double *tflops);

#ifdef __cplusplus
}
#endif
#endif /* CHT_H */
