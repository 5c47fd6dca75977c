/*
 * CPU oracle for the block-sparse quadtree product C = A*B (plain C, FP64).
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg.  It shares no code with the GPU library and
 * is deliberately plain: no blocking, no vectorisation, no reordering beyond
 * what the paper's recursion states.  Build with -ffp-contract=off so that
 * every product and every sum is rounded on its own.
 *
 * Paper, Section 2: a matrix is either identically zero (nil), a small dense
 * leaf, or four quadrants that are again sparse quadtrees; operations are
 * recursive algorithms over the non-nil branches, and a nil operand is handled
 * by a fallback that yields nil.  The multiply below is that recursion:
 *
 *   mul(A, B) = nil                          if A or B is nil,
 *             = dense leaf product           if both are leaves,
 *             = [[A11 B11 + A12 B21, A11 B12 + A12 B22],
 *                [A21 B11 + A22 B21, A21 B12 + A22 B22]]   otherwise,
 *   add(nil, X) = add(X, nil) = X.
 *
 * A leaf of the product that is structurally present is kept even if its
 * values cancel to zero (the product's pattern is the boolean product of the
 * operands' patterns); truncation is a separate operation in the paper.
 * Input leaves whose values are all zero are identically zero, i.e. nil.
 *
 * ORC_MUTANT (0 by default) plants one deliberate mistake, used only by the
 * tests that show the oracle's pins catch such mistakes.
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

typedef struct node {
    double *leaf;      /* non-NULL only at level 0 */
    struct node *q[4]; /* quadrants 11, 12, 21, 22 (index 2*row + col) */
} node;

struct orc_mat {
    int64_t n;
    int32_t b;
    int64_t grid;  /* G = n / b leaves per side */
    int depth;     /* D = ceil(log2 G); the root covers 2^D x 2^D leaves */
    node *root;
};

/* recursion levels (from the root) that are split into OpenMP tasks */
#define PAR_LEVELS 3

static void *xcalloc(size_t n, size_t sz) {
    void *p = calloc(n, sz);
    if (!p && n && sz) {
        fprintf(stderr, "oracle: out of memory\n");
        abort();
    }
    return p;
}

static node *new_node(void) { return (node *)xcalloc(1, sizeof(node)); }

static void free_tree(node *x) {
    if (!x) return;
    free(x->leaf);
    for (int i = 0; i < 4; ++i) free_tree(x->q[i]);
    free(x);
}

static int depth_for(int64_t grid) {
    int d = 0;
    while (((int64_t)1 << d) < grid) ++d;
    return d;
}

static orc_mat *new_mat(int64_t n, int32_t b) {
    orc_mat *m = (orc_mat *)xcalloc(1, sizeof(orc_mat));
    m->n = n;
    m->b = b;
    m->grid = n / b;
    m->depth = depth_for(m->grid);
    return m;
}

/* ---------------------------------------------------------------- build -- */

static int cmp_i64(const void *x, const void *y) {
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    return (a > b) - (a < b);
}

/* Store leaf (I, J) with values v (transposed if trans) in m. */
static void insert_leaf(orc_mat *m, int64_t I, int64_t J, const double *v, int trans) {
    const int bs = m->b;
    node **slot = &m->root;
    for (int lev = m->depth;; --lev) {
        if (!*slot) *slot = new_node();
        if (lev == 0) break;
        int qi = (int)((I >> (lev - 1)) & 1);
        int qj = (int)((J >> (lev - 1)) & 1);
        slot = &(*slot)->q[2 * qi + qj];
    }
    double *leaf = (double *)xcalloc((size_t)bs * bs, sizeof(double));
    for (int r = 0; r < bs; ++r)
        for (int c = 0; c < bs; ++c)
            leaf[(size_t)r * bs + c] = trans ? v[(size_t)c * bs + r] : v[(size_t)r * bs + c];
    (*slot)->leaf = leaf;
}

int orc_build(int64_t n, int32_t b, int64_t nblk, const int32_t *brow,
              const int32_t *bcol, const double *vals, orc_mat **out) {
    if (!out || n <= 0 || b <= 0 || n % b || nblk < 0) return -1;
    if (nblk && (!brow || !bcol || !vals)) return -1;
    int64_t grid = n / b;
    /* coordinates in range and pairwise distinct (zero leaves included) */
    int64_t *keys = (int64_t *)xcalloc(nblk ? nblk : 1, sizeof(int64_t));
    for (int64_t i = 0; i < nblk; ++i) {
        if (brow[i] < 0 || bcol[i] < 0 || brow[i] >= grid || bcol[i] >= grid) {
            free(keys);
            return -1;
        }
        keys[i] = (int64_t)brow[i] * grid + bcol[i];
    }
    qsort(keys, (size_t)nblk, sizeof(int64_t), cmp_i64);
    for (int64_t i = 1; i < nblk; ++i)
        if (keys[i] == keys[i - 1]) {
            free(keys);
            return -3;
        }
    free(keys);

    orc_mat *m = new_mat(n, b);
    size_t lsz = (size_t)b * b;
    for (int64_t i = 0; i < nblk; ++i) {
        const double *v = vals + (size_t)i * lsz;
        int nonzero = 0;
        for (size_t e = 0; e < lsz; ++e)
            if (v[e] != 0.0) { nonzero = 1; break; }
        if (!nonzero) continue; /* identically zero: nil */
        insert_leaf(m, brow[i], bcol[i], v, 0);
    }
    *out = m;
    return 0;
}

/* ------------------------------------------------------------- multiply -- */

/* c = a * b for dense row-major b x b leaves: c_ij = sum_k a_ik b_kj. */
static void leaf_mul(const double *a, const double *bm, double *c, int bs) {
    for (int i = 0; i < bs; ++i)
        for (int j = 0; j < bs; ++j) {
            double s = 0.0;
            for (int k = 0; k < bs; ++k) {
#if ORC_MUTANT == 2
                s += a[(size_t)k * bs + i] * bm[(size_t)k * bs + j];
#else
                s += a[(size_t)i * bs + k] * bm[(size_t)k * bs + j];
#endif
            }
            c[(size_t)i * bs + j] = s;
        }
}

/* x + y, consuming both (either may be nil). */
static node *add(node *x, node *y, int lev, int bs) {
    if (!x) return y;
    if (!y) return x;
    if (lev == 0) {
        size_t lsz = (size_t)bs * bs;
#if ORC_MUTANT == 3
        for (size_t e = 0; e < lsz; ++e) x->leaf[e] -= y->leaf[e];
#else
        for (size_t e = 0; e < lsz; ++e) x->leaf[e] += y->leaf[e];
#endif
        free_tree(y);
        return x;
    }
    for (int i = 0; i < 4; ++i) x->q[i] = add(x->q[i], y->q[i], lev - 1, bs);
    free(y);
    return x;
}

static node *mul(const node *a, const node *b, int lev, int bs,
                 int64_t *npairs, int par) {
    if (!a || !b) return NULL; /* fallback: a nil operand gives nil */
    if (lev == 0) {
        node *c = new_node();
        c->leaf = (double *)xcalloc((size_t)bs * bs, sizeof(double));
        leaf_mul(a->leaf, b->leaf, c->leaf, bs);
#pragma omp atomic
        ++*npairs;
        return c;
    }
    /* t[2*(2i+j)+k] = A_ik * B_kj */
    node *t[8];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k) {
#if ORC_MUTANT == 4
                const node *bk = b->q[2 * j + k];
#else
                const node *bk = b->q[2 * k + j];
#endif
                const node *ak = a->q[2 * i + k];
                node **slot = &t[2 * (2 * i + j) + k];
#pragma omp task firstprivate(ak, bk, slot) if (par > 0)
                *slot = mul(ak, bk, lev - 1, bs, npairs, par - 1);
            }
#pragma omp taskwait
    node *c = new_node();
    int any = 0;
    for (int ij = 0; ij < 4; ++ij) {
#if ORC_MUTANT == 1
        free_tree(t[2 * ij + 1]);
        c->q[ij] = t[2 * ij];
#else
        c->q[ij] = add(t[2 * ij], t[2 * ij + 1], lev - 1, bs);
#endif
        any |= c->q[ij] != NULL;
    }
    if (!any) {
        free(c);
        return NULL;
    }
    return c;
}

int orc_multiply(const orc_mat *A, const orc_mat *B, orc_mat **C,
                 int64_t *npairs) {
    if (!A || !B || !C) return -1;
    if (A->n != B->n || A->b != B->b) return -2;
    orc_mat *m = new_mat(A->n, A->b);
    int64_t np = 0;
#pragma omp parallel
#pragma omp single
    m->root = mul(A->root, B->root, A->depth, A->b, &np, PAR_LEVELS);
    if (npairs) *npairs = np;
    *C = m;
    return 0;
}

/* ---------------------------------------------------- sparse approximate -- */

/* squared Frobenius norm of a subtree */
static double fro2(const node *x, int lev, int bs) {
    if (!x) return 0.0;
    if (lev == 0) {
        double s = 0.0;
        for (size_t e = 0; e < (size_t)bs * bs; ++e) s += x->leaf[e] * x->leaf[e];
        return s;
    }
    double s = 0.0;
    for (int i = 0; i < 4; ++i) s += fro2(x->q[i], lev - 1, bs);
    return s;
}

static node *mul_spamm(const node *a, const node *b, int lev, int bs, double tau,
                       int64_t *npairs) {
    if (!a || !b) return NULL;
#if ORC_MUTANT == 8
    if (fro2(a, lev, bs) * fro2(b, lev, bs) < tau) return NULL; /* squared norms */
#else
    if (sqrt(fro2(a, lev, bs)) * sqrt(fro2(b, lev, bs)) < tau) return NULL;
#endif
    if (lev == 0) {
        node *c = new_node();
        c->leaf = (double *)xcalloc((size_t)bs * bs, sizeof(double));
        leaf_mul(a->leaf, b->leaf, c->leaf, bs);
        ++*npairs;
        return c;
    }
    node *t[8];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k)
                t[2 * (2 * i + j) + k] =
                    mul_spamm(a->q[2 * i + k], b->q[2 * k + j], lev - 1, bs, tau, npairs);
    node *c = new_node();
    int any = 0;
    for (int ij = 0; ij < 4; ++ij) {
        c->q[ij] = add(t[2 * ij], t[2 * ij + 1], lev - 1, bs);
        any |= c->q[ij] != NULL;
    }
    if (!any) {
        free(c);
        return NULL;
    }
    return c;
}

int orc_multiply_spamm(const orc_mat *A, const orc_mat *B, double tau,
                       orc_mat **C, int64_t *npairs) {
    if (!A || !B || !C || !(tau >= 0.0)) return -1;
    if (A->n != B->n || A->b != B->b) return -2;
    orc_mat *m = new_mat(A->n, A->b);
    int64_t np = 0;
    m->root = mul_spamm(A->root, B->root, A->depth, A->b, tau, &np);
    if (npairs) *npairs = np;
    *C = m;
    return 0;
}

/* ------------------------------------------------------- upper triangle -- */

/* The leaves (I, J), I <= J, of a*b for a node on the diagonal of C: the
 * quadrants 11 and 22 are again on the diagonal, quadrant 12 lies wholly
 * above it (every product), quadrant 21 wholly below it (skipped). */
static node *mul_upper(const node *a, const node *b, int lev, int bs,
                       int64_t *npairs, int par) {
    if (!a || !b) return NULL;
    if (lev == 0) return mul(a, b, 0, bs, npairs, 0);
    node *t[8] = {0};
    for (int i = 0; i < 2; ++i)
        for (int j = i; j < 2; ++j)
            for (int k = 0; k < 2; ++k) {
                const node *ak = a->q[2 * i + k], *bk = b->q[2 * k + j];
                node **slot = &t[2 * (2 * i + j) + k];
#if ORC_MUTANT == 5
#pragma omp task firstprivate(ak, bk, slot) if (par > 0)
                *slot = mul_upper(ak, bk, lev - 1, bs, npairs, par - 1);
#else
                if (i == j) {
#pragma omp task firstprivate(ak, bk, slot) if (par > 0)
                    *slot = mul_upper(ak, bk, lev - 1, bs, npairs, par - 1);
                } else {
#pragma omp task firstprivate(ak, bk, slot) if (par > 0)
                    *slot = mul(ak, bk, lev - 1, bs, npairs, par - 1);
                }
#endif
            }
#pragma omp taskwait
    node *c = new_node();
    int any = 0;
    for (int ij = 0; ij < 4; ++ij) {
        c->q[ij] = add(t[2 * ij], t[2 * ij + 1], lev - 1, bs);
        any |= c->q[ij] != NULL;
    }
    if (!any) {
        free(c);
        return NULL;
    }
    return c;
}

int orc_multiply_upper(const orc_mat *A, const orc_mat *B, orc_mat **C,
                       int64_t *npairs) {
    if (!A || !B || !C) return -1;
    if (A->n != B->n || A->b != B->b) return -2;
    orc_mat *m = new_mat(A->n, A->b);
    int64_t np = 0;
#pragma omp parallel
#pragma omp single
    m->root = mul_upper(A->root, B->root, A->depth, A->b, &np, PAR_LEVELS);
    if (npairs) *npairs = np;
    *C = m;
    return 0;
}

/* ------------------------------------------------ transpose / restrict -- */

static node *transpose_rec(const node *x, int lev, int bs) {
    if (!x) return NULL;
    node *t = new_node();
    if (lev == 0) {
        t->leaf = (double *)xcalloc((size_t)bs * bs, sizeof(double));
        for (int i = 0; i < bs; ++i)
            for (int j = 0; j < bs; ++j)
                t->leaf[(size_t)j * bs + i] = x->leaf[(size_t)i * bs + j];
        return t;
    }
    t->q[0] = transpose_rec(x->q[0], lev - 1, bs);
    t->q[1] = transpose_rec(x->q[2], lev - 1, bs);
    t->q[2] = transpose_rec(x->q[1], lev - 1, bs);
    t->q[3] = transpose_rec(x->q[3], lev - 1, bs);
    return t;
}

int orc_transpose(const orc_mat *A, orc_mat **out) {
    if (!A || !out) return -1;
    orc_mat *m = new_mat(A->n, A->b);
    m->root = transpose_rec(A->root, A->depth, A->b);
    *out = m;
    return 0;
}

static node *restrict_rec(const node *x, const node *m, int lev, int bs) {
    if (!m) return NULL;
    node *c = new_node();
    if (lev == 0) {
        c->leaf = (double *)xcalloc((size_t)bs * bs, sizeof(double));
        if (x) memcpy(c->leaf, x->leaf, (size_t)bs * bs * sizeof(double));
        return c;
    }
    for (int i = 0; i < 4; ++i)
        c->q[i] = restrict_rec(x ? x->q[i] : NULL, m->q[i], lev - 1, bs);
    return c;
}

int orc_restrict(const orc_mat *X, const orc_mat *M, orc_mat **out) {
    if (!X || !M || !out) return -1;
    if (X->n != M->n || X->b != M->b) return -2;
    orc_mat *m = new_mat(M->n, M->b);
    m->root = restrict_rec(X->root, M->root, M->depth, M->b);
    *out = m;
    return 0;
}

int orc_backward(const orc_mat *A, const orc_mat *B, const orc_mat *dC,
                 orc_mat **dA, orc_mat **dB) {
    if (!A || !B || !dC || !dA || !dB) return -1;
    if (A->n != B->n || A->b != B->b || dC->n != A->n || dC->b != A->b)
        return -2;
    orc_mat *bt, *at, *p;
    int rc = 0;
    /* dA = (dC * B^T) on A's pattern */
    orc_transpose(B, &bt);
    orc_multiply(dC, bt, &p, NULL);
    rc |= orc_restrict(p, A, dA);
    orc_free(p);
    orc_free(bt);
    /* dB = (A^T * dC) on B's pattern */
    orc_transpose(A, &at);
    orc_multiply(at, dC, &p, NULL);
    rc |= orc_restrict(p, B, dB);
    orc_free(p);
    orc_free(at);
    return rc;
}

/* ------------------------------------------------------------ addition -- */

/* alpha*x + beta*y as a new tree on the union of the two patterns (paper,
 * Section 2.2, matrix addition).  A leaf present on one side only is that
 * side's scaled copy; a leaf present on both is alpha*x + beta*y elementwise
 * (two products, then one sum).  idn != 0 makes y the identity: y is not read,
 * and the leaf (I, I) of y, for every leaf row I < grid, holds 1 on its
 * diagonal and 0 elsewhere. */
static node *add_rec(double alpha, const node *x, double beta, const node *y, int idn,
                     int lev, int bs, int64_t I, int64_t grid) {
    const int ydiag = idn && I < grid; /* this node carries identity leaves */
    if (!x && !y && !ydiag) return NULL;
    node *c = new_node();
    if (lev == 0) {
        size_t lsz = (size_t)bs * bs;
        c->leaf = (double *)xcalloc(lsz, sizeof(double));
        for (int r = 0; r < bs; ++r)
            for (int q = 0; q < bs; ++q) {
                size_t e = (size_t)r * bs + q;
                int have_y = idn ? ydiag : y != NULL;
                double yv = idn ? (r == q ? 1.0 : 0.0) : (y ? y->leaf[e] : 0.0);
#if ORC_MUTANT == 6
                if (x && have_y) c->leaf[e] = alpha * x->leaf[e] + beta * yv;
                else if (x) c->leaf[e] = x->leaf[e];
                else c->leaf[e] = beta * yv;
#else
                if (x && have_y) c->leaf[e] = alpha * x->leaf[e] + beta * yv;
                else if (x) c->leaf[e] = alpha * x->leaf[e];
                else c->leaf[e] = beta * yv;
#endif
            }
        return c;
    }
    const int64_t half = (int64_t)1 << (lev - 1);
    for (int qi = 0; qi < 2; ++qi)
        for (int qj = 0; qj < 2; ++qj) {
            const int k = 2 * qi + qj;
            /* identity leaves lie only in the diagonal quadrants */
            const int sub_idn = idn && qi == qj;
            c->q[k] = add_rec(alpha, x ? x->q[k] : NULL, beta,
                              idn ? NULL : (y ? y->q[k] : NULL), sub_idn, lev - 1, bs,
                              I + qi * half, grid);
        }
    if (!c->q[0] && !c->q[1] && !c->q[2] && !c->q[3]) {
        free(c);
        return NULL;
    }
    return c;
}

int orc_add(double alpha, const orc_mat *A, double beta, const orc_mat *B, orc_mat **out) {
    if (!A || !B || !out) return -1;
    if (A->n != B->n || A->b != B->b) return -2;
    orc_mat *m = new_mat(A->n, A->b);
    m->root = add_rec(alpha, A->root, beta, B->root, 0, A->depth, A->b, 0, A->grid);
    *out = m;
    return 0;
}

int orc_add_identity(double alpha, const orc_mat *A, double beta, orc_mat **out) {
    if (!A || !out) return -1;
    orc_mat *m = new_mat(A->n, A->b);
    m->root = add_rec(alpha, A->root, beta, NULL, 1, A->depth, A->b, 0, A->grid);
    *out = m;
    return 0;
}

/* ---------------------------------------------------------- truncation -- */

typedef struct {
    double key;  /* squared Frobenius norm, or largest magnitude */
    int64_t pos; /* position in Morton order (ties: earlier first) */
} leaf_key;

static int cmp_leaf_key(const void *x, const void *y) {
    const leaf_key *a = (const leaf_key *)x, *b = (const leaf_key *)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->pos > b->pos) - (a->pos < b->pos);
}

int orc_truncate(const orc_mat *M, double eps, int kind, orc_mat **out, double *removed) {
    if (!M || !out || !(eps >= 0.0) || (kind != 0 && kind != 1)) return -1;
    const int64_t nl = orc_nleaves(M);
    const size_t lsz = (size_t)M->b * M->b;
    int32_t *br = (int32_t *)xcalloc(nl ? nl : 1, sizeof(int32_t));
    int32_t *bc = (int32_t *)xcalloc(nl ? nl : 1, sizeof(int32_t));
    double *v = (double *)xcalloc((nl ? nl : 1) * lsz, sizeof(double));
    orc_extract(M, br, bc, v);
    leaf_key *k = (leaf_key *)xcalloc(nl ? nl : 1, sizeof(leaf_key));
    char *drop = (char *)xcalloc(nl ? nl : 1, 1);
    double rem = 0.0;
    for (int64_t l = 0; l < nl; ++l) {
        double s = 0.0;
        for (size_t e = 0; e < lsz; ++e) {
            double a = v[(size_t)l * lsz + e];
            if (kind == 0) s += a * a;
            else if (fabs(a) > s) s = fabs(a);
        }
        k[l].key = s;
        k[l].pos = l;
    }
    if (kind == 0) {
        /* Frobenius-norm control: remove the leaves of smallest norm, in
         * ascending order, while the removed squared norm stays <= eps^2 */
        qsort(k, (size_t)nl, sizeof(leaf_key), cmp_leaf_key);
        double acc = 0.0;
        for (int64_t r = 0; r < nl; ++r) {
#if ORC_MUTANT == 7
            double next = acc + k[nl - 1 - r].key;
            if (!(next <= eps * eps)) break;
            acc = next;
            drop[k[nl - 1 - r].pos] = 1;
#else
            double next = acc + k[r].key;
            if (!(next <= eps * eps)) break;
            acc = next;
            drop[k[r].pos] = 1;
#endif
        }
        rem = sqrt(acc);
    } else {
        /* max-norm control: remove every leaf whose entries are all <= eps */
        for (int64_t l = 0; l < nl; ++l)
            if (k[l].key <= eps) {
                drop[l] = 1;
                if (k[l].key > rem) rem = k[l].key;
            }
    }
    int64_t w = 0;
    for (int64_t l = 0; l < nl; ++l) {
        if (drop[l]) continue;
        br[w] = br[l];
        bc[w] = bc[l];
        memmove(v + (size_t)w * lsz, v + (size_t)l * lsz, lsz * sizeof(double));
        ++w;
    }
    int rc = orc_build(M->n, M->b, w, br, bc, v, out);
    if (removed) *removed = rem;
    free(br);
    free(bc);
    free(v);
    free(k);
    free(drop);
    return rc;
}

/* --------------------------------------------------------------- mirror -- */

int orc_mirror_upper(const orc_mat *U, orc_mat **out) {
    if (!U || !out) return -1;
    const int64_t nl = orc_nleaves(U);
    const size_t lsz = (size_t)U->b * U->b;
    int32_t *br = (int32_t *)xcalloc(nl ? nl : 1, sizeof(int32_t));
    int32_t *bc = (int32_t *)xcalloc(nl ? nl : 1, sizeof(int32_t));
    double *v = (double *)xcalloc((nl ? nl : 1) * lsz, sizeof(double));
    orc_extract(U, br, bc, v);
    int rc = 0;
    for (int64_t l = 0; l < nl; ++l)
        if (br[l] > bc[l]) rc = -1;
    if (rc == 0) {
        orc_mat *m = new_mat(U->n, U->b);
        const int bs = U->b;
        for (int64_t l = 0; l < nl; ++l) {
            double *x = v + (size_t)l * lsz;
#if ORC_MUTANT != 9 /* mutant 9 leaves diagonal leaves as they are */
            if (br[l] == bc[l]) /* diagonal leaf: upper triangle mirrored */
                for (int r = 0; r < bs; ++r)
                    for (int c = 0; c < r; ++c) x[(size_t)r * bs + c] = x[(size_t)c * bs + r];
#endif
            insert_leaf(m, br[l], bc[l], x, 0);
            if (br[l] != bc[l]) insert_leaf(m, bc[l], br[l], x, 1);
        }
        *out = m;
    }
    free(br);
    free(bc);
    free(v);
    return rc;
}

/* --------------------------------------------------- one leaf of A*B -- */

static const double *lookup(const orc_mat *M, int64_t I, int64_t J) {
    const node *x = M->root;
    for (int lev = M->depth; x && lev > 0; --lev) {
        int qi = (int)((I >> (lev - 1)) & 1), qj = (int)((J >> (lev - 1)) & 1);
        x = x->q[2 * qi + qj];
    }
    return x ? x->leaf : NULL;
}

int orc_leaf_product(const orc_mat *A, const orc_mat *B, int64_t I, int64_t J,
                     double *out, int *present) {
    if (!A || !B || !out) return -1;
    if (A->n != B->n || A->b != B->b) return -2;
    if (I < 0 || J < 0 || I >= A->grid || J >= A->grid) return -1;
    int bs = A->b;
    size_t lsz = (size_t)bs * bs;
    double *tmp = (double *)xcalloc(lsz, sizeof(double));
    memset(out, 0, lsz * sizeof(double));
    int any = 0;
    for (int64_t K = 0; K < A->grid; ++K) {
        const double *a = lookup(A, I, K), *b = lookup(B, K, J);
        if (!a || !b) continue;
        leaf_mul(a, b, tmp, bs);
        for (size_t e = 0; e < lsz; ++e) out[e] += tmp[e];
        any = 1;
    }
    free(tmp);
    if (present) *present = any;
    return 0;
}

/* ------------------------------------------------------------- extract -- */

static int64_t count_rec(const node *x, int lev) {
    if (!x) return 0;
    if (lev == 0) return 1;
    int64_t s = 0;
    for (int i = 0; i < 4; ++i) s += count_rec(x->q[i], lev - 1);
    return s;
}

int64_t orc_nleaves(const orc_mat *M) { return M ? count_rec(M->root, M->depth) : 0; }

static void extract_rec(const node *x, int lev, int64_t I, int64_t J, int bs,
                        int32_t *brow, int32_t *bcol, double *vals, int64_t *k) {
    if (!x) return;
    if (lev == 0) {
        brow[*k] = (int32_t)I;
        bcol[*k] = (int32_t)J;
        if (vals)
            memcpy(vals + (size_t)(*k) * bs * bs, x->leaf,
                   (size_t)bs * bs * sizeof(double));
        ++*k;
        return;
    }
    int64_t h = (int64_t)1 << (lev - 1);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            extract_rec(x->q[2 * i + j], lev - 1, I + i * h, J + j * h, bs, brow,
                        bcol, vals, k);
}

int orc_extract(const orc_mat *M, int32_t *brow, int32_t *bcol, double *vals) {
    if (!M) return -1;
    int64_t k = 0;
    extract_rec(M->root, M->depth, 0, 0, M->b, brow, bcol, vals, &k);
    return 0;
}

int64_t orc_dim(const orc_mat *M) { return M ? M->n : 0; }
int32_t orc_leafsize(const orc_mat *M) { return M ? M->b : 0; }

void orc_free(orc_mat *M) {
    if (!M) return;
    free_tree(M->root);
    free(M);
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
