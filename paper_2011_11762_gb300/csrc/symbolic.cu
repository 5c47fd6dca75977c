// Symbolic phase of C = A*B (steps S1-S5): the (A-leaf, B-leaf) pairs, the
// product's leaf pattern, each C leaf's pair segment and the work schedule.
//
// Paper, Section 2: the multiply works level by level on quadrant pairs and
// yields nil whenever an operand is nil, so only pairs of stored leaves that
// meet on an inner index K contribute, and C's stored leaves are exactly the
// (I, J) reached by such a pair.  Flattened, the recursion's leaf-level work
// is the set of triples (I, K, J) with A(I, K) and B(K, J) stored.  Sorting the
// triples by (Morton(I, J), K) groups them per C leaf in Morton order, with
// ascending K inside each group.  All of this is exact integer work.
#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "internal.h"
#include "scan.cuh"

namespace cht {

namespace {

#define GRID_STRIDE(i, n)                                                              \
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < (n); \
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)

// S1: pairs of A leaf (I, K) = stored leaves in row K of B (an element
// loader of the scan that gives each A leaf's pair offset).
struct PairCount {
  const int32_t *a_col;
  const int64_t *b_rowptr;
  __device__ int64_t operator()(int64_t a) const {
    const int32_t K = a_col[a];
    return b_rowptr[K + 1] - b_rowptr[K];
  }
};

// S3: one warp per A leaf writes its pairs: key (Morton(I, J) << L) | K.
__global__ void k_pair_fill(const int32_t *__restrict__ a_row, const int32_t *__restrict__ a_col,
                            int64_t nA, const int64_t *__restrict__ off,
                            const int64_t *__restrict__ b_rowptr,
                            const int32_t *__restrict__ b_rowcol,
                            const int32_t *__restrict__ b_rowleaf, int L, int64_t P,
                            uint64_t *__restrict__ key, int32_t *__restrict__ pa,
                            int32_t *__restrict__ pb, int32_t *__restrict__ idx) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t a = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5; a < nA;
       a += warps) {
    const uint32_t I = static_cast<uint32_t>(a_row[a]);
    const uint32_t K = static_cast<uint32_t>(a_col[a]);
    const int64_t base = off[a], cnt = off[a + 1] - off[a];
    const int64_t rs = b_rowptr[K];
    for (int64_t t = lane; t < cnt; t += 32) {
      const int64_t p = base + t;
      if (p >= P) break;  // (only if the host count were short; checked later)
      const uint32_t J = static_cast<uint32_t>(b_rowcol[rs + t]);
      key[p] = (morton(I, J) << L) | K;
      pa[p] = static_cast<int32_t>(a);
      pb[p] = b_rowleaf[rs + t];
      idx[p] = static_cast<int32_t>(p);
    }
  }
}

// S4 (after the sort): permute the pair payloads into sorted order.
__global__ void k_pair_gather(const int32_t *__restrict__ sidx, int64_t P,
                              const int32_t *__restrict__ pa_in, const int32_t *__restrict__ pb_in,
                              int32_t *__restrict__ pa, int32_t *__restrict__ pb) {
  GRID_STRIDE(i, P) {
    const int32_t s = sidx[i];
    pa[i] = pa_in[s];
    pb[i] = pb_in[s];
  }
}

// S4: a new C leaf starts where the Morton(I, J) part of the key changes.
__device__ inline bool is_head(const uint64_t *skey, int64_t i, int L) {
  return i == 0 || (skey[i] >> L) != (skey[i - 1] >> L);
}
struct HeadFlag {  // scan loader: C leaf index of every pair
  const uint64_t *skey;
  int L;
  __device__ int64_t operator()(int64_t i) const { return is_head(skey, i, L) ? 1 : 0; }
};

// S4: C leaf of every pair, and each C leaf's Morton key, coordinates and
// segment start; *d_nC = cpos[P], the number of C leaves (read from the
// device, so the host need not know it yet).
__global__ void k_segments(const uint64_t *__restrict__ skey, const int64_t *__restrict__ cpos,
                           int64_t P, int L, const int64_t *__restrict__ d_nC,
                           uint64_t *__restrict__ ckey, int32_t *__restrict__ crow,
                           int32_t *__restrict__ ccol, int64_t *__restrict__ cseg,
                           int32_t *__restrict__ pc) {
  GRID_STRIDE(i, P) {
    const bool head = is_head(skey, i, L);
    const int64_t c = cpos[i] - (head ? 0 : 1);
    pc[i] = static_cast<int32_t>(c);
    if (head) {
      const uint64_t m = skey[i] >> L;
      cseg[c] = i;
      ckey[c] = m;
      crow[c] = static_cast<int32_t>(morton_row(m));
      ccol[c] = static_cast<int32_t>(morton_col(m));
    }
    if (i == 0) cseg[*d_nC] = P;
  }
}

// S5: longest-first order key (stable sort keeps Morton order among ties):
// cap - min(len, cap), so that longer segments come first and segments of
// cap pairs or more all count as longest.
constexpr int64_t kLptCap = 0xffff;
__global__ void k_lpt_keys(const int64_t *__restrict__ seg, int64_t n, int64_t cap,
                           uint64_t *__restrict__ key, int32_t *__restrict__ idx) {
  GRID_STRIDE(u, n) {
    int64_t len = seg[u + 1] - seg[u];
    if (len > cap) len = cap;
    key[u] = static_cast<uint64_t>(cap - len);
    idx[u] = static_cast<int32_t>(u);
  }
}

// Statistics of the *d_n C leaves (count read on the device): stats[0] = the
// count, stats[1] = the longest segment, stats[2] = the C leaves of one pair,
// stats[5] = those of 2 .. kFewPairsMax pairs, stats[6] = their pairs; with
// cntB, every pair of those leaves counts on its B leaf; with rowcnt, every
// leaf counts on its leaf row and column.
__global__ void k_c_stats(const int64_t *__restrict__ seg, const uint64_t *__restrict__ ckey,
                          const int64_t *__restrict__ d_n, const int32_t *__restrict__ pb,
                          int32_t *__restrict__ cntB, int32_t *__restrict__ rowcnt,
                          int32_t *__restrict__ colcnt, unsigned long long *__restrict__ stats) {
  const int64_t n = *d_n;
  if (blockIdx.x == 0 && threadIdx.x == 0) stats[0] = static_cast<unsigned long long>(n);
  unsigned long long m = 0, ones = 0, few = 0, virt = 0;
  GRID_STRIDE(u, n) {
    const int64_t p0 = seg[u], len = seg[u + 1] - p0;
    m = max(m, static_cast<unsigned long long>(len));
    if (len <= kFewPairsMax) {
      if (len == 1) {
        ++ones;
      } else {
        ++few;
        virt += static_cast<unsigned long long>(len);
      }
      if (cntB)
        for (int64_t j = 0; j < len; ++j) atomicAdd(&cntB[pb[p0 + j]], 1);
    }
    if (rowcnt) {
      atomicAdd(&rowcnt[morton_row(ckey[u])], 1);
      atomicAdd(&colcnt[morton_col(ckey[u])], 1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    ones += __shfl_xor_sync(0xffffffffu, ones, o);
    few += __shfl_xor_sync(0xffffffffu, few, o);
    virt += __shfl_xor_sync(0xffffffffu, virt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (m) atomicMax(&stats[1], m);
    if (ones) atomicAdd(&stats[2], ones);
    if (few) atomicAdd(&stats[5], few);
    if (virt) atomicAdd(&stats[6], virt);
  }
}

// Groups of up to four units per B leaf: sum of ceil(cnt / 4).
__global__ void k_group_count(const int32_t *__restrict__ cntB, int64_t nB,
                              unsigned long long *__restrict__ out) {
  unsigned long long g = 0;
  GRID_STRIDE(k, nB) g += static_cast<unsigned long long>((cntB[k] + 3) >> 2);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
  if ((threadIdx.x & 31) == 0 && g) atomicAdd(out, g);
}

__global__ void k_iota(int32_t *__restrict__ v, int64_t n) {
  GRID_STRIDE(i, n) v[i] = static_cast<int32_t>(i);
}

// Backward regrouping keys: (unit << L) | minor, payload = pair index.
__global__ void k_regroup_keys(const int32_t *__restrict__ unit, const int32_t *__restrict__ pc,
                               const int32_t *__restrict__ c_minor, int64_t P, int L,
                               uint64_t *__restrict__ key, int32_t *__restrict__ idx) {
  GRID_STRIDE(p, P) {
    key[p] = (static_cast<uint64_t>(unit[p]) << L) | static_cast<uint32_t>(c_minor[pc[p]]);
    idx[p] = static_cast<int32_t>(p);
  }
}

__global__ void k_gather2(const int32_t *__restrict__ sidx, int64_t P,
                          const int32_t *__restrict__ u_in, const int32_t *__restrict__ v_in,
                          int32_t *__restrict__ u_out, int32_t *__restrict__ v_out) {
  GRID_STRIDE(i, P) {
    const int32_t s = sidx[i];
    u_out[i] = u_in[s];
    v_out[i] = v_in[s];
  }
}

// SpAMM filter: keep pair p iff |A leaf| * |B leaf| >= tau (Frobenius norms).
__global__ void k_spamm_keep(const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
                             int64_t P, const double *__restrict__ na,
                             const double *__restrict__ nb, double tau,
                             int32_t *__restrict__ keep) {
  GRID_STRIDE(p, P) keep[p] = (na[pa[p]] * nb[pb[p]] >= tau) ? 1 : 0;
}

__global__ void k_compact_pairs(const int32_t *__restrict__ keep, const int64_t *__restrict__ pos,
                                int64_t P, const uint64_t *__restrict__ key,
                                const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
                                uint64_t *__restrict__ ko, int32_t *__restrict__ ao,
                                int32_t *__restrict__ bo, int32_t *__restrict__ io) {
  GRID_STRIDE(p, P) {
    if (!keep[p]) continue;
    const int64_t q = pos[p];
    ko[q] = key[p];
    ao[q] = pa[p];
    bo[q] = pb[p];
    io[q] = static_cast<int32_t>(q);
  }
}

// Symmetric-square filter: keep pair p iff its C leaf (I, J) has I <= J.
__global__ void k_upper_keep(const uint64_t *__restrict__ key, int64_t P, int L,
                             int32_t *__restrict__ keep) {
  GRID_STRIDE(p, P) {
    const uint64_t m = key[p] >> L;
    keep[p] = morton_row(m) <= morton_col(m) ? 1 : 0;
  }
}

// Frobenius norm of every leaf: one warp per leaf, fixed reduction order.
__global__ void k_leaf_norms(const double *__restrict__ vals, int64_t n, int bb,
                             double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t l = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5; l < n;
       l += warps) {
    const double *v = vals + l * bb;
    double s2 = 0.0;
    for (int e = lane; e < bb; e += 32) s2 = fma(v[e], v[e], s2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) out[l] = sqrt(s2);
  }
}

__global__ void k_count_units(const int32_t *__restrict__ unit, int64_t P, int32_t *__restrict__ cnt) {
  GRID_STRIDE(p, P) atomicAdd(&cnt[unit[p]], 1);
}

// Recompute path: keep a triple only if dC stores leaf (I, J); pc = its index.
__global__ void k_lookup_dc(const uint64_t *__restrict__ key, int64_t P, int L, const int64_t *__restrict__ c_rowptr,
                            const int32_t *__restrict__ c_rowcol,
                            const int32_t *__restrict__ c_rowleaf, int32_t *__restrict__ pc,
                            int32_t *__restrict__ keep) {
  GRID_STRIDE(p, P) {
    const uint64_t m = key[p] >> L;
    const int32_t I = static_cast<int32_t>(morton_row(m)), J = static_cast<int32_t>(morton_col(m));
    int64_t lo = c_rowptr[I], hi = c_rowptr[I + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (c_rowcol[mid] < J) lo = mid + 1; else hi = mid;
    }
    const bool found = lo < c_rowptr[I + 1] && c_rowcol[lo] == J;
    pc[p] = found ? c_rowleaf[lo] : -1;
    keep[p] = found ? 1 : 0;
  }
}

__global__ void k_compact3(const int32_t *__restrict__ keep, const int64_t *__restrict__ pos,
                           int64_t P, const int32_t *__restrict__ a, const int32_t *__restrict__ b,
                           const int32_t *__restrict__ c, int32_t *__restrict__ ao,
                           int32_t *__restrict__ bo, int32_t *__restrict__ co) {
  GRID_STRIDE(p, P) {
    if (!keep[p]) continue;
    const int64_t q = pos[p];
    ao[q] = a[p];
    bo[q] = b[p];
    co[q] = c[p];
  }
}

}  // namespace

// Pairs of a product: sum over K of the A leaves in column K times the B
// leaves in row K, from the patterns' host counts; -1 when a count is missing.
static int64_t host_pair_count(const Pattern &A, const Pattern &B) {
  if (A.colcnt.empty() || B.rowcnt.empty() || A.G != B.G ||
      static_cast<int64_t>(A.colcnt.size()) != A.G || static_cast<int64_t>(B.rowcnt.size()) != B.G)
    return -1;
  int64_t P = 0;
  for (int64_t K = 0; K < A.G; ++K)
    P += static_cast<int64_t>(A.colcnt[K]) * static_cast<int64_t>(B.rowcnt[K]);
  return P;
}

// Triples (I, K, J) of stored A(I,K), B(K,J), sorted by (Morton(I,J), K):
// outputs key[P] (sorted), pa[P], pb[P].  P comes from the patterns' host
// counts (no synchronisation; the device total is copied to *d_ptotal for a
// later check) or, without them, from one synchronisation.
static int make_triples(const Pattern &A, const Pattern &B, cudaStream_t s,
                        DevArray<uint64_t> &skey, DevArray<int32_t> &pa, DevArray<int32_t> &pb,
                        int64_t *P_out, int64_t *d_ptotal, const double *normA = nullptr,
                        const double *normB = nullptr, double tau = 0.0,
                        bool upper_only = false, unsigned long long *z_scan = nullptr,
                        unsigned long long *z_sort = nullptr) {
  const int L = A.L;
  CHT_TRY(ensure_row_index(B, s));
  DevArray<int64_t> off;
  CHT_TRY(off.alloc(A.nnz + 1, s));
  CHT_TRY(scan_exclusive_fn(PairCount{A.bcol.p, B.rowptr.p}, A.nnz, off.p, s, z_scan));
  int64_t P = host_pair_count(A, B);
  if (P < 0) {
    CHT_TRY(read_i64(off.p + A.nnz, &P, s));
  } else if (d_ptotal) {
    CHT_CUDA_TRY(cudaMemcpyAsync(d_ptotal, off.p + A.nnz, sizeof(int64_t),
                                 cudaMemcpyDeviceToDevice, s));
  }
  if (P > 0x7fffffffLL) {
    set_error("%lld leaf pairs exceed the int32 pair index", (long long)P);
    return CHT_ERR_UNSUPPORTED;
  }
  DevArray<uint64_t> key;
  DevArray<int32_t> idx, sidx, pa0, pb0;
  CHT_TRY(key.alloc(P, s));
  CHT_TRY(idx.alloc(P, s));
  CHT_TRY(sidx.alloc(P, s));
  CHT_TRY(pa0.alloc(P, s));
  CHT_TRY(pb0.alloc(P, s));
  CHT_TRY(skey.alloc(P, s));
  CHT_TRY(pa.alloc(P, s));
  CHT_TRY(pb.alloc(P, s));
  if (P > 0) {
    k_pair_fill<<<grid_for(A.nnz * 32, 256), 256, 0, s>>>(A.brow.p, A.bcol.p, A.nnz, off.p,
                                                          B.rowptr.p, B.rowcol.p, B.rowleaf.p, L,
                                                          P, key.p, pa0.p, pb0.p, idx.p);
    CHT_TRY(launched("pair_fill"));
  }
  if (P > 0 && (normA || upper_only)) {
    // sparse approximate product: drop the pairs below the norm threshold;
    // symmetric square: drop the pairs of C leaves below the diagonal
    DevArray<int32_t> keep;
    DevArray<int64_t> pos;
    CHT_TRY(keep.alloc(P, s));
    CHT_TRY(pos.alloc(P + 1, s));
    if (normA) {
      k_spamm_keep<<<grid_for(P, 256), 256, 0, s>>>(pa0.p, pb0.p, P, normA, normB, tau, keep.p);
      CHT_TRY(launched("spamm_keep"));
    } else {
      k_upper_keep<<<grid_for(P, 256), 256, 0, s>>>(key.p, P, L, keep.p);
      CHT_TRY(launched("upper_keep"));
    }
    CHT_TRY(scan_exclusive(keep.p, pos.p, P, s));
    int64_t Pk = 0;
    CHT_TRY(read_i64(pos.p + P, &Pk, s));
    DevArray<uint64_t> key2;
    DevArray<int32_t> pa2, pb2, idx2;
    CHT_TRY(key2.alloc(Pk, s));
    CHT_TRY(pa2.alloc(Pk, s));
    CHT_TRY(pb2.alloc(Pk, s));
    CHT_TRY(idx2.alloc(Pk, s));
    k_compact_pairs<<<grid_for(P, 256), 256, 0, s>>>(keep.p, pos.p, P, key.p, pa0.p, pb0.p,
                                                     key2.p, pa2.p, pb2.p, idx2.p);
    CHT_TRY(launched("compact_pairs"));
    key = std::move(key2);
    pa0 = std::move(pa2);
    pb0 = std::move(pb2);
    idx = std::move(idx2);
    P = Pk;
  }
  if (P > 0) {
    // the fill wrote the pairs in A's (Morton) leaf order, so for one (I, J)
    // in ascending K: a stable sort on the Morton(I, J) bits alone keeps K
    // ascending inside every C leaf
    CHT_TRY(radix_sort_pairs(key.p, idx.p, skey.p, sidx.p, P, 2 * L, s, L,
                             (normA || upper_only) ? nullptr : z_sort));
    k_pair_gather<<<grid_for(P, 256), 256, 0, s>>>(sidx.p, P, pa0.p, pb0.p, pa.p, pb.p);
    CHT_TRY(launched("pair_gather"));
  }
  *P_out = P;
  return CHT_OK;
}

// Longest-first order of n units with segments seg; max_len: the longest
// segment when known (the sort then reads only the bits it needs), else 0.
int schedule_units(const int64_t *seg, int64_t n, int32_t *order, cudaStream_t s,
                   int64_t max_len = 0, unsigned long long *zeroed = nullptr) {
  if (n <= 0) return CHT_OK;
  const int64_t cap = max_len > 0 ? std::min(max_len, kLptCap) : kLptCap;
  if (g_opt.schedule == 1 || (max_len == 1)) {
    // Morton order, or every segment has one pair: the identity
    k_iota<<<grid_for(n, 256), 256, 0, s>>>(order, n);
    return launched("iota");
  }
  DevArray<uint64_t> key, skey;
  DevArray<int32_t> idx;
  CHT_TRY(key.alloc(n, s));
  CHT_TRY(skey.alloc(n, s));
  CHT_TRY(idx.alloc(n, s));
  k_lpt_keys<<<grid_for(n, 256), 256, 0, s>>>(seg, n, cap, key.p, idx.p);
  CHT_TRY(launched("lpt_keys"));
  return radix_sort_pairs(key.p, idx.p, skey.p, order, n, bits_for(cap + 1), s, 0, zeroed);
}

int leaf_norms(const double *vals, int64_t n, int b, double *out, cudaStream_t s) {
  if (n <= 0) return CHT_OK;
  k_leaf_norms<<<grid_for(n * 32, 256), 256, 0, s>>>(vals, n, b * b, out);
  return launched("leaf_norms");
}

int symbolic(const Pattern &A, const Pattern &B, cudaStream_t s, cht_plan **out,
             const double *normA, const double *normB, double tau, bool upper_only) {
  const int L = A.L;
  if (3 * L > 63) {
    set_error("leaf grid of %lld per side is too large for 64-bit pair keys", (long long)A.G);
    return CHT_ERR_UNSUPPORTED;
  }
  auto plan = std::make_unique<cht_plan>();
  plan->id = next_id();
  plan->n = A.n;
  plan->b = A.b;
  plan->nA = A.nnz;
  plan->nB = B.nnz;
  plan->patA = A.id;
  plan->patB = B.id;

  // statistics read in the phase's one synchronisation: [0] C leaves, [1]
  // longest segment, [2] one-pair C leaves, [3] the groups of the split
  // form's units (32-leaves), [4] the device's pair total (checked against
  // the host's count), [5] C leaves of 2 .. kFewPairsMax pairs, [6] their
  // pairs
  // One zeroed device block holds them, then C's leaf counts per row and
  // column (2 G int32, when kept), then the units per B leaf (32-leaves): one
  // memset, and one copy to pinned host memory at the synchronisation.
  constexpr int kStats = 7;
  const bool groups = A.b == 32 && B.nnz > 0;
  const int64_t G = A.G;
  const bool counts = G <= kMaxCountG;
  // When the pair count is known now (host leaf counts, no pair filter) the
  // same block also holds the zeroed state of the phase's two scans and two
  // sorts, so that one memset serves the whole phase.
  const int64_t n_rc = counts ? 2 * G : 0, n_b = groups ? B.nnz : 0;
  const int64_t P_known = host_pair_count(A, B);
  const bool pre = P_known >= 0 && !normA && !upper_only;
  const int64_t w_scan1 = pre ? scan_state_words(A.nnz) : 0;
  const int64_t w_sort = pre ? sort_state_words(P_known, 2 * L, L) : 0;
  const int64_t w_scan2 = pre ? scan_state_words(P_known) : 0;
  const int64_t w_lpt = pre ? sort_state_words(P_known, 16) : 0;
  const int64_t w_counts = (n_rc + n_b + 1) / 2;  // int64 words
  const int64_t words = kStats + w_counts + w_scan1 + w_sort + w_scan2 + w_lpt;
  DevArray<int64_t> stats;
  CHT_TRY(stats.alloc(words, s));
  CHT_CUDA_TRY(cudaMemsetAsync(stats.p, 0, sizeof(int64_t) * words, s));
  int32_t *rc = counts ? reinterpret_cast<int32_t *>(stats.p + kStats) : nullptr;
  int32_t *cntB = groups ? reinterpret_cast<int32_t *>(stats.p + kStats) + n_rc : nullptr;
  auto *zw = reinterpret_cast<unsigned long long *>(stats.p + kStats + w_counts);
  unsigned long long *z_scan1 = pre ? zw : nullptr;
  unsigned long long *z_sort = pre ? zw + w_scan1 : nullptr;
  unsigned long long *z_scan2 = pre ? zw + w_scan1 + w_sort : nullptr;
  unsigned long long *z_lpt = pre ? zw + w_scan1 + w_sort + w_scan2 : nullptr;
  DevArray<uint64_t> skey;
  DevArray<int32_t> pa, pb;
  int64_t P = 0;
  CHT_TRY(make_triples(A, B, s, skey, pa, pb, &P, stats.p + 4, normA, normB, tau, upper_only,
                       z_scan1, z_sort));
  const int64_t P_made = host_pair_count(A, B);  // the count the pair list was sized with
  plan->npairs = P;

  DevArray<int64_t> cpos;
  CHT_TRY(cpos.alloc(P + 1, s));
  CHT_TRY(scan_exclusive_fn(HeadFlag{skey.p, L}, P, cpos.p, s, pre && P == P_known ? z_scan2 : nullptr));
  // C leaves <= P: the C pattern's keys, coordinates and segments are
  // written at that capacity (and kept at it)
  auto C = std::make_shared<Pattern>();
  const int64_t *d_nC = cpos.p + P;
  CHT_TRY(C->mkey.alloc(P, s));
  CHT_TRY(C->brow.alloc(P, s));
  CHT_TRY(C->bcol.alloc(P, s));
  CHT_TRY(plan->cseg.alloc(P + 1, s));
  CHT_TRY(plan->pc.alloc(P, s));
  // (per-B-leaf counts of the split form's units -- 32-leaves: the pairs of
  // C leaves with at most kFewPairsMax pairs -- and the C pattern's leaf
  // counts per row and column live in the statistics block)
  auto *st = reinterpret_cast<unsigned long long *>(stats.p);
  if (P > 0) {
    k_segments<<<grid_for(P, 256), 256, 0, s>>>(skey.p, cpos.p, P, L, d_nC, C->mkey.p,
                                                C->brow.p, C->bcol.p, plan->cseg.p, plan->pc.p);
    CHT_TRY(launched("segments"));
    k_c_stats<<<grid_for(P, 256), 256, 0, s>>>(plan->cseg.p, C->mkey.p, d_nC, pb.p,
                                                cntB, rc, counts ? rc + G : nullptr, st);
    CHT_TRY(launched("c_stats"));
    if (groups) {
      k_group_count<<<grid_for(B.nnz, 256), 256, 0, s>>>(cntB, B.nnz, st + 3);
      CHT_TRY(launched("group_count"));
    }
  } else {
    CHT_CUDA_TRY(cudaMemsetAsync(plan->cseg.p, 0, sizeof(int64_t), s));
  }
  // the statistics and C's counts (not the units per B leaf, which stay on
  // the device) in one copy
  const size_t read_bytes = sizeof(int64_t) * kStats + sizeof(int32_t) * n_rc;
  void *host = nullptr;
  CHT_TRY(pinned_scratch(read_bytes, &host));
  CHT_CUDA_TRY(cudaMemcpyAsync(host, stats.p, read_bytes, cudaMemcpyDeviceToHost, s));
  CHT_CUDA_TRY(cudaStreamSynchronize(s));
  int64_t host_stats[kStats];
  std::memcpy(host_stats, host, sizeof(host_stats));
  if (counts) {
    const int32_t *hc = reinterpret_cast<const int32_t *>(static_cast<const int64_t *>(host) + kStats);
    C->rowcnt.assign(hc, hc + G);
    C->colcnt.assign(hc + G, hc + 2 * G);
  }
  if (P_made >= 0 && host_stats[4] != P_made) {
    set_error("pair count %lld from the leaf counts, %lld on the device", (long long)P_made,
              (long long)host_stats[4]);
    return CHT_ERR_INVALID;
  }
  const int64_t nC = host_stats[0];
  plan->max_seg = host_stats[1];
  if (groups) {
    plan->n_one = host_stats[2];
    plan->n_groups = host_stats[3];
    plan->n_few = host_stats[5];
    plan->n_virt = host_stats[6];
    // the units per B leaf stay where they are: the plan keeps the block
    plan->one_pair_b = cntB;
    plan->sym_block = std::move(stats);
  }

  C->n = A.n;
  C->b = A.b;
  C->G = A.G;
  C->L = L;
  C->nnz = nC;
  C->id = next_id();
  CHT_TRY(plan->order.alloc(nC, s));
  CHT_TRY(schedule_units(plan->cseg.p, nC, plan->order.p, s, plan->max_seg,
                         pre && nC <= P_known ? z_lpt : nullptr));
  plan->pa = std::move(pa);
  plan->pb = std::move(pb);
  plan->C = std::move(C);
  *out = plan.release();
  return CHT_OK;
}

// Regroups triples (pa, pb, pc over C pattern `Cp`) by A leaf (ordered by J)
// and by B leaf (ordered by I) for the two sampled backward products.
static int regroup(const Pattern &A, const Pattern &B, const Pattern &Cp, const int32_t *pa,
                   const int32_t *pb, const int32_t *pc, int64_t P, cudaStream_t s,
                   cht_plan &out) {
  const int L = A.L;
  CHT_TRY(out.segA.alloc(A.nnz + 1, s));
  CHT_TRY(out.segB.alloc(B.nnz + 1, s));
  CHT_TRY(out.dA_c.alloc(P, s));
  CHT_TRY(out.dA_b.alloc(P, s));
  CHT_TRY(out.dB_a.alloc(P, s));
  CHT_TRY(out.dB_c.alloc(P, s));
  CHT_TRY(out.idA.alloc(A.nnz, s));
  CHT_TRY(out.idB.alloc(B.nnz, s));
  DevArray<uint64_t> key, skey;
  DevArray<int32_t> idx, sidx, cnt;
  CHT_TRY(key.alloc(P, s));
  CHT_TRY(skey.alloc(P, s));
  CHT_TRY(idx.alloc(P, s));
  CHT_TRY(sidx.alloc(P, s));
  const int ubitsA = bits_for(A.nnz + 1), ubitsB = bits_for(B.nnz + 1);
  // dA: units = A leaves, minor = J (C leaf column)
  CHT_TRY(cnt.alloc(A.nnz, s));
  CHT_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * cnt.n, s));
  if (P > 0) {
    k_regroup_keys<<<grid_for(P, 256), 256, 0, s>>>(pa, pc, Cp.bcol.p, P, L, key.p, idx.p);
    CHT_TRY(launched("regroup_keys"));
    CHT_TRY(radix_sort_pairs(key.p, idx.p, skey.p, sidx.p, P, ubitsA + L, s));
    k_gather2<<<grid_for(P, 256), 256, 0, s>>>(sidx.p, P, pc, pb, out.dA_c.p, out.dA_b.p);
    CHT_TRY(launched("gather2"));
    k_count_units<<<grid_for(P, 256), 256, 0, s>>>(pa, P, cnt.p);
    CHT_TRY(launched("count_units"));
  }
  CHT_TRY(scan_exclusive(cnt.p, out.segA.p, A.nnz, s));
  // dB: units = B leaves, minor = I (C leaf row)
  CHT_TRY(cnt.alloc(B.nnz, s));
  CHT_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * cnt.n, s));
  if (P > 0) {
    k_regroup_keys<<<grid_for(P, 256), 256, 0, s>>>(pb, pc, Cp.brow.p, P, L, key.p, idx.p);
    CHT_TRY(launched("regroup_keys"));
    CHT_TRY(radix_sort_pairs(key.p, idx.p, skey.p, sidx.p, P, ubitsB + L, s));
    k_gather2<<<grid_for(P, 256), 256, 0, s>>>(sidx.p, P, pa, pc, out.dB_a.p, out.dB_c.p);
    CHT_TRY(launched("gather2"));
    k_count_units<<<grid_for(P, 256), 256, 0, s>>>(pb, P, cnt.p);
    CHT_TRY(launched("count_units"));
  }
  CHT_TRY(scan_exclusive(cnt.p, out.segB.p, B.nnz, s));
  CHT_TRY(schedule_units(out.segA.p, A.nnz, out.idA.p, s));
  CHT_TRY(schedule_units(out.segB.p, B.nnz, out.idB.p, s));
  out.have_bwd = true;
  return CHT_OK;
}

int backward_lists_from_plan(cht_plan &plan, const Pattern &A, const Pattern &B,
                             cudaStream_t s) {
  if (plan.have_bwd) return CHT_OK;
  return regroup(A, B, *plan.C, plan.pa.p, plan.pb.p, plan.pc.p, plan.npairs, s, plan);
}

// Triples restricted to dC's stored leaves, regrouped for the backward.
int backward_lists_recompute(const Pattern &A, const Pattern &B, const Pattern &dC,
                             cudaStream_t s, cht_plan &out) {
  DevArray<uint64_t> skey;
  DevArray<int32_t> pa, pb;
  int64_t P = 0;
  CHT_TRY(make_triples(A, B, s, skey, pa, pb, &P, nullptr));
  CHT_TRY(ensure_row_index(dC, s));
  DevArray<int32_t> pc, keep, ka, kb, kc;
  DevArray<int64_t> pos;
  CHT_TRY(pc.alloc(P, s));
  CHT_TRY(keep.alloc(P, s));
  CHT_TRY(pos.alloc(P + 1, s));
  if (P > 0) {
    k_lookup_dc<<<grid_for(P, 256), 256, 0, s>>>(skey.p, P, A.L, dC.rowptr.p,
                                                 dC.rowcol.p, dC.rowleaf.p, pc.p, keep.p);
    CHT_TRY(launched("lookup_dc"));
  }
  CHT_TRY(scan_exclusive(keep.p, pos.p, P, s));
  int64_t Pk = 0;
  CHT_TRY(read_i64(pos.p + P, &Pk, s));
  CHT_TRY(ka.alloc(Pk, s));
  CHT_TRY(kb.alloc(Pk, s));
  CHT_TRY(kc.alloc(Pk, s));
  if (P > 0) {
    k_compact3<<<grid_for(P, 256), 256, 0, s>>>(keep.p, pos.p, P, pa.p, pb.p, pc.p, ka.p, kb.p,
                                                kc.p);
    CHT_TRY(launched("compact3"));
  }
  out.npairs = Pk;
  return regroup(A, B, dC, ka.p, kb.p, kc.p, Pk, s, out);
}

}  // namespace cht
