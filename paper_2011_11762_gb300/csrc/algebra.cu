// Matrix addition, addition of a scaled identity, and truncation of small
// leaves (paper, Section 2.2: matrix addition including a scaled identity;
// truncation, the removal of small elements with error control).
//
// Addition works on the union of the two Morton-ordered patterns: the keys of
// both operands are concatenated (first operand first), stably radix-sorted,
// and equal neighbours merged, so every output leaf knows its source leaf in
// A and/or B.  The values pass is HBM-bound: one CTA streams a leaf at a time
// with 16-byte loads, alpha*a + beta*b with separately rounded products and
// sum (no fused multiply-add), so the result is the same bit for bit on any
// hardware that rounds to nearest.
//
// Truncation removes whole leaves (a removed leaf becomes nil):
//   Frobenius control: leaves sorted by squared norm (stable: ties keep
//   Morton order), inclusive prefix sums S_r of the sorted squared norms;
//   the removed leaves are the ranks before the first r with S_r > eps^2,
//   so the removed part has Frobenius norm sqrt(S_{m-1}) <= eps;
//   max-norm control: a leaf is removed iff its largest magnitude <= eps.
#include "device.cuh"
#include "internal.h"

namespace cht {

namespace {

constexpr int kLeafThreads = 256;

// ------------------------------------------------------------- addition --

// keys[0..nA) = A's keys, keys[nA..nA+nB) = B's keys (or the diagonal keys
// morton(j, j), j < G, for the identity); payload = position in that list.
__global__ void k_concat_keys(const uint64_t *__restrict__ ka, int64_t nA,
                              const uint64_t *__restrict__ kb, int64_t nB, int identity,
                              uint64_t *__restrict__ keys, int32_t *__restrict__ idx) {
  const int64_t n = nA + nB;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    uint64_t k;
    if (i < nA) {
      k = ka[i];
    } else {
      const int64_t j = i - nA;
      k = identity ? morton(static_cast<uint32_t>(j), static_cast<uint32_t>(j)) : kb[j];
    }
    keys[i] = k;
    idx[i] = static_cast<int32_t>(i);
  }
}

__global__ void k_heads(const uint64_t *__restrict__ skeys, int64_t n, int32_t *__restrict__ head) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    head[i] = (i == 0 || skeys[i] != skeys[i - 1]) ? 1 : 0;
}

// One output leaf per head: its key and its source leaves (-1 = absent).
// Stability puts the A entry of a shared key before the B entry.
__global__ void k_union(const uint64_t *__restrict__ skeys, const int32_t *__restrict__ sidx,
                        const int64_t *__restrict__ pos, int64_t n, int64_t nA,
                        uint64_t *__restrict__ okey, int32_t *__restrict__ ia,
                        int32_t *__restrict__ ib) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (i > 0 && skeys[i] == skeys[i - 1]) continue;
    const int64_t o = pos[i];
    okey[o] = skeys[i];
    const int32_t s0 = sidx[i];
    if (s0 < nA) {
      ia[o] = s0;
      ib[o] = (i + 1 < n && skeys[i + 1] == skeys[i]) ? static_cast<int32_t>(sidx[i + 1] - nA)
                                                      : -1;
    } else {
      ia[o] = -1;
      ib[o] = static_cast<int32_t>(s0 - nA);
    }
  }
}

// Z[o] = alpha*A[ia] + beta*B[ib] (absent side left out); with identity set,
// B[ib] is the identity leaf (1 on its diagonal).  Two elements per thread
// step (16-byte loads and stores); b*b is even for every supported b.
__global__ void __launch_bounds__(kLeafThreads)
k_add_vals(double alpha, const double *__restrict__ A, const int32_t *__restrict__ ia,
           double beta, const double *__restrict__ B, const int32_t *__restrict__ ib,
           int identity, int64_t nout, int b, double *__restrict__ Z) {
  const int bb = b * b;
  for (int64_t o = blockIdx.x; o < nout; o += gridDim.x) {
    const int32_t a = ia[o], c = ib[o];
    const double2 *pa = a >= 0 ? reinterpret_cast<const double2 *>(A + static_cast<int64_t>(a) * bb)
                               : nullptr;
    const double2 *pb = (c >= 0 && !identity)
                            ? reinterpret_cast<const double2 *>(B + static_cast<int64_t>(c) * bb)
                            : nullptr;
    double2 *pz = reinterpret_cast<double2 *>(Z + o * bb);
    for (int e2 = threadIdx.x; e2 < bb / 2; e2 += blockDim.x) {
      double y0 = 0.0, y1 = 0.0;
      if (pb) {
        const double2 t = pb[e2];
        y0 = t.x;
        y1 = t.y;
      } else if (identity && c >= 0) {
        const int e = 2 * e2;
        y0 = (e / b == e % b) ? 1.0 : 0.0;
        y1 = ((e + 1) / b == (e + 1) % b) ? 1.0 : 0.0;
      }
      double2 z;
      if (pa && c >= 0) {
        const double2 x = pa[e2];
        z.x = __dadd_rn(__dmul_rn(alpha, x.x), __dmul_rn(beta, y0));
        z.y = __dadd_rn(__dmul_rn(alpha, x.y), __dmul_rn(beta, y1));
      } else if (pa) {
        const double2 x = pa[e2];
        z.x = __dmul_rn(alpha, x.x);
        z.y = __dmul_rn(alpha, x.y);
      } else {
        z.x = __dmul_rn(beta, y0);
        z.y = __dmul_rn(beta, y1);
      }
      pz[e2] = z;
    }
  }
}

// ----------------------------------------------------------- truncation --

// One warp per leaf: the squared Frobenius norm (kind 0) or the largest
// magnitude (kind 1), in a fixed reduction order.
__global__ void k_leaf_key(const double *__restrict__ vals, int64_t n, int bb, int kind,
                           double *__restrict__ key) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t l = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5; l < n;
       l += warps) {
    const double *v = vals + l * bb;
    double s = 0.0;
    for (int e = lane; e < bb; e += 32) {
      const double x = v[e];
      s = kind == 0 ? fma(x, x, s) : fmax(s, fabs(x));
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double t = __shfl_xor_sync(0xffffffffu, s, off);
      s = kind == 0 ? s + t : fmax(s, t);
    }
    if (lane == 0) key[l] = s;
  }
}

// Non-negative doubles order like their bit patterns.
__global__ void k_key_bits(const double *__restrict__ key, int64_t n, uint64_t *__restrict__ bits,
                           int32_t *__restrict__ idx) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    bits[i] = static_cast<uint64_t>(__double_as_longlong(key[i]));
    idx[i] = static_cast<int32_t>(i);
  }
}

__global__ void k_bits_to_f64(const uint64_t *__restrict__ bits, int64_t n, double *__restrict__ v) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    v[i] = __longlong_as_double(static_cast<long long>(bits[i]));
}

// Inclusive scan of doubles: 1024-element tiles (256 threads x 4), then the
// tile sums, scanned the same way, are added back.
constexpr int kScanThreads = 256, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
k_scan_f64_tile(const double *__restrict__ in, double *__restrict__ out,
                double *__restrict__ tile_sum, int64_t n) {
  __shared__ double sh[kScanThreads];
  const int t = threadIdx.x;
  const int64_t base = blockIdx.x * static_cast<int64_t>(kScanTile) + t * kScanItems;
  double v[kScanItems];
  double run = 0.0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = base + i;
    run += j < n ? in[j] : 0.0;
    v[i] = run;
  }
  sh[t] = run;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {
    const double y = t >= off ? sh[t - off] : 0.0;
    __syncthreads();
    sh[t] += y;
    __syncthreads();
  }
  const double excl = t ? sh[t - 1] : 0.0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = base + i;
    if (j < n) out[j] = excl + v[i];
  }
  if (t == kScanThreads - 1) tile_sum[blockIdx.x] = sh[t];
}

__global__ void k_scan_f64_add(double *__restrict__ out, const double *__restrict__ tile_incl,
                               int64_t n) {
  if (blockIdx.x == 0) return;
  const double off = tile_incl[blockIdx.x - 1];
  const int64_t base = blockIdx.x * static_cast<int64_t>(kScanTile);
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
    const int64_t j = base + i;
    if (j < n) out[j] += off;
  }
}

int scan_inclusive_f64(const double *in, double *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return CHT_OK;
  const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  DevArray<double> tsum, tincl;
  CHT_TRY(tsum.alloc(ntiles, s));
  CHT_TRY(tincl.alloc(ntiles, s));
  k_scan_f64_tile<<<static_cast<unsigned>(ntiles), kScanThreads, 0, s>>>(in, out, tsum.p, n);
  CHT_TRY(launched("scan_f64_tile"));
  if (ntiles > 1) {
    CHT_TRY(scan_inclusive_f64(tsum.p, tincl.p, ntiles, s));
    k_scan_f64_add<<<static_cast<unsigned>(ntiles), kScanThreads, 0, s>>>(out, tincl.p, n);
    CHT_TRY(launched("scan_f64_add"));
  }
  return CHT_OK;
}

// First rank whose inclusive prefix exceeds eps^2 (atomic minimum).
__global__ void k_first_above(const double *__restrict__ S, int64_t n, double eps2,
                              unsigned long long *__restrict__ first) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x)
    if (!(S[r] <= eps2)) atomicMin(first, static_cast<unsigned long long>(r));
}

// keep[leaf] = rank >= m; removed = sqrt(S[m - 1]) (0 when m = 0).
__global__ void k_fro_keep(const int32_t *__restrict__ sidx, const double *__restrict__ S,
                           int64_t n, const unsigned long long *__restrict__ first,
                           int32_t *__restrict__ keep, double *__restrict__ removed) {
  const int64_t m = static_cast<int64_t>(*first);
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    keep[sidx[r]] = r >= m ? 1 : 0;
    if (r == m - 1) *removed = sqrt(S[r]);
  }
}

// Max-norm control: keep iff the largest magnitude > eps; the largest
// removed magnitude by an atomic maximum on its bit pattern.
__global__ void k_max_keep(const double *__restrict__ key, int64_t n, double eps,
                           int32_t *__restrict__ keep, unsigned long long *__restrict__ removed_bits) {
  for (int64_t l = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; l < n;
       l += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const bool k = key[l] > eps;
    keep[l] = k ? 1 : 0;
    if (!k) atomicMax(removed_bits, static_cast<unsigned long long>(__double_as_longlong(key[l])));
  }
}

__global__ void k_compact_leaves(const uint64_t *__restrict__ mkey, const double *__restrict__ vals,
                                 const int32_t *__restrict__ keep, const int64_t *__restrict__ pos,
                                 int64_t n, int bb, uint64_t *__restrict__ okey,
                                 double *__restrict__ ovals) {
  for (int64_t l = blockIdx.x; l < n; l += gridDim.x) {
    if (!keep[l]) continue;
    const int64_t o = pos[l];
    if (threadIdx.x == 0) okey[o] = mkey[l];
    const double2 *src = reinterpret_cast<const double2 *>(vals + l * bb);
    double2 *dst = reinterpret_cast<double2 *>(ovals + o * bb);
    for (int e = threadIdx.x; e < bb / 2; e += blockDim.x) dst[e] = src[e];
  }
}

unsigned leaf_grid(int64_t n) {
  int sms = 0;
  if (num_sms(&sms) != CHT_OK || sms <= 0) sms = 148;
  const int64_t g = static_cast<int64_t>(sms) * 8;
  return static_cast<unsigned>(n < g ? (n > 0 ? n : 1) : g);
}

int new_pattern_like(const Pattern &like, int64_t nnz, cudaStream_t s,
                     std::shared_ptr<Pattern> *out) {
  auto p = std::make_shared<Pattern>();
  p->n = like.n;
  p->b = like.b;
  p->G = like.G;
  p->L = like.L;
  p->nnz = nnz;
  p->id = next_id();
  CHT_TRY(p->mkey.alloc(nnz, s));
  *out = std::move(p);
  return CHT_OK;
}

}  // namespace

int add_matrices(double alpha, cht_mat *A, double beta, cht_mat *B, cudaStream_t s,
                 cht_mat **out) {
  const Pattern &pa = *A->pat;
  const bool identity = B == nullptr;
  if (!identity && (B->pat->n != pa.n || B->pat->b != pa.b)) {
    set_error("addition: operands differ in dimension or leaf size");
    return CHT_ERR_SHAPE;
  }
  const int64_t nA = pa.nnz, nB = identity ? pa.G : B->pat->nnz;
  const int64_t n = nA + nB;
  if (n >= (1LL << 31)) {
    set_error("addition: more than 2^31 - 1 leaves");
    return CHT_ERR_UNSUPPORTED;
  }
  const int bb = pa.b * pa.b;
  DevArray<uint64_t> keys, skeys;
  DevArray<int32_t> idx, sidx, head, ia, ib;
  DevArray<int64_t> pos;
  CHT_TRY(keys.alloc(n, s));
  CHT_TRY(skeys.alloc(n, s));
  CHT_TRY(idx.alloc(n, s));
  CHT_TRY(sidx.alloc(n, s));
  CHT_TRY(head.alloc(n, s));
  CHT_TRY(pos.alloc(n + 1, s));
  if (n > 0) {
    k_concat_keys<<<grid_for(n, 256), 256, 0, s>>>(pa.mkey.p, nA,
                                                   identity ? nullptr : B->pat->mkey.p, nB,
                                                   identity ? 1 : 0, keys.p, idx.p);
    CHT_TRY(launched("concat_keys"));
    CHT_TRY(radix_sort_pairs(keys.p, idx.p, skeys.p, sidx.p, n, 2 * pa.L, s));
    k_heads<<<grid_for(n, 256), 256, 0, s>>>(skeys.p, n, head.p);
    CHT_TRY(launched("heads"));
  }
  CHT_TRY(scan_exclusive(head.p, pos.p, n, s));
  int64_t nout = 0;
  CHT_TRY(read_i64(pos.p + n, &nout, s));
  std::shared_ptr<Pattern> pat;
  CHT_TRY(new_pattern_like(pa, nout, s, &pat));
  CHT_TRY(ia.alloc(nout, s));
  CHT_TRY(ib.alloc(nout, s));
  auto m = std::make_unique<cht_mat>();
  CHT_TRY(m->vals.alloc(static_cast<size_t>(nout) * bb, s));
  if (n > 0) {
    k_union<<<grid_for(n, 256), 256, 0, s>>>(skeys.p, sidx.p, pos.p, n, nA, pat->mkey.p, ia.p,
                                             ib.p);
    CHT_TRY(launched("union"));
    k_add_vals<<<leaf_grid(nout), kLeafThreads, 0, s>>>(
        alpha, A->values(), ia.p, beta, identity ? nullptr : B->values(), ib.p,
        identity ? 1 : 0, nout, pa.b, m->vals.p);
    CHT_TRY(launched("add_vals"));
  }
  CHT_TRY(build_pattern_index(*pat, s));
  m->pat = std::move(pat);
  *out = m.release();
  return CHT_OK;
}

int truncate_matrix(cht_mat *M, double eps, int kind, cudaStream_t s, cht_mat **out,
                    double *removed) {
  const Pattern &p = *M->pat;
  const int64_t n = p.nnz;
  const int bb = p.b * p.b;
  DevArray<double> key, sval, S, drem;
  DevArray<uint64_t> bits, sbits;
  DevArray<int32_t> idx, sidx, keep;
  DevArray<int64_t> pos;
  DevArray<unsigned long long> first;
  CHT_TRY(key.alloc(n, s));
  CHT_TRY(keep.alloc(n, s));
  CHT_TRY(pos.alloc(n + 1, s));
  CHT_TRY(drem.alloc(1, s));
  CHT_TRY(first.alloc(1, s));
  CHT_CUDA_TRY(cudaMemsetAsync(drem.p, 0, sizeof(double), s));
  if (n > 0) {
    k_leaf_key<<<grid_for(n * 32, 256), 256, 0, s>>>(M->values(), n, bb, kind, key.p);
    CHT_TRY(launched("leaf_key"));
    if (kind == CHT_TRUNC_FRO) {
      CHT_TRY(bits.alloc(n, s));
      CHT_TRY(sbits.alloc(n, s));
      CHT_TRY(idx.alloc(n, s));
      CHT_TRY(sidx.alloc(n, s));
      CHT_TRY(sval.alloc(n, s));
      CHT_TRY(S.alloc(n, s));
      k_key_bits<<<grid_for(n, 256), 256, 0, s>>>(key.p, n, bits.p, idx.p);
      CHT_TRY(launched("key_bits"));
      CHT_TRY(radix_sort_pairs(bits.p, idx.p, sbits.p, sidx.p, n, 64, s));
      k_bits_to_f64<<<grid_for(n, 256), 256, 0, s>>>(sbits.p, n, sval.p);
      CHT_TRY(launched("bits_to_f64"));
      CHT_TRY(scan_inclusive_f64(sval.p, S.p, n, s));
      const unsigned long long init = static_cast<unsigned long long>(n);
      CHT_CUDA_TRY(cudaMemcpyAsync(first.p, &init, sizeof(init), cudaMemcpyHostToDevice, s));
      k_first_above<<<grid_for(n, 256), 256, 0, s>>>(S.p, n, eps * eps, first.p);
      CHT_TRY(launched("first_above"));
      k_fro_keep<<<grid_for(n, 256), 256, 0, s>>>(sidx.p, S.p, n, first.p, keep.p, drem.p);
      CHT_TRY(launched("fro_keep"));
    } else {
      k_max_keep<<<grid_for(n, 256), 256, 0, s>>>(
          key.p, n, eps, keep.p, reinterpret_cast<unsigned long long *>(drem.p));
      CHT_TRY(launched("max_keep"));
    }
  }
  CHT_TRY(scan_exclusive(keep.p, pos.p, n, s));
  int64_t nkeep = 0;
  double hrem = 0.0;
  CHT_CUDA_TRY(cudaMemcpyAsync(&hrem, drem.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  CHT_TRY(read_i64(pos.p + n, &nkeep, s));
  std::shared_ptr<Pattern> pat;
  CHT_TRY(new_pattern_like(p, nkeep, s, &pat));
  auto m = std::make_unique<cht_mat>();
  CHT_TRY(m->vals.alloc(static_cast<size_t>(nkeep) * bb, s));
  if (n > 0) {
    k_compact_leaves<<<leaf_grid(n), kLeafThreads, 0, s>>>(p.mkey.p, M->values(), keep.p, pos.p,
                                                           n, bb, pat->mkey.p, m->vals.p);
    CHT_TRY(launched("compact_leaves"));
  }
  CHT_TRY(build_pattern_index(*pat, s));
  m->pat = std::move(pat);
  if (removed) *removed = hrem;
  *out = m.release();
  return CHT_OK;
}

}  // namespace cht
