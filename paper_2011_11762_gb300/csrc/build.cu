// Matrix construction (leaf list -> Morton-ordered leaf array with row and
// column indexes) and extraction to a dense buffer.
//
// Paper, Section 2: a matrix is a sparse quadtree whose nil nodes are the
// identically zero submatrices.  Flattening the quadtree keeps its stored
// leaves in depth-first (Morton) order; an all-zero input leaf is nil and is
// not stored.  Section 2.2 lists construction from index/value vectors and
// extraction of elements; here both work at leaf granularity.
#include "device.cuh"
#include "internal.h"

namespace cht {

namespace {

__global__ void k_make_keys(const int32_t *__restrict__ brow, const int32_t *__restrict__ bcol,
                            int64_t n, int64_t G, uint64_t *__restrict__ keys,
                            int32_t *__restrict__ idx, int *__restrict__ err) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t r = brow[i], c = bcol[i];
    const bool ok = r >= 0 && c >= 0 && r < G && c < G;
    if (!ok) atomicOr(err, 1);
    keys[i] = ok ? morton(static_cast<uint32_t>(r), static_cast<uint32_t>(c)) : 0;
    idx[i] = static_cast<int32_t>(i);
  }
}

// One warp per sorted leaf: duplicate check against the previous key and the
// all-zero test of the leaf's values.
__global__ void k_dup_and_zero(const uint64_t *__restrict__ skeys, const int32_t *__restrict__ sidx,
                               const double *__restrict__ vals, int64_t n, int bb,
                               int32_t *__restrict__ keep, int *__restrict__ err, bool drop_zero) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5; i < n;
       i += warps) {
    if (lane == 0 && i > 0 && skeys[i] == skeys[i - 1]) atomicOr(err, 2);
    const double *v = vals + static_cast<int64_t>(sidx[i]) * bb;
    bool nz = false;
    for (int e = lane; e < bb; e += 32) nz |= (v[e] != 0.0);
    nz = __any_sync(0xffffffffu, nz);
    if (lane == 0) keep[i] = (nz || !drop_zero) ? 1 : 0;
  }
}

__global__ void k_leaf_counts(const uint64_t *__restrict__ key, const int32_t *__restrict__ keep,
                              int64_t n, int64_t G, int32_t *__restrict__ rowcnt,
                              int32_t *__restrict__ colcnt) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (keep && !keep[i]) continue;
    const uint32_t r = morton_row(key[i]), c = morton_col(key[i]);
    if (r < G && c < G) {
      atomicAdd(&rowcnt[r], 1);
      atomicAdd(&colcnt[c], 1);
    }
  }
}

__global__ void k_compact(const uint64_t *__restrict__ skeys, const int32_t *__restrict__ sidx,
                          const int32_t *__restrict__ keep, const int64_t *__restrict__ pos,
                          const double *__restrict__ vin, int64_t n, int bb,
                          uint64_t *__restrict__ mkey, double *__restrict__ vout) {
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    if (!keep[i]) continue;
    const int64_t j = pos[i];
    if (threadIdx.x == 0) mkey[j] = skeys[i];
    const double2 *src = reinterpret_cast<const double2 *>(vin + static_cast<int64_t>(sidx[i]) * bb);
    double2 *dst = reinterpret_cast<double2 *>(vout + j * bb);
    for (int e = threadIdx.x; e < bb / 2; e += blockDim.x) dst[e] = src[e];
  }
}

__global__ void k_decode(const uint64_t *__restrict__ mkey, int64_t n,
                         int32_t *__restrict__ brow, int32_t *__restrict__ bcol) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    brow[i] = static_cast<int32_t>(morton_row(mkey[i]));
    bcol[i] = static_cast<int32_t>(morton_col(mkey[i]));
  }
}

// (row << L) | col and the leaf index, for the row-index sort.
__global__ void k_row_keys(const int32_t *__restrict__ brow, const int32_t *__restrict__ bcol,
                           int64_t n, int L, uint64_t *__restrict__ rkey,
                           int32_t *__restrict__ idx) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    rkey[i] = (static_cast<uint64_t>(brow[i]) << L) | static_cast<uint32_t>(bcol[i]);
    idx[i] = static_cast<int32_t>(i);
  }
}

__global__ void k_count(const int32_t *__restrict__ v, int64_t n, int32_t *__restrict__ cnt) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    atomicAdd(&cnt[v[i]], 1);
}

__global__ void k_split_key(const uint64_t *__restrict__ k, int64_t n, int L,
                            int32_t *__restrict__ low) {
  const uint64_t mask = (1ULL << L) - 1ULL;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    low[i] = static_cast<int32_t>(k[i] & mask);
}

// flag = 1 if any key differs (several threads may store the same 1).
__global__ void k_keys_differ(const uint64_t *__restrict__ x, const uint64_t *__restrict__ y,
                              int64_t n, int *__restrict__ flag) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    if (x[i] != y[i]) *flag = 1;
}

__global__ void k_densify(const double *__restrict__ vals, const int32_t *__restrict__ brow,
                          const int32_t *__restrict__ bcol, int64_t nnz, int b,
                          double *__restrict__ out, int64_t ld) {
  const int bb = b * b;
  for (int64_t l = blockIdx.x; l < nnz; l += gridDim.x) {
    const int64_t r0 = static_cast<int64_t>(brow[l]) * b, c0 = static_cast<int64_t>(bcol[l]) * b;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
      const int r = e / b, c = e % b;
      out[(r0 + r) * ld + c0 + c] = vals[l * bb + e];
    }
  }
}

}  // namespace

int bits_for(int64_t G) {
  int L = 1;
  while ((1LL << L) < G) ++L;
  return L;
}

int build_pattern_index(Pattern &p, cudaStream_t s) {
  const int64_t nnz = p.nnz;
  CHT_TRY(p.brow.alloc(nnz, s));
  CHT_TRY(p.bcol.alloc(nnz, s));
  if (nnz > 0) {
    k_decode<<<grid_for(nnz, 256), 256, 0, s>>>(p.mkey.p, nnz, p.brow.p, p.bcol.p);
    CHT_TRY(launched("decode"));
  }
  return CHT_OK;
}

Pattern::~Pattern() {
  if (rows_ready) cudaEventDestroy(rows_ready);
}

int ensure_row_index(const Pattern &p, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(p.rows_mutex);
  if (p.have_rows) {
    // ordered after the build, whichever stream it ran on
    CHT_CUDA_TRY(cudaStreamWaitEvent(s, p.rows_ready, 0));
    return CHT_OK;
  }
  const int64_t nnz = p.nnz;
  CHT_TRY(p.rowptr.alloc(p.G + 1, s));
  CHT_TRY(p.rowcol.alloc(nnz, s));
  CHT_TRY(p.rowleaf.alloc(nnz, s));
  DevArray<uint64_t> rkey, sk;
  DevArray<int32_t> idx, cnt;
  CHT_TRY(rkey.alloc(nnz, s));
  CHT_TRY(sk.alloc(nnz, s));
  CHT_TRY(idx.alloc(nnz, s));
  CHT_TRY(cnt.alloc(p.G, s));
  if (nnz > 0) {
    k_row_keys<<<grid_for(nnz, 256), 256, 0, s>>>(p.brow.p, p.bcol.p, nnz, p.L, rkey.p, idx.p);
    CHT_TRY(launched("row_keys"));
    // CSR by leaf row: sort by (row, col)
    CHT_TRY(radix_sort_pairs(rkey.p, idx.p, sk.p, p.rowleaf.p, nnz, 2 * p.L, s));
    k_split_key<<<grid_for(nnz, 256), 256, 0, s>>>(sk.p, nnz, p.L, p.rowcol.p);
    CHT_TRY(launched("split_key"));
  }
  CHT_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * p.G, s));
  if (nnz > 0) {
    k_count<<<grid_for(nnz, 256), 256, 0, s>>>(p.brow.p, nnz, cnt.p);
    CHT_TRY(launched("count"));
  }
  CHT_TRY(scan_exclusive(cnt.p, p.rowptr.p, p.G, s));
  if (!p.rows_ready)
    CHT_CUDA_TRY(cudaEventCreateWithFlags(&p.rows_ready, cudaEventDisableTiming));
  CHT_CUDA_TRY(cudaEventRecord(p.rows_ready, s));
  p.have_rows = true;
  return CHT_OK;
}

// Lower-triangle mirror: leaf l (I <= J) is emitted as (I, J) and, off the
// diagonal, also as (J, I) with transposed values; a diagonal leaf keeps its
// upper triangle and mirrors it into its lower one; pos[l] = output slot.
__global__ void k_mirror(const int32_t *__restrict__ brow, const int32_t *__restrict__ bcol,
                         const double *__restrict__ vals, const int64_t *__restrict__ pos,
                         int64_t n, int b, int32_t *__restrict__ orow, int32_t *__restrict__ ocol,
                         double *__restrict__ ovals) {
  const int bb = b * b;
  for (int64_t l = blockIdx.x; l < n; l += gridDim.x) {
    const int32_t I = brow[l], J = bcol[l];
    const int64_t q = pos[l];
    if (threadIdx.x == 0) {
      orow[q] = I;
      ocol[q] = J;
      if (I != J) {
        orow[q + 1] = J;
        ocol[q + 1] = I;
      }
    }
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
      const int r = e / b, c = e % b;
      if (I != J) {
        const double v = vals[l * bb + e];
        ovals[q * bb + e] = v;
        ovals[(q + 1) * bb + c * b + r] = v;
      } else {
        // diagonal leaf: its upper triangle (r <= c) is kept and mirrored
        ovals[q * bb + e] = vals[l * bb + (r <= c ? e : c * b + r)];
      }
    }
  }
}

__global__ void k_mirror_count(const int32_t *__restrict__ brow, const int32_t *__restrict__ bcol,
                               int64_t n, int32_t *__restrict__ cnt, int *__restrict__ err) {
  for (int64_t l = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; l < n;
       l += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t I = brow[l], J = bcol[l];
    if (I > J) atomicOr(err, 1);
    cnt[l] = I == J ? 1 : (I < J ? 2 : 0);
  }
}

int build_matrix(int64_t n, int32_t b, int64_t nblocks, const int32_t *d_brow,
                 const int32_t *d_bcol, const double *d_vals, cudaStream_t s, cht_mat **out,
                 bool drop_zero);

// The full symmetric matrix whose upper triangle (I <= J) U holds.
int mirror_upper(cht_mat *U, cudaStream_t s, cht_mat **out) {
  const Pattern &p = *U->pat;
  const int64_t n = p.nnz;
  DevArray<int32_t> cnt, orow, ocol;
  DevArray<int64_t> pos;
  DevArray<double> ovals;
  DevArray<int> err;
  CHT_TRY(cnt.alloc(n, s));
  CHT_TRY(pos.alloc(n + 1, s));
  CHT_TRY(err.alloc(1, s));
  CHT_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  if (n > 0) {
    k_mirror_count<<<grid_for(n, 256), 256, 0, s>>>(p.brow.p, p.bcol.p, n, cnt.p, err.p);
    CHT_TRY(launched("mirror_count"));
  }
  CHT_TRY(scan_exclusive(cnt.p, pos.p, n, s));
  int64_t total = 0;
  int herr = 0;
  CHT_CUDA_TRY(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CHT_CUDA_TRY(cudaMemcpyAsync(&total, pos.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CHT_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr) {
    set_error("mirror of an upper triangle: a leaf lies below the diagonal");
    return CHT_ERR_INVALID;
  }
  CHT_TRY(orow.alloc(total, s));
  CHT_TRY(ocol.alloc(total, s));
  CHT_TRY(ovals.alloc(static_cast<size_t>(total) * p.b * p.b, s));
  if (n > 0) {
    k_mirror<<<grid_for(n, 1), 256, 0, s>>>(p.brow.p, p.bcol.p, U->values(), pos.p, n, p.b,
                                            orow.p, ocol.p, ovals.p);
    CHT_TRY(launched("mirror"));
  }
  return build_matrix(p.n, p.b, total, orow.p, ocol.p, ovals.p, s, out, false);
}

// Builds a matrix from a device leaf list; see cht_mat_from_blocks.  With
// drop_zero false every given leaf is stored, all-zero or not.
int build_matrix(int64_t n, int32_t b, int64_t nblocks, const int32_t *d_brow,
                 const int32_t *d_bcol, const double *d_vals, cudaStream_t s, cht_mat **out,
                 bool drop_zero) {
  auto pat = std::make_shared<Pattern>();
  pat->n = n;
  pat->b = b;
  pat->G = n / b;
  pat->L = bits_for(pat->G);
  pat->id = next_id();
  const int bb = b * b;

  DevArray<uint64_t> keys, skeys;
  DevArray<int32_t> idx, sidx, keep;
  DevArray<int64_t> pos;
  DevArray<int> err;
  CHT_TRY(keys.alloc(nblocks, s));
  CHT_TRY(skeys.alloc(nblocks, s));
  CHT_TRY(idx.alloc(nblocks, s));
  CHT_TRY(sidx.alloc(nblocks, s));
  CHT_TRY(keep.alloc(nblocks, s));
  CHT_TRY(pos.alloc(nblocks + 1, s));
  CHT_TRY(err.alloc(1, s));
  CHT_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  if (nblocks > 0) {
    k_make_keys<<<grid_for(nblocks, 256), 256, 0, s>>>(d_brow, d_bcol, nblocks, pat->G, keys.p,
                                                       idx.p, err.p);
    CHT_TRY(launched("make_keys"));
    CHT_TRY(radix_sort_pairs(keys.p, idx.p, skeys.p, sidx.p, nblocks, 2 * pat->L, s));
    k_dup_and_zero<<<grid_for(nblocks * 32, 256), 256, 0, s>>>(skeys.p, sidx.p, d_vals, nblocks,
                                                               bb, keep.p, err.p, drop_zero);
    CHT_TRY(launched("dup_and_zero"));
  }
  CHT_TRY(scan_exclusive(keep.p, pos.p, nblocks, s));
  // leaf counts per row and column, read in the same synchronisation
  const int64_t G = pat->G;
  const bool counts = G <= kMaxCountG;
  DevArray<int32_t> cnts;
  if (counts) {
    CHT_TRY(cnts.alloc(2 * G, s));
    CHT_CUDA_TRY(cudaMemsetAsync(cnts.p, 0, sizeof(int32_t) * 2 * G, s));
    CHT_TRY(count_leaves(skeys.p, keep.p, nblocks, G, cnts.p, cnts.p + G, s));
    pat->rowcnt.resize(G);
    pat->colcnt.resize(G);
  }
  int herr = 0;
  int64_t nkeep = 0;
  CHT_CUDA_TRY(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CHT_CUDA_TRY(cudaMemcpyAsync(&nkeep, pos.p + nblocks, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (counts) {
    CHT_CUDA_TRY(cudaMemcpyAsync(pat->rowcnt.data(), cnts.p, sizeof(int32_t) * G,
                                 cudaMemcpyDeviceToHost, s));
    CHT_CUDA_TRY(cudaMemcpyAsync(pat->colcnt.data(), cnts.p + G, sizeof(int32_t) * G,
                                 cudaMemcpyDeviceToHost, s));
  }
  CHT_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr & 1) {
    set_error("leaf coordinate outside the %lld x %lld leaf grid", (long long)pat->G,
              (long long)pat->G);
    return CHT_ERR_INVALID;
  }
  if (herr & 2) {
    set_error("the same leaf coordinate was given twice");
    return CHT_ERR_DUPLICATE;
  }
  pat->nnz = nkeep;
  auto m = std::make_unique<cht_mat>();
  CHT_TRY(pat->mkey.alloc(nkeep, s));
  CHT_TRY(m->vals.alloc(static_cast<size_t>(nkeep) * bb, s));
  if (nblocks > 0) {
    k_compact<<<grid_for(nblocks, 1), 256, 0, s>>>(skeys.p, sidx.p, keep.p, pos.p, d_vals, nblocks,
                                                   bb, pat->mkey.p, m->vals.p);
    CHT_TRY(launched("compact"));
  }
  CHT_TRY(build_pattern_index(*pat, s));
  m->pat = std::move(pat);
  *out = m.release();
  return CHT_OK;
}

int count_leaves(const uint64_t *key, const int32_t *keep, int64_t n, int64_t G,
                 int32_t *rowcnt, int32_t *colcnt, cudaStream_t s) {
  if (n <= 0) return CHT_OK;
  k_leaf_counts<<<grid_for(n, 256), 256, 0, s>>>(key, keep, n, G, rowcnt, colcnt);
  return launched("leaf_counts");
}

int same_leaves(const Pattern &x, const Pattern &y, int *d_flag, cudaStream_t s, bool *same) {
  if (&x == &y || x.id == y.id) {
    *same = true;
    return CHT_OK;
  }
  if (x.n != y.n || x.b != y.b || x.nnz != y.nnz) {
    *same = false;
    return CHT_OK;
  }
  int h = 0;
  if (x.nnz > 0) {
    CHT_CUDA_TRY(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
    k_keys_differ<<<grid_for(x.nnz, 256), 256, 0, s>>>(x.mkey.p, y.mkey.p, x.nnz, d_flag);
    CHT_TRY(launched("keys_differ"));
    CHT_CUDA_TRY(cudaMemcpyAsync(&h, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CHT_CUDA_TRY(cudaStreamSynchronize(s));
  }
  *same = h == 0;
  return CHT_OK;
}

int densify(cht_mat *M, double *d_out, int64_t ld, cudaStream_t s) {
  const Pattern &p = *M->pat;
  CHT_CUDA_TRY(cudaMemset2DAsync(d_out, ld * sizeof(double), 0, p.n * sizeof(double), p.n, s));
  if (p.nnz > 0) {
    k_densify<<<grid_for(p.nnz, 1), 256, 0, s>>>(M->values(), p.brow.p, p.bcol.p, p.nnz, p.b,
                                                 d_out, ld);
    CHT_TRY(launched("densify"));
  }
  return CHT_OK;
}

}  // namespace cht
