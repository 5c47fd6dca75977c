// The C ABI of libcht (declared in include/cht.h): argument checks, handle
// management, allocation and the device status word.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "internal.h"

namespace cht {

// Implemented in the other translation units.
int build_matrix(int64_t n, int32_t b, int64_t nblocks, const int32_t *d_brow,
                 const int32_t *d_bcol, const double *d_vals, cudaStream_t s, cht_mat **out,
                 bool drop_zero);
int mirror_upper(cht_mat *U, cudaStream_t s, cht_mat **out);
int add_matrices(double alpha, cht_mat *A, double beta, cht_mat *B, cudaStream_t s,
                 cht_mat **out);
int truncate_matrix(cht_mat *M, double eps, int kind, cudaStream_t s, cht_mat **out,
                    double *removed);
int densify(cht_mat *M, double *d_out, int64_t ld, cudaStream_t s);
int symbolic(const Pattern &A, const Pattern &B, cudaStream_t s, cht_plan **out,
             const double *normA = nullptr, const double *normB = nullptr, double tau = 0.0,
             bool upper_only = false);
int leaf_norms(const double *vals, int64_t n, int b, double *out, cudaStream_t s);
int backward_lists_from_plan(cht_plan &plan, const Pattern &A, const Pattern &B, cudaStream_t s);
int backward_lists_recompute(const Pattern &A, const Pattern &B, const Pattern &dC,
                             cudaStream_t s, cht_plan &out);
int split_multiply(cht_plan *plan, cht_mat *A, cht_mat *B, int nslices, cudaStream_t s,
                   double *Cvals, double *err_bound);
int batch_create(int32_t count, const cht_plan_t *plans, const cht_mat_t *As,
                 const cht_mat_t *Bs, int mode, int32_t nslices, cudaStream_t s,
                 cht_batch **out);
int batch_run(cht_batch *b, cudaStream_t s);
int batch_output(cht_batch *b, int32_t i, cht_mat **C);
void batch_destroy(cht_batch *b);

Options g_opt;
std::atomic<int64_t> g_launches{0};

namespace {
thread_local char g_last_error[512] = "";
std::atomic<uint64_t> g_next_id{1};
cht_alloc_fn g_alloc = nullptr;
cht_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;
std::mutex g_dev_mutex;
constexpr int kMaxDevices = 64;
int *g_status_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

__device__ int g_status_word;  // the library-wide device status word

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

int current_device(int *dev) {
  CHT_CUDA_TRY(cudaGetDevice(dev));
  if (*dev < 0 || *dev >= kMaxDevices) {
    set_error("device ordinal %d out of range", *dev);
    return CHT_ERR_UNSUPPORTED;
  }
  return CHT_OK;
}
}  // namespace

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what) {
  set_error("CUDA error %s (%s) in %s", cudaGetErrorName(e), cudaGetErrorString(e), what);
  return CHT_ERR_CUDA;
}

int launched(const char *name) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, name);
  return CHT_OK;
}

uint64_t next_id() { return g_next_id.fetch_add(1); }

// Keeps freed blocks in the device's default stream-ordered pool instead of
// returning them to the driver at every synchronisation (this process only).
static void keep_pool_memory() {
  static bool done[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ULL;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done[dev] = true;
}

// Small blocks are cached per (stream, size class) and handed out again on
// the same stream: stream order makes the reuse safe (a block freed after
// work W on stream s is reused only by work queued on s after W), and the
// symbolic phase's dozens of short-lived arrays then cost no allocator call.
// Larger blocks, blocks beyond the cache's cap and any cached block after an
// allocation failure go back to the stream-ordered pool.  The cache keys on
// the stream handle: a caller that destroys a stream while the library's
// work on it is still running, and then gets the same handle for a new
// stream, should synchronise the old one first (as for any stream-ordered
// free).
namespace {
constexpr size_t kCacheMaxBlock = size_t(64) << 20;   // larger: not cached
constexpr size_t kCacheMaxTotal = size_t(1) << 30;    // cached bytes per process
std::mutex g_cache_mutex;
std::map<std::pair<cudaStream_t, size_t>, std::vector<void *>> g_cache;
size_t g_cached_bytes = 0;

size_t size_class(size_t bytes) {
  size_t c = 256;
  while (c < bytes) c <<= 1;
  return c;
}

// Returns every cached block to the pool (after an allocation failure).
void flush_cache() {
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  for (auto &kv : g_cache)
    for (void *p : kv.second) cudaFreeAsync(p, kv.first.first);
  g_cache.clear();
  g_cached_bytes = 0;
  cudaGetLastError();
}
}  // namespace

void *dev_alloc(size_t bytes, cudaStream_t s) {
  if (g_alloc) return g_alloc(bytes, s, g_alloc_ctx);
  const bool cached = bytes <= kCacheMaxBlock;
  const size_t cls = cached ? size_class(bytes) : bytes;
  if (cached) {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    auto it = g_cache.find({s, cls});
    if (it != g_cache.end() && !it->second.empty()) {
      void *p = it->second.back();
      it->second.pop_back();
      g_cached_bytes -= cls;
      return p;
    }
  }
  keep_pool_memory();
  void *p = nullptr;
  if (cudaMallocAsync(&p, cls, s) != cudaSuccess) {
    cudaGetLastError();
    flush_cache();
    if (cudaMallocAsync(&p, cls, s) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (g_free) {
    g_free(p, bytes, s, g_alloc_ctx);
    return;
  }
  if (bytes <= kCacheMaxBlock) {
    const size_t cls = size_class(bytes);
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    if (g_cached_bytes + cls <= kCacheMaxTotal) {
      g_cache[{s, cls}].push_back(p);
      g_cached_bytes += cls;
      return;
    }
  }
  cudaFreeAsync(p, s);
}

int device_status_ptr(int **ptr) {
  int dev = 0;
  CHT_TRY(current_device(&dev));
  std::lock_guard<std::mutex> lock(g_dev_mutex);
  if (!g_status_ptr[dev]) {
    void *p = nullptr;
    CHT_CUDA_TRY(cudaGetSymbolAddress(&p, g_status_word));
    g_status_ptr[dev] = static_cast<int *>(p);
  }
  *ptr = g_status_ptr[dev];
  return CHT_OK;
}

int side_stream(SideStream **out) {
  static thread_local SideStream side[kMaxDevices];
  int dev = 0;
  CHT_TRY(current_device(&dev));
  SideStream &ss = side[dev];
  if (!ss.s) {
    CHT_CUDA_TRY(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
    CHT_CUDA_TRY(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming));
    CHT_CUDA_TRY(cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming));
  }
  *out = &ss;
  return CHT_OK;
}

int pinned_scratch(size_t bytes, void **out) {
  struct Buf {
    void *p = nullptr;
    size_t n = 0;
  };
  static thread_local Buf buf;
  if (buf.n < bytes) {
    if (buf.p) cudaFreeHost(buf.p);
    buf.p = nullptr;
    buf.n = 0;
    size_t n = 4096;
    while (n < bytes) n <<= 1;
    CHT_CUDA_TRY(cudaHostAlloc(&buf.p, n, cudaHostAllocPortable));
    buf.n = n;
  }
  *out = buf.p;
  return CHT_OK;
}

int num_sms(int *sms) {
  int dev = 0;
  CHT_TRY(current_device(&dev));
  if (!g_sms[dev]) {
    int v = 0;
    CHT_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    g_sms[dev] = v;
  }
  *sms = g_sms[dev];
  return CHT_OK;
}

int check_plan_operands(const cht_plan *plan, const cht_mat *A, const cht_mat *B, int *d_flag,
                        cudaStream_t s) {
  if (!plan || !A || !B) {
    set_error("null plan or matrix handle");
    return CHT_ERR_INVALID;
  }
  if (A->pat->n != plan->n || B->pat->n != plan->n || A->pat->b != plan->b ||
      B->pat->b != plan->b || A->pat->nnz != plan->nA || B->pat->nnz != plan->nB) {
    set_error("matrices do not match the plan's operands (n, b or leaf count)");
    return CHT_ERR_SHAPE;
  }
  const bool fastA = A->pat->id == plan->patA, fastB = B->pat->id == plan->patB;
  if (fastA && fastB) return CHT_OK;
  DevArray<int> flag;
  if (!d_flag) {
    CHT_TRY(flag.alloc(1, s));
    d_flag = flag.p;
  }
  bool same = true;
  if (!fastA) {
    if (!plan->opA) same = false;
    else CHT_TRY(same_leaves(*A->pat, *plan->opA, d_flag, s, &same));
    if (!same) {
      set_error("A does not store the leaves of the plan's left operand");
      return CHT_ERR_SHAPE;
    }
  }
  if (!fastB) {
    if (!plan->opB) same = false;
    else CHT_TRY(same_leaves(*B->pat, *plan->opB, d_flag, s, &same));
    if (!same) {
      set_error("B does not store the leaves of the plan's right operand");
      return CHT_ERR_SHAPE;
    }
  }
  return CHT_OK;
}

}  // namespace cht

using namespace cht;

namespace {

bool leaf_ok(int32_t b) { return b >= CHT_MIN_LEAF && b <= CHT_MAX_LEAF && b % 8 == 0; }

int check_pair(cht_mat *A, cht_mat *B) {
  if (!A || !B) {
    set_error("null matrix handle");
    return CHT_ERR_INVALID;
  }
  if (A->pat->n != B->pat->n || A->pat->b != B->pat->b) {
    set_error("shape mismatch: n %lld vs %lld, b %d vs %d", (long long)A->pat->n,
              (long long)B->pat->n, A->pat->b, B->pat->b);
    return CHT_ERR_SHAPE;
  }
  return CHT_OK;
}

// Records the operand patterns in a new plan (see check_plan_operands).
int finish_plan(cht_plan *p, cht_mat *A, cht_mat *B, int64_t *nnzb_C, int64_t *npairs,
                cht_plan_t *out) {
  p->opA = A->pat;
  p->opB = B->pat;
  if (nnzb_C) *nnzb_C = p->C->nnz;
  if (npairs) *npairs = p->npairs;
  *out = p;
  return CHT_OK;
}

// A matrix on the given pattern with uninitialised values.
int new_on_pattern(const std::shared_ptr<Pattern> &pat, uint64_t plan_id, cudaStream_t s,
                   cht_mat **out) {
  auto m = std::make_unique<cht_mat>();
  m->pat = pat;
  m->plan_id = plan_id;
  CHT_TRY(m->vals.alloc(static_cast<size_t>(pat->nnz) * pat->b * pat->b, s));
  *out = m.release();
  return CHT_OK;
}

// Resolves an in/out matrix argument: reuse *io if it has pattern `pat`,
// else create a new one (stored to *io only on success by the caller).
int out_matrix(cht_mat_t *io, const std::shared_ptr<Pattern> &pat, uint64_t plan_id,
               cudaStream_t s, cht_mat **m, bool *created) {
  *created = false;
  if (*io) {
    if ((*io)->pat->id != pat->id) {
      set_error("output matrix does not have the expected pattern");
      return CHT_ERR_INVALID;
    }
    *m = *io;
    return CHT_OK;
  }
  CHT_TRY(new_on_pattern(pat, plan_id, s, m));
  *created = true;
  return CHT_OK;
}

}  // namespace

extern "C" {

int cht_set_allocator(cht_alloc_fn alloc, cht_free_fn free_fn, void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) {
    set_error("allocator and free function must be given together");
    return CHT_ERR_INVALID;
  }
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return CHT_OK;
}

int cht_mat_from_blocks(int64_t n, int32_t b, int64_t nblocks, const int32_t *d_brow,
                        const int32_t *d_bcol, const double *d_vals, void *stream,
                        cht_mat_t *out) {
  if (!out || n <= 0 || !leaf_ok(b) || n % b != 0 || nblocks < 0 || nblocks > 0x7fffffffLL) {
    set_error("invalid shape: n=%lld b=%d nblocks=%lld (need n %% b == 0, %d <= b <= %d, b %% 8 == 0)",
              (long long)n, b, (long long)nblocks, CHT_MIN_LEAF, CHT_MAX_LEAF);
    return CHT_ERR_INVALID;
  }
  if (nblocks > 0 && (!d_brow || !d_bcol || !d_vals)) {
    set_error("null input array");
    return CHT_ERR_INVALID;
  }
  if (reinterpret_cast<uintptr_t>(d_vals) % 16 != 0) {
    set_error("d_vals must be 16-byte aligned");
    return CHT_ERR_INVALID;
  }
  if (bits_for(n / b) > 21) {
    set_error("leaf grid too large (at most 2^21 leaves per side)");
    return CHT_ERR_UNSUPPORTED;
  }
  cht_mat *m = nullptr;
  CHT_TRY(build_matrix(n, b, nblocks, d_brow, d_bcol, d_vals, as_stream(stream), &m, true));
  *out = m;
  return CHT_OK;
}

int cht_mat_info(cht_mat_t M, int64_t *n, int32_t *b, int64_t *nblocks) {
  if (!M) {
    set_error("null matrix handle");
    return CHT_ERR_INVALID;
  }
  if (n) *n = M->pat->n;
  if (b) *b = M->pat->b;
  if (nblocks) *nblocks = M->pat->nnz;
  return CHT_OK;
}

int cht_mat_leaves(cht_mat_t M, double **d_vals, const int32_t **d_brow, const int32_t **d_bcol) {
  if (!M) {
    set_error("null matrix handle");
    return CHT_ERR_INVALID;
  }
  if (d_vals) *d_vals = M->values();
  if (d_brow) *d_brow = M->pat->brow.p;
  if (d_bcol) *d_bcol = M->pat->bcol.p;
  return CHT_OK;
}

int cht_to_dense(cht_mat_t M, double *d_out, int64_t ld, void *stream) {
  if (!M || !d_out || ld < M->pat->n) {
    set_error("invalid dense output (null or ld < n)");
    return CHT_ERR_INVALID;
  }
  return densify(M, d_out, ld, as_stream(stream));
}

int cht_mat_like(cht_mat_t M, void *stream, cht_mat_t *out) {
  if (!M || !out) {
    set_error("null matrix handle or out-pointer");
    return CHT_ERR_INVALID;
  }
  cht_mat *m = nullptr;
  CHT_TRY(new_on_pattern(M->pat, M->plan_id, as_stream(stream), &m));
  *out = m;
  return CHT_OK;
}

int cht_mat_free(cht_mat_t M) {
  if (M && M->view) {
    set_error("batched outputs are views owned by their batch");
    return CHT_ERR_INVALID;
  }
  delete M;
  return CHT_OK;
}

int cht_symbolic_multiply(cht_mat_t A, cht_mat_t B, void *stream, cht_plan_t *out,
                          int64_t *nnzb_C, int64_t *npairs) {
  if (!out) {
    set_error("null plan out-pointer");
    return CHT_ERR_INVALID;
  }
  CHT_TRY(check_pair(A, B));
  cht_plan *p = nullptr;
  CHT_TRY(symbolic(*A->pat, *B->pat, as_stream(stream), &p));
  return finish_plan(p, A, B, nnzb_C, npairs, out);
}

int cht_symbolic_multiply_spamm(cht_mat_t A, cht_mat_t B, double tau, void *stream,
                                cht_plan_t *out, int64_t *nnzb_C, int64_t *npairs) {
  if (!out || !(tau >= 0.0)) {
    set_error("null plan out-pointer or invalid threshold");
    return CHT_ERR_INVALID;
  }
  CHT_TRY(check_pair(A, B));
  cudaStream_t s = as_stream(stream);
  DevArray<double> na, nb;
  CHT_TRY(na.alloc(A->pat->nnz, s));
  CHT_TRY(nb.alloc(B->pat->nnz, s));
  CHT_TRY(leaf_norms(A->values(), A->pat->nnz, A->pat->b, na.p, s));
  CHT_TRY(leaf_norms(B->values(), B->pat->nnz, B->pat->b, nb.p, s));
  cht_plan *p = nullptr;
  CHT_TRY(symbolic(*A->pat, *B->pat, s, &p, na.p, nb.p, tau));
  return finish_plan(p, A, B, nnzb_C, npairs, out);
}

int cht_symbolic_multiply_symsquare(cht_mat_t A, void *stream, cht_plan_t *out,
                                    int64_t *nnzb_C, int64_t *npairs) {
  if (!out || !A) {
    set_error("null matrix or plan out-pointer");
    return CHT_ERR_INVALID;
  }
  cht_plan *p = nullptr;
  CHT_TRY(symbolic(*A->pat, *A->pat, as_stream(stream), &p, nullptr, nullptr, 0.0, true));
  return finish_plan(p, A, A, nnzb_C, npairs, out);
}

int cht_symbolic_multiply_upper(cht_mat_t A, cht_mat_t B, void *stream, cht_plan_t *out,
                                int64_t *nnzb_C, int64_t *npairs) {
  if (!out) {
    set_error("null plan out-pointer");
    return CHT_ERR_INVALID;
  }
  CHT_TRY(check_pair(A, B));
  cht_plan *p = nullptr;
  CHT_TRY(symbolic(*A->pat, *B->pat, as_stream(stream), &p, nullptr, nullptr, 0.0, true));
  return finish_plan(p, A, B, nnzb_C, npairs, out);
}

int cht_mat_mirror_upper(cht_mat_t U, void *stream, cht_mat_t *out) {
  if (!U || !out) {
    set_error("null matrix or out-pointer");
    return CHT_ERR_INVALID;
  }
  cht_mat *m = nullptr;
  CHT_TRY(mirror_upper(U, as_stream(stream), &m));
  *out = m;
  return CHT_OK;
}

int cht_add(double alpha, cht_mat_t A, double beta, cht_mat_t B, void *stream,
            cht_mat_t *out) {
  if (!A || !B || !out) {
    set_error("null matrix or out-pointer");
    return CHT_ERR_INVALID;
  }
  cht_mat *m = nullptr;
  CHT_TRY(add_matrices(alpha, A, beta, B, as_stream(stream), &m));
  *out = m;
  return CHT_OK;
}

int cht_add_identity(double alpha, cht_mat_t A, double beta, void *stream, cht_mat_t *out) {
  if (!A || !out) {
    set_error("null matrix or out-pointer");
    return CHT_ERR_INVALID;
  }
  cht_mat *m = nullptr;
  CHT_TRY(add_matrices(alpha, A, beta, nullptr, as_stream(stream), &m));
  *out = m;
  return CHT_OK;
}

int cht_truncate(cht_mat_t M, double eps, int kind, void *stream, cht_mat_t *out,
                 double *removed) {
  if (!M || !out) {
    set_error("null matrix or out-pointer");
    return CHT_ERR_INVALID;
  }
  if (!(eps >= 0.0) || (kind != CHT_TRUNC_FRO && kind != CHT_TRUNC_MAX)) {
    set_error("truncation: eps must be >= 0 and kind CHT_TRUNC_FRO or CHT_TRUNC_MAX");
    return CHT_ERR_INVALID;
  }
  cht_mat *m = nullptr;
  CHT_TRY(truncate_matrix(M, eps, kind, as_stream(stream), &m, removed));
  *out = m;
  return CHT_OK;
}

int cht_plan_info(cht_plan_t P, int64_t *nnzb_C, int64_t *npairs) {
  if (!P) {
    set_error("null plan");
    return CHT_ERR_INVALID;
  }
  if (nnzb_C) *nnzb_C = P->C->nnz;
  if (npairs) *npairs = P->npairs;
  return CHT_OK;
}

int cht_plan_arrays(cht_plan_t P, const int64_t **d_cseg, const int32_t **d_pair_a,
                    const int32_t **d_pair_b, const int32_t **d_crow, const int32_t **d_ccol,
                    const int32_t **d_order) {
  if (!P) {
    set_error("null plan");
    return CHT_ERR_INVALID;
  }
  if (d_cseg) *d_cseg = P->cseg.p;
  if (d_pair_a) *d_pair_a = P->pa.p;
  if (d_pair_b) *d_pair_b = P->pb.p;
  if (d_crow) *d_crow = P->C->brow.p;
  if (d_ccol) *d_ccol = P->C->bcol.p;
  if (d_order) *d_order = P->order.p;
  return CHT_OK;
}

int cht_plan_free(cht_plan_t P) {
  delete P;
  return CHT_OK;
}

int cht_multiply(cht_plan_t plan, cht_mat_t A, cht_mat_t B, int mode, int32_t nslices,
                 void *stream, cht_mat_t *C, double *max_rel_err_est) {
  if (!plan || !C) {
    set_error("null plan or output pointer");
    return CHT_ERR_INVALID;
  }
  CHT_TRY(check_pair(A, B));
  if (mode != CHT_FP64 && mode != CHT_SPLIT_BF16) {
    set_error("unknown mode %d", mode);
    return CHT_ERR_INVALID;
  }
  cudaStream_t s = as_stream(stream);
  CHT_TRY(check_plan_operands(plan, A, B, nullptr, s));
  cht_mat *m = nullptr;
  bool created = false;
  CHT_TRY(out_matrix(C, plan->C, plan->id, s, &m, &created));
  int rc = CHT_OK;
  double bound = 0.0;
  if (mode == CHT_FP64) {
    GemmWork w{};
    w.X = A->values();
    w.Y = B->values();
    w.Z = m->values();
    w.px = plan->pa.p;
    w.py = plan->pb.p;
    w.seg = plan->cseg.p;
    w.order = plan->order.p;
    w.nunits = plan->C->nnz;
    w.b = plan->b;
    w.nx = A->pat->nnz;
    w.ny = B->pat->nnz;
    w.nz = plan->C->nnz;
    w.npairs = plan->npairs;
    rc = launch_leafgemm_f64(w, s);
    // every output is a dot product of length at most n, computed in FP64:
    // |fl(C) - C| <= gamma_n |A| |B| with gamma_n = n u / (1 - n u)
    const double nu = static_cast<double>(plan->n) * 0x1p-53;
    bound = nu / (1.0 - nu);
  } else {
    rc = split_multiply(plan, A, B, nslices, s, m->values(), &bound);
  }
  if (rc == CHT_OK && max_rel_err_est) {
    rc = cht_sync_status(stream);
    *max_rel_err_est = bound;
  }
  if (rc != CHT_OK) {
    if (created) delete m;
    return rc;
  }
  *C = m;
  return CHT_OK;
}

int cht_multiply_to_host(cht_plan_t plan, cht_mat_t A, cht_mat_t B, void *stream,
                         double *h_C, int32_t nchunks) {
  if (!plan || !h_C || nchunks < 1) {
    set_error("null plan or host buffer, or nchunks < 1");
    return CHT_ERR_INVALID;
  }
  CHT_TRY(check_pair(A, B));
  cudaStream_t s = as_stream(stream);
  CHT_TRY(check_plan_operands(plan, A, B, nullptr, s));
  const int64_t nC = plan->C->nnz;
  DevArray<double> cv;
  CHT_TRY(cv.alloc(static_cast<size_t>(nC) * plan->b * plan->b, s));
  GemmWork w{};
  w.X = A->values();
  w.Y = B->values();
  w.Z = cv.p;
  w.px = plan->pa.p;
  w.py = plan->pb.p;
  w.seg = plan->cseg.p;
  w.nunits = nC;
  w.b = plan->b;
  w.nx = A->pat->nnz;
  w.ny = B->pat->nnz;
  w.nz = nC;
  w.npairs = plan->npairs;
  return multiply_f64_to_host(w, nchunks, h_C, s);
}

int cht_multiply_backward(cht_plan_t plan, cht_mat_t A, cht_mat_t B, cht_mat_t dC,
                          int recompute_pairs, void *stream, cht_mat_t *dA, cht_mat_t *dB) {
  CHT_TRY(check_pair(A, B));
  if (!dC || dC->pat->n != A->pat->n || dC->pat->b != A->pat->b) {
    set_error("dC missing or of another shape");
    return CHT_ERR_SHAPE;
  }
  if (!dA && !dB) return CHT_OK;
  cudaStream_t s = as_stream(stream);
  const Pattern &pa = *A->pat, &pb = *B->pat;
  const bool use_plan = plan && !recompute_pairs && dC->pat->id == plan->C->id &&
                        plan->patA == pa.id && plan->patB == pb.id;
  std::unique_ptr<cht_plan> tmp;
  cht_plan *lists = nullptr;
  if (use_plan) {
    CHT_TRY(backward_lists_from_plan(*plan, pa, pb, s));
    lists = plan;
  } else {
    tmp = std::make_unique<cht_plan>();
    CHT_TRY(backward_lists_recompute(pa, pb, *dC->pat, s, *tmp));
    lists = tmp.get();
  }
  cht_mat *ma = nullptr, *mb = nullptr;
  bool ca = false, cb = false;
  if (dA) CHT_TRY(out_matrix(dA, A->pat, 0, s, &ma, &ca));
  if (dB) {
    int rc = out_matrix(dB, B->pat, 0, s, &mb, &cb);
    if (rc != CHT_OK) {
      if (ca) delete ma;
      return rc;
    }
  }
  int rc = CHT_OK;
  if (ma) {
    GemmWork w{};
    w.X = dC->values();
    w.Y = B->values();
    w.Z = ma->values();
    w.px = lists->dA_c.p;
    w.py = lists->dA_b.p;
    w.seg = lists->segA.p;
    w.order = lists->idA.p;
    w.nunits = pa.nnz;
    w.b = pa.b;
    w.trans_y = 1;
    w.nx = dC->pat->nnz;
    w.ny = pb.nnz;
    w.nz = pa.nnz;
    w.npairs = lists->npairs;
    rc = launch_leafgemm_f64(w, s);
  }
  if (rc == CHT_OK && mb) {
    GemmWork w{};
    w.X = A->values();
    w.Y = dC->values();
    w.Z = mb->values();
    w.px = lists->dB_a.p;
    w.py = lists->dB_c.p;
    w.seg = lists->segB.p;
    w.order = lists->idB.p;
    w.nunits = pb.nnz;
    w.b = pb.b;
    w.trans_x = 1;
    w.nx = pa.nnz;
    w.ny = dC->pat->nnz;
    w.nz = pb.nnz;
    w.npairs = lists->npairs;
    rc = launch_leafgemm_f64(w, s);
  }
  if (rc != CHT_OK) {
    if (ca) delete ma;
    if (cb) delete mb;
    return rc;
  }
  if (dA) *dA = ma;
  if (dB) *dB = mb;
  return CHT_OK;
}

int cht_batch_create(int32_t count, const cht_plan_t *plans, const cht_mat_t *As,
                     const cht_mat_t *Bs, int mode, int32_t nslices, void *stream,
                     cht_batch_t *out) {
  if (!out || count <= 0 || !plans || !As || !Bs) {
    set_error("invalid batch arguments");
    return CHT_ERR_INVALID;
  }
  cht_batch *b = nullptr;
  CHT_TRY(batch_create(count, plans, As, Bs, mode, nslices, as_stream(stream), &b));
  *out = b;
  return CHT_OK;
}

int cht_batch_run(cht_batch_t batch, void *stream) {
  if (!batch) {
    set_error("null batch");
    return CHT_ERR_INVALID;
  }
  return batch_run(batch, as_stream(stream));
}

int cht_batch_output(cht_batch_t batch, int32_t i, cht_mat_t *C) {
  if (!batch || !C) {
    set_error("null batch or output");
    return CHT_ERR_INVALID;
  }
  return batch_output(batch, i, C);
}

int cht_batch_free(cht_batch_t batch) {
  batch_destroy(batch);
  return CHT_OK;
}

int cht_set_option(int option, int64_t value) {
  switch (option) {
    case CHT_OPT_SCHEDULE:
      if (value != 0 && value != 1) break;
      g_opt.schedule = static_cast<int>(value);
      return CHT_OK;
    case CHT_OPT_WAIT_BUDGET_NS:
      if (value < 0) break;
      g_opt.wait_budget_ns = value;
      return CHT_OK;
    case CHT_OPT_CTAS_PER_SM:
      if (value < 0 || value > 32) break;
      g_opt.ctas_per_sm = static_cast<int>(value);
      return CHT_OK;
    case CHT_OPT_FP64_ENGINE:
      if (value < 0 || value > 2) break;
      g_opt.fp64_engine = static_cast<int>(value);
      return CHT_OK;
    case CHT_OPT_SPLIT_SINGLE:
      if (value != 0 && value != 1) break;
      g_opt.split_single = static_cast<int>(value);
      return CHT_OK;
    default:
      break;
  }
  set_error("invalid option %d or value %lld", option, (long long)value);
  return CHT_ERR_INVALID;
}

int cht_get_option(int option, int64_t *value) {
  if (!value) return CHT_ERR_INVALID;
  switch (option) {
    case CHT_OPT_SCHEDULE: *value = g_opt.schedule; return CHT_OK;
    case CHT_OPT_WAIT_BUDGET_NS: *value = g_opt.wait_budget_ns; return CHT_OK;
    case CHT_OPT_CTAS_PER_SM: *value = g_opt.ctas_per_sm; return CHT_OK;
    case CHT_OPT_FP64_ENGINE: *value = g_opt.fp64_engine; return CHT_OK;
    case CHT_OPT_SPLIT_SINGLE: *value = g_opt.split_single; return CHT_OK;
    default: break;
  }
  set_error("invalid option %d", option);
  return CHT_ERR_INVALID;
}

int cht_sync_status(void *stream) {
  cudaStream_t s = as_stream(stream);
  CHT_CUDA_TRY(cudaStreamSynchronize(s));
  int *dptr = nullptr;
  CHT_TRY(device_status_ptr(&dptr));
  int h = 0;
  CHT_CUDA_TRY(cudaMemcpy(&h, dptr, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    CHT_CUDA_TRY(cudaMemset(dptr, 0, sizeof(int)));
    if (h & DEV_STATUS_BAD_INDEX) {
      // (the bounds-checked build; other roles of the kernel then give up
      // through its abort path, which also records a timeout)
      set_error("a kernel met a leaf, pair or unit index outside its array");
      return CHT_ERR_INVALID;
    }
    if (h & DEV_STATUS_TIMEOUT) {
      set_error("a device-side wait ran out of its time budget");
      return CHT_ERR_TIMEOUT;
    }
    set_error("device status word 0x%x", h);
    return CHT_ERR_INVALID;
  }
  return CHT_OK;
}

int64_t cht_launch_count(void) { return g_launches.load(); }

const char *cht_status_str(int status) {
  switch (status) {
    case CHT_OK: return "CHT_OK";
    case CHT_ERR_INVALID: return "CHT_ERR_INVALID";
    case CHT_ERR_SHAPE: return "CHT_ERR_SHAPE";
    case CHT_ERR_DUPLICATE: return "CHT_ERR_DUPLICATE";
    case CHT_ERR_OOM: return "CHT_ERR_OOM";
    case CHT_ERR_CUDA: return "CHT_ERR_CUDA";
    case CHT_ERR_TIMEOUT: return "CHT_ERR_TIMEOUT";
    case CHT_ERR_UNSUPPORTED: return "CHT_ERR_UNSUPPORTED";
    default: return "CHT_ERR_UNKNOWN";
  }
}

const char *cht_last_error(void) { return g_last_error; }

int cht_measure_fp64_peak(int engine, void *stream, double *tflops) {
  if (!tflops || engine < 0 || engine > 3) {
    set_error("invalid engine or null output");
    return CHT_ERR_INVALID;
  }
  return launch_fp64_peak(engine, as_stream(stream), tflops);
}

int cht_measure_fp64_peak_cfg(int engine, int chains, int threads, int ctas_per_sm,
                              void *stream, double *tflops) {
  if (!tflops) {
    set_error("null output");
    return CHT_ERR_INVALID;
  }
  return launch_fp64_peak_cfg(engine, chains, threads, ctas_per_sm, as_stream(stream), tflops);
}

}  // extern "C"
