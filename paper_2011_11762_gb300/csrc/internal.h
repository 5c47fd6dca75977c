// Shared host-side declarations of libcht (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <memory>
#include <mutex>
#include <vector>

#include "cht.h"

namespace cht {

// ----------------------------------------------------------------- errors --
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);  // records, returns CHT_ERR_CUDA

#define CHT_TRY(expr)                \
  do {                               \
    int _rc = (expr);                \
    if (_rc != CHT_OK) return _rc;   \
  } while (0)

#define CHT_CUDA_TRY(call)                                       \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return ::cht::cuda_fail(_e, #call);   \
  } while (0)

// Checks the launch that was just enqueued and counts it.
int launched(const char *name);

extern std::atomic<int64_t> g_launches;

// ---------------------------------------------------------------- options --
struct Options {
  int schedule = 0;               // 0 longest-first, 1 Morton
  int64_t wait_budget_ns = 2000000000LL;
  int ctas_per_sm = 0;            // 0 = auto
  int fp64_engine = 1;            // 0 DMMA, 1 DFMA (measured faster on GB300)
  int split_single = 1;           // 32-leaf split form: one-pair C leaves grouped by B leaf
};
extern Options g_opt;

// Device status word (one per device, zero = OK); kernels OR flags into it.
enum : int { DEV_STATUS_TIMEOUT = 1, DEV_STATUS_BAD_INDEX = 2 };

// Bounds-checked debug build (compiled with -DCHT_BOUNDS_CHECK): the kernels
// test every leaf, pair and unit index they follow against the length of the
// array it indexes before they use it; a failed test records
// DEV_STATUS_BAD_INDEX and the access is skipped (the FP64 kernels skip the
// pair or unit, the split kernels stop through their abort path).  In the
// normal build CHT_INDEX_OK is the constant true and the tests vanish.
#ifdef CHT_BOUNDS_CHECK
#define CHT_INDEX_OK(cond, status) \
  ((cond) || (atomicOr((status), static_cast<int>(::cht::DEV_STATUS_BAD_INDEX)), false))
#else
#define CHT_INDEX_OK(cond, status) true
#endif
int device_status_ptr(int **ptr);
int num_sms(int *sms);
// A second stream of the calling host thread on the current device, with
// two events, for work that can run beside the caller's stream s: record
// `fork` on s and make the side stream wait for it, queue the side work,
// record `join` on the side stream and make s wait for it.  Created at the
// thread's first use on a device and kept.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
int side_stream(SideStream **out);
// Pinned host memory of at least `bytes` for the calling host thread (kept
// and reused: the next call may return the same memory), for device-to-host
// reads that are followed by a synchronisation.
int pinned_scratch(size_t bytes, void **out);

// ------------------------------------------------------------- allocation --
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, size_t bytes, cudaStream_t s);

// A device array released (in stream order) when the owner goes away.
template <class T>
struct DevArray {
  T *p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DevArray() = default;
  DevArray(const DevArray &) = delete;
  DevArray &operator=(const DevArray &) = delete;
  DevArray(DevArray &&o) noexcept { swap(o); }
  DevArray &operator=(DevArray &&o) noexcept {
    reset();
    swap(o);
    return *this;
  }
  ~DevArray() { reset(); }
  void swap(DevArray &o) {
    std::swap(p, o.p);
    std::swap(n, o.n);
    std::swap(s, o.s);
  }
  void reset() {
    if (p) dev_free(p, n * sizeof(T), s);
    p = nullptr;
    n = 0;
  }
  // Allocates max(count, 1) elements; returns CHT_ERR_OOM on failure.
  int alloc(size_t count, cudaStream_t stream) {
    reset();
    size_t c = count ? count : 1;
    p = static_cast<T *>(dev_alloc(c * sizeof(T), stream));
    if (!p) {
      set_error("device allocation of %zu bytes failed", c * sizeof(T));
      return CHT_ERR_OOM;
    }
    n = c;
    s = stream;
    return CHT_OK;
  }
};

// ---------------------------------------------------------------- pattern --
// The stored leaves of a matrix in Morton order, with a row index (CSR) that
// is built the first time a symbolic phase reads it: most product patterns
// are never the right operand of another product, and the index costs two
// radix-sort passes per build.
struct Pattern {
  int64_t n = 0;
  int32_t b = 0;
  int64_t G = 0;   // leaves per side
  int L = 1;       // bits per leaf coordinate, 2^L >= G
  int64_t nnz = 0; // stored leaves
  uint64_t id = 0; // unique per pattern object
  DevArray<uint64_t> mkey;                   // Morton keys, ascending
  DevArray<int32_t> brow, bcol;              // per leaf
  // CSR by leaf row (columns ascending); see ensure_row_index
  mutable DevArray<int64_t> rowptr;          // [G + 1]
  mutable DevArray<int32_t> rowcol, rowleaf; // [nnz]
  mutable bool have_rows = false;
  mutable cudaEvent_t rows_ready = nullptr;  // recorded after the index build
  mutable std::mutex rows_mutex;
  // stored leaves per leaf row and per leaf column, on the host ([G] each;
  // empty when not known, e.g. G > kMaxCountG): read in the synchronisation
  // that sized the pattern, they let the symbolic phase size a product's
  // pair list without one
  std::vector<int32_t> rowcnt, colcnt;
  Pattern() = default;
  Pattern(const Pattern &) = delete;
  Pattern &operator=(const Pattern &) = delete;
  ~Pattern();
};
uint64_t next_id();
int bits_for(int64_t G);
// Most pairs of a C leaf whose pairs the split form's one-pair kernel takes
// as separate units (their exact integer results are summed afterwards; the
// sum of this many stays far inside 64 bits).
constexpr int kFewPairsMax = 4;
// Largest leaf grid side for which patterns keep host leaf counts.
constexpr int64_t kMaxCountG = 1 << 16;
// Adds the leaf counts per row and column of the n Morton keys key[i] with
// keep[i] != 0 (keep null: all) into rowcnt and colcnt ([G] each, device);
// keys outside the G x G grid are skipped.
int count_leaves(const uint64_t *key, const int32_t *keep, int64_t n, int64_t G,
                 int32_t *rowcnt, int32_t *colcnt, cudaStream_t s);
// Fills brow/bcol from the sorted mkey.
int build_pattern_index(Pattern &p, cudaStream_t s);
// Makes p's row index available to work queued on s after this call: built
// on s at the first call, later calls on other streams wait for that build.
int ensure_row_index(const Pattern &p, cudaStream_t s);
// *same = true when x and y store the same leaves (equal n, b and Morton
// keys).  Different pattern objects are compared on the device: d_flag is 4
// bytes of device scratch, and the call synchronises s to read it.
int same_leaves(const Pattern &x, const Pattern &y, int *d_flag, cudaStream_t s, bool *same);

// Blocks for a grid-stride loop over n items: ceil(n / threads), at least 1
// and at most 8 * 65535 (the loops stride by the grid).
inline unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 65535LL * 8) g = 65535LL * 8;
  return static_cast<unsigned>(g);
}

// ------------------------------------------------------------ scan / sort --
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
int scan_exclusive(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
int scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of (key, value) by bits lo_bit .. lo_bit + nbits - 1
// of key.  Passes read whole bytes, so up to 7 bits above that range take
// part in the order too: callers keep them zero.
// `zeroed`: sort_state_words(n, nbits, lo_bit) words of zeroed device memory
// for the sort's histograms and state (used up by the call), or null to
// allocate and clear them here.
int radix_sort_pairs(const uint64_t *kin, const int32_t *vin, uint64_t *kout,
                     int32_t *vout, int64_t n, int nbits, cudaStream_t s, int lo_bit = 0,
                     unsigned long long *zeroed = nullptr);
int64_t sort_state_words(int64_t n, int nbits, int lo_bit = 0);
// Copy of a device int64 to the host (synchronises s).
int read_i64(const int64_t *d, int64_t *h, cudaStream_t s);

// ---------------------------------------------------------------- kernels --
// The grouped leaf-GEMM work description (one output leaf per unit).
struct GemmWork {
  const double *X;        // left operand leaves
  const double *Y;        // right operand leaves
  double *Z;              // output leaves (Z[unit_out[u]] gets the sum)
  const int32_t *px;      // per pair: index into X
  const int32_t *py;      // per pair: index into Y
  const int64_t *seg;     // per output leaf: pair segment [seg[o], seg[o+1])
  const int32_t *order;   // schedule: output leaf of each unit
  int64_t nunits;
  int32_t b;
  int trans_x, trans_y;   // use X^T / Y^T in the product
  // lengths (read by the bounds-checked build): leaves of X, Y and Z, pairs
  int64_t nx, ny, nz, npairs;
};
// Z[o] = sum_p op(X[px[p]]) op(Y[py[p]]) for every unit; FP64.
int launch_leafgemm_f64(const GemmWork &w, cudaStream_t s);
// The same over all w.nunits C leaves (w.order unused) in `nchunks` Morton
// ranges, each copied to h_out (host) while the next is computed.
int multiply_f64_to_host(const GemmWork &w, int64_t nchunks, double *h_out, cudaStream_t s);

// One product of a batch, as the batched kernels see it.
struct ProdDesc {
  const double *X;
  const double *Y;
  double *Z;
  const int32_t *px;
  const int32_t *py;
  const int64_t *seg;
  int32_t b;
  int32_t pad;
  int64_t nx, ny, nz, npairs;  // lengths, as in GemmWork
};
// Batched FP64 multiply: units (product << 32 | output leaf) in one launch;
// maxb = the largest leaf size among the products (32 or 64).
// d_counter: 8 bytes of device scratch, zeroed by the call.
int launch_leafgemm_f64_batch(const ProdDesc *d_prods, int32_t nprods, const int64_t *d_units,
                              int64_t nunits, int maxb, unsigned long long *d_counter,
                              cudaStream_t s);

int launch_fp64_peak(int engine, cudaStream_t s, double *tflops);
int launch_fp64_peak_cfg(int engine, int chains, int threads, int per_sm, cudaStream_t s,
                         double *tflops);

}  // namespace cht

// ------------------------------------------------------------ opaque types --
struct cht_mat {
  std::shared_ptr<cht::Pattern> pat;
  cht::DevArray<double> vals;  // [nnz][b][b]
  uint64_t plan_id = 0;        // plan that produced it (0 = built from blocks)
  bool view = false;           // non-owning view (batched outputs)
  double *view_vals = nullptr;
  double *values() { return view ? view_vals : vals.p; }
};

struct cht_plan {
  uint64_t id = 0;
  int64_t n = 0;
  int32_t b = 0;
  int64_t nA = 0, nB = 0;
  uint64_t patA = 0, patB = 0;       // pattern ids of A and B
  // the operand patterns themselves, kept so that a multiply can check that
  // its operands store the leaves the pair lists index
  std::shared_ptr<cht::Pattern> opA, opB;
  std::shared_ptr<cht::Pattern> C;   // product pattern
  int64_t npairs = 0;
  int64_t max_seg = 0;               // most pairs of any C leaf
  // 32-leaf plans, for the split form's B-leaf groups (read in the symbolic
  // phase's synchronisation; -1: not known): C leaves with one pair, C
  // leaves with 2 .. kFewPairsMax pairs and those leaves' pairs (each pair a
  // unit of its own, summed afterwards), the groups of up to four units
  // sharing a B leaf, and the units per B leaf
  int64_t n_one = -1, n_few = -1, n_virt = -1, n_groups = -1;
  cht::DevArray<int64_t> sym_block;  // the symbolic phase's counters (kept for:)
  const int32_t *one_pair_b = nullptr;  // [nB], inside sym_block
  cht::DevArray<int64_t> cseg;       // [nC + 1]
  cht::DevArray<int32_t> pa, pb, pc; // per pair (sorted by C leaf, then K)
  cht::DevArray<int32_t> order;      // schedule [nC]
  // backward regroupings (built on first use)
  bool have_bwd = false;
  cht::DevArray<int64_t> segA, segB;      // [nA + 1], [nB + 1]
  cht::DevArray<int32_t> dA_c, dA_b;      // pairs grouped by A leaf
  cht::DevArray<int32_t> dB_a, dB_c;      // pairs grouped by B leaf
  cht::DevArray<int32_t> idA, idB;        // identity schedules
  // the split form's grouping of one-pair C leaves (32-leaves), built on
  // first use; owned here, defined in split.cu
  std::shared_ptr<void> split_groups;
};

namespace cht {
// CHT_OK when A and B store the leaves of the plan's operands (the same
// pattern objects, or equal patterns compared with same_leaves); otherwise
// CHT_ERR_SHAPE.  d_flag: 4 bytes of device scratch, or null to allocate.
int check_plan_operands(const cht_plan *plan, const cht_mat *A, const cht_mat *B, int *d_flag,
                        cudaStream_t s);
}  // namespace cht

// A batch of independent products run by one persistent launch.
struct cht_batch {
  int32_t count = 0;
  int mode = CHT_FP64;
  int nslices = 0;
  std::vector<cht_plan *> plans;  // not owned: the caller keeps them alive
  std::vector<cht_mat *> As, Bs;  // not owned
  cht::DevArray<cht::ProdDesc> prods;
  cht::DevArray<int64_t> units;   // (product << 32) | C leaf, in run order
  cht::DevArray<double> cvals;    // every product's C values
  cht::DevArray<unsigned long long> counter;
  int64_t nunits = 0;
  int maxb = 32;                  // largest leaf size among the products
  std::vector<std::unique_ptr<cht_mat>> views;
  void *split_state = nullptr;    // owned by the split path
  ~cht_batch();
};
