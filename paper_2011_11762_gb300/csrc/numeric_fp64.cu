// Numeric phase, FP64 (step S6; also the two sampled products of the
// backward, S8): a persistent grouped leaf-GEMM.
//
// Paper, Section 3: leaf products are dense double-precision matrix products
// (BLAS dgemm on the leaf's blocks); the multiply task adds the products of
// the quadrant pairs.  Here each unit of work is one output leaf o:
//     Z[o] = sum_{p in seg(o)} op(X[px[p]]) * op(Y[py[p]])
// summed in the segment's order (ascending K for the forward product) in
// registers, and stored once -- no atomics.  Units are taken from an atomic
// counter in schedule order (longest segment first by default).
//
// Data movement: each CTA streams its pairs' two leaves (b*b doubles each,
// contiguous) into a ring of shared-memory stages with one-dimensional TMA
// bulk copies completing on an mbarrier per stage.  Every wait is bounded;
// on expiry the CTA records DEV_STATUS_TIMEOUT, drains its copies in flight
// and returns.
//
// Arithmetic: FP64 tensor-core MMA (mma.sync m8n8k4 f64, "DMMA"; engine 0)
// or plain FP64 FMAs from a per-thread register tile (engine 1).
#include <algorithm>
#include <mutex>

#include "device.cuh"
#include "internal.h"

namespace cht {

namespace {

constexpr int kThreads = 128;  // 4 warps, a 2 x 2 grid of warp tiles

// Arithmetic engines: 0 = DMMA (128 threads), 1 = DFMA with a 4 x 8 (b = 64)
// or 2 x 4 (b = 32) register tile per thread (128 threads), 2 = DFMA with a
// 4 x 4 tile per thread (256 threads, b = 64).  GB300 issues about two FP64
// FMAs per clock per SM; with one 128-thread CTA per SM (the 64-leaf ring
// fills shared memory) each scheduler has one warp and its shared-memory
// loads and barriers leave the FP64 pipe idle about 5% of the time; two
// warps per scheduler hide them.
__host__ __device__ constexpr int threads_of(int engine) { return engine == 2 ? 256 : 128; }
constexpr int64_t kDrainBudgetNs = 2000000000LL;

template <int B>
struct LeafCfg {
  static constexpr int kLeaf = B * B;
  static constexpr int kStages = (B == 64) ? 2 : 3;
  static constexpr size_t kSmem = sizeof(double) * 2 * kStages * kLeaf + 16 * kStages;
};

template <int B, bool TX>
__device__ __forceinline__ double ldx(const double *xs, int row, int k) {
  return TX ? xs[k * B + row] : xs[row * B + k];
}
template <int B, bool TY>
__device__ __forceinline__ double ldy(const double *ys, int k, int col) {
  return TY ? ys[col * B + k] : ys[k * B + col];
}

// Per-thread accumulator tile and the compute / store of one leaf product.
template <int B, bool TX, bool TY, int ENGINE>
struct Tile;

// DMMA: warp tile (B/2) x (B/2) = MT x NT tiles of 8 x 8.
template <int B, bool TX, bool TY>
struct Tile<B, TX, TY, 0> {
  static constexpr int WT = B / 2, MT = WT / 8, NT = WT / 8;
  double acc[MT][NT][2];
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < NT; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
  }
  __device__ void mac(const double *xs, const double *ys) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * WT, wn = (warp & 1) * WT;
    const int gr = lane >> 2, gc = lane & 3;
#pragma unroll 4
    for (int k = 0; k < B; k += 4) {
      double a[MT], b[NT];
#pragma unroll
      for (int i = 0; i < MT; ++i) a[i] = ldx<B, TX>(xs, wm + i * 8 + gr, k + gc);
#pragma unroll
      for (int j = 0; j < NT; ++j) b[j] = ldy<B, TY>(ys, k + gc, wn + j * 8 + gr);
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j) dmma_8x8x4(acc[i][j][0], acc[i][j][1], a[i], b[j]);
    }
  }
  __device__ void store(double *z) const {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * WT, wn = (warp & 1) * WT;
    const int gr = lane >> 2, gc = lane & 3;
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        double2 v = make_double2(acc[i][j][0], acc[i][j][1]);
        *reinterpret_cast<double2 *>(z + (wm + i * 8 + gr) * B + wn + j * 8 + 2 * gc) = v;
      }
  }
};

// DFMA: thread tile RM x RN; 16 row groups x 8 column groups of threads.
template <int B, bool TX, bool TY>
struct Tile<B, TX, TY, 1> {
  static constexpr int RM = B / 16, RN = B / 8;
  double acc[RM][RN];
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) acc[i][j] = 0.0;
  }
  __device__ void mac(const double *xs, const double *ys) {
    const int tr = threadIdx.x >> 3, tc = threadIdx.x & 7;
#pragma unroll 2
    for (int k = 0; k < B; ++k) {
      double a[RM], b[RN];
#pragma unroll
      for (int i = 0; i < RM; ++i) a[i] = ldx<B, TX>(xs, tr * RM + i, k);
#pragma unroll
      for (int j = 0; j < RN; ++j) b[j] = ldy<B, TY>(ys, k, tc * RN + j);
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  __device__ void store(double *z) const {
    const int tr = threadIdx.x >> 3, tc = threadIdx.x & 7;
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; j += 2)
        *reinterpret_cast<double2 *>(z + (tr * RM + i) * B + tc * RN + j) =
            make_double2(acc[i][j], acc[i][j + 1]);
  }
};

// DFMA, 256 threads: thread tile RM x RN; 16 row groups x 16 column groups.
template <int B, bool TX, bool TY>
struct Tile<B, TX, TY, 2> {
  static constexpr int RM = B / 16, RN = B / 16;
  double acc[RM][RN];
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) acc[i][j] = 0.0;
  }
  __device__ void mac(const double *xs, const double *ys) {
    const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll 4
    for (int k = 0; k < B; ++k) {
      double a[RM], b[RN];
#pragma unroll
      for (int i = 0; i < RM; ++i) a[i] = ldx<B, TX>(xs, tr * RM + i, k);
#pragma unroll
      for (int j = 0; j < RN; ++j) b[j] = ldy<B, TY>(ys, k, tc * RN + j);
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  __device__ void store(double *z) const {
    const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; j += 2)
        *reinterpret_cast<double2 *>(z + (tr * RM + i) * B + tc * RN + j) =
            make_double2(acc[i][j], acc[i][j + 1]);
  }
};

// One output leaf: Z = sum over the pair segment [p0, p0 + np) of
// op(X[px[p]]) op(Y[py[p]]), with a ring of S shared-memory stages (stage
// pitch `pitch` doubles).  `it` counts the pairs this CTA consumed so far
// (it fixes each stage's mbarrier phase).  Returns false after a timeout
// (recorded in `status`; this CTA's copies in flight have landed).
template <int B, bool TX, bool TY, int ENGINE, int S>
__device__ bool run_unit(const double *__restrict__ X, const double *__restrict__ Y,
                         double *__restrict__ Z, const int32_t *__restrict__ px,
                         const int32_t *__restrict__ py, int64_t p0, int64_t np, double *sx,
                         double *sy, int pitch, uint64_t *full, uint32_t &it, int64_t wait_ns,
                         int *status, int64_t nx, int64_t ny) {
  constexpr int LEAF = B * B;
  constexpr uint32_t kBytes = LEAF * sizeof(double);
  const int tid = threadIdx.x;
  auto issue = [&](int64_t p, uint32_t st) {
    const int64_t ix = px[p], iy = py[p];
    if (CHT_INDEX_OK(ix >= 0 && ix < nx && iy >= 0 && iy < ny, status)) {
      mbar_arrive_expect_tx(&full[st], 2 * kBytes);
      bulk_g2s(sx + st * pitch, X + ix * LEAF, kBytes, &full[st]);
      bulk_g2s(sy + st * pitch, Y + iy * LEAF, kBytes, &full[st]);
    } else {
      mbar_arrive(&full[st]);  // the stage's phase completes without data
    }
  };
  (void)nx;
  (void)ny;
  Tile<B, TX, TY, ENGINE> tile;
  tile.zero();
  if (tid == 0)
    for (int64_t j = 0; j < S - 1 && j < np; ++j) issue(p0 + j, (it + j) % S);
  for (int64_t i = 0; i < np; ++i) {
    if (tid == 0 && i + S - 1 < np) issue(p0 + i + S - 1, (it + i + S - 1) % S);
    const uint32_t st = (it + i) % S, parity = ((it + i) / S) & 1u;
    const bool ok = mbar_wait_bounded(&full[st], parity, wait_ns);
    if (__syncthreads_or(!ok)) {
      // Timed out: record it, let this CTA's copies in flight land, return.
      if (tid == 0) {
        atomicOr(status, DEV_STATUS_TIMEOUT);
        const int64_t issued = (i + S < np) ? i + S : np;
        for (int64_t j = i; j < issued; ++j)
          mbar_wait_bounded(&full[(it + j) % S], ((it + j) / S) & 1u, kDrainBudgetNs);
      }
      __syncthreads();
      return false;
    }
    tile.mac(sx + st * pitch, sy + st * pitch);
    __syncthreads();  // stage st may be refilled after this point
  }
  it += static_cast<uint32_t>(np);
  tile.store(Z);
  return true;
}

template <int B, bool TX, bool TY, int ENGINE>
__global__ void __launch_bounds__(threads_of(ENGINE))
    k_leafgemm_f64(const GemmWork w, int *__restrict__ status, int64_t wait_ns,
                   unsigned long long *__restrict__ next_unit) {
  using Cfg = LeafCfg<B>;
  constexpr int S = Cfg::kStages, LEAF = Cfg::kLeaf;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *sx = reinterpret_cast<double *>(smem_raw);
  double *sy = sx + S * LEAF;
  uint64_t *full = reinterpret_cast<uint64_t *>(sy + S * LEAF);
  __shared__ long long s_unit;

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int st = 0; st < S; ++st) mbar_init(&full[st], 1);
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t it = 0;  // pairs consumed so far by this CTA
  for (;;) {
    if (tid == 0) s_unit = static_cast<long long>(atomicAdd(next_unit, 1ULL));
    __syncthreads();
    const int64_t u = s_unit;
    __syncthreads();
    if (u >= w.nunits) break;
    const int64_t o = w.order[u];
    if (!CHT_INDEX_OK(o >= 0 && o < w.nz, status)) continue;
    const int64_t p0 = w.seg[o], np = w.seg[o + 1] - p0;
    if (!CHT_INDEX_OK(p0 >= 0 && np >= 0 && p0 + np <= w.npairs, status)) continue;
    if (!run_unit<B, TX, TY, ENGINE, S>(w.X, w.Y, w.Z + o * LEAF, w.px, w.py, p0, np, sx, sy,
                                        LEAF, full, it, wait_ns, status, w.nx, w.ny))
      return;
  }
}

// Batched form: units from many products (each with its own leaf size) in
// one launch.  Unit u is product units[u] >> 32, output leaf units[u] & 0xffffffff.
// MAXB is the largest leaf size of the batch: the stage ring is sized for it
// (a batch of 32-leaf products gets the 32-leaf kernel's ring and occupancy).
template <int ENGINE, int MAXB>
__global__ void __launch_bounds__(threads_of(ENGINE))
    k_leafgemm_f64_batch(const ProdDesc *__restrict__ prods, int32_t nprods,
                         const int64_t *__restrict__ units, int64_t nunits,
                         int *__restrict__ status, int64_t wait_ns,
                         unsigned long long *__restrict__ next_unit) {
  (void)nprods;
  constexpr int S = LeafCfg<MAXB>::kStages, PITCH = MAXB * MAXB;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double *sx = reinterpret_cast<double *>(smem_raw);
  double *sy = sx + S * PITCH;
  uint64_t *full = reinterpret_cast<uint64_t *>(sy + S * PITCH);
  __shared__ long long s_unit;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int st = 0; st < S; ++st) mbar_init(&full[st], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t it = 0;
  for (;;) {
    if (tid == 0) s_unit = static_cast<long long>(atomicAdd(next_unit, 1ULL));
    __syncthreads();
    const int64_t u = s_unit;
    __syncthreads();
    if (u >= nunits) break;
    const int64_t packed = units[u];
    if (!CHT_INDEX_OK((packed >> 32) >= 0 && (packed >> 32) < nprods, status)) continue;
    const ProdDesc d = prods[packed >> 32];
    const int64_t o = packed & 0xffffffffLL;
    if (!CHT_INDEX_OK(o < d.nz, status)) continue;
    const int64_t p0 = d.seg[o], np = d.seg[o + 1] - p0;
    if (!CHT_INDEX_OK(p0 >= 0 && np >= 0 && p0 + np <= d.npairs, status)) continue;
    bool ok = false;
    if constexpr (MAXB == 64) {
      if (d.b == 64)
        ok = run_unit<64, false, false, ENGINE, S>(d.X, d.Y, d.Z + o * 4096, d.px, d.py, p0, np,
                                                   sx, sy, PITCH, full, it, wait_ns, status, d.nx, d.ny);
      else
        ok = run_unit<32, false, false, ENGINE, S>(d.X, d.Y, d.Z + o * 1024, d.px, d.py, p0, np,
                                                   sx, sy, PITCH, full, it, wait_ns, status, d.nx, d.ny);
    } else {
      // every product of this batch has 32-leaves
      ok = run_unit<32, false, false, ENGINE, S>(d.X, d.Y, d.Z + o * 1024, d.px, d.py, p0, np, sx,
                                                 sy, PITCH, full, it, wait_ns, status, d.nx, d.ny);
    }
    if (!ok) return;
  }
}

template <int B, bool TX, bool TY, int ENGINE>
int launch_t(const GemmWork &w, cudaStream_t s, int *status, unsigned long long *counter) {
  using Cfg = LeafCfg<B>;
  auto kern = k_leafgemm_f64<B, TX, TY, ENGINE>;
  CHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(Cfg::kSmem)));
  int sms = 0;
  CHT_TRY(num_sms(&sms));
  constexpr int NT = threads_of(ENGINE);
  int per_sm = g_opt.ctas_per_sm;
  if (per_sm <= 0) {
    int occ = 0;
    CHT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, Cfg::kSmem));
    per_sm = std::max(1, occ);
  }
  int64_t grid = std::min<int64_t>(w.nunits, static_cast<int64_t>(sms) * per_sm);
  if (grid < 1) grid = 1;
  kern<<<static_cast<unsigned>(grid), NT, Cfg::kSmem, s>>>(w, status, g_opt.wait_budget_ns,
                                                           counter);
  return launched("leafgemm_f64");
}

template <int B, int ENGINE>
int launch_b(const GemmWork &w, cudaStream_t s, int *status, unsigned long long *counter) {
  if (!w.trans_x && !w.trans_y) return launch_t<B, false, false, ENGINE>(w, s, status, counter);
  if (!w.trans_x && w.trans_y) return launch_t<B, false, true, ENGINE>(w, s, status, counter);
  if (w.trans_x && !w.trans_y) return launch_t<B, true, false, ENGINE>(w, s, status, counter);
  return launch_t<B, true, true, ENGINE>(w, s, status, counter);
}

// ----------------------------------------------------------- FP64 peak --
// Register-resident FP64 throughput kernels for the roofline denominator.
// DFMA: every thread runs CH independent FMA chains a_i <- a_i * y + x (y and
// x kernel arguments, so nothing folds); TILE: a 4 x 8 register tile of
// accumulators updated from 4 + 8 operand registers, the shape of the leaf
// GEMM's inner loop without its shared-memory loads.  DMMA: every warp runs
// CH independent mma.sync m8n8k4 f64 chains.  The results feed a store that
// never happens, so the work cannot be removed.
template <int CH>
__global__ void k_peak_dfma(double *out, int iters, double y, double x0) {
  double a[CH];
  const double x = x0 + 1e-9 * threadIdx.x;
#pragma unroll
  for (int i = 0; i < CH; ++i) a[i] = 1e-3 * i;
  for (int n = 0; n < iters; ++n)
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = fma(a[i], y, x);
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += a[i];
  if (s == 12345.0) out[0] = s;
}

__global__ void k_peak_tile(double *out, int iters, double y, double x0) {
  double a[4], b[8], acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = y * (1.0 + 1e-3 * (i + threadIdx.x));
#pragma unroll
  for (int j = 0; j < 8; ++j) b[j] = x0 * (1.0 - 1e-3 * j);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
  for (int n = 0; n < iters; ++n)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  double s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) s += acc[i][j];
  if (s == 12345.0) out[0] = s;
}

// The leaf GEMM's own inner loop (Tile<B, ..., DFMA>::mac) over one pair of
// B x B leaves held in shared memory, `iters` times: the FP64 kernel's
// arithmetic and shared-memory loads without its copies and unit hand-offs.
template <int B, int ENG>
__global__ void __launch_bounds__(threads_of(ENG)) k_peak_leaf(double *out, int iters, double y,
                                                               double x0) {
  extern __shared__ __align__(16) double peak_smem[];
  double *sx = peak_smem, *sy = peak_smem + B * B;
  for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
    sx[e] = y * (1.0 + 1e-6 * e);
    sy[e] = x0 * (1.0 - 1e-6 * e);
  }
  __syncthreads();
  Tile<B, false, false, ENG> tile;
  tile.zero();
  for (int n = 0; n < iters; ++n) tile.mac(sx, sy);
  double s = 0;
#pragma unroll
  for (int i = 0; i < Tile<B, false, false, ENG>::RM; ++i)
#pragma unroll
    for (int j = 0; j < Tile<B, false, false, ENG>::RN; ++j) s += tile.acc[i][j];
  if (s == 12345.0) out[0] = s;
}

template <int CH>
__global__ void k_peak_dmma(double *out, int iters, double y, double x0) {
  double d[CH][2];
  const double a = x0 + 1e-9 * threadIdx.x, b = y;
#pragma unroll
  for (int i = 0; i < CH; ++i) d[i][0] = d[i][1] = i;
  for (int n = 0; n < iters; ++n)
#pragma unroll
    for (int i = 0; i < CH; ++i) dmma_8x8x4(d[i][0], d[i][1], a, b);
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += d[i][0] + d[i][1];
  if (s == 12345.0) out[0] = s;
}

}  // namespace

int launch_leafgemm_f64(const GemmWork &w, cudaStream_t s) {
  if (w.nunits <= 0) return CHT_OK;
  int *status = nullptr;
  CHT_TRY(device_status_ptr(&status));
  DevArray<unsigned long long> counter;
  CHT_TRY(counter.alloc(1, s));
  CHT_CUDA_TRY(cudaMemsetAsync(counter.p, 0, sizeof(unsigned long long), s));
  const int engine = g_opt.fp64_engine;
  if (w.b == 64)
    return engine == 1   ? launch_b<64, 2>(w, s, status, counter.p)
           : engine == 2 ? launch_b<64, 1>(w, s, status, counter.p)
                         : launch_b<64, 0>(w, s, status, counter.p);
  if (w.b == 32)
    return engine ? launch_b<32, 1>(w, s, status, counter.p) : launch_b<32, 0>(w, s, status, counter.p);
  set_error("leaf size %d: the numeric kernels take b = 32 or b = 64", w.b);
  return CHT_ERR_UNSUPPORTED;
}

namespace {

// Chunk of C leaf u is floor(u * nchunks / nC); inside a chunk the units go
// longest segment first.  key = chunk << 32 | (2^32 - 1 - segment length).
__global__ void k_chunk_keys(const int64_t *__restrict__ seg, int64_t nC, int64_t nchunks,
                             uint64_t *__restrict__ key, int32_t *__restrict__ idx) {
  for (int64_t u = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; u < nC;
       u += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t len = seg[u + 1] - seg[u];
    if (len > 0xffffffffLL) len = 0xffffffffLL;
    const uint64_t chunk = static_cast<uint64_t>(u * nchunks / nC);
    key[u] = (chunk << 32) | (0xffffffffULL - static_cast<uint64_t>(len));
    idx[u] = static_cast<int32_t>(u);
  }
}

}  // namespace

// C = A*B in FP64 with C going to host memory while it is computed: the C
// leaves are cut into `nchunks` contiguous Morton ranges, each computed by
// one launch (longest segment first inside the range) and copied to h_out on
// a second stream as soon as it is done, so the copies overlap the next
// ranges' arithmetic.  The caller's stream waits for the last copy.
int multiply_f64_to_host(const GemmWork &w0, int64_t nchunks, double *h_out, cudaStream_t s) {
  const int64_t nC = w0.nunits;
  if (nC <= 0) return CHT_OK;
  if (nchunks < 1) nchunks = 1;
  if (nchunks > nC) nchunks = nC;
  const int64_t bb = static_cast<int64_t>(w0.b) * w0.b;
  DevArray<uint64_t> key, skey;
  DevArray<int32_t> idx, sidx;
  CHT_TRY(key.alloc(nC, s));
  CHT_TRY(skey.alloc(nC, s));
  CHT_TRY(idx.alloc(nC, s));
  CHT_TRY(sidx.alloc(nC, s));
  {
    int64_t g = (nC + 255) / 256;
    if (g > 65535LL * 8) g = 65535LL * 8;
    k_chunk_keys<<<static_cast<unsigned>(g), 256, 0, s>>>(w0.seg, nC, nchunks, key.p, idx.p);
    CHT_TRY(launched("chunk_keys"));
  }
  CHT_TRY(radix_sort_pairs(key.p, idx.p, skey.p, sidx.p, nC, 32 + bits_for(nchunks + 1), s));
  cudaStream_t cs = nullptr;
  CHT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  int rc = CHT_OK;
  for (int64_t k = 0; k < nchunks && rc == CHT_OK; ++k) {
    const int64_t u0 = (k * nC + nchunks - 1) / nchunks;
    const int64_t u1 = ((k + 1) * nC + nchunks - 1) / nchunks;
    if (u1 <= u0) continue;
    GemmWork w = w0;
    w.order = sidx.p + u0;
    w.nunits = u1 - u0;
    rc = launch_leafgemm_f64(w, s);
    if (rc != CHT_OK) break;
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_out + u0 * bb, w0.Z + u0 * bb, sizeof(double) * (u1 - u0) * bb,
                          cudaMemcpyDeviceToHost, cs);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) rc = cuda_fail(e, "chunk copy");
  }
  // the caller's stream (and the frees of the scratch above) wait for the copies
  cudaEvent_t done;
  cudaError_t e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(done, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, done, 0);
  cudaEventDestroy(done);
  cudaStreamDestroy(cs);
  if (rc == CHT_OK && e != cudaSuccess) rc = cuda_fail(e, "copy stream join");
  return rc;
}

int launch_leafgemm_f64_batch(const ProdDesc *d_prods, int32_t nprods, const int64_t *d_units,
                              int64_t nunits, int maxb, unsigned long long *d_counter,
                              cudaStream_t s) {
  if (nunits <= 0) return CHT_OK;
  int *status = nullptr;
  CHT_TRY(device_status_ptr(&status));
  int sms = 0;
  CHT_TRY(num_sms(&sms));
  const size_t smem = maxb == 64 ? LeafCfg<64>::kSmem : LeafCfg<32>::kSmem;
  // engines as for single products: 64-leaf batches take the 256-thread DFMA
  // tile unless the 128-thread one is asked for
  const int engine = g_opt.fp64_engine == 0 ? 0 : (maxb == 64 && g_opt.fp64_engine == 1) ? 2 : 1;
  auto kern = maxb == 64
                  ? (engine == 2 ? k_leafgemm_f64_batch<2, 64>
                     : engine == 1 ? k_leafgemm_f64_batch<1, 64> : k_leafgemm_f64_batch<0, 64>)
                  : (engine ? k_leafgemm_f64_batch<1, 32> : k_leafgemm_f64_batch<0, 32>);
  const int NT = threads_of(engine);
  CHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)));
  int occ = 0;
  CHT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem));
  const int64_t grid = std::min<int64_t>(nunits, static_cast<int64_t>(sms) * std::max(1, occ));
  CHT_CUDA_TRY(cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), s));
  kern<<<static_cast<unsigned>(grid), NT, smem, s>>>(d_prods, nprods, d_units, nunits,
                                                          status, g_opt.wait_budget_ns,
                                                          d_counter);
  return launched("leafgemm_f64_batch");
}

// One configuration of the FP64 peak kernels: engine 1 = DFMA chains, 2 =
// the DFMA register tile (chains ignored: 32 accumulators), 0 = DMMA chains;
// `threads` per CTA, `per_sm` CTAs per SM on every SM.  The iteration count
// is sized for about 40 ms per launch at 1.2 TFLOP/s; one warm-up launch,
// then one timed launch (CUDA events on s).
int launch_fp64_peak_cfg(int engine, int chains, int threads, int per_sm, cudaStream_t s,
                         double *tflops) {
  const bool chains_ok = engine == 3 ? (chains == 32 || chains == 64)
                                     : (chains == 4 || chains == 8 || chains == 16 ||
                                        chains == 32 || engine == 2);
  if (engine < 0 || engine > 3 || threads < 32 || threads > 1024 || threads % 32 != 0 ||
      per_sm < 1 || per_sm > 32 || !chains_ok ||
      (engine == 3 && threads != 128 && !(threads == 256 && chains == 64))) {
    set_error("FP64 peak: engine 0..3, chains 4/8/16/32 (engine 3: the leaf size, 32 or 64, "
              "with 128 threads, or 64 with 256), threads a multiple of 32 in [32, 1024], "
              "1..32 CTAs per SM");
    return CHT_ERR_INVALID;
  }
  const void *fn = nullptr;
  switch (engine) {
    case 0:
      fn = chains == 4 ? (const void *)k_peak_dmma<4> : chains == 8 ? (const void *)k_peak_dmma<8>
           : chains == 16 ? (const void *)k_peak_dmma<16> : (const void *)k_peak_dmma<32>;
      break;
    case 1:
      fn = chains == 4 ? (const void *)k_peak_dfma<4> : chains == 8 ? (const void *)k_peak_dfma<8>
           : chains == 16 ? (const void *)k_peak_dfma<16> : (const void *)k_peak_dfma<32>;
      break;
    case 2: fn = (const void *)k_peak_tile; break;
    default:
      fn = chains == 32 ? (const void *)k_peak_leaf<32, 1>
           : threads == 256 ? (const void *)k_peak_leaf<64, 2> : (const void *)k_peak_leaf<64, 1>;
  }
  cudaFuncAttributes fa;
  CHT_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
  if (threads > fa.maxThreadsPerBlock) {
    set_error("FP64 peak: %d threads exceed this kernel's %d (registers)", threads,
              fa.maxThreadsPerBlock);
    return CHT_ERR_INVALID;
  }
  int sms = 0;
  CHT_TRY(num_sms(&sms));
  const int grid = sms * per_sm;
  const int ch = engine == 2 ? 32 : chains;
  // FLOPs per iteration per thread (a DMMA's 2 * 8 * 8 * 4 shared by 32 lanes;
  // one leaf product, 2 b^3, shared by the kThreads threads)
  const double per_iter = engine == 0   ? ch * 2.0 * 8 * 8 * 4 / 32.0
                          : engine == 3 ? 2.0 * ch * ch * ch / threads
                                        : ch * 2.0;
  const double target = 4.8e10;  // ~40 ms at 1.2 TFLOP/s
  int64_t iters = static_cast<int64_t>(target / (static_cast<double>(grid) * threads * per_iter));
  iters = std::max<int64_t>(64, std::min<int64_t>(iters, 1 << 24));
  DevArray<double> out;
  CHT_TRY(out.alloc(1, s));
  cudaEvent_t e0, e1;
  CHT_CUDA_TRY(cudaEventCreate(&e0));
  CHT_CUDA_TRY(cudaEventCreate(&e1));
  const double y = 0.999999999, x0 = 1.0;
  const int it = static_cast<int>(iters);
  int rc = CHT_OK;
  for (int rep = 0; rep < 2 && rc == CHT_OK; ++rep) {
    if (rep == 1) cudaEventRecord(e0, s);
    if (engine == 3) {
      // two b x b leaves of dynamic shared memory (64 KB at b = 64)
      const int smem = static_cast<int>(2 * sizeof(double) * ch * ch);
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "fp64 peak smem attribute");
        break;
      }
      if (ch == 32)
        k_peak_leaf<32, 1><<<grid, threads, smem, s>>>(out.p, it, y, x0);
      else if (threads == 256)
        k_peak_leaf<64, 2><<<grid, threads, smem, s>>>(out.p, it, y, x0);
      else
        k_peak_leaf<64, 1><<<grid, threads, smem, s>>>(out.p, it, y, x0);
    } else if (engine == 2) {
      k_peak_tile<<<grid, threads, 0, s>>>(out.p, it, y, x0);
    } else if (engine == 1) {
      switch (ch) {
        case 4: k_peak_dfma<4><<<grid, threads, 0, s>>>(out.p, it, y, x0); break;
        case 8: k_peak_dfma<8><<<grid, threads, 0, s>>>(out.p, it, y, x0); break;
        case 16: k_peak_dfma<16><<<grid, threads, 0, s>>>(out.p, it, y, x0); break;
        default: k_peak_dfma<32><<<grid, threads, 0, s>>>(out.p, it, y, x0); break;
      }
    } else {
      switch (ch) {
        case 4: k_peak_dmma<4><<<grid, threads, 0, s>>>(out.p, it, y, x0); break;
        case 8: k_peak_dmma<8><<<grid, threads, 0, s>>>(out.p, it, y, x0); break;
        case 16: k_peak_dmma<16><<<grid, threads, 0, s>>>(out.p, it, y, x0); break;
        default: k_peak_dmma<32><<<grid, threads, 0, s>>>(out.p, it, y, x0); break;
      }
    }
    rc = launched("fp64_peak");
  }
  float ms = 0.f;
  if (rc == CHT_OK) {
    cudaError_t e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) rc = cuda_fail(e, "fp64 peak timing");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CHT_OK) return rc;
  *tflops = static_cast<double>(grid) * threads * static_cast<double>(iters) * per_iter /
            (ms * 1e-3) / 1e12;
  return CHT_OK;
}

// The best of a small sweep for the engine (chains x CTAs per SM).
int launch_fp64_peak(int engine, cudaStream_t s, double *tflops) {
  double best = 0.0;
  const int chain_set[] = {8, 16, 32};
  const int leaf_set[] = {32, 64};
  const int occ_set[] = {1, 2, 4};
  for (int i = 0; i < (engine == 3 ? 2 : 3); ++i)
    for (int occ : occ_set) {
      double t = 0.0;
      const int ch = engine == 3 ? leaf_set[i] : chain_set[i];
      CHT_TRY(launch_fp64_peak_cfg(engine, ch, engine == 3 ? 128 : 256, occ, s, &t));
      best = std::max(best, t);
    }
  *tflops = best;
  return CHT_OK;
}

}  // namespace cht

// ---------------------------------------------------------------------------
// Allocation-free FP64 multiply (cht_multiply_f64_noalloc in cht.h).
//
// For callers that cannot allocate device memory on the call path.  The only
// scratch the numeric kernel needs -- its 8-byte work counter, which
// cht_multiply takes from the stream-ordered pool on every call -- lives here
// in a file-scope device array instead.  The array's host-side name is only a
// stand-in for the symbol; its device address is looked up once per device
// with cudaGetSymbolAddress and passed to the kernel.
namespace cht {
namespace {
// stated maximum; this call uses 12 bytes: the 8-byte work counter and a
// 4-byte flag for the operand-pattern comparison
constexpr int kNoAllocScratchBytes = 256;
constexpr int kNoAllocMaxDevices = 64;
__device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocScratchBytes / 8];
std::mutex g_noalloc_mutex;
unsigned long long *g_noalloc_ptr[kNoAllocMaxDevices] = {};

int noalloc_scratch(unsigned long long **out) {
  int dev = 0;
  CHT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("device ordinal %d out of range", dev);
    return CHT_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = static_cast<unsigned long long *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return CHT_OK;
}
}  // namespace

}  // namespace cht

extern "C" int cht_multiply_f64_noalloc(cht_plan_t plan, cht_mat_t A, cht_mat_t B, cht_mat_t C,
                                        void *stream) {
  using namespace cht;
  if (!plan || !A || !B || !C) {
    set_error("null plan or matrix handle");
    return CHT_ERR_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long *counter = nullptr;
  CHT_TRY(noalloc_scratch(&counter));
  // operands on other pattern objects are compared with the plan's on the
  // device, the flag in the static array's second word (no allocation)
  CHT_TRY(check_plan_operands(plan, A, B, reinterpret_cast<int *>(counter + 1), s));
  if (C->pat->id != plan->C->id) {
    set_error("C must be a matrix on the plan's product pattern (from cht_multiply or "
              "cht_mat_like of one)");
    return CHT_ERR_INVALID;
  }
  if (plan->C->nnz > 0x7fffffffLL) {
    set_error("%lld output leaves exceed the 2^31 - 1 work units of one call",
              (long long)plan->C->nnz);
    return CHT_ERR_UNSUPPORTED;
  }
  if (plan->b != 32 && plan->b != 64) {
    set_error("leaf size %d: the numeric kernels take b = 32 or b = 64", plan->b);
    return CHT_ERR_UNSUPPORTED;
  }
  if (plan->C->nnz == 0) return CHT_OK;
  int *status = nullptr;
  CHT_TRY(device_status_ptr(&status));
  // the work counter must start at zero; the array keeps the last call's value
  CHT_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
  GemmWork w{};
  w.X = A->values();
  w.Y = B->values();
  w.Z = C->values();
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
  const int engine = g_opt.fp64_engine;
  if (w.b == 64)
    return engine == 1   ? launch_b<64, 2>(w, s, status, counter)
           : engine == 2 ? launch_b<64, 1>(w, s, status, counter)
                         : launch_b<64, 0>(w, s, status, counter);
  return engine ? launch_b<32, 1>(w, s, status, counter) : launch_b<32, 0>(w, s, status, counter);
}

