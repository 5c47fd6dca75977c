// Exclusive prefix sums and a stable LSD radix sort of (uint64 key, int32
// value) pairs: the integer building blocks of the symbolic phase.
#include <algorithm>

#include "internal.h"

namespace cht {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // 2048 elements per CTA

template <class T>
__device__ T block_exclusive_scan(T v, T *total) {
  __shared__ T warp_sums[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T s = lane < kThreads / 32 ? warp_sums[lane] : T(0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T o = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += o;
    }
    if (lane < kThreads / 32) warp_sums[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  T warp_base = warp ? warp_sums[warp - 1] : T(0);
  *total = warp_sums[kThreads / 32 - 1];
  __syncthreads();
  return warp_base + inc - v;
}

template <class Tin>
__global__ void k_tile_reduce(const Tin *__restrict__ in, int64_t n, int64_t *__restrict__ partial) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  int64_t s = 0;
  for (int i = threadIdx.x; i < kTile; i += kThreads) {
    int64_t idx = base + i;
    if (idx < n) s += static_cast<int64_t>(in[idx]);
  }
  int64_t total;
  block_exclusive_scan<int64_t>(s, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

template <class Tin>
__global__ void k_tile_scan(const Tin *__restrict__ in, int64_t n,
                            const int64_t *__restrict__ tile_off, int64_t *__restrict__ out) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + threadIdx.x * kItems;
  int64_t v[kItems];
  int64_t sum = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    int64_t idx = base + j;
    v[j] = idx < n ? static_cast<int64_t>(in[idx]) : 0;
    sum += v[j];
  }
  int64_t total;
  int64_t run = block_exclusive_scan<int64_t>(sum, &total);
  const int64_t off = tile_off ? tile_off[blockIdx.x] : 0;
  run += off;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    int64_t idx = base + j;
    if (idx < n) out[idx] = run;
    run += v[j];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + total;
}

template <class Tin>
int scan_impl(const Tin *in, int64_t *out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    CHT_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return CHT_OK;
  }
  const int64_t ntiles = (n + kTile - 1) / kTile;
  if (ntiles == 1) {
    k_tile_scan<Tin><<<1, kThreads, 0, s>>>(in, n, nullptr, out);
    return launched("tile_scan");
  }
  DevArray<int64_t> partial, poff;
  CHT_TRY(partial.alloc(ntiles, s));
  CHT_TRY(poff.alloc(ntiles + 1, s));
  k_tile_reduce<Tin><<<static_cast<unsigned>(ntiles), kThreads, 0, s>>>(in, n, partial.p);
  CHT_TRY(launched("tile_reduce"));
  CHT_TRY(scan_impl<int64_t>(partial.p, poff.p, ntiles, s));
  k_tile_scan<Tin><<<static_cast<unsigned>(ntiles), kThreads, 0, s>>>(in, n, poff.p, out);
  return launched("tile_scan");
}

// ------------------------------------------------------------ radix sort --

__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                             int32_t *__restrict__ counts, int64_t ntiles) {
  __shared__ int hist[256];
  hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    int64_t idx = base + it * kThreads + threadIdx.x;
    if (idx < n) atomicAdd(&hist[(keys[idx] >> shift) & 255u], 1);
  }
  __syncthreads();
  counts[static_cast<int64_t>(threadIdx.x) * ntiles + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter: within a tile, elements are ranked in index order (the
// tile is walked in kItems rounds of kThreads consecutive elements; inside a
// round, warps in order, lanes in order).
__global__ void k_radix_scatter(const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin,
                                uint64_t *__restrict__ kout, int32_t *__restrict__ vout,
                                int64_t n, int shift, const int64_t *__restrict__ offs,
                                int64_t ntiles) {
  __shared__ int64_t running[256];
  __shared__ int64_t wpos[kThreads / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  running[tid] = offs[static_cast<int64_t>(tid) * ntiles + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) wpos[w][tid] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  for (int it = 0; it < kItems; ++it) {
    const int64_t idx = base + it * kThreads + tid;
    const bool valid = idx < n;
    const uint64_t key = valid ? kin[idx] : 0;
    const int32_t val = valid ? vin[idx] : 0;
    const unsigned digit = valid ? static_cast<unsigned>((key >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wpos[warp][digit] = __popc(peers);
    __syncthreads();
    int64_t r = running[tid];
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
      int64_t c = wpos[w][tid];
      wpos[w][tid] = r;
      r += c;
    }
    running[tid] = r;
    __syncthreads();
    if (valid) {
      const int64_t pos = wpos[warp][digit] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) wpos[w][tid] = 0;
    __syncthreads();
  }
}

}  // namespace

int scan_exclusive(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  return scan_impl<int32_t>(in, out, n, s);
}
int scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, s);
}

int radix_sort_pairs(const uint64_t *kin, const int32_t *vin, uint64_t *kout, int32_t *vout,
                     int64_t n, int nbits, cudaStream_t s) {
  if (n <= 0) return CHT_OK;
  const int npass = std::max(1, (nbits + 7) / 8);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  DevArray<uint64_t> ktmp;
  DevArray<int32_t> vtmp, counts;
  DevArray<int64_t> offs;
  if (npass > 1) {
    CHT_TRY(ktmp.alloc(n, s));
    CHT_TRY(vtmp.alloc(n, s));
  }
  CHT_TRY(counts.alloc(256 * ntiles, s));
  CHT_TRY(offs.alloc(256 * ntiles + 1, s));
  const uint64_t *ksrc = kin;
  const int32_t *vsrc = vin;
  for (int p = 0; p < npass; ++p) {
    const bool to_out = ((npass - 1 - p) % 2) == 0;
    uint64_t *kdst = to_out ? kout : ktmp.p;
    int32_t *vdst = to_out ? vout : vtmp.p;
    const int shift = 8 * p;
    k_radix_hist<<<static_cast<unsigned>(ntiles), kThreads, 0, s>>>(ksrc, n, shift, counts.p,
                                                                     ntiles);
    CHT_TRY(launched("radix_hist"));
    CHT_TRY(scan_exclusive(counts.p, offs.p, 256 * ntiles, s));
    k_radix_scatter<<<static_cast<unsigned>(ntiles), kThreads, 0, s>>>(ksrc, vsrc, kdst, vdst, n,
                                                                        shift, offs.p, ntiles);
    CHT_TRY(launched("radix_scatter"));
    ksrc = kdst;
    vsrc = vdst;
  }
  return CHT_OK;
}

int read_i64(const int64_t *d, int64_t *h, cudaStream_t s) {
  CHT_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CHT_CUDA_TRY(cudaStreamSynchronize(s));
  return CHT_OK;
}

}  // namespace cht
