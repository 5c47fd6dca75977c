// Single-pass exclusive scan with decoupled look-back over tiles of 2048
// elements, on any element loader (so that a count computed on the fly
// needs no array and no launch of its own).
//
// Each tile publishes its own total at once and its inclusive prefix as soon
// as it knows it; a tile finds its exclusive prefix by walking back over its
// predecessors' published words, stopping at the first inclusive one.  Tiles
// take their index from a counter in the order their CTAs start, so every
// tile a CTA waits for belongs to a CTA that is already running and never
// waits for a later tile.  The waits are still bounded: a tile whose wait
// runs out computes its prefix directly from the input (every element before
// it), so the result is exact either way.
#pragma once

#include "device.cuh"
#include "internal.h"

namespace cht {
namespace scan_detail {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // 2048 elements per tile
constexpr int kRadix = 256;
constexpr int64_t kLookbackNs = 2000000000LL;  // a predecessor that long silent: compute directly

// A published word: (value << 2) | flag, flag 1 = the tile's own total,
// 2 = its inclusive prefix (the totals of it and every tile before it);
// 0 = nothing yet.  Values are non-negative and below 2^62.
constexpr unsigned long long kAggregate = 1, kInclusive = 2;
__device__ inline unsigned long long ld_word(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void st_word(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ inline unsigned long long word(int64_t value, unsigned long long flag) {
  return (static_cast<unsigned long long>(value) << 2) | flag;
}

template <class T>
__device__ inline T block_exclusive_scan(T v, T *total) {
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

template <class T>
__device__ inline T block_sum(T v) {
  T total;
  block_exclusive_scan<T>(v, &total);
  return total;
}

// Exclusive prefix of tile `tile` from the published words st[0 .. tile),
// walked back by one warp, 32 tiles at a time: *ok false when a word did not
// appear within the budget.  Called by all 32 lanes of one warp; the result
// is valid in every lane.
__device__ inline int64_t warp_lookback(const unsigned long long *st, int64_t tile, bool *ok) {
  const int lane = threadIdx.x & 31;
  int64_t prefix = 0;
  int64_t end = tile - 1;  // lane l examines tile end - l
  const uint64_t t0 = global_ns();
  while (true) {
    const int64_t idx = end - lane;
    unsigned long long w = idx >= 0 ? ld_word(&st[idx]) : word(0, kInclusive);
    while (!__all_sync(0xffffffffu, (w & 3u) != 0)) {
      const bool late = global_ns() - t0 > static_cast<uint64_t>(kLookbackNs);
      if (__any_sync(0xffffffffu, late)) {
        *ok = false;
        return 0;
      }
      if ((w & 3u) == 0) w = ld_word(&st[idx]);
    }
    // the nearest inclusive word ends the walk; lanes up to it contribute
    const unsigned incl = __ballot_sync(0xffffffffu, (w & 3u) == kInclusive);
    const int stop = incl ? __ffs(incl) - 1 : 31;
    int64_t v = lane <= stop ? static_cast<int64_t>(w >> 2) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    prefix += v;
    if (incl) break;
    end -= 32;
  }
  *ok = true;
  return prefix;
}

// state: [0] tile counter, [1 + t] tile t's published word; zeroed per call.
// load(i) gives element i (non-negative) for 0 <= i < n.
template <class Load>
__global__ void __launch_bounds__(kThreads)
    k_scan(Load load, int64_t n, int64_t *__restrict__ out, unsigned long long *__restrict__ state) {
  __shared__ int64_t s_tile, s_prefix;
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_tile = static_cast<int64_t>(atomicAdd(&state[0], 1ULL));
  __syncthreads();
  const int64_t tile = s_tile;
  unsigned long long *st = state + 1;
  const int64_t base = tile * kTile + threadIdx.x * kItems;
  int64_t v[kItems];
  int64_t sum = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t idx = base + j;
    v[j] = idx < n ? load(idx) : 0;
    sum += v[j];
  }
  int64_t total;
  int64_t run = block_exclusive_scan<int64_t>(sum, &total);
  if (threadIdx.x < 32) {
    if (tile == 0) {
      if (threadIdx.x == 0) {
        st_word(&st[0], word(total, kInclusive));
        s_prefix = 0;
        s_ok = 1;
      }
    } else {
      if (threadIdx.x == 0) st_word(&st[tile], word(total, kAggregate));
      bool ok;
      const int64_t prefix = warp_lookback(st, tile, &ok);
      if (threadIdx.x == 0) {
        s_prefix = prefix;
        s_ok = ok ? 1 : 0;
        if (ok) st_word(&st[tile], word(prefix + total, kInclusive));
      }
    }
  }
  __syncthreads();
  if (!s_ok) {
    // a predecessor stayed silent: the prefix straight from the input
    int64_t part = 0;
    for (int64_t i = threadIdx.x; i < tile * kTile; i += kThreads) part += load(i);
    const int64_t prefix = block_sum<int64_t>(part);
    if (threadIdx.x == 0) {
      s_prefix = prefix;
      st_word(&st[tile], word(prefix + total, kInclusive));
    }
    __syncthreads();
  }
  run += s_prefix;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t idx = base + j;
    if (idx < n) out[idx] = run;
    run += v[j];
  }
  if (threadIdx.x == 0 && (tile + 1) * kTile >= n) out[n] = s_prefix + total;
}

}  // namespace scan_detail

// Words of zeroed state a scan of n elements uses.
inline int64_t scan_state_words(int64_t n) {
  return (n + scan_detail::kTile - 1) / scan_detail::kTile + 1;
}

// out[0..n] = exclusive prefix sums of load(0 .. n), out[n] = the total.
// `zeroed`: scan_state_words(n) words of zeroed device memory for its state
// (used up by the call), or null to allocate and clear them here.
template <class Load>
int scan_exclusive_fn(Load load, int64_t n, int64_t *out, cudaStream_t s,
                      unsigned long long *zeroed = nullptr) {
  using namespace scan_detail;
  if (n <= 0) {
    CHT_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return CHT_OK;
  }
  const int64_t ntiles = (n + kTile - 1) / kTile;
  DevArray<unsigned long long> state;
  unsigned long long *st = zeroed;
  if (!st) {
    CHT_TRY(state.alloc(ntiles + 1, s));
    CHT_CUDA_TRY(cudaMemsetAsync(state.p, 0, sizeof(unsigned long long) * (ntiles + 1), s));
    st = state.p;
  }
  k_scan<Load><<<static_cast<unsigned>(ntiles), kThreads, 0, s>>>(load, n, out, st);
  return launched("scan");
}

}  // namespace cht
