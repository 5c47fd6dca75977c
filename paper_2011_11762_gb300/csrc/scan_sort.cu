// Exclusive prefix sums and a stable LSD radix sort of (uint64 key, int32
// value) pairs: the integer building blocks of the symbolic phase.
//
// Both are single-pass over tiles of 2048 elements with decoupled look-back
// (each tile publishes its own total at once and its inclusive prefix as
// soon as it knows it; a tile finds its exclusive prefix by walking back over
// its predecessors' published words, stopping at the first inclusive one).
// A scan is one launch; a sort is one histogram launch for all digit passes
// and one launch per 8-bit pass.  Tiles take their index from a counter in
// the order their CTAs start, so every tile a CTA waits for belongs to a CTA
// that is already running and never waits for a later tile.  The waits are
// still bounded: a tile whose wait runs out computes its prefix directly
// from the input (every element before it), so the result is exact either
// way.
#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace cht {

namespace {

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

template <class T>
__device__ T block_sum(T v) {
  T total;
  block_exclusive_scan<T>(v, &total);
  return total;
}

// Exclusive prefix of tile `tile` from the published words st[0 .. tile),
// walked back by one warp, 32 tiles at a time: *ok false when a word did not
// appear within the budget.  Called by all 32 lanes of one warp; the result
// is valid in every lane.
__device__ int64_t warp_lookback(const unsigned long long *st, int64_t tile, bool *ok) {
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

// ------------------------------------------------------------------ scan --
// state: [0] tile counter, [1 + t] tile t's published word; zeroed per call.
template <class Tin>
__global__ void __launch_bounds__(kThreads)
    k_scan(const Tin *__restrict__ in, int64_t n, int64_t *__restrict__ out,
           unsigned long long *__restrict__ state) {
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
    v[j] = idx < n ? static_cast<int64_t>(in[idx]) : 0;
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
    for (int64_t i = threadIdx.x; i < tile * kTile; i += kThreads)
      part += static_cast<int64_t>(in[i]);
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

template <class Tin>
int scan_impl(const Tin *in, int64_t *out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    CHT_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return CHT_OK;
  }
  const int64_t ntiles = (n + kTile - 1) / kTile;
  DevArray<unsigned long long> state;
  CHT_TRY(state.alloc(ntiles + 1, s));
  CHT_CUDA_TRY(cudaMemsetAsync(state.p, 0, sizeof(unsigned long long) * (ntiles + 1), s));
  k_scan<Tin><<<static_cast<unsigned>(ntiles), kThreads, 0, s>>>(in, n, out, state.p);
  return launched("scan");
}

// ------------------------------------------------------------ radix sort --
// Digit counts of every pass at once: hist[p * 256 + d] += the keys whose
// digit p (bits 8p .. 8p + 7) is d.
__global__ void __launch_bounds__(kThreads)
    k_sort_hist(const uint64_t *__restrict__ keys, int64_t n, int npass,
                unsigned long long *__restrict__ hist) {
  __shared__ unsigned int h[8 * kRadix];
  for (int i = threadIdx.x; i < npass * kRadix; i += kThreads) h[i] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads) {
    const uint64_t k = keys[i];
    for (int p = 0; p < npass; ++p) atomicAdd(&h[p * kRadix + ((k >> (8 * p)) & 255u)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npass * kRadix; i += kThreads)
    if (h[i]) atomicAdd(&hist[i], static_cast<unsigned long long>(h[i]));
}

// One stable pass on the digit at `shift`.  hist: this pass's 256 digit
// counts; state: [0] tile counter, then per tile 256 published words (one per
// digit).  An element lands at (keys of smaller digits) + (keys of its digit
// in earlier tiles) + (its rank among its digit in this tile, in index order:
// the tile is ranked in kItems rounds of kThreads consecutive elements,
// inside a round warps in order, lanes in order).
__global__ void __launch_bounds__(kThreads)
    k_sort_pass(const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin,
                uint64_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t n, int shift,
                const unsigned long long *__restrict__ hist,
                unsigned long long *__restrict__ state) {
  __shared__ int64_t s_tile;
  __shared__ int wcnt[kThreads / 32][kRadix];
  __shared__ int running[kRadix];
  __shared__ int64_t s_base[kRadix];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = static_cast<int64_t>(atomicAdd(&state[0], 1ULL));
  running[tid] = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) wcnt[w][tid] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t base = tile * kTile;
  uint64_t key[kItems];
  int32_t val[kItems];
  unsigned dig[kItems];
  int rank[kItems];
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t idx = base + it * kThreads + tid;
    const bool valid = idx < n;
    key[it] = valid ? kin[idx] : 0;
    val[it] = valid ? vin[idx] : 0;
    dig[it] = valid ? static_cast<unsigned>((key[it] >> shift) & 255u) : 256u;
  }
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const unsigned d = dig[it];
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int r = __popc(peers & ((1u << lane) - 1u));
    if (d < 256u && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    int run = running[tid];
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
      const int c = wcnt[w][tid];
      wcnt[w][tid] = run;
      run += c;
    }
    running[tid] = run;
    __syncthreads();
    rank[it] = d < 256u ? wcnt[warp][d] + r : 0;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
  }
  // this tile's count of digit tid, published; its prefix over earlier tiles
  unsigned long long *st = state + 1;
  const int cnt = running[tid];
  int64_t prefix = 0;
  bool ok = true;
  if (tile == 0) {
    st_word(&st[tid], word(cnt, kInclusive));
  } else {
    st_word(&st[tile * kRadix + tid], word(cnt, kAggregate));
    const uint64_t t0 = global_ns();
    for (int64_t j = tile - 1; j >= 0;) {
      const unsigned long long w = ld_word(&st[j * kRadix + tid]);
      if ((w & 3u) == 0) {
        if (global_ns() - t0 > static_cast<uint64_t>(kLookbackNs)) {
          ok = false;
          break;
        }
        continue;
      }
      prefix += static_cast<int64_t>(w >> 2);
      if ((w & 3u) == kInclusive) break;
      --j;
    }
    if (ok) st_word(&st[tile * kRadix + tid], word(prefix + cnt, kInclusive));
  }
  if (__syncthreads_or(ok ? 0 : 1)) {
    // a predecessor stayed silent: every digit's prefix straight from the
    // keys before this tile
    running[tid] = 0;
    __syncthreads();
    for (int64_t i = tid; i < base; i += kThreads)
      atomicAdd(&running[(kin[i] >> shift) & 255u], 1);
    __syncthreads();
    prefix = running[tid];
    st_word(&st[tile * kRadix + tid], word(prefix + cnt, kInclusive));
  }
  // keys of smaller digits (every tile)
  int64_t total;
  const int64_t below = block_exclusive_scan<int64_t>(static_cast<int64_t>(hist[tid]), &total);
  s_base[tid] = below + prefix;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    if (dig[it] >= 256u) continue;
    const int64_t pos = s_base[dig[it]] + rank[it];
    if (pos < n) {  // (always, unless the keys changed since the histogram)
      kout[pos] = key[it];
      vout[pos] = val[it];
    }
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
  if (n > 0x7fffffffLL) {
    set_error("radix sort of %lld elements: at most 2^31 - 1", (long long)n);
    return CHT_ERR_UNSUPPORTED;
  }
  const int npass = std::min(8, std::max(1, (nbits + 7) / 8));
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const int64_t per_pass = 1 + ntiles * kRadix;  // counter + published words
  // one zeroed buffer: the histograms of every pass, then each pass's state
  DevArray<unsigned long long> buf;
  CHT_TRY(buf.alloc(npass * kRadix + npass * per_pass, s));
  CHT_CUDA_TRY(cudaMemsetAsync(
      buf.p, 0, sizeof(unsigned long long) * (npass * kRadix + npass * per_pass), s));
  unsigned long long *hist = buf.p, *state = buf.p + npass * kRadix;
  int sms = 0;
  CHT_TRY(num_sms(&sms));
  const int64_t hgrid = std::min<int64_t>(ntiles, 4LL * std::max(sms, 1));
  k_sort_hist<<<static_cast<unsigned>(hgrid), kThreads, 0, s>>>(kin, n, npass, hist);
  CHT_TRY(launched("sort_hist"));
  DevArray<uint64_t> ktmp;
  DevArray<int32_t> vtmp;
  if (npass > 1) {
    CHT_TRY(ktmp.alloc(n, s));
    CHT_TRY(vtmp.alloc(n, s));
  }
  const uint64_t *ksrc = kin;
  const int32_t *vsrc = vin;
  for (int p = 0; p < npass; ++p) {
    const bool to_out = ((npass - 1 - p) % 2) == 0;
    uint64_t *kdst = to_out ? kout : ktmp.p;
    int32_t *vdst = to_out ? vout : vtmp.p;
    k_sort_pass<<<static_cast<unsigned>(ntiles), kThreads, 0, s>>>(
        ksrc, vsrc, kdst, vdst, n, 8 * p, hist + p * kRadix, state + p * per_pass);
    CHT_TRY(launched("sort_pass"));
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
