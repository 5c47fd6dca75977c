// Exclusive prefix sums and a stable LSD radix sort of (uint64 key, int32
// value) pairs: the integer building blocks of the symbolic phase.
//
// Both are single-pass over tiles of 2048 elements with decoupled look-back
// (scan.cuh describes the scheme, its ordering and its bounded waits).  A
// scan is one launch; a sort is one histogram launch for all digit passes and
// one launch per 8-bit pass, each pass publishing and walking back per digit
// in the same way.
#include <algorithm>

#include "scan.cuh"

namespace cht {

namespace {

using namespace scan_detail;

template <class T>
struct ArrayLoad {
  const T *p;
  __device__ int64_t operator()(int64_t i) const { return static_cast<int64_t>(p[i]); }
};

// ------------------------------------------------------------ radix sort --
// Digit counts of every pass at once: hist[p * 256 + d] += the keys whose
// digit p (bits lo + 8p .. lo + 8p + 7) is d.
__global__ void __launch_bounds__(kThreads)
    k_sort_hist(const uint64_t *__restrict__ keys, int64_t n, int npass, int lo,
                unsigned long long *__restrict__ hist) {
  __shared__ unsigned int h[8 * kRadix];
  for (int i = threadIdx.x; i < npass * kRadix; i += kThreads) h[i] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads) {
    const uint64_t k = keys[i];
    for (int p = 0; p < npass; ++p) atomicAdd(&h[p * kRadix + ((k >> (lo + 8 * p)) & 255u)], 1u);
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
  return scan_exclusive_fn(ArrayLoad<int32_t>{in}, n, out, s);
}
int scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  return scan_exclusive_fn(ArrayLoad<int64_t>{in}, n, out, s);
}

int64_t sort_state_words(int64_t n, int nbits, int lo_bit) {
  const int npass = std::min((64 - lo_bit + 7) / 8, std::max(1, (nbits + 7) / 8));
  const int64_t ntiles = (n + kTile - 1) / kTile;
  return npass * kRadix + npass * (1 + ntiles * kRadix);
}

int radix_sort_pairs(const uint64_t *kin, const int32_t *vin, uint64_t *kout, int32_t *vout,
                     int64_t n, int nbits, cudaStream_t s, int lo_bit,
                     unsigned long long *zeroed) {
  if (n <= 0) return CHT_OK;
  if (lo_bit < 0 || lo_bit + nbits > 64) {
    set_error("radix sort on bits %d .. %d of 64-bit keys", lo_bit, lo_bit + nbits - 1);
    return CHT_ERR_INVALID;
  }
  if (n > 0x7fffffffLL) {
    set_error("radix sort of %lld elements: at most 2^31 - 1", (long long)n);
    return CHT_ERR_UNSUPPORTED;
  }
  const int npass = std::min((64 - lo_bit + 7) / 8, std::max(1, (nbits + 7) / 8));
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const int64_t per_pass = 1 + ntiles * kRadix;  // counter + published words
  // one zeroed buffer: the histograms of every pass, then each pass's state
  DevArray<unsigned long long> buf;
  unsigned long long *zb = zeroed;
  if (!zb) {
    CHT_TRY(buf.alloc(npass * kRadix + npass * per_pass, s));
    CHT_CUDA_TRY(cudaMemsetAsync(
        buf.p, 0, sizeof(unsigned long long) * (npass * kRadix + npass * per_pass), s));
    zb = buf.p;
  }
  unsigned long long *hist = zb, *state = zb + npass * kRadix;
  int sms = 0;
  CHT_TRY(num_sms(&sms));
  const int64_t hgrid = std::min<int64_t>(ntiles, 4LL * std::max(sms, 1));
  k_sort_hist<<<static_cast<unsigned>(hgrid), kThreads, 0, s>>>(kin, n, npass, lo_bit, hist);
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
        ksrc, vsrc, kdst, vdst, n, lo_bit + 8 * p, hist + p * kRadix, state + p * per_pass);
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
