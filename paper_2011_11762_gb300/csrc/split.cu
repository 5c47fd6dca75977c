// Split-precision numeric phase (step S7): C = A*B with FP64 operands split
// into bfloat16 digit slices, slice products on the tcgen05 tensor cores
// (kind::f16, FP32 accumulation in TMEM), and an integer recombination.
//
// Splitting (error-free transformation in the style of Ozaki, Ogita, Oishi
// and Rump, Numer. Algorithms 59, 2012): with e_r the frexp exponent of the
// largest |a| in global row r of A (max < 2^e_r) and f_c that of column c of
// B, X = round(a_rk 2^(47 - e_r)) has |X| <= 2^47 and balanced signed base-256
// digits, so
//     a_rk = 2^(e_r+1) * sum_i d_i 2^(-8i),   b_kc = 2^(f_c+1) * sum_j g_j 2^(-8j)
// up to the rounding after the last digit, with |d|, |g| <= 128 (exact in
// bfloat16; a digit product is at most 2^14).  The line exponents are stored
// as e_r + 1 and f_c + 1.  Then
//     C_rc = 2^(e_r + f_c + 2) * sum_t S_t 2^(-8t),   S_t = sum_{i+j=t} sum_k d_i g_j,
// and every S_t is an integer.  Slice pairs with i + j > 7 are dropped (their
// weight is below the 48-bit rounding).
//
// Tensor-core mapping (one CTA per C leaf at a time; b = 64 shown, b = 32 in
// brackets): the A operand of an MMA stacks 2 [4] consecutive slices of the
// A leaf along M = 128, the B operand puts 2 consecutive slices of the B leaf
// side by side (N = 2b).  A block with first slices u, j (both odd) computes
// A_{u+p} B_{j+q} for parts p (rows p*b ..) and column halves q (columns
// q*b ..): diagonal u + j + p + q.  Blocks with equal u + j share TMEM region
// r = (u + j - 2) / 2, so every quadrant of a region holds one diagonal.
//
// Exactness: regions r = 0, 1 (diagonals 2..5 and the parts above them)
// carry the high bits and must be exact.  An FP32 accumulator is exact while
// every partial sum stays at most 2^24, which holds for a window of 8 [32]
// leaf pairs: 2 blocks * 64 * 8 * 2^14 = 2^24 [1 * 32 * 32 * 2^14 = 2^24].  After
// each window the epilogue warps read these regions and add them, converted
// to integers, into int64 accumulators; the next window restarts them.
// Region 2 (weight <= 2^-32 of the leading diagonal) accumulates over the
// whole C leaf in FP32 and is read once.  The final value
//     T = sum_parts (2^8 Q_p + rnd(2^8 (R6 2^-8 + R7 2^-16))) 2^(-8p)
// is an integer in units of 2^-48 of 2^(e_r + f_c + 2); every part and the
// sum are at most K (128/255)^2 2^48 < 2^63 for the unit sizes allowed, so
// the recombination is int64 and the double comes from bit assembly; no
// FP64 arithmetic is used (FP64 is the slowest unit on GB300).
//
// Roles (320 threads): warp 0 = bulk-copy producer, warp 1 = TMEM owner and
// MMA issuer (one thread), warps 2..9 = epilogue (two warps per TMEM lane
// quarter, splitting the columns).  Units are the C leaves in Morton order,
// taken from an atomic counter by the persistent CTAs a chunk at a time (2
// units in the kernel for 64-leaves, 32 in the 32-leaf kernel), so
// neighbouring leaves run together and share their A and B slices through
// L2.  A C leaf with more pairs than a unit may sum is cut into
// pieces added afterwards in FP64.  Every wait is bounded.
#include <algorithm>

#include "device.cuh"
#include "internal.h"
#include "scan.cuh"

namespace cht {

namespace {

constexpr int kW = 8;               // bits per digit
constexpr int kSB = 6;              // B slices (and the split depth s)
constexpr int kRegions = 3;         // TMEM region r holds base diagonal t = 2 + 2r
constexpr int kExactRegions = 2;    // regions with t = 2 and t = 4 are exact
constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int64_t kDrainNs = 2000000000LL;

template <int B>
struct Cfg;
template <>
struct Cfg<64> {
  // N is the MMA width: two B slices side by side (2 b columns)
  static constexpr int N = 128, PARTS = 2, SA = 6, KSTEPS = 4, WINDOW = 8;
};
template <>
struct Cfg<32> {
  static constexpr int N = 64, PARTS = 4, SA = 8, KSTEPS = 2, WINDOW = 32;
};

// MMA blocks (first stacked A slice u, first B slice j; both odd), 1-based.
// Block (u, j) computes A_{u+p} B_{j+q} for every part p and q in {0, 1}
// into TMEM region (u + j - 2) / 2.
template <int B>
struct Blocks;
template <>
struct Blocks<64> {
  static constexpr int NBLK = 6;  // (1,1) (1,3) (3,1) (1,5) (3,3) (5,1)
  __device__ static constexpr int u(int i) { return i <= 1 || i == 3 ? 1 : i == 5 ? 5 : 3; }
  __device__ static constexpr int j(int i) { return i == 0 || i == 2 || i == 5 ? 1 : i == 3 ? 5 : 3; }
};
template <>
struct Blocks<32> {
  static constexpr int NBLK = 4;  // (1,1) (1,3) (1,5) (5,1)
  __device__ static constexpr int u(int i) { return i == 3 ? 5 : 1; }
  __device__ static constexpr int j(int i) { return i == 0 || i == 3 ? 1 : i == 1 ? 3 : 5; }
};

template <int B>
struct Smem {
  // one slice: B rows of B bf16 values (K-major): 128-byte rows with the
  // 128-byte swizzle at b = 64, 64-byte rows with the 64-byte swizzle at b = 32
  static constexpr int TILE = B * B * 2;
  static constexpr int A_BYTES = Cfg<B>::SA * TILE;
  static constexpr int B_BYTES = kSB * TILE;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  // exchange buffer: b = 64 hands part 1 to part 0; b = 32 gathers all 4 parts
  static constexpr int XBUF = (B == 64 ? 1 : Cfg<B>::PARTS) * B * B * 8;
};

// ------------------------------------------------------------ tcgen05 PTX --
__device__ inline void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ inline void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ inline void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ inline void tc_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}
__device__ inline void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                              uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ inline void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 lanes x 32 consecutive 32-bit columns (one column block per thread).
__device__ inline void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ inline void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ inline void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
template <int E>
__device__ inline void tmem_ld(uint32_t taddr, float (&v)[E]);
template <>
__device__ inline void tmem_ld<32>(uint32_t taddr, float (&v)[32]) { tmem_ld32(taddr, v); }
template <>
__device__ inline void tmem_ld<16>(uint32_t taddr, float (&v)[16]) { tmem_ld16(taddr, v); }

// 32 lanes x 16 columns, raw 32-bit words (load / store).
__device__ inline void tmem_ld16u(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ inline void tmem_st16u(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ inline void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle
// layout (rows of 128 bytes, 8-row groups 1024 bytes apart).
__device__ inline uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3ffff) >> 4);  // start address
  d |= static_cast<uint64_t>(1) << 16;                 // leading offset (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;         // stride: 8-row group pitch
  d |= static_cast<uint64_t>(1) << 46;                 // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                 // 128-byte swizzle
  return d;
}
// The same for the 64-byte swizzle layout (rows of 64 bytes, 8-row groups
// 512 bytes apart): the tiles of 32-leaves, whose rows hold 32 bf16 values.
__device__ inline uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3ffff) >> 4);  // start address
  d |= static_cast<uint64_t>(1) << 16;                 // leading offset (unused here)
  d |= static_cast<uint64_t>(512 >> 4) << 32;          // stride: 8-row group pitch
  d |= static_cast<uint64_t>(1) << 46;                 // descriptor version
  d |= static_cast<uint64_t>(4) << 61;                 // 64-byte swizzle
  return d;
}
template <int B>
__device__ inline uint64_t tile_desc(uint32_t saddr) {
  return B == 64 ? sw128_desc(saddr) : sw64_desc(saddr);
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

// Bounded mbarrier wait that also gives up when another role aborted.
__device__ inline bool wait_or_abort(uint64_t *bar, uint32_t parity, int64_t budget_ns,
                                     volatile int *abort_flag) {
  if (budget_ns <= 0) return false;
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (global_ns() - t0 > static_cast<uint64_t>(budget_ns)) return false;
  }
}

// The same wait for a whole warp, with one outcome for all its lanes: every
// lane polls, and the warp goes on only if every lane saw the phase complete.
// The epilogue's tcgen05.ld / st / wait instructions are .sync.aligned (all 32
// lanes must execute them together), so a warp must not split between lanes
// that saw the phase and lanes that saw the abort flag or the deadline.
__device__ inline bool warp_wait_or_abort(uint64_t *bar, uint32_t parity, int64_t budget_ns,
                                          volatile int *abort_flag) {
  const bool ok = wait_or_abort(bar, parity, budget_ns, abort_flag);
  return __all_sync(0xffffffffu, ok);
}

// -------------------------------------------------------- digits / scale --
// The "no exponent" marker (all-zero line); also the byte-0x80 memset value.
constexpr int kNoExp = static_cast<int>(0x80808080u);

// frexp exponent (x in [2^(e-1), 2^e)) from the bits; kNoExp for zero.
__device__ inline int exp_of(double x) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const int biased = static_cast<int>((bits >> 52) & 0x7ff);
  const unsigned long long mant = bits & ((1ULL << 52) - 1);
  if (biased) return biased - 1022;
  if (!mant) return kNoExp;
  return (64 - __clzll(static_cast<long long>(mant))) - 1074;
}

// Magnitude of round(|x| * 2^(nbits - e)) (halves rounded up) and the sign of
// x; e is a stored line exponent (frexp exponent + 1), so the result is at
// most 2^(nbits - 1).
__device__ inline unsigned long long fixed_mag(double x, int e, int nbits, bool *neg) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  *neg = (bits >> 63) != 0;
  const int biased = static_cast<int>((bits >> 52) & 0x7ff);
  unsigned long long mant = bits & ((1ULL << 52) - 1);
  int ex;
  if (biased) {
    mant |= 1ULL << 52;
    ex = biased - 1075;
  } else {
    ex = -1074;
  }
  if (!mant || e == kNoExp) return 0;
  const int sh = ex + nbits - e;
  if (sh >= 0) return mant << sh;  // exact; sh <= nbits - 54
  if (sh <= -55) return 0;         // |x| 2^(nbits-e) < 2^53 2^-55 < 1/2
  return (mant + (1ULL << (-sh - 1))) >> (-sh);
}

// Balanced base-256 digits of a magnitude m <= 2^(8n - 1), least significant
// first: t = ((m + 127) mod 256) - 127, m <- (m - t) / 256, so each digit is
// in [-127, 128] and, with the sign applied, |digit| <= 128.  The recurrence
// runs on 24-bit chunks of m in 32-bit arithmetic: after the three digits of
// a chunk the running value is the carry (0 or 1) into the next chunk.
template <int NDIG>
__device__ inline void balanced_digits(unsigned long long m, bool neg, int (&out)[NDIG]) {
  int v = 0, carry = 0;
#pragma unroll
  for (int g = 0; g < NDIG; ++g) {
    if (g % 3 == 0) v = static_cast<int>((m >> (kW * g)) & 0xffffffULL) + carry;
    const int t = ((v + 127) & 0xff) - 127;
    out[NDIG - 1 - g] = neg ? -t : t;
    v = (v - t) >> kW;
    if (g % 3 == 2) carry = v;
  }
}

// Two integers |t| <= 256 as a bfloat16 pair (both exact in bfloat16).  The
// float with bits 0x4B400000 + t is 1.5 * 2^23 + t, so subtracting 1.5 * 2^23
// gives t exactly; its bfloat16 is the upper half of its bits.  Integer adds,
// one float add and a byte permute replace the slower int-to-float
// conversions.
__device__ inline uint32_t pack_bf16x2(int lo, int hi) {
  const float fl = __int_as_float(0x4B400000 + lo) - 12582912.0f;
  const float fh = __int_as_float(0x4B400000 + hi) - 12582912.0f;
  return __byte_perm(__float_as_uint(fl), __float_as_uint(fh), 0x7632);
}

// Byte offset of logical 16-byte chunk c of row r in a 128-byte-swizzled tile.
__host__ __device__ inline int sw128_offset(int r, int c) {
  return (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4);
}
// The same in a 64-byte-swizzled tile (c < 4): the swizzle XORs the chunk
// index with bits 7 and 8 of the row's byte offset, i.e. with (r >> 1) & 3.
__host__ __device__ inline int sw64_offset(int r, int c) {
  return (r >> 3) * 512 + (r & 7) * 64 + ((c ^ ((r >> 1) & 3)) << 4);
}
// Byte offset of 16-byte chunk c of row r in a slice tile of a b-leaf.
template <int B>
__host__ __device__ inline int tile_offset(int r, int c) {
  return B == 64 ? sw128_offset(r, c) : sw64_offset(r, c);
}

// v * 2^e2 rounded to nearest-even with 64-bit integer operations, |v| < 2^63.
// Outside the normal range of doubles (never for finite inputs of moderate
// range) it falls back to a conversion and ldexp.
__device__ inline double scaled_i64_to_double(long long v, int e2) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? (1ULL << 63) : 0ULL;
  const unsigned long long m = v < 0 ? 0ULL - static_cast<unsigned long long>(v)
                                     : static_cast<unsigned long long>(v);
  int top = 63 - __clzll(static_cast<long long>(m));
  unsigned long long mant;
  const int sh = top - 52;
  if (sh > 0) {
    const unsigned long long rem = m & ((1ULL << sh) - 1ULL), half = 1ULL << (sh - 1);
    mant = m >> sh;
    if (rem > half || (rem == half && (mant & 1ULL))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++top;
      }
    }
  } else {
    mant = m << (-sh);
  }
  const int biased = top + e2 + 1023;
  if (biased <= 0 || biased >= 2047) return ldexp(static_cast<double>(v), e2);
  return __longlong_as_double(static_cast<long long>(
      sgn | (static_cast<unsigned long long>(biased) << 52) | (mant & ((1ULL << 52) - 1))));
}

// The same rounding without branches, in few 32-bit integer operations (the
// FP64 pipe, which a double conversion or multiply would use, is narrow).
// |v| is normalised so that its leading one sits at bit 63 of the word pair
// (hi, lo) -- from the high word when it is non-zero, else from the low one
// -- so that hi and the top 21 bits of lo are the 53-bit significand and the
// low 11 bits of lo decide round-to-nearest-even; adding the significand
// (leading one included) to (exponent - 1) << 52 lets a rounding carry move
// into the exponent.  *ok is false when the result could leave the normal
// range of doubles, and the caller then uses scaled_i64_to_double.  |v| <
// 2^63; v == 0 gives +0 with *ok true (e2 unused); where *ok holds the result
// is bit for bit that of scaled_i64_to_double.
__device__ __forceinline__ double scaled_i64_fast(long long v, int e2, bool *ok) {
  const unsigned long long s = static_cast<unsigned long long>(v >> 63);  // 0 or all ones
  const unsigned long long m = (static_cast<unsigned long long>(v) ^ s) - s;
  const uint32_t mh = static_cast<uint32_t>(m >> 32), ml = static_cast<uint32_t>(m);
  const bool big = mh != 0;
  const uint32_t wh = big ? mh : ml, wl = big ? ml : 0u;
  const int lz = __clz(static_cast<int>(wh));  // 32 when v == 0
  const uint32_t nh = __funnelshift_l(wl, wh, lz), nl = wl << (lz & 31);
  const uint32_t sig_h = nh >> 11, sig_l = __funnelshift_r(nl, nh, 11);
  const uint32_t up = ((nl & 0x7ffu) + (sig_l & 1u) + 0x3ffu) >> 11;
  // exponent field before a rounding carry (unsigned: e2 may be a sentinel
  // when v == 0)
  const uint32_t biased = static_cast<uint32_t>(e2) + (big ? 1086u : 1054u) -
                          static_cast<uint32_t>(lz);
  *ok = wh == 0 || biased - 1u < 2045u;
  const unsigned long long sig = (static_cast<unsigned long long>(sig_h) << 32) | sig_l;
  const unsigned long long bits =
      (static_cast<unsigned long long>((biased - 1u) & 0x7ffu) << 52) + sig + up;
  return wh == 0 ? 0.0 : __longlong_as_double(static_cast<long long>(bits | (s << 63)));
}

// ------------------------------------------------------------ pre-kernels --

// Row exponents of A (stored as frexp exponent + 1): B/16 consecutive
// threads per (leaf, row), 16 consecutive values (eight 16-byte loads) each.
template <int B>
__global__ void k_row_exp(const double *__restrict__ vals, const int32_t *__restrict__ brow,
                          int64_t nleaves, int *__restrict__ row_exp) {
  constexpr int TPR = B / 16;  // threads per row (a power of two dividing 32)
  const int64_t total = nleaves * B * TPR;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t leaf = t / (B * TPR);
    const int r = static_cast<int>((t / TPR) % B), part = static_cast<int>(t % TPR);
    const double2 *src =
        reinterpret_cast<const double2 *>(vals + leaf * B * B + static_cast<int64_t>(r) * B + part * 16);
    int e = kNoExp;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double2 v = src[k];
      e = max(e, max(exp_of(v.x), exp_of(v.y)));
    }
    // the row's threads are consecutive lanes of one warp (total is a
    // multiple of 32, so every lane of a live warp takes part)
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (part == 0 && e != kNoExp)
      atomicMax(&row_exp[static_cast<int64_t>(brow[leaf]) * B + r], e + 1);
  }
}

// Column exponents of B (frexp exponent + 1): thread per (leaf, column);
// consecutive threads read consecutive columns, 16 rows in flight.
template <int B>
__global__ void k_col_exp(const double *__restrict__ vals, const int32_t *__restrict__ bcol,
                          int64_t nleaves, int *__restrict__ col_exp) {
  const int64_t total = nleaves * B;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t leaf = t / B;
    const int c = static_cast<int>(t % B);
    const double *col = vals + leaf * B * B + c;
    int e = kNoExp;
#pragma unroll 16
    for (int k = 0; k < B; ++k) e = max(e, exp_of(col[static_cast<int64_t>(k) * B]));
    if (e != kNoExp) atomicMax(&col_exp[static_cast<int64_t>(bcol[leaf]) * B + c], e + 1);
  }
}

// A slices: thread per (leaf, row r, chunk c of 8 K values).  Leaf layout in
// global memory = the shared-memory image: [SA][B rows][2 B bytes], swizzled
// (128-byte swizzle at b = 64, 64-byte swizzle at b = 32).
template <int B, int SA>
__global__ void k_split_a(const double *__restrict__ vals, const int32_t *__restrict__ brow,
                          int64_t nleaves, const int *__restrict__ row_exp,
                          uint8_t *__restrict__ out) {
  constexpr int CH = B / 8;  // logical chunks per row holding data
  constexpr int TILE = Smem<B>::TILE;
  const int64_t total = nleaves * B * CH;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t leaf = t / (B * CH);
    const int r = static_cast<int>((t / CH) % B), c = static_cast<int>(t % CH);
    const int e = row_exp[static_cast<int64_t>(brow[leaf]) * B + r];
    const double2 *src =
        reinterpret_cast<const double2 *>(vals + leaf * B * B + static_cast<int64_t>(r) * B + c * 8);
    double x[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 v = src[k];
      x[2 * k] = v.x;
      x[2 * k + 1] = v.y;
    }
    int d[SA][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      bool neg;
      const unsigned long long mag = fixed_mag(x[k], e, SA * kW, &neg);
      int dk[SA];
      balanced_digits<SA>(mag, neg, dk);
#pragma unroll
      for (int i = 0; i < SA; ++i) d[i][k] = dk[i];
    }
    uint8_t *base = out + leaf * SA * TILE + tile_offset<B>(r, c);
#pragma unroll
    for (int i = 0; i < SA; ++i) {
      uint4 v;
      v.x = pack_bf16x2(d[i][0], d[i][1]);
      v.y = pack_bf16x2(d[i][2], d[i][3]);
      v.z = pack_bf16x2(d[i][4], d[i][5]);
      v.w = pack_bf16x2(d[i][6], d[i][7]);
      *reinterpret_cast<uint4 *>(base + i * TILE) = v;
    }
  }
}

// B slices, stored transposed (tile row n = column n of the leaf, K-major).
// One block per leaf: the leaf is staged in shared memory with contiguous
// 16-byte loads; thread (column n, chunk c of 8 K values) reads its column
// from shared memory (consecutive threads: consecutive columns, no bank
// conflicts) and writes its 16-byte chunk of every digit plane into a
// shared-memory image of the leaf's slice tiles, which the block then stores
// with contiguous 16-byte writes.
template <int B>
struct SplitBSmem {
  static constexpr int IN = B * (B + 1) * 8;  // the staged leaf (padded rows)
  static constexpr int OUT = kSB * Smem<B>::TILE;  // the slice tiles of one leaf
  static constexpr int TOTAL = IN + OUT;
  static_assert(IN % 16 == 0 && OUT % 16 == 0, "16-byte aligned parts");
};

template <int B>
__global__ void __launch_bounds__(256) k_split_b(const double *__restrict__ vals,
                                                 const int32_t *__restrict__ bcol,
                                                 int64_t nleaves, const int *__restrict__ col_exp,
                                                 uint8_t *__restrict__ out) {
  constexpr int TILE = Smem<B>::TILE;
  constexpr int OUT = SplitBSmem<B>::OUT;
  extern __shared__ __align__(16) uint8_t smem_b[];
  double(*tile)[B + 1] = reinterpret_cast<double(*)[B + 1]>(smem_b);
  uint8_t *img = smem_b + SplitBSmem<B>::IN;
  for (int64_t leaf = blockIdx.x; leaf < nleaves; leaf += gridDim.x) {
    const double2 *src = reinterpret_cast<const double2 *>(vals + leaf * B * B);
    for (int i = threadIdx.x; i < B * B / 2; i += blockDim.x) {
      const double2 v = src[i];
      const int e = 2 * i;
      tile[e / B][e % B] = v.x;
      tile[e / B][e % B + 1] = v.y;
    }
    // reads of the previous leaf's image ended before every thread got here
    __syncthreads();
    const int64_t col0 = static_cast<int64_t>(bcol[leaf]) * B;
    // work items of KV K values of one column: 8 (a 16-byte chunk) at
    // b = 64, 4 (half a chunk) at b = 32, so that all 256 threads have one
    constexpr int KV = B == 32 ? 4 : 8;
    for (int q = threadIdx.x; q < B * (B / KV); q += blockDim.x) {
      const int n = q % B, c = q / B;  // column, item (K values c*KV ..)
      const int f = col_exp[col0 + n];
      int g[kSB][KV];
#pragma unroll
      for (int k = 0; k < KV; ++k) {
        bool neg;
        const unsigned long long mag = fixed_mag(tile[c * KV + k][n], f, kSB * kW, &neg);
        int gk[kSB];
        balanced_digits<kSB>(mag, neg, gk);
#pragma unroll
        for (int j = 0; j < kSB; ++j) g[j][k] = gk[j];
      }
      uint8_t *base = img + tile_offset<B>(n, c * KV / 8) + (c * KV % 8) * 2;
#pragma unroll
      for (int j = 0; j < kSB; ++j) {
        if constexpr (KV == 8) {
          uint4 v;
          v.x = pack_bf16x2(g[j][0], g[j][1]);
          v.y = pack_bf16x2(g[j][2], g[j][3]);
          v.z = pack_bf16x2(g[j][4], g[j][5]);
          v.w = pack_bf16x2(g[j][6], g[j][7]);
          *reinterpret_cast<uint4 *>(base + j * TILE) = v;
        } else {
          uint2 v;
          v.x = pack_bf16x2(g[j][0], g[j][1]);
          v.y = pack_bf16x2(g[j][2], g[j][3]);
          *reinterpret_cast<uint2 *>(base + j * TILE) = v;
        }
      }
    }
    // the image is complete, and the staged leaf is no longer read
    __syncthreads();
    uint4 *dst = reinterpret_cast<uint4 *>(out + leaf * OUT);
    const uint4 *from = reinterpret_cast<const uint4 *>(img);
    for (int i = threadIdx.x; i < OUT / 16; i += blockDim.x) dst[i] = from[i];
  }
}

// ------------------------------------------------------------ main kernel --

// One product as the split kernel sees it.
struct SplitProd {
  const uint8_t *a_slices;  // [nA][SA][tile], tiles in the shared-memory image
  const uint8_t *b_slices;  // [nB][6][tile]
  const int32_t *pa;        // per pair: A leaf (pairs sorted by C leaf, then K)
  const int32_t *pb;        // per pair: B leaf
  const int64_t *cseg;      // per C leaf: pair segment
  const int32_t *crow;
  const int32_t *ccol;
  const int *row_exp;
  const int *col_exp;
  double *C;
  double *const *cptr;      // per unit: output leaf (null: C + unit * b * b)
  int32_t b;
  int32_t pad;
  // lengths (read by the bounds-checked build): A and B leaves, units (the
  // entries of cseg less one), pairs, leaves per side
  int64_t nA, nB, nunits, npairs, G;
};

// Kernel-wide sizes for the largest leaf size a launch serves.
template <int MAXB>
struct KCfg;
template <>
struct KCfg<64> {
  static constexpr int STAGES = 2, STAGE = Smem<64>::STAGE, XBUF = Smem<64>::XBUF, NXB = 1;
  static constexpr int TMEM_COLS = 512;
  static constexpr int CHUNK = 2;  // units taken from the counter at a time
};
template <>
struct KCfg<32> {
  // 4 stages of 28 KB (8 A + 6 B tiles of 2 KB): one-pair units need the
  // copies of several units in flight to hide their latency
  static constexpr int STAGES = 4, STAGE = Smem<32>::STAGE, XBUF = Smem<32>::XBUF, NXB = 2;
  // two accumulator sets of 256 columns: the MMA of unit n + 1 runs while
  // the epilogue still reads unit n
  static constexpr int TMEM_COLS = 512;
  // 32-leaf products often have one or two pairs per C leaf: the producer
  // resolves 32 units at once so their metadata loads overlap
  static constexpr int CHUNK = 32;
};

// One entry of the per-CTA unit queue: a C leaf and everything the MMA and
// epilogue warps need about it, staged in shared memory by the producer.
constexpr int kQueue = 4;
constexpr int16_t kNoExp16 = -32768;
struct alignas(16) Slot {
  double *C;          // the C leaf's values
  int32_t np;         // its leaf pairs
  int32_t b;          // leaf size (0 = no more units)
  int32_t u;          // position in this CTA's unit sequence
  int32_t pad;
  int16_t rexp[64];   // exponents of the leaf's rows of A (kNoExp16: none)
  int16_t cexp[64];   // exponents of the leaf's columns of B
};

template <int MAXB>
constexpr size_t kernel_smem() {
  return static_cast<size_t>(KCfg<MAXB>::STAGES) * KCfg<MAXB>::STAGE +
         KCfg<MAXB>::NXB * KCfg<MAXB>::XBUF + kQueue * sizeof(Slot) + 256 + 1024;
}

// Per-CTA control block (pointers into shared memory).
struct Ctl {
  uint8_t *stage_base;
  int stage_bytes;
  int64_t *xbuf;
  int xbuf_bytes;
  Slot *queue;
  uint64_t *full, *empty, *acc_full, *acc_empty, *drain, *ep_bar, *qfull, *qempty;
  volatile int *abort_flag;
  uint32_t tmem;
  int64_t wait_ns;
};

__device__ inline int16_t exp16(int e) {
  return e == kNoExp ? kNoExp16 : static_cast<int16_t>(max(-32000, min(32000, e)));
}

// One MMA over all K-steps of a leaf pair: A slices u, u + 1 (M = 128) and
// the nb B slices from j on (N = b nb), into TMEM column 64 (u + j - 2); the
// first K-step overwrites when `start`.  (Column block c of the accumulator
// holds diagonal c + 2 + part, so the B slices side by side land on their
// diagonals' blocks.)
template <int NB>
__device__ __forceinline__ void mma64(uint32_t sa, uint32_t sb, uint32_t tmem, int u, int j,
                                      bool start) {
  constexpr uint32_t IDESC = make_idesc(128, 64 * NB);
  const uint64_t ad = tile_desc<64>(sa + (u - 1) * Smem<64>::TILE);
  const uint64_t bd = tile_desc<64>(sb + (j - 1) * Smem<64>::TILE);
  const uint32_t dt = tmem + static_cast<uint32_t>(64 * (u + j - 2));
#pragma unroll
  for (int kk = 0; kk < Cfg<64>::KSTEPS; ++kk)
    tc_mma(dt, ad + 2 * kk, bd + 2 * kk, IDESC, (start && kk == 0) ? 0u : 1u);
}

// The MMA blocks of one leaf pair from stage (sa: A slices, sb: B slices).
// which = 0: all blocks; 1: the blocks of region 2 only; 2: regions 0, 1.
// At b = 64 the slice products are issued as wide MMAs over B slices side
// by side: (A1,2 x B5,6), (A1,2 x B1..4), (A3,4 x B1..4), (A5,6 x B1,2) for
// all regions -- 4 MMAs per K-step instead of 6 blocks, the same 24 slice
// products, each region first written with overwrite -- and, when only one
// side may go (the look-ahead of region 2 before the exact regions are
// released), (A1,2 x B5,6), (A3,4 x B3,4), (A5,6 x B1,2) for region 2 and
// (A1,2 x B1..4), (A3,4 x B1,2) for regions 0, 1.
template <int B>
__device__ __forceinline__ void issue_blocks(uint32_t sa, uint32_t sb, uint32_t tmem,
                                             bool (&fresh)[kRegions], int which) {
  if constexpr (B == 64) {
    if (which == 0) {
      mma64<2>(sa, sb, tmem, 1, 5, fresh[2]);
      mma64<4>(sa, sb, tmem, 1, 1, fresh[0]);
      mma64<4>(sa, sb, tmem, 3, 1, false);
      mma64<2>(sa, sb, tmem, 5, 1, false);
      fresh[0] = fresh[1] = fresh[2] = false;
    } else if (which == 1) {
      mma64<2>(sa, sb, tmem, 1, 5, fresh[2]);
      mma64<2>(sa, sb, tmem, 3, 3, false);
      mma64<2>(sa, sb, tmem, 5, 1, false);
      fresh[2] = false;
    } else {
      mma64<4>(sa, sb, tmem, 1, 1, fresh[0]);
      mma64<2>(sa, sb, tmem, 3, 1, false);
      fresh[0] = fresh[1] = false;
    }
    return;
  }
  using CF = Cfg<B>;
  using SM = Smem<B>;
  constexpr int N = CF::N;
  constexpr uint32_t IDESC = make_idesc(128, N);
#pragma unroll
  for (int bi = 0; bi < Blocks<B>::NBLK; ++bi) {
    const int bu = Blocks<B>::u(bi), bj = Blocks<B>::j(bi);
    const int r = (bu + bj - 2) >> 1;  // region 0..2
    if ((which == 1 && r != 2) || (which == 2 && r == 2)) continue;
    const uint64_t ad = tile_desc<B>(sa + (bu - 1) * SM::TILE);
    const uint64_t bd = tile_desc<B>(sb + (bj - 1) * SM::TILE);  // slices j, j+1
    const uint32_t dt = tmem + static_cast<uint32_t>(r * N);
#pragma unroll
    for (int kk = 0; kk < CF::KSTEPS; ++kk) {
      const uint32_t acc = (fresh[r] && kk == 0) ? 0u : 1u;
      tc_mma(dt, ad + 2 * kk, bd + 2 * kk, IDESC, acc);
    }
    fresh[r] = false;
  }
}

// MMA issuer: all slice-product blocks of one C leaf, window by window.
// Region 2 is not read between windows, so from the second window of a unit
// on, the first pair's region-2 blocks go out before the wait for the
// epilogue to release the exact regions: they cover that hand-off.
template <int B, int S>
__device__ bool mma_unit(int64_t np, uint32_t &k, uint32_t &win, const Ctl &c, uint32_t tmem,
                         uint64_t *acc_full, uint64_t *acc_empty) {
  using CF = Cfg<B>;
  using SM = Smem<B>;
  bool fresh[kRegions];
#pragma unroll
  for (int r = 0; r < kRegions; ++r) fresh[r] = true;
  for (int64_t w0 = 0; w0 < np; w0 += CF::WINDOW, ++win) {
    const bool ahead = w0 != 0;
    if (!ahead) {
      // the epilogue must have read every region of the previous unit
      if (!wait_or_abort(acc_empty, (win & 1u) ^ 1u, c.wait_ns, c.abort_flag)) return false;
      tc_fence_after();
    }
    const int64_t w1 = min(np, w0 + CF::WINDOW);
    for (int64_t i = w0; i < w1; ++i, ++k) {
      const uint32_t st = k % S, ph = (k / S) & 1u;
      if (!wait_or_abort(&c.full[st], ph, c.wait_ns, c.abort_flag)) return false;
      tc_fence_after();
      const uint32_t sa = smem_addr(c.stage_base + st * c.stage_bytes);
      const uint32_t sb = sa + SM::A_BYTES;
      if (i == w0) {
        if (ahead) {
          issue_blocks<B>(sa, sb, tmem, fresh, 1);
          // the epilogue must have read the exact regions of the last window
          if (!wait_or_abort(acc_empty, (win & 1u) ^ 1u, c.wait_ns, c.abort_flag)) return false;
          tc_fence_after();
        }
#pragma unroll
        for (int r = 0; r < kExactRegions; ++r) fresh[r] = true;
        issue_blocks<B>(sa, sb, tmem, fresh, ahead ? 2 : 0);
      } else {
        issue_blocks<B>(sa, sb, tmem, fresh, 0);
      }
      tc_commit(&c.empty[st]);  // frees the stage when these MMAs finish
    }
    tc_commit(acc_full);
  }
  return true;
}

// Epilogue (one of 8 warps): exact windows into int64, final recombination
// and the FP64 store of one C leaf.  `xb` is this unit's exchange buffer.
template <int B, bool SINGLE_FAST>
__device__ bool epi_unit(const Slot &sl, uint32_t &win, uint32_t &epb, int64_t *xb,
                         const Ctl &c, uint32_t tmem, uint64_t *acc_full,
                         uint64_t *acc_empty) {
  using CF = Cfg<B>;
  constexpr int N = CF::N, PARTS = CF::PARTS, WINDOW = CF::WINDOW;
  constexpr int E = B / 2;  // columns of the C leaf per epilogue thread
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3;                // TMEM lane quarter of this warp
  const int half = (warp >= 6) ? 1 : 0;  // which half of the columns
  const int part = (B == 64) ? (q >> 1) : q;
  const int row = (B == 64) ? ((q & 1) * 32 + lane) : lane;
  const int c0 = half * E;
  const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * q) << 16);
  const int64_t np = sl.np;
  // The int64 accumulators of the exact regions live in TMEM columns beyond
  // the MMA regions (2 columns per element: low, high word), so that the
  // exact regions can be copied to registers and released to the MMA at once.
  const uint32_t qbase = lane_base + static_cast<uint32_t>(kRegions * N + half * 2 * E);
  float rl[E];  // low region (t = 6), folded: R6 2^-8 + R7 2^-16
  for (int64_t w0 = 0; w0 < np; w0 += WINDOW, ++win) {
    const bool last = w0 + WINDOW >= np, first = w0 == 0;
    if (!warp_wait_or_abort(acc_full, win & 1u, c.wait_ns, c.abort_flag)) return false;
    tc_fence_after();
    // exact regions r = 0, 1 (base diagonal t = 2 + 2r); column half qq of a
    // region holds diagonal t + part + qq, weight 2^(8 (5 - t - qq)) in
    // units of diagonal 5 + part: ex[2r + qq] is shifted by 8 (3 - 2r - qq)
    float ex[4][E];
#pragma unroll
    for (int r = 0; r < kExactRegions; ++r)
#pragma unroll
      for (int qq = 0; qq < 2; ++qq)
        tmem_ld<E>(lane_base + static_cast<uint32_t>(r * N + qq * B + c0), ex[2 * r + qq]);
    tc_wait_ld();
    if (!last) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);  // the MMA may go on
    }
    long long Q[E];
    // a one-window unit needs no int64 round trip through TMEM (used where
    // the extra live int64 values do not spill: the 32-leaf-only kernel)
    const bool single = SINGLE_FAST && first && last;
    if (single) {
#pragma unroll
      for (int cc = 0; cc < E; ++cc)
        Q[cc] = (static_cast<long long>(__float2int_rn(ex[0][cc])) << 24) +
                (static_cast<long long>(__float2int_rn(ex[1][cc])) << 16) +
                (static_cast<long long>(__float2int_rn(ex[2][cc])) << 8) +
                static_cast<long long>(__float2int_rn(ex[3][cc]));
    } else {
#pragma unroll
      for (int ch = 0; ch < E / 8; ++ch) {
        uint32_t qw[16];
        if (first) {
#pragma unroll
          for (int i = 0; i < 16; ++i) qw[i] = 0;
        } else {
          tmem_ld16u(qbase + 16 * ch, qw);
          tc_wait_ld();
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int cc = ch * 8 + e;
          long long qv = static_cast<long long>(
              (static_cast<unsigned long long>(qw[2 * e + 1]) << 32) | qw[2 * e]);
          qv += (static_cast<long long>(__float2int_rn(ex[0][cc])) << 24) +
                (static_cast<long long>(__float2int_rn(ex[1][cc])) << 16) +
                (static_cast<long long>(__float2int_rn(ex[2][cc])) << 8) +
                static_cast<long long>(__float2int_rn(ex[3][cc]));
          qw[2 * e] = static_cast<uint32_t>(qv);
          qw[2 * e + 1] = static_cast<uint32_t>(static_cast<unsigned long long>(qv) >> 32);
        }
        tmem_st16u(qbase + 16 * ch, qw);
      }
      tc_wait_st();
      if (!last) continue;
    }
    {
      float v[E];
      tmem_ld<E>(lane_base + static_cast<uint32_t>(2 * N + c0), v);
      tc_wait_ld();
#pragma unroll
      for (int cc = 0; cc < E; ++cc) rl[cc] = v[cc] * 0x1p-8f;
      tmem_ld<E>(lane_base + static_cast<uint32_t>(2 * N + B + c0), v);
      tc_wait_ld();
#pragma unroll
      for (int cc = 0; cc < E; ++cc) rl[cc] = fmaf(v[cc], 0x1p-16f, rl[cc]);
    }
    if (!single) {
#pragma unroll
      for (int ch = 0; ch < E / 8; ++ch) {
        uint32_t qw[16];
        tmem_ld16u(qbase + 16 * ch, qw);
        tc_wait_ld();
#pragma unroll
        for (int e = 0; e < 8; ++e)
          Q[ch * 8 + e] = static_cast<long long>(
              (static_cast<unsigned long long>(qw[2 * e + 1]) << 32) | qw[2 * e]);
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(acc_empty);  // the next unit may overwrite TMEM
    // part value in units of 2^-(8 (5 + part) + 8) = 2^-48 after the shift
    // by 8 * part (rounded); the plan limits the window count so that every
    // part fits 64 bits
    auto part_value = [&](int cc) -> long long {
      const long long v = (Q[cc] << 8) + __float2ll_rn(rl[cc] * 256.0f);
      if (part == 0) return v;
      const int sh = kW * part;
      return (v + (1LL << (sh - 1))) >> sh;
    };
    if (B == 64) {
      // the two parts of an element meet in the exchange buffer: part 0
      // converts the first half of this thread's columns, part 1 the second,
      // each handing the other half of its values over (column-major buffer:
      // a warp's lanes, one row each, hit consecutive words)
      constexpr int H = E / 2;
      if (part == 0) {
#pragma unroll
        for (int cc = 0; cc < H; ++cc) xb[(c0 + H + cc) * B + row] = part_value(H + cc);
      } else {
#pragma unroll
        for (int cc = 0; cc < H; ++cc) xb[(c0 + cc) * B + row] = part_value(cc);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(c.ep_bar);
      if (!warp_wait_or_abort(c.ep_bar, epb & 1u, c.wait_ns, c.abort_flag)) return false;
      ++epb;
      const int er = sl.rexp[row];
      const int cb = c0 + (part == 0 ? 0 : H);
      double *dst = sl.C + static_cast<int64_t>(row) * B + cb;
      constexpr int CK = 8;  // elements converted together
#pragma unroll
      for (int c8 = 0; c8 < H; c8 += CK) {
        long long tv[CK];
        double ov[CK];
        bool good = true;
#pragma unroll
        for (int k = 0; k < CK; ++k) {
          const int cc = c8 + k;
          const long long v = part == 0 ? part_value(cc) : part_value(H + cc);
          tv[k] = v + xb[(cb + cc) * B + row];
          const int f = sl.cexp[cb + cc];
          bool ok;
          const double x = scaled_i64_fast(tv[k], er + f - 48, &ok);
          const bool none = er == kNoExp16 || f == kNoExp16;
          good = good && (ok || none);
          ov[k] = none ? 0.0 : x;
        }
        if (!__all_sync(0xffffffffu, good)) {
          // a result outside the normal range of doubles (rare): the exact
          // general conversion
#pragma unroll
          for (int k = 0; k < CK; ++k) {
            const int f = sl.cexp[cb + c8 + k];
            ov[k] = (er == kNoExp16 || f == kNoExp16) ? 0.0
                                                      : scaled_i64_to_double(tv[k], er + f - 48);
          }
        }
#pragma unroll
        for (int k = 0; k < CK; k += 2)
          *reinterpret_cast<double2 *>(dst + c8 + k) = make_double2(ov[k], ov[k + 1]);
      }
    } else {
      // every part into the buffer, then all 256 threads convert 4 elements
      // column-major per part (lanes = rows: no bank conflicts)
#pragma unroll
      for (int cc = 0; cc < E; ++cc)
        xb[(static_cast<int64_t>(part) * B + c0 + cc) * B + row] = part_value(cc);
      __syncwarp();
      if (lane == 0) mbar_arrive(c.ep_bar);
      if (!warp_wait_or_abort(c.ep_bar, epb & 1u, c.wait_ns, c.abort_flag)) return false;
      ++epb;
      const int et = threadIdx.x - 64;  // epilogue thread index
      const int r = et % B, col = (et / B) * 4;
      const int er = sl.rexp[r];
      double o4[4];
      long long t4[4];
      bool good = true;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        long long t = 0;
#pragma unroll
        for (int p = 0; p < PARTS; ++p) t += xb[(static_cast<int64_t>(p) * B + col + j) * B + r];
        t4[j] = t;
        const int f = sl.cexp[col + j];
        bool ok;
        const double x = scaled_i64_fast(t, er + f - 48, &ok);
        const bool none = er == kNoExp16 || f == kNoExp16;
        good = good && (ok || none);
        o4[j] = none ? 0.0 : x;
      }
      if (!__all_sync(0xffffffffu, good)) {
        // a result outside the normal range of doubles (rare)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int f = sl.cexp[col + j];
          o4[j] = (er == kNoExp16 || f == kNoExp16) ? 0.0
                                                    : scaled_i64_to_double(t4[j], er + f - 48);
        }
      }
      double *dst = sl.C + static_cast<int64_t>(r) * B + col;
      *reinterpret_cast<double2 *>(dst) = make_double2(o4[0], o4[1]);
      *reinterpret_cast<double2 *>(dst + 2) = make_double2(o4[2], o4[3]);
    }
  }
  return true;
}

// The persistent split kernel.  Units come from a device counter in order
// (neighbouring C leaves, in Morton order within a product, run together and
// share A and B slices through L2): with `prods` and `units` NULL unit u is C
// leaf u of `single`; with `units` only, C leaf units[u] of `single`;
// otherwise product units[u] >> 32, C leaf units[u] & 0xffffffff.
// `next_unit` (8 bytes, zero at launch) is the unit counter.
template <int MAXB>
__global__ void __launch_bounds__(kThreads, 1)
    k_split_gemm(const SplitProd single, const SplitProd *__restrict__ prods, int32_t nprods,
                 const int64_t *__restrict__ units, int64_t nunits,
                 unsigned long long *__restrict__ next_unit, int *__restrict__ status,
                 int64_t wait_ns) {
  (void)nprods;
  using KC = KCfg<MAXB>;
  constexpr int S = KC::STAGES;
  constexpr int NB = MAXB == 32 ? 2 : 1;  // TMEM accumulator sets
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  const uint32_t raw_addr = smem_addr(smem_raw);
  uint8_t *smem = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  Ctl c;
  c.stage_base = smem;
  c.stage_bytes = KC::STAGE;
  c.xbuf = reinterpret_cast<int64_t *>(smem + S * KC::STAGE);
  c.xbuf_bytes = KC::XBUF;
  c.queue = reinterpret_cast<Slot *>(smem + S * KC::STAGE + KC::NXB * KC::XBUF);
  uint64_t *bars = reinterpret_cast<uint64_t *>(c.queue + kQueue);
  c.full = bars;
  c.empty = bars + S;
  c.qfull = bars + 2 * S;
  c.qempty = c.qfull + kQueue;
  c.acc_full = c.qempty + kQueue;  // [NB]
  c.acc_empty = c.acc_full + 2;     // [NB]
  c.drain = c.acc_full + 4;
  c.ep_bar = c.acc_full + 5;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(c.ep_bar + 2);
  c.abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  c.wait_ns = wait_ns;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&c.full[st], 1);
      mbar_init(&c.empty[st], 1);
    }
    constexpr int kUnitWarps = kEpiWarps;  // a unit's epilogue: all 8 epilogue warps
    for (int i = 0; i < kQueue; ++i) {
      mbar_init(&c.qfull[i], 1);
      mbar_init(&c.qempty[i], 1 + kUnitWarps);  // the MMA thread and the epilogue warps
    }
    for (int bf = 0; bf < 2; ++bf) {
      mbar_init(&c.acc_full[bf], 1);
      mbar_init(&c.acc_empty[bf], kUnitWarps);
      mbar_init(&c.ep_bar[bf], kUnitWarps);
    }
    mbar_init(c.drain, 1);
    *c.abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, KC::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tmem = *tmem_slot;

  auto fail = [&]() {
    atomicOr(status, DEV_STATUS_TIMEOUT);
    *c.abort_flag = 1;
  };

  if (warp == 0) {
    // ------------------------------------------------------- producer --
    // Units are taken kChunk at a time.  Lane l resolves unit u0 + l (its
    // product, C leaf, pair segment, coordinates and the pointers the copies
    // need) so that those loads overlap; then, unit by unit, the line
    // exponents and first pair indices of the next unit are loaded while the
    // current one is staged and its copies are issued.
    constexpr int kChunk = KCfg<MAXB>::CHUNK;
    uint32_t k = 0;  // pairs issued
    uint32_t n = 0;  // queue position
    bool done = false;
    while (!done) {
      unsigned long long u0 = 0;
      if (lane == 0) u0 = atomicAdd(next_unit, static_cast<unsigned long long>(kChunk));
      u0 = __shfl_sync(0xffffffffu, u0, 0);
      int valid_l = 0, b_l = 0, crow_l = 0, ccol_l = 0;
      long long p0_l = 0, p1_l = 0, na_l = 0, nb_l = 0;
      const int *re_l = nullptr, *ce_l = nullptr;
      const int32_t *pa_l = nullptr, *pb_l = nullptr;
      const uint8_t *as_l = nullptr, *bs_l = nullptr;
      double *C_l = nullptr;
      if (lane < kChunk) {
        const unsigned long long u = u0 + lane;
        if (u < static_cast<unsigned long long>(nunits)) {
          valid_l = 1;
          const int64_t packed = units ? units[u] : static_cast<int64_t>(u);
          const int64_t o = units ? (packed & 0xffffffffLL) : packed;
          if (prods && !CHT_INDEX_OK((packed >> 32) >= 0 && (packed >> 32) < nprods, status))
            valid_l = 0;
          const SplitProd &dl = prods && valid_l ? prods[packed >> 32] : single;
          if (valid_l && !CHT_INDEX_OK(o >= 0 && o < dl.nunits, status)) valid_l = 0;
          if (valid_l) {
          b_l = dl.b;
          p0_l = dl.cseg[o];
          p1_l = dl.cseg[o + 1];
          crow_l = dl.crow[o];
          ccol_l = dl.ccol[o];
          if (!CHT_INDEX_OK(p0_l >= 0 && p0_l <= p1_l && p1_l <= dl.npairs && crow_l >= 0 &&
                                crow_l < dl.G && ccol_l >= 0 && ccol_l < dl.G,
                            status))
            valid_l = 0;
          re_l = dl.row_exp;
          ce_l = dl.col_exp;
          pa_l = dl.pa;
          pb_l = dl.pb;
          as_l = dl.a_slices;
          bs_l = dl.b_slices;
          C_l = dl.cptr ? dl.cptr[o] : dl.C + o * dl.b * dl.b;
          na_l = dl.nA;
          nb_l = dl.nB;
          }
        }
      }
      // exponents (rows lane, lane + 32) and the first 32 pair indices of unit j
      struct Pre {
        int re0, re1, ce0, ce1, pa, pb;
      };
      auto fetch = [&](int j) -> Pre {
        Pre q{kNoExp, kNoExp, kNoExp, kNoExp, 0, 0};
        if (!__shfl_sync(0xffffffffu, valid_l, j)) return q;
        const int b = __shfl_sync(0xffffffffu, b_l, j);
        const int64_t cr = __shfl_sync(0xffffffffu, crow_l, j), cc = __shfl_sync(0xffffffffu, ccol_l, j);
        const int *re = reinterpret_cast<const int *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(re_l), j));
        const int *ce = reinterpret_cast<const int *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(ce_l), j));
        const int32_t *pa = reinterpret_cast<const int32_t *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(pa_l), j));
        const int32_t *pb = reinterpret_cast<const int32_t *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(pb_l), j));
        const long long p0 = __shfl_sync(0xffffffffu, p0_l, j), p1 = __shfl_sync(0xffffffffu, p1_l, j);
        q.re0 = re[cr * b + lane];
        q.ce0 = ce[cc * b + lane];
        if (b == 64) {
          q.re1 = re[cr * b + lane + 32];
          q.ce1 = ce[cc * b + lane + 32];
        }
        if (p0 + lane < p1) {
          q.pa = pa[p0 + lane];
          q.pb = pb[p0 + lane];
        }
        return q;
      };
      Pre pre = fetch(0);
      for (int j = 0; j < kChunk && !done; ++j) {
        const int valid = __shfl_sync(0xffffffffu, valid_l, j);
        const Pre cur = pre;
        if (j + 1 < kChunk) pre = fetch(j + 1);  // lands while this unit is staged
        const uint32_t qs = n % kQueue, qph = (n / kQueue) & 1u;
        const bool ok = wait_or_abort(&c.qempty[qs], qph ^ 1u, c.wait_ns, c.abort_flag);
        if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
          if (lane == 0) fail();
          done = true;
          break;
        }
        Slot &sl = c.queue[qs];
        if (!valid) {
          if (lane == 0) {
            sl.b = 0;
            mbar_arrive(&c.qfull[qs]);
          }
          done = true;
          break;
        }
        const int b = __shfl_sync(0xffffffffu, b_l, j);
        const int64_t p0 = __shfl_sync(0xffffffffu, p0_l, j), p1 = __shfl_sync(0xffffffffu, p1_l, j);
        const int32_t *pa = reinterpret_cast<const int32_t *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(pa_l), j));
        const int32_t *pb = reinterpret_cast<const int32_t *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(pb_l), j));
        const uint8_t *a_slices = reinterpret_cast<const uint8_t *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(as_l), j));
        const uint8_t *b_slices = reinterpret_cast<const uint8_t *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(bs_l), j));
        double *Cp = reinterpret_cast<double *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(C_l), j));
        const long long na_j = __shfl_sync(0xffffffffu, na_l, j);
        const long long nb_j = __shfl_sync(0xffffffffu, nb_l, j);
        (void)na_j;
        (void)nb_j;
        sl.rexp[lane] = exp16(cur.re0);
        sl.cexp[lane] = exp16(cur.ce0);
        if (b == 64) {
          sl.rexp[lane + 32] = exp16(cur.re1);
          sl.cexp[lane + 32] = exp16(cur.ce1);
        }
        if (lane == 0) {
          sl.C = Cp;
          sl.np = static_cast<int32_t>(p1 - p0);
          sl.b = b;
          sl.u = static_cast<int32_t>(n);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&c.qfull[qs]);
        ++n;
        const int a_bytes = b == 64 ? Smem<64>::A_BYTES : Smem<32>::A_BYTES;
        const int b_bytes = b == 64 ? Smem<64>::B_BYTES : Smem<32>::B_BYTES;
        for (int64_t base = p0; base < p1 && !done; base += 32) {
          const int64_t pl = base + lane;
          const int32_t pa_v = base == p0 ? cur.pa : (pl < p1 ? pa[pl] : 0);
          const int32_t pb_v = base == p0 ? cur.pb : (pl < p1 ? pb[pl] : 0);
          const int cnt = static_cast<int>(p1 - base < 32 ? p1 - base : 32);
          for (int i = 0; i < cnt; ++i, ++k) {
            const uint32_t st = k % S, ph = (k / S) & 1u;
            const bool w_ok = wait_or_abort(&c.empty[st], ph ^ 1u, c.wait_ns, c.abort_flag);
            const int pa_i = __shfl_sync(0xffffffffu, pa_v, i);
            const int pb_i = __shfl_sync(0xffffffffu, pb_v, i);
            if (!__shfl_sync(0xffffffffu, w_ok ? 1 : 0, 0)) {
              if (lane == 0) fail();
              done = true;
              break;
            }
            if (!CHT_INDEX_OK(pa_i >= 0 && pa_i < na_j && pb_i >= 0 && pb_i < nb_j, status)) {
              // a bad leaf index: stop through the abort path, no copy issued
              if (lane == 0) *c.abort_flag = 1;
              done = true;
              break;
            }
            if (lane == 0) {
              mbar_arrive_expect_tx(&c.full[st], static_cast<uint32_t>(a_bytes + b_bytes));
            }
            __syncwarp();
            // one copy per slice tile, spread over the lanes (many copies in
            // flight instead of two large ones)
            {
              uint8_t *sa = c.stage_base + st * c.stage_bytes;
              const int tile = b == 64 ? Smem<64>::TILE : Smem<32>::TILE;
              const int na = a_bytes / tile, nb = b_bytes / tile;
              if (lane < na)
                bulk_g2s(sa + lane * tile, a_slices + static_cast<int64_t>(pa_i) * a_bytes +
                                               lane * tile,
                         static_cast<uint32_t>(tile), &c.full[st]);
              else if (lane < na + nb)
                bulk_g2s(sa + a_bytes + (lane - na) * tile,
                         b_slices + static_cast<int64_t>(pb_i) * b_bytes + (lane - na) * tile,
                         static_cast<uint32_t>(tile), &c.full[st]);
            }
          }
        }
      }
    }
    if (lane == 0) {
      // copies in flight must land before shared memory goes away (after a
      // normal run these phases completed long ago)
      for (uint32_t j = (k >= S ? k - S : 0); j < k; ++j)
        mbar_wait_bounded(&c.full[j % S], (j / S) & 1u, kDrainNs);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------ MMA issuer --
    if (lane == 0) {
      uint32_t k = 0, win0 = 0, win1 = 0;  // pairs consumed; windows per accumulator set
      for (uint32_t n = 0;; ++n) {
        const uint32_t qs = n % kQueue, qph = (n / kQueue) & 1u;
        if (!wait_or_abort(&c.qfull[qs], qph, c.wait_ns, c.abort_flag)) {
          fail();
          break;
        }
        const int b = c.queue[qs].b;
        const int64_t np = c.queue[qs].np;
        if (b == 0) break;
        mbar_arrive(&c.qempty[qs]);
        bool ok;
        const int bf = NB == 2 ? static_cast<int>(n & 1u) : 0;  // accumulator set
        const uint32_t tm = c.tmem + static_cast<uint32_t>(bf * 256);
        uint32_t w = bf ? win1 : win0;
        if constexpr (MAXB == 64)
          ok = b == 64 ? mma_unit<64, S>(np, k, w, c, tm, &c.acc_full[bf], &c.acc_empty[bf])
                       : mma_unit<32, S>(np, k, w, c, tm, &c.acc_full[bf], &c.acc_empty[bf]);
        else
          ok = mma_unit<32, S>(np, k, w, c, tm, &c.acc_full[bf], &c.acc_empty[bf]);
        if (bf) win1 = w;
        else win0 = w;
        if (!ok) {
          fail();
          break;
        }
      }
      // in-flight MMAs must finish before TMEM is released
      tc_commit(c.drain);
      mbar_wait_bounded(c.drain, 0, kDrainNs);
    }
  } else {
    // -------------------------------------------------------- epilogue --
    uint32_t win0 = 0, win1 = 0, epb = 0;
    for (uint32_t n = 0;; ++n) {
      const uint32_t qs = n % kQueue, qph = (n / kQueue) & 1u;
      if (!warp_wait_or_abort(&c.qfull[qs], qph, c.wait_ns, c.abort_flag)) {
        fail();
        break;
      }
      const Slot &sl = c.queue[qs];
      const int b = sl.b;
      if (b == 0) break;
      int64_t *xb = c.xbuf + (KC::NXB == 2 ? (n & 1u) * (KC::XBUF / 8) : 0);
      bool ok;
      const int bf = NB == 2 ? static_cast<int>(n & 1u) : 0;
      const uint32_t tm = c.tmem + static_cast<uint32_t>(bf * 256);
      uint32_t w = bf ? win1 : win0;
      if constexpr (MAXB == 64)
        ok = b == 64 ? epi_unit<64, false>(sl, w, epb, xb, c, tm, &c.acc_full[bf],
                                           &c.acc_empty[bf])
                     : epi_unit<32, false>(sl, w, epb, xb, c, tm, &c.acc_full[bf],
                                           &c.acc_empty[bf]);
      else
        ok = epi_unit<32, true>(sl, w, epb, xb, c, tm, &c.acc_full[bf], &c.acc_empty[bf]);
      if (bf) win1 = w;
      else win0 = w;
      if (!ok) {
        fail();
        break;
      }
      if constexpr (KC::NXB == 1) {
        // one exchange buffer: part 0 must have read it before the next unit
        __syncwarp();
        if (lane == 0) mbar_arrive(c.ep_bar);
        if (!warp_wait_or_abort(c.ep_bar, epb & 1u, c.wait_ns, c.abort_flag)) {
          fail();
          break;
        }
        ++epb;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&c.qempty[qs]);  // done with the slot
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(c.tmem, KC::TMEM_COLS);
}


// ------------------------------------------------ one-pair C leaves, b = 32 --
// A C leaf with a single leaf pair is one product A(I, K) B(K, J).  These
// leaves are grouped by their B leaf: a group holds up to 4 of them,
// (I_0, J) .. (I_3, J), all with the same B(K, J).  One MMA stacks slice i of
// the group's 4 A leaves along M = 128 (32 rows each) against B slice j
// (N = 32), so TMEM lane quarter q holds C leaf q of the group, and all slice
// diagonals of an element land in the same lane: the epilogue needs no
// exchange between warps.
//
// Slice pairs: exactly those with i + j <= 7 (21 MMAs of K = 32, each two
// K = 16 instructions).  The pairs of diagonal t = i + j accumulate into TMEM
// region t - 2 (32 columns).  A region sums at most 6 pairs of 32 digit
// products of magnitude <= 2^14, below 2^22: exact in FP32.  In units of
// 2^-56 of 2^(e_r + f_c + 2) the element is the integer
//     T = sum_{t=2..7} S_t 2^(56 - 8t)     (|T| < 2^62),
// assembled in int64 by T <- 2^8 T + S_t and converted once.  A uses the
// 8-digit slices of the 32-leaf path (digits 1..6 here), B its 6 digits.
//
// Roles as in k_split_gemm: warp 0 producer (groups taken 8 at a time from a
// device counter; per group one bulk copy of the B leaf's 6 slice tiles, and
// the 24 A tiles -- which land in [slice][unit] order, so no single bulk copy
// can fetch a unit's six -- as 16-byte cp.async copies spread over the 32
// lanes), warp 1 MMA issuer (one thread), warps 2..17 epilogue in two teams
// of 8 that take alternate groups (the epilogue's integer assembly and
// conversion set the pace: while one team waits for its group's slot,
// exponents or accumulators, the other computes), each team two warps per
// lane quarter, 16 columns each.  Two accumulator sets of 192 columns, one
// per team: the MMAs of group n + 1 run while the other team reads group n;
// a warp reads the six regions (8 columns at a time), releases its set, then
// assembles, converts and stores (through a per-warp staging block, as whole
// row pieces).  After the last group the producer publishes one end slot per
// team.  Every wait is bounded.
namespace single32 {
constexpr int kStages = 3;
constexpr int kTile = Smem<32>::TILE;                 // 2 KB
constexpr int kASlices = 6;                           // A digits used
constexpr int kA = kASlices * 4 * kTile;              // [slice][unit][tile]: 48 KB
constexpr int kB = kSB * kTile;                       // 12 KB
constexpr int kStage = kA + kB;
constexpr int kRegionsS = 6;                          // diagonals 2..7
constexpr int kSetCols = 256;                         // accumulator set pitch (192 used)
// 16 epilogue warps in two teams of 8 taking alternate groups (team t the
// groups n with n % 2 == t, in accumulator set t), so that one team's waits
// hide behind the other's arithmetic; in a team two warps per TMEM lane
// quarter, 16 columns each, handled 8 at a time: 18 warps in all
constexpr int kEpi = 16;
constexpr int kTeams = 2;
constexpr int kTeamWarps = kEpi / kTeams;
constexpr int kThreadsS = (2 + kEpi) * 32;
constexpr int kCols = 32 / (kTeamWarps / 4);           // columns per epilogue warp
constexpr int kPiece = 8;                              // columns converted and stored together
// per epilogue warp: a 32 x 8 block of C values, rows padded to 9 doubles
// (few bank conflicts), for stores of whole 64-byte row pieces
constexpr int kStgPitch = kPiece + 1;
constexpr int kStgBytes = 32 * kStgPitch * 8;
constexpr int kChunk = 8;                             // groups per counter step
}  // namespace single32

struct SingleWork {
  const uint8_t *a_slices;  // [nA][8][tile]
  const uint8_t *b_slices;  // [nB][6][tile]
  const int32_t *gb;        // per group: B leaf
  const int32_t *ga;        // per group: 4 A leaves
  // per group: 4 units: C leaf c >= 0 (its one pair), -1 none, or -2 - v:
  // pair v of a C leaf with 2 .. kFewPairsMax pairs, whose exact integer
  // result goes to scratch slot v (summed per C leaf by k_few_sum)
  const int32_t *gc;
  const int32_t *crow, *ccol;
  const int32_t *bcol;      // B leaf columns (a group's C column)
  const int *row_exp, *col_exp;
  double *C;
  int64_t *scratch;         // [nvirt][32][32]
  // C leaves of 2 .. kFewPairsMax pairs: leaf, first scratch slot, pairs
  const int32_t *few_c, *few_v, *few_m;
  int64_t ngroups, nfew, nvirt;
  int64_t nA, nB, nC, G;  // lengths (read by the bounds-checked build)
};

struct alignas(16) GSlot {
  double *C[4];     // output leaves (null: no unit in this quarter)
  const int *row_exp, *col_exp;  // the product's line exponents
  int32_t crow[4];  // the leaves' rows
  int32_t ccol;     // the shared leaf column
  int32_t count;    // units in the group (0: no more groups)
  int32_t raw;      // bit q: unit q writes its exact integers (a scratch slot)
  int32_t pad;
};

constexpr size_t single32_smem() {
  return static_cast<size_t>(single32::kStages) * single32::kStage + kQueue * sizeof(GSlot) +
         single32::kEpi * single32::kStgBytes + 256 + 1024;
}

// Group u is group u of `single` (works NULL), or, in a batch, group
// gunits[u] & 0xffffffff of product gunits[u] >> 32 (works[product]).
__global__ void __launch_bounds__(single32::kThreadsS, 1)
    k_split_single32(const SingleWork single, const SingleWork *__restrict__ works,
                     int32_t nworks, const int64_t *__restrict__ gunits, int64_t ntotal,
                     unsigned long long *__restrict__ next_group, int *__restrict__ status,
                     int64_t wait_ns) {
  (void)nworks;
  using namespace single32;
  constexpr int S = kStages;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_addr(smem_raw);
  uint8_t *smem = smem_raw + ((1024 - (raw_addr & 1023)) & 1023);
  uint8_t *stage_base = smem;
  double *staging = reinterpret_cast<double *>(smem + S * kStage);  // [kEpi][32][kStgPitch]
  GSlot *queue = reinterpret_cast<GSlot *>(smem + S * kStage + kEpi * kStgBytes);
  uint64_t *bars = reinterpret_cast<uint64_t *>(queue + kQueue);
  uint64_t *full = bars, *empty = bars + S, *qfull = bars + 2 * S, *qempty = qfull + kQueue;
  uint64_t *acc_full = qempty + kQueue, *acc_empty = acc_full + 2, *drain = acc_full + 4;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) {
      // the B copy's expect_tx arrival and one cp.async arrival per lane
      mbar_init(&full[st], 1 + 32);
      mbar_init(&empty[st], 1);
    }
    for (int i = 0; i < kQueue; ++i) {
      mbar_init(&qfull[i], 1);
      mbar_init(&qempty[i], 1 + kTeamWarps);
    }
    for (int bf = 0; bf < 2; ++bf) {
      mbar_init(&acc_full[bf], 1);
      mbar_init(&acc_empty[bf], kTeamWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto fail = [&]() {
    atomicOr(status, DEV_STATUS_TIMEOUT);
    *abort_flag = 1;
  };

  if (warp == 0) {
    // ------------------------------------------------------- producer --
    uint32_t n = 0;  // groups staged (queue position and stage count)
    bool done = false;
    while (!done) {
      unsigned long long u0 = 0;
      if (lane == 0) u0 = atomicAdd(next_group, static_cast<unsigned long long>(kChunk));
      u0 = __shfl_sync(0xffffffffu, u0, 0);
      // lane l resolves group u0 + l: its product's descriptor and indices
      const unsigned long long u = u0 + lane;
      int gb_l = 0, ccol_l = 0;
      int ga_l[4] = {0, 0, 0, 0}, gc_l[4] = {-1, -1, -1, -1}, cr_l[4] = {0, 0, 0, 0};
      bool valid_l = lane < kChunk && u < static_cast<unsigned long long>(ntotal);
      int64_t g = 0;
      const SingleWork *wp = &single;
      if (valid_l && works) {
        const int64_t packed = gunits[u];
        if (CHT_INDEX_OK((packed >> 32) >= 0 && (packed >> 32) < nworks, status))
          wp = &works[packed >> 32];
        else
          valid_l = false;
        g = packed & 0xffffffffLL;
      } else {
        g = static_cast<int64_t>(u);
      }
      const SingleWork &w = *wp;
      if (valid_l && !CHT_INDEX_OK(g < w.ngroups, status)) valid_l = false;
      const uint8_t *as_l = w.a_slices, *bs_l = w.b_slices;
      double *C_l = w.C;
      int64_t *sc_l = w.scratch;
      const int *re_l = w.row_exp, *ce_l = w.col_exp;
      if (valid_l) {
        gb_l = w.gb[g];
        bool ok = gb_l >= 0 && gb_l < w.nB;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ga_l[q] = w.ga[4 * g + q];
          gc_l[q] = w.gc[4 * g + q];
          ok = ok && gc_l[q] < w.nC && -2 - static_cast<int64_t>(gc_l[q]) < w.nvirt &&
               (gc_l[q] == -1 || (ga_l[q] >= 0 && ga_l[q] < w.nA));
        }
        ok = ok && gc_l[0] != -1;
        if (!CHT_INDEX_OK(ok, status)) valid_l = false;
      }
      if (valid_l) {
#pragma unroll
        for (int q = 0; q < 4; ++q) cr_l[q] = gc_l[q] >= 0 ? w.crow[gc_l[q]] : 0;
        ccol_l = w.bcol[gb_l];  // the B leaf's column is every unit's C column
        bool ok = ccol_l >= 0 && ccol_l < w.G;
#pragma unroll
        for (int q = 0; q < 4; ++q) ok = ok && cr_l[q] >= 0 && cr_l[q] < w.G;
        if (!CHT_INDEX_OK(ok, status)) valid_l = false;
      }
      for (int j = 0; j < kChunk && !done; ++j) {
        const uint32_t qs = n % kQueue, qph = (n / kQueue) & 1u;
        const bool ok = wait_or_abort(&qempty[qs], qph ^ 1u, wait_ns, abort_flag);
        if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
          if (lane == 0) fail();
          done = true;
          break;
        }
        GSlot &sl = queue[qs];
        const int valid = __shfl_sync(0xffffffffu, valid_l ? 1 : 0, j);
        if (!valid) {
          // one end slot per epilogue team (each team reads every other slot)
          if (lane == 0) {
            sl.count = 0;
            mbar_arrive(&qfull[qs]);
          }
          for (uint32_t t = 1; t < static_cast<uint32_t>(kTeams); ++t) {
            const uint32_t qe = (n + t) % kQueue, qeph = ((n + t) / kQueue) & 1u;
            const bool ok_e = wait_or_abort(&qempty[qe], qeph ^ 1u, wait_ns, abort_flag);
            if (!__shfl_sync(0xffffffffu, ok_e ? 1 : 0, 0)) {
              if (lane == 0) fail();
              break;
            }
            if (lane == 0) {
              queue[qe].count = 0;
              mbar_arrive(&qfull[qe]);
            }
          }
          done = true;
          break;
        }
        int ga[4], gc[4], cr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ga[q] = __shfl_sync(0xffffffffu, ga_l[q], j);
          gc[q] = __shfl_sync(0xffffffffu, gc_l[q], j);
          cr[q] = __shfl_sync(0xffffffffu, cr_l[q], j);
        }
        const uint8_t *a_slices = reinterpret_cast<const uint8_t *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(as_l), j));
        const uint8_t *b_slices = reinterpret_cast<const uint8_t *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(bs_l), j));
        double *Cbase = reinterpret_cast<double *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(C_l), j));
        int64_t *scratch = reinterpret_cast<int64_t *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(sc_l), j));
        const int *row_exp = reinterpret_cast<const int *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(re_l), j));
        const int *col_exp = reinterpret_cast<const int *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<long long>(ce_l), j));
        const int gbv = __shfl_sync(0xffffffffu, gb_l, j);
        const int ccv = __shfl_sync(0xffffffffu, ccol_l, j);
        int count = 0, raw = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          count += gc[q] != -1 ? 1 : 0;
          raw |= gc[q] <= -2 ? 1 << q : 0;
        }
        if (lane < 4) {
          const int c = gc[lane];
          sl.C[lane] = c >= 0    ? Cbase + static_cast<int64_t>(c) * 1024
                       : c <= -2 ? reinterpret_cast<double *>(
                                       scratch + (-2 - static_cast<int64_t>(c)) * 1024)
                                 : nullptr;
          sl.crow[lane] = cr[lane];
        }
        if (lane == 0) {
          sl.ccol = ccv;
          sl.count = count;
          sl.raw = raw;
          sl.row_exp = row_exp;
          sl.col_exp = col_exp;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&qfull[qs]);
        // the group's tiles: B slices 1..6 (one copy) and A slices 1..6 of
        // each unit into [slice][unit]
        const uint32_t st = n % S, ph = (n / S) & 1u;
        const bool w_ok = wait_or_abort(&empty[st], ph ^ 1u, wait_ns, abort_flag);
        if (!__shfl_sync(0xffffffffu, w_ok ? 1 : 0, 0)) {
          if (lane == 0) fail();
          done = true;
          break;
        }
        uint8_t *sa = stage_base + st * kStage;
        if (lane == 0) {
          mbar_arrive_expect_tx(&full[st], static_cast<uint32_t>(kB));
          bulk_g2s(sa + kA, b_slices + static_cast<int64_t>(gbv) * kB, static_cast<uint32_t>(kB),
                   &full[st]);
        }
        // A tile (unit q, slice i) -> sa + (i * 4 + q) tiles; lane l copies
        // 16-byte chunks l, l + 32, .. of every tile (coalesced)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (gc[q] == -1) continue;
          const uint8_t *src = a_slices + static_cast<int64_t>(ga[q]) * Cfg<32>::SA * kTile;
#pragma unroll
          for (int i = 0; i < kASlices; ++i)
#pragma unroll
            for (int c = lane; c < kTile / 16; c += 32)
              cp_async16(sa + (i * 4 + q) * kTile + c * 16, src + i * kTile + c * 16);
        }
        cp_async_arrive_noinc(&full[st]);  // when this lane's copies have landed
        ++n;
      }
    }
    // copies in flight land before shared memory goes away
    cp_async_wait_all();
    if (lane == 0) {
      for (uint32_t j = (n >= S ? n - S : 0); j < n; ++j)
        mbar_wait_bounded(&full[j % S], (j / S) & 1u, kDrainNs);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------ MMA issuer --
    if (lane == 0) {
      for (uint32_t n = 0;; ++n) {
        const uint32_t qs = n % kQueue, qph = (n / kQueue) & 1u;
        if (!wait_or_abort(&qfull[qs], qph, wait_ns, abort_flag)) {
          fail();
          break;
        }
        if (queue[qs].count == 0) break;
        mbar_arrive(&qempty[qs]);
        // accumulator set bf: the epilogue must have read the group before
        // last (the previous user of this set)
        const uint32_t bf = n & 1u, use = n >> 1;
        if (!wait_or_abort(&acc_empty[bf], (use & 1u) ^ 1u, wait_ns, abort_flag)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t st = n % S, ph = (n / S) & 1u;
        if (!wait_or_abort(&full[st], ph, wait_ns, abort_flag)) {
          fail();
          break;
        }
        // the A tiles came through the generic proxy (cp.async): order them
        // before the tensor core's (async proxy) reads
        fence_proxy_async_smem();
        tc_fence_after();
        const uint32_t sa = smem_addr(stage_base + st * kStage), sb = sa + kA;
        const uint32_t set = tmem + bf * kSetCols;
        // A digit i meets B digits 1..7-i: the B slice tiles lie one after
        // the other (32 rows each, the same 8-row group stride), so one MMA
        // of N = 32 (7 - i) rows of B covers them, writing regions i - 1..5
        // (columns 32 (i - 1) on); digit 1's MMA covers all six regions and
        // starts them
        const uint64_t bd = sw64_desc(sb);
#pragma unroll
        for (int i = 1; i <= kASlices; ++i) {
          const uint32_t idesc = make_idesc(128, 32 * (7 - i));
          const uint64_t ad = sw64_desc(sa + (i - 1) * 4 * kTile);
          const uint32_t dt = set + static_cast<uint32_t>((i - 1) * 32);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            tc_mma(dt, ad + 2 * kk, bd + 2 * kk, idesc, (i == 1 && kk == 0) ? 0u : 1u);
        }
        tc_commit(&empty[st]);  // the stage is free when these MMAs finish
        tc_commit(&acc_full[bf]);
      }
      tc_commit(drain);
      mbar_wait_bounded(drain, 0, kDrainNs);
    }
  } else {
    // -------------------------------------------------------- epilogue --
    const int e = warp - 2;                     // epilogue warp 0..15
    const int team = e / kTeamWarps;            // takes the groups n = team, team + 2, ..
    const int q = warp & 3;                     // lane quarter = unit of the group
    const int c0 = ((e % kTeamWarps) >> 2) * kCols;  // this warp's kCols columns
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * q) << 16);
    double *stg = staging + e * 32 * kStgPitch;
    for (uint32_t n = static_cast<uint32_t>(team);; n += kTeams) {
      const uint32_t qs = n % kQueue, qph = (n / kQueue) & 1u;
      if (!warp_wait_or_abort(&qfull[qs], qph, wait_ns, abort_flag)) {
        fail();
        break;
      }
      const GSlot &sl = queue[qs];
      if (sl.count == 0) break;
      double *Cq = sl.C[q];
      const bool raw = (sl.raw >> q) & 1;  // exact integers to a scratch slot
      // line exponents (loaded while the MMAs run)
      const int er =
          Cq && !raw ? sl.row_exp[static_cast<int64_t>(sl.crow[q]) * 32 + lane] : kNoExp;
      int fc[kCols];
#pragma unroll
      for (int c = 0; c < kCols; ++c)
        fc[c] = sl.col_exp[static_cast<int64_t>(sl.ccol) * 32 + c0 + c];
      const uint32_t bf = n & 1u, use = n >> 1;  // (bf == team)
      if (!warp_wait_or_abort(&acc_full[bf], use & 1u, wait_ns, abort_flag)) {
        fail();
        break;
      }
      tc_fence_after();
      // the six diagonals of 8 columns at a time (all six regions in one TMEM
      // round trip).  A region holds an integer of magnitude below 2^22:
      // adding 1.5 * 2^23 moves it, exactly, into [2^23, 2^24), where the
      // float's bit pattern is 0x4B400000 plus the integer (no
      // float-to-integer conversion); two regions combine in 32 bits
      // (S_t 2^8 + S_t+1 < 2^31 in magnitude) and the three pairs in 64:
      // T = P_0 2^32 + P_1 2^16 + P_2
      long long T[kCols];
#pragma unroll
      for (int h = 0; h < kCols / kPiece; ++h) {
        const uint32_t base = lane_base + bf * kSetCols + c0 + h * kPiece;
        float v[kRegionsS][kPiece];
#pragma unroll
        for (int r = 0; r < kRegionsS; ++r) tmem_ld8(base + static_cast<uint32_t>(r * 32), v[r]);
        tc_wait_ld();
#pragma unroll
        for (int c = 0; c < kPiece; ++c) {
          uint32_t u[kRegionsS];
#pragma unroll
          for (int r = 0; r < kRegionsS; ++r) u[r] = __float_as_uint(v[r][c] + 12582912.0f);
          constexpr uint32_t kBias = 257u * 0x4B400000u;  // both offsets of a pair
          const int p0 = static_cast<int>(u[0] * 256u + u[1] - kBias);
          const int p1 = static_cast<int>(u[2] * 256u + u[3] - kBias);
          const int p2 = static_cast<int>(u[4] * 256u + u[5] - kBias);
          T[h * kPiece + c] = static_cast<long long>(p0) * 0x100000000LL +
                              static_cast<long long>(p1) * 0x10000LL + p2;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[bf]);  // the MMA may reuse this set
      if (Cq) {
        // convert this lane's row (its own exponents), stage the warp's
        // 32 x 8 block, and store it as row pieces of 8 doubles; twice
        // (a line without stored values -- exponent kNoExp -- has zero
        // digits, so T = 0 there and converts to +0 whatever the exponent)
        const uint32_t eb = static_cast<uint32_t>(er) - 56u;
#pragma unroll
        for (int h = 0; h < kCols / kPiece; ++h) {
          bool good = true;
          if (raw) {
            // the integers themselves (their bit patterns pass through the
            // staging block and the stores unchanged)
#pragma unroll
            for (int c = 0; c < kPiece; ++c)
              stg[lane * kStgPitch + c] = __longlong_as_double(T[h * kPiece + c]);
          } else {
#pragma unroll
            for (int c = 0; c < kPiece; ++c) {
              bool ok;
              const double x = scaled_i64_fast(
                  T[h * kPiece + c],
                  static_cast<int>(eb + static_cast<uint32_t>(fc[h * kPiece + c])), &ok);
              good = good && ok;
              stg[lane * kStgPitch + c] = x;
            }
          }
          if (!__all_sync(0xffffffffu, good)) {
            // a result outside the normal range of doubles somewhere in the
            // warp (rare): the exact general conversion for this lane's row
#pragma unroll
            for (int c = 0; c < kPiece; ++c)
              stg[lane * kStgPitch + c] = scaled_i64_to_double(
                  T[h * kPiece + c],
                  static_cast<int>(eb + static_cast<uint32_t>(fc[h * kPiece + c])));
          }
          __syncwarp();
          constexpr int kRowsPer = 32 / kPiece;  // rows stored by one instruction
          const int col = lane % kPiece, sub = lane / kPiece;
#pragma unroll
          for (int k = 0; k < 32 / kRowsPer; ++k) {
            const int row = kRowsPer * k + sub;
            Cq[row * 32 + c0 + h * kPiece + col] = stg[row * kStgPitch + col];
          }
          __syncwarp();  // the staging block is read before it is written again
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&qempty[qs]);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// Scratch of one operand pair: line exponents and slices.
struct Operands {
  DevArray<int> row_exp, col_exp;
  DevArray<uint8_t> a_sl, b_sl;
};

int alloc_operands(const Pattern &pa, const Pattern &pb, cudaStream_t s, Operands &op) {
  const int b = pa.b;
  const size_t a_bytes = b == 64 ? Smem<64>::A_BYTES : Smem<32>::A_BYTES;
  const size_t b_bytes = b == 64 ? Smem<64>::B_BYTES : Smem<32>::B_BYTES;
  CHT_TRY(op.row_exp.alloc(pa.n, s));
  CHT_TRY(op.col_exp.alloc(pa.n, s));
  CHT_TRY(op.a_sl.alloc(static_cast<size_t>(pa.nnz) * a_bytes, s));
  CHT_TRY(op.b_sl.alloc(static_cast<size_t>(pb.nnz) * b_bytes, s));
  return CHT_OK;
}

// Exponents and slices of A and B (the pre-kernels of one product).  With
// `side`, B's two kernels run on the side stream, beside A's (the two
// chains share nothing; both are short and latency-bound on small products),
// and s waits for them at the end.
template <int B>
int split_operands(const cht_mat *A, const cht_mat *Bm, cudaStream_t s, Operands &op,
                   bool side = false) {
  using CF = Cfg<B>;
  const Pattern &pa = *A->pat, &pb = *Bm->pat;
  // kNoExp fill (every byte 0x80)
  CHT_CUDA_TRY(cudaMemsetAsync(op.row_exp.p, 0x80, sizeof(int) * pa.n, s));
  CHT_CUDA_TRY(cudaMemsetAsync(op.col_exp.p, 0x80, sizeof(int) * pa.n, s));
  const double *av = const_cast<cht_mat *>(A)->values();
  const double *bv = const_cast<cht_mat *>(Bm)->values();
  SideStream *ss = nullptr;
  cudaStream_t sb = s;
  if (side && pa.nnz > 0 && pb.nnz > 0) {
    CHT_TRY(side_stream(&ss));
    CHT_CUDA_TRY(cudaEventRecord(ss->fork, s));
    CHT_CUDA_TRY(cudaStreamWaitEvent(ss->s, ss->fork, 0));
    sb = ss->s;
  }
  if (pa.nnz > 0) {
    k_row_exp<B><<<grid_for(pa.nnz * B * (B / 16), 256), 256, 0, s>>>(av, pa.brow.p, pa.nnz,
                                                                      op.row_exp.p);
    CHT_TRY(launched("row_exp"));
  }
  if (pb.nnz > 0) {
    k_col_exp<B><<<grid_for(pb.nnz * B, 256), 256, 0, sb>>>(bv, pb.bcol.p, pb.nnz, op.col_exp.p);
    CHT_TRY(launched("col_exp"));
  }
  if (pa.nnz > 0) {
    k_split_a<B, CF::SA><<<grid_for(pa.nnz * B * (B / 8), 256), 256, 0, s>>>(
        av, pa.brow.p, pa.nnz, op.row_exp.p, op.a_sl.p);
    CHT_TRY(launched("split_a"));
  }
  if (pb.nnz > 0) {
    int sms = 0;
    CHT_TRY(num_sms(&sms));
    const int64_t nblk = std::min<int64_t>(pb.nnz, static_cast<int64_t>(sms) * 8);
    constexpr int smem = SplitBSmem<B>::TOTAL;
    CHT_CUDA_TRY(cudaFuncSetAttribute(k_split_b<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      smem));
    k_split_b<B><<<static_cast<unsigned>(nblk), 256, smem, sb>>>(bv, pb.bcol.p, pb.nnz,
                                                                 op.col_exp.p, op.b_sl.p);
    CHT_TRY(launched("split_b"));
  }
  if (ss) {
    CHT_CUDA_TRY(cudaEventRecord(ss->join, ss->s));
    CHT_CUDA_TRY(cudaStreamWaitEvent(s, ss->join, 0));
  }
  return CHT_OK;
}

SplitProd make_prod(const cht_plan *plan, const Operands &op, double *Cvals) {
  SplitProd d{};
  d.a_slices = op.a_sl.p;
  d.b_slices = op.b_sl.p;
  d.pa = plan->pa.p;
  d.pb = plan->pb.p;
  d.cseg = plan->cseg.p;
  d.crow = plan->C->brow.p;
  d.ccol = plan->C->bcol.p;
  d.row_exp = op.row_exp.p;
  d.col_exp = op.col_exp.p;
  d.C = Cvals;
  d.b = plan->b;
  d.nA = plan->nA;
  d.nB = plan->nB;
  d.nunits = plan->C->nnz;
  d.npairs = plan->npairs;
  d.G = plan->C->G;
  return d;
}

template <int MAXB>
int launch_split(const SplitProd &single, const SplitProd *prods, int32_t nprods,
                 const int64_t *units, int64_t nunits, unsigned long long *counter,
                 cudaStream_t s) {
  if (nunits <= 0) return CHT_OK;
  CHT_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
  int *status = nullptr;
  CHT_TRY(device_status_ptr(&status));
  int sms = 0;
  CHT_TRY(num_sms(&sms));
  auto kern = k_split_gemm<MAXB>;
  constexpr size_t smem = kernel_smem<MAXB>();
  CHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)));
  const int64_t grid = std::min<int64_t>(nunits, sms);
  kern<<<static_cast<unsigned>(grid), kThreads, smem, s>>>(single, prods, nprods, units, nunits,
                                                          counter, status, g_opt.wait_budget_ns);
  return launched("split_gemm");
}

// Pairs one unit may sum.  Every window adds at most 2^24 * 2^32 to an int64
// part (127 windows fit), and the final sum of a C element, in units of 2^-48
// of 2^(e_r + f_c + 2), is at most K * (128/255)^2 * 2^48 with K = b * pairs,
// so it stays below 2^63 for K <= 65024 (b = 64) and K <= 128000 (b = 32).
int max_unit_pairs(int b) { return b == 64 ? 127 * Cfg<64>::WINDOW : 4000; }

// Long segments: a C leaf with more pairs than one unit may sum is cut into
// np = ceil(len / maxp) pieces of ceil(len / np) pairs; each piece is a unit
// whose exact split-form sum goes to a scratch leaf, and the pieces are then
// added in FP64, in piece order.
__global__ void k_piece_count(const int64_t *__restrict__ cseg, int64_t nC, int maxp,
                              int32_t *__restrict__ npiece, int32_t *__restrict__ nscratch) {
  for (int64_t o = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; o < nC;
       o += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t len = cseg[o + 1] - cseg[o];
    const int32_t np = len > maxp ? static_cast<int32_t>((len + maxp - 1) / maxp) : 1;
    npiece[o] = np;
    nscratch[o] = np > 1 ? np : 0;
  }
}

__global__ void k_piece_fill(const int64_t *__restrict__ cseg, const int32_t *__restrict__ crow,
                             const int32_t *__restrict__ ccol, int64_t nC,
                             const int32_t *__restrict__ npiece, const int64_t *__restrict__ vpos,
                             const int64_t *__restrict__ tpos, double *C, double *scratch, int bb,
                             int64_t *__restrict__ vseg, int32_t *__restrict__ vrow,
                             int32_t *__restrict__ vcol, double **__restrict__ vptr) {
  for (int64_t o = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; o < nC;
       o += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p0 = cseg[o], len = cseg[o + 1] - p0;
    const int32_t np = npiece[o];
    const int64_t plen = (len + np - 1) / np;
    for (int32_t q = 0; q < np; ++q) {
      const int64_t v = vpos[o] + q;
      const int64_t start = p0 + q * plen;
      vseg[v] = start < p0 + len ? start : p0 + len;
      vrow[v] = crow[o];
      vcol[v] = ccol[o];
      vptr[v] = np > 1 ? scratch + (tpos[o] + q) * bb : C + o * bb;
    }
    if (o == nC - 1) vseg[vpos[o] + np] = cseg[nC];
  }
}

__global__ void k_piece_reduce(const int32_t *__restrict__ npiece, const int64_t *__restrict__ tpos,
                               int64_t nC, const double *__restrict__ scratch, int bb,
                               double *__restrict__ C) {
  for (int64_t o = blockIdx.x; o < nC; o += gridDim.x) {
    const int32_t np = npiece[o];
    if (np < 2) continue;
    const double *src = scratch + tpos[o] * bb;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
      double acc = src[e];
      for (int32_t q = 1; q < np; ++q) acc += src[static_cast<int64_t>(q) * bb + e];
      C[o * bb + e] = acc;
    }
  }
}

// The units of one product whose longest segment exceeds one unit's limit.
struct PieceUnits {
  DevArray<int32_t> npiece, nscratch, vrow, vcol;
  DevArray<int64_t> vpos, tpos, vseg;
  DevArray<double *> vptr;
  DevArray<double> scratch;
  int64_t nv = 0;
};

int make_pieces(const cht_plan *plan, double *Cvals, cudaStream_t s, PieceUnits &pu) {
  const int64_t nC = plan->C->nnz;
  const int bb = plan->b * plan->b;
  CHT_TRY(pu.npiece.alloc(nC, s));
  CHT_TRY(pu.nscratch.alloc(nC, s));
  CHT_TRY(pu.vpos.alloc(nC + 1, s));
  CHT_TRY(pu.tpos.alloc(nC + 1, s));
  k_piece_count<<<grid_for(nC, 256), 256, 0, s>>>(plan->cseg.p, nC, max_unit_pairs(plan->b),
                                                  pu.npiece.p, pu.nscratch.p);
  CHT_TRY(launched("piece_count"));
  CHT_TRY(scan_exclusive(pu.npiece.p, pu.vpos.p, nC, s));
  CHT_TRY(scan_exclusive(pu.nscratch.p, pu.tpos.p, nC, s));
  int64_t nt = 0;
  CHT_CUDA_TRY(cudaMemcpyAsync(&pu.nv, pu.vpos.p + nC, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CHT_TRY(read_i64(pu.tpos.p + nC, &nt, s));
  CHT_TRY(pu.vseg.alloc(pu.nv + 1, s));
  CHT_TRY(pu.vrow.alloc(pu.nv, s));
  CHT_TRY(pu.vcol.alloc(pu.nv, s));
  CHT_TRY(pu.vptr.alloc(pu.nv, s));
  CHT_TRY(pu.scratch.alloc(static_cast<size_t>(nt) * bb, s));
  k_piece_fill<<<grid_for(nC, 256), 256, 0, s>>>(plan->cseg.p, plan->C->brow.p, plan->C->bcol.p,
                                                 nC, pu.npiece.p, pu.vpos.p, pu.tpos.p, Cvals,
                                                 pu.scratch.p, bb, pu.vseg.p, pu.vrow.p,
                                                 pu.vcol.p, pu.vptr.p);
  return launched("piece_fill");
}

// Units (product << 32 | unit) of one product, in order.
__global__ void k_pack_units(int64_t n, int64_t prod, int64_t off, int64_t *__restrict__ units) {
  for (int64_t u = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; u < n;
       u += static_cast<int64_t>(gridDim.x) * blockDim.x)
    units[off + u] = (prod << 32) | u;
}

// ------------------------------------- grouping of the one-pair C leaves --
// The units of the one-pair kernel are the pairs of the C leaves with at
// most kFewPairsMax pairs: a one-pair C leaf is one unit writing its C leaf;
// a C leaf of 2 .. kFewPairsMax pairs gives one unit per pair, each writing
// its exact integer result (in units of 2^(e_r + f_c - 54), the same for
// every pair of the leaf) to a scratch slot, and k_few_sum adds them and
// converts once: the exact sum of the method's slice products (i + j <= 7)
// over the leaf's pairs, rounded once.  Units are grouped by their B leaf (groups in B's leaf order, i.e.
// Morton order of (K, J): neighbouring groups share A leaves of nearby inner
// indices K through L2), at most 4 per group; the C leaves with more pairs
// form the general kernel's unit list.  The symbolic phase counted the units
// per B leaf (cntB), so B leaf k's groups start at the prefix sum of
// ceil(cnt / 4), and each unit takes a slot in its B leaf's run by an atomic
// counter: the order inside a run, of the scratch slots and of the general
// kernel's list is not fixed, which changes no result -- every C leaf is
// computed on its own and every sum is exact.
struct GroupsOf {  // scan loader: groups of B leaf k
  const int32_t *cntB;
  __device__ int64_t operator()(int64_t k) const { return (cntB[k] + 3) >> 2; }
};

__global__ void k_group_place(const int64_t *__restrict__ cseg, int64_t nC,
                              const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
                              const int64_t *__restrict__ gstart, int32_t *__restrict__ fill,
                              unsigned long long *__restrict__ counters,
                              int32_t *__restrict__ gb, int32_t *__restrict__ ga,
                              int32_t *__restrict__ gc, int64_t *__restrict__ more,
                              int32_t *__restrict__ few_c, int32_t *__restrict__ few_v,
                              int32_t *__restrict__ few_m) {
  for (int64_t o = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; o < nC;
       o += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = cseg[o];
    const int64_t len = cseg[o + 1] - p;
    const int m = len > kFewPairsMax ? kFewPairsMax + 1 : static_cast<int>(len);
    if (m > kFewPairsMax) {
      more[atomicAdd(&counters[0], 1ULL)] = o;
      continue;
    }
    int64_t v0 = 0;
    if (m > 1) {
      const int64_t f = static_cast<int64_t>(atomicAdd(&counters[1], 1ULL));
      v0 = static_cast<int64_t>(atomicAdd(&counters[2], static_cast<unsigned long long>(m)));
      few_c[f] = static_cast<int32_t>(o);
      few_v[f] = static_cast<int32_t>(v0);
      few_m[f] = m;
    }
    for (int j = 0; j < m; ++j) {
      const int32_t k = pb[p + j];
      const int slot = atomicAdd(&fill[k], 1);
      const int64_t g = gstart[k] + (slot >> 2);
      const int q = slot & 3;
      ga[4 * g + q] = pa[p + j];
      gc[4 * g + q] = m == 1 ? static_cast<int32_t>(o) : static_cast<int32_t>(-2 - (v0 + j));
      if (q == 0) gb[g] = k;
    }
  }
}

// C leaves of 2 .. kFewPairsMax pairs: the sum of their units' exact
// integers, converted once with the leaf's line exponents.  One CTA per leaf;
// `fewunits` packs (product << 32) | leaf for a batch (works non-null).
__global__ void __launch_bounds__(256)
    k_few_sum(const SingleWork single, const SingleWork *__restrict__ works, int32_t nworks,
              const int64_t *__restrict__ fewunits, int64_t ntotal, int *__restrict__ status) {
  for (int64_t u = blockIdx.x; u < ntotal; u += gridDim.x) {
    const SingleWork *wp = &single;
    int64_t f = u;
    if (works) {
      const int64_t packed = fewunits[u];
      if (!CHT_INDEX_OK((packed >> 32) >= 0 && (packed >> 32) < nworks, status)) continue;
      wp = &works[packed >> 32];
      f = packed & 0xffffffffLL;
    }
    const SingleWork &w = *wp;
    if (!CHT_INDEX_OK(f < w.nfew, status)) continue;
    const int32_t o = w.few_c[f], v0 = w.few_v[f], m = w.few_m[f];
    if (!CHT_INDEX_OK(o >= 0 && o < w.nC && v0 >= 0 && m >= 2 && m <= kFewPairsMax &&
                          static_cast<int64_t>(v0) + m <= w.nvirt,
                      status))
      continue;
    const int64_t I = w.crow[o], J = w.ccol[o];
    if (!CHT_INDEX_OK(I >= 0 && I < w.G && J >= 0 && J < w.G, status)) continue;
    const int64_t *src = w.scratch + static_cast<int64_t>(v0) * 1024;
    double *dst = w.C + static_cast<int64_t>(o) * 1024;
    // each thread: 4 consecutive elements of one row, every slot's values
    // loaded at once (16-byte loads), then summed, converted and stored
    for (int e0 = threadIdx.x * 4; e0 < 1024; e0 += blockDim.x * 4) {
      longlong2 part[kFewPairsMax][2];
#pragma unroll
      for (int j = 0; j < kFewPairsMax; ++j) {
        if (j < m) {
          const longlong2 *p = reinterpret_cast<const longlong2 *>(src + j * 1024 + e0);
          part[j][0] = p[0];
          part[j][1] = p[1];
        } else {
          part[j][0] = make_longlong2(0, 0);
          part[j][1] = make_longlong2(0, 0);
        }
      }
      const int er = w.row_exp[I * 32 + (e0 >> 5)];
      const int4 fc = *reinterpret_cast<const int4 *>(w.col_exp + J * 32 + (e0 & 31));
      long long t[4] = {0, 0, 0, 0};
#pragma unroll
      for (int j = 0; j < kFewPairsMax; ++j) {
        t[0] += part[j][0].x;
        t[1] += part[j][0].y;
        t[2] += part[j][1].x;
        t[3] += part[j][1].y;
      }
      const int f[4] = {fc.x, fc.y, fc.z, fc.w};
      double x[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        // (an empty line of A or B has zero digits: t = 0 converts to +0)
        const int e2 = static_cast<int>(static_cast<uint32_t>(er) + static_cast<uint32_t>(f[k]) - 56u);
        bool ok;
        x[k] = scaled_i64_fast(t[k], e2, &ok);
        if (!ok) x[k] = scaled_i64_to_double(t[k], e2);
      }
      reinterpret_cast<double2 *>(dst + e0)[0] = make_double2(x[0], x[1]);
      reinterpret_cast<double2 *>(dst + e0)[1] = make_double2(x[2], x[3]);
    }
  }
}

struct SingleGroups {
  DevArray<int32_t> gb, ga, gc;  // per group: B leaf; 4 A leaves; 4 units (see SingleWork::gc)
  DevArray<int64_t> more;        // C leaves with more than kFewPairsMax pairs
  DevArray<int32_t> few_c, few_v, few_m;  // C leaves of 2 .. kFewPairsMax pairs
  int64_t ngroups = 0, nmore = 0, nsingle = 0, nfew = 0, nvirt = 0;
};

int build_single_groups(const cht_plan *plan, cudaStream_t s, SingleGroups &g) {
  const int64_t nC = plan->C->nnz, nB = plan->nB;
  if (plan->n_one < 0 || plan->n_few < 0 || plan->n_virt < 0 || plan->n_groups < 0 ||
      plan->one_pair_b == nullptr) {
    set_error("the plan carries no unit counts (a 32-leaf plan from the symbolic phase does)");
    return CHT_ERR_INVALID;
  }
  g.nsingle = plan->n_one;
  g.nfew = plan->n_few;
  g.nvirt = plan->n_virt;
  g.nmore = nC - plan->n_one - plan->n_few;
  g.ngroups = plan->n_groups;
  const int64_t ng = g.ngroups;
  DevArray<int64_t> gstart;
  DevArray<int32_t> fill;
  DevArray<unsigned long long> counters;
  CHT_TRY(gstart.alloc(nB + 1, s));
  CHT_TRY(fill.alloc(nB, s));
  CHT_TRY(counters.alloc(3, s));
  CHT_TRY(g.gb.alloc(ng, s));
  CHT_TRY(g.ga.alloc(4 * ng, s));
  CHT_TRY(g.gc.alloc(4 * ng, s));
  CHT_TRY(g.more.alloc(g.nmore, s));
  CHT_TRY(g.few_c.alloc(g.nfew, s));
  CHT_TRY(g.few_v.alloc(g.nfew, s));
  CHT_TRY(g.few_m.alloc(g.nfew, s));
  if (nC == 0) return CHT_OK;
  CHT_TRY(scan_exclusive_fn(GroupsOf{plan->one_pair_b}, nB, gstart.p, s));
  CHT_CUDA_TRY(cudaMemsetAsync(fill.p, 0, sizeof(int32_t) * nB, s));
  CHT_CUDA_TRY(cudaMemsetAsync(counters.p, 0, sizeof(unsigned long long) * 3, s));
  CHT_CUDA_TRY(cudaMemsetAsync(g.ga.p, 0, sizeof(int32_t) * 4 * ng, s));
  CHT_CUDA_TRY(cudaMemsetAsync(g.gc.p, 0xff, sizeof(int32_t) * 4 * ng, s));  // -1
  k_group_place<<<grid_for(nC, 256), 256, 0, s>>>(
      plan->cseg.p, nC, plan->pa.p, plan->pb.p, gstart.p, fill.p, counters.p, g.gb.p, g.ga.p,
      g.gc.p, g.more.p, g.few_c.p, g.few_v.p, g.few_m.p);
  return launched("group_place");
}

int launch_few_sum(const SingleWork &w, const SingleWork *works, int32_t nworks,
                   const int64_t *fewunits, int64_t ntotal, cudaStream_t s) {
  if (ntotal <= 0) return CHT_OK;
  int *status = nullptr;
  CHT_TRY(device_status_ptr(&status));
  int sms = 0;
  CHT_TRY(num_sms(&sms));
  const int64_t grid = std::min<int64_t>(ntotal, 16LL * std::max(sms, 1));
  k_few_sum<<<static_cast<unsigned>(grid), 256, 0, s>>>(w, works, nworks, fewunits, ntotal,
                                                        status);
  return launched("few_sum");
}

// One launch over `ntotal` groups: those of `w` (works NULL), or the groups
// gunits[] of the batch's products works[0 .. nworks).
int launch_single32(const SingleWork &w, const SingleWork *works, int32_t nworks,
                    const int64_t *gunits, int64_t ntotal, unsigned long long *counter,
                    cudaStream_t s) {
  if (ntotal <= 0) return CHT_OK;
  CHT_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
  int *status = nullptr;
  CHT_TRY(device_status_ptr(&status));
  int sms = 0;
  CHT_TRY(num_sms(&sms));
  constexpr size_t smem = single32_smem();
  CHT_CUDA_TRY(cudaFuncSetAttribute(k_split_single32,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)));
  const int64_t grid = std::min<int64_t>((ntotal + single32::kChunk - 1) / single32::kChunk, sms);
  k_split_single32<<<static_cast<unsigned>(std::max<int64_t>(grid, 1)), single32::kThreadsS,
                     smem, s>>>(
      w, works, nworks, gunits, ntotal, counter, status, g_opt.wait_budget_ns);
  return launched("split_single32");
}

// Packed units (product << 32) | list[u] of one product.
__global__ void k_pack_list(int64_t n, int64_t prod, const int64_t *__restrict__ list,
                            int64_t off, int64_t *__restrict__ units) {
  for (int64_t u = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; u < n;
       u += static_cast<int64_t>(gridDim.x) * blockDim.x)
    units[off + u] = (prod << 32) | list[u];
}

// The one-pair kernel's view of one product.
SingleWork make_single_work(const cht_plan *plan, const Operands &op, const SingleGroups &g,
                            const Pattern &bpat, double *Cvals, int64_t *scratch) {
  SingleWork sw{};
  sw.a_slices = op.a_sl.p;
  sw.b_slices = op.b_sl.p;
  sw.gb = g.gb.p;
  sw.ga = g.ga.p;
  sw.gc = g.gc.p;
  sw.crow = plan->C->brow.p;
  sw.ccol = plan->C->bcol.p;
  sw.row_exp = op.row_exp.p;
  sw.col_exp = op.col_exp.p;
  sw.bcol = bpat.bcol.p;
  sw.C = Cvals;
  sw.scratch = scratch;
  sw.few_c = g.few_c.p;
  sw.few_v = g.few_v.p;
  sw.few_m = g.few_m.p;
  sw.ngroups = g.ngroups;
  sw.nfew = g.nfew;
  sw.nvirt = g.nvirt;
  sw.nA = plan->nA;
  sw.nB = plan->nB;
  sw.nC = plan->C->nnz;
  sw.G = plan->C->G;
  return sw;
}

// The plan's one-pair groups, built at its first use and kept in the plan.
int plan_groups(cht_plan *plan, cudaStream_t s, const SingleGroups **out) {
  if (!plan->split_groups) {
    auto g = std::make_shared<SingleGroups>();
    CHT_TRY(build_single_groups(plan, s, *g));
    plan->split_groups = g;
  }
  *out = static_cast<const SingleGroups *>(plan->split_groups.get());
  return CHT_OK;
}

struct SplitBatch {
  std::vector<Operands> ops;
  std::vector<PieceUnits> pieces;  // per product; used where has_pieces
  std::vector<char> has_pieces;
  std::vector<char> one_pair;      // product's one-pair leaves go to the one-pair kernel
  DevArray<int64_t> units;         // the general kernel's units (when own_units)
  int64_t nunits = 0;
  bool own_units = false;
  DevArray<SplitProd> prods;
  DevArray<SingleWork> works;      // the one-pair kernel's product table
  DevArray<int64_t> gunits;        // (product << 32) | group, every one-pair product
  int64_t ngunits = 0;
  std::vector<DevArray<int64_t>> scratch;  // per product: few-pair units' integers
  DevArray<int64_t> fewunits;      // (product << 32) | few-pair leaf
  int64_t nfewunits = 0;
  DevArray<unsigned long long> counter;
  int maxb = 32;
};

}  // namespace

int split_multiply(cht_plan *plan, cht_mat *A, cht_mat *B, int nslices, cudaStream_t s,
                   double *Cvals, double *err_bound) {
  if (nslices != 0 && nslices != kSB) {
    set_error("the split form uses %d slices (nslices = 0 or %d)", kSB, kSB);
    return CHT_ERR_UNSUPPORTED;
  }
  const int b = plan->b;
  if (b != 32 && b != 64) {
    set_error("leaf size %d: the split form takes b = 32 or b = 64", b);
    return CHT_ERR_UNSUPPORTED;
  }
  // elementwise bound relative to 2^(e_r + f_c): K (s + 3) 2^(-s w) with
  // K <= n, plus the FP32 rounding of the low regions (below 2^-50)
  *err_bound = static_cast<double>(plan->n) * (kSB + 3) * 0x1p-48 + 0x1p-50;
  const bool pieces = plan->max_seg > max_unit_pairs(b);
  const bool one_pair = b == 32 && !pieces && g_opt.split_single;
  // the plan's one-pair groups first (their build synchronises when the
  // symbolic phase did not count them, and should then not wait for the
  // slicing pre-kernels)
  const SingleGroups *groups = nullptr;
  if (one_pair) CHT_TRY(plan_groups(plan, s, &groups));
  Operands op;
  CHT_TRY(alloc_operands(*A->pat, *B->pat, s, op));
  if (b == 64)
    CHT_TRY(split_operands<64>(A, B, s, op, true));
  else
    CHT_TRY(split_operands<32>(A, B, s, op, true));
  SplitProd d = make_prod(plan, op, Cvals);
  DevArray<unsigned long long> counter;
  CHT_TRY(counter.alloc(1, s));
  int64_t nunits = plan->C->nnz;
  PieceUnits pu;
  if (pieces) {
    CHT_TRY(make_pieces(plan, Cvals, s, pu));
    d.cseg = pu.vseg.p;
    d.crow = pu.vrow.p;
    d.ccol = pu.vcol.p;
    d.cptr = pu.vptr.p;
    d.nunits = pu.nv;
    nunits = pu.nv;
  }
  if (one_pair) {
    // the pairs of C leaves with at most kFewPairsMax pairs grouped by B
    // leaf (and the few-pair leaves' sums); the others by the general kernel
    const SingleGroups *g = groups;
    DevArray<int64_t> scratch;
    CHT_TRY(scratch.alloc(static_cast<size_t>(g->nvirt) * 1024, s));
    const SingleWork sw = make_single_work(plan, op, *g, *B->pat, Cvals, scratch.p);
    CHT_TRY(launch_single32(sw, nullptr, 0, nullptr, sw.ngroups, counter.p, s));
    CHT_TRY(launch_few_sum(sw, nullptr, 0, nullptr, g->nfew, s));
    if (g->nmore > 0) CHT_TRY(launch_split<32>(d, nullptr, 0, g->more.p, g->nmore, counter.p, s));
    return CHT_OK;
  }
  if (b == 64)
    CHT_TRY(launch_split<64>(d, nullptr, 0, nullptr, nunits, counter.p, s));
  else
    CHT_TRY(launch_split<32>(d, nullptr, 0, nullptr, nunits, counter.p, s));
  if (pieces) {
    const int64_t nC = plan->C->nnz;
    k_piece_reduce<<<static_cast<unsigned>(std::min<int64_t>(nC, 65535LL * 8)), 256, 0, s>>>(
        pu.npiece.p, pu.tpos.p, nC, pu.scratch.p, b * b, Cvals);
    CHT_TRY(launched("piece_reduce"));
  }
  return CHT_OK;
}

int split_batch_prepare(cht_batch *bt, cudaStream_t s) {
  if (bt->nslices != 0 && bt->nslices != kSB) {
    set_error("the split form uses %d slices (nslices = 0 or %d)", kSB, kSB);
    return CHT_ERR_UNSUPPORTED;
  }
  auto sb = std::make_unique<SplitBatch>();
  std::vector<SplitProd> host(bt->count);
  std::vector<SingleWork> works(bt->count);
  sb->ops.resize(bt->count);
  sb->pieces.resize(bt->count);
  sb->has_pieces.assign(bt->count, 0);
  sb->one_pair.assign(bt->count, 0);
  sb->scratch.resize(bt->count);
  bool own = false;
  for (int32_t i = 0; i < bt->count; ++i) {
    cht_plan *plan = bt->plans[i];
    CHT_TRY(alloc_operands(*bt->As[i]->pat, *bt->Bs[i]->pat, s, sb->ops[i]));
    host[i] = make_prod(plan, sb->ops[i], bt->views[i]->view_vals);
    sb->maxb = std::max(sb->maxb, static_cast<int>(plan->b));
    if (plan->max_seg > max_unit_pairs(plan->b)) {
      // long segments: this product's units become pieces (see make_pieces)
      PieceUnits &pu = sb->pieces[i];
      CHT_TRY(make_pieces(plan, bt->views[i]->view_vals, s, pu));
      host[i].cseg = pu.vseg.p;
      host[i].crow = pu.vrow.p;
      host[i].ccol = pu.vcol.p;
      host[i].cptr = pu.vptr.p;
      host[i].nunits = pu.nv;
      sb->has_pieces[i] = 1;
      own = true;
    } else if (plan->b == 32 && g_opt.split_single) {
      // as cht_multiply: one-pair C leaves to the one-pair kernel
      const SingleGroups *g = nullptr;
      CHT_TRY(plan_groups(plan, s, &g));
      CHT_TRY(sb->scratch[i].alloc(static_cast<size_t>(g->nvirt) * 1024, s));
      works[i] = make_single_work(plan, sb->ops[i], *g, *bt->Bs[i]->pat,
                                  bt->views[i]->view_vals, sb->scratch[i].p);
      sb->one_pair[i] = 1;
      sb->ngunits += g->ngroups;
      sb->nfewunits += g->nfew;
      own = true;
    }
  }
  if (own) {
    // the general kernel's units, every product's in order: its pieces, its
    // C leaves of two or more pairs (one-pair products), or all its C leaves
    int64_t total = 0;
    for (int32_t i = 0; i < bt->count; ++i) {
      const SingleGroups *g = static_cast<const SingleGroups *>(bt->plans[i]->split_groups.get());
      total += sb->has_pieces[i] ? sb->pieces[i].nv
               : sb->one_pair[i] ? g->nmore
                                 : bt->plans[i]->C->nnz;
    }
    if (total > 0x7fffffffLL || sb->ngunits > 0x7fffffffLL || sb->nfewunits > 0x7fffffffLL) {
      set_error("batch has too many work units");
      return CHT_ERR_UNSUPPORTED;
    }
    CHT_TRY(sb->units.alloc(total, s));
    CHT_TRY(sb->gunits.alloc(sb->ngunits, s));
    CHT_TRY(sb->fewunits.alloc(sb->nfewunits, s));
    int64_t off = 0, goff = 0, foff = 0;
    for (int32_t i = 0; i < bt->count; ++i) {
      const SingleGroups *g = static_cast<const SingleGroups *>(bt->plans[i]->split_groups.get());
      if (sb->one_pair[i]) {
        if (g->nmore > 0) {
          k_pack_list<<<grid_for(g->nmore, 256), 256, 0, s>>>(g->nmore, i, g->more.p, off,
                                                              sb->units.p);
          CHT_TRY(launched("pack_list"));
        }
        off += g->nmore;
        if (g->ngroups > 0) {
          k_pack_units<<<grid_for(g->ngroups, 256), 256, 0, s>>>(g->ngroups, i, goff,
                                                                 sb->gunits.p);
          CHT_TRY(launched("pack_units"));
        }
        goff += g->ngroups;
        if (g->nfew > 0) {
          k_pack_units<<<grid_for(g->nfew, 256), 256, 0, s>>>(g->nfew, i, foff,
                                                              sb->fewunits.p);
          CHT_TRY(launched("pack_units"));
        }
        foff += g->nfew;
        continue;
      }
      const int64_t n = sb->has_pieces[i] ? sb->pieces[i].nv : bt->plans[i]->C->nnz;
      if (n > 0) {
        k_pack_units<<<grid_for(n, 256), 256, 0, s>>>(n, i, off, sb->units.p);
        CHT_TRY(launched("pack_units"));
      }
      off += n;
    }
    sb->nunits = total;
    sb->own_units = true;
  }
  CHT_TRY(sb->prods.alloc(bt->count, s));
  CHT_TRY(sb->works.alloc(bt->count, s));
  CHT_TRY(sb->counter.alloc(1, s));
  CHT_CUDA_TRY(cudaMemcpyAsync(sb->prods.p, host.data(), sizeof(SplitProd) * bt->count,
                               cudaMemcpyHostToDevice, s));
  CHT_CUDA_TRY(cudaMemcpyAsync(sb->works.p, works.data(), sizeof(SingleWork) * bt->count,
                               cudaMemcpyHostToDevice, s));
  CHT_CUDA_TRY(cudaStreamSynchronize(s));
  bt->split_state = sb.release();
  return CHT_OK;
}

int split_batch_run(cht_batch *bt, cudaStream_t s) {
  auto *sb = static_cast<SplitBatch *>(bt->split_state);
  for (int32_t i = 0; i < bt->count; ++i) {
    if (bt->plans[i]->b == 64)
      CHT_TRY(split_operands<64>(bt->As[i], bt->Bs[i], s, sb->ops[i]));
    else
      CHT_TRY(split_operands<32>(bt->As[i], bt->Bs[i], s, sb->ops[i]));
  }
  const SplitProd none{};
  const int64_t *units = sb->own_units ? sb->units.p : bt->units.p;
  const int64_t nunits = sb->own_units ? sb->nunits : bt->nunits;
  if (sb->ngunits > 0)
    CHT_TRY(launch_single32(SingleWork{}, sb->works.p, bt->count, sb->gunits.p, sb->ngunits,
                            sb->counter.p, s));
  CHT_TRY(launch_few_sum(SingleWork{}, sb->works.p, bt->count, sb->fewunits.p, sb->nfewunits, s));
  if (sb->maxb == 64)
    CHT_TRY(launch_split<64>(none, sb->prods.p, bt->count, units, nunits, sb->counter.p, s));
  else
    CHT_TRY(launch_split<32>(none, sb->prods.p, bt->count, units, nunits, sb->counter.p, s));
  for (int32_t i = 0; i < bt->count; ++i) {
    if (!sb->has_pieces[i]) continue;
    const cht_plan *plan = bt->plans[i];
    const int64_t nC = plan->C->nnz;
    k_piece_reduce<<<static_cast<unsigned>(std::min<int64_t>(nC, 65535LL * 8)), 256, 0, s>>>(
        sb->pieces[i].npiece.p, sb->pieces[i].tpos.p, nC, sb->pieces[i].scratch.p,
        plan->b * plan->b, bt->views[i]->view_vals);
    CHT_TRY(launched("piece_reduce"));
  }
  return CHT_OK;
}

void split_batch_release(cht_batch *bt) {
  delete static_cast<SplitBatch *>(bt->split_state);
  bt->split_state = nullptr;
}

}  // namespace cht
