// Device helpers shared by the kernels: Morton codes, mbarriers, bulk copies
// and bounded waits.  All waits are bounded; no kernel traps.
#pragma once

#include <cstdint>

namespace cht {

// ------------------------------------------------------------ Morton keys --
// Quadrant order of the quadtree is 11, 12, 21, 22 (index 2*row_bit +
// col_bit), so bit k of the row goes to bit 2k+1 and bit k of the column to
// bit 2k: ascending keys = depth-first quadtree order.
__host__ __device__ inline uint64_t spread_bits(uint64_t x) {
  x &= 0xffffffffULL;
  x = (x | (x << 16)) & 0x0000ffff0000ffffULL;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffULL;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0fULL;
  x = (x | (x << 2)) & 0x3333333333333333ULL;
  x = (x | (x << 1)) & 0x5555555555555555ULL;
  return x;
}
__host__ __device__ inline uint32_t gather_bits(uint64_t x) {
  x &= 0x5555555555555555ULL;
  x = (x | (x >> 1)) & 0x3333333333333333ULL;
  x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0fULL;
  x = (x | (x >> 4)) & 0x00ff00ff00ff00ffULL;
  x = (x | (x >> 8)) & 0x0000ffff0000ffffULL;
  x = (x | (x >> 16)) & 0x00000000ffffffffULL;
  return static_cast<uint32_t>(x);
}
__host__ __device__ inline uint64_t morton(uint32_t row, uint32_t col) {
  return (spread_bits(row) << 1) | spread_bits(col);
}
__host__ __device__ inline uint32_t morton_row(uint64_t key) { return gather_bits(key >> 1); }
__host__ __device__ inline uint32_t morton_col(uint64_t key) { return gather_bits(key); }

// ----------------------------------------------------------------- timers --
__device__ inline uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// -------------------------------------------------------------- mbarriers --
__device__ inline uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ inline void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ inline void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ inline void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ inline void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ inline void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ inline void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity to complete, for at most
// budget_ns nanoseconds (budget 0: gives up at once).  Returns false when the
// budget ran out.
__device__ inline bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int64_t budget_ns) {
  if (budget_ns <= 0) return false;
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > static_cast<uint64_t>(budget_ns)) return false;
  }
}

// ----------------------------------------------------------- bulk copies --
// One-dimensional TMA bulk copy global -> shared, completing on `bar` with
// `bytes` transaction bytes.  Addresses 16-byte aligned, bytes % 16 == 0.
__device__ inline void bulk_g2s(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ------------------------------------------------- 16-byte async copies --
// One 16-byte global -> shared copy (cp.async, cached in L2 only).  Both
// addresses 16-byte aligned.
__device__ inline void cp_async16(void *dst_smem, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src)
               : "memory");
}
// An arrival on `bar` once every cp.async this thread issued so far has
// landed; the barrier's expected count must include it (.noinc).
__device__ inline void cp_async_arrive_noinc(uint64_t *bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ------------------------------------------------------------- FP64 DMMA --
// D (8x8) += A (8x4, row) * B (4x8, col), FP64 tensor-core MMA.
// Lane l holds A[l/4][l%4], B[l%4][l/4], D[l/4][2*(l%4) + {0, 1}].
__device__ inline void dmma_8x8x4(double &d0, double &d1, double a, double b) {
  asm volatile(
      "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
      : "+d"(d0), "+d"(d1)
      : "d"(a), "d"(b));
}

}  // namespace cht
