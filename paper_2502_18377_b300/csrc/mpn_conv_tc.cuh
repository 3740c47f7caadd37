// Convolution of the learned warm start on the 5th-generation tensor cores:
// an implicit GEMM per 3x3x3 tap with tcgen05.mma (kind::f16, BF16 x BF16 ->
// FP32), the accumulator of a tile in tensor memory.
//
// A CTA owns tiles of 128 consecutive points and loops over them
// (persistent), with three roles that wait on one another only through
// mbarriers:
//   * warps 0-3 (thread m = row m of a tile) copy, for TPS taps at a time,
//     their neighbours' CI input channels (16-byte cp.async, zero-filled
//     outside the grid) into the next slot of a ring of operand tiles A
//     (TPS x 128 x CI, K-major) in shared memory; each thread's copies
//     arrive on the slot's "full" barrier when they land, so copies are in
//     flight without holding registers;
//   * one thread of warp 4 waits for a full slot, orders the landed copies
//     before the tensor core's reads (proxy fence), issues per tap CI/16 MMAs of
//     M = 128, N = CO, K = 16 into one of the tile's NACC accumulators (128
//     TMEM lanes x CO FP32 columns each; tap k into accumulator k mod NACC, so
//     consecutive MMAs do not wait for one another; two tiles' sets used in
//     turn), commits the slot's MMAs to its "empty" barrier, and after the 27th
//     tap to the accumulator set's "full" barrier;
//   * warps 5-8 read a full accumulator set back with tcgen05.ld (warp w
//     reads lanes 32 (w mod 4) ..), add its NACC accumulators, arrive on its
//     "empty" barrier and apply bias, ReLU and the output conversion.
// The weights of all 27 taps (B operands, CO x CI, K-major) stay in shared
// memory.  Every wait is bounded; a wait that gives up sets an error word.
//
// Shared-memory operands use the canonical K-major layout without swizzling:
// 8 x 16-byte core matrices (8 rows of 8 BF16), stored contiguously; within
// an operand of one MMA the core matrices adjacent in K are LBO = 128 bytes
// apart and those adjacent in M (or N) SBO = 256 bytes apart.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace tc {

constexpr int TM = 128;          // points per tile (MMA M)
constexpr int TPB = 288;         // warps 0-3 gather, warp 4 issues the MMAs, warps 5-8 drain the accumulators
constexpr unsigned LBO = 128, SBO = 256;
constexpr int WAIT_LIMIT = 1 << 22;

__host__ __device__ constexpr int ks_of(int CI) { return CI / 16; }
// accumulators per tile: tap k accumulates into accumulator k mod NACC, so the
// tensor core has NACC independent chains (the epilogue adds them)
constexpr int NACC = 4;
// TMEM columns of a CTA: two tiles in turn x NACC accumulators x CO (a power
// of two >= 32)
__host__ __device__ constexpr int tmem_cols(int CO) { return 2 * NACC * CO <= 32 ? 32 : (2 * NACC * CO <= 64 ? 64 : (2 * NACC * CO <= 128 ? 128 : 256)); }
// resident CTAs per SM the tensor memory (512 columns) allows
__host__ __device__ constexpr int tmem_ctas(int CO) { return 512 / tmem_cols(CO); }
// bytes of one MMA's operand tile of R rows x 16 K: R/8 core-matrix rows of 2
__host__ __device__ constexpr int op_bytes(int R) { return (R / 8) * 256; }
// operand slots in the ring (taps the gathers run ahead of the MMAs)
__host__ __device__ constexpr int slots(int CI) { return CI == 16 ? 4 : 2; }
// taps per slot: one commit per slot (a commit per tap kept the tensor core
// from overlapping the taps' MMAs)
constexpr int TPS = 3;
// shared-memory layout (bytes): weights, the ring of A slots, barriers
// (full and empty per slot, accumulator full and empty per accumulator), TMEM address
__host__ __device__ constexpr int w_bytes(int CI, int CO) { return 27 * ks_of(CI) * op_bytes(CO); }
__host__ __device__ constexpr int a_bytes(int CI) { return TPS * ks_of(CI) * op_bytes(TM); }
__host__ __device__ constexpr int smem_used(int CI, int CO) {
  return w_bytes(CI, CO) + slots(CI) * a_bytes(CI) + 8 * (2 * slots(CI) + 4) + 16;
}
// the dynamic shared memory a launch requests: at least what keeps more than
// tmem_ctas(CO) CTAs from sharing an SM (233,472 bytes per SM, 1 KB of them
// reserved per CTA), so a CTA's TMEM allocation never has to wait
__host__ __device__ constexpr int smem_bytes(int CI, int CO) {
  return smem_used(CI, CO) > 233472 / (tmem_ctas(CO) + 1) ? smem_used(CI, CO) : 233472 / (tmem_ctas(CO) + 1);
}

// offset of the 16-byte chunk (row r, K chunk kc of 8 elements) in an operand
// tile of one MMA
__host__ __device__ constexpr unsigned chunk_off(int r, int kc) {
  return (unsigned)((r >> 3) * SBO + kc * LBO + (r & 7) * 16);
}

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4),
// descriptor version 1 (bits 46-47), no base offset, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo = SBO) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Row-staged variant (rows of n_y % 128 == 0): a tile is 128 consecutive y
// points of one (t, x) row, and M-row r of its MMAs is the point
// y0 + (r >> 3) + 16 (r & 7).  Each (t + dt, x + dx) input row the tile needs
// is staged once, as 18 core-matrix rows c' (K-major, CI/8 chunks of 8
// channels) whose row k holds the point y0 - 1 + c' + 16 k; the operand of the
// tap with y offset dy then starts dy + 1 core-matrix rows in (SBO =
// CI/8 x 128 bytes), so the three y taps of a row share one staging.  A ring
// slot holds the three x rows of one time plane (nine taps, one commit).
__host__ __device__ constexpr int rb_bytes(int CI) { return 18 * (CI / 8) * 128; }      // one staged row
__host__ __device__ constexpr int rs_bytes(int CI) { return 3 * rb_bytes(CI); }         // one slot (3 rows)
__host__ __device__ constexpr int rslots(int CI) { return CI == 16 ? 4 : 2; }
__host__ __device__ constexpr int rsmem_used(int CI, int CO) {
  return w_bytes(CI, CO) + rslots(CI) * rs_bytes(CI) + 8 * (2 * rslots(CI) + 4) + 16;
}
__host__ __device__ constexpr int rsmem_bytes(int CI, int CO) {
  return rsmem_used(CI, CO) > 233472 / (tmem_ctas(CO) + 1) ? rsmem_used(CI, CO) : 233472 / (tmem_ctas(CO) + 1);
}
// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s32(b)) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(s32(b)), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
// 16-byte asynchronous copy global -> shared (zero-filled when src_bytes = 0),
// and an arrival on an mbarrier when all of this thread's copies so far land
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_arrive(uint64_t* b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(s32(b)) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// one MMA: D (TMEM) (+)= A (smem) x B (smem)
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               :: "r"(dtmem), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}
// arrive on the mbarrier when every MMA this thread issued so far completes
__device__ __forceinline__ void commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s32(b)) : "memory");
}

}  // namespace tc
