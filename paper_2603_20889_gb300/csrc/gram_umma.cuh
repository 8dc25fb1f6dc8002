// Blackwell 5th-generation tensor-core (tcgen05) primitives and the tile layout of the
// Gram products C = Y^T Y of the Gram methods (paper Sec. 3.1).
//
// The exact bf16 digit slicing of gram_tc.cuh is kept (seven balanced base-128 digits per
// value, digit-pair products with p + q <= 6 (0-based) summed exactly in FP32), but the
// products run as tcgen05.mma with the accumulators in tensor memory (TMEM):
//  * Digit planes are stored in shared memory in the canonical K-major layout without
//    swizzle: 8 x 8 core matrices of 128 contiguous bytes (8 columns c x 8 rows r), core
//    matrices along r 128 B apart (LBO), 8-column groups KT x 16 B apart (SBO).  A plane
//    holds NC columns x KT rows (16 KB); the planes follow each other.
//  * One MMA has M = 128 = SP = 128 / NC consecutive planes p0..p0+SP-1 stacked (their
//    columns are the rows of A), N = NC (one plane q as B) and K = 16 rows.  Because the
//    planes are contiguous, the stacked A is one descriptor.  Lane L of the accumulator
//    holds plane p0 + L / NC, column L % NC; all MMAs with the same t = p0 + q share one
//    accumulator block of NC columns, in which lane group k carries digit weight t + k.
//  * Seven blocks (t = 0..6) cover every pair with p + q <= 6 (0-based); lane groups whose
//    weight exceeds 6 hold products beyond the truncation and are not read.  The plane
//    after the last one (p = 7) is never needed, so whatever lies there is harmless.
//  * Per block and tile at most ceil(7 / SP) pairs x KT rows x 64^2 < 2^24 add up: every FP32
//    accumulator is an exact integer.  One thread issues the MMAs and commits them to an
//    mbarrier; all warps then read TMEM (each warp its lane quarter) and fold the blocks,
//    scaled by 2^(e_i + e_j - 12 - 7w), into double-float accumulators that move into FP64
//    (in an L2-resident workspace block) every few tiles.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace ql {

template <int NC>
struct UmmaShape {
  static constexpr int T = 256;
  static constexpr int KT = 8192 / NC;        // rows per tile
  static constexpr int ND = 7;                // digit planes
  static constexpr int SP = 128 / NC;         // planes stacked in the MMA's M dimension
  static constexpr int PLANE = NC * KT * 2;   // bytes per digit plane (16 KB)
  static constexpr int LBO = 128;             // bytes between core matrices along the rows
  static constexpr int SBO = KT * 16;         // bytes between 8-column groups
  static constexpr int TCOLS = 7 * NC <= 128 ? 128 : (7 * NC <= 256 ? 256 : 512);  // TMEM columns
  static_assert(NC == 16 || NC == 32 || NC == 64, "M = 128 needs 128 / NC stacked planes");
  static constexpr int PAIRS_MAX = (ND + SP - 1) / SP;  // MMA pairs per accumulator block
  static_assert(PAIRS_MAX * KT * 64 * 64 < (1 << 24), "exact FP32 digit sums");
};

template <int NC, typename S>
struct UmmaSmem {
  using Sh = UmmaShape<NC>;
  static constexpr int LDS = Sh::KT + 16 / (int)sizeof(S);  // padded staged column
  static constexpr int LDY = Sh::KT + 4;                     // padded double-float column of Y
  static constexpr size_t kDigits = (size_t)Sh::ND * Sh::PLANE;
  static constexpr size_t kOffStage = kDigits;
  static constexpr size_t kStage = sizeof(S) * (size_t)NC * LDS;
  static constexpr size_t kYdf = 8 * (size_t)NC * LDY;
  static constexpr size_t kRed = 8 * (size_t)128 * NC;       // end of launch: per-lane partials
  static constexpr size_t kStageMax0 = kStage > kYdf ? kStage : kYdf;
  static constexpr size_t kStageMax = kStageMax0 > kRed ? kStageMax0 : kRed;
  static constexpr size_t kOffPow = (kOffStage + kStageMax + 15) / 16 * 16;
  static constexpr size_t kOffExpo = kOffPow + 4 * NC;
  static constexpr size_t kOffColmax = kOffExpo + 4 * NC;
  static constexpr size_t kOffGexp = kOffColmax + 4 * NC;
  static constexpr size_t kOffMisc = kOffGexp + 4 * NC;
  static constexpr size_t kOffBar = (kOffMisc + 64 * 4 + 15) / 16 * 16;  // MMA barrier, load barrier, TMEM slot
  static constexpr size_t kMain = kOffBar + 24;
  static constexpr size_t kEpi = 8 * (4 * (size_t)NC * (NC + 1) + 8 * (NC + 1)) + 64 * 4 + 16;
  static constexpr size_t kBytes = kMain > kEpi ? kMain : kEpi;
  static_assert(kStageMax >= (size_t)Sh::PLANE, "plane 7 reads stay inside shared memory");
};

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), descriptor version 1,
// no swizzle.
QL_DEV uint64_t umma_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

QL_DEV void tmem_alloc(uint32_t* slot, uint32_t ncols) {  // whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(slot)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
}
QL_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols));
}
QL_DEV void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
QL_DEV void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
      smem_addr(mbar)));
}
QL_DEV void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mbar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
}
QL_DEV bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
      "selp.b32 %0, 1, 0, P1;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(mbar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for the phase with the given parity; gives up after `limit` clocks (default 2^32,
// about 2 s) and returns false.
QL_DEV bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity, long long limit = 1ll << 32) {
  const long long t0 = clock64();
  while (!mbar_try_wait(mbar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
QL_DEV void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(mbar)) : "memory");
}
QL_DEV void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mbar)), "r"(bytes)
               : "memory");
}
// One contiguous global -> shared copy by the bulk-copy engine; its bytes count against the
// mbarrier's expected transaction bytes.  Addresses 16-byte aligned, size a multiple of 16.
QL_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(mbar))
               : "memory");
}
QL_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
QL_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Make this thread's generic-proxy shared-memory writes visible to the tensor core.
QL_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
QL_DEV void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// N consecutive 32-bit TMEM columns of this thread's lane (32x32b shape, whole warp).
QL_DEV void tmem_ld(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}
QL_DEV void tmem_ld(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
QL_DEV void tmem_ld(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
QL_DEV void tmem_ld(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

}  // namespace ql
