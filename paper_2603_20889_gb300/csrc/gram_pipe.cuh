// Pipelined first Gram pass on tcgen05 (C = X^T X, paper Sec. 3.1, Algorithm 1 step 1, and
// the first pass of SVQB2) for the 16-, 32- and 64-column classes.
//
// The products are the exact bf16 digit products of gram_umma.cuh, arranged so that the
// tensor core, the CUDA cores and the copy engine work on different tiles at once:
//  * Warp roles.  Sixteen slicer warps cut tiles into digit planes and read the accumulators
//    out; one control warp issues the bulk copies (one column per lane, two tiles ahead) and
//    the MMAs.  They meet only at mbarriers: "stage read" per raw stage (slicers -> control:
//    the next copy into it may start), "digits ready" per digit buffer (slicers -> control),
//    "MMAs done" per digit buffer (tcgen05.commit -> slicers) and "tile landed" per raw stage
//    (copy engine -> slicers).  The slicers vote among themselves on a named barrier.
//  * A tile holds 4096 elements (KT = 4096 / NC rows).  Two raw stages and two digit
//    buffers alternate: while the MMAs of tile t run, the slicers cut tile t + 1 and the
//    copy of tile t + 2 is in flight.
//  * Every value is cut into EIGHT balanced base-128 digits (56 bits) relative to a running
//    per-column scale 2^e (|x| < 2^e), not a per-tile one.  Because the scale stays fixed
//    across tiles, the MMAs of many tiles accumulate in the same tensor-memory blocks; the
//    blocks are read out only every G = 16 tiles (the most that keeps every FP32 sum an exact
//    integer: 16 x KT rows x (7 / SP + 1) pairs x 64^2 <= 2^24), or when a tile's column
//    maximum exceeds the scale (the scale is then raised to that maximum plus 2 bits).
//    Relative to the largest element the fixed point keeps at least 53 bits; the dropped
//    digit pairs (p + q >= 8) weigh below 2^-52 of the column scales' product.
//  * Pair (p, q) of the digit planes weighs 2^(e_i + e_j - 12 - 7 (p + q)).  One MMA is
//    128 x 128 x 16: A stacks SP = 128 / NC planes p0..p0+SP-1 (its rows), B stacks planes
//    q0..q0+SP-1 (its columns), K = 16 rows of X.  The MMAs with the same p0 + q0 share one
//    block of 128 accumulator columns at (p0 + q0) NC; lane k NC + i, column l NC + j of it
//    carries weight p0 + q0 + k + l, so the combination tb = (p0 + q0) + l of a lane sits at
//    column tb NC + j and weighs tb + k.  Combinations of weight above 7 are not read.
//  * The read-out folds the blocks into double-float sums, kept with an FP64 level in an
//    L2-resident workspace block per CTA (touched only at read-outs, so no registers hold
//    them); the double-float sums move into the FP64 level every 16 read-outs.  At the end
//    the CTA's partial Gram matrix goes to the workspace and the last CTA runs the common
//    epilogue.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "gram.cuh"
#include "gram_tc.cuh"
#include "gram_umma.cuh"

namespace ql {

template <int NC>
struct PipeShape {
  static constexpr int TS = 512;              // slicer threads: 16 warps, 4 per TMEM lane quarter
  static constexpr int T = TS + 32;           // and the control warp (17 warps: up to 96 registers each)
  static constexpr int UPT = 512 / TS;        // 8-row units per slicer and tile
  static constexpr int KT = 4096 / NC;        // rows per tile: 64, 128, 256
  static constexpr int ND = 8;                // digit planes
  static constexpr int SP = 128 / NC;         // planes stacked in the MMA's M = N = 128
  static constexpr int PLANE = NC * KT * 2;   // bytes per digit plane (8 KB)
  static constexpr int DBUF = ND * PLANE;     // one tile's digit planes (64 KB)
  static constexpr int LBO = 128;             // bytes between core matrices along the rows
  static constexpr int SBO = KT * 16;         // bytes between 8-column groups
  static constexpr int TCOLS = 8 * NC;        // tensor-memory columns: 128, 256, 512
  static constexpr int PAIRS_MAX = 7 / SP + 1;  // MMAs per accumulator block and k-step
  static constexpr int G = 16;                // tiles summed in tensor memory per read-out
  static constexpr int SLACK = 2;             // bits of headroom above a new column maximum
  static constexpr int HALF = NC / (TS / 128);  // accumulator columns per slicer thread
  static constexpr int DF_FLUSH = 16;         // read-outs per double-float -> FP64 move
  static_assert(NC == 16 || NC == 32 || NC == 64, "M = N = 128 needs 128 / NC stacked planes");
  static_assert(NC * KT / 8 == UPT * TS, "units of 8 rows of one column, UPT per slicer thread");
  static_assert((long long)G * KT * PAIRS_MAX * 4096 <= (1LL << 24), "exact FP32 digit sums");
};

template <int NC, typename S, int XF = kXNone>
struct PipeSmem {
  using Sh = PipeShape<NC>;
  // a staged tile is KT / RPB boxes of RPB rows (128 bytes) x NC columns, written by the
  // tensor copy with the 128-byte swizzle: column c of box k is the 128-byte line
  // k NC + c, whose 16-byte chunk q sits at chunk position q ^ (c & 7) (the right-hand
  // side of least squares, a column of its own, is copied unswizzled)
  static constexpr int RPB = 128 / (int)sizeof(S);            // rows per box
  static constexpr int NBOX = Sh::KT / RPB;                   // boxes per tile
  static constexpr size_t kOffDig = 0;                       // 2 digit buffers (1024-aligned)
  static constexpr size_t kRaw = sizeof(S) * (size_t)NC * Sh::KT;
  static constexpr size_t kOffRaw = kOffDig + 2 * (size_t)Sh::DBUF;  // 2 raw stages
  static constexpr size_t kOffPow = kOffRaw + 2 * kRaw;
  static constexpr size_t kOffScale = kOffPow + 4 * NC;       // running scale exponents
  static constexpr size_t kOffColmax = kOffScale + 4 * NC;
  static constexpr size_t kOffMisc = kOffColmax + 4 * NC;
  // barriers: MMAs done [2], tile landed [2], digits ready [2], stage read [2]; then the
  // TMEM slot, the new-group flags [2] and the failure flags of the two roles
  static constexpr size_t kOffBar = (kOffMisc + 64 * 4 + 15) / 16 * 16;
  static constexpr size_t kOffSlot = kOffBar + 64;
  static constexpr size_t kMain = kOffSlot + 32;
  static constexpr size_t kRed = 8 * (size_t)128 * NC;       // end of chunk: per-lane sums (in the digits)
  static constexpr size_t kEpi = 8 * (4 * (size_t)NC * (NC + 1) + 8 * (NC + 1)) + 64 * 4 + 16;
  // later passes (Y = X M'): the M' digits as mma.sync B fragments [8-column block][k-step]
  // [digit][lane], the column exponents of X (whole matrix) and of M', and the CTA's entry
  // decision
  static constexpr int NCB = NC / 8, KSTEPS = NC / 16;
  static constexpr size_t kOffBq = (kMain + 15) / 16 * 16;
  static constexpr size_t kBq = XF == kXNone ? 0 : sizeof(uint2) * NCB * KSTEPS * 7 * 32;
  static constexpr size_t kOffGexp = kOffBq + kBq;
  static constexpr size_t kOffFexp = kOffGexp + 4 * NC;
  static constexpr size_t kOffEntry = kOffFexp + 4 * NC;
  static constexpr size_t kBytes = XF == kXNone ? kMain : kOffEntry + 16;
  static_assert(kEpi <= kOffPow, "the epilogue's shared memory stays below the scales and barriers");
  static_assert(kRed <= 2 * (size_t)Sh::DBUF, "per-lane sums fit in the digit buffers");
};

// Barrier state of a pipelined Gram CTA, carried from one work item to the next: the parity
// of each barrier pair's next phase, and whether every bounded wait so far succeeded
// (uniform across the CTA).  Each thread keeps its own copy; a role only uses its own bits.
struct PipeBars {
  uint32_t mpar = 0;  // bit b: next phase of "MMAs done" b (slicers) / "stage read" and "digits ready" b (control)
  uint32_t lpar = 0;  // bit b: next phase of "tile landed" b
  bool ok = true;
};

template <int NC, typename S>
QL_DEV uint32_t pipe_cta_begin(unsigned char* smem) {
  using Sm = PipeSmem<NC, S>;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Sm::kOffSlot);
  if ((threadIdx.x >> 5) == 0) tmem_alloc(tslot, PipeShape<NC>::TCOLS);
  if (threadIdx.x == 0) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Sm::kOffBar);
    for (int i = 0; i < 4; ++i) mbar_init(bar + i, 1);
    for (int i = 4; i < 8; ++i) mbar_init(bar + i, PipeShape<NC>::TS / 32);  // one arrival per slicer warp
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *tslot;
}

// Named barrier 1 among the slicer warps (barrier 0 is __syncthreads), with a vote.
template <int COUNT>
QL_DEV void slicer_sync() {
  asm volatile("bar.sync 1, %0;\n" ::"n"(COUNT) : "memory");
}
template <int COUNT>
QL_DEV bool slicer_or(bool p) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "n"(COUNT)
      : "memory");
  return r != 0;
}
template <int COUNT>
QL_DEV bool slicer_and(bool p) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "n"(COUNT)
      : "memory");
  return r != 0;
}

// One box of a rank-2 tensor map (x = row, innermost; y = column) into shared memory, its
// bytes counted on the mbarrier.  x must be a multiple of 16 bytes' worth of elements.
QL_DEV void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_addr(mbar))
      : "memory");
}

// The 8 rows r0..r0+7 of column c of a staged tile (see PipeSmem: boxes of RPB rows, 128-byte
// swizzle; swz = c & 7, or 0 for the unswizzled right-hand-side column); r0 is a multiple of 8.
template <int NC, typename S>
QL_DEV void load8_swz(S (&v)[8], const unsigned char* stage, int c, int r0, int swz) {
  constexpr int RPB = 128 / (int)sizeof(S), EPC = 16 / (int)sizeof(S);  // rows per box, per chunk
  const unsigned char* line = stage + (size_t)((r0 / RPB) * NC + c) * 128;
  const int q0 = (r0 % RPB) / EPC;
#pragma unroll
  for (int q = 0; q < 8 / EPC; ++q) {
    const float4 t = *reinterpret_cast<const float4*>(line + (((q0 + q) ^ swz) << 4));
    const S* e = reinterpret_cast<const S*>(&t);
#pragma unroll
    for (int j = 0; j < EPC; ++j) v[q * EPC + j] = e[j];
  }
}

// Sign, biased double exponent and 53-bit significand of a stored element (0 for zero).
QL_DEV void split_elem(double x, unsigned& neg, int& E, unsigned long long& sig) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  neg = (unsigned)(b >> 63);
  E = (int)((b >> 52) & 0x7ff);
  sig = (b & 0xfffffffffffffull) | (1ull << 52);
}
QL_DEV void split_elem(float x, unsigned& neg, int& E, unsigned long long& sig) {
  const unsigned b = __float_as_uint(x);
  neg = b >> 31;
  const int ef = (int)((b >> 23) & 0xff);
  E = ef == 0 ? 0 : ef + 896;
  sig = (unsigned long long)((b & 0x7fffffu) | 0x800000u) << 29;
}
QL_DEV int elem_exponent(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); }
QL_DEV int elem_exponent(float x) {
  const int ef = (int)((__float_as_uint(x) >> 23) & 0xff);
  return ef == 0 ? 0 : ef + 896;
}

// Eight balanced base-128 digits of a signed fixed-point value |N| < 2^55.  With
// Nb = N + kDigitBias8 (64 added to every digit position, the top one included), every
// digit is a bit field of Nb: digit p >= 1 is ((Nb >> 7 (7 - p)) & 127) - 64 and digit 0 is
// (Nb >> 49) - 64; all lie in [-64, 64] (Nb is positive and below 2^57).
constexpr unsigned long long kDigitBias8 =
    64ULL * ((1ULL << 49) + (1ULL << 42) + (1ULL << 35) + (1ULL << 28) + (1ULL << 21) + (1ULL << 14) + (1ULL << 7) + 1ULL);

// Nb = N + kDigitBias8 of one element, N = rint(x 2^(55 - e)) its round-to-nearest (ties to
// even) fixed point relative to the scale exponent Es >= E (e = Es - 1022, |x| < 2^e, so
// |N| < 2^55).  The common case, a shift of at most 31 bits, runs on 32-bit words (one
// funnel shift, and the dropped word decides the rounding); smaller elements take the
// 64-bit form.
template <typename S>
QL_DEV unsigned long long biased_fixed56(S x, int Es) {
  unsigned neg;
  int E;
  unsigned long long sig;
  split_elem(x, neg, E, sig);
  const int sh = Es - E - 2;
  unsigned long long q;
  if (E == 0) {
    q = 0ull;
  } else if (sh <= 31) {
    const unsigned sh_ = (unsigned)(sig >> 32), sl = (unsigned)sig;
    if (sh <= 0) {
      q = sig << (-sh);  // E >= Es - 2: exact
    } else {
      const unsigned ql = __funnelshift_r(sl, sh_, sh), qh = sh_ >> sh;
      const unsigned rem = sl << (32 - sh), half = 0x80000000u;
      const unsigned up = (rem > half || (rem == half && (ql & 1u))) ? 1u : 0u;
      q = (((unsigned long long)qh << 32) | ql) + up;
    }
  } else if (sh >= 54) {
    q = 0ull;  // below a quarter of the last place
  } else {
    q = sig >> sh;
    const unsigned long long rem = sig << (64 - sh), half = 1ull << 63;
    q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
  }
  const unsigned long long m = neg ? ~0ull : 0ull;
  return (q ^ m) + (kDigitBias8 + (neg ? 1ull : 0ull));  // N + bias, N = +-q
}

// Digit p of two elements (rows r, r + 1) as one bf16x2 word (row r in the lower half):
// the fields f (digit + 64, in [0, 128]) become bf16(128 + f) by their bits 0x4300 + f,
// and subtracting 192 leaves the digit exactly.
template <int P>
QL_DEV unsigned digit_word(unsigned long long A, unsigned long long B) {
  constexpr int SH = 7 * (7 - P);
  constexpr unsigned MASK = P == 0 ? 0x00ff00ffu : 0x007f007fu;
  const unsigned fa = (unsigned)(A >> SH), fb = (unsigned)(B >> SH);
  const unsigned w = (__byte_perm(fa, fb, 0x5410) & MASK) | 0x43004300u;
  const __nv_bfloat162 r =
      __hsub2(*reinterpret_cast<const __nv_bfloat162*>(&w), __floats2bfloat162_rn(192.0f, 192.0f));
  return *reinterpret_cast<const unsigned*>(&r);
}

// The same for the seven digits of the 48-bit convention (fixed48_of_double + kDigitBias,
// see gram_tc.cuh) of two elements, given Nb7 = N + kDigitBias + kDigitTop7: the top digit's
// field then reads (Nb7 >> 42) in [0, 128] and digit p's (Nb7 >> 7 (6 - p)) & 127.
constexpr unsigned long long kDigitTop7 = 64ULL << 42;
template <int P>
QL_DEV unsigned digit_word7(unsigned long long A, unsigned long long B) {
  constexpr int SH = 7 * (6 - P);
  constexpr unsigned MASK = P == 0 ? 0x00ff00ffu : 0x007f007fu;
  const unsigned fa = (unsigned)(A >> SH), fb = (unsigned)(B >> SH);
  const unsigned w = (__byte_perm(fa, fb, 0x5410) & MASK) | 0x43004300u;
  const __nv_bfloat162 r =
      __hsub2(*reinterpret_cast<const __nv_bfloat162*>(&w), __floats2bfloat162_rn(192.0f, 192.0f));
  return *reinterpret_cast<const unsigned*>(&r);
}

}  // namespace ql
