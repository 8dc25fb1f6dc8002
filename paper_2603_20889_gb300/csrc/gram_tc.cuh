// Tensor-core Gram pass (bf16 mma.sync) with exact digit slicing.
//
// The Gram products C = Y^T Y of the Gram methods (paper Sec. 3.1, "tsmttsm" and the
// fused second-pass kernels) are dense contractions over the m rows, so they run on the
// tensor cores.  FP64-level accuracy comes from splitting every value exactly into bf16
// digits:  for each row tile and column c, e_c is the smallest power of two above the
// column's largest |y|;  y 2^(48 - e_c) is rounded to the nearest integer N (ties to even,
// |N| <= 2^48) and written in balanced base 128,
//   N = sum_{k=0..6} d_k 128^(6-k),  d_1..d_6 in [-64, 63], d_0 in [-64, 64],
// so y ~= sum_k d_k 2^(e_c - 6 - 7k) with a rounding error below 2^(e_c - 49) that is as
// often positive as negative.  Every digit is an integer that bf16 holds exactly, every
// product |d_p d_q| <= 2^12 is exact, and the tensor cores sum at most 7 digit pairs over at
// most 128 rows per accumulator, far below 2^24: every FP32 accumulator is an exact integer.
// Products with the same weight w = p + q share one accumulator, for w <= 6; each is scaled
// by 2^(e_i + e_j - 12 - 7w) (exact) and folded into a double-float per C entry, and the
// double-float sums are moved into FP64 every few tiles.  The dropped pairs (w >= 7) involve
// only the lower digits d_1..d_6, which are centred on zero: per row they weigh less than
// 2^-49 of 2^(e_i + e_j) and have mean zero (the squares d_k^2 that do not cancel, k >= 4,
// weigh 2^-56 and less), so they average out over the rows instead of biasing C, as digits
// of one sign (truncation) would.
//
// The second pass forms Y = X M (M = R1^{-1} or B1) on the tensor cores as well.  X is sliced
// at the column scale e_k of the whole matrix (the first pass records it), so that
//   X M = sum_{p,q} 2^(-12 - 7(p+q)) dX_p M'  with  M' = diag(2^e_k) M,
// a scale that no longer depends on k.  M' is sliced once per CTA, column by column, into
// bf16 digits that stay in registers as MMA B fragments for the whole launch; per 16 x 8
// block of Y the 28 digit pairs again accumulate exactly in FP32 per weight, and the seven
// weights are summed into one double-float per element.  Y is then sliced at its own
// per-tile column scale and fed to the Gram products above.
//
// Warp layout of the Gram products (8 warps): the C tiles (16-row blocks x 8-column blocks)
// are grouped by row block into units of up to 2 column blocks, and the row tile is split
// into KS parts, so that every warp owns the same number of units.  Per 16-row k-step a
// unit loads the A fragments of all 7 digits and the B fragments of all 7 digits once and
// issues the 28 digit-pair MMAs from registers (one shared-memory fragment load feeds up to
// 7 MMAs).  In the product Y = X M' a warp owns one 8-column block of Y and 8 of its 16-row
// blocks.
#pragma once

#include "common.cuh"

namespace ql {

template <int NC>
struct TcShape {
  static constexpr int T = 256;
  static constexpr int KT = 8192 / NC;                // rows per shared-memory tile
  static constexpr int LDR = KT + 8;                  // padded digit row (conflict-free ldmatrix)
  static constexpr int ND = 7;                        // digits per value
  static constexpr int MR = NC < 16 ? 1 : NC / 16;    // 16-row blocks of C
  static constexpr int NCB = NC / 8;                  // 8-column blocks of C
  static constexpr int TILES = MR * NCB;
  static constexpr int G = NCB < 2 ? NCB : 2;         // column blocks per warp unit
  static constexpr int GROUPS = TILES / G;
  static constexpr int KS = GROUPS >= 8 ? 1 : 8 / GROUPS;  // row parts
  static constexpr int UNITS = GROUPS * KS;
  static constexpr int U = UNITS / 8;                 // units per warp
  static constexpr int KPART = KT / KS;               // rows per unit and tile
  static_assert(UNITS % 8 == 0, "8 warps");
  static_assert(KPART <= 128 && KPART % 16 == 0, "exact FP32 digit sums");
};

template <int NC, typename S>
struct TcSmem {
  using Sh = TcShape<NC>;
  static constexpr int LDY = Sh::KT + 4;                    // padded double-float row of Y
  static constexpr size_t kStage = sizeof(S) * NC * Sh::KT;
  static constexpr size_t kYdf = 8 * (size_t)NC * LDY;      // second pass: Y tile, same region
  static constexpr size_t kStageMax = kStage > kYdf ? kStage : kYdf;
  static constexpr size_t kSlices = 2 * (size_t)Sh::ND * NC * Sh::LDR;
  static constexpr size_t kOffSlices = (kStageMax + 127) / 128 * 128;
  static constexpr size_t kOffPow = kOffSlices + kSlices;          // float 2^e_c per column
  static constexpr size_t kOffExpo = kOffPow + 4 * NC;             // int max exponent per column
  static constexpr size_t kOffColmax = kOffExpo + 4 * NC;          // int, range check
  static constexpr size_t kOffGexp = kOffColmax + 4 * NC;          // int, column exponents of X
  static constexpr size_t kOffZero = (kOffGexp + 4 * NC + 15) / 16 * 16;
  static constexpr size_t kOffMisc = kOffZero + 16;
  static constexpr size_t kMain = kOffMisc + 64 * 4;
  static constexpr size_t kEpi = 8 * (4 * (size_t)NC * (NC + 1) + 8 * (NC + 1)) + 64 * 4 + 16;
  static constexpr size_t kBytes = kMain > kEpi ? kMain : kEpi;
};

QL_DEV void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_addr(p)));
}
QL_DEV void ldsm_x2(unsigned& r0, unsigned& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(smem_addr(p)));
}
// Four 8x8 b16 matrices, each stored with its rows as memory columns (ldmatrix .trans).
QL_DEV void ldsm_x4_t(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_addr(p)));
}
QL_DEV void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Balanced base-128 digits of a signed 48-bit fixed-point value N (|N| <= 2^48).  With
// Nb = N + kDigitBias (64 added to every digit position below the top one), digit k >= 1
// is ((Nb >> 7 (6 - k)) & 127) - 64 and digit 0 is Nb >> 42 (arithmetic shift).
constexpr long long kDigitBias =
    64LL * ((1LL << 35) + (1LL << 28) + (1LL << 21) + (1LL << 14) + (1LL << 7) + 1LL);
constexpr int kDigitScaleLog2 = 12;  // a digit pair (p, q) weighs 2^(e_i + e_j - 12 - 7 (p + q))

template <int K>
QL_DEV int balanced_digit(long long Nb) {
  if constexpr (K == 0) {
    return (int)(Nb >> 42);
  } else {
    return (int)((Nb >> (7 * (6 - K))) & 127) - 64;
  }
}
QL_DEV int balanced_digit_rt(long long Nb, int k) {
  return k == 0 ? (int)(Nb >> 42) : (int)((Nb >> (7 * (6 - k))) & 127) - 64;
}

// Bits of the float holding the small integer d (|d| <= 2^21): (1.5 2^23 + d) - 1.5 2^23.
// Its upper 16 bits are d in bf16, exact for |d| <= 256.
QL_DEV unsigned float_bits_of_small_int(int d) {
  return __float_as_uint(__fsub_rn(__int_as_float(0x4B400000 + d), 12582912.0f));
}
QL_DEV unsigned bf16_of_small_int(int d) { return float_bits_of_small_int(d) >> 16; }
// Two digits as a bf16x2 register (lo in the lower half).
QL_DEV unsigned bf16x2_of_ints(int lo, int hi) {
  return __byte_perm(float_bits_of_small_int(lo), float_bits_of_small_int(hi), 0x7632);
}

// Round-to-nearest (ties to even) signed fixed point of a double relative to the column's
// largest biased exponent Emax: N = rint(x 2^(48 - e)), e = Emax - 1022 (|x| < 2^e).
QL_DEV long long fixed48_of_double(double x, int Emax) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7ff);
  if (E == 0) return 0;
  const int sh = 5 + Emax - E;  // x 2^(48 - e) = sig 2^-sh
  if (sh >= 64) return 0;
  const unsigned long long sig = (bits & 0xfffffffffffffull) | (1ull << 52);
  unsigned long long q = sig >> sh;
  const unsigned long long r = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  q += (r > half || (r == half && (q & 1ull))) ? 1ull : 0ull;
  return (bits >> 63) ? -(long long)q : (long long)q;
}

// Same for a float (a stored FP32 element, or one part of a double-float) with Efmax the
// largest biased float exponent of the column: N = rint(f 2^(48 - e)), e = Efmax - 126.
QL_DEV long long fixed48_of_float(float f, int Efmax) {
  const unsigned b = __float_as_uint(f);
  const int Ef = (int)((b >> 23) & 0xff);
  if (Ef == 0) return 0;
  const unsigned long long sig = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
  const int sl = Ef - Efmax + 24;  // f 2^(48 - e) = sig 2^sl
  unsigned long long q;
  if (sl >= 0) {
    q = sig << sl;
  } else {
    const int sh = -sl;
    if (sh >= 26) return 0;
    q = sig >> sh;
    const unsigned long long r = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    q += (r > half || (r == half && (q & 1ull))) ? 1ull : 0ull;
  }
  return (b >> 31) ? -(long long)q : (long long)q;
}

}  // namespace ql
