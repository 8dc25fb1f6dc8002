// Gram-matrix passes of the Q-less Cholesky-QR2 and SVQB2 methods (paper Sec. 3.1,
// Algorithm 1; kernels "tsmttsm", "tsmRttsmR" and "tsmmttsmm").
//
// One launch computes C = Y^T Y for Y = X (first pass) or Y = X M (second pass, with M =
// R1^{-1} upper triangular for CholQR2 or M = B1 = U1 L1^{-1/2} for SVQB2), where the
// product X M is formed tile by tile in shared memory and never written back (the
// "on the fly" second pass).  Each CTA streams its row tiles (cp.async staging, one tile
// ahead), converts them to the working arithmetic once, applies M, and accumulates 4 x 4
// blocks of the upper triangle of C in registers over row slices.  The CTA partials are
// reduced in a fixed order by the last CTA to finish (no atomics on the data, so results
// are bitwise reproducible), which then runs the n x n FP64 epilogue of the pass.
#pragma once

#include "common.cuh"

namespace ql {

enum GramXform : int { kXNone = 0, kXUpper = 1, kXFull = 2 };

template <int NC>
struct GramShape {
  static constexpr int BS = NC < 4 ? NC : 4;      // block edge of C
  static constexpr int NB = NC / BS;              // blocks per dimension
  static constexpr int NBT = NB * (NB + 1) / 2;   // blocks on/above the diagonal
  static constexpr int T = NC == 64 ? 288 : NC == 32 ? 288 : NC == 16 ? 160 : NC == 8 ? 192 : 256;
  static constexpr int SL = T / NBT >= 1 ? T / NBT : 1;  // row slices
  static constexpr int B = 4096 / NC;             // rows per tile
};

template <int NC, typename S, typename Ar>
struct GramSmem {
  using Sh = GramShape<NC>;
  using V = typename Ar::T;
  static constexpr size_t kStage = sizeof(S) * NC * Sh::B;
  static constexpr size_t kY = sizeof(V) * NC * Sh::B;
  static constexpr size_t kRed = sizeof(V) * Sh::SL * Sh::NBT * Sh::BS * Sh::BS;
  static constexpr size_t kYY = 2 * kY > kRed ? 2 * kY : kRed;  // Y0, Y1 (or the slice reduction)
  static constexpr size_t kM = sizeof(V) * NC * NC;
  static constexpr size_t kEpi = sizeof(double) * (5 * NC * (NC + 1) + 8 * (NC + 1));  // n x n FP64, ld NC + 1
  static constexpr size_t kOffY = (kStage + 15) / 16 * 16;
  static constexpr size_t kOffM = kOffY + kYY;
  static constexpr size_t kOffMisc = kOffM + kM;
  static constexpr size_t kMain = kOffMisc + 64 * sizeof(int) + NC * sizeof(int);
  static constexpr size_t kBytes = kMain > kEpi + 64 * sizeof(int) + 16 ? kMain : kEpi + 64 * sizeof(int) + 16;
};

}  // namespace ql
