// Q-less Householder TSQR device code (paper Sec. 3.2, Algorithms 2-4).
//
// A CTA owns a contiguous range of row blocks ("tiles") of X.  Each tile of b rows is
// staged HBM -> shared memory with cp.async (issued one tile ahead, Algorithm 3's
// asynchronous copy), moved into registers, and folded into the CTA's running triangle R
// by the in-place trapezoidal Householder QR of [R; W] (Algorithm 4).  The per-CTA
// triangles are merged by a binary R-tree inside the same launch (Algorithm 2's second
// stage, replaced by "last CTA done" merges of triangle pairs), in FP64.
//
// Register tile layout: T threads = TC column groups x TR row threads.  Thread (cg, tr)
// holds rows tr + q*TR (q < RPT) of the columns c = cg + k*TC (k < NCT = NC/TC), so the
// work per Householder step shrinks evenly for every thread.  One shared-memory reduction
// per column step yields the pivot column's norm and all its dot products at once:
// for x = [R_jj; W(:,j)] and beta = -sign(R_jj) ||x||, v = x - beta e_1, the reflector
// H = I - v v^T / (-beta v_1) (v_1 = R_jj - beta) updates column c > j by
//   f_c = (W(:,j)^T W(:,c) + v_1 R_jc) / (-beta v_1),   R_jc -= v_1 f_c,   W(:,c) -= W(:,j) f_c.
//
// Precision.  The running triangle R is carried across the CTA's tiles in triple-float
// (double-float policy) or FP64.  With a = |R_jj|, b = |beta| = a + delta, s = sign(R_jj)
// and d_c = W(:,j)^T W(:,c), the update of row j reads
//   beta = -s (a + delta),  delta = ||W(:,j)||^2 / (a + ||x||),
//   R_jc  <- -R_jc + (delta R_jc - s d_c) / b,
//   f_c    = (d_c / (a + b) + s R_jc) / b,
// so the working arithmetic only forms the corrections delta and (delta R_jc - s d_c) / b,
// which are of the size of this tile's contribution; the sign flip is exact and the
// correction is added to the carried value with an error far below FP64's.  The rounding
// errors of the corrections are relative to one tile's rows, independent from tile to
// tile, and average out over the tiles instead of accumulating in R (double-float rounding
// on R itself would grow like the square root of the number of tiles).
#pragma once

#include "common.cuh"

namespace ql {

// Parameters of one TSQR problem as seen by the device code.
template <typename S>
struct TsqrProblem {
  ColSource<S> src;  // columns of X (or of [A b])
  int64_t m;         // rows
  int n;             // columns (<= NC)
  int vec16;         // every column starts 16-byte aligned (16-byte copies)
};

// Workspace views for one R-tree.
struct TreeView {
  double* slots;   // R triangles, n x n each (ld n), one per tree node
  int* counters;   // one arrival counter per internal node
  int* flags;      // [0]: range flag (double-float out of range), [1]: nonfinite
  int leaves;      // number of leaves (CTAs contributing a triangle)
};

// Arity of the R-tree for NC columns: for narrow X a merge costs little arithmetic and each
// tree level mostly costs its synchronisation (an arrival counter, L2 round trips), so wide
// nodes cut the levels; for wide X a merge costs O(n^3) FP64 per child and binary nodes
// keep that on fewer CTAs in sequence.
template <int NC>
constexpr int tree_arity() {
  return NC <= 8 ? 16 : (NC <= 16 ? 4 : 2);
}

template <int NC, int TC, int RPT, int T>
struct TsqrShape {
  static constexpr int TR = T / TC;        // row threads per column group
  static constexpr int NCT = NC / TC;      // columns held by one thread
  static constexpr int B = TR * RPT;       // rows per tile
  // staging depth: for wide X one buffer (the next tile lands while the current one is
  // factored from registers; the factorisation is long enough to cover the copy, and more
  // shared memory would cost CTAs per SM).  Very narrow X factors a tile quickly, so two
  // tiles stay in flight.
  static constexpr int STAGES = NC <= 4 ? 2 : 1;
  static_assert(NC % TC == 0, "column groups must divide NC");
  static_assert(TR % 16 == 0 || TR == T, "row threads per group must be a multiple of 16");
};

// Shared-memory layout of the TSQR kernels.
template <int NC, int TC, int RPT, int T, typename S, typename Ar>
struct TsqrSmem {
  using Sh = TsqrShape<NC, TC, RPT, T>;
  using V = typename Ar::T;
  static constexpr size_t kStage = sizeof(S) * NC * Sh::B;           // one staged tile
  static constexpr size_t kStages = kStage * Sh::STAGES;
  static constexpr size_t kMerge = sizeof(double) * tree_arity<NC>() * NC * NC;  // [Ra; Rb_1..Rb_{A-1}]
  static constexpr size_t kArena = kStages > kMerge ? kStages : kMerge;
  static constexpr size_t kR = (sizeof(typename Ar::RT) * NC * NC + 15) / 16 * 16;  // running triangle (carried type)
  static constexpr size_t kPart = sizeof(V) * NC * Sh::TR;           // column partial sums
  static constexpr size_t kPiv = (TC > 1) ? sizeof(V) * Sh::B : 0;   // pivot broadcast
  static constexpr size_t kF = sizeof(V) * NC;                       // reflector coefficients
  static constexpr size_t kOffR = (kArena + 15) / 16 * 16;
  static constexpr size_t kOffPart = kOffR + kR;
  static constexpr size_t kOffPiv = kOffPart + kPart;
  static constexpr size_t kOffF = kOffPiv + kPiv;
  static constexpr size_t kOffCn = kOffF + kF;                       // running column norms
  static constexpr size_t kOffMisc = kOffCn + sizeof(V) * NC;        // int[16] + int[NC]
  static constexpr size_t kOffSd = (kOffMisc + (16 + NC) * sizeof(int) + 15) / 16 * 16;
  static constexpr size_t kOffBeta = kOffSd + 2 * sizeof(double) * NC;  // FP64 scratch, then the new diagonal
  static constexpr size_t kBytes = kOffBeta + 16;
};

template <int P>
QL_DEV void group_reduce2(double& a, double& b) {
#pragma unroll
  for (int o = P / 2; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
}
template <int P>
QL_DEV void group_reduce2(df& a, df& b) {
#pragma unroll
  for (int o = P / 2; o > 0; o >>= 1) {
    a = df_add(a, shfl_xor(a, o));
    b = df_add(b, shfl_xor(b, o));
  }
}

__host__ __device__ constexpr int pow2_floor(int x) { return x >= 32 ? 32 : x >= 16 ? 16 : x >= 8 ? 8 : x >= 4 ? 4 : x >= 2 ? 2 : 1; }

// ---------------------------------------------------------------------------------------
// The CTA-level factorisation state and its tile loop.
// ---------------------------------------------------------------------------------------
template <int NC, int TC, int RPT, int T, typename S, typename Ar>
struct TsqrCta {
  using Sh = TsqrShape<NC, TC, RPT, T>;
  using Sm = TsqrSmem<NC, TC, RPT, T, S, Ar>;
  using V = typename Ar::T;
  static constexpr int TR = Sh::TR, NCT = Sh::NCT, B = Sh::B;

  using RT = typename Ar::RT;
  S* stage;     // [NC][B]
  RT* R;        // [NC][NC], R[j * NC + c] = R(j, c) in the carried type (triple-float or FP64)
  RT* beta_s;   // the new diagonal of the current column step
  V* part;      // [NC][TR]
  V* piv;       // [B]
  V* fco;       // [NC]
  V* cn;        // [NC] sum over finished rows i < j of R(i, c)^2 within the current tile
  int* misc;    // scalars
  int* colmax;  // [NC] per-column max biased exponent (range check)
  double* arena;  // aliases the stage: [Ra; Rb] during the R-tree
  double* sd;     // FP64 scratch [2 NC]

  int tid, cg, tr;

  QL_DEV void init(unsigned char* smem) {
    stage = reinterpret_cast<S*>(smem);
    arena = reinterpret_cast<double*>(smem);
    R = reinterpret_cast<RT*>(smem + Sm::kOffR);
    beta_s = reinterpret_cast<RT*>(smem + Sm::kOffBeta);
    part = reinterpret_cast<V*>(smem + Sm::kOffPart);
    piv = reinterpret_cast<V*>(smem + Sm::kOffPiv);
    fco = reinterpret_cast<V*>(smem + Sm::kOffF);
    cn = reinterpret_cast<V*>(smem + Sm::kOffCn);
    misc = reinterpret_cast<int*>(smem + Sm::kOffMisc);
    colmax = misc + 16;
    sd = reinterpret_cast<double*>(smem + Sm::kOffSd);
    tid = threadIdx.x;
    cg = tid / TR;
    tr = tid % TR;
  }

  QL_DEV void reset_r() {
    for (int i = tid; i < NC * NC; i += T) R[i] = Ar::r_zero();
    for (int i = tid; i < NC; i += T) colmax[i] = 0;
  }

  // Issue the cp.async copies of rows [row0, row0 + B) of all NC columns into stage
  // buffer `buf` (one commit group per tile).
  QL_DEV void issue_tile(const TsqrProblem<S>& p, int64_t row0, int buf = 0) {
    constexpr int PER = B / T > 0 ? B / T : 1;
    S* st = stage + (size_t)buf * NC * B;
    if (p.vec16) {  // 16-byte copies; the rows past m are zero-filled
      constexpr int EPV = 16 / (int)sizeof(S);  // elements per copy
      constexpr int NV = B / EPV;               // copies per column
      constexpr int PERV = NV / T > 0 ? NV / T : 1;
#pragma unroll 1
      for (int c = 0; c < NC; ++c) {
        const S* col = p.src.col(c < p.n ? c : 0);
        const bool cvalid = c < p.n;
#pragma unroll
        for (int e = 0; e < PERV; ++e) {
          const int v = tid + e * T;
          if (NV % T == 0 || v < NV) {
            const int64_t row = row0 + (int64_t)v * EPV;
            const int64_t left = cvalid ? p.m - row : 0;
            const int bytes = left <= 0 ? 0 : (left >= EPV ? 16 : (int)left * (int)sizeof(S));
            cp_async_16(st + c * B + v * EPV, bytes > 0 ? col + row : col, bytes);
          }
        }
      }
      cp_async_commit();
      return;
    }
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
      const S* col = p.src.col(c < p.n ? c : 0);
      bool cvalid = c < p.n;
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        int r = tid + e * T;
        if (B % T == 0 || r < B) {
          int64_t row = row0 + r;
          bool v = cvalid && row < p.m;
          cp_async_elem<S>(st + c * B + r, v ? col + row : col, v);
        }
      }
    }
    cp_async_commit();
  }

  // Stage -> registers (with the range bookkeeping of the double-float policy: the
  // column's largest exponent is reduced over the lanes that share the column, then one
  // shared-memory atomic per column and warp records it).
  QL_DEV void stage_to_regs(V (&w)[RPT][NCT], int buf = 0) {
    const S* stage = this->stage + (size_t)buf * NC * B;
    constexpr unsigned kHalf = TR >= 32 ? 0xffffffffu : 0x0000ffffu;
    const unsigned gmask = TR >= 32 ? 0xffffffffu : (((tid & 31) < 16) ? kHalf : (kHalf << 16));
#pragma unroll
    for (int k = 0; k < NCT; ++k) {
      int c = cg + k * TC;
      unsigned emax = 0;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        int E;
        w[q][k] = Ar::load(stage[c * B + tr + q * TR], E);
        emax = max(emax, (unsigned)E);
      }
      if constexpr (Ar::kRangeChecked) {
        emax = __reduce_max_sync(gmask, emax);
        if ((tid & (TR >= 32 ? 31 : 15)) == 0 && emax > 0) atomicMax(&colmax[c], (int)emax);
      }
    }
  }

  // Group reduction of two values over P consecutive lanes (P a power of two <= 32).
  QL_DEV static void group_reduce_rt(V& a, V& b, int P) {
    for (int o = P >> 1; o > 0; o >>= 1) {
      a = Ar::add(a, Ar::shfl(a, o));
      b = Ar::add(b, Ar::shfl(b, o));
    }
  }

  // One Householder column step j of the trapezoidal QR of [R; W].  The loop over j is
  // not unrolled (the unrolled form overflows the instruction cache); register indices
  // stay compile-time: every local column k is processed under a warp-uniform test on j.
  QL_DEV void column_step(V (&w)[RPT][NCT], int j) {
    const int kj = j / TC;  // local index of column j in its owner group
    V pv[RPT];
    if constexpr (TC == 1) {
#pragma unroll
      for (int q = 0; q < RPT; ++q) pv[q] = w[q][0];
#pragma unroll
      for (int k = 1; k < NCT; ++k)
        if (kj == k) {
#pragma unroll
          for (int q = 0; q < RPT; ++q) pv[q] = w[q][k];
        }
    } else {
      if (cg == j % TC) {
#pragma unroll
        for (int k = 0; k < NCT; ++k)
          if (kj == k) {
#pragma unroll
            for (int q = 0; q < RPT; ++q) piv[tr + q * TR] = w[q][k];
          }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < RPT; ++q) pv[q] = piv[tr + q * TR];
    }
    // partial dot products W(:,j)^T W(:,c) over my rows, for my columns c >= j
#pragma unroll
    for (int k = 0; k < NCT; ++k) {
      const int c = cg + k * TC;
      if (c >= j) {
        typename Ar::Acc acc = Ar::acc_zero();
#pragma unroll
        for (int q = 0; q < RPT; ++q) Ar::acc_fma(acc, pv[q], w[q][k]);
        part[c * TR + tr] = Ar::acc_get(acc);
      }
    }
    __syncthreads();
    // column totals and reflector coefficients: P threads per column c in [j, NC)
    {
      const int NV = NC - j;
      int P = pow2_floor(T / NV);
      if (P > TR) P = pow2_floor(TR);
      const int vi = tid / P, li = tid % P;
      const bool active = vi < NV;
      const int c = j + (active ? vi : 0);
      V d = Ar::zero(), nr = Ar::zero();
      if (active) {
        for (int t = li; t < TR; t += P) {
          d = Ar::add(d, part[c * TR + t]);
          nr = Ar::add(nr, part[j * TR + t]);
        }
      }
      group_reduce_rt(d, nr, P);
      if (active && li == 0) {
        // Householder preserves the 2-norm of column j of [R; W]: cn[j] + x1^2 + nr is its
        // norm at the start of the tile.  A remainder below kTau of it is rounding residue
        // (a tile with fewer independent rows than columns): no reflector is built from it.
        const RT x1r = R[j * NC + j];
        const V x1 = Ar::r_get(x1r);
        V rem = Ar::add(Ar::mul(x1, x1), nr);
        bool skip = Ar::is_zero(nr) || Ar::le(rem, Ar::mul(Ar::add(cn[j], rem), Ar::tau2()));
        if (skip) {
          fco[c] = Ar::zero();  // H = I
          if (c == j) misc[0] = 0;
          if (c > j) {
            V rjc = Ar::r_get(R[j * NC + c]);
            cn[c] = Ar::add(cn[c], Ar::mul(rjc, rjc));
          }
        } else {
          const bool neg = Ar::r_negative(x1r);  // s = sign(R_jj), sign(0) = +1
          const V a = neg ? Ar::neg(x1) : x1;
          const V q = Ar::recip(Ar::add(a, Ar::sqrt_(rem)));  // 1 / (a + ||x||)
          const V delta = Ar::mul(nr, q);                    // |beta| - a
          if (c == j) {
            const RT b = Ar::r_add(neg ? Ar::r_neg(x1r) : x1r, delta);  // |beta| = a + delta
            *beta_s = neg ? b : Ar::r_neg(b);  // beta = -s |beta|, written into R after the barrier
            misc[0] = 1;
          } else {
            const V ib = Ar::recip(Ar::add(a, delta));  // 1 / |beta|
            const RT rjcr = R[j * NC + c];
            const V rjc = Ar::r_get(rjcr);
            const V sdc = neg ? Ar::neg(d) : d;      // s d_c
            const V srjc = neg ? Ar::neg(rjc) : rjc;  // s R_jc
            const V corr = Ar::mul(Ar::sub(Ar::mul(delta, rjc), sdc), ib);
            R[j * NC + c] = Ar::r_add(Ar::r_neg(rjcr), corr);  // -R_jc + corr
            const V rn = Ar::sub(corr, rjc);
            cn[c] = Ar::add(cn[c], Ar::mul(rn, rn));
            fco[c] = Ar::mul(Ar::add(Ar::mul(d, q), srjc), ib);
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && misc[0]) R[j * NC + j] = *beta_s;
    // update my columns c > j
#pragma unroll
    for (int k = 0; k < NCT; ++k) {
      const int c = cg + k * TC;
      if (c > j) {
        V f = fco[c];
#pragma unroll
        for (int q = 0; q < RPT; ++q) w[q][k] = Ar::sub_mul(w[q][k], pv[q], f);
      }
    }
  }

  // Fold the register tile into R: the in-place trapezoidal Householder QR of [R; W]
  // (Algorithm 4, one reflector per column).
  QL_DEV void factor_tile(V (&w)[RPT][NCT], int n) {
#pragma unroll 1
    for (int j = 0; j < n; ++j) column_step(w, j);
  }

  // Process tiles [t0, t1) of problem p (tile t covers rows [row_base + t*B, ...)).
  QL_DEV void run(const TsqrProblem<S>& p, int64_t row_base, int64_t t0, int64_t t1) {
    constexpr int ST = Sh::STAGES;
    V w[RPT][NCT];
    if (t0 >= t1) return;
#pragma unroll
    for (int s = 0; s < ST; ++s) {  // prologue: ST tiles in flight (empty groups past the end)
      if (t0 + s < t1)
        issue_tile(p, row_base + (t0 + s) * B, s);
      else
        cp_async_commit();
    }
    for (int64_t t = t0; t < t1; ++t) {
      const int buf = (int)((t - t0) % ST);
      cp_async_wait_group<ST - 1>();  // this tile's group has landed
      __syncthreads();
      stage_to_regs(w, buf);
      for (int i = tid; i < NC; i += T) cn[i] = Ar::zero();
      __syncthreads();
      if (t + ST < t1)
        issue_tile(p, row_base + (t + ST) * B, buf);
      else
        cp_async_commit();
      factor_tile(w, p.n);
    }
    cp_async_wait_all();
    __syncthreads();
  }

  // Range verdict of this CTA (double-float policy): every nonzero column max exponent
  // must lie in [kDfEminLimit, df_emax_limit(m)] (the running column norms, formed in the
  // working arithmetic, reach sqrt(m) max|x|).
  QL_DEV bool out_of_range(int n, int64_t m) {
    if constexpr (!Ar::kRangeChecked) return false;
    const int emax = df_emax_limit(m);
    bool bad = false;
    for (int c = 0; c < n; ++c) {
      int e = colmax[c];
      if (e != 0 && (e < kDfEminLimit || e > emax)) bad = true;
    }
    return bad;
  }
};

// ---------------------------------------------------------------------------------------
// FP64 merge of stacked triangles: Ra <- R of [Ra; Rb_0; ...; Rb_{nb-1}] (n x n upper
// triangles in shared memory, ld NC; the Rb follow each other, NC x NC apart).  Column j's
// reflector touches Ra(j, :) and rows 0..j of every Rb (their untouched parts stay upper
// triangular), so nb + 1 triangles merge in n column steps, not nb n.  One thread per
// trailing column; remainders below kTauF64 of their column's norm are treated as rounding
// residue (no reflector), as in the tile factorisation.
// ---------------------------------------------------------------------------------------
constexpr double kTauF64Sq = 0x1p-92;  // (2^-46)^2

template <int NC, int T>
QL_DEV void merge_stack_f64(double* Ra, double* Rbs, int nb, int n, double* sd) {
  int tid = threadIdx.x;
  double* cnm = sd + NC;  // sum over finished rows i < j of Ra(i, c)^2
  for (int c = tid; c < NC; c += T) cnm[c] = 0.0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    double x1 = Ra[j * NC + j];
    for (int c = j + tid; c < n; c += T) {
      double s = 0.0;
      for (int b = 0; b < nb; ++b) {
        const double* Rb = Rbs + (size_t)b * NC * NC;
        for (int i = 0; i <= j; ++i) s = fma(Rb[i * NC + j], Rb[i * NC + c], s);
      }
      sd[c] = s;
    }
    __syncthreads();
    double nr = sd[j];
    double rem = fma(x1, x1, nr);
    bool skip = nr == 0.0 || rem <= kTauF64Sq * (cnm[j] + rem);
    if (!skip) {
      double nrm = sqrt(rem);
      double beta = x1 < 0.0 ? nrm : -nrm;
      double v1 = x1 - beta;
      double g = -1.0 / (beta * v1);
      for (int c = j + 1 + tid; c < n; c += T) {
        double f = fma(v1, Ra[j * NC + c], sd[c]) * g;
        double rn = fma(-v1, f, Ra[j * NC + c]);
        Ra[j * NC + c] = rn;
        cnm[c] = fma(rn, rn, cnm[c]);
        for (int b = 0; b < nb; ++b) {
          double* Rb = Rbs + (size_t)b * NC * NC;
          for (int i = 0; i <= j; ++i) Rb[i * NC + c] = fma(-Rb[i * NC + j], f, Rb[i * NC + c]);
        }
      }
      if (tid == 0) Ra[j * NC + j] = beta;
    } else {
      for (int c = j + 1 + tid; c < n; c += T) cnm[c] = fma(Ra[j * NC + c], Ra[j * NC + c], cnm[c]);
    }
    __syncthreads();
  }
}

// Copy an n x n triangle from global (ld n) into shared (ld NC), zero-padded to NC.
template <int NC, int T>
QL_DEV void load_tri(double* dst, const double* src, int n) {
  for (int i = threadIdx.x; i < NC * NC; i += T) {
    int r = i / NC, c = i % NC;
    dst[i] = (r < n && c < n && r <= c) ? __ldcg(src + (size_t)c * n + r) : 0.0;
  }
}
template <int NC, int T>
QL_DEV void store_tri(double* dst, const double* src, int n) {
  for (int i = threadIdx.x; i < n * n; i += T) {
    int c = i / n, r = i % n;
    __stcg(dst + i, r <= c ? src[r * NC + c] : 0.0);
  }
}

// Climb the A-ary R-tree from leaf `leaf`, whose triangle is already in slot(0, leaf).
// Node i of a level has the children A i .. A i + A - 1 of the level below; the last child
// CTA to arrive (one arrival counter per node) merges all of them and carries the result
// up.  Returns true in exactly one CTA (the root owner), with the final triangle in Ra
// (shared, ld NC).  `arena` holds Ra followed by room for A - 1 more triangles (A at most
// tree_arity<NC>(), which sizes it).  Slots of
// level l start at sum_{l' < l} width_l'; counters at sum_{l' < l} width_{l' + 1}.
template <int NC, int T>
QL_DEV bool climb_tree(const TreeView& tv, int leaf, int n, double* arena, double* sd, int* s_flag, int A) {
  double* Ra = arena;
  double* Rbs = arena + NC * NC;
  __syncthreads();  // the leaf slot was written by all threads of this CTA
  int width = tv.leaves, idx = leaf;
  size_t slot_base = 0, cnt_base = 0;
  if (width == 1) {
    load_tri<NC, T>(Ra, tv.slots, n);
    __syncthreads();
    return true;
  }
  while (width > 1) {
    const int parent = idx / A, first = parent * A;
    const int cnt = min(A, width - first);
    const int next_width = (width + A - 1) / A;
    if (cnt > 1) {
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        int old = atomicAdd(&tv.counters[cnt_base + parent], 1);
        *s_flag = old;
        if (old == cnt - 1) tv.counters[cnt_base + parent] = 0;  // reset for the next call
      }
      __syncthreads();
      if (*s_flag != cnt - 1) return false;  // a sibling merges
      __threadfence();
      const double* c0 = tv.slots + (slot_base + (size_t)first) * (size_t)n * n;
      load_tri<NC, T>(Ra, c0, n);
      for (int b = 1; b < cnt; ++b) load_tri<NC, T>(Rbs + (size_t)(b - 1) * NC * NC, c0 + (size_t)b * n * n, n);
      __syncthreads();
      merge_stack_f64<NC, T>(Ra, Rbs, cnt - 1, n, sd);
    } else {
      load_tri<NC, T>(Ra, tv.slots + (slot_base + (size_t)idx) * (size_t)n * n, n);
      __syncthreads();
    }
    cnt_base += (size_t)next_width;
    slot_base += (size_t)width;
    width = next_width;
    idx = parent;
    if (width > 1) {
      store_tri<NC, T>(tv.slots + (slot_base + (size_t)idx) * (size_t)n * n, Ra, n);
      __syncthreads();
    }
  }
  return true;
}

// Tree sizes for `leaves` leaves and arity A: total slots and counters.  Arity 2 bounds
// every larger arity (the workspace is sized with it).
inline size_t tree_slots(int leaves, int A = 2) {
  size_t s = 0;
  for (int w = leaves;; w = (w + A - 1) / A) {
    s += (size_t)w;
    if (w <= 1) break;
  }
  return s;
}
inline size_t tree_counters(int leaves, int A = 2) {
  size_t s = 0;
  for (int w = leaves; w > 1; w = (w + A - 1) / A) s += (size_t)((w + A - 1) / A);
  return s + 1;
}

}  // namespace ql
