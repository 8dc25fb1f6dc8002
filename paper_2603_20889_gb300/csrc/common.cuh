// Shared device building blocks of the qless kernels: double-float arithmetic, the two
// arithmetic policies (double-float on the FP32 pipes, native FP64), cp.async staging and
// the small FP64 n x n routines that run inside the "last CTA done" epilogues.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "../../include/qless.h"

#define QL_DEV __device__ __forceinline__

namespace ql {

constexpr int kMaxN = 64;

// ---------------------------------------------------------------------------------------
// Double-float ("df"): value = hi + lo with |lo| <= ulp(hi).  Error-free transformations
// use the _rn intrinsics so that nvcc never contracts or reassociates them.
//   two_sum (Knuth), fast_two_sum (Dekker, |a| >= |b|), two_prod via FMA.
// ---------------------------------------------------------------------------------------
struct df {
  float hi, lo;
};

QL_DEV void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
QL_DEV void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
QL_DEV df df_make(float hi, float lo) {
  df r;
  fast_two_sum(hi, lo, r.hi, r.lo);
  return r;
}
QL_DEV df df_add(df a, df b) {  // "sloppy" sum: absolute error ~ u^2 (|a| + |b|)
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_make(s, e);
}
QL_DEV df df_neg(df a) { return df{-a.hi, -a.lo}; }
QL_DEV df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
// Products keep the lo * lo term: it is below 2^-48 of the product but has a fixed sign for
// squares (a dropped lo^2 biases every sum of squares low by about 2^-50).
QL_DEV df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.lo, e));
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_make(p, e);
}
// a - b * c, one renormalisation.  Used for updates w -= v f whose b.lo * c.lo term changes
// sign with the row (v.lo), so it is left out (it would only add cost, not remove a bias).
QL_DEV df df_sub_mul(df a, df b, df c) {
  float p = __fmul_rn(b.hi, c.hi);
  float e = __fmaf_rn(b.hi, c.hi, -p);
  e = __fmaf_rn(b.hi, c.lo, e);
  e = __fmaf_rn(b.lo, c.hi, e);
  float s, t;
  two_sum(a.hi, -p, s, t);
  t = __fadd_rn(t, __fsub_rn(a.lo, e));
  return df_make(s, t);
}
// 1 / b from the float reciprocal q and r = 1 - q b: 1 / b = q (1 + r + r^2 + ...).  The
// second-order term q r^2 is kept: one Newton step alone always falls short (by q r^2 >= 0,
// about 2^-50 on average), a one-signed error that would accumulate over many updates.
QL_DEV df df_recip(df b) {
  float q = __fdiv_rn(1.0f, b.hi);
  float p = __fmul_rn(q, b.hi);
  float e = __fmaf_rn(q, b.hi, -p);
  e = __fmaf_rn(q, b.lo, e);
  float r = __fsub_rn(__fsub_rn(1.0f, p), e);  // 1 - q b
  return df_make(q, __fmul_rn(__fmaf_rn(r, r, r), q));
}
// sqrt(a), a >= 0: sqrtf plus the series correction d - d^2 / (2 s), d = r / (2 s),
// r = a - s^2 (one Newton step alone always overshoots by about d^2 / (2 s)).
QL_DEV df df_sqrt(df a) {
  if (a.hi <= 0.0f) return df{0.0f, 0.0f};
  float s = __fsqrt_rn(a.hi);
  float p = __fmul_rn(s, s);
  float e = __fmaf_rn(s, s, -p);
  float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);
  float is2 = __fdiv_rn(0.5f, s);
  float d = __fmul_rn(r, is2);
  return df_make(s, __fmaf_rn(-__fmul_rn(d, d), is2, d));
}
QL_DEV double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
QL_DEV df df_from_double_rn(double x) {  // used only on n x n data
  float hi = __double2float_rn(x);
  float lo = __double2float_rn(x - (double)hi);
  return df{hi, lo};
}

// Split an IEEE double into a double-float without the FP64 pipe (the scarce resource on
// this GPU): hi = the top 24 significand bits (truncated, built with integer operations),
// lo = the remaining 29 bits converted to float with rounding, so |x - (hi + lo)| <=
// 2^-48 |x|.  Doubles outside [2^-103, 2^127) give 0 (the range check rejects them); the
// biased exponent E of x is returned for that check.
QL_DEV df df_split_double(double x, int& E) {
  unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  unsigned int hw = (unsigned int)(bits >> 32), lw = (unsigned int)bits;
  unsigned int sign = hw & 0x80000000u;
  E = (int)((hw >> 20) & 0x7ffu);
  if (E < 920 || E > 1150) return df{0.0f, 0.0f};
  unsigned int hb = sign | ((unsigned int)(E - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
  float scale = __int_as_float((int)((unsigned int)(E - 919) << 23));  // 2^(E - 1046)
  float lo = __fmul_rn(__fmul_rn(__uint2float_rn(lw & 0x1fffffffu), 1.862645149230957e-09f), scale);
  df r;
  r.hi = __int_as_float((int)hb);
  r.lo = sign ? -lo : lo;
  return r;
}

// Triple-float ("tf"): value = hi + mid + lo, about 72 significant bits, built from the
// same error-free transformations.  Used for values carried across many updates (the
// running TSQR triangle), where double-float rounding would accumulate.
struct tf {
  float hi, mid, lo;
};
QL_DEV tf tf_neg(tf a) { return tf{-a.hi, -a.mid, -a.lo}; }
QL_DEV df tf_to_df(tf a) { return df{a.hi, a.mid}; }
QL_DEV double tf_to_double(tf a) { return ((double)a.hi + (double)a.mid) + (double)a.lo; }
// a + b (tf + df): exact two-sums of the leading parts, the third-order terms (below
// 2^-48 of the result) summed in FP32, then renormalised; error about 2^-72 |a + b|.
QL_DEV tf tf_add_df(tf a, df b) {
  float s0, e0, s1, e1, s2, e2, h, u, m, l;
  two_sum(a.hi, b.hi, s0, e0);
  two_sum(a.mid, b.lo, s1, e1);
  two_sum(s1, e0, s2, e2);
  const float t = __fadd_rn(__fadd_rn(e1, e2), a.lo);
  two_sum(s0, s2, h, u);
  two_sum(u, t, m, l);
  return tf{h, m, l};
}

QL_DEV df shfl_xor(df a, int mask) {
  return df{__shfl_xor_sync(0xffffffffu, a.hi, mask), __shfl_xor_sync(0xffffffffu, a.lo, mask)};
}

// ---------------------------------------------------------------------------------------
// Arithmetic policies.  T is the working element; Acc an unnormalised dot-product
// accumulator; load() converts one stored element and reports its biased IEEE-double
// exponent in E for the range check (only the double-float policy needs it).
// ---------------------------------------------------------------------------------------
struct ArithDF {
  using T = df;
  struct Acc {
    float hi, lo;
  };
  static constexpr bool kRangeChecked = true;
  QL_DEV static T zero() { return df{0.0f, 0.0f}; }
  // Convert one stored element; E receives its biased IEEE-double exponent (0 for zero).
  QL_DEV static T load(double x, int& E) { return df_split_double(x, E); }
  QL_DEV static T load(float x, int& E) {
    int e = (__float_as_int(x) >> 23) & 0xff;
    E = e == 0 ? 0 : e + 896;  // rebias to the double exponent scale
    return e == 0 ? df{0.0f, 0.0f} : df{x, 0.0f};
  }
  QL_DEV static Acc acc_zero() { return Acc{0.0f, 0.0f}; }
  QL_DEV static void acc_fma(Acc& acc, T a, T b) {  // acc += a * b (lo * lo kept, see df_mul)
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.lo, e));
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    two_sum(acc.hi, p, s, t);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
  }
  QL_DEV static T acc_get(Acc a) { return df_make(a.hi, a.lo); }
  QL_DEV static T add(T a, T b) { return df_add(a, b); }
  QL_DEV static T sub(T a, T b) { return df_sub(a, b); }
  QL_DEV static T mul(T a, T b) { return df_mul(a, b); }
  QL_DEV static T sub_mul(T a, T b, T c) { return df_sub_mul(a, b, c); }
  QL_DEV static T recip(T a) { return df_recip(a); }
  QL_DEV static T sqrt_(T a) { return df_sqrt(a); }
  QL_DEV static T neg(T a) { return df_neg(a); }
  QL_DEV static bool is_zero(T a) { return a.hi == 0.0f; }
  QL_DEV static bool negative(T a) { return a.hi < 0.0f; }
  QL_DEV static bool le(T a, T b) { return a.hi <= b.hi; }  // approximate order suffices
  QL_DEV static T tau2() { return df{0x1p-80f, 0.0f}; }      // (2^-40)^2: negligible remainder
  QL_DEV static double to_double(T a) { return df_to_double(a); }
  QL_DEV static T from_double(double x) { return df_from_double_rn(x); }
  QL_DEV static T shfl(T a, int mask) { return shfl_xor(a, mask); }
  // Values carried across tiles (the running TSQR triangle): triple-float, so that their
  // many small updates round at about 2^-72 instead of double-float's 2^-48.
  using RT = tf;
  QL_DEV static RT r_zero() { return tf{0.0f, 0.0f, 0.0f}; }
  QL_DEV static T r_get(RT r) { return tf_to_df(r); }
  QL_DEV static bool r_negative(RT r) { return r.hi < 0.0f; }
  QL_DEV static RT r_neg(RT r) { return tf_neg(r); }
  QL_DEV static RT r_add(RT r, T c) { return tf_add_df(r, c); }  // r + c
  QL_DEV static double r_to_double(RT r) { return tf_to_double(r); }
};

struct ArithF64 {
  using T = double;
  using Acc = double;
  static constexpr bool kRangeChecked = false;
  QL_DEV static T zero() { return 0.0; }
  QL_DEV static T load(double x, int& E) {
    E = 0;
    return x;
  }
  QL_DEV static T load(float x, int& E) {
    E = 0;
    return (double)x;
  }
  QL_DEV static Acc acc_zero() { return 0.0; }
  QL_DEV static void acc_fma(Acc& acc, T a, T b) { acc = fma(a, b, acc); }
  QL_DEV static T acc_get(Acc a) { return a; }
  QL_DEV static T add(T a, T b) { return a + b; }
  QL_DEV static T sub(T a, T b) { return a - b; }
  QL_DEV static T mul(T a, T b) { return a * b; }
  QL_DEV static T sub_mul(T a, T b, T c) { return fma(-b, c, a); }
  QL_DEV static T recip(T a) { return 1.0 / a; }
  QL_DEV static T sqrt_(T a) { return a > 0.0 ? sqrt(a) : 0.0; }
  QL_DEV static T neg(T a) { return -a; }
  QL_DEV static bool is_zero(T a) { return a == 0.0; }
  QL_DEV static bool negative(T a) { return a < 0.0; }
  QL_DEV static bool le(T a, T b) { return a <= b; }
  QL_DEV static T tau2() { return 0x1p-92; }  // (2^-46)^2: negligible remainder
  QL_DEV static double to_double(T a) { return a; }
  QL_DEV static T from_double(double x) { return x; }
  QL_DEV static T shfl(T a, int mask) { return __shfl_xor_sync(0xffffffffu, a, mask); }
  using RT = double;
  QL_DEV static RT r_zero() { return 0.0; }
  QL_DEV static T r_get(RT r) { return r; }
  QL_DEV static bool r_negative(RT r) { return r < 0.0; }
  QL_DEV static RT r_neg(RT r) { return -r; }
  QL_DEV static RT r_add(RT r, T c) { return r + c; }
  QL_DEV static double r_to_double(RT r) { return r; }
};

// Range accepted by the double-float kernels: every nonzero block-column maximum |x| in
// [2^-40, 2^50] (biased double exponents 983..1073); the per-thread minimum exponent is
// only used to detect columns whose block maximum is tiny.
constexpr int kDfEmaxLimit = 1023 + 50;
constexpr int kDfEminLimit = 1023 - 40;
// Kernels whose double-float values include sums of squares over all m rows (column norms
// and Gram entries, up to m max|x|^2) also need m 2^(2 (e + 1)) <= 2^124 for a biased
// exponent limit 1023 + e: the upper limit drops by half a binade per doubling of m
// (e = 48 at m = 2^25, 47 at m = 2^28) and stays at most 50.
__host__ __device__ inline int df_emax_limit(int64_t m) {
  int bits = 0;
  while (bits < 62 && ((int64_t)1 << bits) < m) ++bits;  // ceil(log2 m)
  const int e = (122 - bits) / 2;
  return 1023 + (e < 50 ? e : 50);
}

// ---------------------------------------------------------------------------------------
// cp.async staging (Ampere-style per-thread async copies; any element-aligned address).
// ---------------------------------------------------------------------------------------
template <int I, int N, typename F>
QL_DEV void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

QL_DEV unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

QL_DEV void cp_async_8(void* smem, const void* gmem, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_addr(smem)), "l"(gmem),
               "r"(valid ? 8 : 0));
}
QL_DEV void cp_async_4(void* smem, const void* gmem, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr(smem)), "l"(gmem),
               "r"(valid ? 4 : 0));
}
// 16-byte copy (both addresses 16-byte aligned) of which the first src_bytes (0..16) are
// read and the rest zero-filled.
QL_DEV void cp_async_16(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(smem)), "l"(gmem), "r"(src_bytes));
}
QL_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
QL_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <int N>
QL_DEV void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename S>
QL_DEV void cp_async_elem(S* smem, const S* gmem, bool valid);
template <>
QL_DEV void cp_async_elem<double>(double* smem, const double* gmem, bool valid) {
  cp_async_8(smem, gmem, valid);
}
template <>
QL_DEV void cp_async_elem<float>(float* smem, const float* gmem, bool valid) {
  cp_async_4(smem, gmem, valid);
}

// Column pointer of the logical matrix [A b]: columns < nA come from A (ld lda), column nA
// (if any) from the vector b.  Used so least squares reads [A b] in place.
template <typename S>
struct ColSource {
  const S* A;
  int64_t lda;
  const S* b;
  int nA;
  QL_DEV const S* col(int c) const { return c < nA ? A + (int64_t)c * lda : b; }
};

}  // namespace ql
