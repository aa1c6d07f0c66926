// Device-side double-double (DD) and quad-double (QD) arithmetic.
//
// A DD number is an unevaluated sum hi + lo of two doubles and a QD number an
// unevaluated sum of four (Kouya 2015, Section 1: "two or four connected
// double precision floating-point numbers"). Every operation below is spelled
// with explicit round-to-nearest intrinsics so that nvcc can neither contract
// a product and a sum into an FMA nor reassociate: the operation sequences
// are pinned, and the Simple kernels that use them reproduce a plain CPU
// restatement of the same sequences bit for bit.
//
// Published algorithms used:
//   TwoSum (Knuth, TAOCP vol. 2) and FastTwoSum (Dekker 1971): s + e = a + b
//     exactly;
//   TwoProd with FMA: p + e = a * b exactly (no underflow);
//   DD product: TwoProd of the leading limbs, both cross products folded into
//     the error by FMA, FastTwoSum renormalisation;
//   DD sum: accurate double-word addition (Joldes, Muller, Popescu 2017),
//     relative error <= 3 u^2;
//   QD sum: limbs merged by decreasing magnitude, then renormalisation by
//     VecSum and a compaction pass (Joldes, Marty, Muller, Popescu 2016);
//   QD product: limb products of order <= 2 by TwoProd, order-3 terms summed
//     plainly (the orders kept by Hida, Li, Bailey 2001), the terms sorted
//     by decreasing magnitude, then the same renormalisation;
//   QD quotient: long division, five double digits.
#pragma once

#include <cstdint>

namespace ddg {

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  double bv = __dsub_rn(s, a);
  double av = __dsub_rn(s, bv);
  e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  e = __dsub_rn(b, __dsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  p = __dmul_rn(a, b);
  e = __fma_rn(a, b, -p);
}

struct dd_t {
  double hi, lo;
};

__device__ __forceinline__ dd_t dd_mul(dd_t a, dd_t b) {
  double p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fma_rn(a.hi, b.lo, e);
  e = __fma_rn(a.lo, b.hi, e);
  dd_t r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dd_t dd_add(dd_t a, dd_t b) {
  double sh, sl, th, tl;
  two_sum(a.hi, b.hi, sh, sl);
  two_sum(a.lo, b.lo, th, tl);
  sl = __dadd_rn(sl, th);
  fast_two_sum(sh, sl, sh, sl);
  sl = __dadd_rn(sl, tl);
  dd_t r;
  fast_two_sum(sh, sl, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dd_t dd_neg(dd_t a) { return dd_t{-a.hi, -a.lo}; }

// DD quotient a / b by long division: three double quotient digits, each
// remainder formed with the DD product and sum above (relative error a few
// units of 2^-104).
__device__ __forceinline__ dd_t dd_div(dd_t a, dd_t b) {
  const double q1 = __ddiv_rn(a.hi, b.hi);
  dd_t r = dd_add(a, dd_mul(dd_t{-q1, 0.0}, b));
  const double q2 = __ddiv_rn(r.hi, b.hi);
  r = dd_add(r, dd_mul(dd_t{-q2, 0.0}, b));
  const double q3 = __ddiv_rn(r.hi, b.hi);
  dd_t q;
  fast_two_sum(q1, q2, q.hi, q.lo);
  return dd_add(q, dd_t{q3, 0.0});
}

// 1 / b in DD by one Newton step from the double reciprocal y0: with
// r = 1 - b y0 (two FMAs; |r| <= 2^-52), 1 / b = y0 (1 + r + r^2 + ...), so
// y0 + y0 r (1 + r) is accurate to ~2^-105. Short dependency chain: a
// GB300 SM issues a single thread's FP64 instructions slowly, and the LU's
// pivot reciprocal sits on its critical path.
__device__ __forceinline__ dd_t dd_recip(dd_t b) {
  const double y0 = __ddiv_rn(1.0, b.hi);
  double r = __fma_rn(-b.hi, y0, 1.0);
  r = __fma_rn(-b.lo, y0, r);
  const double c = __dmul_rn(y0, r);
  dd_t y;
  fast_two_sum(y0, __fma_rn(c, r, c), y.hi, y.lo);
  return y;
}

// |a| > |b| as DD numbers (compares hi, then the lo of the same sign).
__device__ __forceinline__ bool dd_abs_greater(dd_t a, dd_t b) {
  const double ah = fabs(a.hi), bh = fabs(b.hi);
  const double al = a.hi < 0.0 ? -a.lo : a.lo;
  const double bl = b.hi < 0.0 ? -b.lo : b.lo;
  return ah > bh || (ah == bh && al > bl);
}

struct qd_t {
  double x[4];
};

// VecSum from the last (smallest) term up, then a top-down compaction that
// emits a limb each time the running TwoSum leaves a nonzero error. N is a
// compile-time count so that the term array stays in registers.
template <int N>
__device__ __forceinline__ qd_t qd_renorm(const double (&x)[N]) {
  double t[N];
  double s = x[N - 1];
#pragma unroll
  for (int i = N - 2; i >= 0; --i) two_sum(x[i], s, s, t[i + 1]);
  t[0] = s;
  qd_t r;
  r.x[0] = r.x[1] = r.x[2] = r.x[3] = 0.0;
  int k = 0;
  s = t[0];
#pragma unroll
  for (int i = 1; i < N; ++i) {
    double s2, e;
    two_sum(s, t[i], s2, e);
    if (k < 4) {
      if (e != 0.0) {
        // a limb is complete
        if (k == 0) r.x[0] = s2;
        else if (k == 1) r.x[1] = s2;
        else if (k == 2) r.x[2] = s2;
        else r.x[3] = s2;
        ++k;
        s = e;
      } else {
        s = s2;
      }
    }
  }
  if (k < 4) {
    if (k == 0) r.x[0] = s;
    else if (k == 1) r.x[1] = s;
    else if (k == 2) r.x[2] = s;
    else r.x[3] = s;
  }
  return r;
}

__device__ __forceinline__ qd_t qd_add(const qd_t& a, const qd_t& b) {
  double m[8];
  int i = 0, j = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    double ai = i == 0 ? a.x[0] : i == 1 ? a.x[1] : i == 2 ? a.x[2] : a.x[3];
    double bj = j == 0 ? b.x[0] : j == 1 ? b.x[1] : j == 2 ? b.x[2] : b.x[3];
    bool take_a = (j == 4) || (i < 4 && fabs(ai) >= fabs(bj));
    m[t] = take_a ? ai : bj;
    if (take_a) ++i; else ++j;
  }
  return qd_renorm<8>(m);
}

// Stable sort by decreasing magnitude: odd-even transposition (N rounds of
// adjacent compare-exchanges that swap only on a strictly larger magnitude,
// so equal magnitudes keep their order). The keys are the magnitude bits,
// compared as integers, so the sort runs on the integer pipe. The product's
// terms are listed by order (i + j of a_i b_j); a limb far below its
// position (a QD number close to a short one, e.g. an integer plus a tiny
// correction) puts tiny terms among larger ones, and the renormalisation
// below needs them in decreasing order to keep four full limbs.
template <int N>
__device__ __forceinline__ void sort_by_magnitude(double (&t)[N]) {
  unsigned long long k[N];
#pragma unroll
  for (int i = 0; i < N; ++i) k[i] = (unsigned long long)__double_as_longlong(t[i]) & 0x7FFFFFFFFFFFFFFFull;
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int i = r & 1; i + 1 < N; i += 2)
      if (k[i + 1] > k[i]) {
        const unsigned long long kk = k[i];
        k[i] = k[i + 1];
        k[i + 1] = kk;
        const double tt = t[i];
        t[i] = t[i + 1];
        t[i + 1] = tt;
      }
}

__device__ __forceinline__ qd_t qd_mul(const qd_t& a, const qd_t& b) {
  double p00, q00, p01, q01, p10, q10, p02, q02, p11, q11, p20, q20;
  two_prod(a.x[0], b.x[0], p00, q00);
  two_prod(a.x[0], b.x[1], p01, q01);
  two_prod(a.x[1], b.x[0], p10, q10);
  two_prod(a.x[0], b.x[2], p02, q02);
  two_prod(a.x[1], b.x[1], p11, q11);
  two_prod(a.x[2], b.x[0], p20, q20);
  double o3 = __dmul_rn(a.x[0], b.x[3]);
  o3 = __fma_rn(a.x[1], b.x[2], o3);
  o3 = __fma_rn(a.x[2], b.x[1], o3);
  o3 = __fma_rn(a.x[3], b.x[0], o3);
  o3 = __dadd_rn(o3, q02);
  o3 = __dadd_rn(o3, q11);
  o3 = __dadd_rn(o3, q20);
  double t[10] = {p00, p01, p10, q00, p02, p11, p20, q01, q10, o3};
  sort_by_magnitude(t);
  return qd_renorm<10>(t);
}

__device__ __forceinline__ qd_t qd_neg(const qd_t& a) {
  return qd_t{{-a.x[0], -a.x[1], -a.x[2], -a.x[3]}};
}

// QD quotient a / b by long division: five double quotient digits, each
// remainder formed with the QD product and sum above, renormalised.
__device__ __forceinline__ qd_t qd_div(const qd_t& a, const qd_t& b) {
  double q[5];
  qd_t r = a;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    q[k] = __ddiv_rn(r.x[0], b.x[0]);
    r = qd_add(r, qd_neg(qd_mul(qd_t{{q[k], 0.0, 0.0, 0.0}}, b)));
  }
  q[4] = __ddiv_rn(r.x[0], b.x[0]);
  return qd_renorm<5>(q);
}

// 1 / b in QD: the DD reciprocal y1 (~2^-105), then one Newton step in QD:
// e = 1 - b y1 (QD product and sum; |e| ~ 2^-105, accurate to ~2^-210),
// 1 / b = y1 (1 + e + e^2 + ...) ~ y1 + y1 e + y1 e0^2. About a quarter of
// the instructions of the long division.
__device__ __forceinline__ qd_t qd_recip(const qd_t& b) {
  const dd_t y1 = dd_recip(dd_t{b.x[0], b.x[1]});
  const qd_t p = qd_mul(b, qd_t{{y1.hi, y1.lo, 0.0, 0.0}});
  const qd_t e = qd_add(qd_t{{1.0, 0.0, 0.0, 0.0}}, qd_neg(p));
  const dd_t c = dd_mul(y1, dd_t{e.x[0], e.x[1]});
  const double c2 = __dmul_rn(c.hi, e.x[0]);
  const double t[5] = {y1.hi, y1.lo, c.hi, c.lo, c2};
  return qd_renorm<5>(t);
}

// ---------------------------------------------------------------------------
// Limb-generic wrappers so that kernels can be written once for DD and QD.
template <int L> struct num;
template <> struct num<2> {
  using T = dd_t;
  static __device__ __forceinline__ T zero() { return dd_t{0.0, 0.0}; }
  static __device__ __forceinline__ T add(const T& a, const T& b) { return dd_add(a, b); }
  static __device__ __forceinline__ T mul(const T& a, const T& b) { return dd_mul(a, b); }
  static __device__ __forceinline__ T neg(const T& a) { return dd_neg(a); }
  static __device__ __forceinline__ T div(const T& a, const T& b) { return dd_div(a, b); }
  static __device__ __forceinline__ T recip(const T& b) { return dd_recip(b); }
  static __device__ __forceinline__ T one() { return dd_t{1.0, 0.0}; }
  static __device__ __forceinline__ double lead(const T& a) { return a.hi; }
  static __device__ __forceinline__ double second(const T& a) { return a.lo; }
  static __device__ __forceinline__ T load(const double* const* p, int64_t off) {
    return dd_t{p[0][off], p[1][off]};
  }
  static __device__ __forceinline__ void store(double* const* p, int64_t off, const T& v) {
    p[0][off] = v.hi;
    p[1][off] = v.lo;
  }
};
template <> struct num<4> {
  using T = qd_t;
  static __device__ __forceinline__ T zero() { return qd_t{{0.0, 0.0, 0.0, 0.0}}; }
  static __device__ __forceinline__ T add(const T& a, const T& b) { return qd_add(a, b); }
  static __device__ __forceinline__ T mul(const T& a, const T& b) { return qd_mul(a, b); }
  static __device__ __forceinline__ T neg(const T& a) { return qd_neg(a); }
  static __device__ __forceinline__ T div(const T& a, const T& b) { return qd_div(a, b); }
  static __device__ __forceinline__ T recip(const T& b) { return qd_recip(b); }
  static __device__ __forceinline__ T one() { return qd_t{{1.0, 0.0, 0.0, 0.0}}; }
  static __device__ __forceinline__ double lead(const T& a) { return a.x[0]; }
  static __device__ __forceinline__ double second(const T& a) { return a.x[1]; }
  static __device__ __forceinline__ T load(const double* const* p, int64_t off) {
    return qd_t{{p[0][off], p[1][off], p[2][off], p[3][off]}};
  }
  static __device__ __forceinline__ void store(double* const* p, int64_t off, const T& v) {
    p[0][off] = v.x[0];
    p[1][off] = v.x[1];
    p[2][off] = v.x[2];
    p[3][off] = v.x[3];
  }
};

}  // namespace ddg
