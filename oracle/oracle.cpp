// CPU oracle for double-double (DD) and quad-double (QD) matrix products.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
// load this file; only the tests, the smoke check and the benchmark's CPU
// baseline do. It shares no code, header or constant table with the CUDA
// library.
//
// What it computes (Kouya 2015, "Performance evaluation of multiple precision
// matrix multiplications using parallelized Strassen and Winograd
// algorithms"):
//   * Section 2, Eq. 1 ("Simple"): c_ij = sum_{k=1..l} a_ik b_kj, taken as a
//     plain triple loop, c_ij starting from 0 (or from C for the update
//     modes), k ascending, one DD/QD multiply then one DD/QD add per term.
//   * DD and QD numbers (Section 1: two or four connected doubles). The
//     paper uses the QD library's dd_real / qd_real; their operation
//     sequences are not printed in the paper, so the sequences below are the
//     published error-free-transformation algorithms, written from their
//     definitions:
//       TwoSum (Knuth, TAOCP vol. 2), FastTwoSum (Dekker 1971),
//       TwoProd via FMA (exact product error),
//       DD product: leading TwoProd, both cross products folded in by FMA,
//         FastTwoSum renormalisation (the low*low term is dropped);
//       DD sum: the accurate double-word addition (two TwoSums, two
//         FastTwoSum renormalisations; Joldes, Muller, Popescu 2017);
//       QD sum: the eight limbs merged by decreasing magnitude, then an
//         expansion renormalisation (VecSum followed by a compaction pass,
//         Joldes, Marty, Muller, Popescu 2016);
//       QD product: all limb products of order <= 2 (in units of the limb
//         spacing) by TwoProd, order-3 products and errors summed plainly,
//         the terms sorted by decreasing magnitude, then the same
//         renormalisation (Hida, Li, Bailey 2001 keep the same orders).
//   * An exact checker: a Kulisch-style long accumulator that forms every
//     limb product exactly (integer significands, __int128) and returns, per
//     output entry, the exact error (C_exact - C_computed) rounded to double.
//   * An exact residual checker b - A x for the Section 4 linear systems
//     (DD or QD) and unblocked DD and QD LU with partial pivoting for
//     reference solutions (QD quotients by long division).
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fno-fast-math (every
// product and sum below must round exactly once; fma is always spelled out).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>
#include <algorithm>

namespace {

// ---------------------------------------------------------------- EFTs ----
inline void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  double bv = s - a;
  double av = s - bv;
  e = (a - av) + (b - bv);
}
inline void fast_two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  e = b - (s - a);
}
inline void two_prod(double a, double b, double& p, double& e) {
  p = a * b;
  e = std::fma(a, b, -p);
}

// ------------------------------------------------------------------ DD ----
struct dd { double hi, lo; };

inline dd dd_mul(dd a, dd b) {
  double p, e;
  two_prod(a.hi, b.hi, p, e);
  e = std::fma(a.hi, b.lo, e);
  e = std::fma(a.lo, b.hi, e);
  dd r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

inline dd dd_add(dd a, dd b) {
  double sh, sl, th, tl;
  two_sum(a.hi, b.hi, sh, sl);
  two_sum(a.lo, b.lo, th, tl);
  sl = sl + th;
  fast_two_sum(sh, sl, sh, sl);
  sl = sl + tl;
  dd r;
  fast_two_sum(sh, sl, r.hi, r.lo);
  return r;
}

// ------------------------------------------------------------------ QD ----
struct qd { double x[4]; };

// Renormalise an n-term expansion (roughly decreasing magnitudes) to 4 limbs:
// VecSum from the smallest term up (error-free), then a top-down compaction
// that emits a limb whenever the running TwoSum leaves a nonzero error.
inline qd renorm(const double* x, int n) {
  double t[16];
  double s = x[n - 1];
  for (int i = n - 2; i >= 0; --i) two_sum(x[i], s, s, t[i + 1]);
  t[0] = s;
  qd r{{0.0, 0.0, 0.0, 0.0}};
  int k = 0;
  s = t[0];
  for (int i = 1; i < n; ++i) {
    double s2, e;
    two_sum(s, t[i], s2, e);
    if (e != 0.0) {
      r.x[k++] = s2;
      if (k == 4) return r;
      s = e;
    } else {
      s = s2;
    }
  }
  r.x[k] = s;
  return r;
}

inline qd qd_add(const qd& a, const qd& b) {
  double m[8];
  int i = 0, j = 0;
  for (int t = 0; t < 8; ++t) {
    if (j == 4 || (i < 4 && std::fabs(a.x[i]) >= std::fabs(b.x[j]))) m[t] = a.x[i++];
    else m[t] = b.x[j++];
  }
  return renorm(m, 8);
}

inline qd qd_mul(const qd& a, const qd& b) {
  double p00, q00, p01, q01, p10, q10, p02, q02, p11, q11, p20, q20;
  two_prod(a.x[0], b.x[0], p00, q00);
  two_prod(a.x[0], b.x[1], p01, q01);
  two_prod(a.x[1], b.x[0], p10, q10);
  two_prod(a.x[0], b.x[2], p02, q02);
  two_prod(a.x[1], b.x[1], p11, q11);
  two_prod(a.x[2], b.x[0], p20, q20);
  double o3 = a.x[0] * b.x[3];
  o3 = std::fma(a.x[1], b.x[2], o3);
  o3 = std::fma(a.x[2], b.x[1], o3);
  o3 = std::fma(a.x[3], b.x[0], o3);
  o3 = o3 + q02;
  o3 = o3 + q11;
  o3 = o3 + q20;
  double t[10] = {p00, p01, p10, q00, p02, p11, p20, q01, q10, o3};
  // decreasing magnitude, ties in the order above (a limb far below its
  // position would otherwise leave tiny terms among larger ones)
  std::stable_sort(t, t + 10, [](double x, double y) { return std::fabs(x) > std::fabs(y); });
  return renorm(t, 10);
}

// ------------------------------------------------------------ threading ---
template <class F>
void parallel_for(int64_t count, int nthreads, F f) {
  if (nthreads <= 1 || count < 2) {
    for (int64_t i = 0; i < count; ++i) f(i);
    return;
  }
  if (nthreads > count) nthreads = (int)count;
  std::vector<std::thread> th;
  th.reserve(nthreads);
  for (int t = 0; t < nthreads; ++t) {
    th.emplace_back([=]() {
      for (int64_t i = t; i < count; i += nthreads) f(i);
    });
  }
  for (auto& x : th) x.join();
}

// ------------------------------------------------------------- Kulisch ----
// Long fixed-point accumulator: digit d holds bits [32 d, 32 d + 32) of the
// value scaled by 2^-EMIN. Digits are signed 64-bit and carries are resolved
// only when the value is read, so each digit absorbs 2^31 additions.
struct Kulisch {
  static constexpr int EMIN = -2240;  // below the smallest product of doubles
  static constexpr int ND = 142;      // 4544 bits: covers every double product
  int64_t w[ND];
  Kulisch() { std::memset(w, 0, sizeof(w)); }

  static inline void decode(double x, uint64_t& m, int& e, bool& neg) {
    uint64_t bits;
    std::memcpy(&bits, &x, 8);
    neg = (bits >> 63) != 0;
    int be = (int)((bits >> 52) & 0x7FF);
    uint64_t frac = bits & ((uint64_t(1) << 52) - 1);
    if (be == 0) { m = frac; e = -1074; }
    else { m = frac | (uint64_t(1) << 52); e = be - 1075; }
  }
  // add sign * v * 2^e, v < 2^107
  inline void add_scaled(unsigned __int128 v, int e, bool neg) {
    if (v == 0) return;
    int pos = e - EMIN;
    int d = pos >> 5, r = pos & 31;
    // v << r spans at most 139 bits: five digits
    unsigned __int128 lo = v << r;                // bits 0..127 of v << r
    uint64_t top = r ? (uint64_t)(v >> (128 - r)) : 0;  // bits 128.. of v << r
    int64_t s = neg ? -1 : 1;
    w[d] += s * (int64_t)(uint32_t)(lo);
    w[d + 1] += s * (int64_t)(uint32_t)(lo >> 32);
    w[d + 2] += s * (int64_t)(uint32_t)(lo >> 64);
    w[d + 3] += s * (int64_t)(uint32_t)(lo >> 96);
    w[d + 4] += s * (int64_t)(uint32_t)(top);
  }
  inline void add_double(double x, bool negate) {
    uint64_t m; int e; bool neg;
    decode(x, m, e, neg);
    add_scaled(m, e, neg != negate);
  }
  inline void add_product(double x, double y, bool negate) {
    uint64_t mx, my; int ex, ey; bool nx, ny;
    decode(x, mx, ex, nx);
    decode(y, my, ey, ny);
    add_scaled((unsigned __int128)mx * my, ex + ey, (nx != ny) != negate);
  }
  // Value rounded to nearest double (ties to even, with a sticky bit for
  // everything below the 96-bit window): the correctly rounded value.
  double to_double() const {
    uint32_t dig[ND];
    int64_t c = 0;
    for (int i = 0; i < ND; ++i) {
      int64_t v = w[i] + c;
      dig[i] = (uint32_t)v;
      c = v >> 32;  // arithmetic shift: floor division by 2^32
    }
    bool neg = c < 0;
    if (neg) {  // two's complement negation of the digit string
      uint64_t carry = 1;
      for (int i = 0; i < ND; ++i) {
        uint64_t v = (uint64_t)(uint32_t)(~dig[i]) + carry;
        dig[i] = (uint32_t)v;
        carry = v >> 32;
      }
    }
    int top = ND - 1;
    while (top >= 0 && dig[top] == 0) --top;
    if (top < 0) return 0.0;
    auto at = [&](int i) -> uint64_t { return i >= 0 ? dig[i] : 0; };
    unsigned __int128 win = ((unsigned __int128)at(top) << 64) | (at(top - 1) << 32) | at(top - 2);
    bool sticky = false;
    for (int i = top - 3; i >= 0; --i)
      if (dig[i]) { sticky = true; break; }
    int lz = __builtin_clz(dig[top]);
    int rs = 43 - lz;  // leading one (bit 95 - lz) moves to bit 52
    uint64_t keep = (uint64_t)(win >> rs);
    unsigned __int128 rem = win & ((((unsigned __int128)1) << rs) - 1);
    unsigned __int128 half = ((unsigned __int128)1) << (rs - 1);
    if (rem > half || (rem == half && (sticky || (keep & 1)))) keep += 1;
    double v = std::ldexp((double)keep, rs + (top - 2) * 32 + EMIN);
    return neg ? -v : v;
  }
};

}  // namespace

extern "C" {

// ------------------------------------------------------- scalar ops -------
void orc_two_sum(double a, double b, double* out) { two_sum(a, b, out[0], out[1]); }
void orc_two_prod(double a, double b, double* out) { two_prod(a, b, out[0], out[1]); }
void orc_dd_mul(const double* a, const double* b, double* out) {
  dd r = dd_mul({a[0], a[1]}, {b[0], b[1]});
  out[0] = r.hi; out[1] = r.lo;
}
void orc_dd_add(const double* a, const double* b, double* out) {
  dd r = dd_add({a[0], a[1]}, {b[0], b[1]});
  out[0] = r.hi; out[1] = r.lo;
}
void orc_qd_mul(const double* a, const double* b, double* out) {
  qd x, y;
  for (int i = 0; i < 4; ++i) { x.x[i] = a[i]; y.x[i] = b[i]; }
  qd r = qd_mul(x, y);
  for (int i = 0; i < 4; ++i) out[i] = r.x[i];
}
void orc_qd_add(const double* a, const double* b, double* out) {
  qd x, y;
  for (int i = 0; i < 4; ++i) { x.x[i] = a[i]; y.x[i] = b[i]; }
  qd r = qd_add(x, y);
  for (int i = 0; i < 4; ++i) out[i] = r.x[i];
}
void orc_renorm(const double* x, int n, double* out) {
  qd r = renorm(x, n);
  for (int i = 0; i < 4; ++i) out[i] = r.x[i];
}
// Exact sum of sign_i * x_i * y_i (y may be null: plain sum), rounded.
double orc_exact_dot(int64_t n, const double* x, const double* y, const int* neg) {
  Kulisch acc;
  for (int64_t i = 0; i < n; ++i) {
    bool s = neg ? neg[i] != 0 : false;
    if (y) acc.add_product(x[i], y[i], s);
    else acc.add_double(x[i], s);
  }
  return acc.to_double();
}

// ------------------------------------------------------ Simple GEMMs ------
// mode: 0 C := A B, 1 C := C + A B, 2 C := C - A B.
// Planes are row-major with leading dimensions lda, ldb, ldc (in doubles).
int orc_dd_gemm_simple(int64_t m, int64_t l, int64_t n,
                       const double* Ahi, const double* Alo, int64_t lda,
                       const double* Bhi, const double* Blo, int64_t ldb,
                       double* Chi, double* Clo, int64_t ldc, int mode, int nthreads) {
  if (m < 0 || l < 0 || n < 0 || mode < 0 || mode > 2) return 1;
  parallel_for(m, nthreads, [&](int64_t i) {
    for (int64_t j = 0; j < n; ++j) {
      dd c{0.0, 0.0};
      if (mode != 0) c = dd{Chi[i * ldc + j], Clo[i * ldc + j]};
      for (int64_t k = 0; k < l; ++k) {
        dd a{Ahi[i * lda + k], Alo[i * lda + k]};
        if (mode == 2) { a.hi = -a.hi; a.lo = -a.lo; }
        dd b{Bhi[k * ldb + j], Blo[k * ldb + j]};
        c = dd_add(c, dd_mul(a, b));
      }
      Chi[i * ldc + j] = c.hi;
      Clo[i * ldc + j] = c.lo;
    }
  });
  return 0;
}

int orc_qd_gemm_simple(int64_t m, int64_t l, int64_t n,
                       const double* const* A, int64_t lda,
                       const double* const* B, int64_t ldb,
                       double* const* C, int64_t ldc, int mode, int nthreads) {
  if (m < 0 || l < 0 || n < 0 || mode < 0 || mode > 2) return 1;
  parallel_for(m, nthreads, [&](int64_t i) {
    for (int64_t j = 0; j < n; ++j) {
      qd c{{0.0, 0.0, 0.0, 0.0}};
      if (mode != 0) for (int t = 0; t < 4; ++t) c.x[t] = C[t][i * ldc + j];
      for (int64_t k = 0; k < l; ++k) {
        qd a, b;
        for (int t = 0; t < 4; ++t) {
          a.x[t] = A[t][i * lda + k];
          b.x[t] = B[t][k * ldb + j];
          if (mode == 2) a.x[t] = -a.x[t];
        }
        c = qd_add(c, qd_mul(a, b));
      }
      for (int t = 0; t < 4; ++t) C[t][i * ldc + j] = c.x[t];
    }
  });
  return 0;
}

// ----------------------------------------------------- exact checker ------
// For each listed entry (rows[t], cols[t]) (all m*n entries in row-major
// order when count < 0) writes err[t] = (exact value - computed value),
// rounded, where exact = [C0] +/- sum_k a_ik b_kj over all limbs and the
// computed value is the sum of the limbs of C at that entry.
// limbs: 2 (DD) or 4 (QD). A, B, C, C0 are arrays of `limbs` plane pointers;
// C0 may be null (mode 0).
int orc_gemm_error(int limbs, int64_t m, int64_t l, int64_t n,
                   const double* const* A, int64_t lda,
                   const double* const* B, int64_t ldb,
                   const double* const* C, int64_t ldc,
                   const double* const* C0, int mode,
                   int64_t count, const int64_t* rows, const int64_t* cols,
                   double* err, int nthreads) {
  if (limbs != 2 && limbs != 4) return 1;
  int64_t total = count < 0 ? m * n : count;
  parallel_for(total, nthreads, [&](int64_t t) {
    int64_t i = count < 0 ? t / n : rows[t];
    int64_t j = count < 0 ? t % n : cols[t];
    Kulisch acc;
    bool neg = mode == 2;
    for (int64_t k = 0; k < l; ++k)
      for (int p = 0; p < limbs; ++p) {
        double a = A[p][i * lda + k];
        if (a == 0.0) continue;
        for (int q = 0; q < limbs; ++q) {
          double b = B[q][k * ldb + j];
          if (b != 0.0) acc.add_product(a, b, neg);
        }
      }
    if (mode != 0 && C0)
      for (int p = 0; p < limbs; ++p) acc.add_double(C0[p][i * ldc + j], false);
    for (int p = 0; p < limbs; ++p) acc.add_double(C[p][i * ldc + j], true);
    err[t] = acc.to_double();
  });
  return 0;
}

// Exact value of entries of A B rounded to double (for closed-form tests).
int orc_gemm_exact(int limbs, int64_t m, int64_t l, int64_t n,
                   const double* const* A, int64_t lda,
                   const double* const* B, int64_t ldb,
                   double* out, int nthreads) {
  parallel_for(m * n, nthreads, [&](int64_t t) {
    int64_t i = t / n, j = t % n;
    Kulisch acc;
    for (int64_t k = 0; k < l; ++k)
      for (int p = 0; p < limbs; ++p)
        for (int q = 0; q < limbs; ++q)
          acc.add_product(A[p][i * lda + k], B[q][k * ldb + j], false);
    out[t] = acc.to_double();
  });
  return 0;
}

// ------------------------------------------------------------ LU ----------
// Exact residual r = b - A x per row (A: n x n DD, x and b: n x nrhs DD,
// row-major), rounded to double. Section 4, Eq. 2.
int orc_dd_residual(int64_t n, int64_t nrhs,
                    const double* Ahi, const double* Alo, int64_t lda,
                    const double* Xhi, const double* Xlo, int64_t ldx,
                    const double* Bhi, const double* Blo, int64_t ldb,
                    double* r, int nthreads) {
  parallel_for(n * nrhs, nthreads, [&](int64_t t) {
    int64_t i = t / nrhs, c = t % nrhs;
    Kulisch acc;
    acc.add_double(Bhi[i * ldb + c], false);
    acc.add_double(Blo[i * ldb + c], false);
    for (int64_t k = 0; k < n; ++k) {
      const double a[2] = {Ahi[i * lda + k], Alo[i * lda + k]};
      const double x[2] = {Xhi[k * ldx + c], Xlo[k * ldx + c]};
      for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q)
          if (a[p] != 0.0 && x[q] != 0.0) acc.add_product(a[p], x[q], true);
    }
    r[t] = acc.to_double();
  });
  return 0;
}

// The same exact residual for DD (limbs = 2) or QD (limbs = 4) operands,
// each argument an array of limb planes.
int orc_residual(int limbs, int64_t n, int64_t nrhs, const double* const* A, int64_t lda,
                 const double* const* X, int64_t ldx, const double* const* B, int64_t ldb,
                 double* r, int nthreads) {
  parallel_for(n * nrhs, nthreads, [&](int64_t t) {
    int64_t i = t / nrhs, c = t % nrhs;
    Kulisch acc;
    for (int p = 0; p < limbs; ++p) acc.add_double(B[p][i * ldb + c], false);
    for (int64_t k = 0; k < n; ++k)
      for (int p = 0; p < limbs; ++p)
        for (int q = 0; q < limbs; ++q) {
          const double a = A[p][i * lda + k], x = X[q][k * ldx + c];
          if (a != 0.0 && x != 0.0) acc.add_product(a, x, true);
        }
    r[t] = acc.to_double();
  });
  return 0;
}

// QD quotient a / b by long division: each digit is the leading limb of the
// running remainder over the leading limb of b, the remainder loses that
// digit times b (QD arithmetic), and five digits are renormalised.
inline qd qd_div(const qd& a, const qd& b) {
  double q[5];
  qd r = a;
  for (int k = 0; k < 5; ++k) {
    q[k] = r.x[0] / b.x[0];
    if (k < 4) {
      qd t = qd_mul(qd{{-q[k], 0.0, 0.0, 0.0}}, b);
      r = qd_add(r, t);
    }
  }
  return renorm(q, 5);
}

// Unblocked right-looking QD LU (Section 4 with block size 1), in place on
// four limb planes, the pivot rule of the DD version on the first two limbs
// (|x0|, then x1 with the sign of x0); l_ij = a_ij / a_jj by qd_div.
int orc_qd_getrf(int64_t n, double* const* A, int64_t lda, int64_t* ipiv, int pivot) {
  auto at = [&](int64_t i, int64_t c) {
    return qd{{A[0][i * lda + c], A[1][i * lda + c], A[2][i * lda + c], A[3][i * lda + c]}};
  };
  auto put = [&](int64_t i, int64_t c, const qd& v) {
    for (int q = 0; q < 4; ++q) A[q][i * lda + c] = v.x[q];
  };
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = j;
    if (pivot) {
      double bh = std::fabs(A[0][j * lda + j]);
      double bl = A[0][j * lda + j] < 0 ? -A[1][j * lda + j] : A[1][j * lda + j];
      for (int64_t i = j + 1; i < n; ++i) {
        double h = std::fabs(A[0][i * lda + j]);
        double lo = A[0][i * lda + j] < 0 ? -A[1][i * lda + j] : A[1][i * lda + j];
        if (h > bh || (h == bh && lo > bl)) { bh = h; bl = lo; p = i; }
      }
    }
    ipiv[j] = p;
    if (p != j)
      for (int64_t c = 0; c < n; ++c)
        for (int q = 0; q < 4; ++q) std::swap(A[q][p * lda + c], A[q][j * lda + c]);
    const qd piv = at(j, j);
    if (piv.x[0] == 0.0 && piv.x[1] == 0.0 && piv.x[2] == 0.0 && piv.x[3] == 0.0) return (int)(1 + j);
    for (int64_t i = j + 1; i < n; ++i) {
      const qd l = qd_div(at(i, j), piv);
      put(i, j, l);
      const qd nl{{-l.x[0], -l.x[1], -l.x[2], -l.x[3]}};
      for (int64_t c = j + 1; c < n; ++c) put(i, c, qd_add(at(i, c), qd_mul(nl, at(j, c))));
    }
  }
  return 0;
}

void orc_qd_div(const double* a, const double* b, double* out) {
  qd r = qd_div(qd{{a[0], a[1], a[2], a[3]}}, qd{{b[0], b[1], b[2], b[3]}});
  for (int q = 0; q < 4; ++q) out[q] = r.x[q];
}

// Unblocked right-looking DD LU (Section 4 steps 1-3 with block size 1),
// in place, with partial pivoting when pivot != 0: the pivot of column j is
// the first row index i >= j maximising |a_ij| compared as DD (hi, then lo
// with the sign of hi). ipiv[j] = chosen row (0-based). Returns 0, or
// 1 + j for an exactly zero pivot in column j.
int orc_dd_getrf(int64_t n, double* Ahi, double* Alo, int64_t lda, int64_t* ipiv, int pivot) {
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = j;
    if (pivot) {
      double bh = std::fabs(Ahi[j * lda + j]);
      double bl = Ahi[j * lda + j] < 0 ? -Alo[j * lda + j] : Alo[j * lda + j];
      for (int64_t i = j + 1; i < n; ++i) {
        double h = std::fabs(Ahi[i * lda + j]);
        double lo = Ahi[i * lda + j] < 0 ? -Alo[i * lda + j] : Alo[i * lda + j];
        if (h > bh || (h == bh && lo > bl)) { bh = h; bl = lo; p = i; }
      }
    }
    ipiv[j] = p;
    if (p != j)
      for (int64_t c = 0; c < n; ++c) {
        std::swap(Ahi[p * lda + c], Ahi[j * lda + c]);
        std::swap(Alo[p * lda + c], Alo[j * lda + c]);
      }
    dd piv{Ahi[j * lda + j], Alo[j * lda + j]};
    if (piv.hi == 0.0 && piv.lo == 0.0) return (int)(1 + j);
    for (int64_t i = j + 1; i < n; ++i) {
      // l_ij = a_ij / piv by one Newton step on the DD quotient
      dd a{Ahi[i * lda + j], Alo[i * lda + j]};
      double q1 = a.hi / piv.hi;
      dd r = dd_add(a, dd_mul({-q1, 0.0}, piv));
      double q2 = r.hi / piv.hi;
      dd rr = dd_add(r, dd_mul({-q2, 0.0}, piv));
      double q3 = rr.hi / piv.hi;
      dd q;
      fast_two_sum(q1, q2, q.hi, q.lo);
      q = dd_add(q, {q3, 0.0});
      Ahi[i * lda + j] = q.hi;
      Alo[i * lda + j] = q.lo;
      dd nq{-q.hi, -q.lo};
      for (int64_t c = j + 1; c < n; ++c) {
        dd u{Ahi[j * lda + c], Alo[j * lda + c]};
        dd v{Ahi[i * lda + c], Alo[i * lda + c]};
        dd w = dd_add(v, dd_mul(nq, u));
        Ahi[i * lda + c] = w.hi;
        Alo[i * lda + c] = w.lo;
      }
    }
  }
  return 0;
}

}  // extern "C"
