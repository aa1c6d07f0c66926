// Fixed-point integer arithmetic for DD / QD numbers on the integer pipe.
//
// GB300 retires 2 FP64 instructions per clock per SM but 64 IMAD and ~128
// other integer instructions, so the library's DD / QD arithmetic runs on
// the integer pipe wherever it is hot:
//   * operands: an expansion x0 + x1 + ... summed exactly into a W-word
//     integer M at the scale of x0 (to_fixed), or placed at a common scale
//     shared by several operands (add_at);
//   * products: the leading words of M_a M_b by multiword multiplication
//     (mul_top), placed into a two's-complement window (place_shr);
//   * windows: wide accumulators (Kulisch-style, only as wide as the
//     products' range needs) whose scale is fixed from the largest operands,
//     so the sums are exact; bits below the window are truncated;
//   * rounding back: acc_chunks / from_fixed / operand_to_limbs.
//
// Word layout: acc[0] is the least significant 32-bit word; the top word
// carries the sign. A double x is unpacked as |x| = (m1:m0) 2^(e - 1075) with
// m1 holding the hidden bit (e >= 1; zero and subnormals have e = 1).
//
// The helpers are __host__ __device__ so that their bit manipulation can be
// checked on the host against exact arithmetic.
#pragma once

#include <cstdint>
#include <cstring>

namespace ddg {
namespace fx {

struct unpacked {
  uint32_t m0, m1;  // significand, m1 < 2^21
  int e;            // biased exponent, >= 1
  uint32_t s;       // sign bit
};

__host__ __device__ __forceinline__ uint64_t dbits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}

__host__ __device__ __forceinline__ double bitsd(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}

__host__ __device__ __forceinline__ unpacked unpack(double x) {
  const uint64_t b = dbits(x);
  const uint32_t hi = (uint32_t)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7FF);
  unpacked u;
  u.m0 = (uint32_t)b;
  u.m1 = (hi & 0xFFFFFu) | (e ? 0x100000u : 0u);
  u.e = e ? e : 1;
  u.s = hi >> 31;
  return u;
}

// Biased exponent field of x (0 for zero / subnormal).
__host__ __device__ __forceinline__ int expfield(double x) {
  return (int)((dbits(x) >> 52) & 0x7FF);
}

// (hi:lo << r) >> 32, r in [0, 31]
__host__ __device__ __forceinline__ uint32_t shl_funnel(uint32_t lo, uint32_t hi, int r) {
#ifdef __CUDA_ARCH__
  return __funnelshift_l(lo, hi, r);
#else
  return (uint32_t)(((((uint64_t)hi) << 32) | lo) << r >> 32);
#endif
}

__host__ __device__ __forceinline__ int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

// acc += (d XOR mask) + neg, mask = -neg: adds d, or subtracts it when neg = 1.
template <int NW>
__host__ __device__ __forceinline__ void acc_add(uint32_t (&A)[NW], const uint32_t (&d)[NW], uint32_t neg) {
  const uint32_t m = 0u - neg;
#ifdef __CUDA_ARCH__
  if constexpr (NW == 6) {
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %6, 0xFFFFFFFF;\n\t"
        "addc.cc.u32 %0, %0, %7;\n\t"
        "addc.cc.u32 %1, %1, %8;\n\t"
        "addc.cc.u32 %2, %2, %9;\n\t"
        "addc.cc.u32 %3, %3, %10;\n\t"
        "addc.cc.u32 %4, %4, %11;\n\t"
        "addc.u32 %5, %5, %12;\n\t}"
        : "+r"(A[0]), "+r"(A[1]), "+r"(A[2]), "+r"(A[3]), "+r"(A[4]), "+r"(A[5])
        : "r"(neg), "r"(d[0] ^ m), "r"(d[1] ^ m), "r"(d[2] ^ m), "r"(d[3] ^ m), "r"(d[4] ^ m),
          "r"(d[5] ^ m));
  } else if constexpr (NW == 9) {
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %9, 0xFFFFFFFF;\n\t"
        "addc.cc.u32 %0, %0, %10;\n\t"
        "addc.cc.u32 %1, %1, %11;\n\t"
        "addc.cc.u32 %2, %2, %12;\n\t"
        "addc.cc.u32 %3, %3, %13;\n\t"
        "addc.cc.u32 %4, %4, %14;\n\t"
        "addc.cc.u32 %5, %5, %15;\n\t"
        "addc.cc.u32 %6, %6, %16;\n\t"
        "addc.cc.u32 %7, %7, %17;\n\t"
        "addc.u32 %8, %8, %18;\n\t}"
        : "+r"(A[0]), "+r"(A[1]), "+r"(A[2]), "+r"(A[3]), "+r"(A[4]), "+r"(A[5]), "+r"(A[6]),
          "+r"(A[7]), "+r"(A[8])
        : "r"(neg), "r"(d[0] ^ m), "r"(d[1] ^ m), "r"(d[2] ^ m), "r"(d[3] ^ m), "r"(d[4] ^ m),
          "r"(d[5] ^ m), "r"(d[6] ^ m), "r"(d[7] ^ m), "r"(d[8] ^ m));
  } else {
    static_assert(NW == 6 || NW == 9, "accumulator width");
  }
#else
  uint64_t c = neg;
  for (int t = 0; t < NW; ++t) {
    const uint64_t v = (uint64_t)A[t] + (uint64_t)(d[t] ^ m) + c;
    A[t] = (uint32_t)v;
    c = v >> 32;
  }
#endif
}

// 128-bit right shift of p by s >= 1 bits (bits shifted out are dropped).
__host__ __device__ __forceinline__ void shr128(uint32_t (&p)[4], int s) {
  uint64_t lo = ((uint64_t)p[1] << 32) | p[0];
  uint64_t hi = ((uint64_t)p[3] << 32) | p[2];
  if (s >= 128) {
    lo = 0;
    hi = 0;
  } else if (s >= 64) {
    lo = s == 64 ? hi : hi >> (s - 64);
    hi = 0;
  } else if (s > 0) {
    lo = (lo >> s) | (hi << (64 - s));
    hi >>= s;
  }
  p[0] = (uint32_t)lo;
  p[1] = (uint32_t)(lo >> 32);
  p[2] = (uint32_t)hi;
  p[3] = (uint32_t)(hi >> 32);
}

// Add sign * p * 2^pos (in units of the accumulator's least significant bit)
// into A. WF is the word index that positions in [32 (WF - 1), 32 WF + 31]
// fall into on the fast path (two candidate word offsets, one select per
// word); any other position takes the general path.
template <int NW, int WF>
__host__ __device__ __forceinline__ void place(uint32_t (&A)[NW], uint32_t (&p)[4], int pos, uint32_t neg) {
  uint32_t d[NW];
  if (pos >= 32 * (WF - 1) && pos < 32 * (WF + 1)) {
    const int r = pos & 31;
    const bool hiw = (pos >> 5) == WF;
    const uint32_t q0 = p[0] << r;
    const uint32_t q1 = shl_funnel(p[0], p[1], r);
    const uint32_t q2 = shl_funnel(p[1], p[2], r);
    const uint32_t q3 = shl_funnel(p[2], p[3], r);
    const uint32_t q4 = shl_funnel(p[3], 0u, r);
    const uint32_t q[5] = {q0, q1, q2, q3, q4};
#pragma unroll
    for (int t = 0; t < NW; ++t) {
      const int jl = t - (WF - 1), jh = t - WF;  // piece index for each candidate offset
      const uint32_t vl = (jl >= 0 && jl < 5) ? q[jl < 0 ? 0 : (jl > 4 ? 4 : jl)] : 0u;
      const uint32_t vh = (jh >= 0 && jh < 5) ? q[jh < 0 ? 0 : (jh > 4 ? 4 : jh)] : 0u;
      d[t] = hiw ? vh : vl;
    }
  } else {
    if (pos < 0) {
      shr128(p, -pos);
      pos = 0;
    }
    const int w = pos >> 5, r = pos & 31;
    const uint32_t q0 = p[0] << r;
    const uint32_t q1 = shl_funnel(p[0], p[1], r);
    const uint32_t q2 = shl_funnel(p[1], p[2], r);
    const uint32_t q3 = shl_funnel(p[2], p[3], r);
    const uint32_t q4 = shl_funnel(p[3], 0u, r);
    const uint32_t q[5] = {q0, q1, q2, q3, q4};
#pragma unroll
    for (int t = 0; t < NW; ++t) {
      uint32_t v = 0u;
#pragma unroll
      for (int c = 0; c < 5; ++c)
        if (t - c >= 0) v = (w == t - c) ? q[c] : v;
      d[t] = v;
    }
  }
  acc_add<NW>(A, d, neg);
}

// Power of two 2^k as a double for k in [-2044, 2046], as the product of
// two factors that are both normal (the product rounds only if subnormal).
__host__ __device__ __forceinline__ double pow2_product(double x, int k) {
  const int k1 = k / 2, k2 = k - k1;
  const double f1 = bitsd((uint64_t)(k1 + 1023) << 52);
  const double f2 = bitsd((uint64_t)(k2 + 1023) << 52);
#ifdef __CUDA_ARCH__
  return __dmul_rn(__dmul_rn(x, f1), f2);
#else
  return (x * f1) * f2;
#endif
}

// Magnitude and sign of a two's-complement accumulator.
template <int NW>
__host__ __device__ __forceinline__ uint32_t acc_abs(uint32_t (&A)[NW]) {
  const uint32_t neg = A[NW - 1] >> 31;
  const uint32_t m = 0u - neg;
  uint64_t c = neg;
#pragma unroll
  for (int t = 0; t < NW; ++t) {
    const uint64_t v = (uint64_t)(A[t] ^ m) + c;
    A[t] = (uint32_t)v;
    c = v >> 32;
  }
  return neg;
}

// Whether the two's-complement NW-word A has magnitude below 2^bits
// (0 < bits < 32 NW); A is not changed.
template <int NW>
__host__ __device__ __forceinline__ bool acc_mag_below(const uint32_t (&A)[NW], int bits) {
  const uint32_t m = 0u - (A[NW - 1] >> 31);
  uint64_t c = m & 1u;
  bool below = true;
  const int w = bits >> 5, r = bits & 31;
#pragma unroll
  for (int t = 0; t < NW; ++t) {
    const uint64_t v = (uint64_t)(A[t] ^ m) + c;
    const uint32_t x = (uint32_t)v;
    c = v >> 32;
    if (t > w && x != 0u) below = false;
    if (t == w && (x >> r) != 0u) below = false;
  }
  return below;
}

// B = A shifted up by whole words so that A's highest nonzero word lands in
// B[NW - 1]; returns the index of that word in A, or -1 if A = 0. A barrel
// shifter (conditional shifts by 8, 4, 2, 1 words with fixed indices): no
// select over a computed word index, a form that was seen miscompiled at
// -O3 on this toolchain.
template <int NW>
__host__ __device__ __forceinline__ int acc_top_align(const uint32_t (&A)[NW], uint32_t (&B)[NW]) {
  int top = -1;
#pragma unroll
  for (int t = 0; t < NW; ++t) {
    if (A[t] != 0u) top = t;
    B[t] = A[t];
  }
  const int s = NW - 1 - top;
#pragma unroll
  for (int step = 8; step >= 1; step >>= 1) {
    if (step >= NW) continue;
    const bool on = top >= 0 && (s & step) != 0;
#pragma unroll
    for (int t = NW - 1; t >= 0; --t) B[t] = on ? (t >= step ? B[t - step] : 0u) : B[t];
  }
  return top;
}

// Split the magnitude |A| into K chunks of 53 bits from its leading bit down:
// |A| ~= sum_c chunk[c] * 2^(exp[c]) (in units of the LSB), truncated below.
// Returns false if A is zero.
template <int NW, int K>
__host__ __device__ __forceinline__ bool acc_chunks(const uint32_t (&A)[NW], uint64_t (&chunk)[K], int (&exp)[K]) {
  uint32_t B[NW];
  const int top = acc_top_align<NW>(A, B);
  if (top < 0) return false;
  // the top word and the words below it as a bit string g (MSB first)
  constexpr int G = (53 * K + 31) / 32 + 2;  // words needed below the leading bit
  uint32_t g[G];
#pragma unroll
  for (int i = 0; i < G; ++i) g[i] = i < NW ? B[NW - 1 - (i < NW ? i : 0)] : 0u;
  const int lz = clz32(g[0]);
  // left-align: shift the string so that the leading one is bit 31 of g[0]
#pragma unroll
  for (int i = 0; i < G; ++i) g[i] = shl_funnel(i + 1 < G ? g[i + 1] : 0u, g[i], lz);
  const int lead = 32 * top + 31 - lz;  // bit position of the leading one
#pragma unroll
  for (int c = 0; c < K; ++c) {
    // bits [53 c, 53 c + 53) of the aligned string, counted from the top
    const int b0 = 53 * c;
    const int w = b0 >> 5, o = b0 & 31;
    const uint64_t x = ((uint64_t)g[w] << 32) | g[w + 1];
    const uint32_t y = g[w + 2];
    // 96 bits x:y starting at bit offset o; take 53 bits
    const uint64_t top64 = (o == 0) ? x : ((x << o) | ((uint64_t)y >> (32 - o)));
    chunk[c] = top64 >> 11;
    exp[c] = lead - 52 - b0;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Per-operand fixed-point form (the Block kernel's second scheme).
//
// A DD / QD number x = x0 + x1 + ... is converted once, when its tile is
// staged, into an unsigned W-word integer M with |x| ~= M 2^(f - 1075 -
// (32 W - 53)), f = the biased exponent field of x0 (1 for zero and
// subnormals) and the sign of x0: x0's 53-bit significand fills the top of
// M and each further limb is added or subtracted at its own offset
// (truncated toward zero below bit 0, i.e. 2^-(32 W - 1) of |x|). Since the
// expansion is normalised, 0 <= M < 2^(32 W). Returns f | (sign << 16).
template <int L, int W>
__host__ __device__ __forceinline__ int to_fixed(const double (&x)[L], uint32_t (&M)[W]) {
#pragma unroll
  for (int w = 0; w < W; ++w) M[w] = 0u;
  const unpacked u0 = unpack(x[0]);
  if (u0.m0 == 0u && u0.m1 == 0u) return 1;
  constexpr int TOP = 32 * W - 53;  // bit offset of x0's significand
#pragma unroll
  for (int q = 0; q < L; ++q) {
    const unpacked u = q == 0 ? u0 : unpack(x[q]);
    int sh = q == 0 ? TOP : (u.e - u0.e) + TOP;  // bit offset of this limb's LSB
    uint64_t m = ((uint64_t)u.m1 << 32) | u.m0;
    if (m == 0u || sh <= -53) continue;
    if (sh < 0) {
      m >>= -sh;
      sh = 0;
    }
    // the limb as W words at offset sh (53 bits span at most 3 words)
    const int wo = sh >> 5, r = sh & 31;
    const uint32_t p0 = (uint32_t)m << r;
    const uint32_t p1 = shl_funnel((uint32_t)m, (uint32_t)(m >> 32), r);
    const uint32_t p2 = shl_funnel((uint32_t)(m >> 32), 0u, r);
    const uint32_t neg = q == 0 ? 0u : (u.s ^ u0.s);
    const uint32_t msk = 0u - neg;
    uint64_t c = neg;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t d = w == wo ? p0 : (w == wo + 1 ? p1 : (w == wo + 2 ? p2 : 0u));
      const uint64_t v = (uint64_t)M[w] + (d ^ msk) + c;
      M[w] = (uint32_t)v;
      c = v >> 32;
    }
  }
  return u0.e | (int)(u0.s << 16);
}

// The K = 2 W - D leading words of a b from the column sums of the partial
// products with i + j >= D (Comba order, a three-word running sum; the
// columns below D and their carries are dropped). The result is below the
// exact floor(a b / 2^(32 D)) by less than (D + 1) 2^32 units.
template <int W, int D>
__host__ __device__ __forceinline__ void mul_top(const uint32_t (&a)[W], const uint32_t (&b)[W],
                                                 uint32_t (&p)[2 * W - D]) {
  uint32_t c0 = 0u, c1 = 0u, c2 = 0u;
#pragma unroll
  for (int k = D; k <= 2 * W - 2; ++k) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int j = k - i;
      if (j < 0 || j >= W) continue;
#ifdef __CUDA_ARCH__
      // the carry out of the high word goes to c2 by an add (integer ALU
      // pipe), leaving the IMAD pipe to the two multiplies: QD +8%, DD +1%
      asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
          "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
          "addc.u32 %2, %2, 0;"
          : "+r"(c0), "+r"(c1), "+r"(c2)
          : "r"(a[i]), "r"(b[j]));
#else
      const uint64_t pr = (uint64_t)a[i] * b[j];
      const uint64_t lo = (uint64_t)c0 + (uint32_t)pr;
      const uint64_t hi = (uint64_t)c1 + (uint32_t)(pr >> 32) + (lo >> 32);
      c0 = (uint32_t)lo;
      c1 = (uint32_t)hi;
      c2 += (uint32_t)(hi >> 32);
#endif
    }
    p[k - D] = c0;
    c0 = c1;
    c1 = c2;
    c2 = 0u;
  }
  p[2 * W - 1 - D] = c0;
}

// q = the W words of a b at columns W .. 2 W - 1 (column c: 2^(32 c)) from
// the partial products a_i b_j with i + j >= W, and of those with
// i + j = W - 1 only the high halves (their low halves, the products below
// and all their carries are left out): q is below floor(a b / 2^(32 W)) by
// less than 2 W. Column by column, a three-word running sum; on the device
// 16 IMAD for W = 4 (6 products x 2 + 4 high halves). The product of the
// pre-shifted DD Block form (fx_pre.cuh).
template <int W>
__host__ __device__ __forceinline__ void mul_top_hi(const uint32_t (&a)[W], const uint32_t (&b)[W],
                                                    uint32_t (&q)[W]) {
  constexpr int D = W - 1;
#ifdef __CUDA_ARCH__
  uint32_t c0 = 0u, c1 = __umulhi(a[0], b[D]), c2 = 0u;
#pragma unroll
  for (int i = 1; i < W; ++i)
    asm("mad.hi.cc.u32 %0, %2, %3, %0;\n\t"
        "addc.u32 %1, %1, 0;"
        : "+r"(c1), "+r"(c2)
        : "r"(a[i]), "r"(b[D - i]));
#pragma unroll
  for (int k = W; k <= 2 * W - 2; ++k) {
    c0 = c1;
    c1 = c2;
    c2 = 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int j = k - i;
      if (j < 0 || j >= W) continue;
      if (k < 2 * W - 2) {
        asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
            "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
            "addc.u32 %2, %2, 0;"
            : "+r"(c0), "+r"(c1), "+r"(c2)
            : "r"(a[i]), "r"(b[j]));
      } else {  // the top column: a b < 2^(64 W), no carry out of it
        asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\t"
            "madc.hi.u32 %1, %2, %3, %1;"
            : "+r"(c0), "+r"(c1)
            : "r"(a[i]), "r"(b[j]));
      }
    }
    q[k - W] = c0;
  }
  q[W - 1] = c1;
#else
  // the same sum with 64-bit column accumulators
  uint64_t col[2 * W + 1] = {};
  for (int i = 0; i < W; ++i)
    for (int j = 0; j < W; ++j) {
      const uint64_t pr = (uint64_t)a[i] * b[j];
      if (i + j == D) {
        col[W] += pr >> 32;
      } else if (i + j >= W) {
        col[i + j] += (uint32_t)pr;
        col[i + j + 1] += pr >> 32;
      }
    }
  uint64_t carry = 0;
  for (int k = W; k < 2 * W; ++k) {
    const uint64_t v = col[k] + carry;
    q[k - W] = (uint32_t)v;
    carry = v >> 32;
  }
#endif
}

// (hi:lo >> r) low word, r in [0, 31]
__host__ __device__ __forceinline__ uint32_t shr_funnel(uint32_t lo, uint32_t hi, int r) {
#ifdef __CUDA_ARCH__
  return __funnelshift_r(lo, hi, r);
#else
  return (uint32_t)(((((uint64_t)hi) << 32) | lo) >> r);
#endif
}

// acc += (d XOR m) + (m & 1) for a mask m = 0 (add d) or ~0 (subtract d).
template <int NW>
__host__ __device__ __forceinline__ void acc_add_mask(uint32_t (&A)[NW], const uint32_t (&d)[NW], uint32_t m) {
#ifdef __CUDA_ARCH__
  if constexpr (NW == 6) {
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %6, %6;\n\t"  // carry = top bit of the mask
        "madc.lo.cc.u32 %0, %7, 1, %0;\n\t"
        "madc.lo.cc.u32 %1, %8, 1, %1;\n\t"
        "madc.lo.cc.u32 %2, %9, 1, %2;\n\t"
        "madc.lo.cc.u32 %3, %10, 1, %3;\n\t"
        "madc.lo.cc.u32 %4, %11, 1, %4;\n\t"
        "madc.lo.u32 %5, %12, 1, %5;\n\t}"
        : "+r"(A[0]), "+r"(A[1]), "+r"(A[2]), "+r"(A[3]), "+r"(A[4]), "+r"(A[5])
        : "r"(m), "r"(d[0] ^ m), "r"(d[1] ^ m), "r"(d[2] ^ m), "r"(d[3] ^ m), "r"(d[4] ^ m),
          "r"(d[5] ^ m));
  } else if constexpr (NW == 9) {
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %9, %9;\n\t"
        "madc.lo.cc.u32 %0, %10, 1, %0;\n\t"
        "madc.lo.cc.u32 %1, %11, 1, %1;\n\t"
        "madc.lo.cc.u32 %2, %12, 1, %2;\n\t"
        "madc.lo.cc.u32 %3, %13, 1, %3;\n\t"
        "madc.lo.cc.u32 %4, %14, 1, %4;\n\t"
        "madc.lo.cc.u32 %5, %15, 1, %5;\n\t"
        "madc.lo.cc.u32 %6, %16, 1, %6;\n\t"
        "madc.lo.cc.u32 %7, %17, 1, %7;\n\t"
        "madc.lo.u32 %8, %18, 1, %8;\n\t}"
        : "+r"(A[0]), "+r"(A[1]), "+r"(A[2]), "+r"(A[3]), "+r"(A[4]), "+r"(A[5]), "+r"(A[6]),
          "+r"(A[7]), "+r"(A[8])
        : "r"(m), "r"(d[0] ^ m), "r"(d[1] ^ m), "r"(d[2] ^ m), "r"(d[3] ^ m), "r"(d[4] ^ m),
          "r"(d[5] ^ m), "r"(d[6] ^ m), "r"(d[7] ^ m), "r"(d[8] ^ m));
  } else {
    static_assert(NW == 6 || NW == 9, "accumulator width");
  }
#else
  uint64_t c = m >> 31;
  for (int t = 0; t < NW; ++t) {
    const uint64_t v = (uint64_t)A[t] + (uint64_t)(d[t] ^ m) + c;
    A[t] = (uint32_t)v;
    c = v >> 32;
  }
#endif
}

// A += sign * floor(p / 2^sh) for a K-word p, sh >= 0 and the sign as a
// mask m (0: add, ~0: subtract); bits shifted out are dropped. Fast path for
// sh < 32 (a funnel shift per word); larger shifts take the general path.
template <int NW, int K>
__host__ __device__ __forceinline__ void place_shr(uint32_t (&A)[NW], const uint32_t (&p)[K], int sh,
                                                   uint32_t m) {
  static_assert(K <= NW, "product wider than the window");
  uint32_t d[NW];
  const int r = sh & 31;
  if (sh < 32) {
#pragma unroll
    for (int t = 0; t < NW; ++t) d[t] = t < K ? shr_funnel(p[t], t + 1 < K ? p[t + 1] : 0u, r) : 0u;
  } else {
    const int w = sh >> 5;
#pragma unroll
    for (int t = 0; t < NW; ++t) {
      uint32_t v = 0u;
#pragma unroll
      for (int s = 1; s < K; ++s) {
        if (t + s >= K) continue;
        const uint32_t x = shr_funnel(p[t + s], t + s + 1 < K ? p[t + s + 1] : 0u, r);
        v = (w == s) ? x : v;
      }
      d[t] = v;
    }
  }
  acc_add_mask<NW>(A, d, m);
}

// ---------------------------------------------------------------------------
// Exact sums of DD / QD numbers (the quadrant passes).
//
// All operands of one element are placed at a common scale, unit
// 2^(emax - 1075 - top) with emax the largest leading-limb exponent field
// among them, as signed NW-word integers (limbs below bit 0 truncated toward
// zero: 2^-(top + 52) of the largest operand); sums and differences are then
// exact multiword additions, and each result is converted back once.

// V += sign * x (x an expansion of L limbs) at the common scale.
template <int L, int NW>
__host__ __device__ __forceinline__ void add_at(uint32_t (&V)[NW], const double (&x)[L], int emax, int top,
                                                uint32_t negate) {
#pragma unroll
  for (int q = 0; q < L; ++q) {
    const unpacked u = unpack(x[q]);
    uint64_t m = ((uint64_t)u.m1 << 32) | u.m0;
    int sh = (u.e - emax) + top;
    if (m == 0u || sh <= -53) continue;
    if (sh < 0) {
      m >>= -sh;
      sh = 0;
    }
    const int wo = sh >> 5, r = sh & 31;
    const uint32_t p0 = (uint32_t)m << r;
    const uint32_t p1 = shl_funnel((uint32_t)m, (uint32_t)(m >> 32), r);
    const uint32_t p2 = shl_funnel((uint32_t)(m >> 32), 0u, r);
    const uint32_t msk = 0u - (u.s ^ negate);
    uint64_t c = msk & 1u;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t d = w == wo ? p0 : (w == wo + 1 ? p1 : (w == wo + 2 ? p2 : 0u));
      const uint64_t v = (uint64_t)V[w] + (d ^ msk) + c;
      V[w] = (uint32_t)v;
      c = v >> 32;
    }
  }
}

// R = X + Y or X - Y (two's complement, NW words).
template <int NW>
__host__ __device__ __forceinline__ void vadd(uint32_t (&R)[NW], const uint32_t (&X)[NW], const uint32_t (&Y)[NW],
                                              bool sub) {
  const uint32_t msk = sub ? 0xFFFFFFFFu : 0u;
  uint64_t c = sub ? 1u : 0u;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint64_t v = (uint64_t)X[w] + (Y[w] ^ msk) + c;
    R[w] = (uint32_t)v;
    c = v >> 32;
  }
}

// mag 2^e2 with the sign bit neg as a double (mag < 2^54): the bit pattern
// is assembled on the integer pipe when the result is a normal number; other
// cases take the FP64 scaling.
__host__ __device__ __forceinline__ double make_double(uint64_t mag, int e2, uint32_t neg) {
  if (mag == 0u) return neg ? -0.0 : 0.0;
  const int lz = clz32((uint32_t)(mag >> 32)) + ((mag >> 32) == 0u ? clz32((uint32_t)mag) : 0);
  const int sh = 11 - lz;  // leading one to bit 52
  const uint64_t m = sh >= 0 ? (mag >> sh) : (mag << -sh);
  const int be = e2 + sh + 1075;
  if (be >= 1 && be <= 2046 && (sh <= 0 || (mag & ((1ull << sh) - 1u)) == 0u))
    return bitsd(((uint64_t)neg << 63) | ((uint64_t)be << 52) | (m & 0xFFFFFFFFFFFFFull));
  const double v = pow2_product((double)mag, e2 < -2044 ? -2044 : (e2 > 2046 ? 2046 : e2));
  return neg ? -v : v;
}

template <int L, int W>
__host__ __device__ __forceinline__ void operand_to_limbs(const uint32_t (&M)[W], int e, uint32_t s, double (&out)[L]);
template <int NW, int W>
__host__ __device__ __forceinline__ int acc_normalize(const uint32_t (&A)[NW], uint32_t (&M)[W]);

// The L-limb expansion nearest the signed integer V 2^lsb (V is destroyed).
// QD: the leading 224 bits of |V| rounded greedily limb by limb
// (operand_to_limbs: canonical). DD:
// the leading L 53-bit pieces of |V| and the next bit, turned into balanced
// digits from the least significant end (a digit >= 2^52 becomes digit -
// 2^53 and carries one into the next), so the leading limb is |V| rounded to
// 53 bits and each further limb is at most half a unit of the one above.
// Bits below the L + 1 pieces are truncated. For L = 2 this is the DD
// nearest V (hi = V rounded to 53 bits, |lo| <= ulp(hi) / 2).
template <int L, int NW>
__host__ __device__ __forceinline__ void from_fixed_balanced(uint32_t (&V)[NW], int lsb, double (&out)[L]);

template <int L, int NW>
__host__ __device__ __forceinline__ void from_fixed(uint32_t (&V)[NW], int lsb, double (&out)[L]) {
  if constexpr (L == 4) {
    const uint32_t neg = acc_abs<NW>(V);
    uint32_t M[7];
    const int p = acc_normalize<NW, 7>(V, M);
    if (p < 0) {
#pragma unroll
      for (int q = 0; q < L; ++q) out[q] = 0.0;
      return;
    }
    operand_to_limbs<4, 7>(M, p + lsb + 1023, neg, out);
  } else {
    from_fixed_balanced<L, NW>(V, lsb, out);
  }
}

// The balanced-digit form of the above for any L (V is destroyed): the
// leading L 53-bit pieces and the next bit of |V| as balanced digits; for
// L = 2 the nearest DD, for L = 4 a nonoverlapping expansion that a QD
// renormalisation turns canonical.
template <int L, int NW>
__host__ __device__ __forceinline__ void from_fixed_balanced(uint32_t (&V)[NW], int lsb, double (&out)[L]) {
  const uint32_t neg = acc_abs<NW>(V);
  uint64_t ch[L + 1];
  int ex[L + 1];
  if (!acc_chunks<NW, L + 1>(V, ch, ex)) {
#pragma unroll
    for (int q = 0; q < L; ++q) out[q] = 0.0;
    return;
  }
  uint64_t c = ch[L] >> 52;  // the bit after the last piece
#pragma unroll
  for (int q = L - 1; q >= 0; --q) {
    int64_t v = (int64_t)ch[q] + (int64_t)c;
    c = 0u;
    if (q > 0 && v >= (int64_t)1 << 52) {
      v -= (int64_t)1 << 53;
      c = 1u;
    }
    const uint32_t dn = v < 0 ? 1u : 0u;
    out[q] = make_double((uint64_t)(v < 0 ? -v : v), lsb + ex[q], neg ^ dn);
  }
}

// ---------------------------------------------------------------------------
// Fixed-point scalars for latency-bound kernels (the LU's triangular solves).

// M = the W leading words of the nonnegative NW-word integer A, its leading
// one moved to bit 32 W - 1 (bits shifted out below are dropped); returns
// the position of A's leading one, or -1 if A = 0 (M = 0).
template <int NW, int W>
__host__ __device__ __forceinline__ int acc_normalize(const uint32_t (&A)[NW], uint32_t (&M)[W]) {
  static_assert(W <= NW, "operand wider than the source");
  uint32_t B[NW];
  const int top = acc_top_align<NW>(A, B);
  if (top < 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) M[w] = 0u;
    return -1;
  }
  const int lz = clz32(B[NW - 1]);
#pragma unroll
  for (int i = 0; i < W; ++i) M[W - 1 - i] = shl_funnel(NW - 2 - i >= 0 ? B[NW - 2 - i] : 0u, B[NW - 1 - i], lz);
  return 32 * top + 31 - lz;
}

// Arithmetic right shift of the two's-complement NW-word A by s >= 0 bits
// (word shifts by a barrel shifter with fixed indices, then a funnel shift).
template <int NW>
__host__ __device__ __forceinline__ void acc_sar(uint32_t (&A)[NW], int s) {
  if (s <= 0) return;
  const uint32_t fill = (A[NW - 1] >> 31) ? 0xFFFFFFFFu : 0u;
  const int w = s >> 5, r = s & 31;
  if (w >= NW) {
#pragma unroll
    for (int t = 0; t < NW; ++t) A[t] = fill;
    return;
  }
#pragma unroll
  for (int step = 8; step >= 1; step >>= 1) {
    if (step >= NW) continue;
    const bool on = (w & step) != 0;
#pragma unroll
    for (int t = 0; t < NW; ++t) A[t] = on ? (t + step < NW ? A[t + step < NW ? t + step : 0] : fill) : A[t];
  }
  if (r != 0) {
#pragma unroll
    for (int t = 0; t < NW; ++t) A[t] = shr_funnel(A[t], t + 1 < NW ? A[t + 1 < NW ? t + 1 : 0] : fill, r);
  }
}

// The expansion of L limbs nearest M 2^(e - 1075 - (32 W - 53)) (M with its
// leading one at bit 32 W - 1, sign s), greedily: each limb is the
// remaining value rounded to 53 bits (half up), the remainder kept exactly
// in W words and renormalised. Canonical (each limb at most half a unit
// in the last place of the one above) and integer-only except for
// assembling the doubles.
template <int L, int W>
__host__ __device__ __forceinline__ void operand_to_limbs(const uint32_t (&M)[W], int e, uint32_t s, double (&out)[L]) {
  uint32_t R[W];
#pragma unroll
  for (int w = 0; w < W; ++w) R[w] = M[w];
  int lead = e;  // exponent field of R's leading bit (R normalised)
  uint32_t neg = s;
#pragma unroll
  for (int q = 0; q < L; ++q) {
    // top 53 bits and the rounding bit of the normalised R
    const uint64_t top64 = ((uint64_t)R[W - 1] << 32) | R[W - 2];
    uint64_t h = top64 >> 11;                 // 53 bits
    const uint32_t rb = (uint32_t)(top64 >> 10) & 1u;
    if (h == 0u) {
#pragma unroll
      for (int t = q; t < L; ++t) out[t] = 0.0;
      return;
    }
    out[q] = make_double(h + rb, lead - 1075, neg);
    if (q + 1 == L) break;
    // remainder: R - (h + rb) 2^(32 W - 53); below the top 53 bits R holds
    // the rest r; if rb, the remainder is -(2^(32 W - 53) - r)
    R[W - 1] = 0u;
    R[W - 2] &= 0x7FFu;  // bits below the leading 53 (32 W - 53 = 32 (W - 2) + 11)
    if (rb) {
      // rounded up: the remainder is -(2^(32 W - 53) - r) with r >= 2^(32 W - 54)
      // the rest, i.e. the low 32 W - 53 bits of -r
      uint64_t c = 1u;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const uint64_t v = (uint64_t)(~R[w]) + c;
        R[w] = (uint32_t)v;
        c = v >> 32;
      }
      R[W - 1] = 0u;
      R[W - 2] &= 0x7FFu;
      neg ^= 1u;
    }
    uint32_t Rn[W];
    const int p = acc_normalize<W, W>(R, Rn);
    if (p < 0) {
#pragma unroll
      for (int t = q + 1; t < L; ++t) out[t] = 0.0;
      return;
    }
    lead -= (32 * W - 1) - p;
#pragma unroll
    for (int w = 0; w < W; ++w) R[w] = Rn[w];
  }
}

}  // namespace fx
}  // namespace ddg
