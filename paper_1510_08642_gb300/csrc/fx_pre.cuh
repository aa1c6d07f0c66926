// The pre-shifted form of the DD / QD Block product (Kouya 2015, Section 2,
// Block with DD / QD arithmetic), shared by the tile kernel (block_fx.cu)
// and the narrow kernel (gemv_fx.cu), so that both give the same bits.
//
// Each operand is shifted once, at staging, to the largest exponent of its
// row of A / column of B (its W words keep 22 bits beyond the 106 that DD
// needs with W = 4, 12 beyond QD's 212 with W = 7), so that all products of
// an output share one scale and add into the window with no shift. Of each
// product only the words at columns D + 1 .. 2 W - 1 (D = W - 1) are
// formed: the columns below, which land in window word 0, are left out,
// except the high halves of the column-D partial products, which carry into
// column D + 1 (fx::mul_top_hi).
//
// Error per term in window units (word 0 = 1 unit): the operands'
// truncation at their row / column maximum < 2^33, the columns left out and
// their carries < 2 W 2^32: < 2^35.33 (DD) / 2^36 (QD). Over l terms that
// is below l 2^-106 |S| (DD) / l 2^-209 |S| (QD) once the window sum keeps
// |S| >= 2^keep units (keep = 142 / 245; the largest product is below
// 2^160 / 2^256 units): within the elementwise bounds (2 l + 4) 2^-106
// (DD) / (2 l + 4) 2^-209 (QD) of sum_k |a_ik b_kj|. Both errors are zero
// when every operand's bits lie in its top two words at the shared scale
// (within 64 bits of its row / column maximum: small integers, for
// instance); such products are exact.
//
// An output whose window keeps fewer bits is recomputed on its own in the
// shifted form (every product to its own scale), by the whole warp with the
// lanes splitting k (warp_shifted_one), and, if that window too keeps fewer
// than 53 L bits, with the window at its largest term: each output's result
// depends on its own row and column only.
#pragma once

#include <cstdint>

#include "fx.cuh"
#include "fx_round.cuh"

namespace ddg {

template <int L> struct fxpre;
template <> struct fxpre<2> { static constexpr int keep = 142; };
template <> struct fxpre<4> { static constexpr int keep = 245; };

// M >> s for a W-word M (bits shifted out dropped; 0 for s >= 32 W): a
// funnel shift per word, then whole-word steps of 2 and 1 at fixed indices.
template <int W>
__host__ __device__ __forceinline__ void shr_words(uint32_t (&M)[W], int s) {
  if (s <= 0) return;
  if (s >= 32 * W) {
#pragma unroll
    for (int t = 0; t < W; ++t) M[t] = 0u;
    return;
  }
  const int r = s & 31, q = s >> 5;
#pragma unroll
  for (int t = 0; t < W; ++t) M[t] = fx::shr_funnel(M[t], t + 1 < W ? M[t + 1] : 0u, r);
  if (q >= 4) {
#pragma unroll
    for (int t = 0; t < W; ++t) M[t] = t + 4 < W ? M[t + 4] : 0u;
  }
  if (q & 2) {
#pragma unroll
    for (int t = 0; t < W; ++t) M[t] = t + 2 < W ? M[t + 2] : 0u;
  }
  if (q & 1) {
#pragma unroll
    for (int t = 0; t < W; ++t) M[t] = t + 1 < W ? M[t + 1] : 0u;
  }
}

// acc (window words 1 .. NW - 1; word 0 stays 0) += the term q (W = NW - 2
// words) with sign mask s (0 or ~0): (q XOR s, s) plus the carry s & 1
// (two's complement; word 0 of -q is 0).
#ifdef __CUDACC__
__device__ __forceinline__ void pre_add(uint32_t (&acc)[5], const uint32_t (&q)[4], uint32_t s) {
  asm("{\n\t.reg .u32 t;\n\t"
      "add.cc.u32 t, %9, %9;\n\t"
      "addc.cc.u32 %0, %0, %5;\n\t"
      "addc.cc.u32 %1, %1, %6;\n\t"
      "addc.cc.u32 %2, %2, %7;\n\t"
      "addc.cc.u32 %3, %3, %8;\n\t"
      "addc.u32 %4, %4, %9;\n\t}"
      : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2]), "+r"(acc[3]), "+r"(acc[4])
      : "r"(q[0] ^ s), "r"(q[1] ^ s), "r"(q[2] ^ s), "r"(q[3] ^ s), "r"(s));
}

__device__ __forceinline__ void pre_add(uint32_t (&acc)[8], const uint32_t (&q)[7], uint32_t s) {
  asm("{\n\t.reg .u32 t;\n\t"
      "add.cc.u32 t, %15, %15;\n\t"
      "addc.cc.u32 %0, %0, %8;\n\t"
      "addc.cc.u32 %1, %1, %9;\n\t"
      "addc.cc.u32 %2, %2, %10;\n\t"
      "addc.cc.u32 %3, %3, %11;\n\t"
      "addc.cc.u32 %4, %4, %12;\n\t"
      "addc.cc.u32 %5, %5, %13;\n\t"
      "addc.cc.u32 %6, %6, %14;\n\t"
      "addc.u32 %7, %7, %15;\n\t}"
      : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2]), "+r"(acc[3]), "+r"(acc[4]), "+r"(acc[5]), "+r"(acc[6]),
        "+r"(acc[7])
      : "r"(q[0] ^ s), "r"(q[1] ^ s), "r"(q[2] ^ s), "r"(q[3] ^ s), "r"(q[4] ^ s), "r"(q[5] ^ s), "r"(q[6] ^ s),
        "r"(s));
}

#endif

// The NW-word window (word 0 = 0) of the pre-shifted accumulator.
template <int NW>
__host__ __device__ __forceinline__ void pre_window(const uint32_t (&acc)[NW - 1], uint32_t (&w)[NW]) {
  w[0] = 0u;
#pragma unroll
  for (int t = 0; t < NW - 1; ++t) w[t + 1] = acc[t];
}

}  // namespace ddg
