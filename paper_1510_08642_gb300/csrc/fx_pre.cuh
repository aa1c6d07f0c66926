// The pre-shifted form of the DD Block product (Kouya 2015, Section 2,
// Block with DD arithmetic), shared by the tile kernel (block_fx.cu) and
// the narrow kernel (gemv_fx.cu), so that both give the same bits.
//
// Each operand is shifted once, at staging, to the largest exponent of its
// row of A / column of B (its W = 4 words keep 22 bits beyond the 106 that
// DD needs), so that all products of an output share one scale and add
// into the window with no shift. Of each product only the words at columns
// D + 1 .. 2 W - 1 (D = W - 1) are formed: the columns below, which land in
// window word 0, are left out, except the high halves of the column-D
// partial products, which carry into column D + 1 (mul_top_hi).
//
// Error per term in window units (word 0 = 1 unit): the operands'
// truncation at their row / column maximum < 2^33, the columns left out and
// their carries < 2^35: < 2^35.33. Over l terms < l 2^35.33 units, which is
// below l 2^-106 |S| once the window sum keeps |S| >= 2^keep units
// (keep = 142): within the elementwise bound (2 l + 4) 2^-106
// sum_k |a_ik b_kj|. Both errors are zero when every operand's bits lie in
// its top two words at the shared scale (within 64 bits of its row / column
// maximum: small integers, for instance); such products are exact.
//
// An output whose window keeps fewer bits is recomputed on its own in the
// shifted form (every product to its own scale; fx_shifted_one), and, if
// that window too keeps fewer than 106 bits, with the window at its largest
// term (fx_rescue): each output's result depends on its own row and column
// only.
#pragma once

#include <cstdint>

#include "fx.cuh"
#include "fx_round.cuh"

namespace ddg {

template <int L> struct fxpre { static constexpr bool on = false; };
template <> struct fxpre<2> { static constexpr bool on = true; static constexpr int keep = 142; };

// M >> s for a W-word M (bits shifted out dropped; 0 for s >= 32 W): a
// funnel shift per word, then whole-word steps of 2 and 1 at fixed indices.
template <int W>
__device__ __forceinline__ void shr_words(uint32_t (&M)[W], int s) {
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

// acc (window words 1 .. 5; word 0 stays 0) += the term q with sign mask s
// (0 or ~0): (q XOR s, s) plus the carry s & 1 (two's complement; word 0 of
// -q is 0).
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

// The 6-word window (word 0 = 0) of the pre-shifted accumulator.
__device__ __forceinline__ void pre_window(const uint32_t (&acc)[5], uint32_t (&w)[6]) {
  w[0] = 0u;
#pragma unroll
  for (int t = 0; t < 5; ++t) w[t + 1] = acc[t];
}

}  // namespace ddg
