// Window constants of the integer-pipe products and the rounding of a
// finished window to DD / QD (the epilogue shared by the Block kernel and
// the column-vector kernel).
//
// Operands are W-word fixed-point integers (fx::to_fixed, the leading
// limb's significand LSB at bit 32 W - 53); a product keeps the K = 2 W - D
// leading words of M_a M_b (fx::mul_top) and is shifted into an NW-word
// two's-complement window by the operands' distances below the largest
// exponent fields f_a (row of A) and f_b (column of B). The window's LSB then
// has exponent f_a + f_b + LSB0:
//   DD: W = 4, D = 3: unit of M is 2^(e - 1150), word D is 2^96 of M_a M_b,
//       LSB0 = 96 - 2 * 1150 = -2204;
//   QD: W = 7, D = 6: unit 2^(e - 1246), word D is 2^192, LSB0 = -2300.
#pragma once

#include "arith.cuh"
#include "fx.cuh"

namespace ddg {

template <int L> struct fxwin;
template <> struct fxwin<2> {
  static constexpr int W = 4, D = 3, K = 2 * W - D, NW = 6, LSB0 = -2204;
};
template <> struct fxwin<4> {
  static constexpr int W = 7, D = 6, K = 2 * W - D, NW = 9, LSB0 = -2300;
};

// chunk 2^k with the sign mask neg; 0 below the subnormal range
__device__ __forceinline__ double fx_scaled(uint64_t chunk, int k, uint32_t neg) {
  if (chunk == 0 || k < -2044) return 0.0;
  double v = fx::pow2_product(__ull2double_rn(chunk), k > 2046 ? 2046 : k);
  return neg ? -v : v;
}

// The window A (consumed: replaced by its magnitude) rounded to DD / QD,
// its LSB having exponent lsb: the magnitude cut into 53-bit chunks from its
// leading bit, each converted exactly, then renormalised (two_sum for DD,
// qd_renorm for QD).
template <int L, int NW>
__device__ __forceinline__ typename num<L>::T window_round(uint32_t (&A)[NW], int lsb) {
  const uint32_t neg = fx::acc_abs<NW>(A);
  typename num<L>::T v;
  if constexpr (L == 2) {
    uint64_t ch[2];
    int ex[2];
    double hi = 0.0, lo = 0.0;
    if (fx::acc_chunks<NW, 2>(A, ch, ex)) {
      hi = fx_scaled(ch[0], lsb + ex[0], neg);
      lo = fx_scaled(ch[1], lsb + ex[1], neg);
    }
    two_sum(hi, lo, v.hi, v.lo);
  } else {
    uint64_t ch[4];
    int ex[4];
    double x[4] = {0.0, 0.0, 0.0, 0.0};
    if (fx::acc_chunks<NW, 4>(A, ch, ex)) {
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = fx_scaled(ch[q], lsb + ex[q], neg);
    }
    v = qd_renorm<4>(x);
  }
  return v;
}

}  // namespace ddg
