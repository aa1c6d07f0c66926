// Fixed-point scalars on the integer pipe for the LU's latency-bound steps
// (triangular solves, column updates, pivot reciprocals): a DD / QD value is
// an exact two's-complement window of NW 32-bit words with an anchor
// exponent, or a W-word operand M with its leading one at bit 32 W - 1
// (value M 2^(e - 1075 - (32 W - 53)), e the exponent field, s the sign).
// Host and device; pinned on the host against exact integers.
#pragma once

#include <cstdint>

#include "fx.cuh"

namespace ddg {

// Fixed-point widths of the triangular bases: operands as W-word integers
// (fx::to_fixed), products' K = 2 W - D leading words, NW-word windows
// with an operand of exponent field A at bit TOPA (so that a product of
// exponent fields e_l + e_x = A + 1023 lands at shift 0).
template <int L> struct tfx;
template <> struct tfx<2> { static constexpr int W = 4, D = 3, K = 5, NW = 6, TOPA = 106; };
template <> struct tfx<4> { static constexpr int W = 7, D = 6, K = 8, NW = 9, TOPA = 202; };

// One lane's running value x = acc 2^(A - 1075 - TOPA) as a fixed-point
// operand: leading one at bit 32 W - 1 of M, exponent field e, sign s; z set
// when the value is zero.
template <int L>
__host__ __device__ __forceinline__ void window_operand(const uint32_t (&acc)[tfx<L>::NW], int A, uint32_t (&M)[tfx<L>::W],
                                               int& e, uint32_t& s, bool& z) {
  constexpr int NW = tfx<L>::NW, W = tfx<L>::W;
  uint32_t mag[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) mag[w] = acc[w];
  s = fx::acc_abs<NW>(mag);
  const int p = fx::acc_normalize<NW, W>(mag, M);
  z = p < 0;
  e = p + A - 52 - tfx<L>::TOPA;
}

// acc -= (l x) for fixed-point operands l = (Ml, el, sl), x = (Mx, ex, sx):
// the product's leading words placed into the window, which moves up
// (arithmetic shift, A grows) when the product would not fit below its top.
template <int L>
__host__ __device__ __forceinline__ void window_sub_product(uint32_t (&acc)[tfx<L>::NW], int& A, const uint32_t (&Ml)[tfx<L>::W],
                                                   int el, uint32_t sl, const uint32_t (&Mx)[tfx<L>::W], int ex,
                                                   uint32_t sx) {
  constexpr int W = tfx<L>::W, D = tfx<L>::D, K = tfx<L>::K, NW = tfx<L>::NW;
  uint32_t P[K];
  fx::mul_top<W, D>(Ml, Mx, P);
  int shl = el + ex - A - 1023;
  if (shl > 0) {
    fx::acc_sar<NW>(acc, shl);
    A += shl;
    shl = 0;
  }
  fx::place_shr<NW, K>(acc, P, -shl, (sl ^ sx) ? 0u : 0xFFFFFFFFu);
}

// acc := the operand (M, e, s) exactly, as the window of anchor
// A = e + TOPA - (32 W - 53) (so that acc = +-M).
template <int L>
__host__ __device__ __forceinline__ void window_from_operand(uint32_t (&acc)[tfx<L>::NW], int& A, const uint32_t (&M)[tfx<L>::W],
                                                    int e, uint32_t s) {
  constexpr int W = tfx<L>::W, NW = tfx<L>::NW;
  A = e + tfx<L>::TOPA - (32 * W - 53);
  const uint32_t msk = s ? 0xFFFFFFFFu : 0u;
  uint64_t cy = msk & 1u;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint64_t v = (uint64_t)((w < W ? M[w] : 0u) ^ msk) + cy;
    acc[w] = (uint32_t)v;
    cy = v >> 32;
  }
}

// 1 / b in QD on the integer pipe from an approximation y0 + y1 of 1 / b
// (a DD reciprocal, ~2^-105): two Newton steps y := y + y (1 - b y), with
// 1 - b y and the update exact in fixed-point windows (up to the dropped
// partial products, ~2^-219) and y kept at 224 bits between the steps;
// rounded to QD once.
__host__ __device__ __forceinline__ void qd_recip_refine(const double (&b)[4], double y0, double y1, double (&out)[4]) {
  constexpr int W = tfx<4>::W, NW = tfx<4>::NW;
  uint32_t Mb[W], My[W];
  const int esb = fx::to_fixed<4, W>(b, Mb);
  const double yq[4] = {y0, y1, 0.0, 0.0};
  const int esy = fx::to_fixed<4, W>(yq, My);
  const int eb = esb & 0xFFFF;
  const uint32_t sb = (uint32_t)esb >> 16;
  int ey = esy & 0xFFFF;
  uint32_t sy = (uint32_t)esy >> 16;
  const double one[4] = {1.0, 0.0, 0.0, 0.0};
#pragma unroll 1
  for (int it = 0; it < 2; ++it) {
    uint32_t acc[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) acc[w] = 0u;
    int A = 1023;
    fx::add_at<4, NW>(acc, one, A, tfx<4>::TOPA, 0u);
    window_sub_product<4>(acc, A, Mb, eb, sb, My, ey, sy);  // 1 - b y
    uint32_t Me[W], se;
    int ee;
    bool ze;
    window_operand<4>(acc, A, Me, ee, se, ze);
    if (ze) break;
    int A2;
    window_from_operand<4>(acc, A2, My, ey, sy);
    window_sub_product<4>(acc, A2, My, ey, sy, Me, ee, se ^ 1u);  // + y e
    bool zy;
    window_operand<4>(acc, A2, My, ey, sy, zy);
  }
  fx::operand_to_limbs<4, W>(My, ey, sy, out);
}


}  // namespace ddg
