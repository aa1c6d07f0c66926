// Elementwise accuracy of the integer-pipe Block product (Kouya 2015,
// Section 2, Block with DD / QD arithmetic: every c_ij is accurate relative
// to its own sum_k |a_ik b_kj|).
//
// The Block kernels fix the window of an output c_ij from the largest
// exponent field of row i of A (f_a) and of column j of B (f_b): the window
// keeps 2^-159 (DD) / 2^-255 (QD) of 2^(f_a + f_b) and truncates below. When
// the two maxima sit at different k and every actual product a_ik b_kj is
// far below 2^(f_a + f_b) (row [2^200, 2^-200] times column [2^-200,
// 2^200]: both products are 1, the window sees nothing), the truncation is
// not small relative to sum_k |a_ik b_kj|.
//
// Test and rescue: the window sum S (in window units, error < l units) is
// accepted when |S| >= 2^(53 L); then sum_k |a_ik b_kj| >= |c_ij| >= 2^(53 L
// - 1) units and the truncation, l units, is within 2 l 2^-(53 L) of it.
// Otherwise the output is recomputed with its window anchored at its own
// largest term: E = max_k (f(a_ik) + f(b_kj)) over the nonzero pairs, each
// term shifted by E - f(a_ik) - f(b_kj), window LSB at 2^(E + LSB0). The
// truncation per term is then below 2^-158 (DD) / 2^-254 (QD) of
// max_k |a_ik b_kj| <= sum_k |a_ik b_kj|. Ordinary inputs (no cancellation
// beyond 2^-53 of max|a_i.| max|b_.j|) never take the rescue, and their bits
// are those of the plain window.
#pragma once

#include "fx_round.cuh"
#include "kernels.cuh"

namespace ddg {

// Significant window bits an output must keep to skip the rescue.
template <int L> struct fxkeep { static constexpr int bits = 53 * L; };

// Exponent fields f(a) + f(b) of the pair (a, b) at offsets ao of A and bo
// of B (fields >= 1, as fx::to_fixed gives them), or -1 if a or b is zero.
template <int L, bool PRE>
__device__ __forceinline__ int fx_pair_field(const mat& A, const mat& B, const fxop& Ax, const fxop& Bx, int64_t ao,
                                             int64_t bo) {
  if constexpr (PRE) {
    const int fa = Ax.f[ao], fb = Bx.f[bo];
    if (fa == FX_ZERO || fb == FX_ZERO) return -1;
    return (fa & 0xFFFF) + (fb & 0xFFFF);
  } else {
    const double a = A.p[0][ao], b = B.p[0][bo];
    if ((fx::dbits(a) << 1) == 0u || (fx::dbits(b) << 1) == 0u) return -1;
    return max(fx::expfield(a), 1) + max(fx::expfield(b), 1);
  }
}

// acc += a b placed E - f(a) - f(b) bits below the window top of anchor E.
template <int L, bool PRE>
__device__ __forceinline__ void fx_pair_place(const mat& A, const mat& B, const fxop& Ax, const fxop& Bx, int64_t ao,
                                              int64_t bo, int E, uint32_t (&acc)[fxwin<L>::NW]) {
  using F = fxwin<L>;
  constexpr int W = F::W, D = F::D, K = F::K, NW = F::NW;
  const int e = fx_pair_field<L, PRE>(A, B, Ax, Bx, ao, bo);
  if (e < 0 || E - e >= 32 * K) return;  // zero, or every bit below the window
  uint32_t ma[W], mb[W];
  uint32_t sgn;
  if constexpr (PRE) {
    constexpr int WV = (W + 3) / 4;
    uint32_t wa[4 * WV], wb[4 * WV];
#pragma unroll
    for (int v = 0; v < WV; ++v) {
      const uint4 qa = Ax.w[ao * WV + v], qb = Bx.w[bo * WV + v];
      wa[4 * v] = qa.x; wa[4 * v + 1] = qa.y; wa[4 * v + 2] = qa.z; wa[4 * v + 3] = qa.w;
      wb[4 * v] = qb.x; wb[4 * v + 1] = qb.y; wb[4 * v + 2] = qb.z; wb[4 * v + 3] = qb.w;
    }
#pragma unroll
    for (int t = 0; t < W; ++t) ma[t] = wa[t], mb[t] = wb[t];
    sgn = (((Ax.f[ao] ^ Bx.f[bo]) >> 16) & 1) ? 0xFFFFFFFFu : 0u;
  } else {
    double xa[L], xb[L];
#pragma unroll
    for (int q = 0; q < L; ++q) xa[q] = A.p[q][ao], xb[q] = B.p[q][bo];
    const int ea = fx::to_fixed<L, W>(xa, ma);
    const int eb = fx::to_fixed<L, W>(xb, mb);
    sgn = ((ea ^ eb) >> 16) ? 0xFFFFFFFFu : 0u;
  }
  uint32_t p[K];
  fx::mul_top<W, D>(ma, mb, p);
  fx::place_shr<NW, K>(acc, p, E - e, sgn);
}

template <int L> struct fxacc {
  uint32_t w[fxwin<L>::NW];
  int lsb;
};

// The window sum of output c_ij with its window anchored at E (every term
// placed E - f(a_ik) - f(b_kj) bits below the window top, as fx_pair_place),
// by one thread; with E = f_a + f_b (the row / column maxima) this is the
// window of the Block kernels' shifted form, term for term.
template <int L, bool PRE>
__device__ __forceinline__ void fx_window_at(int64_t l, const mat& A, const mat& B, const fxop& Ax, const fxop& Bx,
                                             int64_t gi, int64_t gj, int E, uint32_t (&w)[fxwin<L>::NW]) {
  const int64_t ald = PRE ? Ax.ld : A.ld, bld = PRE ? Bx.ld : B.ld;
#pragma unroll
  for (int t = 0; t < fxwin<L>::NW; ++t) w[t] = 0u;
  for (int64_t k = 0; k < l; ++k) fx_pair_place<L, PRE>(A, B, Ax, Bx, gi * ald + k, k * bld + gj, E, w);
}

// One output c_ij recomputed by one thread with the window anchored at its
// largest term (two passes over k; rare, kept out of line so that the
// Block kernels' main loops are compiled as without it).
template <int L, bool PRE>
__device__ __noinline__ fxacc<L> fx_rescue(int64_t l, mat A, mat B, fxop Ax, fxop Bx, int64_t gi, int64_t gj) {
  const int64_t ald = PRE ? Ax.ld : A.ld, bld = PRE ? Bx.ld : B.ld;
  int E = -1;
  for (int64_t k = 0; k < l; ++k) E = max(E, fx_pair_field<L, PRE>(A, B, Ax, Bx, gi * ald + k, k * bld + gj));
  fxacc<L> r;
#pragma unroll
  for (int w = 0; w < fxwin<L>::NW; ++w) r.w[w] = 0u;
  r.lsb = 0;
  if (E < 0) return r;  // every term is zero
  fx_window_at<L, PRE>(l, A, B, Ax, Bx, gi, gj, E, r.w);
  r.lsb = E + fxwin<L>::LSB0;
  return r;
}

// Output c_ij in the shifted form with window anchor fab = f_a + f_b, and,
// if that window keeps fewer than 53 L bits, the rescue: the result the
// Block kernels' shifted form gives for it (one thread, out of line).
template <int L, bool PRE>
__device__ __noinline__ fxacc<L> fx_shifted_one(int64_t l, mat A, mat B, fxop Ax, fxop Bx, int64_t gi, int64_t gj,
                                                int fab) {
  fxacc<L> r;
  fx_window_at<L, PRE>(l, A, B, Ax, Bx, gi, gj, fab, r.w);
  r.lsb = fab + fxwin<L>::LSB0;
  if (fx::acc_mag_below<fxwin<L>::NW>(r.w, fxkeep<L>::bits)) r = fx_rescue<L, PRE>(l, A, B, Ax, Bx, gi, gj);
  return r;
}

}  // namespace ddg
