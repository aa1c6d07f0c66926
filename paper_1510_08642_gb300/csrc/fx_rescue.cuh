// Elementwise accuracy of the integer-pipe Block product (Kouya 2015,
// Section 2, Block with DD / QD arithmetic: every c_ij is accurate relative
// to its own sum_k |a_ik b_kj|): the per-output paths behind the
// pre-shifted form (fx_pre.cuh).
//
// Shifted form: each term a_ik b_kj of an output is formed at its own scale
// (fx::mul_top of the operands' full words) and placed E - f(a_ik) - f(b_kj)
// bits below the top of a window anchored at E; with E = f_a + f_b (the
// largest exponent fields of row i of A and column j of B) the window keeps
// 2^-159 (DD) / 2^-255 (QD) of 2^(f_a + f_b) and truncates below. When the
// two maxima sit at different k and every actual product a_ik b_kj is far
// below 2^(f_a + f_b) (row [2^200, 2^-200] times column [2^-200, 2^200]:
// both products are 1, the window sees nothing), that truncation is not
// small relative to sum_k |a_ik b_kj|.
//
// Test and rescue: the window sum S (in window units, error < l units) is
// accepted when |S| >= 2^(53 L); then sum_k |a_ik b_kj| >= |c_ij| >= 2^(53 L
// - 1) units and the truncation, l units, is within 2 l 2^-(53 L) of it.
// Otherwise the output is recomputed with its window anchored at its own
// largest term: E = max_k (f(a_ik) + f(b_kj)) over the nonzero pairs, window
// LSB at 2^(E + LSB0). The truncation per term is then below 2^-158 (DD) /
// 2^-254 (QD) of max_k |a_ik b_kj| <= sum_k |a_ik b_kj|.
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

// The exact sum of the 32 lanes' windows, in every lane (a butterfly of
// multiword two's-complement additions; the order does not matter).
template <int NW>
__device__ __forceinline__ void warp_window_sum(uint32_t (&w)[NW]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    uint32_t o[NW];
#pragma unroll
    for (int t = 0; t < NW; ++t) o[t] = __shfl_xor_sync(0xffffffffu, w[t], off);
    fx::acc_add_mask<NW>(w, o, 0u);
  }
}

// Output c_ij in the shifted form by one whole warp (warp-uniform
// arguments; the lanes split k): the window at anchor fab = f_a + f_b, and,
// if it keeps fewer than 53 L bits, the window at the largest term. The
// same terms and exact sums whatever the order; the result in every lane.
template <int L, bool PRE>
__device__ __forceinline__ fxacc<L> warp_shifted_one(int64_t l, const mat& A, const mat& B, const fxop& Ax,
                                                     const fxop& Bx, int64_t gi, int64_t gj, int fab) {
  constexpr int NW = fxwin<L>::NW;
  const int lane = threadIdx.x & 31;
  const int64_t ald = PRE ? Ax.ld : A.ld, bld = PRE ? Bx.ld : B.ld;
  fxacc<L> r;
#pragma unroll
  for (int t = 0; t < NW; ++t) r.w[t] = 0u;
  for (int64_t k = lane; k < l; k += 32) fx_pair_place<L, PRE>(A, B, Ax, Bx, gi * ald + k, k * bld + gj, fab, r.w);
  warp_window_sum<NW>(r.w);
  r.lsb = fab + fxwin<L>::LSB0;
  if (fx::acc_mag_below<NW>(r.w, fxkeep<L>::bits)) {
    int E = -1;
    for (int64_t k = lane; k < l; k += 32) E = max(E, fx_pair_field<L, PRE>(A, B, Ax, Bx, gi * ald + k, k * bld + gj));
    E = __reduce_max_sync(0xffffffffu, E);
#pragma unroll
    for (int t = 0; t < NW; ++t) r.w[t] = 0u;
    r.lsb = 0;
    if (E >= 0) {
      for (int64_t k = lane; k < l; k += 32)
        fx_pair_place<L, PRE>(A, B, Ax, Bx, gi * ald + k, k * bld + gj, E, r.w);
      warp_window_sum<NW>(r.w);
      r.lsb = E + fxwin<L>::LSB0;
    }
  }
  return r;
}

}  // namespace ddg
