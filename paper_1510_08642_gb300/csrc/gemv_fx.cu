// Block product for narrow right operands (n <= GEMV_MAX_N columns of B and
// C): the same integer-pipe multiply-add and window as the Block kernel
// (Kouya 2015, Section 2, Block; block_fx.cu), arranged as a dot product per
// output. The Block kernel's 16 x 32 output tile leaves most of its columns
// idle when n is tiny (b = A 1, and the triangular solves of an LU solve
// with one right-hand side, Section 4 Eq. 2), and each of its few CTAs runs
// the whole k loop alone; here one warp takes one output c_ij and its lanes
// split k:
//   * the largest exponent fields of row i of A and column j of B (a warp
//     max reduction) fix the window scale, exactly as in the Block kernel;
//   * lane t accumulates the terms k = t, t + 32, ... into its own window
//     in the pre-shifted form (fx::to_fixed, shr_words, fx::mul_top_hi);
//   * the 32 windows are summed exactly across the warp (butterfly of
//     multiword two's-complement additions; the window has 32 bits of
//     headroom, enough for l < 2^31 terms in any order);
//   * lane 0 rounds the window once (window_round) and applies the mode.
//   * an output whose window keeps fewer than fxpre<L>::keep bits is
//     recomputed by the warp in the shifted form, and then, if it keeps
//     fewer than 53 L significant bits, with the window at its own largest
//     term (warp_shifted_one, fx_rescue.cuh), as in the Block kernel.
// The result is the one the Block kernel's arithmetic defines: every term
// carries the same truncations, and the window sum is exact, so the order
// of the terms does not matter.
#include "fx_pre.cuh"
#include "fx_rescue.cuh"
#include "fx_round.cuh"
#include "kernels.cuh"

namespace ddg {

namespace {

constexpr int GV_WARPS = 8;  // outputs per CTA

template <int L>
__device__ __forceinline__ void load_limbs(const mat& M, int64_t off, double (&x)[L]) {
#pragma unroll
  for (int q = 0; q < L; ++q) x[q] = M.p[q][off];
}

template <int L>
__global__ void __launch_bounds__(32 * GV_WARPS) gemv_fx_kernel(int64_t m, int64_t l, int64_t n, mat A, mat B,
                                                                mat C, int mode) {
  using F = fxwin<L>;
  constexpr int W = F::W, NW = F::NW;
  const int lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * GV_WARPS + (threadIdx.x >> 5);
  if (e >= m * n) return;  // warp-uniform
  const int64_t i = e / n, j = e % n;
  const int64_t arow = i * A.ld;

  int fa = 1, fb = 1;
  for (int64_t k = lane; k < l; k += 32) {
    fa = max(fa, fx::expfield(A.p[0][arow + k]));
    fb = max(fb, fx::expfield(B.p[0][k * B.ld + j]));
  }
  fa = __reduce_max_sync(0xffffffffu, fa);
  fb = __reduce_max_sync(0xffffffffu, fb);

  using N = num<L>;
  auto finish = [&](uint32_t(&w)[NW], int lsb) {
    typename N::T v = window_round<L, NW>(w, lsb);
    const int64_t off = i * C.ld + j;
    if (mode == MODE_ADD) v = N::add(N::load(C.p, off), v);
    else if (mode == MODE_SUB) v = N::add(N::load(C.p, off), N::neg(v));
    N::store(C.p, off, v);
  };
  {
    // the pre-shifted form (fx_pre.cuh), as the tile kernel stages it; its
    // window is kept when it reaches fxpre<L>::keep bits
    uint32_t pa[NW - 1];
#pragma unroll
    for (int t = 0; t < NW - 1; ++t) pa[t] = 0u;
    for (int64_t k = lane; k < l; k += 32) {
      double xa[L], xb[L];
      load_limbs<L>(A, arow + k, xa);
      load_limbs<L>(B, k * B.ld + j, xb);
      uint32_t ma[W], mb[W];
      const int ea = fx::to_fixed<L, W>(xa, ma);
      const int eb = fx::to_fixed<L, W>(xb, mb);
      const bool za = (fx::dbits(xa[0]) << 1) == 0u, zb = (fx::dbits(xb[0]) << 1) == 0u;
      shr_words<W>(ma, za ? 32 * W : fa - (ea & 0xFFFF));
      shr_words<W>(mb, zb ? 32 * W : fb - (eb & 0xFFFF));
      const uint32_t sa = ((ea >> 16) & 1) && !za ? 0xFFFFFFFFu : 0u;
      const uint32_t sb = ((eb >> 16) & 1) && !zb ? 0xFFFFFFFFu : 0u;
      uint32_t q[W];
      fx::mul_top_hi<W>(ma, mb, q);
      pre_add(pa, q, sa ^ sb);
    }
    uint32_t acc[NW];
    pre_window<NW>(pa, acc);
    warp_window_sum<NW>(acc);
    if (!fx::acc_mag_below<NW>(acc, fxpre<L>::keep)) {  // warp-uniform: every lane holds the total
      if (lane == 0) finish(acc, fa + fb + F::LSB0);
      return;
    }
  }
  // below the threshold: the shifted form by the whole warp, then, if
  // needed, the window at the largest term (fx_rescue.cuh)
  fxacc<L> x = warp_shifted_one<L, false>(l, A, B, fxop{}, fxop{}, i, j, fa + fb);
  if (lane == 0) finish(x.w, x.lsb);
}

}  // namespace

cudaError_t launch_gemv_fx(int limbs, int64_t m, int64_t l, int64_t n, mat A, mat B, mat C, int mode,
                           cudaStream_t s) {
  if (m == 0 || n == 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  const unsigned grid = (unsigned)((m * n + GV_WARPS - 1) / GV_WARPS);
  if (limbs == 2) gemv_fx_kernel<2><<<grid, 32 * GV_WARPS, 0, s>>>(m, l, n, A, B, C, mode);
  else gemv_fx_kernel<4><<<grid, 32 * GV_WARPS, 0, s>>>(m, l, n, A, B, C, mode);
  cudaError_t e = cudaGetLastError();
  if (ev) {
    const double bytes = 8.0 * limbs * ((double)m * l + (double)l * n + (double)m * n * (mode == MODE_SET ? 1 : 2));
    prof_end_launch(s, ev, PROF_GEMV, (double)m * (double)l * (double)n, bytes);
  }
  return e;
}

}  // namespace ddg
