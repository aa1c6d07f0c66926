// Block product with fixed-point accumulation on the integer pipe (Kouya
// 2015, Section 2, Block: C_ij = sum_k A_ik B_kj over tiles; the recursion's
// base case).
//
// GB300 retires 2 FP64 instructions per clock per SM but 64 IMAD and 128
// other integer instructions, so the multiply-add runs without FP64:
//   * staging: every element of the A and B tiles is converted once into a
//     W-word fixed-point integer M (its limbs summed exactly at their own
//     offsets below the leading limb's significand; W = 4 words for DD,
//     7 for QD; fx::to_fixed) and shifted to the largest exponent of its
//     row of A / column of B; its sign kept as a mask (fx_pre.cuh);
//   * multiply-add: the upper W words of M_a M_b (fx::mul_top_hi: the
//     partial products with i + j >= W and the high halves of those with
//     i + j = W - 1; 16 IMAD for DD, 49 for QD), added unshifted into a
//     two's-complement window of NW = W + 2 words per output whose scale
//     is fixed before the k loop from those maxima;
//   * epilogue: the window rounded to DD / QD once; an output that keeps
//     too few window bits is recomputed by its warp in the shifted form and
//     rescued if needed (fx_rescue.cuh).
// Conversion once per operand: a tile of A is staged by every CTA of its row
// of tiles (n / BN of them) and a tile of B by m / BM CTAs, so converting on
// the fly repeats to_fixed for each element that often. For products with
// many tiles the conversion runs once per element in its own elementwise
// kernel (fx_convert_kernel, into scratch the caller provides) and the Block
// kernel stages the converted words by plain copies (block_fxc_kernel); the
// words, shifts and therefore the results are the same bits either way.
// Error per term and the acceptance test: fx_pre.cuh; the sum in the window
// is exact for l < 2^31; one final rounding to DD / QD.
#include <algorithm>
#include <type_traits>

#include "arith.cuh"
#include "fx.cuh"
#include "fx_pre.cuh"
#include "fx_rescue.cuh"
#include "fx_round.cuh"
#include "kernels.cuh"

namespace ddg {

namespace {

template <int L> struct fxcfg;
template <> struct fxcfg<2> : fxwin<2> {
  static constexpr int BM = 16, BN = 32, BK = 16, TM = 2, TN = 2;
  static constexpr int MINB = 8;  // resident CTAs per SM (register cap 64; 7 at 72 measured 3% slower)
};
template <> struct fxcfg<4> : fxwin<4> {
  static constexpr int BM = 8, BN = 32, BK = 16, TM = 1, TN = 2;
  static constexpr int MINB = 8;
};


}  // namespace

// Operand tiles in fixed-point form: the W words of each element as WV
// 16-byte vectors (vector v of all elements in one plane, so that a warp's
// reads of consecutive elements are consecutive), and per element its shift
// below the largest exponent of its row (A) / column (B) and its sign mask.
// The A tile is padded by one row: its staging writes run along k.
template <int L>
struct fx_smem {
  static constexpr int WV = (fxcfg<L>::W + 3) / 4;
  uint4 Aw[WV][fxcfg<L>::BK][fxcfg<L>::BM + 1];
  uint4 Bw[WV][fxcfg<L>::BK][fxcfg<L>::BN];
  int As[fxcfg<L>::BK][fxcfg<L>::BM + 1];  // sign masks (0 or -1)
  int Bs[fxcfg<L>::BK][fxcfg<L>::BN];
  int row_f[fxcfg<L>::BM], col_f[fxcfg<L>::BN];
};

namespace {

// Store one element's words shifted to its row / column maximum fmax
// (fx_pre.cuh; a zero stores 0) and its sign mask.
template <int L>
__device__ __forceinline__ void put_staged(uint32_t (&M)[4 * fx_smem<L>::WV], bool zero, int f, int fmax, uint4* w,
                                           int stride, int* sgn) {
  constexpr int W = fxcfg<L>::W, WV = fx_smem<L>::WV;
  shr_words<W>(*reinterpret_cast<uint32_t(*)[W]>(M), zero ? 32 * W : fmax - (f & 0xFFFF));
#pragma unroll
  for (int v = 0; v < WV; ++v) w[v * stride] = make_uint4(M[4 * v], M[4 * v + 1], M[4 * v + 2], M[4 * v + 3]);
  *sgn = ((f >> 16) & 1) && !zero ? -1 : 0;
}

// Convert one element (to_fixed) and stage it.
template <int L>
__device__ __forceinline__ void stage(const double (&x)[L], int fmax, uint4* w, int stride, int* sgn) {
  constexpr int W = fxcfg<L>::W, WV = (W + 3) / 4;
  uint32_t M[4 * WV];
  uint32_t(&Mw)[W] = *reinterpret_cast<uint32_t(*)[W]>(M);
  const int es = fx::to_fixed<L, W>(x, Mw);
#pragma unroll
  for (int t = W; t < 4 * WV; ++t) M[t] = 0u;
  const bool zero = (fx::dbits(x[0]) << 1) == 0u;
  put_staged<L>(M, zero, es, fmax, w, stride, sgn);
}

// The same staging from a converted operand: its words and f as to_fixed
// gave them.
template <int L>
__device__ __forceinline__ void stage_pre(bool ok, const fxop& X, int64_t e, int fmax, uint4* w, int stride,
                                          int* sgn) {
  constexpr int WV = fx_smem<L>::WV;
  uint32_t M[4 * WV];
#pragma unroll
  for (int v = 0; v < WV; ++v) {
    const uint4 q = ok ? X.w[e * WV + v] : make_uint4(0u, 0u, 0u, 0u);
    M[4 * v] = q.x; M[4 * v + 1] = q.y; M[4 * v + 2] = q.z; M[4 * v + 3] = q.w;
  }
  const int f = ok ? X.f[e] : FX_ZERO;
  put_staged<L>(M, f == FX_ZERO, f, fmax, w, stride, sgn);
}

}  // namespace

// Largest exponent field of the leading limb per row of A and column of B
// for the tile at (i0, j0), into sm.row_f / sm.col_f (at least 1).
template <int L, bool PRE>
__device__ __forceinline__ void fx_maxima(int64_t m, int64_t l, int64_t n, const mat& A, const mat& B, int64_t i0,
                                          int64_t j0, fx_smem<L>& sm, const fxop& Ax, const fxop& Bx) {
  using P = fxcfg<L>;
  constexpr int BM = P::BM, BN = P::BN, TM = P::TM, TN = P::TN;
  constexpr int NT = (BN / TN) * (BM / TM);
  auto& row_f = sm.row_f;
  auto& col_f = sm.col_f;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int c = tid; c < BN; c += NT) col_f[c] = 1;
  for (int r = warp; r < BM; r += NT / 32) {
    int f = 1;
    const int64_t gi = i0 + r;
    if (gi < m) {
      if constexpr (PRE) {
        for (int64_t k = lane; k < l; k += 32) f = max(f, Ax.f[gi * Ax.ld + k] & 0xFFFF);
      } else {
        for (int64_t k = lane; k < l; k += 32) f = max(f, fx::expfield(A.p[0][gi * A.ld + k]));
      }
    }
    f = __reduce_max_sync(0xffffffffu, f);
    if (lane == 0) row_f[r] = f;
  }
  __syncthreads();
  {
    const int c = tid % BN;
    const int64_t gj = j0 + c;
    int f = 1;
    if (gj < n) {
      if constexpr (PRE) {
        for (int64_t k = tid / BN; k < l; k += NT / BN) f = max(f, Bx.f[k * Bx.ld + gj] & 0xFFFF);
      } else {
        for (int64_t k = tid / BN; k < l; k += NT / BN) f = max(f, fx::expfield(B.p[0][k * B.ld + gj]));
      }
    }
    atomicMax(&col_f[c], f);
  }
  __syncthreads();
}

// The tile in the pre-shifted form (fx_pre.cuh).
template <int L, bool PRE>
__device__ __forceinline__ void fx_pre(int64_t m, int64_t l, int64_t n, const mat& A, const mat& B, const mat& C,
                                       int mode, int64_t i0, int64_t j0, fx_smem<L>& sm, const fxop& Ax,
                                       const fxop& Bx) {
  using P = fxcfg<L>;
  constexpr int BM = P::BM, BN = P::BN, BK = P::BK, TM = P::TM, TN = P::TN, NW = P::NW, W = P::W;
  constexpr int WV = fx_smem<L>::WV, NP = NW - 1;
  static_assert(NW == W + 2, "pre-shifted form: window of W + 2 words");
  constexpr int NX = BN / TN, NY = BM / TM, NT = NX * NY;
  auto& row_f = sm.row_f;
  auto& col_f = sm.col_f;
  const int tid = threadIdx.x;
  const int tx = tid % NX, ty = tid / NX;

  // window words 1 .. NW - 1 (word 0 stays 0)
  uint32_t acc[TM][TN][NP];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c)
#pragma unroll
      for (int w = 0; w < NP; ++w) acc[r][c][w] = 0u;
  for (int64_t k0 = 0; k0 < l; k0 += BK) {
#pragma unroll
    for (int idx = tid; idx < BM * BK; idx += NT) {
      const int r = idx / BK, c = idx % BK;
      const int64_t gi = i0 + r, gk = k0 + c;
      const bool ok = gi < m && gk < l;
      if constexpr (PRE) {
        stage_pre<L>(ok, Ax, gi * Ax.ld + gk, row_f[r], &sm.Aw[0][c][r], BK * (BM + 1), &sm.As[c][r]);
      } else {
        double x[L];
#pragma unroll
        for (int q = 0; q < L; ++q) x[q] = ok ? A.p[q][gi * A.ld + gk] : 0.0;
        stage<L>(x, row_f[r], &sm.Aw[0][c][r], BK * (BM + 1), &sm.As[c][r]);
      }
    }
#pragma unroll
    for (int idx = tid; idx < BK * BN; idx += NT) {
      const int r = idx / BN, c = idx % BN;
      const int64_t gk = k0 + r, gj = j0 + c;
      const bool ok = gk < l && gj < n;
      if constexpr (PRE) {
        stage_pre<L>(ok, Bx, gk * Bx.ld + gj, col_f[c], &sm.Bw[0][r][c], BK * BN, &sm.Bs[r][c]);
      } else {
        double x[L];
#pragma unroll
        for (int q = 0; q < L; ++q) x[q] = ok ? B.p[q][gk * B.ld + gj] : 0.0;
        stage<L>(x, col_f[c], &sm.Bw[0][r][c], BK * BN, &sm.Bs[r][c]);
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int kk = 0; kk < BK; ++kk) {
      uint32_t a[TM][4 * WV], b[TN][4 * WV], sa[TM], sb[TN];
#pragma unroll
      for (int r = 0; r < TM; ++r) {
#pragma unroll
        for (int v = 0; v < WV; ++v) {
          const uint4 q = sm.Aw[v][kk][ty + r * NY];
          a[r][4 * v] = q.x; a[r][4 * v + 1] = q.y; a[r][4 * v + 2] = q.z; a[r][4 * v + 3] = q.w;
        }
        sa[r] = (uint32_t)sm.As[kk][ty + r * NY];
      }
#pragma unroll
      for (int c = 0; c < TN; ++c) {
#pragma unroll
        for (int v = 0; v < WV; ++v) {
          const uint4 q = sm.Bw[v][kk][tx + c * NX];
          b[c][4 * v] = q.x; b[c][4 * v + 1] = q.y; b[c][4 * v + 2] = q.z; b[c][4 * v + 3] = q.w;
        }
        sb[c] = (uint32_t)sm.Bs[kk][tx + c * NX];
      }
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) {
          uint32_t q[W];
          fx::mul_top_hi<W>(*reinterpret_cast<const uint32_t(*)[W]>(a[r]),
                            *reinterpret_cast<const uint32_t(*)[W]>(b[c]), q);
          pre_add(acc[r][c], q, sa[r] ^ sb[c]);
        }
    }
    __syncthreads();
  }

  using N = num<L>;
  auto finish = [&](int64_t gi, int64_t gj, uint32_t(&w)[NW], int lsb) {
    typename N::T v = window_round<L, NW>(w, lsb);
    const int64_t off = gi * C.ld + gj;
    if (mode == MODE_ADD) v = N::add(N::load(C.p, off), v);
    else if (mode == MODE_SUB) v = N::add(N::load(C.p, off), N::neg(v));
    N::store(C.p, off, v);
  };
  uint32_t redo = 0u;  // outputs below fxpre<L>::keep window bits, bit r TN + c
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const int64_t gi = i0 + ty + r * NY, gj = j0 + tx + c * NX;
      if (gi < m && gj < n) {
        uint32_t w[NW];
        pre_window<NW>(acc[r][c], w);
        if (fx::acc_mag_below<NW>(w, fxpre<L>::keep)) {
          redo |= 1u << (r * TN + c);
          continue;
        }
        finish(gi, gj, w, row_f[ty + r * NY] + col_f[tx + c * NX] + P::LSB0);
      }
    }
  // Such outputs one at a time in the shifted form, each by the whole warp
  // (the lanes split k; a warp-uniform loop), when no accumulator is live
  // any more; the owning lane stores the result.
  const int lane = tid & 31;
  unsigned pend = __ballot_sync(0xffffffffu, redo != 0u);
  while (pend) {
    const int src = __ffs((int)pend) - 1;
    const uint32_t msrc = __shfl_sync(0xffffffffu, redo, src);
    const int t = __ffs((int)msrc) - 1;
    const int ts = (tid & ~31) + src, txs = ts % NX, tys = ts / NX;
    const int r = t / TN, c = t % TN;
    const int64_t gi = i0 + tys + r * NY, gj = j0 + txs + c * NX;
    fxacc<L> x = warp_shifted_one<L, PRE>(l, A, B, Ax, Bx, gi, gj, row_f[tys + r * NY] + col_f[txs + c * NX]);
    if (lane == src) {
      finish(gi, gj, x.w, x.lsb);
      redo &= ~(1u << t);
    }
    pend = __ballot_sync(0xffffffffu, redo != 0u);
  }
}

// One BM x BN tile of C at (i0, j0): C (mode) A B restricted to the tile,
// in the pre-shifted form (fx_pre.cuh). PRE: the operands come converted in
// Ax, Bx (A and B are then not read).
template <int L, bool PRE>
__device__ __forceinline__ void fx_tile(int64_t m, int64_t l, int64_t n, const mat& A, const mat& B,
                                        const mat& C, int mode, int64_t i0, int64_t j0, fx_smem<L>& sm,
                                        const fxop& Ax, const fxop& Bx) {
  fx_maxima<L, PRE>(m, l, n, A, B, i0, j0, sm, Ax, Bx);
  fx_pre<L, PRE>(m, l, n, A, B, C, mode, i0, j0, sm, Ax, Bx);
}

template <int L>
__global__ void __launch_bounds__(128, fxcfg<L>::MINB) block_fx_kernel(int64_t m, int64_t l, int64_t n, mat A, mat B,
                                                       mat C, int mode) {
  __shared__ fx_smem<L> sm;
  fx_tile<L, false>(m, l, n, A, B, C, mode, (int64_t)blockIdx.y * fxcfg<L>::BM,
                    (int64_t)blockIdx.x * fxcfg<L>::BN, sm, fxop{}, fxop{});
}

// The Block kernel on converted operands (A, B given only by their fxop):
// blockIdx.z picks one of G.count products of the same shape.
template <int L>
__global__ void __launch_bounds__(128, fxcfg<L>::MINB) block_fxc_kernel(int64_t m, int64_t l, int64_t n,
                                                                        fxc_group G, int mode) {
  __shared__ fx_smem<L> sm;
  const int z = blockIdx.z;
  fx_tile<L, true>(m, l, n, mat{}, mat{}, G.C[z], mode, (int64_t)blockIdx.y * fxcfg<L>::BM,
                   (int64_t)blockIdx.x * fxcfg<L>::BN, sm, G.A[z], G.B[z]);
}

// Element (r, c) of X converted (to_fixed) into the dense fxop layout with
// ld = cols: its word vectors at w[(r cols + c) WV ...], f at f[r cols + c].
template <int L>
__device__ __forceinline__ void convert_elem(const mat& X, int64_t r, int64_t c, int64_t cols, uint4* __restrict__ w,
                                             int* __restrict__ f) {
  constexpr int W = fxcfg<L>::W, WV = fx_smem<L>::WV;
  double x[L];
#pragma unroll
  for (int q = 0; q < L; ++q) x[q] = X.p[q][r * X.ld + c];
  uint32_t M[4 * WV];
  uint32_t(&Mw)[W] = *reinterpret_cast<uint32_t(*)[W]>(M);
  const int es = fx::to_fixed<L, W>(x, Mw);
#pragma unroll
  for (int t = W; t < 4 * WV; ++t) M[t] = 0u;
  const bool zero = (fx::dbits(x[0]) << 1) == 0u;
  const int64_t e = r * cols + c;
#pragma unroll
  for (int v = 0; v < WV; ++v) w[e * WV + v] = make_uint4(M[4 * v], M[4 * v + 1], M[4 * v + 2], M[4 * v + 3]);
  f[e] = zero ? FX_ZERO : es;
}

// Every element of up to FX_CONV_MAX operands converted once, each into the
// dense layout of fxop (ld = cols): blockIdx.z = operand, thread = column,
// CTA row = matrix row.
template <int L>
__global__ void __launch_bounds__(256) fx_convert_kernel(fx_conv_jobs J) {
  const fx_conv_job& jb = J.job[blockIdx.z];
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= jb.cols) return;
  for (int64_t r = blockIdx.y; r < jb.rows; r += gridDim.y) convert_elem<L>(jb.X, r, c, jb.cols, jb.w, jb.f);
}

// The same for a device-resident list of operands (batch plans): job t owns
// the tiles [tile0, tile0 + rows tiles_x), each one row by 256 columns;
// CTA b takes tiles b, b + gridDim.x, ... (no CTA waits on another).
template <int L>
__global__ void __launch_bounds__(256) grouped_convert_kernel(const fx_ctask* __restrict__ tasks, int ntasks,
                                                              int64_t total) {
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].tile0 <= t) lo = mid;
      else hi = mid - 1;
    }
    const fx_ctask& jb = tasks[lo];
    const int64_t local = t - jb.tile0;
    const int64_t r = local / jb.tiles_x;
    const int64_t c = (local - r * jb.tiles_x) * 256 + threadIdx.x;
    if (c < jb.cols) convert_elem<L>(jb.X, r, c, jb.cols, jb.w, jb.f);
  }
}

// Grouped persistent launch: every CTA takes the next tile of the task list
// (tiles numbered task by task, tasks sorted by decreasing l by the planner)
// from a global counter until none is left. No CTA waits on another.
template <int L>
__global__ void __launch_bounds__(128, fxcfg<L>::MINB - 1) grouped_fx_kernel(const gtask* __restrict__ tasks, int ntasks,
                                                         int64_t total, unsigned long long* counter) {
  __shared__ fx_smem<L> sm;
  __shared__ int64_t st;
  for (;;) {
    if (threadIdx.x == 0) st = (int64_t)atomicAdd(counter, 1ULL);
    __syncthreads();
    const int64_t t = st;
    __syncthreads();
    if (t >= total) break;
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].tile0 <= t) lo = mid;
      else hi = mid - 1;
    }
    const gtask g = tasks[lo];
    const int64_t local = t - g.tile0;
    const int64_t bi = local / g.tiles_n, bj = local % g.tiles_n;
    fx_tile<L, false>(g.m, g.l, g.n, g.A, g.B, g.C, g.mode, bi * fxcfg<L>::BM, bj * fxcfg<L>::BN, sm, fxop{},
                      fxop{});
    __syncthreads();
  }
}

// The grouped launch on converted operands (batch plans).
template <int L>
__global__ void __launch_bounds__(128, fxcfg<L>::MINB - 1) grouped_fxc_kernel(const gctask* __restrict__ tasks,
                                                                              int ntasks, int64_t total,
                                                                              unsigned long long* counter) {
  __shared__ fx_smem<L> sm;
  __shared__ int64_t st;
  for (;;) {
    if (threadIdx.x == 0) st = (int64_t)atomicAdd(counter, 1ULL);
    __syncthreads();
    const int64_t t = st;
    __syncthreads();
    if (t >= total) break;
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].tile0 <= t) lo = mid;
      else hi = mid - 1;
    }
    const gctask g = tasks[lo];
    const int64_t local = t - g.tile0;
    const int64_t bi = local / g.tiles_n, bj = local % g.tiles_n;
    fx_tile<L, true>(g.m, g.l, g.n, mat{}, mat{}, g.C, g.mode, bi * fxcfg<L>::BM, bj * fxcfg<L>::BN, sm, g.A, g.B);
    __syncthreads();
  }
}

// DD and QD tiles of one task list in one persistent launch (a batch plan
// with one leaf launch): every CTA takes the next tile from the global
// counter, whatever its task's limb count, and converts its tiles as they
// are staged (the bits of the converted-operand kernels). No CTA waits on
// another.
union fx_smem_any {
  fx_smem<2> d;
  fx_smem<4> q;
};

__global__ void __launch_bounds__(128, fxcfg<2>::MINB - 1) grouped_mixed_kernel(const gtask* __restrict__ tasks,
                                                                              int ntasks, int64_t total,
                                                                              unsigned long long* counter) {
  __shared__ fx_smem_any sm;
  __shared__ int64_t st;
  for (;;) {
    if (threadIdx.x == 0) st = (int64_t)atomicAdd(counter, 1ULL);
    __syncthreads();
    const int64_t t = st;
    __syncthreads();
    if (t >= total) break;
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].tile0 <= t) lo = mid;
      else hi = mid - 1;
    }
    const gtask g = tasks[lo];
    const int64_t local = t - g.tile0;
    const int64_t bi = local / g.tiles_n, bj = local % g.tiles_n;
    if (g.limbs == 2)
      fx_tile<2, false>(g.m, g.l, g.n, g.A, g.B, g.C, g.mode, bi * fxcfg<2>::BM, bj * fxcfg<2>::BN, sm.d, fxop{},
                        fxop{});
    else
      fx_tile<4, false>(g.m, g.l, g.n, g.A, g.B, g.C, g.mode, bi * fxcfg<4>::BM, bj * fxcfg<4>::BN, sm.q, fxop{},
                        fxop{});
    __syncthreads();
  }
}

void fx_tile_shape(int limbs, int* bm, int* bn) {
  *bm = limbs == 2 ? fxcfg<2>::BM : fxcfg<4>::BM;
  *bn = limbs == 2 ? fxcfg<2>::BN : fxcfg<4>::BN;
}

cudaError_t launch_grouped_fx(int limbs, const gtask* tasks, int ntasks, int64_t total_tiles,
                              unsigned long long* counter, double ops, cudaStream_t s) {
  if (ntasks == 0 || total_tiles == 0) return cudaSuccess;
  int dev = 0, sms = 0;  // the current device's (a cheap runtime query; no shared cache)
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  const int per_sm = (limbs == 2 ? fxcfg<2>::MINB : fxcfg<4>::MINB) - 1;  // resident CTAs per SM
  const int64_t grid = std::min<int64_t>(total_tiles, (int64_t)sms * per_sm);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  if (limbs == 2) grouped_fx_kernel<2><<<(unsigned)grid, 128, 0, s>>>(tasks, ntasks, total_tiles, counter);
  else grouped_fx_kernel<4><<<(unsigned)grid, 128, 0, s>>>(tasks, ntasks, total_tiles, counter);
  e = cudaGetLastError();
  if (ev) prof_end_launch(s, ev, PROF_BLOCK, ops, 0.0);
  return e;
}

cudaError_t launch_grouped_mixed(const gtask* tasks, int ntasks, int64_t total_tiles, unsigned long long* counter,
                                 double ops, cudaStream_t s) {
  if (ntasks == 0 || total_tiles == 0) return cudaSuccess;
  int dev = 0, sms = 0;  // the current device's (a cheap runtime query; no shared cache)
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  const int64_t grid = std::min<int64_t>(total_tiles, (int64_t)sms * (fxcfg<2>::MINB - 1));
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  grouped_mixed_kernel<<<(unsigned)grid, 128, 0, s>>>(tasks, ntasks, total_tiles, counter);
  e = cudaGetLastError();
  if (ev) prof_end_launch(s, ev, PROF_BLOCK, ops, 0.0);
  return e;
}

namespace {
inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }
inline size_t wv_of(int limbs) { return limbs == 2 ? fx_smem<2>::WV : fx_smem<4>::WV; }
}  // namespace

cudaError_t launch_grouped_fxc(int limbs, const gctask* tasks, int ntasks, int64_t total_tiles,
                               unsigned long long* counter, double ops, cudaStream_t s) {
  if (ntasks == 0 || total_tiles == 0) return cudaSuccess;
  int dev = 0, sms = 0;  // the current device's (a cheap runtime query; no shared cache)
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  const int per_sm = (limbs == 2 ? fxcfg<2>::MINB : fxcfg<4>::MINB) - 1;
  const int64_t grid = std::min<int64_t>(total_tiles, (int64_t)sms * per_sm);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  if (limbs == 2) grouped_fxc_kernel<2><<<(unsigned)grid, 128, 0, s>>>(tasks, ntasks, total_tiles, counter);
  else grouped_fxc_kernel<4><<<(unsigned)grid, 128, 0, s>>>(tasks, ntasks, total_tiles, counter);
  e = cudaGetLastError();
  if (ev) prof_end_launch(s, ev, PROF_BLOCK, ops, 0.0);
  return e;
}

int64_t convert_tiles(int64_t rows, int64_t cols) { return rows * ((cols + 255) / 256); }

cudaError_t launch_grouped_convert(int limbs, const fx_ctask* tasks, int ntasks, int64_t total_tiles, double elems,
                                   cudaStream_t s) {
  if (ntasks == 0 || total_tiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(total_tiles, 152 * 8);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  if (limbs == 2) grouped_convert_kernel<2><<<grid, 256, 0, s>>>(tasks, ntasks, total_tiles);
  else grouped_convert_kernel<4><<<grid, 256, 0, s>>>(tasks, ntasks, total_tiles);
  cudaError_t e = cudaGetLastError();
  if (ev) prof_end_launch(s, ev, PROF_CONVERT, elems, elems * (8.0 * limbs + 16.0 * wv_of(limbs) + 4.0));
  return e;
}

cudaError_t launch_block_fx(int limbs, int64_t m, int64_t l, int64_t n, mat A, mat B, mat C,
                            int mode, cudaStream_t s) {
  if (m == 0 || n == 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  if (limbs == 2) {
    dim3 grid((unsigned)((n + fxcfg<2>::BN - 1) / fxcfg<2>::BN), (unsigned)((m + fxcfg<2>::BM - 1) / fxcfg<2>::BM));
    block_fx_kernel<2><<<grid, 128, 0, s>>>(m, l, n, A, B, C, mode);
  } else {
    dim3 grid((unsigned)((n + fxcfg<4>::BN - 1) / fxcfg<4>::BN), (unsigned)((m + fxcfg<4>::BM - 1) / fxcfg<4>::BM));
    block_fx_kernel<4><<<grid, 128, 0, s>>>(m, l, n, A, B, C, mode);
  }
  cudaError_t e = cudaGetLastError();
  if (ev) {
    const double macs = (double)m * (double)l * (double)n;
    const double bytes = 8.0 * limbs * ((double)m * l + (double)l * n + (double)m * n * (mode == MODE_SET ? 1 : 2));
    prof_end_launch(s, ev, PROF_BLOCK, macs, bytes);
  }
  return e;
}

size_t fxop_bytes(int limbs, int64_t rows, int64_t cols) {
  const size_t elems = (size_t)rows * (size_t)cols;
  return al256(elems * 16 * wv_of(limbs)) + al256(elems * 4);
}

cudaError_t launch_fx_convert(int limbs, int count, const int64_t* rows, const int64_t* cols, const mat* X,
                              char* const* buf, fxop* out, cudaStream_t s) {
  if (count < 1 || count > FX_CONV_MAX) return cudaErrorInvalidValue;
  fx_conv_jobs J{};
  J.count = count;
  int64_t max_rows = 0, max_cols = 0;
  double elems = 0.0;
  for (int t = 0; t < count; ++t) {
    uint4* w = reinterpret_cast<uint4*>(buf[t]);
    int* f = reinterpret_cast<int*>(buf[t] + al256((size_t)rows[t] * (size_t)cols[t] * 16 * wv_of(limbs)));
    J.job[t] = fx_conv_job{rows[t], cols[t], X[t], w, f};
    out[t] = fxop{w, f, cols[t]};
    max_rows = std::max(max_rows, rows[t]);
    max_cols = std::max(max_cols, cols[t]);
    elems += (double)rows[t] * (double)cols[t];
  }
  if (max_rows == 0 || max_cols == 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  const dim3 grid((unsigned)((max_cols + 255) / 256), (unsigned)std::min<int64_t>(max_rows, 65535), (unsigned)count);
  if (limbs == 2) fx_convert_kernel<2><<<grid, 256, 0, s>>>(J);
  else fx_convert_kernel<4><<<grid, 256, 0, s>>>(J);
  cudaError_t e = cudaGetLastError();
  if (ev) prof_end_launch(s, ev, PROF_CONVERT, elems, elems * (8.0 * limbs + 16.0 * wv_of(limbs) + 4.0));
  return e;
}

bool block_fx_converts(int limbs, int64_t m, int64_t l, int64_t n) {
  (void)limbs;
  // each operand element is otherwise converted once per CTA row / column
  // of tiles: worth a separate pass once the grid is a few tiles each way
  return l >= 32 && m >= 64 && n >= 64;
}

size_t block_fx_scratch_bytes(int limbs, int64_t m, int64_t l, int64_t n) {
  return fxop_bytes(limbs, m, l) + fxop_bytes(limbs, l, n);
}

cudaError_t launch_block_fxc(int limbs, int64_t m, int64_t l, int64_t n, const fxop* Ax, const fxop* Bx,
                             const mat* C, int count, int mode, cudaStream_t s) {
  if (count < 1 || count > FXC_GROUP_MAX) return cudaErrorInvalidValue;
  if (m == 0 || n == 0) return cudaSuccess;
  nvtx_range nv("ddg.leaf x%d %lldx%lldx%lld", count, (long long)m, (long long)l, (long long)n);
  fxc_group G{};
  for (int t = 0; t < count; ++t) G.A[t] = Ax[t], G.B[t] = Bx[t], G.C[t] = C[t];
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  if (limbs == 2) {
    dim3 grid((unsigned)((n + fxcfg<2>::BN - 1) / fxcfg<2>::BN), (unsigned)((m + fxcfg<2>::BM - 1) / fxcfg<2>::BM),
              (unsigned)count);
    block_fxc_kernel<2><<<grid, 128, 0, s>>>(m, l, n, G, mode);
  } else {
    dim3 grid((unsigned)((n + fxcfg<4>::BN - 1) / fxcfg<4>::BN), (unsigned)((m + fxcfg<4>::BM - 1) / fxcfg<4>::BM),
              (unsigned)count);
    block_fxc_kernel<4><<<grid, 128, 0, s>>>(m, l, n, G, mode);
  }
  cudaError_t e = cudaGetLastError();
  if (ev) {
    const double macs = (double)count * (double)m * (double)l * (double)n;
    const double bytes = (double)count * 8.0 * limbs *
                         ((double)m * l + (double)l * n + (double)m * n * (mode == MODE_SET ? 1 : 2));
    prof_end_launch(s, ev, PROF_BLOCK, macs, bytes);
  }
  return e;
}

cudaError_t launch_block_fx_converted(int limbs, int64_t m, int64_t l, int64_t n, mat A, mat B, mat C, int mode,
                                      void* scratch, cudaStream_t s) {
  if (m == 0 || n == 0) return cudaSuccess;
  if (l == 0) return launch_block_fx(limbs, m, l, n, A, B, C, mode, s);
  char* buf[2] = {static_cast<char*>(scratch), static_cast<char*>(scratch) + fxop_bytes(limbs, m, l)};
  const int64_t rows[2] = {m, l}, cols[2] = {l, n};
  const mat X[2] = {A, B};
  fxop op[2];
  cudaError_t e = launch_fx_convert(limbs, 2, rows, cols, X, buf, op, s);
  if (e != cudaSuccess) return e;
  return launch_block_fxc(limbs, m, l, n, &op[0], &op[1], &C, 1, mode, s);
}

int block_fx_fp64_ops_per_mac(int limbs) { return limbs == 2 || limbs == 4 ? 0 : -1; }

}  // namespace ddg
