// Block product with exact fixed-point accumulation (Kouya 2015, Section 2,
// Block: C_ij = sum_k A_ik B_kj over tiles; the recursion's base case).
//
// Same tiling as block.cu (CTA tile of C, k-slabs of the limb planes staged
// in shared memory, a register micro-tile per thread), but the multiply-add
// moves the exact part of every product to the integer pipe (fx.cuh):
//   DD: a_hi b_hi exactly (integer significand product) into a 192-bit
//       window accumulator; the cross terms a_hi b_lo + a_lo b_hi by two FMAs
//       into an FP64 sum (they are 2^-53 below the leading product, so one
//       rounding per term is 2^-106 relative). 2 FP64 instructions per
//       multiply-add instead of 12 (TwoSum scheme) or 27 (DD multiply then
//       DD add).
//   QD: the six limb products of order <= 2 exactly into a 288-bit window;
//       the four order-3 products by FMA into an FP64 sum. 4 FP64
//       instructions per multiply-add instead of 113 / ~218.
// Before the k loop every CTA scans its row panel of A and column panel of B
// for the largest exponent per row / column; the window of c_ij is scaled so
// that sum_k |a_ik0 b_kj0| < 2^31 times the largest product fits below the
// sign bit, making the integer accumulation exact for l < 2^31.
// Error: truncation below the window (2^-159 resp. 2^-255 of the largest
// product of row i and column j, per term) plus one rounding per FP64 term
// and the final rounding to DD/QD.
#include <algorithm>

#include "arith.cuh"
#include "fx.cuh"
#include "kernels.cuh"

namespace ddg {

namespace {

template <int L> struct fxcfg;
template <> struct fxcfg<2> {
  static constexpr int BM = 16, BN = 32, BK = 16, TM = 2, TN = 2, NW = 6;
  static constexpr int POS0 = 53;     // pos of a product = (ea - fa) + (eb - fb) + POS0
  static constexpr int LSB0 = -2203;  // LSB exponent = fa + fb + LSB0
};
template <> struct fxcfg<4> {
  static constexpr int BM = 8, BN = 32, BK = 8, TM = 1, TN = 2, NW = 9;
  static constexpr int POS0 = 149;
  static constexpr int LSB0 = -2299;
};

__device__ __forceinline__ double scaled(uint64_t chunk, int k, uint32_t neg) {
  if (chunk == 0 || k < -2044) return 0.0;
  double v = fx::pow2_product(__ull2double_rn(chunk), k > 2046 ? 2046 : k);
  return neg ? -v : v;
}

}  // namespace

template <int L>
struct fx_smem {
  double As[L][fxcfg<L>::BK][fxcfg<L>::BM];
  double Bs[L][fxcfg<L>::BK][fxcfg<L>::BN];
  int row_f[fxcfg<L>::BM], col_f[fxcfg<L>::BN];
};

// One BM x BN tile of C at (i0, j0): C (mode) A B restricted to the tile.
template <int L>
__device__ __forceinline__ void fx_tile(int64_t m, int64_t l, int64_t n, const mat& A, const mat& B,
                                        const mat& C, int mode, int64_t i0, int64_t j0, fx_smem<L>& sm) {
  using P = fxcfg<L>;
  constexpr int BM = P::BM, BN = P::BN, BK = P::BK, TM = P::TM, TN = P::TN, NW = P::NW;
  constexpr int NX = BN / TN, NY = BM / TM, NT = NX * NY;
  static_assert(NT == 128, "block kernel assumes 128 threads");
  auto& As = sm.As;
  auto& Bs = sm.Bs;
  auto& row_f = sm.row_f;
  auto& col_f = sm.col_f;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tid % NX, ty = tid / NX;

  // ---- largest exponent field of the leading limb, per row of A / column of B
  for (int c = tid; c < BN; c += NT) col_f[c] = 1;
  for (int r = warp; r < BM; r += NT / 32) {
    int f = 1;
    const int64_t gi = i0 + r;
    if (gi < m)
      for (int64_t k = lane; k < l; k += 32) f = max(f, fx::expfield(A.p[0][gi * A.ld + k]));
    f = __reduce_max_sync(0xffffffffu, f);
    if (lane == 0) row_f[r] = f;
  }
  __syncthreads();
  {
    const int c = tid % BN;
    const int64_t gj = j0 + c;
    int f = 1;
    if (gj < n)
      for (int64_t k = tid / BN; k < l; k += NT / BN) f = max(f, fx::expfield(B.p[0][k * B.ld + gj]));
    atomicMax(&col_f[c], f);
  }
  __syncthreads();

  int base[TM][TN];
  uint32_t acc[TM][TN][NW];
  double ef[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      base[r][c] = P::POS0 - row_f[ty + r * NY] - col_f[tx + c * NX];
      ef[r][c] = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) acc[r][c][w] = 0u;
    }

  for (int64_t k0 = 0; k0 < l; k0 += BK) {
#pragma unroll
    for (int idx = tid; idx < BM * BK; idx += NT) {
      const int r = idx / BK, c = idx % BK;
      const int64_t gi = i0 + r, gk = k0 + c;
      const bool ok = gi < m && gk < l;
#pragma unroll
      for (int q = 0; q < L; ++q) As[q][c][r] = ok ? A.p[q][gi * A.ld + gk] : 0.0;
    }
#pragma unroll
    for (int idx = tid; idx < BK * BN; idx += NT) {
      const int r = idx / BN, c = idx % BN;
      const int64_t gk = k0 + r, gj = j0 + c;
      const bool ok = gk < l && gj < n;
#pragma unroll
      for (int q = 0; q < L; ++q) Bs[q][r][c] = ok ? B.p[q][gk * B.ld + gj] : 0.0;
    }
    __syncthreads();
#pragma unroll 1
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM][L], b[TN][L];
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int q = 0; q < L; ++q) a[r][q] = As[q][kk][ty + r * NY];
#pragma unroll
      for (int c = 0; c < TN; ++c)
#pragma unroll
        for (int q = 0; q < L; ++q) b[c][q] = Bs[q][kk][tx + c * NX];
      if constexpr (L == 2) {
        fx::unpacked ua[TM], ub[TN];
#pragma unroll
        for (int r = 0; r < TM; ++r) ua[r] = fx::unpack(a[r][0]);
#pragma unroll
        for (int c = 0; c < TN; ++c) ub[c] = fx::unpack(b[c][0]);
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
          for (int c = 0; c < TN; ++c) {
            uint32_t p[4];
            fx::mant_mul(ua[r], ub[c], p);
            fx::place<NW, 1>(acc[r][c], p, ua[r].e + ub[c].e + base[r][c], ua[r].s ^ ub[c].s);
            ef[r][c] = __fma_rn(a[r][0], b[c][1], ef[r][c]);
            ef[r][c] = __fma_rn(a[r][1], b[c][0], ef[r][c]);
          }
      } else {
        fx::unpacked ua[TM][3], ub[TN][3];
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
          for (int q = 0; q < 3; ++q) ua[r][q] = fx::unpack(a[r][q]);
#pragma unroll
        for (int c = 0; c < TN; ++c)
#pragma unroll
          for (int q = 0; q < 3; ++q) ub[c][q] = fx::unpack(b[c][q]);
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
          for (int c = 0; c < TN; ++c) {
            uint32_t p[4];
            const int bs = base[r][c];
#define DDG_PAIR(I, J, WF)                                                                  \
            fx::mant_mul(ua[r][I], ub[c][J], p);                                            \
            fx::place<NW, WF>(acc[r][c], p, ua[r][I].e + ub[c][J].e + bs, ua[r][I].s ^ ub[c][J].s);
            DDG_PAIR(0, 0, 4)
            DDG_PAIR(0, 1, 3)
            DDG_PAIR(1, 0, 3)
            DDG_PAIR(0, 2, 1)
            DDG_PAIR(1, 1, 1)
            DDG_PAIR(2, 0, 1)
#undef DDG_PAIR
            double e = ef[r][c];
            e = __fma_rn(a[r][0], b[c][3], e);
            e = __fma_rn(a[r][1], b[c][2], e);
            e = __fma_rn(a[r][2], b[c][1], e);
            e = __fma_rn(a[r][3], b[c][0], e);
            ef[r][c] = e;
          }
      }
    }
    __syncthreads();
  }

  using N = num<L>;
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const int64_t gi = i0 + ty + r * NY, gj = j0 + tx + c * NX;
      if (gi < m && gj < n) {
        const int lsb = row_f[ty + r * NY] + col_f[tx + c * NX] + P::LSB0;
        const uint32_t neg = fx::acc_abs<NW>(acc[r][c]);
        typename N::T v;
        if constexpr (L == 2) {
          uint64_t ch[2];
          int ex[2];
          double hi = 0.0, lo = 0.0;
          if (fx::acc_chunks<NW, 2>(acc[r][c], ch, ex)) {
            hi = scaled(ch[0], lsb + ex[0], neg);
            lo = scaled(ch[1], lsb + ex[1], neg);
          }
          double s, e1;
          two_sum(hi, ef[r][c], s, e1);
          two_sum(s, __dadd_rn(e1, lo), v.hi, v.lo);
        } else {
          uint64_t ch[4];
          int ex[4];
          double x[5] = {0.0, 0.0, 0.0, 0.0, ef[r][c]};
          if (fx::acc_chunks<NW, 4>(acc[r][c], ch, ex)) {
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = scaled(ch[q], lsb + ex[q], neg);
          }
          v = qd_renorm<5>(x);
        }
        const int64_t off = gi * C.ld + gj;
        if (mode == MODE_ADD) v = N::add(N::load(C.p, off), v);
        else if (mode == MODE_SUB) v = N::add(N::load(C.p, off), N::neg(v));
        N::store(C.p, off, v);
      }
    }
}

template <int L>
__global__ void __launch_bounds__(128) block_fx_kernel(int64_t m, int64_t l, int64_t n, mat A, mat B,
                                                       mat C, int mode) {
  __shared__ fx_smem<L> sm;
  fx_tile<L>(m, l, n, A, B, C, mode, (int64_t)blockIdx.y * fxcfg<L>::BM,
             (int64_t)blockIdx.x * fxcfg<L>::BN, sm);
}

// Grouped persistent launch: every CTA takes the next tile of the task list
// (tiles numbered task by task, tasks sorted by decreasing l by the planner)
// from a global counter until none is left. No CTA waits on another.
template <int L>
__global__ void __launch_bounds__(128) grouped_fx_kernel(const gtask* __restrict__ tasks, int ntasks,
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
    fx_tile<L>(g.m, g.l, g.n, g.A, g.B, g.C, g.mode, bi * fxcfg<L>::BM, bj * fxcfg<L>::BN, sm);
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
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  const int per_sm = limbs == 2 ? 5 : 3;  // resident CTAs per SM (register limited)
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
    prof_end_launch(s, ev, PROF_BLOCK, macs * block_fx_fp64_ops_per_mac(limbs), bytes);
  }
  return e;
}

int block_fx_fp64_ops_per_mac(int limbs) { return limbs == 2 ? 2 : 4; }

}  // namespace ddg
