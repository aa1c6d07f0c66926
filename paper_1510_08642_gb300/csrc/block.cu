// Block product (Kouya 2015, Section 2): C_ij = sum_{k=1..L} A_ik B_kj over
// tiles, also the base case at which the Strassen / Winograd recursion stops
// (Section 3, n_min).
//
// GB300 design. The FP64 pipe of a GB300 SM retires only 2 FP64 instructions
// per clock (measured: ~6.0e11 DFMA/s on 152 SMs, 1/64 of the FP32 rate), so
// a DD/QD product is bound by FP64 instruction issue, not by memory: a
// 32x64 DD tile with a 16-deep k-slab does 32768 multiply-adds (~393K FP64
// instructions) per 24 KB staged. The kernel therefore
//   * stages k-slabs of the hi/lo (or four QD) planes in shared memory with
//     coalesced loads (the bandwidth need is tiny; no TMA pipeline is needed
//     to keep the FP64 pipe fed),
//   * gives every thread a register micro-tile (4x4 DD, 2x2 QD) whose
//     independent accumulations hide FP64 latency with one warp per SMSP,
//   * and cuts FP64 instructions per multiply-add instead of the generic
//     "DD multiply then DD add" (27 FP64 ops for DD):
//       DD: c is kept as (S, E). The leading products p = a_hi b_hi are summed
//         into S error-free by TwoSum, TwoProd's error, both cross products
//         and TwoSum's error go into E in plain FP64. 12 FP64 ops per
//         multiply-add. Elementwise error <= (l + 4) u^2 sum_k |a_ik b_kj|
//         (u = 2^-53), far inside the 8 l 2^-104 normwise bound.
//       QD: c is kept as four levels S0..S3 by order of magnitude (in units
//         of the limb spacing u). Products of order 0..2 are TwoProd'd, and
//         the terms of levels 0..2 are added by TwoSum with their errors
//         pushed one level down; level 3 is a plain sum. 113 FP64 ops per
//         multiply-add instead of ~220 for the pinned QD multiply-then-add.
//   The result is renormalised once per output entry.
#include "arith.cuh"
#include "kernels.cuh"

namespace ddg {

namespace {

struct acc_dd {
  double S, E;
  __device__ __forceinline__ void init() { S = 0.0; E = 0.0; }
  __device__ __forceinline__ void mac(const double* a, const double* b) {
    const double ah = a[0], al = a[1], bh = b[0], bl = b[1];
    double p = __dmul_rn(ah, bh);
    double e = __fma_rn(ah, bh, -p);
    E = __fma_rn(ah, bl, E);
    E = __fma_rn(al, bh, E);
    double s = __dadd_rn(S, p);
    double bv = __dsub_rn(s, S);
    double av = __dsub_rn(s, bv);
    double t = __dadd_rn(__dsub_rn(S, av), __dsub_rn(p, bv));
    S = s;
    E = __dadd_rn(E, __dadd_rn(t, e));
  }
  __device__ __forceinline__ dd_t result() const {
    dd_t r;
    two_sum(S, E, r.hi, r.lo);
    return r;
  }
};
constexpr int kOpsDD = 12;

struct acc_qd {
  double S0, S1, S2, S3;
  __device__ __forceinline__ void init() { S0 = S1 = S2 = S3 = 0.0; }
  __device__ __forceinline__ void mac(const double* a, const double* b) {
    double p00, q00, p01, q01, p10, q10, p02, q02, p11, q11, p20, q20;
    two_prod(a[0], b[0], p00, q00);
    two_prod(a[0], b[1], p01, q01);
    two_prod(a[1], b[0], p10, q10);
    two_prod(a[0], b[2], p02, q02);
    two_prod(a[1], b[1], p11, q11);
    two_prod(a[2], b[0], p20, q20);
    double o3 = __dmul_rn(a[0], b[3]);
    o3 = __fma_rn(a[1], b[2], o3);
    o3 = __fma_rn(a[2], b[1], o3);
    o3 = __fma_rn(a[3], b[0], o3);
    double t0, u1, u2, u3, u4, v[9];
    two_sum(S0, p00, S0, t0);
    two_sum(S1, p01, S1, u1);
    two_sum(S1, p10, S1, u2);
    two_sum(S1, q00, S1, u3);
    two_sum(S1, t0, S1, u4);
    two_sum(S2, p02, S2, v[0]);
    two_sum(S2, p11, S2, v[1]);
    two_sum(S2, p20, S2, v[2]);
    two_sum(S2, q01, S2, v[3]);
    two_sum(S2, q10, S2, v[4]);
    two_sum(S2, u1, S2, v[5]);
    two_sum(S2, u2, S2, v[6]);
    two_sum(S2, u3, S2, v[7]);
    two_sum(S2, u4, S2, v[8]);
    double w = __dadd_rn(o3, q02);
    w = __dadd_rn(w, q11);
    w = __dadd_rn(w, q20);
#pragma unroll
    for (int i = 0; i < 9; ++i) w = __dadd_rn(w, v[i]);
    S3 = __dadd_rn(S3, w);
  }
  __device__ __forceinline__ qd_t result() const {
    const double x[4] = {S0, S1, S2, S3};
    return qd_renorm<4>(x);
  }
};
constexpr int kOpsQD = 12 + 4 + 6 * 14 + 13;  // 113

template <int L> struct blk;
template <> struct blk<2> {
  static constexpr int BM = 32, BN = 64, BK = 16, TM = 4, TN = 4;
  using acc = acc_dd;
};
template <> struct blk<4> {
  static constexpr int BM = 16, BN = 32, BK = 8, TM = 2, TN = 2;
  using acc = acc_qd;
};

}  // namespace

template <int L>
__global__ void __launch_bounds__(128) block_kernel(int64_t m, int64_t l, int64_t n, mat A, mat B,
                                                    mat C, int mode) {
  using P = blk<L>;
  constexpr int BM = P::BM, BN = P::BN, BK = P::BK, TM = P::TM, TN = P::TN;
  constexpr int NX = BN / TN, NY = BM / TM, NT = NX * NY;
  static_assert(NT == 128, "block kernel assumes 128 threads");
  __shared__ double As[L][BK][BM];
  __shared__ double Bs[L][BK][BN];

  const int tid = threadIdx.x;
  const int tx = tid % NX, ty = tid / NX;
  const int64_t i0 = (int64_t)blockIdx.y * BM;
  const int64_t j0 = (int64_t)blockIdx.x * BN;

  typename P::acc acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c].init();

  for (int64_t k0 = 0; k0 < l; k0 += BK) {
    // A tile BM x BK, stored k-major; B tile BK x BN.
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
#pragma unroll 2
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
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c].mac(a[r], b[c]);
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
        typename N::T v = acc[r][c].result();
        const int64_t off = gi * C.ld + gj;
        if (mode == MODE_ADD) v = N::add(N::load(C.p, off), v);
        else if (mode == MODE_SUB) v = N::add(N::load(C.p, off), N::neg(v));
        N::store(C.p, off, v);
      }
    }
}

cudaError_t launch_block(int limbs, int64_t m, int64_t l, int64_t n, mat A, mat B, mat C,
                         int mode, cudaStream_t s) {
  if (m == 0 || n == 0) return cudaSuccess;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  if (limbs == 2) {
    dim3 grid((unsigned)((n + blk<2>::BN - 1) / blk<2>::BN), (unsigned)((m + blk<2>::BM - 1) / blk<2>::BM));
    block_kernel<2><<<grid, 128, 0, s>>>(m, l, n, A, B, C, mode);
  } else {
    dim3 grid((unsigned)((n + blk<4>::BN - 1) / blk<4>::BN), (unsigned)((m + blk<4>::BM - 1) / blk<4>::BM));
    block_kernel<4><<<grid, 128, 0, s>>>(m, l, n, A, B, C, mode);
  }
  cudaError_t e = cudaGetLastError();
  if (ev) {
    const double macs = (double)m * (double)l * (double)n;
    const double bytes = 8.0 * limbs * ((double)m * l + (double)l * n + (double)m * n * (mode == MODE_SET ? 1 : 2));
    prof_end_launch(s, ev, PROF_BLOCK, macs, bytes);
  }
  return e;
}

int block_fp64_ops_per_mac(int limbs) { return limbs == 2 ? kOpsDD : kOpsQD; }

}  // namespace ddg
