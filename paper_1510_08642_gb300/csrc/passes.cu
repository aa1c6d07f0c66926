// Fused quadrant add/sub passes of one Strassen or Winograd recursion level
// (Kouya 2015, Section 2: the Strassen algorithm [Strassen 1969] and
// Winograd's variant, whose sub-products are computed in parallel in
// Figs. 1-2; the figures' formulas are the standard ones restated below).
//
// Each pass reads every input quadrant once and writes every output once,
// with all sums of one level fused into a single kernel; the chained
// Winograd sums (S2 = S1 - A11, S4 = A12 - S2, ...) stay in registers.
// Winograd (7 products, 15 additions):
//   S1 = A21 + A22, S2 = S1 - A11, S3 = A11 - A21, S4 = A12 - S2
//   T1 = B12 - B11, T2 = B22 - T1, T3 = B22 - B12, T4 = T2 - B21
//   P1 = A11 B11, P2 = A12 B21, P3 = S4 B22, P4 = A22 T4,
//   P5 = S1 T1,  P6 = S2 T2,  P7 = S3 T3
//   C11 = P1 + P2, U2 = P1 + P6, U3 = U2 + P7, U4 = U2 + P5,
//   C12 = U4 + P3, C21 = U3 - P4, C22 = U3 + P5
// Strassen (7 products, 18 additions):
//   M1 = (A11 + A22)(B11 + B22), M2 = (A21 + A22) B11, M3 = A11 (B12 - B22),
//   M4 = A22 (B21 - B11), M5 = (A11 + A12) B22, M6 = (A21 - A11)(B11 + B12),
//   M7 = (A12 - A22)(B21 + B22)
//   C11 = M1 + M4 - M5 + M7, C12 = M3 + M5, C21 = M2 + M4,
//   C22 = M1 - M2 + M3 + M6
// Every sum is exact in fixed point on the integer pipe (one rounding per
// output): the accurate DD / QD additions of arith.cuh cost 20 / 91 FP64
// instructions each, which made these O(n^2) passes FP64-issue bound on
// GB300 rather than HBM bound.
#include <algorithm>

#include "arith.cuh"
#include "fx.cuh"
#include "kernels.cuh"

namespace ddg {


// Fixed-point width per limb count: NW words, the largest operand's leading
// significand at bit TOP (headroom for sums of up to 8 operands below the
// sign bit).
template <int L> struct pfx;
template <> struct pfx<2> { static constexpr int NW = 5, TOP = 32 * 5 - 58; };
template <> struct pfx<4> { static constexpr int NW = 9, TOP = 32 * 9 - 58; };

// One element (i, j) of a fused pass. The operands (and C for the update
// modes) are placed at one common scale as exact integers on the integer
// pipe (fx::add_at), every sum of the pass is an exact multiword addition,
// and each output is rounded back once (fx::from_fixed). Error per output: one rounding to DD / QD (a DD output is
// the DD nearest the exact sum, up to 2^-(top + 52) of the largest operand).
template <int L, int KIND>
__device__ __forceinline__ void pass_elem(const pass_args& a, int mode, int64_t i, int64_t j) {
  using N = num<L>;
  using T = typename N::T;
  constexpr int NW = pfx<L>::NW, TOP = pfx<L>::TOP;
  using V = uint32_t[NW];
  constexpr int NIN = (KIND == PASS_WINOGRAD_C || KIND == PASS_STRASSEN_C) ? 7 : (KIND == PASS_COMBINE ? 1 : 4);
  constexpr int NOUT = (KIND == PASS_STRASSEN_A || KIND == PASS_STRASSEN_B) ? 5 : (KIND == PASS_COMBINE ? 1 : 4);
  constexpr bool UPD = KIND == PASS_WINOGRAD_C || KIND == PASS_STRASSEN_C || KIND == PASS_COMBINE;
  const bool upd = UPD && mode != MODE_SET;
  double x[NIN][L], c[NOUT][L];
#pragma unroll
  for (int q = 0; q < NIN; ++q) {
    const int64_t off = i * a.in[q].ld + j;
#pragma unroll
    for (int t = 0; t < L; ++t) x[q][t] = a.in[q].p[t][off];
  }
  int emax = 1;
#pragma unroll
  for (int q = 0; q < NIN; ++q) emax = max(emax, fx::expfield(x[q][0]));
  if (upd) {
#pragma unroll
    for (int q = 0; q < NOUT; ++q) {
      const int64_t off = i * a.out[q].ld + j;
#pragma unroll
      for (int t = 0; t < L; ++t) c[q][t] = a.out[q].p[t][off];
      emax = max(emax, fx::expfield(c[q][0]));
    }
  }
  V X[NIN];
#pragma unroll
  for (int q = 0; q < NIN; ++q) {
#pragma unroll
    for (int w = 0; w < NW; ++w) X[q][w] = 0u;
    fx::add_at<L, NW>(X[q], x[q], emax, TOP, 0u);
  }
  const int lsb = emax - 1075 - TOP;
  auto put = [&](int q, V& r) {
    if (UPD && upd) {
      if (mode == MODE_SUB) {  // r := -r, then + C: C - sum
        uint32_t cy = 1u;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const uint64_t v = (uint64_t)(~r[w]) + cy;
          r[w] = (uint32_t)v;
          cy = (uint32_t)(v >> 32);
        }
      }
      fx::add_at<L, NW>(r, c[q], emax, TOP, 0u);
    }
    double o[L];
    fx::from_fixed<L, NW>(r, lsb, o);  // canonical DD / QD
    T v;
    if constexpr (L == 2) v = dd_t{o[0], o[1]};
    else v = qd_t{{o[0], o[1], o[2], o[3]}};
    N::store(a.out[q].p, i * a.out[q].ld + j, v);
  };
  V r0, r1, r2;
  if constexpr (KIND == PASS_WINOGRAD_A) {
    // x: A11, A12, A21, A22 -> S1, S2, S3, S4
    fx::vadd<NW>(r0, X[2], X[3], false);  // S1 = A21 + A22
    fx::vadd<NW>(r1, r0, X[0], true);     // S2 = S1 - A11
    fx::vadd<NW>(r2, X[1], r1, true);     // S4 = A12 - S2
    put(0, r0);
    put(1, r1);
    put(3, r2);
    fx::vadd<NW>(r0, X[0], X[2], true);   // S3 = A11 - A21
    put(2, r0);
  } else if constexpr (KIND == PASS_WINOGRAD_B) {
    // x: B11, B12, B21, B22 -> T1, T2, T3, T4
    fx::vadd<NW>(r0, X[1], X[0], true);   // T1 = B12 - B11
    fx::vadd<NW>(r1, X[3], r0, true);     // T2 = B22 - T1
    fx::vadd<NW>(r2, r1, X[2], true);     // T4 = T2 - B21
    put(0, r0);
    put(1, r1);
    put(3, r2);
    fx::vadd<NW>(r0, X[3], X[1], true);   // T3 = B22 - B12
    put(2, r0);
  } else if constexpr (KIND == PASS_WINOGRAD_C) {
    // x: P1 .. P7 -> C11, C12, C21, C22 (mode)
    V u2, u3;
    fx::vadd<NW>(u2, X[0], X[5], false);  // U2 = P1 + P6
    fx::vadd<NW>(u3, u2, X[6], false);    // U3 = U2 + P7
    fx::vadd<NW>(r0, X[0], X[1], false);  // C11 = P1 + P2
    put(0, r0);
    fx::vadd<NW>(r0, u2, X[4], false);    // U4 = U2 + P5
    fx::vadd<NW>(r1, r0, X[2], false);    // C12 = U4 + P3
    put(1, r1);
    fx::vadd<NW>(r0, u3, X[3], true);     // C21 = U3 - P4
    put(2, r0);
    fx::vadd<NW>(r0, u3, X[4], false);    // C22 = U3 + P5
    put(3, r0);
  } else if constexpr (KIND == PASS_STRASSEN_A) {
    // x: A11, A12, A21, A22
    fx::vadd<NW>(r0, X[0], X[3], false); put(0, r0);  // A11 + A22
    fx::vadd<NW>(r0, X[2], X[3], false); put(1, r0);  // A21 + A22
    fx::vadd<NW>(r0, X[0], X[1], false); put(2, r0);  // A11 + A12
    fx::vadd<NW>(r0, X[2], X[0], true);  put(3, r0);  // A21 - A11
    fx::vadd<NW>(r0, X[1], X[3], true);  put(4, r0);  // A12 - A22
  } else if constexpr (KIND == PASS_STRASSEN_B) {
    // x: B11, B12, B21, B22
    fx::vadd<NW>(r0, X[0], X[3], false); put(0, r0);  // B11 + B22
    fx::vadd<NW>(r0, X[1], X[3], true);  put(1, r0);  // B12 - B22
    fx::vadd<NW>(r0, X[2], X[0], true);  put(2, r0);  // B21 - B11
    fx::vadd<NW>(r0, X[0], X[1], false); put(3, r0);  // B11 + B12
    fx::vadd<NW>(r0, X[2], X[3], false); put(4, r0);  // B21 + B22
  } else if constexpr (KIND == PASS_STRASSEN_C) {
    // x: M1 .. M7
    fx::vadd<NW>(r0, X[0], X[3], false);  // M1 + M4
    fx::vadd<NW>(r1, r0, X[4], true);     // - M5
    fx::vadd<NW>(r0, r1, X[6], false);    // + M7
    put(0, r0);
    fx::vadd<NW>(r0, X[2], X[4], false); put(1, r0);  // M3 + M5
    fx::vadd<NW>(r0, X[1], X[3], false); put(2, r0);  // M2 + M4
    fx::vadd<NW>(r0, X[0], X[1], true);   // M1 - M2
    fx::vadd<NW>(r1, r0, X[2], false);    // + M3
    fx::vadd<NW>(r0, r1, X[5], false);    // + M6
    put(3, r0);
  } else {  // PASS_COMBINE
#pragma unroll
    for (int w = 0; w < NW; ++w) r0[w] = X[0][w];
    put(0, r0);
  }
}

template <int L, int KIND>
__global__ void __launch_bounds__(256) pass_kernel(int64_t rows, int64_t cols, pass_args a, int mode) {
  const int64_t j = (int64_t)blockIdx.x * 32 + threadIdx.x;
  if (j >= cols) return;
  for (int64_t i = (int64_t)blockIdx.y * 8 + threadIdx.y; i < rows; i += (int64_t)gridDim.y * 8)
    pass_elem<L, KIND>(a, mode, i, j);
}

// Grouped pass launch: tiles of 8 x 32 elements of every task, numbered task
// by task; CTAs stride over the tiles.
template <int L, int KIND>
__global__ void __launch_bounds__(256) grouped_pass_kernel(const ptask* __restrict__ tasks, int ntasks,
                                                           int64_t total) {
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].tile0 <= t) lo = mid;
      else hi = mid - 1;
    }
    const ptask& g = tasks[lo];
    const int64_t local = t - g.tile0;
    const int64_t i = (local / g.tiles_x) * 8 + threadIdx.y;
    const int64_t j = (local % g.tiles_x) * 32 + threadIdx.x;
    if (i < g.rows && j < g.cols) pass_elem<L, KIND>(g.a, g.mode, i, j);
  }
}

template <int L>
static void launch_kind(int kind, dim3 g, dim3 b, cudaStream_t s, int64_t rows, int64_t cols,
                        const pass_args& a, int mode) {
  switch (kind) {
    case PASS_WINOGRAD_A: pass_kernel<L, PASS_WINOGRAD_A><<<g, b, 0, s>>>(rows, cols, a, mode); break;
    case PASS_WINOGRAD_B: pass_kernel<L, PASS_WINOGRAD_B><<<g, b, 0, s>>>(rows, cols, a, mode); break;
    case PASS_WINOGRAD_C: pass_kernel<L, PASS_WINOGRAD_C><<<g, b, 0, s>>>(rows, cols, a, mode); break;
    case PASS_STRASSEN_A: pass_kernel<L, PASS_STRASSEN_A><<<g, b, 0, s>>>(rows, cols, a, mode); break;
    case PASS_STRASSEN_B: pass_kernel<L, PASS_STRASSEN_B><<<g, b, 0, s>>>(rows, cols, a, mode); break;
    case PASS_STRASSEN_C: pass_kernel<L, PASS_STRASSEN_C><<<g, b, 0, s>>>(rows, cols, a, mode); break;
    default: pass_kernel<L, PASS_COMBINE><<<g, b, 0, s>>>(rows, cols, a, mode); break;
  }
}

template <int L>
static void launch_grouped_kind(int kind, unsigned grid, cudaStream_t s, const ptask* t, int nt, int64_t total) {
  dim3 b(32, 8);
  switch (kind) {
    case PASS_WINOGRAD_A: grouped_pass_kernel<L, PASS_WINOGRAD_A><<<grid, b, 0, s>>>(t, nt, total); break;
    case PASS_WINOGRAD_B: grouped_pass_kernel<L, PASS_WINOGRAD_B><<<grid, b, 0, s>>>(t, nt, total); break;
    case PASS_WINOGRAD_C: grouped_pass_kernel<L, PASS_WINOGRAD_C><<<grid, b, 0, s>>>(t, nt, total); break;
    case PASS_STRASSEN_A: grouped_pass_kernel<L, PASS_STRASSEN_A><<<grid, b, 0, s>>>(t, nt, total); break;
    case PASS_STRASSEN_B: grouped_pass_kernel<L, PASS_STRASSEN_B><<<grid, b, 0, s>>>(t, nt, total); break;
    case PASS_STRASSEN_C: grouped_pass_kernel<L, PASS_STRASSEN_C><<<grid, b, 0, s>>>(t, nt, total); break;
    default: grouped_pass_kernel<L, PASS_COMBINE><<<grid, b, 0, s>>>(t, nt, total); break;
  }
}

cudaError_t launch_grouped_pass(int limbs, int kind, const ptask* tasks, int ntasks, int64_t total_tiles,
                                cudaStream_t s) {
  if (ntasks == 0 || total_tiles == 0) return cudaSuccess;
  nvtx_range nv("ddg.grouped pass kind %d", kind);
  const unsigned grid = (unsigned)std::min<int64_t>(total_tiles, 152 * 16);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (limbs == 2) launch_grouped_kind<2>(kind, grid, s, tasks, ntasks, total_tiles);
  else launch_grouped_kind<4>(kind, grid, s, tasks, ntasks, total_tiles);
  return cudaGetLastError();
}

cudaError_t launch_pass(int limbs, int kind, int64_t rows, int64_t cols, const mat* in, int nin,
                        const mat* out, int nout, int mode, cudaStream_t s) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  nvtx_range nv("ddg.pass kind %d %lldx%lld", kind, (long long)rows, (long long)cols);
  pass_args a{};
  for (int q = 0; q < nin && q < 7; ++q) a.in[q] = in[q];
  for (int q = 0; q < nout && q < 5; ++q) a.out[q] = out[q];
  dim3 block(32, 8);
  int64_t gy = (rows + 7) / 8;
  if (gy > 65535) gy = 65535;
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)gy);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  if (limbs == 2) launch_kind<2>(kind, grid, block, s, rows, cols, a, mode);
  else launch_kind<4>(kind, grid, block, s, rows, cols, a, mode);
  cudaError_t e = cudaGetLastError();
  if (ev) {
    // sums per element and elements moved per element, by pass kind
    static const int adds[7] = {4, 4, 7, 5, 5, 8, 0};
    const bool upd = mode != MODE_SET && (kind == PASS_WINOGRAD_C || kind == PASS_STRASSEN_C || kind == PASS_COMBINE);
    const int nadd = adds[kind] + (upd ? nout : 0);
    const double elems = (double)rows * (double)cols;
    const double moved = (double)(nin + nout + (upd ? nout : 0));
    prof_end_launch(s, ev, PROF_PASS, elems * nadd, elems * moved * limbs * 8.0);
  }
  return e;
}

// FP64 instructions of one accurate DD / QD sum of arith.cuh (DD 20: two
// TwoSums, two FastTwoSums, two adds; QD: the merge compares 7 and two
// 7-step TwoSum chains 84), which the fixed-point passes replace.
int add_fp64_ops(int limbs) { return limbs == 2 ? 20 : 91; }

}  // namespace ddg
