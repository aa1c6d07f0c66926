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
// Every sum is the accurate DD / QD addition of arith.cuh. On GB300 these
// passes are FP64-issue bound rather than HBM bound (20 FP64 instructions per
// DD sum against 48 bytes moved); they are O(n^2) against the O(n^3)
// products.
#include <algorithm>

#include "arith.cuh"
#include "kernels.cuh"

namespace ddg {


// One element (i, j) of a fused pass.
template <int L, int KIND>
__device__ __forceinline__ void pass_elem(const pass_args& a, int mode, int64_t i, int64_t j) {
  using N = num<L>;
  using T = typename N::T;
  auto ld = [&](int q) { return N::load(a.in[q].p, i * a.in[q].ld + j); };
  auto st = [&](int q, const T& v) { N::store(a.out[q].p, i * a.out[q].ld + j, v); };
  auto st_mode = [&](int q, const T& v) {
    const int64_t off = i * a.out[q].ld + j;
    if (mode == MODE_SET) N::store(a.out[q].p, off, v);
    else if (mode == MODE_ADD) N::store(a.out[q].p, off, N::add(N::load(a.out[q].p, off), v));
    else N::store(a.out[q].p, off, N::add(N::load(a.out[q].p, off), N::neg(v)));
  };
  auto add = [](const T& x, const T& y) { return N::add(x, y); };
  auto sub = [](const T& x, const T& y) { return N::add(x, N::neg(y)); };
  if constexpr (KIND == PASS_WINOGRAD_A) {
    const T x11 = ld(0), x12 = ld(1), x21 = ld(2), x22 = ld(3);
    const T s1 = add(x21, x22);
    const T s2 = sub(s1, x11);
    st(0, s1);
    st(1, s2);
    st(2, sub(x11, x21));
    st(3, sub(x12, s2));
  } else if constexpr (KIND == PASS_WINOGRAD_B) {
    const T x11 = ld(0), x12 = ld(1), x21 = ld(2), x22 = ld(3);
    const T t1 = sub(x12, x11);
    const T t2 = sub(x22, t1);
    st(0, t1);
    st(1, t2);
    st(2, sub(x22, x12));
    st(3, sub(t2, x21));
  } else if constexpr (KIND == PASS_WINOGRAD_C) {
    const T p1 = ld(0), p2 = ld(1), p3 = ld(2), p4 = ld(3), p5 = ld(4), p6 = ld(5), p7 = ld(6);
    const T u2 = add(p1, p6);
    const T u3 = add(u2, p7);
    const T u4 = add(u2, p5);
    st_mode(0, add(p1, p2));
    st_mode(1, add(u4, p3));
    st_mode(2, sub(u3, p4));
    st_mode(3, add(u3, p5));
  } else if constexpr (KIND == PASS_STRASSEN_A) {
    const T x11 = ld(0), x12 = ld(1), x21 = ld(2), x22 = ld(3);
    st(0, add(x11, x22));
    st(1, add(x21, x22));
    st(2, add(x11, x12));
    st(3, sub(x21, x11));
    st(4, sub(x12, x22));
  } else if constexpr (KIND == PASS_STRASSEN_B) {
    const T x11 = ld(0), x12 = ld(1), x21 = ld(2), x22 = ld(3);
    st(0, add(x11, x22));
    st(1, sub(x12, x22));
    st(2, sub(x21, x11));
    st(3, add(x11, x12));
    st(4, add(x21, x22));
  } else if constexpr (KIND == PASS_STRASSEN_C) {
    const T m1 = ld(0), m2 = ld(1), m3 = ld(2), m4 = ld(3), m5 = ld(4), m6 = ld(5), m7 = ld(6);
    st_mode(0, add(sub(add(m1, m4), m5), m7));
    st_mode(1, add(m3, m5));
    st_mode(2, add(m2, m4));
    st_mode(3, add(add(sub(m1, m2), m3), m6));
  } else {  // PASS_COMBINE
    st_mode(0, ld(0));
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
  const unsigned grid = (unsigned)std::min<int64_t>(total_tiles, 152 * 16);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (limbs == 2) launch_grouped_kind<2>(kind, grid, s, tasks, ntasks, total_tiles);
  else launch_grouped_kind<4>(kind, grid, s, tasks, ntasks, total_tiles);
  return cudaGetLastError();
}

cudaError_t launch_pass(int limbs, int kind, int64_t rows, int64_t cols, const mat* in, int nin,
                        const mat* out, int nout, int mode, cudaStream_t s) {
  if (rows == 0 || cols == 0) return cudaSuccess;
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
    prof_end_launch(s, ev, PROF_PASS, elems * nadd * add_fp64_ops(limbs), elems * moved * limbs * 8.0);
  }
  return e;
}

// FP64 instructions of one accurate sum: DD 20 (two TwoSums, two FastTwoSums,
// two adds); QD: the merge compares 7 and two 7-step TwoSum chains 84.
int add_fp64_ops(int limbs) { return limbs == 2 ? 20 : 91; }

}  // namespace ddg
