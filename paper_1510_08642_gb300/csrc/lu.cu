// DD and QD LU decomposition and solve (Kouya 2015, Section 4): the blocked
// right-looking LU whose trailing update A22 := A22 - L21 U12 (step 3, the
// underlined product) is a DD / QD matrix product, here the library's
// product with mode SUB and the caller's algorithm (Winograd by default),
// and the solution of A x = b (Eq. 2) by forward and back substitution. One
// code path for both precisions (template on the limb count).
//
// Steps per block column of width K (the paper's K = alpha n_min):
//   1. panel: for each column j of the block, pivot search (the first row of
//      largest |a_ij| compared as DD; skipped in the paper's no-pivot mode),
//      swap of the two whole rows, DD quotients l_ij = a_ij (1 / a_jj) and
//      the rank-1 update of the next columns: one grid launch per column
//      (quotients, update, partial arg-maxes of the next column), whose last
//      CTA to finish chooses and swaps the next pivot (an atomic counter; no
//      CTA waits for another). Wide block columns are factored
//      recursively in halves (left half, triangular solve and Block update of
//      the right half, right half), so the rank-1 updates in pinned DD
//      arithmetic stay within 16 columns.
//   2. U12 := L11^-1 A12 by a recursive triangular solve whose off-diagonal
//      updates are Block products (base case: 32-row triangles, one warp per
//      right-hand column: a GB300 SM issues FP64 slowly, so the chain of DD
//      operations per warp is kept short).
//   3. A22 := A22 - L21 U12 through the matrix product.
// The loop runs while columns remain; the last block has min(K, remaining)
// columns (the paper's garbled loop end, read as "until no columns remain").
#include <algorithm>
#include <cstdlib>
#include <functional>
#include <map>
#include <mutex>
#include <string>

#include <cooperative_groups.h>

#include "arith.cuh"
#include "fx.cuh"
#include "fxscalar.cuh"
#include "kernels.cuh"

namespace ddg {

namespace cg = cooperative_groups;

namespace {

constexpr int RB = 8;        // rows per CTA in the column kernels (many CTAs: the
                             // rank-1 updates of a column spread over the SMs)
constexpr int TB = 32;       // triangle size of the substitution base case (one warp)
constexpr int KMAX = 512;    // widest block column
constexpr int PANEL_BASE = 16;  // widest panel factored column by column
// DD column steps (quotients and rank-1 updates of a panel): the exact
// fixed-point form on the integer pipe, as for QD (false), or the DD
// sequences on the FP64 pipe (true). The FP64 pipe retires 2 instructions
// per clock per SM, so with the panel's rows spread over all SMs in one
// launch the integer form is the faster one.
constexpr bool kDDColumnFP64 = false;

// Pivot candidates compare by integer keys of |x| (leading limb magnitude,
// then the second limb with the leading limb's sign): no FP64 compare
// instructions on the pivot search's critical path.
struct partial_t {
  unsigned long long kh, kl;
  int64_t idx;
};

// Per-call device state of the column steps (large enough for a QD value).
struct col_state {
  unsigned int counter;  // CTAs finished in the current launch
  unsigned int pad;
  double rinv[4];        // 1 / pivot of the column being eliminated (0 if zero)
};

template <int L>
__device__ __forceinline__ typename num<L>::T ldA(const mat& A, int64_t i, int64_t j) {
  return num<L>::load(A.p, i * A.ld + j);
}
template <int L>
__device__ __forceinline__ void stA(const mat& A, int64_t i, int64_t j, const typename num<L>::T& v) {
  num<L>::store(A.p, i * A.ld + j, v);
}

__device__ __forceinline__ unsigned long long dkey(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);  // order of doubles
}

template <int L>
__device__ __forceinline__ partial_t cand(const typename num<L>::T& v, int64_t i) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(num<L>::lead(v));
  const double s2 = num<L>::second(v);
  return partial_t{b & 0x7FFFFFFFFFFFFFFFull, dkey((b >> 63) ? -s2 : s2), i};
}

__device__ __forceinline__ partial_t none() { return partial_t{0ull, 0ull, INT64_MAX}; }

// Is a a better pivot than b: larger |x|, ties to the smaller row index.
__device__ __forceinline__ bool better(const partial_t& a, const partial_t& b) {
  if (a.kh != b.kh) return a.kh > b.kh;
  if (a.kl != b.kl) return a.kl > b.kl;
  return a.idx < b.idx;
}

__device__ __forceinline__ void warp_best(partial_t& v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    partial_t w{__shfl_xor_sync(0xffffffffu, v.kh, o), __shfl_xor_sync(0xffffffffu, v.kl, o),
                __shfl_xor_sync(0xffffffffu, v.idx, o)};
    if (better(w, v)) v = w;
  }
}

template <int L>
__device__ __forceinline__ bool is_zero(const typename num<L>::T& v) {
  const double* x = reinterpret_cast<const double*>(&v);
  bool z = true;
#pragma unroll
  for (int q = 0; q < L; ++q)
    z = z && (((unsigned long long)__double_as_longlong(x[q]) & 0x7FFFFFFFFFFFFFFFull) == 0ull);
  return z;
}

template <int L>
__device__ __forceinline__ typename num<L>::T get_rinv(const col_state* cs) {
  typename num<L>::T v;
  double* x = reinterpret_cast<double*>(&v);
#pragma unroll
  for (int q = 0; q < L; ++q) x[q] = cs->rinv[q];
  return v;
}

// The window rounded to an L-limb expansion and stored.
template <int L>
__device__ __forceinline__ void window_store(uint32_t (&acc)[tfx<L>::NW], int A, const mat& X, int64_t i, int64_t c) {
  double o[L];
  fx::from_fixed<L, tfx<L>::NW>(acc, A - 1075 - tfx<L>::TOPA, o);
  typename num<L>::T v;
  if constexpr (L == 2) v = dd_t{o[0], o[1]};
  else v = qd_t{{o[0], o[1], o[2], o[3]}};
  stA<L>(X, i, c, v);
}

// Triangle entries staged in fixed-point form, lane-contiguous: Tw[k][w][i]
// is word w of entry (i, k), Te[k][i] its exponent field | sign << 16.
template <int L>
struct tri_smem {
  uint32_t Tw[TB][tfx<L>::W][TB];
  int Te[TB][TB];
};

template <int L>
__device__ __forceinline__ void stage_triangle(tri_smem<L>& sm, const mat& T, int64_t m, bool upper) {
  constexpr int W = tfx<L>::W;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int i = e / TB, k = e % TB;
    const bool use = i < m && k < m && (upper ? k > i : k < i);
    double x[L];
#pragma unroll
    for (int q = 0; q < L; ++q) x[q] = use ? T.p[q][i * T.ld + k] : 0.0;
    uint32_t M[W];
    const int es = fx::to_fixed<L, W>(x, M);
#pragma unroll
    for (int w = 0; w < W; ++w) sm.Tw[k][w][i] = M[w];
    sm.Te[k][i] = es;
  }
}

// Executed by the last CTA of a launch (all its threads): choose the pivot
// of column j from the partial arg-maxes (or row j without pivoting),
// record it, flag an exactly zero pivot, swap rows j and p within the
// columns [c0, c1) of the narrow panel being factored (the other columns
// receive the interchanges in one pass per panel, lu_laswp_kernel), and
// publish 1 / pivot for the quotients of column j.
template <int L>
__device__ void finish_pivot(int64_t n, const mat& A, int64_t j, int64_t c0, int64_t c1, int64_t nparts,
                             const partial_t* part, int64_t* ipiv, int64_t* info, int pivot, col_state* cs) {
  using T = typename num<L>::T;
  __shared__ partial_t sbest[8];
  __shared__ int64_t sp;
  const int tid = threadIdx.x;
  if (pivot) {
    partial_t v = none();
    for (int64_t t = tid; t < nparts; t += blockDim.x) {
      const partial_t q = part[t];
      if (better(q, v)) v = q;
    }
    warp_best(v);
    if ((tid & 31) == 0) sbest[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (better(sbest[w], v)) v = sbest[w];
      sp = (v.idx >= j && v.idx < n) ? v.idx : j;
    }
  } else if (tid == 0) {
    sp = j;
  }
  __syncthreads();
  const int64_t p = sp;
  if (p != j) {
    for (int64_t c = c0 + tid; c < c1; c += blockDim.x)
#pragma unroll
      for (int q = 0; q < L; ++q) {
        double* rj = A.p[q] + j * A.ld + c;
        double* rp = A.p[q] + p * A.ld + c;
        const double t = *rj;
        *rj = *rp;
        *rp = t;
      }
  }
  __syncthreads();
  if (tid == 0) {
    ipiv[j] = p;
    const T piv = ldA<L>(A, j, j);
    const bool zero = is_zero<L>(piv);
    if (zero && *info == 0) *info = j + 1;
    T r = num<L>::zero();
    if (!zero) {
      if constexpr (L == 4) {
        const dd_t y = dd_recip(dd_t{piv.x[0], piv.x[1]});
        qd_recip_refine(piv.x, y.hi, y.lo, r.x);
      }
      else r = num<L>::recip(piv);
    }
    const double* x = reinterpret_cast<const double*>(&r);
#pragma unroll
    for (int q = 0; q < L; ++q) cs->rinv[q] = x[q];
    cs->counter = 0u;
  }
}

// Am I the last CTA of this launch to get here? (publishes this CTA's
// global writes first; no CTA waits for another)
__device__ __forceinline__ bool last_block(col_state* cs) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&cs->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

}  // namespace

// First column j of a narrow panel [j, pe): partial arg-maxes of column j
// over rows [j, n) (RB rows per CTA), then the last CTA chooses and swaps
// the pivot.
template <int L>
__global__ void __launch_bounds__(256) lu_start_kernel(int64_t n, mat A, int64_t j, int64_t pe, partial_t* part,
                                                       int64_t* ipiv, int64_t* info, int pivot,
                                                       col_state* cs) {
  const int tid = threadIdx.x;
  if (pivot && tid < 32) {
    const int64_t i = j + (int64_t)blockIdx.x * RB + tid;
    partial_t v = i < n ? cand<L>(ldA<L>(A, i, j), i) : none();
    warp_best(v);
    if (tid == 0) part[blockIdx.x] = v;
  }
  if (last_block(cs)) finish_pivot<L>(n, A, j, j, pe, gridDim.x, part, ipiv, info, pivot, cs);
}

// Column j of the narrow panel [c0, pe) (its pivot row already in place,
// 1 / pivot in cs): quotients l_ij = a_ij (1 / a_jj) for rows below j,
// rank-1 update of columns (j, pe) of those rows; then, if column j + 1
// belongs to the same panel, the partial arg-maxes of the updated column
// j + 1 and, in the last CTA, its pivot. For QD the quotients and updates
// run on the integer pipe: operands as W-word fixed-point integers, each
// quotient one multiword product (kept at full width for the updates,
// stored rounded), each update a - l u exact in a window and rounded once.
template <int L>
__global__ void __launch_bounds__(256) lu_col_kernel(int64_t n, mat A, int64_t c0, int64_t j, int64_t pe,
                                                     partial_t* part, int64_t* ipiv, int64_t* info,
                                                     int pivot, col_state* cs) {
  using N = num<L>;
  constexpr int W = tfx<L>::W, D = tfx<L>::D, K = tfx<L>::K, NW = tfx<L>::NW;
  constexpr int TOPW = 32 * W - 53;
  __shared__ uint32_t uw[PANEL_BASE][W];  // pe - j - 1 < PANEL_BASE
  __shared__ int ue[PANEL_BASE];           // exponent field | sign << 16, or -1 for zero
  __shared__ uint32_t lw[RB][W];
  __shared__ int le[RB], ls[RB];           // exponent field, sign; le = -1 for zero
  const int tid = threadIdx.x;
  const int64_t r0 = j + 1 + (int64_t)blockIdx.x * RB;
  const int rows = (int)(n - r0 < RB ? n - r0 : RB);
  const int cols = (int)(pe - j - 1);
  if constexpr (L == 2 && kDDColumnFP64) {
    // DD on the FP64 pipe (7 + 20 instructions per update)
    using T = typename N::T;
    __shared__ T u[PANEL_BASE];
    __shared__ T lq[RB];
    const T rinv = get_rinv<L>(cs);
    const bool zero = is_zero<L>(rinv);
    if (tid < rows) {
      T l = N::zero();
      if (!zero) {
        l = N::mul(ldA<L>(A, r0 + tid, j), rinv);
        stA<L>(A, r0 + tid, j, l);
      }
      lq[tid] = l;
    }
    for (int c = tid; c < cols; c += blockDim.x) u[c] = ldA<L>(A, j, j + 1 + c);
    __syncthreads();
    for (int e = tid; e < rows * cols; e += blockDim.x) {
      const int r = e / cols, c = e % cols;
      const int64_t i = r0 + r, jc = j + 1 + c;
      stA<L>(A, i, jc, N::add(ldA<L>(A, i, jc), N::mul(N::neg(lq[r]), u[c])));
    }
  } else {
  if (tid < rows) {
    le[tid] = -1;
    double rv[L];
#pragma unroll
    for (int q = 0; q < L; ++q) rv[q] = cs->rinv[q];
    if ((fx::dbits(rv[0]) << 1) != 0u) {
      double a[L];
#pragma unroll
      for (int q = 0; q < L; ++q) a[q] = A.p[q][(r0 + tid) * A.ld + j];
      if ((fx::dbits(a[0]) << 1) != 0u) {
        uint32_t Ma[W], Mr[W], P[K], Ml[W];
        const int ea = fx::to_fixed<L, W>(a, Ma), er = fx::to_fixed<L, W>(rv, Mr);
        fx::mul_top<W, D>(Ma, Mr, P);
        const int p = fx::acc_normalize<K, W>(P, Ml);
        const int el = p + (ea & 0xFFFF) + (er & 0xFFFF) - 1075 - 2 * TOPW + 32 * D - 52;
        const int sl = ((ea ^ er) >> 16) & 1;
        // store l rounded to DD / QD
        double o[L];
        fx::operand_to_limbs<L, W>(Ml, el, (uint32_t)sl, o);
        typename N::T v;
        if constexpr (L == 2) v = dd_t{o[0], o[1]};
        else v = qd_t{{o[0], o[1], o[2], o[3]}};
        stA<L>(A, r0 + tid, j, v);
#pragma unroll
        for (int w = 0; w < W; ++w) lw[tid][w] = Ml[w];
        le[tid] = el;
        ls[tid] = sl;
      }
    }
  }
  for (int c = tid; c < cols; c += blockDim.x) {
    double u[L];
#pragma unroll
    for (int q = 0; q < L; ++q) u[q] = A.p[q][j * A.ld + j + 1 + c];
    uint32_t M[W];
    const int es = fx::to_fixed<L, W>(u, M);
#pragma unroll
    for (int w = 0; w < W; ++w) uw[c][w] = M[w];
    ue[c] = (fx::dbits(u[0]) << 1) == 0u ? -1 : es;
  }
  __syncthreads();
  for (int e = tid; e < rows * cols; e += blockDim.x) {
    const int r = e / cols, c = e % cols;
    if (le[r] < 0 || ue[c] < 0) continue;  // l = 0 or u = 0: nothing to subtract
    const int64_t i = r0 + r, jc = j + 1 + c;
    double a[L];
#pragma unroll
    for (int q = 0; q < L; ++q) a[q] = A.p[q][i * A.ld + jc];
    int Aw = max(1, fx::expfield(a[0]));
    uint32_t acc[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) acc[w] = 0u;
    fx::add_at<L, NW>(acc, a, Aw, tfx<L>::TOPA, 0u);
    uint32_t Ml[W], Mu[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      Ml[w] = lw[r][w];
      Mu[w] = uw[c][w];
    }
    window_sub_product<L>(acc, Aw, Ml, le[r], (uint32_t)ls[r], Mu, ue[c] & 0xFFFF, (uint32_t)ue[c] >> 16);
    window_store<L>(acc, Aw, A, i, jc);
  }
  }
  if (j + 1 >= pe) return;  // the next panel starts with lu_start_kernel
  __syncthreads();
  if (pivot && tid < 32) {
    partial_t v = tid < rows ? cand<L>(ldA<L>(A, r0 + tid, j + 1), r0 + tid) : none();
    warp_best(v);
    if (tid == 0) part[blockIdx.x] = v;
  }
  if (last_block(cs)) finish_pivot<L>(n, A, j + 1, c0, pe, gridDim.x, part, ipiv, info, pivot, cs);
}

// ---------------------------------------------------------------------------
// One launch per narrow panel (the Section 4 step 1 panel factorisation of
// PANEL_BASE columns, all its column steps in one cooperative kernel).
//
// The rows [c0, n) are split into G contiguous chunks of R rows, one per
// CTA; each CTA keeps its rows of the panel in shared memory for the whole
// panel. Per column j one grid barrier: before it, every CTA publishes its
// best pivot candidate together with that row's panel values, and the
// owner of row j publishes row j (double-buffered slots, so that a CTA one
// column ahead never overwrites what a slower CTA still reads); after it,
// every CTA picks the same pivot from the G candidates, takes the pivot row
// from the winner's slot, performs its part of the row interchange, forms
// 1 / pivot, its quotients and its rank-1 updates with the same arithmetic
// as the per-column kernels. All CTAs are co-resident (cooperative launch);
// the barrier's wait is bounded and a CTA that gives up records -1 in
// *info and returns.
constexpr int PR_MAX = 64;  // rows per CTA kept in shared memory

struct pub_t {
  partial_t c;
  double row[PANEL_BASE * 4];  // the candidate's panel row, L doubles per entry
};

struct panel_sync {
  unsigned int count;  // arrivals at the current barrier
  unsigned int gen;    // completed barriers
};

constexpr unsigned int PANEL_WAIT_TRIES = 1u << 22;

// Barrier of the G co-resident CTAs; false if the wait ran out (then *info
// = -1) or another CTA gave up before.
__device__ __forceinline__ bool panel_barrier(panel_sync* ps, unsigned int& gen, unsigned int G, int64_t* info) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned int g = gen;
    __threadfence();
    if (atomicAdd(&ps->count, 1u) == G - 1u) {
      atomicExch(&ps->count, 0u);
      __threadfence();
      atomicExch(&ps->gen, g + 1u);
    } else {
      unsigned int i = 0;
      while (*reinterpret_cast<volatile unsigned int*>(&ps->gen) == g) {
        if (++i > PANEL_WAIT_TRIES || *reinterpret_cast<volatile int64_t*>(info) < 0) {
          ok = 0;
          atomicExch(reinterpret_cast<unsigned long long*>(info), (unsigned long long)(int64_t)-1);
          break;
        }
        if (i > 32) __nanosleep(64);
      }
    }
    __threadfence();
    gen = g + 1u;
  }
  __syncthreads();
  return ok != 0;
}

template <int L>
__device__ __forceinline__ void put_row(double* dst, const typename num<L>::T* src, int w) {
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    const double* x = reinterpret_cast<const double*>(&src[c]);
#pragma unroll
    for (int q = 0; q < L; ++q) dst[c * L + q] = x[q];
  }
}

// Reads of what other CTAs published bypass L1 (__ldcg): the slots are
// reused every other column and L1 is not coherent across SMs.
template <int L>
__device__ __forceinline__ void get_row(typename num<L>::T* dst, const double* src, int w) {
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    double* x = reinterpret_cast<double*>(&dst[c]);
#pragma unroll
    for (int q = 0; q < L; ++q) x[q] = __ldcg(src + c * L + q);
  }
}

__device__ __forceinline__ partial_t get_cand(const partial_t* p) {
  return partial_t{__ldcg(&p->kh), __ldcg(&p->kl), (int64_t)__ldcg(reinterpret_cast<const long long*>(&p->idx))};
}

// One column step of a panel held in shared memory: the quotients
// l_ij = a_ij (1 / a_jj) of this CTA's rows below j and the rank-1 update of
// their columns (j, w), with the per-column kernels' arithmetic (exact
// fixed-point form on the integer pipe). rows: nr rows starting at global row
// r_lo; prow: the pivot row; scratch in shared memory.
template <int L>
struct panel_scratch {
  typename num<L>::T* lq;
  uint32_t (*lw)[tfx<L>::W];
  int* le;
  int* ls;
  uint32_t (*uw)[tfx<L>::W];
  int* ue;
};

template <int L>
__device__ __forceinline__ void panel_column_step(typename num<L>::T (*rows)[PANEL_BASE], int nr, int64_t r_lo,
                                                  int64_t j, int jc, int w, const typename num<L>::T* prow,
                                                  const typename num<L>::T rinv, const panel_scratch<L>& sc) {
  using N = num<L>;
  using T = typename N::T;
  constexpr int W = tfx<L>::W, D = tfx<L>::D, K = tfx<L>::K, NW = tfx<L>::NW;
  constexpr int TOPW = 32 * W - 53;
  const int tid = threadIdx.x;
  T* lq = sc.lq;
  uint32_t (*lw)[W] = sc.lw;
  uint32_t (*uw)[W] = sc.uw;
  int *le = sc.le, *ls = sc.ls, *ue = sc.ue;
  (void)lq;
  const bool zero = is_zero<L>(rinv);
  const int cols = w - jc - 1;
  if (!zero) {
    if constexpr (L == 2 && kDDColumnFP64) {
      for (int r = tid; r < nr; r += blockDim.x) {
        T l = N::zero();
        if (r_lo + r > j) {
          l = N::mul(rows[r][jc], rinv);
          rows[r][jc] = l;
        }
        lq[r] = l;
      }
      __syncthreads();
      for (int e = tid; e < nr * cols; e += blockDim.x) {
        const int r = e / cols, c = jc + 1 + e % cols;
        if (r_lo + r > j) rows[r][c] = N::add(rows[r][c], N::mul(N::neg(lq[r]), prow[c]));
      }
    } else {
      for (int r = tid; r < nr; r += blockDim.x) {
        le[r] = -1;
        const T a = rows[r][jc];
        if (r_lo + r > j && !is_zero<L>(a)) {
          const double* ax = reinterpret_cast<const double*>(&a);
          const double* rx = reinterpret_cast<const double*>(&rinv);
          double av[L], rv[L];
#pragma unroll
          for (int q = 0; q < L; ++q) av[q] = ax[q], rv[q] = rx[q];
          uint32_t Ma[W], Mr[W], P[K], Ml[W];
          const int ea = fx::to_fixed<L, W>(av, Ma), er = fx::to_fixed<L, W>(rv, Mr);
          fx::mul_top<W, D>(Ma, Mr, P);
          const int pp = fx::acc_normalize<K, W>(P, Ml);
          const int el = pp + (ea & 0xFFFF) + (er & 0xFFFF) - 1075 - 2 * TOPW + 32 * D - 52;
          const int sl = ((ea ^ er) >> 16) & 1;
          double o[L];
          fx::operand_to_limbs<L, W>(Ml, el, (uint32_t)sl, o);
          T lv;
          double* lx = reinterpret_cast<double*>(&lv);
#pragma unroll
          for (int q = 0; q < L; ++q) lx[q] = o[q];
          rows[r][jc] = lv;
#pragma unroll
          for (int t = 0; t < W; ++t) lw[r][t] = Ml[t];
          le[r] = el;
          ls[r] = sl;
        }
      }
      for (int c = tid; c < cols; c += blockDim.x) {
        const double* ux = reinterpret_cast<const double*>(&prow[jc + 1 + c]);
        double u[L];
#pragma unroll
        for (int q = 0; q < L; ++q) u[q] = ux[q];
        uint32_t M[W];
        const int es = fx::to_fixed<L, W>(u, M);
#pragma unroll
        for (int t = 0; t < W; ++t) uw[c][t] = M[t];
        ue[c] = (fx::dbits(u[0]) << 1) == 0u ? -1 : es;
      }
      __syncthreads();
      for (int e = tid; e < nr * cols; e += blockDim.x) {
        const int r = e / cols, c = e % cols;
        if (le[r] < 0 || ue[c] < 0) continue;  // l = 0 or u = 0: nothing to subtract
        const double* ax = reinterpret_cast<const double*>(&rows[r][jc + 1 + c]);
        double a[L];
#pragma unroll
        for (int q = 0; q < L; ++q) a[q] = ax[q];
        int Aw = max(1, fx::expfield(a[0]));
        uint32_t acc[NW];
#pragma unroll
        for (int t = 0; t < NW; ++t) acc[t] = 0u;
        fx::add_at<L, NW>(acc, a, Aw, tfx<L>::TOPA, 0u);
        uint32_t Ml[W], Mu[W];
#pragma unroll
        for (int t = 0; t < W; ++t) {
          Ml[t] = lw[r][t];
          Mu[t] = uw[c][t];
        }
        window_sub_product<L>(acc, Aw, Ml, le[r], (uint32_t)ls[r], Mu, ue[c] & 0xFFFF, (uint32_t)ue[c] >> 16);
        double o[L];
        fx::from_fixed<L, NW>(acc, Aw - 1075 - tfx<L>::TOPA, o);
        double* dx = reinterpret_cast<double*>(&rows[r][jc + 1 + c]);
#pragma unroll
        for (int q = 0; q < L; ++q) dx[q] = o[q];
      }
    }
  }
}

// The interchanges of one panel (row c0 + t with row piv[t], t < w, in
// order) applied to the columns outside [c0, pe), spread over the grid's
// threads (all CTAs of the launch, column slices of their own: nothing
// else touches those columns during the panel). piv: this CTA's copy of the
// panel's pivots in shared memory. In batches of SWAP_BATCH pivots (at most
// 2 SWAP_BATCH rows each, their composed permutation worked out once per
// CTA): the batches in order give the interchanges in order.
constexpr int SWAP_BATCH = 8;

template <int L>
__device__ __forceinline__ void panel_swaps(int64_t n, const mat& A, int64_t c0, int64_t pe, const int64_t* piv,
                                           int w, unsigned int cta, unsigned int ctas) {
  __shared__ int64_t dst[2 * SWAP_BATCH], src[2 * SWAP_BATCH];
  __shared__ int cnt;
  const int64_t outside = n - (pe - c0);
  for (int t0 = 0; t0 < w; t0 += SWAP_BATCH) {
    __syncthreads();
    if (threadIdx.x == 0) {
      int c = 0;
      auto slot = [&](int64_t r) {
        for (int t = 0; t < c; ++t)
          if (dst[t] == r) return t;
        dst[c] = r;
        src[c] = r;
        return c++;
      };
      for (int t = t0; t < w && t < t0 + SWAP_BATCH; ++t) {
        const int64_t k = c0 + t, p = piv[t];
        if (p == k || p < 0 || p >= n) continue;
        const int a = slot(k), b = slot(p);
        const int64_t x = src[a];
        src[a] = src[b];
        src[b] = x;
      }
      cnt = c;
    }
    __syncthreads();
    const int nrows = cnt;
    if (nrows == 0) continue;
    for (int64_t e = (int64_t)cta * blockDim.x + threadIdx.x; e < outside * L; e += (int64_t)ctas * blockDim.x) {
      const int q = (int)(e / outside);
      int64_t col = e % outside;
      if (col >= c0) col += pe - c0;
      double v[2 * SWAP_BATCH];
#pragma unroll
      for (int t = 0; t < 2 * SWAP_BATCH; ++t)
        if (t < nrows) v[t] = A.p[q][src[t] * A.ld + col];
#pragma unroll
      for (int t = 0; t < 2 * SWAP_BATCH; ++t)
        if (t < nrows) A.p[q][dst[t] * A.ld + col] = v[t];
    }
  }
}

template <int L>
__global__ void __launch_bounds__(256) lu_panel_kernel(int64_t n, mat A, int64_t c0, int64_t pe, int64_t R,
                                                       int64_t* ipiv, int64_t* info, int pivot, pub_t* pub,
                                                       double* rowj, panel_sync* ps, int extra) {
  using N = num<L>;
  using T = typename N::T;
  constexpr int W = tfx<L>::W;
  __shared__ T rows[PR_MAX][PANEL_BASE];
  __shared__ T prow[PANEL_BASE];  // the pivot row (row j after the interchange)
  __shared__ T lq[PR_MAX];        // DD quotients
  __shared__ uint32_t lw[PR_MAX][W], uw[PANEL_BASE][W];  // QD fixed-point quotients / pivot row
  __shared__ int le[PR_MAX], ls[PR_MAX], ue[PANEL_BASE];
  __shared__ partial_t sbest[8];
  __shared__ T srinv;
  __shared__ int64_t piv_s[PANEL_BASE];  // the panel's pivots, for panel_swaps
  const int tid = threadIdx.x, nw = blockDim.x >> 5;
  const int w = (int)(pe - c0);
  const unsigned int G = gridDim.x;
  const unsigned int arrivals = G + (unsigned int)extra;  // extra > 0 only in the wait test
  const int64_t r_lo = c0 + (int64_t)blockIdx.x * R;
  const int64_t left = n - r_lo;
  const int nr = left <= 0 ? 0 : (int)(left < R ? left : R);
  unsigned int gen = *reinterpret_cast<volatile unsigned int*>(&ps->gen);
  for (int e = tid; e < nr * w; e += blockDim.x) rows[e / w][e % w] = ldA<L>(A, r_lo + e / w, c0 + e % w);
  __syncthreads();

  for (int64_t j = c0; j < pe; ++j) {
    const int jc = (int)(j - c0);
    pub_t* slot = pub + (size_t)(jc & 1) * G;
    double* rj = rowj + (size_t)(jc & 1) * PANEL_BASE * 4;
    // ---- this CTA's best candidate (rows i >= j), published with its row
    partial_t v = none();
    if (pivot) {
      for (int r = tid; r < nr; r += blockDim.x)
        if (r_lo + r >= j) {
          const partial_t q = cand<L>(rows[r][jc], r_lo + r);
          if (better(q, v)) v = q;
        }
      warp_best(v);
      if ((tid & 31) == 0) sbest[tid >> 5] = v;
      __syncthreads();
      v = sbest[0];
      for (int k = 1; k < nw; ++k)
        if (better(sbest[k], v)) v = sbest[k];
      if (v.idx != INT64_MAX) put_row<L>(slot[blockIdx.x].row, rows[v.idx - r_lo], w);
    }
    if (tid == 0) slot[blockIdx.x].c = v;
    if (j >= r_lo && j < r_lo + nr) put_row<L>(rj, rows[j - r_lo], w);
    if (!panel_barrier(ps, gen, arrivals, info)) return;
    // ---- the pivot: the best of the G candidates (a strict order: every
    // CTA picks the same), or row j without pivoting
    partial_t b = none();
    if (pivot) {
      for (unsigned int k = tid; k < G; k += blockDim.x) {
        const partial_t q = get_cand(&slot[k].c);
        if (better(q, b)) b = q;
      }
      warp_best(b);
      __syncthreads();
      if ((tid & 31) == 0) sbest[tid >> 5] = b;
      __syncthreads();
      b = sbest[0];
      for (int k = 1; k < nw; ++k)
        if (better(sbest[k], b)) b = sbest[k];
    }
    const bool pv = pivot && b.idx >= j && b.idx < n;
    const int64_t p = pv ? b.idx : j;
    if (tid == 0) piv_s[jc] = p;
    if (pv) get_row<L>(prow, slot[(b.idx - c0) / R].row, w);
    else get_row<L>(prow, rj, w);
    __syncthreads();
    // ---- the interchange of rows j and p within the panel
    if (j >= r_lo && j < r_lo + nr)
      for (int c = tid; c < w; c += blockDim.x) rows[j - r_lo][c] = prow[c];
    if (p != j && p >= r_lo && p < r_lo + nr) get_row<L>(rows[p - r_lo], rj, w);
    if (tid == 0) {
      const T piv = prow[jc];
      const bool zero = is_zero<L>(piv);
      if (blockIdx.x == 0) {
        ipiv[j] = p;
        if (zero && *info == 0) *info = j + 1;
      }
      T r = N::zero();
      if (!zero) {
        if constexpr (L == 4) {
          const dd_t y = dd_recip(dd_t{piv.x[0], piv.x[1]});
          qd_recip_refine(piv.x, y.hi, y.lo, r.x);
        } else {
          r = N::recip(piv);
        }
      }
      srinv = r;
    }
    __syncthreads();
    // ---- quotients l_ij = a_ij (1 / a_jj) and the rank-1 update of the
    // columns (j, pe) of this CTA's rows below j
    const T rinv = srinv;
    panel_column_step<L>(rows, nr, r_lo, j, jc, w, prow, rinv,
                         panel_scratch<L>{lq, lw, le, ls, uw, ue});
    __syncthreads();
  }
  for (int e = tid; e < nr * w; e += blockDim.x) stA<L>(A, r_lo + e / w, c0 + e % w, rows[e / w][e % w]);
  if (pivot) panel_swaps<L>(n, A, c0, pe, piv_s, w, blockIdx.x, G);
}

// ---------------------------------------------------------------------------
// The same panel factorisation by one thread-block cluster (up to 16 CTAs;
// distributed shared memory): each CTA holds up to RCL_MAX rows of the
// panel in shared memory; per column, after a cluster barrier every CTA
// reads the CTAs' candidates and the pivot row and row j straight from the
// owners' shared memory, a second cluster barrier lets the owners
// interchange the rows, and the column step follows. The barriers are the
// hardware's (every CTA passes every one of them; no spin-wait), and the
// arithmetic is panel_column_step's, so the factors are the same bits as the
// grid form's and the per-column kernels'.
constexpr int RCL_MAX = 256;  // rows per CTA of the cluster form

template <int L>
struct cl_smem {
  typename num<L>::T rows[RCL_MAX][PANEL_BASE];
  typename num<L>::T prow[PANEL_BASE], oldj[PANEL_BASE];
  typename num<L>::T lq[RCL_MAX];
  uint32_t lw[RCL_MAX][tfx<L>::W], uw[PANEL_BASE][tfx<L>::W];
  int le[RCL_MAX], ls[RCL_MAX], ue[PANEL_BASE];
  partial_t cand, sbest[8];
  typename num<L>::T rinv;
  int64_t piv[PANEL_BASE];  // the panel's pivots, for panel_swaps
};

template <int L>
__global__ void __launch_bounds__(256) lu_panel_cluster_kernel(int64_t n, mat A, int64_t c0, int64_t pe, int64_t R,
                                                               int64_t* ipiv, int64_t* info, int pivot) {
  using N = num<L>;
  using T = typename N::T;
  extern __shared__ __align__(16) unsigned char cl_raw[];
  cl_smem<L>& sm = *reinterpret_cast<cl_smem<L>*>(cl_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned int rank = cluster.block_rank(), CS = cluster.num_blocks();
  const int tid = threadIdx.x, nw = blockDim.x >> 5;
  const int w = (int)(pe - c0);
  const int64_t r_lo = c0 + (int64_t)rank * R;
  const int64_t left = n - r_lo;
  const int nr = left <= 0 ? 0 : (int)(left < R ? left : R);
  for (int e = tid; e < nr * w; e += blockDim.x) sm.rows[e / w][e % w] = ldA<L>(A, r_lo + e / w, c0 + e % w);
  __syncthreads();

  for (int64_t j = c0; j < pe; ++j) {
    const int jc = (int)(j - c0);
    // ---- this CTA's best candidate (rows i >= j)
    partial_t v = none();
    if (pivot) {
      for (int r = tid; r < nr; r += blockDim.x)
        if (r_lo + r >= j) {
          const partial_t q = cand<L>(sm.rows[r][jc], r_lo + r);
          if (better(q, v)) v = q;
        }
      warp_best(v);
      if ((tid & 31) == 0) sm.sbest[tid >> 5] = v;
      __syncthreads();
      v = sm.sbest[0];
      for (int k = 1; k < nw; ++k)
        if (better(sm.sbest[k], v)) v = sm.sbest[k];
    }
    if (tid == 0) sm.cand = v;
    cluster.sync();  // candidates and rows visible to the whole cluster
    // ---- the pivot (every CTA the same), the pivot row and row j from their owners
    if (tid < 32) {
      partial_t b = none();
      if (pivot && (unsigned int)tid < CS) b = *cluster.map_shared_rank(&sm.cand, (unsigned int)tid);
      warp_best(b);
      if (tid == 0) sm.sbest[0] = b;
    }
    __syncthreads();
    const partial_t b = sm.sbest[0];
    const int64_t p = (pivot && b.idx >= j && b.idx < n) ? b.idx : j;
    if (tid == 0) sm.piv[jc] = p;
    {
      const unsigned int op = (unsigned int)((p - c0) / R), oj = (unsigned int)((j - c0) / R);
      const T* rp = cluster.map_shared_rank(&sm.rows[0][0], op) + (p - c0 - (int64_t)op * R) * PANEL_BASE;
      const T* rjp = cluster.map_shared_rank(&sm.rows[0][0], oj) + (j - c0 - (int64_t)oj * R) * PANEL_BASE;
      for (int c = tid; c < w; c += blockDim.x) {
        sm.prow[c] = rp[c];
        sm.oldj[c] = rjp[c];
      }
    }
    cluster.sync();  // every CTA has read the two rows before their owners change them
    // ---- the interchange of rows j and p within the panel
    if (j >= r_lo && j < r_lo + nr)
      for (int c = tid; c < w; c += blockDim.x) sm.rows[j - r_lo][c] = sm.prow[c];
    if (p != j && p >= r_lo && p < r_lo + nr)
      for (int c = tid; c < w; c += blockDim.x) sm.rows[p - r_lo][c] = sm.oldj[c];
    if (tid == 0) {
      const T piv = sm.prow[jc];
      const bool zero = is_zero<L>(piv);
      if (rank == 0) {
        ipiv[j] = p;
        if (zero && *info == 0) *info = j + 1;
      }
      T r = N::zero();
      if (!zero) {
        if constexpr (L == 4) {
          const dd_t y = dd_recip(dd_t{piv.x[0], piv.x[1]});
          qd_recip_refine(piv.x, y.hi, y.lo, r.x);
        } else {
          r = N::recip(piv);
        }
      }
      sm.rinv = r;
    }
    __syncthreads();
    panel_column_step<L>(sm.rows, nr, r_lo, j, jc, w, sm.prow, sm.rinv,
                         panel_scratch<L>{sm.lq, sm.lw, sm.le, sm.ls, sm.uw, sm.ue});
    __syncthreads();
  }
  for (int e = tid; e < nr * w; e += blockDim.x) stA<L>(A, r_lo + e / w, c0 + e % w, sm.rows[e / w][e % w]);
  if (pivot) panel_swaps<L>(n, A, c0, pe, sm.piv, w, rank, CS);
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// The interchanges ipiv[k0 .. k1) (in order, at most PANEL_BASE) applied to
// every column outside [k0, k1) (the per-column kernels' panels; the fused
// panel kernels do this themselves): panel_swaps over the grid.
template <int L>
__global__ void lu_laswp_kernel(int64_t n, mat A, int64_t k0, int64_t k1, const int64_t* ipiv) {
  __shared__ int64_t piv[PANEL_BASE];
  const int w = (int)(k1 - k0);
  for (int t = threadIdx.x; t < w; t += blockDim.x) piv[t] = ipiv[k0 + t];
  panel_swaps<L>(n, A, k0, k1, piv, w, blockIdx.x, gridDim.x);
}

template <int L>
__device__ __forceinline__ typename num<L>::T shfl(const typename num<L>::T& v, int k) {
  typename num<L>::T r;
  const double* x = reinterpret_cast<const double*>(&v);
  double* y = reinterpret_cast<double*>(&r);
#pragma unroll
  for (int q = 0; q < L; ++q) y[q] = __shfl_sync(0xffffffffu, x[q], k);
  return r;
}

// X := L^-1 X for a unit lower triangle (m <= TB rows): one warp per column
// of X, lane i holding row i as an exact fixed-point window on the integer
// pipe. At step k lane k's value is final: it is normalised to a W-word
// operand and broadcast by shuffles, and the lanes below subtract l_ik x_k
// (W-word product, one placement). Each value is rounded to DD / QD once,
// at the end. (The FP64 form of this loop ran a single warp's DD / QD
// chain through an FP64 pipe that issues one warp instruction per 16
// cycles per SM.)
template <int L>
__global__ void __launch_bounds__(128) trsm_lower_unit_base(int64_t m, int64_t r, mat Lm, mat X) {
  constexpr int W = tfx<L>::W, NW = tfx<L>::NW;
  __shared__ tri_smem<L> sm;
  stage_triangle<L>(sm, Lm, m, false);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (c >= r) return;
  double b[L];
#pragma unroll
  for (int q = 0; q < L; ++q) b[q] = lane < m ? X.p[q][lane * X.ld + c] : 0.0;
  int A = max(1, fx::expfield(b[0]));
  uint32_t acc[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) acc[w] = 0u;
  fx::add_at<L, NW>(acc, b, A, tfx<L>::TOPA, 0u);
  for (int k = 0; k < (int)m; ++k) {
    uint32_t Mx[W], sx;
    int ex;
    bool zx;
    window_operand<L>(acc, A, Mx, ex, sx, zx);
#pragma unroll
    for (int w = 0; w < W; ++w) Mx[w] = __shfl_sync(0xffffffffu, Mx[w], k);
    ex = __shfl_sync(0xffffffffu, ex, k);
    sx = __shfl_sync(0xffffffffu, sx, k);
    zx = __shfl_sync(0xffffffffu, (int)zx, k) != 0;
    if (lane > k && lane < m && !zx) {
      uint32_t Ml[W];
#pragma unroll
      for (int w = 0; w < W; ++w) Ml[w] = sm.Tw[k][w][lane];
      const int es = sm.Te[k][lane];
      window_sub_product<L>(acc, A, Ml, es & 0xFFFF, (uint32_t)es >> 16, Mx, ex, sx);
    }
  }
  if (lane < m) window_store<L>(acc, A, X, lane, c);
}

// X := U^-1 X for an upper triangle with nonzero diagonal (m <= TB rows),
// one warp per column as above, from the last row up. Each lane forms the
// reciprocal of its diagonal entry once (DD / QD Newton step) as a
// fixed-point operand; at step k lane k multiplies its value by it, the
// quotient is broadcast and the lanes above subtract u_ik x_k.
template <int L>
__global__ void __launch_bounds__(128) trsm_upper_base(int64_t m, int64_t r, mat U, mat X) {
  using N = num<L>;
  constexpr int W = tfx<L>::W, D = tfx<L>::D, K = tfx<L>::K, NW = tfx<L>::NW;
  __shared__ tri_smem<L> sm;
  stage_triangle<L>(sm, U, m, true);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (c >= r) return;
  uint32_t Mr[W];
  int er;
  uint32_t sr;
  {
    const typename N::T d = lane < m ? ldA<L>(U, lane, lane) : N::one();
    const typename N::T ri = N::recip(d);
    const int es = fx::to_fixed<L, W>(*reinterpret_cast<const double(*)[L]>(&ri), Mr);
    er = es & 0xFFFF;
    sr = (uint32_t)es >> 16;
  }
  double b[L];
#pragma unroll
  for (int q = 0; q < L; ++q) b[q] = lane < m ? X.p[q][lane * X.ld + c] : 0.0;
  int A = max(1, fx::expfield(b[0]));
  uint32_t acc[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) acc[w] = 0u;
  fx::add_at<L, NW>(acc, b, A, tfx<L>::TOPA, 0u);
  for (int k = (int)m - 1; k >= 0; --k) {
    // x = value * (1 / u_kk): the product's K words normalised to W words
    uint32_t Ma[W], sa;
    int ea;
    bool za;
    window_operand<L>(acc, A, Ma, ea, sa, za);
    uint32_t P[K], Mx[W];
    fx::mul_top<W, D>(Ma, Mr, P);
    const int p = fx::acc_normalize<K, W>(P, Mx);
    // P ~ Ma Mr 2^(32 D - 2 TOPW - 2150 + ea + er) with TOPW = 32 W - 53
    int ex = p + ea + er - 1075 - 2 * (32 * W - 53) + 32 * D - 52;
    uint32_t sx = sa ^ sr;
    bool zx = za || p < 0;
    if (lane == k) {
      // lane k's final value x_k (kept exactly as its window)
      if (zx) {
#pragma unroll
        for (int w = 0; w < NW; ++w) acc[w] = 0u;
      } else {
        window_from_operand<L>(acc, A, Mx, ex, sx);
      }
    }
#pragma unroll
    for (int w = 0; w < W; ++w) Mx[w] = __shfl_sync(0xffffffffu, Mx[w], k);
    ex = __shfl_sync(0xffffffffu, ex, k);
    sx = __shfl_sync(0xffffffffu, sx, k);
    zx = __shfl_sync(0xffffffffu, (int)zx, k) != 0;
    if (lane < k && !zx) {
      uint32_t Mu[W];
#pragma unroll
      for (int w = 0; w < W; ++w) Mu[w] = sm.Tw[k][w][lane];
      const int es = sm.Te[k][lane];
      window_sub_product<L>(acc, A, Mu, es & 0xFFFF, (uint32_t)es >> 16, Mx, ex, sx);
    }
  }
  if (lane < m) window_store<L>(acc, A, X, lane, c);
}

// Row permutation of the interchanges ipiv[0..n): perm[i] = source row of
// row i after all swaps, built by one thread in shared memory when it fits.
__global__ void lu_perm_kernel(int64_t n, const int64_t* ipiv, int64_t* perm) {
  extern __shared__ int32_t sperm[];
  const bool in_smem = n <= 12288;
  if (threadIdx.x != 0) return;
  if (in_smem) {
    for (int64_t i = 0; i < n; ++i) sperm[i] = (int32_t)i;
    for (int64_t j = 0; j < n; ++j) {
      const int64_t p = ipiv[j];
      if (p != j && p >= 0 && p < n) {
        const int32_t t = sperm[j];
        sperm[j] = sperm[p];
        sperm[p] = t;
      }
    }
    for (int64_t i = 0; i < n; ++i) perm[i] = sperm[i];
  } else {
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t j = 0; j < n; ++j) {
      const int64_t p = ipiv[j];
      if (p != j && p >= 0 && p < n) {
        const int64_t t = perm[j];
        perm[j] = perm[p];
        perm[p] = t;
      }
    }
  }
}

template <int L>
__global__ void lu_gather_kernel(int64_t n, int64_t r, const int64_t* perm, mat B, mat X) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * r) return;
  const int64_t i = e / r, c = e % r;
  stA<L>(X, i, c, ldA<L>(B, perm[i], c));
}

// ------------------------------------------------------------------ host --
static ddg_opts block_opts() {
  ddg_opts o;
  ddg_opts_default(&o);
  o.algo = DDG_BLOCK;
  return o;
}

static cudaError_t counted(cudaError_t e) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

// X := L^-1 X (L unit lower, m x m), X m x r.
template <int L>
static ddg_status trsm_lower_unit(int64_t m, int64_t r, const mat& Lm, const mat& X, cudaStream_t s) {
  if (m == 0 || r == 0) return DDG_OK;
  if (m <= TB) {
    trsm_lower_unit_base<L><<<(unsigned)((r + 3) / 4), 128, 0, s>>>(m, r, Lm, X);
    return counted(cudaGetLastError()) == cudaSuccess ? DDG_OK : set_error(DDG_ECUDA, "trsm launch");
  }
  const int64_t m1 = std::max<int64_t>(TB, (m / 2) / TB * TB);
  ddg_status st = trsm_lower_unit<L>(m1, r, Lm, X, s);
  if (st != DDG_OK) return st;
  st = gemm_run(L, m - m1, m1, r, view(Lm, m1, 0), X, view(X, m1, 0), MODE_SUB, block_opts(), s);
  if (st != DDG_OK) return st;
  return trsm_lower_unit<L>(m - m1, r, view(Lm, m1, m1), view(X, m1, 0), s);
}

// X := U^-1 X (U upper, m x m), X m x r.
template <int L>
static ddg_status trsm_upper(int64_t m, int64_t r, const mat& U, const mat& X, cudaStream_t s) {
  if (m == 0 || r == 0) return DDG_OK;
  if (m <= TB) {
    trsm_upper_base<L><<<(unsigned)((r + 3) / 4), 128, 0, s>>>(m, r, U, X);
    return counted(cudaGetLastError()) == cudaSuccess ? DDG_OK : set_error(DDG_ECUDA, "trsm launch");
  }
  const int64_t m1 = std::max<int64_t>(TB, (m / 2) / TB * TB);
  ddg_status st = trsm_upper<L>(m - m1, r, view(U, m1, m1), view(X, m1, 0), s);
  if (st != DDG_OK) return st;
  st = gemm_run(L, m1, m - m1, r, view(U, 0, m1), view(X, m1, 0), X, MODE_SUB, block_opts(), s);
  if (st != DDG_OK) return st;
  return trsm_upper<L>(m1, r, U, X, s);
}

static bool bad_planes(int L, const mat& M, int64_t rows, int64_t cols) {
  if (rows == 0 || cols == 0) return false;
  if (M.ld < cols || M.ld < 1) return true;
  for (int q = 0; q < L; ++q)
    if (!M.p[q]) return true;
  return false;
}

// Cluster size of the cluster panel form on this device (16, else 8), 0 if
// neither can be resident with the form's shared memory; per device, once.
template <int L>
static int cluster_panel_size() {
  static std::mutex mu;
  static std::map<int, int> known;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = known.find(dev);
  if (it != known.end()) return it->second;
  int cs = 0, cl = 0;
  cudaDeviceGetAttribute(&cl, cudaDevAttrClusterLaunch, dev);
  const void* f = (const void*)lu_panel_cluster_kernel<L>;
  if (cl && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(cl_smem<L>)) ==
                cudaSuccess &&
      cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    for (int c : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)c;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)c);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = sizeof(cl_smem<L>);
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, f, &cfg) == cudaSuccess && nclusters >= 1) {
        cs = c;
        break;
      }
    }
  }
  cudaGetLastError();
  known[dev] = cs;
  return cs;
}

template <int L>
static ddg_status getrf_impl(const char* name, int64_t n, const mat& M, int64_t* ipiv, int32_t K,
                             int32_t pivot, const ddg_opts* opts, int64_t* info, void* stream) {
  clear_error();
  const std::string nm(name);
  if (n < 0) return set_error(DDG_EINVAL, nm + ": negative size");
  if (K < 1 || K > KMAX) return set_error(DDG_EINVAL, nm + ": block size K must be in [1, 512]");
  if (pivot != 0 && pivot != 1) return set_error(DDG_EINVAL, nm + ": pivot must be 0 or 1");
  if (bad_planes(L, M, n, n)) return set_error(DDG_EINVAL, nm + ": A: null plane or ld < n");
  if (n > 0 && !ipiv) return set_error(DDG_EINVAL, nm + ": ipiv is null");
  ddg_opts o;
  ddg_opts_default(&o);
  if (opts) o = *opts;
  if (o.algo < DDG_SIMPLE || o.algo > DDG_OZAKI2_TC || o.cutoff < 1 || o.accum < 0 || o.accum > 2 ||
      (o.pad != 0 && o.pad != 1) || (o.streams != 0 && o.streams != 1 && o.streams != 7))
    return set_error(DDG_EINVAL, nm + ": invalid options");
  if (n == 0) return DDG_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t maxparts = (n + RB - 1) / RB;
  // Panel forms, fastest first: one thread-block cluster (CS CTAs holding a
  // few rows each, below), the cooperative grid (one CTA per SM at most, up
  // to PR_MAX rows each), the per-column kernels. DDG_LU_PANEL = "cluster",
  // "grid" or "columns" restricts the choice to that form and the ones after
  // it, an explicit "cluster" taking the cluster form up to RCL_MAX rows per
  // CTA (tests use it to cover every form; all give the same bits).
  int dev = 0, nsm = 0, coop = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_panel_kernel<L>, 256, 0);
  cudaGetLastError();
  const char* env = std::getenv("DDG_LU_PANEL");
  const std::string form = env ? env : "cluster";
  const bool fused_ok = coop && per_sm >= 1 && nsm > 0 && form != "columns";
  const int CS = form == "cluster" ? cluster_panel_size<L>() : 0;
  // the cluster form only while its CTAs hold few rows: its 16 SMs are
  // throughput-bound on the rank-1 updates of taller panels, where the grid
  // form's 152 SMs win despite the slower grid barrier (sweep of the rows
  // per CTA on GB300: DD best at 128, QD at 32)
  const int64_t cl_rows = form == "cluster" && !env ? (L == 2 ? 128 : 32) : RCL_MAX;
  const int64_t gmax = std::max(1, nsm);
  const size_t pub_bytes = 2 * sizeof(pub_t) * (size_t)gmax;
  const size_t bytes = sizeof(partial_t) * (size_t)maxparts + 512 + pub_bytes + 2 * PANEL_BASE * 4 * 8 + 256;
  void* ws = nullptr;
  if (ddg::ws_alloc(&ws, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return set_error(DDG_ENOMEM, nm + ": scratch allocation failed");
  }
  partial_t* part = reinterpret_cast<partial_t*>(static_cast<char*>(ws) + 512);
  char* after = static_cast<char*>(ws) + 512 + sizeof(partial_t) * (size_t)maxparts;
  pub_t* pub = reinterpret_cast<pub_t*>(after);
  double* rowj = reinterpret_cast<double*>(after + pub_bytes);
  panel_sync* psync = reinterpret_cast<panel_sync*>(after + pub_bytes + 2 * PANEL_BASE * 4 * 8);
  int64_t* dinfo = info ? info : reinterpret_cast<int64_t*>(ws);
  col_state* cs = reinterpret_cast<col_state*>(static_cast<char*>(ws) + 256);
  ddg_status st = DDG_OK;
  auto cu = [&](cudaError_t e) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (e != cudaSuccess && st == DDG_OK) st = set_error(DDG_ECUDA, nm + ": " + cudaGetErrorString(e));
  };
  if (cudaMemsetAsync(dinfo, 0, sizeof(int64_t), s) != cudaSuccess ||
      cudaMemsetAsync(cs, 0, sizeof(col_state), s) != cudaSuccess ||
      cudaMemsetAsync(psync, 0, sizeof(panel_sync), s) != cudaSuccess)
    st = set_error(DDG_ECUDA, nm + ": memset");
  // Panel of columns [c0, c0 + w), rows [c0, n): per-column kernels for
  // narrow panels; wider ones split in halves (left half, its triangular
  // solve and Block update of the right half, then the right half), so the
  // rank-1 updates stay within PANEL_BASE columns and the rest of the panel
  // work runs in the Block kernel.
  std::function<void(int64_t, int64_t)> panel = [&](int64_t c0, int64_t w) {
    if (st != DDG_OK || w <= 0) return;
    if (w <= PANEL_BASE) {
      nvtx_range nv("ddg.getrf panel %lld", (long long)c0);
      const int64_t pe = c0 + w;
      const int64_t prow = n - c0;
      if (CS > 0 && (prow + CS - 1) / CS <= cl_rows) {
        const int64_t Rc = (prow + CS - 1) / CS;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)CS;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)CS);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = sizeof(cl_smem<L>);
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cu(cudaLaunchKernelEx(&cfg, lu_panel_cluster_kernel<L>, n, M, c0, pe, Rc, ipiv, dinfo, (int)pivot));
        return;  // the kernel applies the panel's interchanges outside it too
      }
      const int64_t R = std::max<int64_t>(8, (prow + gmax - 1) / gmax);
      if (fused_ok && R <= PR_MAX) {
        const unsigned G = (unsigned)((prow + R - 1) / R);
        int64_t nn = n, cc0 = c0, ppe = pe, RR = R;
        int piv = pivot, extra = 0;
        mat MM = M;
        int64_t* ip = ipiv;
        void* args[] = {&nn, &MM, &cc0, &ppe, &RR, &ip, &dinfo, &piv, &pub, &rowj, &psync, &extra};
        cu(cudaLaunchCooperativeKernel((const void*)lu_panel_kernel<L>, dim3(G), dim3(256), args, 0, s));
        return;  // the kernel applies the panel's interchanges outside it too
      }
      const int64_t nstart = pivot ? (n - c0 + RB - 1) / RB : 1;
      lu_start_kernel<L><<<(unsigned)nstart, 256, 0, s>>>(n, M, c0, pe, part, ipiv, dinfo, pivot, cs);
      cu(cudaGetLastError());
      for (int64_t j = c0; j < pe && j + 1 < n && st == DDG_OK; ++j) {
        const int64_t blocks = (n - j - 1 + RB - 1) / RB;
        lu_col_kernel<L><<<(unsigned)blocks, 256, 0, s>>>(n, M, c0, j, pe, part, ipiv, dinfo, pivot, cs);
        cu(cudaGetLastError());
      }
      if (pivot && st == DDG_OK) {
        lu_laswp_kernel<L><<<(unsigned)((n * L + 127) / 128), 128, 0, s>>>(n, M, c0, pe, ipiv);
        cu(cudaGetLastError());
      }
      return;
    }
    const int64_t w1 = std::max<int64_t>(PANEL_BASE, (w / 2) / PANEL_BASE * PANEL_BASE);
    panel(c0, w1);
    if (st != DDG_OK) return;
    const int64_t w2 = w - w1, c1 = c0 + w1;
    st = trsm_lower_unit<L>(w1, w2, view(M, c0, c0), view(M, c0, c1), s);
    if (st != DDG_OK) return;
    if (n - c1 > 0)
      st = gemm_run(L, n - c1, w1, w2, view(M, c1, c0), view(M, c0, c1), view(M, c1, c1), MODE_SUB,
                    block_opts(), s);
    if (st != DDG_OK) return;
    panel(c1, w2);
  };
  for (int64_t j0 = 0; j0 < n && st == DDG_OK; j0 += K) {
    const int64_t pe = std::min<int64_t>(n, j0 + K);
    panel(j0, pe - j0);
    if (st != DDG_OK || pe >= n) break;
    const int64_t kb = pe - j0, rest = n - pe;
    st = trsm_lower_unit<L>(kb, rest, view(M, j0, j0), view(M, j0, pe), s);
    if (st != DDG_OK) break;
    // Section 4 step 3: A22 := A22 - L21 U12
    nvtx_range nv("ddg.getrf trailing update %lld", (long long)pe);
    st = gemm_run(L, rest, kb, rest, view(M, pe, j0), view(M, j0, pe), view(M, pe, pe), MODE_SUB, o, s);
  }
  int64_t hinfo = 0;
  if (st == DDG_OK && !info) {
    if (cudaMemcpyAsync(&hinfo, dinfo, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = set_error(DDG_ECUDA, nm + ": reading the pivot status");
  }
  ddg::ws_free(ws, s);
  if (st == DDG_OK && hinfo < 0)
    return set_error(DDG_ETIMEOUT, nm + ": a bounded device wait of the panel kernel ran out");
  if (st == DDG_OK && hinfo != 0)
    return set_error(DDG_ESINGULAR, nm + ": exactly zero pivot in column " + std::to_string(hinfo - 1));
  return st;
}

// Test support: one panel of a 64 x 64 DD matrix in 8 CTAs whose grid
// barrier expects one arrival more than there are CTAs, so that every CTA's
// bounded wait runs out; synchronous. DDG_ETIMEOUT when info came back -1.
ddg_status lu_panel_wait_test() {
  const int64_t n = 64;
  char* buf = nullptr;
  const size_t mat_bytes = 2 * n * n * sizeof(double);
  const size_t bytes = mat_bytes + n * sizeof(int64_t) + 64 + 2 * 8 * sizeof(pub_t) + 2 * PANEL_BASE * 4 * 8 + 64;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) return set_error(DDG_ENOMEM, "wait test: allocation failed");
  cudaMemset(buf, 0, bytes);
  mat M{};
  M.p[0] = reinterpret_cast<double*>(buf);
  M.p[1] = M.p[0] + n * n;
  M.ld = n;
  int64_t* ipiv = reinterpret_cast<int64_t*>(buf + mat_bytes);
  int64_t* info = ipiv + n;
  pub_t* pub = reinterpret_cast<pub_t*>(buf + mat_bytes + n * sizeof(int64_t) + 64);
  double* rowj = reinterpret_cast<double*>(reinterpret_cast<char*>(pub) + 2 * 8 * sizeof(pub_t));
  panel_sync* ps = reinterpret_cast<panel_sync*>(rowj + 2 * PANEL_BASE * 4);
  int64_t nn = n, c0 = 0, pe = PANEL_BASE, R = 8;
  int piv = 1, extra = 1;
  void* args[] = {&nn, &M, &c0, &pe, &R, &ipiv, &info, &piv, &pub, &rowj, &ps, &extra};
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)lu_panel_kernel<2>, dim3(8), dim3(256), args, 0, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int64_t h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, info, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return set_error(DDG_ECUDA, std::string("wait test: ") + cudaGetErrorString(e));
  return h < 0 ? set_error(DDG_ETIMEOUT, "panel barrier wait ran out (as intended)") : DDG_OK;
}

template <int L>
static ddg_status getrs_impl(const char* name, int64_t n, int64_t nrhs, const mat& LUm, const int64_t* ipiv,
                             const mat& Bm, void* stream) {
  clear_error();
  const std::string nm(name);
  if (n < 0 || nrhs < 0) return set_error(DDG_EINVAL, nm + ": negative size");
  if (bad_planes(L, LUm, n, n) || bad_planes(L, Bm, n, nrhs))
    return set_error(DDG_EINVAL, nm + ": null plane or ld too small");
  if (n > 0 && !ipiv) return set_error(DDG_EINVAL, nm + ": ipiv is null");
  if (n == 0 || nrhs == 0) return DDG_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t plane = ((size_t)n * nrhs * sizeof(double) + 255) & ~(size_t)255;
  const size_t bytes = L * plane + (((size_t)n * sizeof(int64_t) + 255) & ~(size_t)255);
  void* ws = nullptr;
  if (ddg::ws_alloc(&ws, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return set_error(DDG_ENOMEM, nm + ": scratch allocation failed");
  }
  char* base = static_cast<char*>(ws);
  mat X{};
  X.ld = nrhs;
  for (int q = 0; q < L; ++q) X.p[q] = reinterpret_cast<double*>(base + q * plane);
  int64_t* perm = reinterpret_cast<int64_t*>(base + L * plane);
  ddg_status st = DDG_OK;
  const size_t sm = n <= 12288 ? (size_t)n * sizeof(int32_t) : 0;
  lu_perm_kernel<<<1, 32, sm, s>>>(n, ipiv, perm);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    const int64_t tot = n * nrhs;
    lu_gather_kernel<L><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, nrhs, perm, Bm, X);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) st = set_error(DDG_ECUDA, nm + ": " + cudaGetErrorString(e));
  if (st == DDG_OK) st = trsm_lower_unit<L>(n, nrhs, LUm, X, s);
  if (st == DDG_OK) st = trsm_upper<L>(n, nrhs, LUm, X, s);
  if (st == DDG_OK)
    for (int q = 0; q < L && st == DDG_OK; ++q)
      if (cudaMemcpy2DAsync(Bm.p[q], Bm.ld * sizeof(double), X.p[q], nrhs * sizeof(double),
                            nrhs * sizeof(double), n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        st = set_error(DDG_ECUDA, nm + ": copy-back");
  ddg::ws_free(ws, s);
  return st;
}

}  // namespace ddg

extern "C" {

ddg_status dd_getrf(int64_t n, dd_mat A, int64_t* ipiv, int32_t K, int32_t pivot, const ddg_opts* opts,
                    int64_t* info, void* stream) {
  const ddg::mat M{{A.hi, A.lo, nullptr, nullptr}, A.ld};
  return ddg::getrf_impl<2>("dd_getrf", n, M, ipiv, K, pivot, opts, info, stream);
}

ddg_status dd_getrs(int64_t n, int64_t nrhs, dd_mat LU, const int64_t* ipiv, dd_mat B, void* stream) {
  const ddg::mat L{{LU.hi, LU.lo, nullptr, nullptr}, LU.ld};
  const ddg::mat Bm{{B.hi, B.lo, nullptr, nullptr}, B.ld};
  return ddg::getrs_impl<2>("dd_getrs", n, nrhs, L, ipiv, Bm, stream);
}

ddg_status qd_getrf(int64_t n, qd_mat A, int64_t* ipiv, int32_t K, int32_t pivot, const ddg_opts* opts,
                    int64_t* info, void* stream) {
  const ddg::mat M{{A.x[0], A.x[1], A.x[2], A.x[3]}, A.ld};
  return ddg::getrf_impl<4>("qd_getrf", n, M, ipiv, K, pivot, opts, info, stream);
}

ddg_status qd_getrs(int64_t n, int64_t nrhs, qd_mat LU, const int64_t* ipiv, qd_mat B, void* stream) {
  const ddg::mat L{{LU.x[0], LU.x[1], LU.x[2], LU.x[3]}, LU.ld};
  const ddg::mat Bm{{B.x[0], B.x[1], B.x[2], B.x[3]}, B.ld};
  return ddg::getrs_impl<4>("qd_getrs", n, nrhs, L, ipiv, Bm, stream);
}

}  // extern "C"
