// DD LU decomposition and solve (Kouya 2015, Section 4): the blocked
// right-looking LU whose trailing update A22 := A22 - L21 U12 (step 3, the
// underlined product) is a DD matrix product, here dd_gemm with mode SUB and
// the caller's algorithm (Winograd by default), and the solution of A x = b
// (Eq. 2) by forward and back substitution.
//
// Steps per block column of width K (the paper's K = alpha n_min):
//   1. panel: for each column j of the block, pivot search (the first row of
//      largest |a_ij| compared as DD; skipped in the paper's no-pivot mode),
//      swap of the two whole rows, DD quotients l_ij = a_ij / a_jj and the
//      rank-1 update of the next columns. One single-CTA launch (pivot +
//      swap) and one grid launch (quotients + update + partial arg-max of
//      the next column) per column. Wide block columns are factored
//      recursively in halves (left half, triangular solve and Block update of
//      the right half, right half), so the rank-1 updates in pinned DD
//      arithmetic stay within 16 columns.
//   2. U12 := L11^-1 A12 by a recursive triangular solve whose off-diagonal
//      updates are Block products (base case: 8-row triangles in one kernel,
//      one thread per right-hand column: a GB300 SM issues FP64 slowly, so
//      the per-thread chain of DD operations is kept short).
//   3. A22 := A22 - L21 U12 through the matrix product.
// The loop runs while columns remain; the last block has min(K, remaining)
// columns (the paper's garbled loop end, read as "until no columns remain").
#include <algorithm>
#include <functional>
#include <string>

#include "arith.cuh"
#include "kernels.cuh"

namespace ddg {

namespace {

constexpr int RB = 32;       // rows per CTA in the column kernels
constexpr int TB = 8;        // triangle size of the substitution base case
constexpr int KMAX = 512;    // widest block column
constexpr int PANEL_BASE = 16;  // widest panel factored column by column

struct partial_t {
  double hi, lo;
  int64_t idx;
};

__device__ __forceinline__ dd_t ldA(const mat& A, int64_t i, int64_t j) {
  return dd_t{A.p[0][i * A.ld + j], A.p[1][i * A.ld + j]};
}
__device__ __forceinline__ void stA(const mat& A, int64_t i, int64_t j, dd_t v) {
  A.p[0][i * A.ld + j] = v.hi;
  A.p[1][i * A.ld + j] = v.lo;
}

// Is candidate (v, i) a better pivot than (w, k): larger |x|, ties to the
// smaller row index.
__device__ __forceinline__ bool better(dd_t v, int64_t i, dd_t w, int64_t k) {
  if (dd_abs_greater(v, w)) return true;
  if (dd_abs_greater(w, v)) return false;
  return i < k;
}

__device__ __forceinline__ void warp_argmax(dd_t& v, int64_t& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd_t w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    int64_t k = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(w, k, v, i)) {
      v = w;
      i = k;
    }
  }
}

}  // namespace

// Partial arg-max of column j over rows [r0, n): one warp per RB rows.
__global__ void __launch_bounds__(32) lu_argmax_kernel(int64_t n, mat A, int64_t j, int64_t r0,
                                                       partial_t* part) {
  const int64_t i = r0 + (int64_t)blockIdx.x * RB + threadIdx.x;
  dd_t v{0.0, 0.0};
  int64_t idx = INT64_MAX;
  if (i < n) {
    v = ldA(A, i, j);
    idx = i;
  }
  warp_argmax(v, idx);
  if (threadIdx.x == 0) part[blockIdx.x] = partial_t{v.hi, v.lo, idx};
}

// Pivot of column j: reduce the partial arg-maxes (or take row j), record
// it, flag an exactly zero pivot, and swap rows j and p across all columns.
__global__ void __launch_bounds__(256) lu_pivot_kernel(int64_t n, mat A, int64_t j, int64_t nparts,
                                                       const partial_t* part, int64_t* ipiv,
                                                       int64_t* info, int pivot) {
  __shared__ dd_t sv[8];
  __shared__ int64_t si[8];
  __shared__ int64_t sp;
  const int tid = threadIdx.x;
  if (pivot) {
    dd_t v{0.0, 0.0};
    int64_t idx = INT64_MAX;
    for (int64_t t = tid; t < nparts; t += blockDim.x) {
      const partial_t q = part[t];
      const dd_t w{q.hi, q.lo};
      if (better(w, q.idx, v, idx)) {
        v = w;
        idx = q.idx;
      }
    }
    warp_argmax(v, idx);
    if ((tid & 31) == 0) {
      sv[tid >> 5] = v;
      si[tid >> 5] = idx;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (better(sv[w], si[w], v, idx)) {
          v = sv[w];
          idx = si[w];
        }
      sp = (idx >= j && idx < n) ? idx : j;
    }
  } else if (tid == 0) {
    sp = j;
  }
  __syncthreads();
  const int64_t p = sp;
  if (tid == 0) {
    ipiv[j] = p;
    const dd_t d = ldA(A, p, j);
    if (d.hi == 0.0 && d.lo == 0.0 && *info == 0) *info = j + 1;
  }
  if (p != j) {
    for (int64_t c = tid; c < n; c += blockDim.x)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        double* rj = A.p[q] + j * A.ld + c;
        double* rp = A.p[q] + p * A.ld + c;
        const double t = *rj;
        *rj = *rp;
        *rp = t;
      }
  }
}

// Quotients l_ij = a_ij / a_jj for rows below j, rank-1 update of columns
// (j, pe) of those rows, and (optionally) the partial arg-max of column j+1.
__global__ void __launch_bounds__(256) lu_update_kernel(int64_t n, mat A, int64_t j, int64_t pe,
                                                        partial_t* part, int want_argmax) {
  __shared__ dd_t u[KMAX];
  __shared__ dd_t lq[RB];
  const int tid = threadIdx.x;
  const int64_t r0 = j + 1 + (int64_t)blockIdx.x * RB;
  const int rows = (int)(n - r0 < RB ? n - r0 : RB);
  const int cols = (int)(pe - j - 1);
  const dd_t piv = ldA(A, j, j);
  const bool zero = piv.hi == 0.0 && piv.lo == 0.0;
  if (tid < rows) {
    dd_t l{0.0, 0.0};
    if (!zero) {
      l = dd_div(ldA(A, r0 + tid, j), piv);
      stA(A, r0 + tid, j, l);
    }
    lq[tid] = l;
  }
  for (int c = tid; c < cols; c += blockDim.x) u[c] = ldA(A, j, j + 1 + c);
  __syncthreads();
  for (int e = tid; e < rows * cols; e += blockDim.x) {
    const int r = e / cols, c = e % cols;
    const int64_t i = r0 + r, jc = j + 1 + c;
    stA(A, i, jc, dd_add(ldA(A, i, jc), dd_mul(dd_neg(lq[r]), u[c])));
  }
  if (want_argmax) {
    __syncthreads();
    if (tid < 32) {
      dd_t v{0.0, 0.0};
      int64_t idx = INT64_MAX;
      if (tid < rows) {
        v = ldA(A, r0 + tid, j + 1);
        idx = r0 + tid;
      }
      warp_argmax(v, idx);
      if (tid == 0) part[blockIdx.x] = partial_t{v.hi, v.lo, idx};
    }
  }
}

// X := L^-1 X for a unit lower triangle L (m <= TB rows), one thread per
// column of X; the triangle is staged in shared memory.
__global__ void __launch_bounds__(128) trsm_lower_unit_base(int64_t m, int64_t r, mat Lm, mat X) {
  __shared__ dd_t T[TB][TB];
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int i = e / TB, k = e % TB;
    T[i][k] = (i < m && k < i) ? ldA(Lm, i, k) : dd_t{0.0, 0.0};
  }
  __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= r) return;
  dd_t x[TB];
#pragma unroll
  for (int i = 0; i < TB; ++i) {
    dd_t acc = i < m ? ldA(X, i, c) : dd_t{0.0, 0.0};
#pragma unroll
    for (int k = 0; k < i; ++k) acc = dd_add(acc, dd_mul(dd_neg(T[i][k]), x[k]));
    x[i] = acc;
    if (i < m) stA(X, i, c, acc);
  }
}

// X := U^-1 X for an upper triangle U with nonzero diagonal (m <= TB rows).
__global__ void __launch_bounds__(128) trsm_upper_base(int64_t m, int64_t r, mat U, mat X) {
  __shared__ dd_t T[TB][TB];
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int i = e / TB, k = e % TB;
    T[i][k] = (i < m && k < m && k >= i) ? ldA(U, i, k) : dd_t{i == k ? 1.0 : 0.0, 0.0};
  }
  __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= r) return;
  dd_t x[TB];
#pragma unroll
  for (int i = TB - 1; i >= 0; --i) {
    dd_t acc = i < m ? ldA(X, i, c) : dd_t{0.0, 0.0};
#pragma unroll
    for (int k = i + 1; k < TB; ++k) acc = dd_add(acc, dd_mul(dd_neg(T[i][k]), x[k]));
    x[i] = dd_div(acc, T[i][i]);
    if (i < m) stA(X, i, c, x[i]);
  }
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

__global__ void lu_gather_kernel(int64_t n, int64_t r, const int64_t* perm, mat B, mat X) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * r) return;
  const int64_t i = e / r, c = e % r;
  stA(X, i, c, ldA(B, perm[i], c));
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
static ddg_status trsm_lower_unit(int64_t m, int64_t r, const mat& Lm, const mat& X, cudaStream_t s) {
  if (m == 0 || r == 0) return DDG_OK;
  if (m <= TB) {
    trsm_lower_unit_base<<<(unsigned)((r + 127) / 128), 128, 0, s>>>(m, r, Lm, X);
    return counted(cudaGetLastError()) == cudaSuccess ? DDG_OK : set_error(DDG_ECUDA, "trsm launch");
  }
  const int64_t m1 = std::max<int64_t>(TB, (m / 2) / TB * TB);
  ddg_status st = trsm_lower_unit(m1, r, Lm, X, s);
  if (st != DDG_OK) return st;
  st = gemm_run(2, m - m1, m1, r, view(Lm, m1, 0), X, view(X, m1, 0), MODE_SUB, block_opts(), s);
  if (st != DDG_OK) return st;
  return trsm_lower_unit(m - m1, r, view(Lm, m1, m1), view(X, m1, 0), s);
}

// X := U^-1 X (U upper, m x m), X m x r.
static ddg_status trsm_upper(int64_t m, int64_t r, const mat& U, const mat& X, cudaStream_t s) {
  if (m == 0 || r == 0) return DDG_OK;
  if (m <= TB) {
    trsm_upper_base<<<(unsigned)((r + 127) / 128), 128, 0, s>>>(m, r, U, X);
    return counted(cudaGetLastError()) == cudaSuccess ? DDG_OK : set_error(DDG_ECUDA, "trsm launch");
  }
  const int64_t m1 = std::max<int64_t>(TB, (m / 2) / TB * TB);
  ddg_status st = trsm_upper(m - m1, r, view(U, m1, m1), view(X, m1, 0), s);
  if (st != DDG_OK) return st;
  st = gemm_run(2, m1, m - m1, r, view(U, 0, m1), view(X, m1, 0), X, MODE_SUB, block_opts(), s);
  if (st != DDG_OK) return st;
  return trsm_upper(m1, r, U, X, s);
}

static bool bad_dd(const dd_mat& M, int64_t rows, int64_t cols) {
  if (rows == 0 || cols == 0) return false;
  return !M.hi || !M.lo || M.ld < cols || M.ld < 1;
}

}  // namespace ddg

extern "C" {

ddg_status dd_getrf(int64_t n, dd_mat A, int64_t* ipiv, int32_t K, int32_t pivot, const ddg_opts* opts,
                    int64_t* info, void* stream) {
  using namespace ddg;
  clear_error();
  if (n < 0) return set_error(DDG_EINVAL, "negative size");
  if (K < 1 || K > KMAX) return set_error(DDG_EINVAL, "block size K must be in [1, 512]");
  if (pivot != 0 && pivot != 1) return set_error(DDG_EINVAL, "pivot must be 0 or 1");
  if (bad_dd(A, n, n)) return set_error(DDG_EINVAL, "A: null plane or ld < n");
  if (n > 0 && !ipiv) return set_error(DDG_EINVAL, "ipiv is null");
  ddg_opts o;
  ddg_opts_default(&o);
  if (opts) o = *opts;
  if (o.algo < DDG_SIMPLE || o.algo > DDG_WINOGRAD || o.cutoff < 1 || (o.accum != 0 && o.accum != 1) ||
      (o.pad != 0 && o.pad != 1) || (o.streams != 0 && o.streams != 1 && o.streams != 7))
    return set_error(DDG_EINVAL, "invalid options");
  if (n == 0) return DDG_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const mat M{{A.hi, A.lo, nullptr, nullptr}, A.ld};
  const int64_t maxparts = (n + RB - 1) / RB;
  const size_t bytes = sizeof(partial_t) * (size_t)maxparts + 256;
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return set_error(DDG_ENOMEM, "dd_getrf: scratch allocation failed");
  }
  partial_t* part = reinterpret_cast<partial_t*>(static_cast<char*>(ws) + 256);
  int64_t* dinfo = info ? info : reinterpret_cast<int64_t*>(ws);
  ddg_status st = DDG_OK;
  auto cu = [&](cudaError_t e) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (e != cudaSuccess && st == DDG_OK) st = set_error(DDG_ECUDA, std::string("dd_getrf: ") + cudaGetErrorString(e));
  };
  if (cudaMemsetAsync(dinfo, 0, sizeof(int64_t), s) != cudaSuccess) st = set_error(DDG_ECUDA, "memset");
  // Panel of columns [c0, c0 + w), rows [c0, n): per-column kernels for
  // narrow panels; wider ones split in halves (left half, its triangular
  // solve and Block update of the right half, then the right half), so the
  // rank-1 updates in pinned DD arithmetic stay within PANEL_BASE columns and
  // the rest of the panel work runs in the Block kernel.
  std::function<void(int64_t, int64_t)> panel = [&](int64_t c0, int64_t w) {
    if (st != DDG_OK || w <= 0) return;
    if (w <= PANEL_BASE) {
      const int64_t pe = c0 + w;
      for (int64_t j = c0; j < pe && st == DDG_OK; ++j) {
        const int64_t nparts = (n - j + RB - 1) / RB;
        if (pivot && j == c0) {
          lu_argmax_kernel<<<(unsigned)nparts, 32, 0, s>>>(n, M, j, j, part);
          cu(cudaGetLastError());
        }
        lu_pivot_kernel<<<1, 256, 0, s>>>(n, M, j, nparts, part, ipiv, dinfo, pivot);
        cu(cudaGetLastError());
        if (j + 1 < n) {
          const int64_t blocks = (n - j - 1 + RB - 1) / RB;
          lu_update_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, M, j, pe, part, (pivot && j + 1 < pe) ? 1 : 0);
          cu(cudaGetLastError());
        }
      }
      return;
    }
    const int64_t w1 = std::max<int64_t>(PANEL_BASE, (w / 2) / PANEL_BASE * PANEL_BASE);
    panel(c0, w1);
    if (st != DDG_OK) return;
    const int64_t w2 = w - w1, c1 = c0 + w1;
    st = trsm_lower_unit(w1, w2, view(M, c0, c0), view(M, c0, c1), s);
    if (st != DDG_OK) return;
    if (n - c1 > 0)
      st = gemm_run(2, n - c1, w1, w2, view(M, c1, c0), view(M, c0, c1), view(M, c1, c1), MODE_SUB,
                    block_opts(), s);
    if (st != DDG_OK) return;
    panel(c1, w2);
  };
  for (int64_t j0 = 0; j0 < n && st == DDG_OK; j0 += K) {
    const int64_t pe = std::min<int64_t>(n, j0 + K);
    panel(j0, pe - j0);
    if (st != DDG_OK || pe >= n) break;
    const int64_t kb = pe - j0, rest = n - pe;
    st = trsm_lower_unit(kb, rest, view(M, j0, j0), view(M, j0, pe), s);
    if (st != DDG_OK) break;
    // Section 4 step 3: A22 := A22 - L21 U12
    st = gemm_run(2, rest, kb, rest, view(M, pe, j0), view(M, j0, pe), view(M, pe, pe), MODE_SUB, o, s);
  }
  int64_t hinfo = 0;
  if (st == DDG_OK && !info) {
    if (cudaMemcpyAsync(&hinfo, dinfo, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = set_error(DDG_ECUDA, "dd_getrf: reading the pivot status");
  }
  cudaFreeAsync(ws, s);
  if (st == DDG_OK && hinfo != 0)
    return set_error(DDG_ESINGULAR, "dd_getrf: exactly zero pivot in column " + std::to_string(hinfo - 1));
  return st;
}

ddg_status dd_getrs(int64_t n, int64_t nrhs, dd_mat LU, const int64_t* ipiv, dd_mat B, void* stream) {
  using namespace ddg;
  clear_error();
  if (n < 0 || nrhs < 0) return set_error(DDG_EINVAL, "negative size");
  if (bad_dd(LU, n, n) || bad_dd(B, n, nrhs)) return set_error(DDG_EINVAL, "null plane or ld too small");
  if (n > 0 && !ipiv) return set_error(DDG_EINVAL, "ipiv is null");
  if (n == 0 || nrhs == 0) return DDG_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const mat L{{LU.hi, LU.lo, nullptr, nullptr}, LU.ld};
  const mat Bm{{B.hi, B.lo, nullptr, nullptr}, B.ld};
  const size_t plane = ((size_t)n * nrhs * sizeof(double) + 255) & ~(size_t)255;
  const size_t bytes = 2 * plane + (((size_t)n * sizeof(int64_t) + 255) & ~(size_t)255);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return set_error(DDG_ENOMEM, "dd_getrs: scratch allocation failed");
  }
  char* base = static_cast<char*>(ws);
  const mat X{{reinterpret_cast<double*>(base), reinterpret_cast<double*>(base + plane), nullptr, nullptr}, nrhs};
  int64_t* perm = reinterpret_cast<int64_t*>(base + 2 * plane);
  ddg_status st = DDG_OK;
  const size_t sm = n <= 12288 ? (size_t)n * sizeof(int32_t) : 0;
  lu_perm_kernel<<<1, 32, sm, s>>>(n, ipiv, perm);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    const int64_t tot = n * nrhs;
    lu_gather_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, nrhs, perm, Bm, X);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) st = set_error(DDG_ECUDA, std::string("dd_getrs: ") + cudaGetErrorString(e));
  if (st == DDG_OK) st = trsm_lower_unit(n, nrhs, L, X, s);
  if (st == DDG_OK) st = trsm_upper(n, nrhs, L, X, s);
  if (st == DDG_OK)
    for (int q = 0; q < 2 && st == DDG_OK; ++q)
      if (cudaMemcpy2DAsync(Bm.p[q], Bm.ld * sizeof(double), X.p[q], nrhs * sizeof(double),
                            nrhs * sizeof(double), n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        st = set_error(DDG_ECUDA, "dd_getrs: copy-back");
  cudaFreeAsync(ws, s);
  return st;
}

}  // extern "C"
