// C-ABI entry points dd_gemm / qd_gemm and the Strassen / Winograd recursion
// (Kouya 2015, Section 2 and Figs. 1-2; Section 3 for n_min).
//
// Recursion. A level splits A (m x l), B (l x n) and C into quadrants while
// min(m, l, n) > cutoff. One fused pass forms the left operands of the seven
// sub-products, one the right operands, the seven products recurse, and one
// fused pass combines them into C (passes.cu). The paper runs the seven
// sub-products of a level in seven OpenMP sections; here the seven products
// of the top level are forked onto seven CUDA streams (event fork/join on the
// caller's stream), and each stream runs its sub-tree depth-first, which keeps
// 7x more thread blocks in flight than one product alone when the recursion
// reaches small base cases.
//
// Odd sizes (the paper measures n = 1023 and 1025 but does not say how they
// are handled). Default: peel. The even leading part recurses; the last
// column of A / row of B (odd l) is added by a rank-1 Block product, the last
// column of C (odd n) and the last row (odd m) are Block products. Option
// pad = 1: copy A, B (and C) into zero-padded buffers whose sizes are
// multiples of 2^depth, recurse, copy the result back.
//
// Temporaries. Sizes are planned by a dry run of the same recursion, then one
// block is taken from the stream-ordered allocator. Each fork branch has a
// stack of its own: nodes below the top level run in stream order, so a
// node's temporaries are reused by its next sibling. Total for a square n:
// about 15 (n/2)^2 (1 + 7/3) DD/QD entries. Each stack also has one area for
// the converted operands of its Block base cases (they run in stream order
// too), sized by its largest base case.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "ddgemm.h"
#include "kernels.cuh"

namespace ddg {

std::atomic<uint64_t> g_launches{0};
static thread_local std::string g_err;

static ddg_status fail(ddg_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

void clear_error() { g_err.clear(); }
ddg_status set_error(ddg_status st, const std::string& msg) { return fail(st, msg); }

#define DDG_CUDA(x)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (x);                                                                \
    if (e_ != cudaSuccess) return fail(DDG_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define DDG_TRY(x)                       \
  do {                                   \
    ddg_status s_ = (x);                 \
    if (s_ != DDG_OK) return s_;         \
  } while (0)

// ------------------------------------------------------------ stream pool --
static constexpr int kMaxDev = 64;
static std::mutex g_pool_mu;
static bool g_pool_init[kMaxDev];
static cudaStream_t g_pool[kMaxDev][7];

static ddg_status stream_pool(cudaStream_t** out) {
  int dev = 0;
  DDG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return fail(DDG_ENOTSUP, "device index out of range");
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool_init[dev]) {
    for (int i = 0; i < 7; ++i)
      DDG_CUDA(cudaStreamCreateWithFlags(&g_pool[dev][i], cudaStreamNonBlocking));
    g_pool_init[dev] = true;
  }
  *out = g_pool[dev];
  return DDG_OK;
}

// ------------------------------------------------------------- recursion --
static inline size_t plane_bytes(int64_t rows, int64_t cols) {
  size_t b = (size_t)rows * (size_t)cols * sizeof(double);
  return (b + 255) & ~(size_t)255;
}

struct Ctx {
  int L = 2;
  int accum = 0;
  int algo = DDG_WINOGRAD;
  int cutoff = 512;
  int nstreams = 7;
  bool dry = true;
  char* base = nullptr;
  size_t region_off[8] = {0};
  size_t peak[8] = {0};
  // Block base cases with operands converted once (accum 0): their scratch
  // area per region (offset, size); off for accum 2 and the fixed scratch
  bool convert = true;
  size_t leaf_off[8] = {0};
  size_t leaf_peak[8] = {0};
  cudaStream_t* pool = nullptr;
  // While a fork branch is planned, its launches are collected here and
  // issued afterwards round-robin with the other branches' (see level()).
  std::vector<std::function<cudaError_t()>>* q = nullptr;
};

// Where launch_fx_convert puts an operand converted into buf: the word
// vectors first, then f, 256-byte aligned (its layout).
static fxop fxop_at(int L, char* buf, int64_t rows, int64_t cols) {
  const size_t words = ((size_t)rows * (size_t)cols * 16 * (L == 2 ? 1 : 2) + 255) & ~(size_t)255;
  return fxop{reinterpret_cast<const uint4*>(buf), reinterpret_cast<const int*>(buf + words), cols};
}

// Issue a launch now, or queue it for the branch being collected.
static cudaError_t issue(Ctx& c, std::function<cudaError_t()> fn) {
  if (c.q) {
    c.q->push_back(std::move(fn));
    return cudaSuccess;
  }
  return fn();
}

static mat alloc_mat(Ctx& c, int region, size_t& sp, int64_t rows, int64_t cols) {
  mat M{};
  M.ld = std::max<int64_t>(cols, 1);
  for (int q = 0; q < c.L; ++q) {
    if (!c.dry) M.p[q] = reinterpret_cast<double*>(c.base + c.region_off[region] + sp);
    sp += plane_bytes(rows, cols);
  }
  c.peak[region] = std::max(c.peak[region], sp);
  return M;
}

static ddg_status zero_mat(const Ctx& c, const mat& M, int64_t rows, int64_t cols, cudaStream_t s) {
  for (int q = 0; q < c.L; ++q)
    DDG_CUDA(cudaMemset2DAsync(M.p[q], M.ld * sizeof(double), 0, cols * sizeof(double), rows, s));
  return DDG_OK;
}

static ddg_status copy_mat(const Ctx& c, const mat& dst, const mat& src, int64_t rows, int64_t cols,
                           cudaStream_t s) {
  for (int q = 0; q < c.L; ++q)
    DDG_CUDA(cudaMemcpy2DAsync(dst.p[q], dst.ld * sizeof(double), src.p[q], src.ld * sizeof(double),
                               cols * sizeof(double), rows, cudaMemcpyDeviceToDevice, s));
  return DDG_OK;
}

// Is the base case m x l x n a Block product on operands converted once?
static bool converts(const Ctx& c, int64_t m, int64_t l, int64_t n) {
  return c.accum == 0 && c.convert && n > GEMV_MAX_N && block_fx_converts(c.L, m, l, n);
}

// The base case on stack `region`; a dry run only sizes its scratch.
static cudaError_t base_case(Ctx& c, int region, int64_t m, int64_t l, int64_t n, const mat& A,
                             const mat& B, const mat& C, int mode, cudaStream_t s) {
  const int L = c.L;
  if (c.accum == 1)
    return c.dry ? cudaSuccess : issue(c, [=] { return launch_block(L, m, l, n, A, B, C, mode, s); });
  if (n <= GEMV_MAX_N)
    return c.dry ? cudaSuccess : issue(c, [=] { return launch_gemv_fx(L, m, l, n, A, B, C, mode, s); });
  if (converts(c, m, l, n)) {
    if (c.dry) {
      c.leaf_peak[region] = std::max(c.leaf_peak[region], block_fx_scratch_bytes(c.L, m, l, n));
      return cudaSuccess;
    }
    char* scratch = c.base + c.leaf_off[region];
    return issue(c, [=] { return launch_block_fx_converted(L, m, l, n, A, B, C, mode, scratch, s); });
  }
  return c.dry ? cudaSuccess : issue(c, [=] { return launch_block_fx(L, m, l, n, A, B, C, mode, s); });
}

static bool splits(const Ctx& c, int64_t m, int64_t l, int64_t n) {
  if (c.algo != DDG_STRASSEN && c.algo != DDG_WINOGRAD) return false;
  const int64_t mn = std::min(m, std::min(l, n));
  return mn >= 2 && mn > c.cutoff;
}

static ddg_status rec(Ctx& c, int64_t m, int64_t l, int64_t n, const mat& A, const mat& B,
                      const mat& C, int mode, cudaStream_t s, int region, size_t sp, int depth);

// One recursion level on even m, l, n.
static ddg_status level(Ctx& c, int64_t m, int64_t l, int64_t n, const mat& A, const mat& B,
                        const mat& C, int mode, cudaStream_t s, int region, size_t sp, int depth) {
  const int64_t h = m / 2, k = l / 2, w = n / 2;
  const mat A11 = view(A, 0, 0), A12 = view(A, 0, k), A21 = view(A, h, 0), A22 = view(A, h, k);
  const mat B11 = view(B, 0, 0), B12 = view(B, 0, w), B21 = view(B, k, 0), B22 = view(B, k, w);
  const mat C11 = view(C, 0, 0), C12 = view(C, 0, w), C21 = view(C, h, 0), C22 = view(C, h, w);
  const bool win = c.algo == DDG_WINOGRAD;
  const int nl = win ? 4 : 5;  // left / right operand temporaries
  mat SL[5] = {}, SR[5] = {}, P[7] = {};
  for (int i = 0; i < nl; ++i) SL[i] = alloc_mat(c, region, sp, h, k);
  for (int i = 0; i < nl; ++i) SR[i] = alloc_mat(c, region, sp, k, w);
  for (int i = 0; i < 7; ++i) P[i] = alloc_mat(c, region, sp, h, w);

  const int L = c.L;
  if (!c.dry) {
    const mat qa[4] = {A11, A12, A21, A22};
    const mat qb[4] = {B11, B12, B21, B22};
    const mat sl[5] = {SL[0], SL[1], SL[2], SL[3], SL[4]}, sr[5] = {SR[0], SR[1], SR[2], SR[3], SR[4]};
    DDG_CUDA(issue(c, [=] {
      return launch_pass(L, win ? PASS_WINOGRAD_A : PASS_STRASSEN_A, h, k, qa, 4, sl, nl, MODE_SET, s);
    }));
    DDG_CUDA(issue(c, [=] {
      return launch_pass(L, win ? PASS_WINOGRAD_B : PASS_STRASSEN_B, k, w, qb, 4, sr, nl, MODE_SET, s);
    }));
  }
  // the seven sub-products
  mat lhs[7], rhs[7];
  if (win) {  // P1 = A11 B11, P2 = A12 B21, P3 = S4 B22, P4 = A22 T4, P5 = S1 T1, P6 = S2 T2, P7 = S3 T3
    const mat L_[7] = {A11, A12, SL[3], A22, SL[0], SL[1], SL[2]};
    const mat R_[7] = {B11, B21, B22, SR[3], SR[0], SR[1], SR[2]};
    for (int i = 0; i < 7; ++i) { lhs[i] = L_[i]; rhs[i] = R_[i]; }
  } else {  // M1..M7 of Strassen 1969
    const mat L_[7] = {SL[0], SL[1], A11, A22, SL[2], SL[3], SL[4]};
    const mat R_[7] = {SR[0], B11, SR[1], SR[2], B22, SR[3], SR[4]};
    for (int i = 0; i < 7; ++i) { lhs[i] = L_[i]; rhs[i] = R_[i]; }
  }
  // Children that are Block base cases on converted operands: their 14
  // operands are converted in one launch (into the stack's leaf area) and
  // the seven products, all of one shape, run as one launch on s. This keeps
  // each stream's queue short and fills the GPU even when one leaf product
  // alone has few tiles.
  if (!splits(c, h, k, w) && converts(c, h, k, w)) {
    const size_t bl = fxop_bytes(c.L, h, k), br = fxop_bytes(c.L, k, w);
    c.leaf_peak[region] = std::max(c.leaf_peak[region], 7 * (bl + br));
    if (!c.dry) {
      char* area = c.base + c.leaf_off[region];
      int64_t rows[14], cols[14];
      mat X[14];
      char* buf[14];
      fxop op[14];
      for (int i = 0; i < 7; ++i) {
        rows[i] = h, cols[i] = k, X[i] = lhs[i], buf[i] = area + i * bl;
        rows[7 + i] = k, cols[7 + i] = w, X[7 + i] = rhs[i], buf[7 + i] = area + 7 * bl + i * br;
      }
      for (int t = 0; t < 14; ++t) op[t] = fxop_at(L, buf[t], rows[t], cols[t]);
      struct node_args {
        int64_t rows[14], cols[14];
        mat X[14];
        char* buf[14];
        fxop op[14];
        mat P[7], qc[4];
      };
      auto na = std::make_shared<node_args>();
      std::copy(rows, rows + 14, na->rows);
      std::copy(cols, cols + 14, na->cols);
      std::copy(X, X + 14, na->X);
      std::copy(buf, buf + 14, na->buf);
      std::copy(op, op + 14, na->op);
      std::copy(P, P + 7, na->P);
      na->qc[0] = C11, na->qc[1] = C12, na->qc[2] = C21, na->qc[3] = C22;
      DDG_CUDA(issue(c, [=] {
        fxop out[14];
        return launch_fx_convert(L, 14, na->rows, na->cols, na->X, na->buf, out, s);
      }));
      DDG_CUDA(issue(c, [=] { return launch_block_fxc(L, h, k, w, &na->op[0], &na->op[7], na->P, 7, MODE_SET, s); }));
      DDG_CUDA(issue(c, [=] {
        return launch_pass(L, win ? PASS_WINOGRAD_C : PASS_STRASSEN_C, h, w, na->P, 7, na->qc, 4, mode, s);
      }));
    }
    return DDG_OK;
  }
  auto child = [&](int i, cudaStream_t cs, int reg, size_t rsp) -> ddg_status {
    return rec(c, h, k, w, lhs[i], rhs[i], P[i], MODE_SET, cs, reg, rsp, depth + 1);
  };
  const bool fork = depth == 0 && c.nstreams == 7;
  if (fork) {
    // Each branch's launches are collected first and then issued
    // round-robin over the seven streams: issued branch after branch, a deep
    // recursion fills one stream's queue and blocks the host before the
    // later branches have started.
    cudaEvent_t ev_fork = nullptr, ev_join[7] = {nullptr};
    std::vector<std::function<cudaError_t()>> branch[7];
    if (!c.dry) {
      DDG_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
      DDG_CUDA(cudaEventRecord(ev_fork, s));
    }
    for (int i = 0; i < 7; ++i) {
      cudaStream_t cs = c.dry ? s : c.pool[i];
      if (!c.dry) DDG_CUDA(cudaStreamWaitEvent(cs, ev_fork, 0));
      c.q = c.dry ? nullptr : &branch[i];
      const ddg_status st = child(i, cs, 1 + i, 0);
      c.q = nullptr;
      DDG_TRY(st);
    }
    if (!c.dry) {
      size_t most = 0;
      for (int i = 0; i < 7; ++i) most = std::max(most, branch[i].size());
      for (size_t j = 0; j < most; ++j)
        for (int i = 0; i < 7; ++i)
          if (j < branch[i].size()) DDG_CUDA(branch[i][j]());
    }
    for (int i = 0; i < 7; ++i) {
      if (!c.dry) {
        DDG_CUDA(cudaEventCreateWithFlags(&ev_join[i], cudaEventDisableTiming));
        DDG_CUDA(cudaEventRecord(ev_join[i], c.pool[i]));
        DDG_CUDA(cudaStreamWaitEvent(s, ev_join[i], 0));
      }
    }
    if (!c.dry) {
      DDG_CUDA(cudaEventDestroy(ev_fork));
      for (int i = 0; i < 7; ++i) DDG_CUDA(cudaEventDestroy(ev_join[i]));
    }
  } else {
    for (int i = 0; i < 7; ++i) DDG_TRY(child(i, s, region, sp));
  }
  if (!c.dry) {
    const mat qc[4] = {C11, C12, C21, C22};
    const mat pp[7] = {P[0], P[1], P[2], P[3], P[4], P[5], P[6]};
    DDG_CUDA(issue(c, [=] {
      return launch_pass(L, win ? PASS_WINOGRAD_C : PASS_STRASSEN_C, h, w, pp, 7, qc, 4, mode, s);
    }));
  }
  return DDG_OK;
}

static ddg_status rec(Ctx& c, int64_t m, int64_t l, int64_t n, const mat& A, const mat& B,
                      const mat& C, int mode, cudaStream_t s, int region, size_t sp, int depth) {
  if (m == 0 || n == 0) return DDG_OK;
  if (l == 0) return (mode == MODE_SET && !c.dry) ? zero_mat(c, C, m, n, s) : DDG_OK;
  if (!splits(c, m, l, n)) {
    DDG_CUDA(base_case(c, region, m, l, n, A, B, C, mode, s));
    return DDG_OK;
  }
  const int64_t m2 = m & ~int64_t(1), l2 = l & ~int64_t(1), n2 = n & ~int64_t(1);
  if (!c.dry) nvtxRangePushA(depth == 0 ? "ddg.level 0" : depth == 1 ? "ddg.level 1" : depth == 2 ? "ddg.level 2"
                                                        : depth == 3 ? "ddg.level 3" : "ddg.level 4+");
  const ddg_status lst = level(c, m2, l2, n2, A, B, C, mode, s, region, sp, depth);
  if (!c.dry) nvtxRangePop();
  DDG_TRY(lst);
  if (l2 != l)  // C[:m2, :n2] (+/-)= A[:m2, l2] B[l2, :n2]
    DDG_CUDA(base_case(c, region, m2, 1, n2, view(A, 0, l2), view(B, l2, 0), C,
                       mode == MODE_SUB ? MODE_SUB : MODE_ADD, s));
  if (n2 != n)
    DDG_CUDA(base_case(c, region, m2, l, 1, A, view(B, 0, n2), view(C, 0, n2), mode, s));
  if (m2 != m)
    DDG_CUDA(base_case(c, region, 1, l, n, view(A, m2, 0), B, view(C, m2, 0), mode, s));
  return DDG_OK;
}

// Top level: optional padding around the recursion.
static ddg_status top(Ctx& c, int64_t m, int64_t l, int64_t n, const mat& A, const mat& B,
                      const mat& C, int mode, bool pad, cudaStream_t s) {
  if (!pad || !splits(c, m, l, n)) return rec(c, m, l, n, A, B, C, mode, s, 0, 0, 0);
  int depth = 0;
  for (int64_t t = std::min(m, std::min(l, n)); t >= 2 && t > c.cutoff; t = (t + 1) / 2) ++depth;
  const int64_t mult = int64_t(1) << depth;
  auto up = [&](int64_t x) { return (x + mult - 1) / mult * mult; };
  const int64_t mp = up(m), lp = up(l), np = up(n);
  if (mp == m && lp == l && np == n) return rec(c, m, l, n, A, B, C, mode, s, 0, 0, 0);
  size_t sp = 0;
  mat Ap = alloc_mat(c, 0, sp, mp, lp), Bp = alloc_mat(c, 0, sp, lp, np), Cp = alloc_mat(c, 0, sp, mp, np);
  if (!c.dry) {
    DDG_TRY(zero_mat(c, Ap, mp, lp, s));
    DDG_TRY(zero_mat(c, Bp, lp, np, s));
    DDG_TRY(copy_mat(c, Ap, A, m, l, s));
    DDG_TRY(copy_mat(c, Bp, B, l, n, s));
    if (mode != MODE_SET) DDG_TRY(copy_mat(c, Cp, C, m, n, s));
  }
  DDG_TRY(rec(c, mp, lp, np, Ap, Bp, Cp, mode, s, 0, sp, 0));
  if (!c.dry) DDG_TRY(copy_mat(c, C, Cp, m, n, s));
  return DDG_OK;
}

// ----------------------------------------------------------- validation --
static bool bad_mat(int L, const mat& M, int64_t rows, int64_t cols, const char* name,
                    std::string& why) {
  if (rows == 0 || cols == 0) return false;
  if (M.ld < cols || M.ld < 1) {
    why = std::string(name) + ": ld smaller than the column count";
    return true;
  }
  for (int q = 0; q < L; ++q)
    if (!M.p[q]) {
      why = std::string(name) + ": null limb plane";
      return true;
    }
  return false;
}

// Do the element sets of two strided regions X (xr x xc) and Y (yr x yc)
// share an address? Exact when both have the same leading dimension (views
// into one matrix, e.g. L21, U12 and A22 of an LU step); otherwise the
// conservative test on the address ranges.
static bool region_overlap(const double* x, int64_t xr, int64_t xc, int64_t xld, const double* y,
                           int64_t yr, int64_t yc, int64_t yld) {
  const char* x0 = reinterpret_cast<const char*>(x);
  const char* x1 = reinterpret_cast<const char*>(x + (xr - 1) * xld + xc);
  const char* y0 = reinterpret_cast<const char*>(y);
  const char* y1 = reinterpret_cast<const char*>(y + (yr - 1) * yld + yc);
  if (!(x0 < y1 && y0 < x1)) return false;
  const std::ptrdiff_t db = y0 - x0;
  if (xld != yld || db % (std::ptrdiff_t)sizeof(double) != 0) return true;
  int64_t d = db / (std::ptrdiff_t)sizeof(double);
  int64_t dr = d >= 0 ? d / xld : -((-d + xld - 1) / xld);
  int64_t dc = d - dr * xld;  // 0 <= dc < ld
  // Y's element (r, c) is X's (r + dr, c + dc) if c + dc < ld, else (r + dr + 1, c + dc - ld)
  auto rect = [&](int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
    return r0 < xr && 0 < r1 && c0 < xc && 0 < c1 && r0 < r1 && c0 < c1;
  };
  if (rect(dr, dr + yr, dc, std::min(dc + yc, xld))) return true;
  if (dc + yc > xld && rect(dr + 1, dr + 1 + yr, 0, dc + yc - xld)) return true;
  return false;
}

bool overlaps(int L, const mat& X, int64_t xr, int64_t xc, const mat& Y, int64_t yr, int64_t yc) {
  if (xr == 0 || xc == 0 || yr == 0 || yc == 0) return false;
  for (int p = 0; p < L; ++p)
    for (int q = 0; q < L; ++q)
      if (region_overlap(X.p[p], xr, xc, X.ld, Y.p[q], yr, yc, Y.ld)) return true;
  return false;
}

ddg_status gemm_run(int L, int64_t m, int64_t l, int64_t n, const mat& A, const mat& B, const mat& C,
                    int mode, const ddg_opts& o, cudaStream_t s);

static ddg_status gemm_entry(int L, int64_t m, int64_t l, int64_t n, const mat& A, const mat& B,
                             const mat& C, int mode, const ddg_opts* opts, void* stream) {
  g_err.clear();
  ddg_opts o;
  ddg_opts_default(&o);
  if (opts) o = *opts;
  if (m < 0 || l < 0 || n < 0) return fail(DDG_EINVAL, "negative size");
  if (mode < DDG_SET || mode > DDG_SUB) return fail(DDG_EINVAL, "mode must be DDG_SET, DDG_ADD or DDG_SUB");
  if (o.algo < DDG_SIMPLE || o.algo > DDG_OZAKI2_TC) return fail(DDG_EINVAL, "unknown algo");
  if (o.algo == DDG_OZAKI2 || o.algo == DDG_OZAKI2_TC ? (o.slices != 0 && (o.slices < 2 || o.slices > 40))
                           : (o.slices != 0 && (o.slices < 2 || o.slices > (L == 2 ? 18 : 32))))
    return fail(DDG_EINVAL, "slices must be 0 or in [2, 18] (DD) / [2, 32] (QD); moduli in [2, 40]");
  if (o.cutoff < 1) return fail(DDG_EINVAL, "cutoff must be >= 1");
  if (o.pad != 0 && o.pad != 1) return fail(DDG_EINVAL, "pad must be 0 or 1");
  if (o.streams != 0 && o.streams != 1 && o.streams != 7) return fail(DDG_EINVAL, "streams must be 0, 1 or 7");
  if (o.accum < 0 || o.accum > 2) return fail(DDG_EINVAL, "accum must be 0, 1 or 2");
  for (int i = 0; i < 2; ++i)
    if (o.reserved[i] != 0) return fail(DDG_EINVAL, "reserved option fields must be zero");
  std::string why;
  if (bad_mat(L, A, m, l, "A", why) || bad_mat(L, B, l, n, "B", why) || bad_mat(L, C, m, n, "C", why))
    return fail(DDG_EINVAL, why);
  if (overlaps(L, C, m, n, A, m, l) || overlaps(L, C, m, n, B, l, n))
    return fail(DDG_EINVAL, "C overlaps A or B");
  if (m > (int64_t)65535 * 8 || n > ((int64_t)1 << 36)) return fail(DDG_EINVAL, "matrix too large");
  return gemm_run(L, m, l, n, A, B, C, mode, o, reinterpret_cast<cudaStream_t>(stream));
}

ddg_status gemm_run(int L, int64_t m, int64_t l, int64_t n, const mat& A, const mat& B, const mat& C,
                    int mode, const ddg_opts& o, cudaStream_t s) {
  if (m == 0 || n == 0) return DDG_OK;
  nvtx_range nv("ddg.gemm L%d algo %d %lldx%lldx%lld", L, o.algo, (long long)m, (long long)l, (long long)n);

  if (o.algo == DDG_SIMPLE) {
    DDG_CUDA(launch_simple(L, m, l, n, A, B, C, mode, s));
    return DDG_OK;
  }
  if (o.algo == DDG_OZAKI) {
    if (m > 65535) return fail(DDG_EINVAL, "DDG_OZAKI: m must be <= 65535");
    if (l == 0) {
      Ctx z;
      z.L = L;
      return mode == MODE_SET ? zero_mat(z, C, m, n, s) : DDG_OK;
    }
    return ozaki_gemm(L, m, l, n, A, B, C, mode, o.slices ? o.slices : (L == 2 ? 16 : 32), s);
  }
  if (o.algo == DDG_OZAKI2 || o.algo == DDG_OZAKI2_TC) {
    if (L != 2) return fail(DDG_ENOTSUP, "DDG_OZAKI2: DD only (the moduli <= 256 give at most ~2^369)");
    if (m > 65535) return fail(DDG_EINVAL, "DDG_OZAKI2: m must be <= 65535");
    if (l == 0) {
      Ctx z;
      z.L = L;
      return mode == MODE_SET ? zero_mat(z, C, m, n, s) : DDG_OK;
    }
    return ozaki_crt_gemm(m, l, n, A, B, C, mode, o.slices ? o.slices : 32, o.algo == DDG_OZAKI2_TC, s);
  }
  Ctx c;
  c.L = L;
  c.accum = o.accum;
  c.algo = o.algo;
  c.cutoff = o.cutoff;
  c.nstreams = o.streams == 1 ? 1 : 7;
  if (splits(c, m, l, n) && c.nstreams == 7) DDG_TRY(stream_pool(&c.pool));
  // plan (a Block product alone plans its converted operands only); if the
  // workspace with converted operands cannot be had, plan again with tiles
  // converted as they are staged (the same bits, less workspace)
  void* ws = nullptr;
  size_t total = 0;
  for (;;) {
    c.dry = true;
    for (int r = 0; r < 8; ++r) c.peak[r] = c.leaf_peak[r] = 0;
    DDG_TRY(top(c, m, l, n, A, B, C, mode, o.pad == 1, s));
    total = 0;
    bool converted = false;
    for (int r = 0; r < 8; ++r) {
      c.region_off[r] = total;
      total += (c.peak[r] + 255) & ~(size_t)255;
    }
    for (int r = 0; r < 8; ++r) {
      c.leaf_off[r] = total;
      total += (c.leaf_peak[r] + 255) & ~(size_t)255;
      converted = converted || c.leaf_peak[r] > 0;
    }
    if (!total) break;
    cudaError_t e = ddg::ws_alloc(&ws, total, s);
    if (e == cudaSuccess) break;
    cudaGetLastError();
    ws = nullptr;
    if (!converted)
      return fail(DDG_ENOMEM, "cudaMallocAsync of " + std::to_string(total) + " bytes: " + cudaGetErrorString(e));
    c.convert = false;
  }
  // run
  c.dry = false;
  c.base = static_cast<char*>(ws);
  ddg_status st = top(c, m, l, n, A, B, C, mode, o.pad == 1, s);
  if (ws) {
    cudaError_t e = ddg::ws_free(ws, s);
    if (st == DDG_OK && e != cudaSuccess) return fail(DDG_ECUDA, std::string("cudaFreeAsync: ") + cudaGetErrorString(e));
  }
  return st;
}

}  // namespace ddg

extern "C" {

void ddg_opts_default(ddg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->algo = DDG_WINOGRAD;
  o->cutoff = 512;
  o->pad = 0;
  o->streams = 7;
  o->accum = 0;
}

ddg_status dd_gemm(int64_t m, int64_t l, int64_t n, dd_mat A, dd_mat B, dd_mat C, int32_t mode,
                   const ddg_opts* opts, void* stream) {
  ddg::mat a{{A.hi, A.lo, nullptr, nullptr}, A.ld};
  ddg::mat b{{B.hi, B.lo, nullptr, nullptr}, B.ld};
  ddg::mat c{{C.hi, C.lo, nullptr, nullptr}, C.ld};
  return ddg::gemm_entry(2, m, l, n, a, b, c, mode, opts, stream);
}

ddg_status qd_gemm(int64_t m, int64_t l, int64_t n, qd_mat A, qd_mat B, qd_mat C, int32_t mode,
                   const ddg_opts* opts, void* stream) {
  ddg::mat a{{A.x[0], A.x[1], A.x[2], A.x[3]}, A.ld};
  ddg::mat b{{B.x[0], B.x[1], B.x[2], B.x[3]}, B.ld};
  ddg::mat c{{C.x[0], C.x[1], C.x[2], C.x[3]}, C.ld};
  return ddg::gemm_entry(4, m, l, n, a, b, c, mode, opts, stream);
}

int32_t ddg_block_fp64_ops_per_mac(int32_t limbs, int32_t accum) {
  if ((limbs != 2 && limbs != 4) || accum < 0 || accum > 2) return -1;
  return accum != 1 ? ddg::block_fx_fp64_ops_per_mac(limbs) : ddg::block_fp64_ops_per_mac(limbs);
}

int32_t ddg_ozaki2_precision(int32_t moduli, int64_t l) {
  if (moduli < 2 || moduli > 40 || l < 1) return -1;
  const int P = ddg::ozaki_crt_precision(moduli, l);
  return P >= 1 ? P : -1;
}

const char* ddg_last_error(void) { return ddg::g_err.c_str(); }

uint64_t ddg_kernel_launches(void) { return ddg::g_launches.load(std::memory_order_relaxed); }

ddg_status ddg_test_bounded_wait(int32_t which) {
  ddg::clear_error();
  if (which == 0) {
    const cudaError_t e = ddg::crt_tc_wait_test();
    if (e != cudaSuccess) return ddg::set_error(DDG_ECUDA, std::string("wait test: ") + cudaGetErrorString(e));
    return ddg::crt_tc_timeouts(false) > 0 ? ddg::set_error(DDG_ETIMEOUT, "tensor-core wait ran out (as intended)")
                                           : DDG_OK;
  }
  if (which == 1) return ddg::lu_panel_wait_test();
  return ddg::set_error(DDG_EINVAL, "ddg_test_bounded_wait: which must be 0 or 1");
}

int32_t ddg_device_timeouts(int32_t reset) {
  if (cudaDeviceSynchronize() != cudaSuccess) return -1;
  return ddg::crt_tc_timeouts(reset != 0);
}

}  // extern "C"

// ------------------------------------------------ allocation-free variant --
// dd_gemm_noalloc: the same Strassen / Winograd product as dd_gemm, for
// callers that must not allocate device memory at call time. Its recursion
// temporaries live in one fixed array compiled into this library, so every
// GPU that loads the library keeps kNoAllocScratchBytes reserved until the
// process exits. Host code cannot use the array's name as a device address;
// the address is looked up once per device with cudaGetSymbolAddress.
namespace ddg {

static constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kMaxDev];

// Device address of the fixed scratch on the current device (looked up on the
// first call per device, with that device current).
static ddg_status noalloc_scratch(void** out) {
  int dev = 0;
  DDG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return fail(DDG_ENOTSUP, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    DDG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return DDG_OK;
}

static ddg_status gemm_noalloc_entry(int64_t m, int64_t l, int64_t n, const mat& A, const mat& B,
                                     const mat& C, int mode, const ddg_opts* opts, void* stream) {
  g_err.clear();
  const int L = 2;
  ddg_opts o;
  ddg_opts_default(&o);
  if (opts) o = *opts;
  if (m < 0 || l < 0 || n < 0) return fail(DDG_EINVAL, "negative size");
  if (mode < DDG_SET || mode > DDG_SUB) return fail(DDG_EINVAL, "mode must be DDG_SET, DDG_ADD or DDG_SUB");
  if (o.algo < DDG_SIMPLE || o.algo > DDG_OZAKI2_TC) return fail(DDG_EINVAL, "unknown algo");
  if (o.algo == DDG_OZAKI2 || o.algo == DDG_OZAKI2_TC ? (o.slices != 0 && (o.slices < 2 || o.slices > 40))
                           : (o.slices != 0 && (o.slices < 2 || o.slices > (L == 2 ? 18 : 32))))
    return fail(DDG_EINVAL, "slices must be 0 or in [2, 18] (DD) / [2, 32] (QD); moduli in [2, 40]");
  if (o.cutoff < 1) return fail(DDG_EINVAL, "cutoff must be >= 1");
  if (o.pad != 0 && o.pad != 1) return fail(DDG_EINVAL, "pad must be 0 or 1");
  if (o.accum < 0 || o.accum > 2) return fail(DDG_EINVAL, "accum must be 0, 1 or 2");
  for (int i = 0; i < 2; ++i)
    if (o.reserved[i] != 0) return fail(DDG_EINVAL, "reserved option fields must be zero");
  std::string why;
  if (bad_mat(L, A, m, l, "A", why) || bad_mat(L, B, l, n, "B", why) || bad_mat(L, C, m, n, "C", why))
    return fail(DDG_EINVAL, why);
  if (overlaps(L, C, m, n, A, m, l) || overlaps(L, C, m, n, B, l, n))
    return fail(DDG_EINVAL, "C overlaps A or B");
  if (m > (int64_t)65535 * 8 || n > ((int64_t)1 << 36)) return fail(DDG_EINVAL, "matrix too large");
  if (o.algo == DDG_OZAKI || o.algo == DDG_OZAKI2 || o.algo == DDG_OZAKI2_TC)
    return fail(DDG_EINVAL, "dd_gemm_noalloc: the INT8 / BF16 residue products need a workspace; use dd_gemm");
  if (m == 0 || n == 0) return DDG_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (o.algo == DDG_SIMPLE) {
    DDG_CUDA(launch_simple(L, m, l, n, A, B, C, mode, s));
    return DDG_OK;
  }
  Ctx c;
  c.L = L;
  c.accum = o.accum;
  c.algo = o.algo;
  c.cutoff = o.cutoff;
  c.nstreams = 1;     // no forking: no streams or events are created
  c.convert = false;  // Block base cases convert their tiles on the fly
  if (!splits(c, m, l, n)) {
    if (l == 0) return mode == MODE_SET ? zero_mat(c, C, m, n, s) : DDG_OK;
    c.dry = false;
    DDG_CUDA(base_case(c, 0, m, l, n, A, B, C, mode, s));
    return DDG_OK;
  }
  c.dry = true;
  DDG_TRY(top(c, m, l, n, A, B, C, mode, o.pad == 1, s));
  size_t total = 0;
  for (int r = 0; r < 8; ++r) {
    c.region_off[r] = total;
    total += (c.peak[r] + 255) & ~(size_t)255;
  }
  if (total > kNoAllocScratchBytes)
    return fail(DDG_EINVAL, "dd_gemm_noalloc: this product needs " + std::to_string(total) +
                                " bytes of scratch; the fixed scratch holds " +
                                std::to_string(kNoAllocScratchBytes) +
                                " (use dd_gemm, a larger cutoff, or a smaller problem)");
  void* base = nullptr;
  DDG_TRY(noalloc_scratch(&base));
  c.dry = false;
  c.base = static_cast<char*>(base);
  // Every temporary is written in full before it is read (operand passes,
  // Block products in set mode, memset of padding), so stale contents of the
  // shared scratch never reach a result.
  return top(c, m, l, n, A, B, C, mode, o.pad == 1, s);
}

}  // namespace ddg

extern "C" ddg_status dd_gemm_noalloc(int64_t m, int64_t l, int64_t n, dd_mat A, dd_mat B, dd_mat C,
                                      int32_t mode, const ddg_opts* opts, void* stream) {
  ddg::mat a{{A.hi, A.lo, nullptr, nullptr}, A.ld};
  ddg::mat b{{B.hi, B.lo, nullptr, nullptr}, B.ld};
  ddg::mat c{{C.hi, C.lo, nullptr, nullptr}, C.ld};
  return ddg::gemm_noalloc_entry(m, l, n, a, b, c, mode, opts, stream);
}
