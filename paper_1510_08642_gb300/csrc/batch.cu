// Batched DD/QD products: many independent, uneven C (mode) A B problems as
// a handful of grouped persistent launches (the Block base case of Kouya
// 2015, Section 2, and its Strassen / Winograd recursion, applied to a whole
// batch at once).
//
// A batch plan expands every problem's recursion breadth-first:
//   pre[d]   fused operand passes of all nodes at depth d (top-down),
//   leaves   every base-case Block product of every problem, plus the border
//            products of peeled odd rows / columns (they touch disjoint parts
//            of C), in one grouped launch per limb count: the products with
//            enough tiles (block_fx_converts) after one grouped launch that
//            converts all their operands to fixed-point words, the others
//            converting tiles as they are staged (the same bits either way),
//   post[d]  fused combination passes at depth d (bottom-up), each followed
//            by the rank-1 fix-ups of odd inner dimensions at that depth.
// Passes of the same depth, kind and limb count share one grouped launch.
// All temporaries and the device task lists are allocated once when the plan
// is created, so running a plan allocates nothing; the run can be captured
// into a CUDA graph and replayed (use_graph = 1).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ddgemm.h"
#include "kernels.cuh"

namespace ddg {

namespace {

struct Launch {
  int type;  // 0 pass, 1 grouped Block, 2 grouped conversion, 3 grouped Block on converted operands,
            // 4 grouped Block of DD and QD tasks together (one leaf launch)
  int limbs;
  int kind;
  size_t task_off;  // byte offset of the task array in the plan's buffer
  int ntasks;
  int64_t total;
  size_t counter_off;
  double ops;  // multiply-adds (grouped Block launches) or converted elements
};

struct Builder {
  bool dry = true;
  char* base = nullptr;
  size_t off = 0;  // temporaries
  // (depth, limbs, kind) -> tasks
  std::map<std::tuple<int, int, int>, std::vector<ptask>> pre, post;
  std::map<std::tuple<int, int>, std::vector<gtask>> fix;  // (depth, limbs)
  std::vector<gtask> leaves[5];
  int maxdepth = 0;
  double leaf_macs = 0.0;

  mat alloc(int L, int64_t rows, int64_t cols) {
    mat M{};
    M.ld = std::max<int64_t>(cols, 1);
    const size_t bytes = (((size_t)rows * (size_t)cols * sizeof(double)) + 255) & ~(size_t)255;
    for (int q = 0; q < L; ++q) {
      if (!dry) M.p[q] = reinterpret_cast<double*>(base + off);
      off += bytes;
    }
    return M;
  }
};

bool splits_b(int algo, int cutoff, int64_t m, int64_t l, int64_t n) {
  if (algo != DDG_STRASSEN && algo != DDG_WINOGRAD) return false;
  const int64_t mn = std::min(m, std::min(l, n));
  return mn >= 2 && mn > cutoff;
}

gtask leaf(int64_t m, int64_t l, int64_t n, const mat& A, const mat& B, const mat& C, int mode) {
  gtask t{};
  t.m = m;
  t.l = l;
  t.n = n;
  t.A = A;
  t.B = B;
  t.C = C;
  t.mode = mode;
  return t;
}

ptask pass(int64_t rows, int64_t cols, const mat* in, int nin, const mat* out, int nout, int mode) {
  ptask t{};
  t.rows = rows;
  t.cols = cols;
  for (int q = 0; q < nin; ++q) t.a.in[q] = in[q];
  for (int q = 0; q < nout; ++q) t.a.out[q] = out[q];
  t.mode = mode;
  return t;
}

void expand(Builder& b, int L, int algo, int cutoff, int64_t m, int64_t l, int64_t n, const mat& A,
            const mat& B, const mat& C, int mode, int depth) {
  if (m == 0 || n == 0) return;
  b.maxdepth = std::max(b.maxdepth, depth);
  if (!splits_b(algo, cutoff, m, l, n)) {
    b.leaves[L].push_back(leaf(m, l, n, A, B, C, mode));
    b.leaf_macs += (double)m * l * n;
    return;
  }
  const int64_t m2 = m & ~int64_t(1), l2 = l & ~int64_t(1), n2 = n & ~int64_t(1);
  if (n2 != n) b.leaves[L].push_back(leaf(m2, l, 1, A, view(B, 0, n2), view(C, 0, n2), mode));
  if (m2 != m) b.leaves[L].push_back(leaf(1, l, n, view(A, m2, 0), B, view(C, m2, 0), mode));
  if (l2 != l)
    b.fix[{depth, L}].push_back(
        leaf(m2, 1, n2, view(A, 0, l2), view(B, l2, 0), C, mode == MODE_SUB ? MODE_SUB : MODE_ADD));
  const int64_t h = m2 / 2, k = l2 / 2, w = n2 / 2;
  const mat A11 = view(A, 0, 0), A12 = view(A, 0, k), A21 = view(A, h, 0), A22 = view(A, h, k);
  const mat B11 = view(B, 0, 0), B12 = view(B, 0, w), B21 = view(B, k, 0), B22 = view(B, k, w);
  const mat C11 = view(C, 0, 0), C12 = view(C, 0, w), C21 = view(C, h, 0), C22 = view(C, h, w);
  const bool win = algo == DDG_WINOGRAD;
  const int nl = win ? 4 : 5;
  mat SL[5], SR[5], P[7];
  for (int i = 0; i < nl; ++i) SL[i] = b.alloc(L, h, k);
  for (int i = 0; i < nl; ++i) SR[i] = b.alloc(L, k, w);
  for (int i = 0; i < 7; ++i) P[i] = b.alloc(L, h, w);
  const mat qa[4] = {A11, A12, A21, A22};
  const mat qb[4] = {B11, B12, B21, B22};
  const mat qc[4] = {C11, C12, C21, C22};
  const int ka = win ? PASS_WINOGRAD_A : PASS_STRASSEN_A;
  const int kb = win ? PASS_WINOGRAD_B : PASS_STRASSEN_B;
  const int kc = win ? PASS_WINOGRAD_C : PASS_STRASSEN_C;
  b.pre[{depth, L, ka}].push_back(pass(h, k, qa, 4, SL, nl, MODE_SET));
  b.pre[{depth, L, kb}].push_back(pass(k, w, qb, 4, SR, nl, MODE_SET));
  if (win) {
    const mat Lh[7] = {A11, A12, SL[3], A22, SL[0], SL[1], SL[2]};
    const mat Rh[7] = {B11, B21, B22, SR[3], SR[0], SR[1], SR[2]};
    for (int i = 0; i < 7; ++i) expand(b, L, algo, cutoff, h, k, w, Lh[i], Rh[i], P[i], MODE_SET, depth + 1);
  } else {
    const mat Lh[7] = {SL[0], SL[1], A11, A22, SL[2], SL[3], SL[4]};
    const mat Rh[7] = {SR[0], B11, SR[1], SR[2], B22, SR[3], SR[4]};
    for (int i = 0; i < 7; ++i) expand(b, L, algo, cutoff, h, k, w, Lh[i], Rh[i], P[i], MODE_SET, depth + 1);
  }
  b.post[{depth, L, kc}].push_back(pass(h, w, P, 7, qc, 4, mode));
}

}  // namespace

}  // namespace ddg

struct ddg_batch_s {
  int dev = 0;
  char* buf = nullptr;
  size_t bytes = 0;
  std::vector<ddg::Launch> launches;
  int use_graph = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels_per_run = 0;
  cudaStream_t create_stream = nullptr;
  ddg_batch_stats stats{};
};

namespace ddg {

static ddg_status enqueue(ddg_batch_s* b, cudaStream_t s) {
  for (const Launch& L : b->launches) {
    cudaError_t e;
    if (L.type == 0)
      e = launch_grouped_pass(L.limbs, L.kind, reinterpret_cast<const ptask*>(b->buf + L.task_off), L.ntasks,
                              L.total, s);
    else if (L.type == 1)
      e = launch_grouped_fx(L.limbs, reinterpret_cast<const gtask*>(b->buf + L.task_off), L.ntasks, L.total,
                            reinterpret_cast<unsigned long long*>(b->buf + L.counter_off), L.ops, s);
    else if (L.type == 2)
      e = launch_grouped_convert(L.limbs, reinterpret_cast<const fx_ctask*>(b->buf + L.task_off), L.ntasks,
                                 L.total, L.ops, s);
    else if (L.type == 4)
      e = launch_grouped_mixed(reinterpret_cast<const gtask*>(b->buf + L.task_off), L.ntasks, L.total,
                               reinterpret_cast<unsigned long long*>(b->buf + L.counter_off), L.ops, s);
    else
      e = launch_grouped_fxc(L.limbs, reinterpret_cast<const gctask*>(b->buf + L.task_off), L.ntasks, L.total,
                             reinterpret_cast<unsigned long long*>(b->buf + L.counter_off), L.ops, s);
    if (e != cudaSuccess) return set_error(DDG_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  }
  return DDG_OK;
}

// Do the limb planes of X (xr x xc) and Y (yr x yc) share an element?
// (gemm.cu: exact for views with one leading dimension, else conservative.)
bool overlaps(int L, const mat& X, int64_t xr, int64_t xc, const mat& Y, int64_t yr, int64_t yc);

static bool bad_problem(const ddg_problem& p, std::string& why) {
  const int L = p.limbs;
  if (L != 2 && L != 4) { why = "limbs must be 2 or 4"; return true; }
  if (p.m < 0 || p.l < 0 || p.n < 0) { why = "negative size"; return true; }
  if (p.mode < DDG_SET || p.mode > DDG_SUB) { why = "bad mode"; return true; }
  if (p.algo != DDG_BLOCK && p.algo != DDG_STRASSEN && p.algo != DDG_WINOGRAD) {
    why = "batched algo must be DDG_BLOCK, DDG_STRASSEN or DDG_WINOGRAD";
    return true;
  }
  if (p.cutoff < 1) { why = "cutoff must be >= 1"; return true; }
  auto bad = [&](double* const* x, int64_t ld, int64_t r, int64_t c, const char* nm) {
    if (r == 0 || c == 0) return false;
    if (ld < c || ld < 1) { why = std::string(nm) + ": ld too small"; return true; }
    for (int q = 0; q < L; ++q)
      if (!x[q]) { why = std::string(nm) + ": null plane"; return true; }
    return false;
  };
  if (bad(p.A, p.lda, p.m, p.l, "A") || bad(p.B, p.ldb, p.l, p.n, "B") || bad(p.C, p.ldc, p.m, p.n, "C"))
    return true;
  auto planes = [&](double* const* x, int64_t ld) {
    return mat{{x[0], x[1], L == 4 ? x[2] : nullptr, L == 4 ? x[3] : nullptr}, ld};
  };
  const mat A = planes(p.A, p.lda), B = planes(p.B, p.ldb), C = planes(p.C, p.ldc);
  if (overlaps(L, C, p.m, p.n, A, p.m, p.l) || overlaps(L, C, p.m, p.n, B, p.l, p.n)) {
    why = "C overlaps A or B";
    return true;
  }
  return false;
}

}  // namespace ddg

extern "C" {

ddg_status ddg_batch_create(ddg_batch* out, int32_t count, const ddg_problem* probs, int32_t use_graph,
                            void* stream) {
  return ddg_batch_create_ex(out, count, probs, use_graph, 0, stream);
}

ddg_status ddg_batch_create_ex(ddg_batch* out, int32_t count, const ddg_problem* probs, int32_t use_graph,
                               int32_t flags, void* stream) {
  using namespace ddg;
  clear_error();
  if (!out) return set_error(DDG_EINVAL, "out is null");
  *out = nullptr;
  if (count < 0 || (count > 0 && !probs)) return set_error(DDG_EINVAL, "bad problem list");
  if (use_graph != 0 && use_graph != 1) return set_error(DDG_EINVAL, "use_graph must be 0 or 1");
  if (flags & ~DDG_BATCH_ONE_LEAF_LAUNCH) return set_error(DDG_EINVAL, "unknown batch flags");
  const bool one_leaf = (flags & DDG_BATCH_ONE_LEAF_LAUNCH) != 0;
  for (int32_t i = 0; i < count; ++i) {
    std::string why;
    if (bad_problem(probs[i], why)) return set_error(DDG_EINVAL, "problem " + std::to_string(i) + ": " + why);
  }
  auto build = [&](Builder& bld) {
    for (int32_t i = 0; i < count; ++i) {
      const ddg_problem& p = probs[i];
      const mat A{{p.A[0], p.A[1], p.limbs == 4 ? p.A[2] : nullptr, p.limbs == 4 ? p.A[3] : nullptr}, p.lda};
      const mat B{{p.B[0], p.B[1], p.limbs == 4 ? p.B[2] : nullptr, p.limbs == 4 ? p.B[3] : nullptr}, p.ldb};
      const mat C{{p.C[0], p.C[1], p.limbs == 4 ? p.C[2] : nullptr, p.limbs == 4 ? p.C[3] : nullptr}, p.ldc};
      expand(bld, p.limbs, p.algo, p.cutoff, p.m, p.l, p.n, A, B, C, p.mode, 0);
    }
  };
  Builder dry;
  build(dry);
  const size_t temps = (dry.off + 255) & ~(size_t)255;
  // converted operands of the leaves that convert, after the temporaries
  auto conv_bytes = [](int L, const gtask& g) {
    return fxop_bytes(L, g.m, g.l) + fxop_bytes(L, g.l, g.n);
  };
  size_t convs = 0;
  if (!one_leaf)
    for (int L : {2, 4})
      for (const gtask& g : dry.leaves[L])
        if (block_fx_converts(L, g.m, g.l, g.n)) convs += conv_bytes(L, g);
  // without room for the converted operands every leaf converts its tiles
  // as they are staged (the same bits)
  bool conv_ok = true;
  size_t lists = temps + convs;
  auto* b = new ddg_batch_s();
  b->use_graph = use_graph;
  if (cudaGetDevice(&b->dev) != cudaSuccess) {
    delete b;
    return set_error(DDG_ECUDA, "cudaGetDevice");
  }
  Builder real;
  real.dry = false;
  // task arrays are laid out after the temporaries; the real pass fills them
  std::vector<char> host;
  auto push_tasks = [&](const void* data, size_t bytes) {
    const size_t at = (host.size() + 255) & ~(size_t)255;
    host.resize(at + bytes);
    std::memcpy(host.data() + at, data, bytes);
    return lists + at;
  };
  // temporaries, then the task lists (bounded from the dry expansion)
  std::vector<Launch> launches;
  {
    size_t tb = 0;
    for (auto& kv : dry.pre) tb += ((kv.second.size() * sizeof(ptask) + 255) & ~(size_t)255);
    for (auto& kv : dry.post) tb += ((kv.second.size() * sizeof(ptask) + 255) & ~(size_t)255);
    for (auto& kv : dry.fix) tb += ((kv.second.size() * sizeof(gtask) + 255) & ~(size_t)255) + 256;
    for (int L : {2, 4}) {
      const size_t nl = dry.leaves[L].size();
      tb += ((nl * sizeof(gtask) + 255) & ~(size_t)255) + 256;   // leaves converting tiles as staged
      tb += ((nl * sizeof(gctask) + 255) & ~(size_t)255) + 256;  // leaves on converted operands
      tb += ((2 * nl * sizeof(fx_ctask) + 255) & ~(size_t)255);  // their conversions
    }
    b->bytes = lists + tb + 4096;
  }
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  if (ddg::ws_alloc(reinterpret_cast<void**>(&b->buf), std::max<size_t>(b->bytes, 256), cs) != cudaSuccess) {
    cudaGetLastError();
    b->buf = nullptr;
    if (convs) {
      conv_ok = false;
      b->bytes -= convs;
      lists = temps;
      if (ddg::ws_alloc(reinterpret_cast<void**>(&b->buf), std::max<size_t>(b->bytes, 256), cs) != cudaSuccess) {
        cudaGetLastError();
        b->buf = nullptr;
      }
    }
    if (!b->buf) {
      delete b;
      return set_error(DDG_ENOMEM, "ddg_batch_create: workspace of " + std::to_string(b->bytes) + " bytes");
    }
  }
  real.base = b->buf;
  build(real);
  auto number_g = [&](std::vector<gtask>& v, int L) {
    int bm, bn;
    fx_tile_shape(L, &bm, &bn);
    std::stable_sort(v.begin(), v.end(), [](const gtask& x, const gtask& y) { return x.l > y.l; });
    int64_t t0 = 0;
    for (auto& g : v) {
      g.tiles_n = (int)((g.n + bn - 1) / bn);
      g.tile0 = t0;
      t0 += (int64_t)((g.m + bm - 1) / bm) * g.tiles_n;
    }
    return t0;
  };
  auto number_p = [&](std::vector<ptask>& v) {
    int64_t t0 = 0;
    for (auto& p : v) {
      p.tiles_x = (int)((p.cols + 31) / 32);
      p.tile0 = t0;
      t0 += ((p.rows + 7) / 8) * p.tiles_x;
    }
    return t0;
  };
  auto add_g = [&](std::vector<gtask>& v, int L) {
    if (v.empty()) return;
    const int64_t total = number_g(v, L);
    Launch la{1, L, 0, 0, (int)v.size(), total, 0, 0.0};
    for (const gtask& g : v) la.ops += (double)g.m * g.l * g.n;  // multiply-adds
    la.task_off = push_tasks(v.data(), v.size() * sizeof(gtask));
    const uint64_t zero = 0;
    la.counter_off = push_tasks(&zero, sizeof(zero));
    launches.push_back(la);
    b->stats.leaf_tiles += total;
  };
  auto add_p = [&](std::vector<ptask>& v, int L, int kind) {
    if (v.empty()) return;
    const int64_t total = number_p(v);
    Launch la{0, L, kind, 0, (int)v.size(), total, 0, 0.0};
    la.task_off = push_tasks(v.data(), v.size() * sizeof(ptask));
    launches.push_back(la);
    b->stats.pass_tasks += (int64_t)v.size();
  };
  // the leaves that convert: their operands' buffers, conversion tasks and
  // product tasks; the others stay in the staged-conversion launch
  size_t cursor = temps;
  auto add_converted = [&](std::vector<gtask>& v, int L) {
    std::vector<gtask> plain;
    std::vector<gctask> conv;
    std::vector<fx_ctask> jobs;
    int64_t ctiles = 0;
    double elems = 0.0;
    auto job = [&](int64_t rows, int64_t cols, const mat& X, fxop* out) {
      char* buf = b->buf + cursor;
      cursor += fxop_bytes(L, rows, cols);
      fx_ctask j{};
      j.rows = rows;
      j.cols = cols;
      j.X = X;
      j.w = reinterpret_cast<uint4*>(buf);
      j.f = reinterpret_cast<int*>(buf + (((size_t)rows * cols * 16 * (L == 2 ? 1 : 2) + 255) & ~(size_t)255));
      j.tiles_x = (cols + 255) / 256;
      j.tile0 = ctiles;
      ctiles += convert_tiles(rows, cols);
      elems += (double)rows * cols;
      jobs.push_back(j);
      *out = fxop{j.w, j.f, cols};
    };
    for (const gtask& g : v) {
      if (!conv_ok || !block_fx_converts(L, g.m, g.l, g.n)) {
        plain.push_back(g);
        continue;
      }
      gctask c{};
      c.m = g.m;
      c.l = g.l;
      c.n = g.n;
      c.C = g.C;
      c.mode = g.mode;
      job(g.m, g.l, g.A, &c.A);
      job(g.l, g.n, g.B, &c.B);
      conv.push_back(c);
    }
    if (!jobs.empty()) {
      Launch la{2, L, 0, 0, (int)jobs.size(), ctiles, 0, elems};
      la.task_off = push_tasks(jobs.data(), jobs.size() * sizeof(fx_ctask));
      launches.push_back(la);
    }
    if (!conv.empty()) {
      int bm, bn;
      fx_tile_shape(L, &bm, &bn);
      std::stable_sort(conv.begin(), conv.end(), [](const gctask& x, const gctask& y) { return x.l > y.l; });
      int64_t t0 = 0;
      double macs = 0.0;
      for (auto& g : conv) {
        g.tiles_n = (int)((g.n + bn - 1) / bn);
        g.tile0 = t0;
        t0 += (int64_t)((g.m + bm - 1) / bm) * g.tiles_n;
        macs += (double)g.m * g.l * g.n;
      }
      Launch la{3, L, 0, 0, (int)conv.size(), t0, 0, macs};
      la.task_off = push_tasks(conv.data(), conv.size() * sizeof(gctask));
      const uint64_t zero = 0;
      la.counter_off = push_tasks(&zero, sizeof(zero));
      launches.push_back(la);
      b->stats.leaf_tiles += t0;
    }
    add_g(plain, L);
  };
  for (int d = 0; d <= real.maxdepth; ++d)
    for (auto& kv : real.pre)
      if (std::get<0>(kv.first) == d) add_p(kv.second, std::get<1>(kv.first), std::get<2>(kv.first));
  if (one_leaf) {
    // every base-case product of both limb counts in one persistent launch,
    // tiles converted as they are staged (the converted-operand bits)
    std::vector<gtask> all;
    for (int L : {2, 4}) {
      b->stats.leaf_tasks += (int64_t)real.leaves[L].size();
      for (gtask g : real.leaves[L]) {
        g.limbs = L;
        all.push_back(g);
      }
    }
    if (!all.empty()) {
      std::stable_sort(all.begin(), all.end(), [](const gtask& x, const gtask& y) {
        return (double)x.l * x.limbs * x.limbs > (double)y.l * y.limbs * y.limbs;  // longest tiles first
      });
      int64_t t0 = 0;
      double macs = 0.0;
      for (auto& g : all) {
        int bm, bn;
        fx_tile_shape(g.limbs, &bm, &bn);
        g.tiles_n = (int)((g.n + bn - 1) / bn);
        g.tile0 = t0;
        t0 += (int64_t)((g.m + bm - 1) / bm) * g.tiles_n;
        macs += (double)g.m * g.l * g.n;
      }
      Launch la{4, 0, 0, 0, (int)all.size(), t0, 0, macs};
      la.task_off = push_tasks(all.data(), all.size() * sizeof(gtask));
      const uint64_t zero = 0;
      la.counter_off = push_tasks(&zero, sizeof(zero));
      launches.push_back(la);
      b->stats.leaf_tiles += t0;
    }
  } else {
    for (int L : {2, 4}) {
      b->stats.leaf_tasks += (int64_t)real.leaves[L].size();
      add_converted(real.leaves[L], L);
    }
  }
  for (int d = real.maxdepth; d >= 0; --d) {
    for (auto& kv : real.post)
      if (std::get<0>(kv.first) == d) add_p(kv.second, std::get<1>(kv.first), std::get<2>(kv.first));
    for (auto& kv : real.fix)
      if (std::get<0>(kv.first) == d) add_g(kv.second, std::get<1>(kv.first));
  }
  if (cursor != lists || lists + host.size() > b->bytes) {
    ddg::ws_free(b->buf, cs);
    delete b;
    return set_error(DDG_ECUDA, "ddg_batch_create: task list larger than planned");
  }
  // pageable source: the copy is staged before the call returns
  if (!host.empty() &&
      cudaMemcpyAsync(b->buf + lists, host.data(), host.size(), cudaMemcpyHostToDevice, cs) != cudaSuccess) {
    ddg::ws_free(b->buf, cs);
    delete b;
    return set_error(DDG_ECUDA, "ddg_batch_create: task upload");
  }
  b->launches = launches;
  b->kernels_per_run = (int)launches.size();
  b->stats.problems = count;
  b->stats.launches_per_run = (int64_t)launches.size();
  b->stats.workspace_bytes = (uint64_t)b->bytes;
  b->stats.leaf_macs = real.leaf_macs;
  if (use_graph && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    ddg::ws_free(b->buf, cs);
    delete b;
    return set_error(DDG_ECUDA, "ddg_batch_create: capture stream");
  }
  b->create_stream = cs;
  *out = b;
  return DDG_OK;
}

ddg_status ddg_batch_run(ddg_batch b, void* stream) {
  using namespace ddg;
  clear_error();
  if (!b) return set_error(DDG_EINVAL, "null batch");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!b->use_graph) return enqueue(b, s);
  if (!b->exec) {
    // the capture stream must see the plan's upload, queued on the create stream
    if (cudaStreamSynchronize(b->create_stream) != cudaSuccess)
      return set_error(DDG_ECUDA, "ddg_batch_run: waiting for the plan upload");
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return set_error(DDG_ECUDA, "ddg_batch_run: begin capture");
    ddg_status st = enqueue(b, b->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (st != DDG_OK) return st;
    if (e != cudaSuccess) return set_error(DDG_ECUDA, std::string("ddg_batch_run: end capture: ") + cudaGetErrorString(e));
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
      b->exec = nullptr;
      return set_error(DDG_ECUDA, "ddg_batch_run: graph instantiate");
    }
  } else {
    // launches inside the graph are counted at each replay
    g_launches.fetch_add((uint64_t)b->kernels_per_run, std::memory_order_relaxed);
  }
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return set_error(DDG_ECUDA, std::string("ddg_batch_run: graph launch: ") + cudaGetErrorString(e));
  return DDG_OK;
}

ddg_status ddg_batch_get_stats(ddg_batch b, ddg_batch_stats* st) {
  if (!b || !st) return ddg::set_error(DDG_EINVAL, "null argument");
  *st = b->stats;
  return DDG_OK;
}

ddg_status ddg_batch_destroy(ddg_batch b, void* stream) {
  if (!b) return DDG_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->dev);
  ddg_status st = DDG_OK;
  if (b->exec || b->cap) {
    // a graph may still be running: wait for the device before destroying it
    if (cudaDeviceSynchronize() != cudaSuccess) st = ddg::set_error(DDG_ECUDA, "ddg_batch_destroy: sync");
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
  }
  if (b->buf && ddg::ws_free(b->buf, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess && st == DDG_OK)
    st = ddg::set_error(DDG_ECUDA, "ddg_batch_destroy: free");
  cudaSetDevice(cur);
  delete b;
  return st;
}

ddg_status dd_gemm_batched(int32_t count, const ddg_problem* probs, void* stream) {
  ddg_batch b = nullptr;
  ddg_status st = ddg_batch_create(&b, count, probs, 0, stream);
  if (st != DDG_OK) return st;
  st = ddg_batch_run(b, stream);
  ddg_status st2 = ddg_batch_destroy(b, stream);
  return st != DDG_OK ? st : st2;
}

}  // extern "C"
