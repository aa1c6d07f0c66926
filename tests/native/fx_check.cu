// Host driver for the fixed-point helpers of the Block kernel (fx.cuh):
// reads commands from stdin and prints results, so that the Python test can
// compare them with exact integer arithmetic. Host code only (no kernels).
//   T L x0 .. x(L-1)          -> to_fixed: es M[0] .. M[W-1]   (W = 4 / 7)
//   M W D a[0..W-1] b[0..W-1]  -> mul_top: p[0 .. 2W-D-1]
//   H W a[0..W-1] b[0..W-1]    -> mul_top_hi: q[0 .. W-1]           (W = 4 / 7)
//   S L fa fb xa(L) xb(L)      -> the pre-shifted term a b at the window of the
//                                 fields fa, fb: window words 0 .. NW-1 (L = 2 / 4)
//   P NW K sh neg acc[0..NW-1] p[0..K-1] -> place_shr: acc[0 .. NW-1]
//   N NW W A[0..NW-1]          -> acc_normalize: p M[0..W-1]   (6,4) / (9,7)
//   R NW s A[0..NW-1]          -> acc_sar: A[0..NW-1]          (NW = 6 / 9)
//   O L e s M[0..W-1]          -> operand_to_limbs: limbs (hex)  (L = 2: W = 4, 4: W = 7)
//   Q b0..b3 y0 y1             -> qd_recip_refine: 4 limbs (hex)
//   F L x(L) l(L) y(L)         -> window: x - l y, rounded to L limbs (hex)
//   A L emax top n (sign x0 .. x(L-1)) x n -> add_at into V (NW = 5 / 9),
//                              then from_fixed: V[0..NW-1] ; limbs (hex)
//   B NW bits A[0..NW-1]       -> acc_mag_below: 0 / 1          (NW = 6 / 9)
// Doubles are read as 16 hex digits of their bit pattern.
#include <cinttypes>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "fx.cuh"
#include "fx_pre.cuh"
#include "fxscalar.cuh"

using namespace ddg;

template <class... A>
static void scan(const char* f, A... a) {
  if (std::scanf(f, a...) != (int)sizeof...(A)) std::exit(2);
}

static double rd() {
  unsigned long long b;
  scan("%llx", &b);
  return fx::bitsd(b);
}

template <int L, int W>
static void do_fixed() {
  double x[L];
  for (int q = 0; q < L; ++q) x[q] = rd();
  uint32_t M[W];
  const int es = fx::to_fixed<L, W>(x, M);
  std::printf("%d", es);
  for (int w = 0; w < W; ++w) std::printf(" %u", M[w]);
  std::printf("\n");
}

template <int W, int D>
static void do_mul() {
  uint32_t a[W], b[W], p[2 * W - D];
  for (int i = 0; i < W; ++i) scan("%u", &a[i]);
  for (int i = 0; i < W; ++i) scan("%u", &b[i]);
  fx::mul_top<W, D>(a, b, p);
  for (int i = 0; i < 2 * W - D; ++i) std::printf("%u%c", p[i], i + 1 < 2 * W - D ? ' ' : '\n');
}

template <int W>
static void do_mul_hi() {
  uint32_t a[W], b[W], q[W];
  for (int i = 0; i < W; ++i) scan("%u", &a[i]);
  for (int i = 0; i < W; ++i) scan("%u", &b[i]);
  fx::mul_top_hi<W>(a, b, q);
  for (int i = 0; i < W; ++i) std::printf("%u%c", q[i], i + 1 < W ? ' ' : '\n');
}

// The pre-shifted form's term (fx_pre.cuh) on the host: the operands
// shifted to the fields fa, fb, the product's upper words (mul_top_hi) and
// the sign, as the window words 1 .. NW-1 (word 0 = 0) of that one term.
template <int L, int W, int NW>
static void do_pre_term() {
  int fa, fb;
  scan("%d %d", &fa, &fb);
  double xa[L], xb[L];
  for (int q = 0; q < L; ++q) xa[q] = rd();
  for (int q = 0; q < L; ++q) xb[q] = rd();
  uint32_t ma[W], mb[W];
  const int ea = fx::to_fixed<L, W>(xa, ma), eb = fx::to_fixed<L, W>(xb, mb);
  const bool za = (fx::dbits(xa[0]) << 1) == 0u, zb = (fx::dbits(xb[0]) << 1) == 0u;
  shr_words<W>(ma, za ? 32 * W : fa - (ea & 0xFFFF));
  shr_words<W>(mb, zb ? 32 * W : fb - (eb & 0xFFFF));
  const bool neg = ((((ea >> 16) & 1) != 0) && !za) != ((((eb >> 16) & 1) != 0) && !zb);
  uint32_t q[W];
  fx::mul_top_hi<W>(ma, mb, q);
  uint32_t acc[NW - 1] = {};
  for (int t = 0; t < W; ++t) acc[t] = q[t];
  if (neg) {  // two's complement of (q, 0)
    uint64_t c = 1;
    for (int t = 0; t < NW - 1; ++t) {
      const uint64_t v = (uint64_t)(acc[t] ^ 0xFFFFFFFFu) + c;
      acc[t] = (uint32_t)v;
      c = v >> 32;
    }
  }
  uint32_t w[NW];
  pre_window<NW>(acc, w);
  for (int i = 0; i < NW; ++i) std::printf("%u%c", w[i], i + 1 < NW ? ' ' : '\n');
}

template <int NW, int K>
static void do_place() {
  int sh;
  unsigned neg;
  scan("%d %u", &sh, &neg);
  uint32_t acc[NW], p[K];
  for (int i = 0; i < NW; ++i) scan("%u", &acc[i]);
  for (int i = 0; i < K; ++i) scan("%u", &p[i]);
  fx::place_shr<NW, K>(acc, p, sh, neg ? 0xFFFFFFFFu : 0u);
  for (int i = 0; i < NW; ++i) std::printf("%u%c", acc[i], i + 1 < NW ? ' ' : '\n');
}

template <int L, int NW>
static void do_sum() {
  int emax, top, n;
  scan("%d %d %d", &emax, &top, &n);
  uint32_t V[NW] = {0};
  for (int i = 0; i < n; ++i) {
    unsigned sg;
    scan("%u", &sg);
    double x[L];
    for (int q = 0; q < L; ++q) x[q] = rd();
    fx::add_at<L, NW>(V, x, emax, top, sg);
  }
  for (int w = 0; w < NW; ++w) std::printf("%u ", V[w]);
  double out[L];
  fx::from_fixed<L, NW>(V, emax - 1075 - top, out);
  std::printf(";");
  for (int q = 0; q < L; ++q) std::printf(" %016llx", (unsigned long long)fx::dbits(out[q]));
  std::printf("\n");
}

template <int NW, int W>
static void do_norm() {
  uint32_t A[NW], M[W];
  for (int i = 0; i < NW; ++i) scan("%u", &A[i]);
  const int p = fx::acc_normalize<NW, W>(A, M);
  std::printf("%d", p);
  for (int i = 0; i < W; ++i) std::printf(" %u", M[i]);
  std::printf("\n");
}

template <int NW>
static void do_sar() {
  int sh;
  scan("%d", &sh);
  uint32_t A[NW];
  for (int i = 0; i < NW; ++i) scan("%u", &A[i]);
  fx::acc_sar<NW>(A, sh);
  for (int i = 0; i < NW; ++i) std::printf("%u%c", A[i], i + 1 < NW ? ' ' : '\n');
}

template <int L, int W>
static void do_limbs() {
  int e;
  unsigned sg;
  scan("%d %u", &e, &sg);
  uint32_t M[W];
  for (int i = 0; i < W; ++i) scan("%u", &M[i]);
  double out[L];
  fx::operand_to_limbs<L, W>(M, e, sg, out);
  for (int q = 0; q < L; ++q) std::printf("%016llx%c", (unsigned long long)fx::dbits(out[q]), q + 1 < L ? ' ' : '\n');
}

template <int L>
static void do_fms() {
  constexpr int W = ddg::tfx<L>::W, NW = ddg::tfx<L>::NW;
  double x[L], l[L], y[L];
  for (int q = 0; q < L; ++q) x[q] = rd();
  for (int q = 0; q < L; ++q) l[q] = rd();
  for (int q = 0; q < L; ++q) y[q] = rd();
  uint32_t acc[NW] = {0}, Ml[W], My[W];
  int A = fx::expfield(x[0]) > 1 ? fx::expfield(x[0]) : 1;
  fx::add_at<L, NW>(acc, x, A, ddg::tfx<L>::TOPA, 0u);
  const int el = fx::to_fixed<L, W>(l, Ml), ey = fx::to_fixed<L, W>(y, My);
  if ((fx::dbits(l[0]) << 1) != 0u && (fx::dbits(y[0]) << 1) != 0u)
    ddg::window_sub_product<L>(acc, A, Ml, el & 0xFFFF, (uint32_t)el >> 16, My, ey & 0xFFFF, (uint32_t)ey >> 16);
  double out[L];
  fx::from_fixed<L, NW>(acc, A - 1075 - ddg::tfx<L>::TOPA, out);
  for (int q = 0; q < L; ++q) std::printf("%016llx%c", (unsigned long long)fx::dbits(out[q]), q + 1 < L ? ' ' : '\n');
}

template <int NW>
static void do_below() {
  int bits;
  scan("%d", &bits);
  uint32_t A[NW];
  for (int i = 0; i < NW; ++i) scan("%u", &A[i]);
  std::printf("%d\n", fx::acc_mag_below<NW>(A, bits) ? 1 : 0);
}

static void do_recip() {
  double b[4], out[4];
  for (int q = 0; q < 4; ++q) b[q] = rd();
  const double y0 = rd(), y1 = rd();
  ddg::qd_recip_refine(b, y0, y1, out);
  for (int q = 0; q < 4; ++q) std::printf("%016llx%c", (unsigned long long)fx::dbits(out[q]), q < 3 ? ' ' : '\n');
}

int main() {
  char cmd[4];
  while (std::scanf("%3s", cmd) == 1) {
    int a, b;
    if (cmd[0] == 'T') {
      scan("%d", &a);
      if (a == 2) do_fixed<2, 4>();
      else do_fixed<4, 7>();
    } else if (cmd[0] == 'M') {
      scan("%d %d", &a, &b);
      if (a == 4) do_mul<4, 3>();
      else do_mul<7, 6>();
    } else if (cmd[0] == 'S') {
      scan("%d", &a);
      if (a == 2) do_pre_term<2, 4, 6>();
      else do_pre_term<4, 7, 9>();
    } else if (cmd[0] == 'H') {
      scan("%d", &a);
      if (a == 4) do_mul_hi<4>();
      else do_mul_hi<7>();
    } else if (cmd[0] == 'F') {
      scan("%d", &a);
      if (a == 2) do_fms<2>();
      else do_fms<4>();
    } else if (cmd[0] == 'Q') {
      do_recip();
    } else if (cmd[0] == 'O') {
      scan("%d", &a);
      if (a == 2) do_limbs<2, 4>();
      else do_limbs<4, 7>();
    } else if (cmd[0] == 'N') {
      scan("%d %d", &a, &b);
      if (a == 6) do_norm<6, 4>();
      else do_norm<9, 7>();
    } else if (cmd[0] == 'R') {
      scan("%d", &a);
      if (a == 6) do_sar<6>();
      else do_sar<9>();
    } else if (cmd[0] == 'A') {
      scan("%d", &a);
      if (a == 2) do_sum<2, 5>();
      else do_sum<4, 9>();
    } else if (cmd[0] == 'B') {
      scan("%d", &a);
      if (a == 6) do_below<6>();
      else do_below<9>();
    } else if (cmd[0] == 'P') {
      scan("%d %d", &a, &b);
      if (a == 6) do_place<6, 5>();
      else do_place<9, 8>();
    }
  }
  return 0;
}
