// Host driver for the fixed-point helpers of the Block kernel (fx.cuh):
// reads commands from stdin and prints results, so that the Python test can
// compare them with exact integer arithmetic. Host code only (no kernels).
//   T L x0 .. x(L-1)          -> to_fixed: es M[0] .. M[W-1]   (W = 4 / 7)
//   M W D a[0..W-1] b[0..W-1]  -> mul_top: p[0 .. 2W-D-1]
//   P NW K sh neg acc[0..NW-1] p[0..K-1] -> place_shr: acc[0 .. NW-1]
// Doubles are read as 16 hex digits of their bit pattern.
#include <cinttypes>
#include <cstdio>
#include <cstring>

#include "fx.cuh"

using namespace ddg;

static double rd() {
  unsigned long long b;
  if (std::scanf("%llx", &b) != 1) return 0.0;
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
  for (int i = 0; i < W; ++i) std::scanf("%u", &a[i]);
  for (int i = 0; i < W; ++i) std::scanf("%u", &b[i]);
  fx::mul_top<W, D>(a, b, p);
  for (int i = 0; i < 2 * W - D; ++i) std::printf("%u%c", p[i], i + 1 < 2 * W - D ? ' ' : '\n');
}

template <int NW, int K>
static void do_place() {
  int sh;
  unsigned neg;
  std::scanf("%d %u", &sh, &neg);
  uint32_t acc[NW], p[K];
  for (int i = 0; i < NW; ++i) std::scanf("%u", &acc[i]);
  for (int i = 0; i < K; ++i) std::scanf("%u", &p[i]);
  fx::place_shr<NW, K>(acc, p, sh, neg ? 0xFFFFFFFFu : 0u);
  for (int i = 0; i < NW; ++i) std::printf("%u%c", acc[i], i + 1 < NW ? ' ' : '\n');
}

int main() {
  char cmd[4];
  while (std::scanf("%3s", cmd) == 1) {
    int a, b;
    if (cmd[0] == 'T') {
      std::scanf("%d", &a);
      if (a == 2) do_fixed<2, 4>();
      else do_fixed<4, 7>();
    } else if (cmd[0] == 'M') {
      std::scanf("%d %d", &a, &b);
      if (a == 4) do_mul<4, 3>();
      else do_mul<7, 6>();
    } else if (cmd[0] == 'P') {
      std::scanf("%d %d", &a, &b);
      if (a == 6) do_place<6, 5>();
      else do_place<9, 8>();
    }
  }
  return 0;
}
