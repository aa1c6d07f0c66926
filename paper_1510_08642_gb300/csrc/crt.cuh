// Moduli of the CRT (Ozaki scheme II) DD product and their reduction
// constants, shared by its two product engines: INT8 mma.sync (ozaki.cu)
// and BF16 tcgen05 (ozaki_tc.cu). The residue products of both are exact
// integers, so both give the same residues and the same bits.
#pragma once

#include <cstdint>

namespace ddg {

constexpr int CRT_MAXN = 40;

// The CRT moduli: the 40 largest pairwise-coprime integers <= 256, taken
// greedily from 256 downward.
__host__ __device__ constexpr int crt_mod(int t) {
  constexpr int tab[CRT_MAXN] = {256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199,
                                 197, 193, 191, 181, 179, 173, 167, 163, 157, 151, 149, 139, 137, 131,
                                 127, 113, 109, 107, 103, 101, 97,  89,  83,  79,  73,  71};
  return tab[t];
}

// 2^e mod m (for the digit-wise residues of the split).
__host__ __device__ constexpr uint32_t crt_pow2_mod(int e, uint32_t m) {
  uint32_t r = 1u % m;
  for (int i = 0; i < e; ++i) r = (r * 2u) % m;
  return r;
}

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
constexpr bool crt_mods_ok() {
  for (int a = 0; a < CRT_MAXN; ++a) {
    if (crt_mod(a) < 2 || crt_mod(a) > 256 || (a > 0 && crt_mod(a) >= crt_mod(a - 1))) return false;
    for (int b = 0; b < a; ++b)
      if (gcd_c(crt_mod(a), crt_mod(b)) != 1) return false;
  }
  return true;
}
static_assert(crt_mods_ok(), "CRT moduli must be pairwise coprime, decreasing, <= 256");

// Reduction constants of each CRT modulus for the GEMM epilogue: for
// |v| <= 2^30, u = v + bias (bias = m ceil(2^30 / m)) lies in [0, 2^32) and
// u mod m = u - m q with q = umulhi(u, floor(2^32 / m)) or q + 1. Fixed at
// compile time (constant memory, no per-call state).
struct crt_red {
  uint32_t m[CRT_MAXN], magic[CRT_MAXN], bias[CRT_MAXN];
};
constexpr crt_red make_crt_red() {
  crt_red r{};
  for (int t = 0; t < CRT_MAXN; ++t) {
    const uint32_t m = (uint32_t)crt_mod(t);
    r.m[t] = m;
    r.magic[t] = (uint32_t)((1ull << 32) / m);
    r.bias[t] = m * (((1u << 30) + m - 1u) / m);
  }
  return r;
}
// Each translation unit that reduces residues keeps its own copy.
static __constant__ crt_red c_crt_red = make_crt_red();

}  // namespace ddg
