// DD product by error-free splitting into INT8 slices (the Ozaki scheme,
// Ozaki, Ogita, Oishi 2012), as a precision alternative to the integer-pipe
// Block kernel for the DD product C := A B of Kouya 2015, Section 2, Eq. 1.
//
// Split (integer pipe, no FP64). Row i of A is scaled by 2^-ea_i, where
// 2^ea_i bounds every |a_ik|, and rounded to the integer
//   X_ik = round(a_ik 2^(T - ea_i)),   T = 6 + 7 (s - 1),
// then written in balanced base 128: X = sum_p d_p 128^(s-p), d_p in
// [-64, 63] for p >= 2 and d_1 in [-64, 64]. The digits of slice p form an
// int8 matrix alpha^(p); B is split the same way per column j (beta^(q),
// stored transposed so that both operands are k-contiguous).
// Products (INT8 tensor cores, mma.sync m16n8k32 with INT32 accumulation;
// tcgen05 has no INT8 kind on sm_103a). Slice pairs of equal weight
// 2^(-12 - 7 (p + q - 2)) are summed by concatenating along k: for each
// diagonal r = p + q = 2 .. s + 1,
//   D_r = sum_{p + q = r} alpha^(p) beta^(q),
// exact in INT32 while (r - 1) l 2^12 < 2^31. Pairs with p + q > s + 1 are
// dropped (their weight is below the slices' own rounding).
// Recombination (integer pipe): V_ij = sum_r D_r 2^(7 (s + 1 - r)) exactly in
// a 192-bit fixed-point word, then c_ij = V_ij 2^(ea_i + fb_j - T - 6), rounded
// to DD (and combined with C for the update modes).
// Error per entry <= l (s + 3) 2^(-7 s) 2^(ea_i + fb_j) (slice rounding and
// dropped pairs) plus the final DD rounding.
//
// CRT variant (Ozaki, Uchino, Imamura 2025, "Ozaki scheme II"; DD only).
// Rows of A and columns of B are scaled and rounded to integers X, Y with
// |X|, |Y| <= 2^P as above (T = P); Z = X Y is then an integer matrix with
// |Z| <= l 2^(2P). Instead of slicing X into digits, take N pairwise-coprime
// moduli m_t <= 256 with M = prod m_t > 2 l 2^(2P): the residues X mod m_t
// and Y mod m_t fit in int8, one INT8 product per modulus gives Z mod m_t
// (INT32 accumulation, exact for l <= 2^16, reduced mod m_t in the
// epilogue), and the Chinese remainder theorem recovers Z exactly:
//   Z = (sum_t r_t c_t) mod M, c_t = (M / m_t) ((M / m_t)^-1 mod m_t),
// taken in (-M/2, M/2). N products instead of s (s + 1) / 2: N = 32 gives
// P = 113 at l = 4096 with 32 INT8 products, where slicing needs 136 for
// the same precision.
#include <algorithm>
#include <mutex>
#include <set>
#include <cuda_bf16.h>
#include <cmath>
#include <cstring>
#include <string>

#include "arith.cuh"
#include "fx.cuh"
#include "crt.cuh"
#include "kernels.cuh"

namespace ddg {

namespace {

constexpr int OBM = 128, OBN = 128, OBK = 64, OST = 3, OROW = OBK + 16;
constexpr int STAGE_BYTES = (OBM + OBN) * OROW;
constexpr int OZ_SMEM = OST * STAGE_BYTES;
constexpr int OZ_MAXS = 40;  // most slices (QD: 32; DD: 18) or CRT moduli (40)
constexpr int CRT_NW = 10;   // 320-bit CRT reconstruction word
constexpr int CRT_PMAX = 120;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(const void* p, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s));
}

__device__ __forceinline__ void mma_s8(int (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

}  // namespace

// Largest exponent field of the leading limb per row (byrow) or per column.
__global__ void oz_exp_kernel(int64_t rows, int64_t cols, mat X, int byrow, int* ex) {
  if (byrow) {
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    int f = 1;
    for (int64_t k = lane; k < cols; k += 32) f = max(f, fx::expfield(X.p[0][r * X.ld + k]));
    f = __reduce_max_sync(0xffffffffu, f);
    if (lane == 0) ex[r] = f;
  } else {
    // 32 columns per CTA, its 8 warps splitting the rows (coalesced rows of
    // 32 doubles), then a shared-memory reduction over the warps
    __shared__ int part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * 32 + lane;
    int f = 1;
    if (c < cols)
      for (int64_t k = w; k < rows; k += 8) f = max(f, fx::expfield(X.p[0][k * X.ld + c]));
    part[w][lane] = f;
    __syncthreads();
    if (w == 0 && c < cols) {
#pragma unroll
      for (int t = 1; t < 8; ++t) f = max(f, part[t][lane]);
      ex[c] = f;
    }
  }
}

// Balanced base-128 digits of round(x 2^(T - e)) for x = the sum of the L
// limbs, where 2^e bounds |x| (field = biased exponent with |x0| <
// 2^(field - 1022)). The limbs are placed exactly (bits below 2^-64 units
// truncated toward zero) in a fixed-point word of NW 32-bit words, rounded
// half up to the integer X, and X is cut into digits from the least
// significant end: d_p = the balanced residue of X mod 128, X = (X - d_p) / 128.
template <int L>
__device__ __forceinline__ void oz_integer(const double (&x)[L], int field, int T,
                                           unsigned long long (&X)[L == 2 ? 2 : 4]) {
  constexpr int NW = L == 2 ? 6 : 9;   // split word: 192 / 288 bits
  constexpr int KW = L == 2 ? 2 : 4;   // X in 64-bit words (X < 2^T)
  uint32_t acc[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) acc[w] = 0u;
  // LSB of acc = 2^(e - T - 64); a double M 2^(E - 1075) sits at E - field + T + 11
#pragma unroll
  for (int q = 0; q < L; ++q) {
    fx::unpacked u = fx::unpack(x[q]);
    uint32_t p[4] = {u.m0, u.m1, 0u, 0u};
    if (q == 0) fx::place<NW, (L == 2 ? 3 : 6)>(acc, p, u.e - field + T + 11, u.s);
    else fx::place<NW, (L == 2 ? 2 : 4)>(acc, p, u.e - field + T + 11, u.s);
  }
  // X = floor((acc + 2^63) / 2^64): round half up to an integer
  uint32_t half[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) half[w] = w == 1 ? 0x80000000u : 0u;
  fx::acc_add<NW>(acc, half, 0u);
#pragma unroll
  for (int k = 0; k < KW; ++k) {
    const int w0 = 2 + 2 * k, w1 = 3 + 2 * k;
    const uint32_t lo = w0 < NW ? acc[w0 < NW ? w0 : 0] : 0u;
    // sign-extend past the top word
    const uint32_t sext = (acc[NW - 1] >> 31) ? 0xFFFFFFFFu : 0u;
    const uint32_t hi = w1 < NW ? acc[w1 < NW ? w1 : 0] : sext;
    X[k] = ((unsigned long long)hi << 32) | lo;
  }
}

template <int L>
__device__ __forceinline__ void oz_digits(const double (&x)[L], int field, int s, int8_t* out,
                                          int64_t stride) {
  constexpr int KW = L == 2 ? 2 : 4;
  unsigned long long X[KW];
  oz_integer<L>(x, field, 6 + 7 * (s - 1), X);
  for (int p = s; p >= 2; --p) {
    int d = (int)(X[0] & 127u);
    d = d >= 64 ? d - 128 : d;
    // X -= d (multiword, two's complement), then X >>= 7 (arithmetic)
    const unsigned long long dd = (unsigned long long)(long long)d;
    const unsigned long long ext = d < 0 ? ~0ull : 0ull;
    unsigned long long carry = 0;
#pragma unroll
    for (int k = 0; k < KW; ++k) {
      const unsigned long long sub = k == 0 ? dd : ext;
      const unsigned long long r = X[k] - sub - carry;
      carry = (X[k] < sub) || (X[k] - sub < carry) ? 1ull : 0ull;
      X[k] = r;
    }
#pragma unroll
    for (int k = 0; k < KW - 1; ++k) X[k] = (X[k] >> 7) | (X[k + 1] << 57);
    X[KW - 1] = (unsigned long long)((long long)X[KW - 1] >> 7);
    out[(int64_t)(p - 1) * stride] = (int8_t)d;
  }
  out[0] = (int8_t)(int)(long long)X[0];  // remaining top digit in [-64, 64]
}


// Residues of the integer round(x 2^(P - e)) modulo m_0 .. m_(N-1), each as
// an int8 representative (r or r - m_t). |X| < 2^121 is taken as four 32-bit
// words w_k; X mod m = sum_k (w_k mod m) (2^(32 k) mod m) mod m, with every
// modulus a compile-time constant (the loop is unrolled), so each reduction
// is a multiply-high sequence on the integer pipe.
// A residue or digit stored as an int8 (mma.sync operands) or as a bf16
// (tcgen05 operands; every integer of magnitude <= 256 is exact in bf16).
__device__ __forceinline__ void oz_put(int8_t* p, int v) { *p = (int8_t)v; }
__device__ __forceinline__ void oz_put(__nv_bfloat16* p, int v) { *p = __int2bfloat16_rn(v); }

template <typename T>
__device__ __forceinline__ void oz_residues(const double (&x)[2], int field, int N, int P, T* out,
                                            int64_t stride) {
  unsigned long long X[2];
  oz_integer<2>(x, field, P, X);
  const bool neg = (long long)X[1] < 0;
  if (neg) {  // |X| (128-bit two's complement negate)
    X[0] = ~X[0] + 1ull;
    X[1] = ~X[1] + (X[0] == 0ull ? 1ull : 0ull);
  }
  // |X| <= 2^120 as six 21-bit digits d_k: X mod m = (sum_k d_k (2^(21 k)
  // mod m)) mod m, the sum below 6 2^21 255 < 2^32, so one 32-bit
  // multiply-add per digit and one reduction per modulus
  uint32_t d[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int b = 21 * k;  // bit offset of digit k in the 128-bit |X|
    const unsigned long long lo = b < 64 ? X[0] >> b : 0ull;
    const unsigned long long hi = b == 0 ? 0ull : (b < 64 ? X[1] << (64 - b) : X[1] >> (b - 64));
    d[k] = (uint32_t)(lo | hi) & 0x1FFFFFu;
  }
#pragma unroll
  for (int t = 0; t < CRT_MAXN; ++t) {
    if (t < N) {
      const uint32_t m = (uint32_t)crt_mod(t);
      uint32_t acc = 0u;
#pragma unroll
      for (int k = 0; k < 6; ++k) acc += d[k] * crt_pow2_mod(21 * k, m);
      uint32_t r = acc % m;
      if (neg && r != 0u) r = m - r;
      oz_put(out + (int64_t)t * stride, r < 128u ? (int)r : (int)r - (int)m);
    }
  }
}

// Slices of A (per row) into As[s][mpad][lpad], of B (per column, stored
// transposed) into Bs[s][npad][lpad]; padding is zero. With CRT, the N
// residue planes instead (s = N, T = P).
template <int L, bool CRT, typename T = int8_t>
__global__ void oz_split_a_kernel(int64_t m, int64_t l, mat A, const int* ex, int s, int P, int64_t mpad,
                                  int64_t lpad, T* As) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (k >= lpad) return;
  const int64_t stride = mpad * lpad;
  T* out = As + i * lpad + k;
  if (i < m && k < l) {
    double x[L];
#pragma unroll
    for (int q = 0; q < L; ++q) x[q] = A.p[q][i * A.ld + k];
    if constexpr (CRT) oz_residues(x, ex[i], s, P, out, stride);
    else oz_digits<L>(x, ex[i], s, out, stride);
  } else {
    for (int p = 0; p < s; ++p) oz_put(out + (int64_t)p * stride, 0);
  }
}

template <int L, bool CRT, typename T = int8_t>
__global__ void oz_split_b_kernel(int64_t l, int64_t n, mat B, const int* ex, int s, int P, int64_t npad,
                                  int64_t lpad, T* Bs) {
  // tile: 32 k x 32 j; digits staged in shared memory and written k-contiguous
  __shared__ int8_t t[OZ_MAXS][32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int64_t k0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  for (int kk = ty; kk < 32; kk += 8) {
    const int64_t k = k0 + kk, j = j0 + tx;
    int8_t dig[OZ_MAXS];
    if (k < l && j < n) {
      double x[L];
#pragma unroll
      for (int q = 0; q < L; ++q) x[q] = B.p[q][k * B.ld + j];
      if constexpr (CRT) oz_residues(x, ex[j], s, P, dig, 1);
      else oz_digits<L>(x, ex[j], s, dig, 1);
    } else {
      for (int p = 0; p < s; ++p) dig[p] = 0;
    }
    for (int p = 0; p < s; ++p) t[p][tx][kk] = dig[p];
  }
  __syncthreads();
  const int64_t stride = npad * lpad;
  for (int jj = ty; jj < 32; jj += 8) {
    const int64_t j = j0 + jj, k = k0 + tx;
    if (j < npad && k < lpad)
      for (int p = 0; p < s; ++p) oz_put(Bs + (int64_t)p * stride + j * lpad + k, t[p][jj][tx]);
  }
}


// Slices: D[r - 2] = sum_{p + q = r} alpha^(p) beta^(q) for the diagonal of
// blockIdx.z (z = 0 is the longest diagonal, r = s + 1, scheduled first).
// CRT: R[t] = (alpha^(t) beta^(t)) mod m_t as bytes, t = blockIdx.z.
template <bool CRT>
__global__ void __launch_bounds__(256) oz_gemm_kernel(int64_t mpad, int64_t npad, int64_t lpad, int s,
                                                      const int8_t* __restrict__ As,
                                                      const int8_t* __restrict__ Bs, int32_t* D,
                                                      uint8_t* R) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps: 64 x 32 each
  const int r = CRT ? 0 : s + 1 - (int)blockIdx.z;
  const int nseg = CRT ? 1 : r - 1;
  const int64_t m0 = (int64_t)blockIdx.y * OBM, n0 = (int64_t)blockIdx.x * OBN;
  const int kps = (int)(lpad / OBK);
  const int total = nseg * kps;

  auto load = [&](int q, int stage) {
    const int seg = q / kps, kk = q % kps;
    const int pa = CRT ? (int)blockIdx.z + 1 : seg + 1, pb = CRT ? pa : r - pa;
    const int8_t* ga = As + (int64_t)(pa - 1) * mpad * lpad + m0 * lpad + (int64_t)kk * OBK;
    const int8_t* gb = Bs + (int64_t)(pb - 1) * npad * lpad + n0 * lpad + (int64_t)kk * OBK;
    uint8_t* sa = smem + stage * STAGE_BYTES;
    uint8_t* sb = sa + OBM * OROW;
#pragma unroll
    for (int c = tid; c < OBM * OBK / 16; c += 256) {
      const int row = c >> 2, col = (c & 3) * 16;
      cp_async16(sa + row * OROW + col, ga + row * lpad + col);
      cp_async16(sb + row * OROW + col, gb + row * lpad + col);
    }
  };

  int acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0;

#pragma unroll
  for (int q = 0; q < OST - 1; ++q) {
    if (q < total) load(q, q);
    cp_commit();
  }
  for (int q = 0; q < total; ++q) {
    cp_wait<OST - 2>();
    __syncthreads();
    if (q + OST - 1 < total) load(q + OST - 1, (q + OST - 1) % OST);
    cp_commit();
    const uint8_t* sa = smem + (q % OST) * STAGE_BYTES;
    const uint8_t* sb = sa + OBM * OROW;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t af[4][4], bf[4][2];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        const int row = wm * 64 + mi * 16 + (lane & 15);
        const int col = ks * 32 + (lane >> 4) * 16;
        ldsm_x4(sa + row * OROW + col, af[mi][0], af[mi][1], af[mi][2], af[mi][3]);
      }
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {
        const int row = wn * 32 + nj * 16 + (lane & 7) + ((lane >> 4) << 3);
        const int col = ks * 32 + ((lane >> 3) & 1) * 16;
        ldsm_x4(sb + row * OROW + col, bf[2 * nj][0], bf[2 * nj][1], bf[2 * nj + 1][0], bf[2 * nj + 1][1]);
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_s8(acc[mi][ni], af[mi], bf[ni][0], bf[ni][1]);
    }
  }
  cp_wait<0>();
  const int g = lane >> 2, tq = lane & 3;
  if constexpr (CRT) {
    const int t = blockIdx.z;
    const uint32_t m = c_crt_red.m[t], magic = c_crt_red.magic[t], bias = c_crt_red.bias[t];
    auto res = [&](int v) -> uint32_t {
      const uint32_t u = (uint32_t)v + bias;
      uint32_t x = u - __umulhi(u, magic) * m;
      return x >= m ? x - m : x;
    };
    uint8_t* Rt = R + (int64_t)t * mpad * npad;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int64_t row = m0 + wm * 64 + mi * 16 + g;
        const int64_t col = n0 + wn * 32 + ni * 8 + 2 * tq;
        *reinterpret_cast<uchar2*>(Rt + row * npad + col) =
            make_uchar2((uint8_t)res(acc[mi][ni][0]), (uint8_t)res(acc[mi][ni][1]));
        *reinterpret_cast<uchar2*>(Rt + (row + 8) * npad + col) =
            make_uchar2((uint8_t)res(acc[mi][ni][2]), (uint8_t)res(acc[mi][ni][3]));
      }
    return;
  }
  int32_t* Dr = D + (int64_t)(r - 2) * mpad * npad;
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const int64_t row = m0 + wm * 64 + mi * 16 + g;
      const int64_t col = n0 + wn * 32 + ni * 8 + 2 * tq;
      *reinterpret_cast<int2*>(Dr + row * npad + col) = make_int2(acc[mi][ni][0], acc[mi][ni][1]);
      *reinterpret_cast<int2*>(Dr + (row + 8) * npad + col) = make_int2(acc[mi][ni][2], acc[mi][ni][3]);
    }
}

// C (mode) sum_r D_r 2^(ea_i + fb_j - 12 - 7 (r - 2)), exact in a 192-bit
// (DD) or 288-bit (QD) word, rounded once: DD = leading 53 bits and the next
// 53 (truncated), summed by TwoSum; QD = four such 53-bit pieces,
// renormalised.
template <int L>
__global__ void oz_recombine_kernel(int64_t m, int64_t n, int s, int64_t mpad, int64_t npad,
                                    const int32_t* D, const int* exa, const int* exb, mat C, int mode) {
  constexpr int NW = L == 2 ? 6 : 9;
  using N = num<L>;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j >= n || i >= m) return;
  uint32_t acc[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) acc[w] = 0u;
  const int64_t plane = mpad * npad;
  for (int r = 2; r <= s + 1; ++r) {
    const int32_t v = D[(int64_t)(r - 2) * plane + i * npad + j];
    const int sh = 7 * (s + 1 - r);
    const int w = sh >> 5, b = sh & 31;
    const long long x = (long long)v * (long long)(1u << b);  // |x| < 2^62
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)((unsigned long long)x >> 32);
    const uint32_t ext = x < 0 ? 0xFFFFFFFFu : 0u;
    uint32_t d[NW];
#pragma unroll
    for (int t = 0; t < NW; ++t) d[t] = t < w ? 0u : (t == w ? lo : (t == w + 1 ? hi : ext));
    fx::acc_add<NW>(acc, d, 0u);
  }
  const int T = 6 + 7 * (s - 1);
  // a ~ 2^(ea - T) sum_p d_p 128^(s - p), likewise b, so
  // c = 2^(ea + fb - 2T) sum_r D_r 128^(2s - r) = V 2^(ea + fb - T - 6),
  // with ea = exa - 1022, fb = exb - 1022.
  const int lsb = (exa[i] - 1022) + (exb[j] - 1022) - T - 6;
  const uint32_t neg = fx::acc_abs<NW>(acc);
  uint64_t ch[L];
  int ex[L];
  double x[L];
#pragma unroll
  for (int q = 0; q < L; ++q) x[q] = 0.0;
  if (fx::acc_chunks<NW, L>(acc, ch, ex)) {
#pragma unroll
    for (int q = 0; q < L; ++q) {
      const int k = lsb + ex[q];
      double v = (ch[q] == 0 || k < -2044) ? 0.0 : fx::pow2_product(__ull2double_rn(ch[q]), k > 2046 ? 2046 : k);
      x[q] = neg ? -v : v;
    }
  }
  typename N::T v;
  if constexpr (L == 2) {
    two_sum(x[0], x[1], v.hi, v.lo);
  } else {
    v = qd_renorm<4>(x);
  }
  const int64_t off = i * C.ld + j;
  if (mode == MODE_ADD) v = N::add(N::load(C.p, off), v);
  else if (mode == MODE_SUB) v = N::add(N::load(C.p, off), N::neg(v));
  N::store(C.p, off, v);
}

// CRT reconstruction constants for N moduli (passed by value).
struct crt_consts {
  uint32_t c[CRT_MAXN][2 * CRT_NW];  // c_t = (M / m_t) ((M / m_t)^-1 mod m_t) as 16-bit digits
  uint32_t M[CRT_NW];
  uint32_t halfM[CRT_NW];        // floor(M / 2)
  double inv_scaled;             // 2^(32 (wt - 2)) / M
  float inv_scaled_f;            // the same in FP32 (the quotient estimate)
  int wt;                        // highest word of sum_t r_t c_t that can be nonzero (>= 2)
};

// C (mode) Z 2^(ea_i + fb_j - 2P), Z from its residues by the CRT:
// S = sum_t r_t c_t (the constants as 16-bit digits: every digit column
// sums below 40 2^24 < 2^30 in a 32-bit register; carries propagated once
// at the end), q = floor(S / M) from
// the three top words (off by at most one, corrected), Z = S - q M in
// [0, M), then Z - M if Z > M / 2; rounded to DD as in the slice scheme.
__global__ void oz_crt_recombine_kernel(int64_t m, int64_t n, int N, int P, int64_t mpad, int64_t npad,
                                        const uint8_t* __restrict__ R, const int* exa, const int* exb,
                                        mat C, int mode, crt_consts cc) {
  using Nm = num<2>;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j >= n || i >= m) return;
  const int64_t plane = mpad * npad;
  uint32_t w[2 * CRT_NW];
#pragma unroll
  for (int k = 0; k < 2 * CRT_NW; ++k) w[k] = 0u;
#pragma unroll
  for (int t = 0; t < CRT_MAXN; ++t) {  // unrolled: static indices into the constants
    if (t < N) {
      const uint32_t r = R[(int64_t)t * plane + i * npad + j];
#pragma unroll
      for (int k = 0; k < 2 * CRT_NW; ++k) w[k] += r * cc.c[t][k];  // < 40 * 2^24
    }
  }
  uint32_t S[CRT_NW];
  uint32_t carry = 0u;
#pragma unroll
  for (int k = 0; k < CRT_NW; ++k) {
    const uint32_t lo = w[2 * k] + carry;             // < 2^31
    const uint32_t hi = w[2 * k + 1] + (lo >> 16);    // < 2^31
    S[k] = (lo & 0xFFFFu) | (hi << 16);
    carry = hi >> 16;
  }
  // q estimate from words wt, wt - 1, wt - 2 (selected without dynamic indexing)
  uint32_t s2 = 0u, s1 = 0u, s0 = 0u;
#pragma unroll
  for (int k = 0; k < CRT_NW; ++k) {
    s2 = k == cc.wt ? S[k] : s2;
    s1 = k == cc.wt - 1 ? S[k] : s1;
    s0 = k == cc.wt - 2 ? S[k] : s0;
  }
  // q < N 2^8 <= 2^14: in FP32 (relative error a few 2^-24, so q is off by
  // less than 2^-8 before the floor, i.e. at most one either way, which the
  // correction below absorbs; all three words count when M is small)
  const float sf = __fmaf_rn(__fmaf_rn(__uint2float_rn(s2), 4294967296.0f, __uint2float_rn(s1)), 4294967296.0f,
                             __uint2float_rn(s0));
  const uint32_t q = (uint32_t)floorf(__fmul_rn(sf, cc.inv_scaled_f));
  // Z = S - q M
  uint32_t Z[CRT_NW];
  unsigned long long pc = 0ull;
  uint32_t borrow = 0u;
#pragma unroll
  for (int k = 0; k < CRT_NW; ++k) {
    const unsigned long long pm = (unsigned long long)q * cc.M[k] + pc;
    pc = pm >> 32;
    const uint32_t sub = (uint32_t)pm;
    const unsigned long long d = (unsigned long long)S[k] - sub - borrow;
    Z[k] = (uint32_t)d;
    borrow = (uint32_t)(d >> 63);
  }
  // correct q by one either way: Z < 0 -> Z += M; Z >= M -> Z -= M
  auto add_m = [&](uint32_t sgn) {  // Z += M (sgn = 0) or Z -= M (sgn = 1)
    const uint32_t msk = 0u - sgn;
    unsigned long long c = sgn;
#pragma unroll
    for (int k = 0; k < CRT_NW; ++k) {
      const unsigned long long v = (unsigned long long)Z[k] + (cc.M[k] ^ msk) + c;
      Z[k] = (uint32_t)v;
      c = v >> 32;
    }
  };
  auto greater = [&](const uint32_t (&b)[CRT_NW]) {  // Z > b (both nonnegative)
    int res = 0;
#pragma unroll
    for (int k = 0; k < CRT_NW; ++k) res = Z[k] > b[k] ? 1 : (Z[k] < b[k] ? -1 : res);
    return res > 0;
  };
  auto is_neg = [&]() { return (Z[CRT_NW - 1] >> 31) != 0u; };
  if (is_neg()) add_m(0u);
  else {
    // Z >= M  <=>  Z > M - 1; compare against M directly
    int res = 0;
#pragma unroll
    for (int k = 0; k < CRT_NW; ++k) res = Z[k] > cc.M[k] ? 1 : (Z[k] < cc.M[k] ? -1 : res);
    if (res >= 0) add_m(1u);
  }
  if (greater(cc.halfM)) add_m(1u);  // symmetric range: Z - M < 0
  const int lsb = (exa[i] - 1022) + (exb[j] - 1022) - 2 * P;
  const uint32_t neg = fx::acc_abs<CRT_NW>(Z);
  uint64_t ch[2];
  int ex[2];
  dd_t v{0.0, 0.0};
  if (fx::acc_chunks<CRT_NW, 2>(Z, ch, ex)) {
    const int e0 = lsb + ex[0];  // chunk 0 in [2^52, 2^53) at 2^e0, chunk 1 at 2^(e0 - 53)
    if (e0 >= -1000 && e0 <= 960) {
      // two_sum(chunk 0, chunk 1) on the integer pipe: the head rounded to
      // nearest (ties to even) at 2^e0, the remainder exact; the same bits
      uint64_t h = ch[0];
      int64_t lo = (int64_t)ch[1];
      const uint64_t half = 1ull << 52;
      if (ch[1] > half || (ch[1] == half && (h & 1ull))) {
        h += 1ull;
        lo -= (int64_t)1 << 53;
      }
      v.hi = fx::make_double(h, e0, neg);
      v.lo = lo == 0 ? 0.0 : fx::make_double((uint64_t)(lo < 0 ? -lo : lo), e0 - 53, neg ^ (lo < 0 ? 1u : 0u));
    } else {
      double x[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int e = lsb + ex[k];
        double w = (ch[k] == 0 || e < -2044) ? 0.0 : fx::pow2_product(__ull2double_rn(ch[k]), e > 2046 ? 2046 : e);
        x[k] = neg ? -w : w;
      }
      two_sum(x[0], x[1], v.hi, v.lo);
    }
  }
  const int64_t off = i * C.ld + j;
  if (mode == MODE_ADD) v = Nm::add(Nm::load(C.p, off), v);
  else if (mode == MODE_SUB) v = Nm::add(Nm::load(C.p, off), Nm::neg(v));
  Nm::store(C.p, off, v);
}

// ------------------------------------------------------------------ host --
static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// The INT8 kernels' shared-memory attribute, once per device (thread-safe).
static void set_gemm_attrs() {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(dev)) return;
  cudaFuncSetAttribute(oz_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
  cudaFuncSetAttribute(oz_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
  done.insert(dev);
}

// Multiword helpers for the CRT constants (little-endian 32-bit words).
using bigw = uint32_t[CRT_NW];
static void big_mul_small(bigw& a, uint32_t k) {
  uint64_t c = 0;
  for (int i = 0; i < CRT_NW; ++i) {
    const uint64_t v = (uint64_t)a[i] * k + c;
    a[i] = (uint32_t)v;
    c = v >> 32;
  }
}
static uint32_t big_div_small(bigw& a, uint32_t k) {  // a /= k, returns a mod k
  uint64_t r = 0;
  for (int i = CRT_NW - 1; i >= 0; --i) {
    const uint64_t v = (r << 32) | a[i];
    a[i] = (uint32_t)(v / k);
    r = v % k;
  }
  return (uint32_t)r;
}
static int big_bitlen(const bigw& a) {
  for (int i = CRT_NW - 1; i >= 0; --i)
    if (a[i]) return 32 * i + 32 - __builtin_clz(a[i]);
  return 0;
}
static uint32_t inv_mod(uint32_t a, uint32_t m) {  // a^-1 mod m (gcd(a, m) = 1), extended Euclid
  int64_t t0 = 0, t1 = 1, r0 = m, r1 = a % m;
  while (r1 != 0) {
    const int64_t q = r0 / r1;
    int64_t x = r0 - q * r1; r0 = r1; r1 = x;
    x = t0 - q * t1; t0 = t1; t1 = x;
  }
  return (uint32_t)((t0 % (int64_t)m + m) % m);
}

// Integer scaling precision for N moduli and inner dimension l:
// P = min(120, floor((bitlen(M) - 2 - ceil(log2 l)) / 2)), so l 2^(2P) < M / 2.
static int crt_precision(int N, int64_t l, crt_consts* cc) {
  bigw M = {0};
  M[0] = 1;
  for (int t = 0; t < N; ++t) big_mul_small(M, (uint32_t)crt_mod(t));
  const int B = big_bitlen(M);
  int clog = 0;
  while (((int64_t)1 << clog) < l) ++clog;
  const int P = std::min(CRT_PMAX, (B - 2 - clog) / 2);
  if (cc) {
    std::memset(cc, 0, sizeof(*cc));
    for (int k = 0; k < CRT_NW; ++k) cc->M[k] = M[k];
    for (int t = 0; t < N; ++t) {
      const uint32_t mt = (uint32_t)crt_mod(t);
      bigw Mt;
      for (int k = 0; k < CRT_NW; ++k) Mt[k] = M[k];
      big_div_small(Mt, mt);  // exact
      bigw tmp;
      for (int k = 0; k < CRT_NW; ++k) tmp[k] = Mt[k];
      const uint32_t y = inv_mod(big_div_small(tmp, mt), mt);
      big_mul_small(Mt, y);
      for (int k = 0; k < CRT_NW; ++k) {
        cc->c[t][2 * k] = Mt[k] & 0xFFFFu;
        cc->c[t][2 * k + 1] = Mt[k] >> 16;
      }
    }
    for (int k = 0; k < CRT_NW; ++k)
      cc->halfM[k] = (M[k] >> 1) | (k + 1 < CRT_NW ? (M[k + 1] << 31) : 0u);
    cc->wt = std::max(2, (B + 13) / 32);
    double md = 0.0;
    for (int k = CRT_NW - 1; k >= 0; --k) md = md * 4294967296.0 + (double)M[k];
    cc->inv_scaled = std::ldexp(1.0 / md, 32 * (cc->wt - 2));
    cc->inv_scaled_f = (float)cc->inv_scaled;
  }
  return P;
}

ddg_status ozaki_gemm(int L, int64_t m, int64_t l, int64_t n, const mat& A, const mat& B, const mat& C,
                      int mode, int s, cudaStream_t st) {
  if (m == 0 || n == 0) return DDG_OK;
  // X < 2^T must fit the digit loop and the split word: T <= 125 (DD, 192
  // bits) or T <= 223 (QD, 288 bits)
  const int smax = L == 2 ? 18 : 32;
  if (s < 2 || s > smax)
    return set_error(DDG_EINVAL, "ozaki slices must be in [2, " + std::to_string(smax) + "]");
  const int64_t mpad = (m + OBM - 1) / OBM * OBM, npad = (n + OBN - 1) / OBN * OBN;
  const int64_t lpad = std::max<int64_t>(OBK, (l + OBK - 1) / OBK * OBK);
  if ((int64_t)s * lpad * 4096 >= ((int64_t)1 << 31))
    return set_error(DDG_EINVAL, "ozaki: s * l too large for exact INT32 accumulation");
  const size_t bA = al256((size_t)s * mpad * lpad), bB = al256((size_t)s * npad * lpad);
  const size_t bD = al256((size_t)s * mpad * npad * 4), bE = al256((size_t)(m + n) * 4);
  void* ws = nullptr;
  if (ddg::ws_alloc(&ws, bA + bB + bD + bE, st) != cudaSuccess) {
    cudaGetLastError();
    return set_error(DDG_ENOMEM, "ozaki: workspace allocation failed");
  }
  char* base = static_cast<char*>(ws);
  int8_t* As = reinterpret_cast<int8_t*>(base);
  int8_t* Bs = reinterpret_cast<int8_t*>(base + bA);
  int32_t* D = reinterpret_cast<int32_t*>(base + bA + bB);
  int* exa = reinterpret_cast<int*>(base + bA + bB + bD);
  int* exb = exa + m;
  set_gemm_attrs();
  cudaEvent_t ev = nullptr;
  auto launched = [&]() { g_launches.fetch_add(1, std::memory_order_relaxed); };
  oz_exp_kernel<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(m, l, A, 1, exa);
  launched();
  oz_exp_kernel<<<(unsigned)((n + 31) / 32), 256, 0, st>>>(l, n, B, 0, exb);
  launched();
  const dim3 ga((unsigned)((lpad + 255) / 256), (unsigned)mpad), gb((unsigned)(npad / 32), (unsigned)(lpad / 32));
  if (L == 2) {
    oz_split_a_kernel<2, false><<<ga, 256, 0, st>>>(m, l, A, exa, s, 0, mpad, lpad, As);
    oz_split_b_kernel<2, false><<<gb, dim3(32, 8), 0, st>>>(l, n, B, exb, s, 0, npad, lpad, Bs);
  } else {
    oz_split_a_kernel<4, false><<<ga, 256, 0, st>>>(m, l, A, exa, s, 0, mpad, lpad, As);
    oz_split_b_kernel<4, false><<<gb, dim3(32, 8), 0, st>>>(l, n, B, exb, s, 0, npad, lpad, Bs);
  }
  launched();
  launched();
  prof_begin_launch(st, &ev);
  oz_gemm_kernel<false><<<dim3((unsigned)(npad / OBN), (unsigned)(mpad / OBM), (unsigned)s), 256, OZ_SMEM, st>>>(
      mpad, npad, lpad, s, As, Bs, D, nullptr);
  launched();
  cudaError_t e = cudaGetLastError();
  if (ev) {
    const double pairs = 0.5 * s * (s + 1);
    prof_end_launch(st, ev, PROF_OZAKI, 2.0 * pairs * (double)mpad * (double)npad * (double)lpad,
                    (double)s * (mpad + npad) * lpad + 4.0 * s * mpad * npad);
  }
  if (e == cudaSuccess) {
    const dim3 gr((unsigned)((n + 255) / 256), (unsigned)m);
    if (L == 2) oz_recombine_kernel<2><<<gr, 256, 0, st>>>(m, n, s, mpad, npad, D, exa, exb, C, mode);
    else oz_recombine_kernel<4><<<gr, 256, 0, st>>>(m, n, s, mpad, npad, D, exa, exb, C, mode);
    launched();
    e = cudaGetLastError();
  }
  ddg::ws_free(ws, st);
  if (e != cudaSuccess) return set_error(DDG_ECUDA, std::string("ozaki: ") + cudaGetErrorString(e));
  return DDG_OK;
}

ddg_status ozaki_crt_gemm(int64_t m, int64_t l, int64_t n, const mat& A, const mat& B, const mat& C, int mode,
                          int N, bool tc, cudaStream_t st) {
  if (m == 0 || n == 0) return DDG_OK;
  if (N < 2 || N > CRT_MAXN)
    return set_error(DDG_EINVAL, "ozaki2: moduli must be in [2, " + std::to_string(CRT_MAXN) + "]");
  const int64_t nb = tc ? 2 * OBN : OBN;  // the tensor-core tiles are 256 columns wide
  const int64_t mpad = (m + OBM - 1) / OBM * OBM, npad = (n + nb - 1) / nb * nb;
  const int64_t lpad = std::max<int64_t>(OBK, (l + OBK - 1) / OBK * OBK);
  if (lpad > 65536) return set_error(DDG_EINVAL, "ozaki2: l must be <= 65536 (exact INT32 residue products)");
  crt_consts cc;
  const int P = crt_precision(N, l, &cc);
  if (P < 1) return set_error(DDG_EINVAL, "ozaki2: too few moduli for this l");
  const size_t esz = tc ? 2 : 1;  // residues as bf16 (tensor cores) or int8 (mma.sync)
  const size_t bA = al256((size_t)N * mpad * lpad * esz), bB = al256((size_t)N * npad * lpad * esz);
  const size_t bR = al256((size_t)N * mpad * npad), bE = al256((size_t)(m + n) * 4);
  void* ws = nullptr;
  if (ddg::ws_alloc(&ws, bA + bB + bR + bE, st) != cudaSuccess) {
    cudaGetLastError();
    return set_error(DDG_ENOMEM, "ozaki2: workspace allocation failed");
  }
  char* base = static_cast<char*>(ws);
  uint8_t* R = reinterpret_cast<uint8_t*>(base + bA + bB);
  int* exa = reinterpret_cast<int*>(base + bA + bB + bR);
  int* exb = exa + m;
  set_gemm_attrs();
  cudaEvent_t ev = nullptr;
  auto launched = [&]() { g_launches.fetch_add(1, std::memory_order_relaxed); };
  nvtxRangePushA(tc ? "ddg.crt split (bf16)" : "ddg.crt split (int8)");
  oz_exp_kernel<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(m, l, A, 1, exa);
  launched();
  oz_exp_kernel<<<(unsigned)((n + 31) / 32), 256, 0, st>>>(l, n, B, 0, exb);
  launched();
  const dim3 ga((unsigned)((lpad + 255) / 256), (unsigned)mpad), gb((unsigned)(npad / 32), (unsigned)(lpad / 32));
  cudaError_t e = cudaSuccess;
  if (tc) {
    __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(base);
    __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(base + bA);
    oz_split_a_kernel<2, true, __nv_bfloat16><<<ga, 256, 0, st>>>(m, l, A, exa, N, P, mpad, lpad, As);
    launched();
    oz_split_b_kernel<2, true, __nv_bfloat16><<<gb, dim3(32, 8), 0, st>>>(l, n, B, exb, N, P, npad, lpad, Bs);
    launched();
    e = cudaGetLastError();
    nvtxRangePop();
    nvtx_range nv("ddg.crt residue products (tcgen05) N %d", N);
    if (e == cudaSuccess) e = launch_crt_tc(N, mpad, npad, lpad, As, Bs, R, st);
  } else {
    int8_t* As = reinterpret_cast<int8_t*>(base);
    int8_t* Bs = reinterpret_cast<int8_t*>(base + bA);
    oz_split_a_kernel<2, true><<<ga, 256, 0, st>>>(m, l, A, exa, N, P, mpad, lpad, As);
    launched();
    oz_split_b_kernel<2, true><<<gb, dim3(32, 8), 0, st>>>(l, n, B, exb, N, P, npad, lpad, Bs);
    launched();
    nvtxRangePop();
    nvtx_range nv("ddg.crt residue products (int8) N %d", N);
    prof_begin_launch(st, &ev);
    oz_gemm_kernel<true><<<dim3((unsigned)(npad / OBN), (unsigned)(mpad / OBM), (unsigned)N), 256, OZ_SMEM, st>>>(
        mpad, npad, lpad, N, As, Bs, nullptr, R);
    launched();
    e = cudaGetLastError();
    if (ev)
      prof_end_launch(st, ev, PROF_OZAKI, 2.0 * N * (double)mpad * (double)npad * (double)lpad,
                      (double)N * (mpad + npad) * lpad + (double)N * mpad * npad);
  }
  if (e == cudaSuccess) {
    nvtx_range nv2("ddg.crt reconstruction");
    const dim3 gr((unsigned)((n + 255) / 256), (unsigned)m);
    oz_crt_recombine_kernel<<<gr, 256, 0, st>>>(m, n, N, P, mpad, npad, R, exa, exb, C, mode, cc);
    launched();
    e = cudaGetLastError();
  }
  ddg::ws_free(ws, st);
  if (e != cudaSuccess) return set_error(DDG_ECUDA, std::string("ozaki2: ") + cudaGetErrorString(e));
  return DDG_OK;
}

int ozaki_crt_precision(int N, int64_t l) { return crt_precision(N, l, nullptr); }

}  // namespace ddg
