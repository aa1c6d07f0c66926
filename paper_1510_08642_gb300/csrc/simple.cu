// Simple product (Kouya 2015, Section 2, Eq. 1): c_ij = sum_{k=1..l} a_ik b_kj.
//
// One thread per output entry; k runs in ascending order and each term is one
// DD/QD multiply followed by one DD/QD add, with c_ij starting from zero (or
// from C for the update modes). With the operation sequences pinned in
// arith.cuh this reproduces a plain CPU triple loop bit for bit. It is the
// reference-order kernel, not a fast one: the paper's Table 1 shows the same
// loop is the slowest of the four algorithms.
#include "arith.cuh"
#include "kernels.cuh"

namespace ddg {

template <int L>
__global__ void __launch_bounds__(256) simple_kernel(int64_t m, int64_t l, int64_t n, mat A,
                                                     mat B, mat C, int mode) {
  using N = num<L>;
  const int64_t j = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t i = (int64_t)blockIdx.y * 8 + threadIdx.y;
  if (i >= m || j >= n) return;
  typename N::T c = mode == MODE_SET ? N::zero() : N::load(C.p, i * C.ld + j);
  for (int64_t k = 0; k < l; ++k) {
    typename N::T a = N::load(A.p, i * A.ld + k);
    if (mode == MODE_SUB) a = N::neg(a);
    typename N::T b = N::load(B.p, k * B.ld + j);
    c = N::add(c, N::mul(a, b));
  }
  N::store(C.p, i * C.ld + j, c);
}

cudaError_t launch_simple(int limbs, int64_t m, int64_t l, int64_t n, mat A, mat B, mat C,
                          int mode, cudaStream_t s) {
  if (m == 0 || n == 0) return cudaSuccess;
  dim3 block(32, 8);
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + 7) / 8));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(s, &ev);
  if (limbs == 2) simple_kernel<2><<<grid, block, 0, s>>>(m, l, n, A, B, C, mode);
  else simple_kernel<4><<<grid, block, 0, s>>>(m, l, n, A, B, C, mode);
  cudaError_t e = cudaGetLastError();
  if (ev) {
    const double macs = (double)m * (double)l * (double)n;
    // DD multiply 7 + accurate add 20; QD by the op counts of arith.cuh
    prof_end_launch(s, ev, PROF_SIMPLE, macs * (limbs == 2 ? 27.0 : 218.0),
                    8.0 * limbs * ((double)m * l * n * 2 + (double)m * n));
  }
  return e;
}

}  // namespace ddg
