// Internal interface between the C-ABI layer and the CUDA kernels.
#pragma once

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace ddg {

// NVTX range over a scope of host code that issues work (a product, a
// recursion level, a fused pass, a CRT stage, an LU phase); a no-op unless
// a profiler that records NVTX is attached.
struct nvtx_range {
  explicit nvtx_range(const char* name) { nvtxRangePushA(name); }
  template <class... Args>
  nvtx_range(const char* fmt, Args... args) {
    char buf[96];
    std::snprintf(buf, sizeof(buf), fmt, args...);
    nvtxRangePushA(buf);
  }
  ~nvtx_range() { nvtxRangePop(); }
  nvtx_range(const nvtx_range&) = delete;
  nvtx_range& operator=(const nvtx_range&) = delete;
};

// A matrix of L limb planes (L = 2 for DD, 4 for QD), each row-major with
// leading dimension ld (in doubles). Unused plane pointers are null.
struct mat {
  double* p[4];
  int64_t ld;
};

inline mat view(const mat& M, int64_t r0, int64_t c0) {
  mat v = M;
  for (int k = 0; k < 4; ++k)
    if (v.p[k]) v.p[k] += r0 * M.ld + c0;
  return v;
}

// Count of kernel launches issued by the library (all kernels, all threads).
extern std::atomic<uint64_t> g_launches;

// Launch profiling hooks (profile.cu); no-ops unless ddg_profile_begin ran.
enum ProfKind {
  PROF_SIMPLE = 0, PROF_BLOCK = 1, PROF_PASS = 2, PROF_OZAKI = 3, PROF_GEMV = 4, PROF_CONVERT = 5,
  PROF_TENSOR = 6  // tcgen05 residue products
};
bool prof_enabled();
void prof_begin_launch(cudaStream_t s, cudaEvent_t* start);
void prof_end_launch(cudaStream_t s, cudaEvent_t start, int kind, double ops, double bytes);

enum Mode { MODE_SET = 0, MODE_ADD = 1, MODE_SUB = 2 };

// Quadrant pass kinds (fused add/sub passes of one recursion level).
enum PassKind {
  PASS_WINOGRAD_A = 0,  // S1..S4 from A11, A12, A21, A22
  PASS_WINOGRAD_B = 1,  // T1..T4 from B11, B12, B21, B22
  PASS_WINOGRAD_C = 2,  // C11..C22 from P1..P7
  PASS_STRASSEN_A = 3,  // five left operands of M1..M7
  PASS_STRASSEN_B = 4,  // five right operands of M1..M7
  PASS_STRASSEN_C = 5,  // C11..C22 from M1..M7
  PASS_COMBINE = 6,     // C := C (+/-) X  (used after padding)
};

// Eq. 1 Simple product, one thread per c_ij, k ascending (pinned sequence).
cudaError_t launch_simple(int limbs, int64_t m, int64_t l, int64_t n, mat A, mat B, mat C,
                          int mode, cudaStream_t s);

// Block product C (mode) A B on CTA tiles (the recursion base case).
// launch_block: TwoSum accumulation on the FP64 pipe (block.cu);
// launch_block_fx: exact fixed-point accumulation of the leading products on
// the integer pipe (block_fx.cu).
cudaError_t launch_block_fx(int limbs, int64_t m, int64_t l, int64_t n, mat A, mat B, mat C,
                            int mode, cudaStream_t s);
int block_fx_fp64_ops_per_mac(int limbs);

// Operands converted to fixed-point words once (launch_fx_convert), for the
// Block kernel on converted operands (launch_block_fxc): element (r, c) of a
// rows x cols operand has its 16-byte word vectors at w[(r ld + c) WV + v]
// (WV = 1 for DD, 2 for QD), and at f[r ld + c] its leading limb's exponent
// field (>= 1) | sign << 16, or FX_ZERO for a zero; ld = cols.
struct fxop {
  const uint4* w;
  const int* f;
  int64_t ld;
};
constexpr int FX_ZERO = (int)0x80000000u;
constexpr int FX_CONV_MAX = 14;  // operands per conversion launch
struct fx_conv_job {
  int64_t rows, cols;
  mat X;
  uint4* w;
  int* f;
};
struct fx_conv_jobs {
  fx_conv_job job[FX_CONV_MAX];
  int count;
};
// Device bytes of one converted rows x cols operand (256-byte multiple).
size_t fxop_bytes(int limbs, int64_t rows, int64_t cols);
// Convert `count` <= FX_CONV_MAX operands X[t] (rows[t] x cols[t]) in one
// launch into buf[t] (fxop_bytes each, 256-byte aligned); out[t] describes
// the result.
cudaError_t launch_fx_convert(int limbs, int count, const int64_t* rows, const int64_t* cols, const mat* X,
                              char* const* buf, fxop* out, cudaStream_t s);
// The Block product on converted operands, the same bits as launch_block_fx:
// count <= FXC_GROUP_MAX products C[t] (mode) A[t] B[t] of one shape in one
// launch (blockIdx.z = t).
constexpr int FXC_GROUP_MAX = 7;
struct fxc_group {
  fxop A[FXC_GROUP_MAX], B[FXC_GROUP_MAX];
  mat C[FXC_GROUP_MAX];
};
cudaError_t launch_block_fxc(int limbs, int64_t m, int64_t l, int64_t n, const fxop* Ax, const fxop* Bx,
                             const mat* C, int count, int mode, cudaStream_t s);
// Both steps for one product, scratch = block_fx_scratch_bytes (used in
// stream order on s). block_fx_converts: whether the shape gains from it
// (a tile of A is otherwise converted by each of the n / BN CTAs that stage
// it, a tile of B by m / BM).
bool block_fx_converts(int limbs, int64_t m, int64_t l, int64_t n);
size_t block_fx_scratch_bytes(int limbs, int64_t m, int64_t l, int64_t n);
cudaError_t launch_block_fx_converted(int limbs, int64_t m, int64_t l, int64_t n, mat A, mat B, mat C, int mode,
                                      void* scratch, cudaStream_t s);

// The same product for n <= GEMV_MAX_N columns: one warp per output, lanes
// splitting k (gemv_fx.cu); the Block base case dispatches to it.
constexpr int64_t GEMV_MAX_N = 8;
cudaError_t launch_gemv_fx(int limbs, int64_t m, int64_t l, int64_t n, mat A, mat B, mat C, int mode,
                           cudaStream_t s);

// One product of a grouped launch (device-resident task list). Tiles are
// numbered consecutively: task t owns tiles [tile0, tile0 + tiles_m tiles_n).
struct gtask {
  int64_t m, l, n;
  mat A, B, C;
  int mode;
  int tiles_n;
  int64_t tile0;
  int limbs;  // 2 or 4; read by the mixed launch (launch_grouped_mixed) only
};
// DD and QD tasks of one list in one persistent launch (tiles converted as
// they are staged; each task's tiles numbered with its own limb count's
// tile shape, fx_tile_shape).
cudaError_t launch_grouped_mixed(const gtask* tasks, int ntasks, int64_t total_tiles, unsigned long long* counter,
                                 double ops, cudaStream_t s);
void fx_tile_shape(int limbs, int* bm, int* bn);

// Grouped conversion (batch plans): operand t (rows x cols of X) into w, f
// (fxop layout, ld = cols), owning the tiles [tile0, tile0 + rows tiles_x)
// of one row by 256 columns (convert_tiles).
struct fx_ctask {
  int64_t rows, cols;
  mat X;
  uint4* w;
  int* f;
  int64_t tile0;
  int64_t tiles_x;
};
int64_t convert_tiles(int64_t rows, int64_t cols);
cudaError_t launch_grouped_convert(int limbs, const fx_ctask* tasks, int ntasks, int64_t total_tiles, double elems,
                                   cudaStream_t s);
// One product of a grouped launch on converted operands (tiles as gtask).
struct gctask {
  int64_t m, l, n;
  fxop A, B;
  mat C;
  int mode;
  int tiles_n;
  int64_t tile0;
};
cudaError_t launch_grouped_fxc(int limbs, const gctask* tasks, int ntasks, int64_t total_tiles,
                               unsigned long long* counter, double ops, cudaStream_t s);
cudaError_t launch_grouped_fx(int limbs, const gtask* tasks, int ntasks, int64_t total_tiles,
                              unsigned long long* counter, double ops, cudaStream_t s);
cudaError_t launch_block(int limbs, int64_t m, int64_t l, int64_t n, mat A, mat B, mat C,
                         int mode, cudaStream_t s);

// Operands of one fused pass: up to 7 input and 5 output quadrants.
struct pass_args {
  mat in[7];
  mat out[5];
};

// One pass of a grouped launch: tiles of 8 x 32 elements numbered from tile0.
struct ptask {
  int64_t rows, cols;
  pass_args a;
  int mode;
  int tiles_x;
  int64_t tile0;
};
cudaError_t launch_grouped_pass(int limbs, int kind, const ptask* tasks, int ntasks, int64_t total_tiles,
                                cudaStream_t s);

// One fused quadrant pass over a rows x cols quadrant grid.
cudaError_t launch_pass(int limbs, int kind, int64_t rows, int64_t cols, const mat* in, int nin,
                        const mat* out, int nout, int mode, cudaStream_t s);

// FP64 instructions of one accurate DD / QD addition as used by the passes.
int add_fp64_ops(int limbs);

}  // namespace ddg

#include "ddgemm.h"

namespace ddg {

// Error text of the calling host thread (ddg_last_error).
void clear_error();
ddg_status set_error(ddg_status st, const std::string& msg);

// Temporaries of a call: the library's workspace pool of the current device
// (pool.cu), stream-ordered like cudaMallocAsync / cudaFreeAsync.
cudaError_t ws_alloc(void** p, size_t bytes, cudaStream_t s);
cudaError_t ws_free(void* p, cudaStream_t s);

// C (mode) A B with options o (validated by the caller): the body of
// dd_gemm / qd_gemm, used by the LU routines.
ddg_status gemm_run(int L, int64_t m, int64_t l, int64_t n, const mat& A, const mat& B, const mat& C,
                    int mode, const ddg_opts& o, cudaStream_t s);

// DD product by residues and the Chinese remainder theorem (Ozaki scheme
// II), N moduli (ozaki.cu); the residue products on the INT8 mma.sync path
// (tc = false) or as BF16 on the tcgen05 tensor cores (tc = true, the same
// bits); the integer scaling precision it uses.
ddg_status ozaki_crt_gemm(int64_t m, int64_t l, int64_t n, const mat& A, const mat& B, const mat& C, int mode,
                          int N, bool tc, cudaStream_t st);

// The tcgen05 residue products (ozaki_tc.cu): N BF16 residue planes of A
// (mpad x lpad, k contiguous) and of B (npad x lpad, B transposed) in, N
// byte planes of the product's residues (mpad x npad) out; mpad, npad
// multiples of 128, lpad a multiple of 64 and <= 65536. crt_tc_timeouts:
// how many CTAs of that kernel gave up a bounded wait (reset: set to 0).
cudaError_t launch_crt_tc(int N, int64_t mpad, int64_t npad, int64_t lpad, const void* As, const void* Bs,
                          uint8_t* R, cudaStream_t st);
int crt_tc_timeouts(bool reset);
cudaError_t crt_tc_wait_test();     // test support (ozaki_tc.cu)
ddg_status lu_panel_wait_test();    // test support (lu.cu)
int ozaki_crt_precision(int N, int64_t l);

// DD / QD product by INT8 slices (Ozaki scheme), s slices (ozaki.cu).
ddg_status ozaki_gemm(int L, int64_t m, int64_t l, int64_t n, const mat& A, const mat& B, const mat& C,
                      int mode, int s, cudaStream_t st);

// Number of FP64 instructions of one multiply-accumulate in the Block
// kernel's inner loop (counted from its source), for the roofline.
int block_fp64_ops_per_mac(int limbs);

}  // namespace ddg
