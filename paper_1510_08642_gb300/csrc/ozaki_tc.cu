// Residue products of the CRT DD product (Ozaki scheme II) on the
// fifth-generation tensor cores: tcgen05.mma kind::f16 with BF16 operands
// and FP32 accumulation in tensor memory, operands staged by TMA.
//
// The DD product C := A B (Kouya 2015, Section 2, Eq. 1) by the Chinese
// remainder theorem (ozaki.cu) needs, for every modulus m_t, the integer
// matrix product of the residue matrices X mod m_t (m x l) and Y mod m_t
// (l x n), reduced mod m_t. Balanced residues lie in [-128, 127], so they
// are exact BF16 values and each product a_ik b_kj is an integer of
// magnitude <= 2^14. Summed in FP32, 256 such terms stay within 2^22 and
// every partial sum is an exactly representable integer, whatever the
// order or the alignment the tensor core uses; so the k loop runs in chunks
// of 256 terms, each chunk accumulated in tensor memory from zero and then
// drained exactly into 32-bit integer sums in registers (x + 1.5 2^23 holds
// the integer x in its low bits for |x| <= 2^22). The integer sums
// (|sum| <= l 2^14 <= 2^30) are reduced mod m_t and stored as bytes, the
// same residues the INT8 mma.sync kernel writes; the CRT reconstruction
// that follows is shared.
//
// Kernel layout (one persistent CTA per SM, 320 threads; tiles of 128 rows
// of A by 256 columns of B, so that a 48 KB stage feeds twice the MMA work
// of a 128 x 128 tile for 1.5 times the bytes):
//   warp 0: TMA producer (one lane): 64-wide k blocks of A (128 rows) and B
//           (256 rows of the transposed B) as 128 x 64 BF16 boxes
//           (128-byte rows, 128-byte swizzle) into a ring of 4 stages;
//   warp 1: allocates all 512 tensor-memory columns (two 128 x 256 FP32
//           accumulators) and issues the MMAs (one lane): per k block four
//           128 x 256 x 16 MMAs, per 256-term chunk one accumulator,
//           alternating, so that the drain of one chunk overlaps the MMAs
//           of the next;
//   warps 2-9: drain: warp w reads lanes 32 (w mod 4) .. + 31 of the
//           accumulator (one row of the tile per thread, tcgen05.ld
//           32x32b), columns 128 ((w - 2) / 4) .. + 127, adds the chunk
//           into 128 integer sums, releases the accumulator; at the end of
//           a tile reduces mod m_t and writes its 128 residues of the row.
// Tiles (modulus t, 128-row block, 256-column block) are taken in that
// order, CTA b taking tiles b, b + gridDim.x, ... (no CTA waits on another):
// consecutive tiles share a modulus, so the 152 resident tiles read one
// modulus's residue planes (2 x 32 MB at n = 4096) through the L2.
// Every wait on an mbarrier gives up after a bounded number of tries; the
// CTA then records the timeout, lets its copies and MMAs in flight finish,
// frees its tensor memory and returns.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched at run time)
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "crt.cuh"
#include "kernels.cuh"

namespace ddg {

namespace {

constexpr int TBM = 128, TBN = 256, TBK = 64;  // tile; a k block is one 128-byte BF16 row
constexpr int TST = 4;                          // shared-memory stages (48 KB each)
constexpr int DRAIN_WARPS = 8;                  // two per tensor-memory lane quarter
constexpr int DCOLS = TBN / 2;                  // accumulator columns per draining warp
constexpr int TCHUNK = 256;                     // terms per exact FP32 accumulation
constexpr int KB_PER_CHUNK = TCHUNK / TBK;
constexpr int A_BYTES = TBM * TBK * 2, B_BYTES = TBN * TBK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 2 * TBN;
constexpr int TC_THREADS = 32 * (2 + DRAIN_WARPS);
// barriers: full[TST], empty[TST], acc_full[2], acc_empty[2], drained; then
// the tensor-memory address and the abort flag
constexpr int BAR_BYTES = 8 * (2 * TST + 5) + 8;
constexpr int TC_SMEM = 1024 + TST * STAGE_BYTES + BAR_BYTES;
constexpr uint32_t WAIT_TRIES = 1u << 22;  // ~ seconds with the suspend hint below

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                           ((uint32_t)(TBM >> 4) << 24);

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzle: start address >> 4 (bits 0-13), leading byte offset
// 16 >> 4 (bits 16-29; unused for this layout), stride byte offset 1024 >> 4
// between 8-row groups (bits 32-45), the constant 0b001 (bits 46-48),
// swizzle mode 2 = 128 bytes (bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Wait for the phase of parity `parity` of the barrier; false if the CTA
// was aborted or the wait ran out (then the CTA is aborted and the timeout
// counted).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, int* timeouts) {
  for (uint32_t i = 0; i < WAIT_TRIES; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (*abort) return false;
    if (i > 16) __nanosleep(256);
  }
  *abort = 1;
  atomicAdd(timeouts, 1);
  return false;
}

// The same wait ignoring the abort flag (draining work in flight on exit).
__device__ __forceinline__ void mbar_wait_exit(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < WAIT_TRIES; ++i) {
    if (mbar_try(bar, parity)) return;
    if (i > 16) __nanosleep(256);
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}

// Arrive once on the barrier when every tcgen05.mma issued so far by this
// thread has completed.
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 32 consecutive 32-bit columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct tc_args {
  int64_t mt, nt;      // 128-row / 128-column blocks per modulus
  int64_t mpad, npad;  // rows of one modulus's A plane / B plane
  int kblocks;         // lpad / 64
  int N;               // moduli
  uint8_t* R;          // residues of the product: N planes of mpad x npad bytes
  int* timeouts;       // incremented by a CTA whose wait ran out
  int idle_producer;   // test support: 1 = the TMA producer issues nothing
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    crt_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, tc_args g) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment for the 128-byte swizzle atoms
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sbase = smem_raw + (base - raw);
  const uint32_t bars = base + TST * STAGE_BYTES;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (TST + s); };
  auto acc_full = [&](int b) { return bars + 8u * (2 * TST + b); };
  auto acc_empty = [&](int b) { return bars + 8u * (2 * TST + 2 + b); };
  const uint32_t drained = bars + 8u * (2 * TST + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sbase + TST * STAGE_BYTES + 8 * (2 * TST + 5));
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t per_mod = g.mt * g.nt, total = per_mod * g.N;
  const int nchunks = (g.kblocks + KB_PER_CHUNK - 1) / KB_PER_CHUNK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TST; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), DRAIN_WARPS);  // one arrival per draining warp
    }
    mbar_init(drained, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    if (lane == 0 && !g.idle_producer) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      uint32_t armed = 0, armed_par = 0;  // stages armed, and the parity of their last arming
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < total && ok; tile += gridDim.x) {
        const int64_t t = tile / per_mod, rem = tile % per_mod;
        const int ya = (int)(t * g.mpad + (rem / g.nt) * TBM);
        const int yb = (int)(t * g.npad + (rem % g.nt) * TBN);
        for (int kb = 0; kb < g.kblocks; ++kb) {
          if (!mbar_wait(empty(stage), phase ^ 1u, abort, g.timeouts)) {
            ok = false;
            break;
          }
          const uint32_t sa = base + stage * STAGE_BYTES;
          mbar_expect_tx(full(stage), STAGE_BYTES);
          tma_load_2d(sa, &tmA, kb * TBK, ya, full(stage));
          tma_load_2d(sa + A_BYTES, &tmB, kb * TBK, yb, full(stage));
          tma_load_2d(sa + A_BYTES + B_BYTES / 2, &tmB, kb * TBK, yb + TBN / 2, full(stage));
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          if (++stage == TST) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // the copies this thread started have landed before the CTA leaves
      for (int s = 0; s < TST; ++s)
        if ((armed >> s) & 1u) mbar_wait_exit(full(s), (armed_par >> s) & 1u);
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------- MMA issue
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t accn = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < total && ok; tile += gridDim.x) {
        for (int c = 0; c < nchunks && ok; ++c, ++accn) {
          const uint32_t b = accn & 1u, use = accn >> 1;
          if (!mbar_wait(acc_empty(b), (use & 1u) ^ 1u, abort, g.timeouts)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + b * TBN;
          const int kb0 = c * KB_PER_CHUNK, kb1 = min(g.kblocks, kb0 + KB_PER_CHUNK);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(full(stage), phase, abort, g.timeouts)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = base + stage * STAGE_BYTES;
            const uint64_t da = sdesc(sa), db = sdesc(sa + A_BYTES);
#pragma unroll
            for (int kk = 0; kk < TBK / 16; ++kk)  // 16 BF16 = 32 bytes further along the swizzled row
              tc_mma(d, da + 2u * kk, db + 2u * kk, (kb > kb0 || kk > 0) ? 1u : 0u);
            tc_commit(empty(stage));  // the stage is free once these MMAs have read it
            if (++stage == TST) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (ok) tc_commit(acc_full(b));
        }
      }
      // every MMA issued by this thread has completed before TMEM is freed
      tc_commit(drained);
      mbar_wait_exit(drained, 0);
    }
  } else {
    // --------------------------------------------------------------- drain
    const int q = warp & 3;                 // lanes 32 q .. 32 q + 31 of tensor memory
    const int h = (warp - 2) >> 2;          // columns h DCOLS .. h DCOLS + DCOLS - 1
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * DCOLS);
    uint32_t accn = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < total && ok; tile += gridDim.x) {
      int sum[DCOLS];
#pragma unroll
      for (int j = 0; j < DCOLS; ++j) sum[j] = 0;
      for (int c = 0; c < nchunks; ++c, ++accn) {
        const uint32_t b = accn & 1u, use = accn >> 1;
        // a warp-uniform outcome: the loads below are .sync.aligned
        if (!__all_sync(0xffffffffu, mbar_wait(acc_full(b), use & 1u, abort, g.timeouts))) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int piece = 0; piece < DCOLS / 32; ++piece) {
          uint32_t v[32];
          tc_ld32(lane_base + b * TBN + piece * 32, v);
#pragma unroll
          for (int j = 0; j < 32; ++j)  // exact: |v| <= 2^22
            sum[piece * 32 + j] += __float_as_int(__fadd_rn(__uint_as_float(v[j]), 12582912.0f)) - 0x4B400000;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty(b));
      }
      if (!ok) break;
      const int64_t t = tile / per_mod, rem = tile % per_mod;
      const int64_t row = (rem / g.nt) * TBM + q * 32 + lane, col0 = (rem % g.nt) * TBN + h * DCOLS;
      const uint32_t m = c_crt_red.m[t], magic = c_crt_red.magic[t], bias = c_crt_red.bias[t];
      uint4* out = reinterpret_cast<uint4*>(g.R + (t * g.mpad + row) * g.npad + col0);
#pragma unroll
      for (int v16 = 0; v16 < DCOLS / 16; ++v16) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uint32_t word = 0u;
#pragma unroll
          for (int bb = 0; bb < 4; ++bb) {
            const uint32_t u = (uint32_t)sum[v16 * 16 + e * 4 + bb] + bias;
            uint32_t x = u - __umulhi(u, magic) * m;
            x = x >= m ? x - m : x;
            word |= x << (8 * bb);
          }
          w[e] = word;
        }
        out[v16] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// cuTensorMapEncodeTiled, fetched from the driver once.
typedef CUresult (*encode_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_fn get_encoder() {
  static std::once_flag once;
  static encode_fn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<encode_fn>(p);
  });
  return fn;
}

// A rows x lpad BF16 plane set (rows = N planes stacked) as a 2D tensor with
// 64 x 128 boxes and 128-byte swizzle.
bool make_map(CUtensorMap* map, const __nv_bfloat16* p, int64_t rows, int64_t lpad) {
  encode_fn enc = get_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)lpad, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)lpad * 2};
  const cuuint32_t box[2] = {TBK, 128};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

__device__ int g_tc_timeouts;

}  // namespace

cudaError_t launch_crt_tc(int N, int64_t mpad, int64_t npad, int64_t lpad, const void* As_, const void* Bs_,
                          uint8_t* R, cudaStream_t st) {
  const __nv_bfloat16* As = static_cast<const __nv_bfloat16*>(As_);
  const __nv_bfloat16* Bs = static_cast<const __nv_bfloat16*>(Bs_);
  if (mpad % TBM || npad % TBN || lpad % TBK || N < 1 || N > CRT_MAXN) return cudaErrorInvalidValue;
  if ((int64_t)N * mpad > INT32_MAX || (int64_t)N * npad > INT32_MAX) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, As, (int64_t)N * mpad, lpad) || !make_map(&mb, Bs, (int64_t)N * npad, lpad))
    return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  {
    static std::mutex mu;
    static bool attr_set[64];
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
      const cudaError_t a = cudaFuncSetAttribute(crt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
      if (a != cudaSuccess) return a;
      attr_set[dev] = true;
    }
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  int* timeouts = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&timeouts), g_tc_timeouts);
  if (e != cudaSuccess) return e;
  tc_args a{mpad / TBM, npad / TBN, mpad, npad, (int)(lpad / TBK), N, R, timeouts, 0};
  const int64_t tiles = a.mt * a.nt * N;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, sms);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEvent_t ev = nullptr;
  prof_begin_launch(st, &ev);
  crt_tc_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(ma, mb, a);
  e = cudaGetLastError();
  if (ev)
    prof_end_launch(st, ev, PROF_TENSOR, 2.0 * N * (double)mpad * (double)npad * (double)lpad,
                    2.0 * N * (mpad + npad) * (double)lpad + (double)N * mpad * npad);
  return e;
}

// Test support: one CTA of the kernel on a 128 x 64 x 256 problem with its
// TMA producer idle, so that the MMA thread's wait on the first stage runs
// out; synchronous. Returns the CUDA status of the launch and the wait.
cudaError_t crt_tc_wait_test() {
  __nv_bfloat16 *a = nullptr, *b = nullptr;
  uint8_t* r = nullptr;
  cudaError_t e = cudaMalloc(&a, 128 * 64 * 2);
  if (e == cudaSuccess) e = cudaMalloc(&b, TBN * 64 * 2);
  if (e == cudaSuccess) e = cudaMalloc(&r, 128 * TBN);
  if (e == cudaSuccess) e = cudaMemset(a, 0, 128 * 64 * 2);
  if (e == cudaSuccess) e = cudaMemset(b, 0, TBN * 64 * 2);
  CUtensorMap ma, mb;
  if (e == cudaSuccess && (!make_map(&ma, a, 128, 64) || !make_map(&mb, b, TBN, 64))) e = cudaErrorInvalidValue;
  int* timeouts = nullptr;
  if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&timeouts), g_tc_timeouts);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(crt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e == cudaSuccess) {
    tc_args t{1, 1, 128, TBN, 1, 1, r, timeouts, 1};
    g_launches.fetch_add(1, std::memory_order_relaxed);
    crt_tc_kernel<<<1, TC_THREADS, TC_SMEM>>>(ma, mb, t);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(a);
  cudaFree(b);
  cudaFree(r);
  return e;
}

int crt_tc_timeouts(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_timeouts, sizeof(int)) != cudaSuccess) return -1;
  if (reset) {
    const int z = 0;
    cudaMemcpyToSymbol(g_tc_timeouts, &z, sizeof(int));
  }
  return v;
}

}  // namespace ddg
