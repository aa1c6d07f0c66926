/*
 * ddgemm: double-double (DD, 106-bit) and quad-double (QD, 212-bit) dense
 * matrix products and LU solves on one GB300 GPU (sm_103a).
 *
 * The operations are those of T. Kouya, "Performance evaluation of multiple
 * precision matrix multiplications using parallelized Strassen and Winograd
 * algorithms" (2015):
 *   - C := A B of any m x l x n (Section 2, Eq. 1) by the Simple, Block,
 *     Strassen and Winograd algorithms (Section 2; Section 3 names the
 *     recursion cutoff n_min, at which the self-recursive call stops);
 *   - LU decomposition whose trailing update A22 := A22 - L21 U12 is such a
 *     product (Section 4, steps 1-3), and the solution of A x = b (Eq. 2).
 *
 * Conventions for every entry point
 *   - A DD matrix is two row-major planes of doubles in device memory (hi and
 *     lo), a QD matrix four (x[0] leading .. x[3]); element (i, j) of plane p
 *     is p[i * ld + j], with ld >= number of columns (ld >= 1). The value of
 *     an entry is the exact sum of its limbs; inputs are expected normalised
 *     (|lo| <= ulp(hi)/2, and likewise between QD limbs); non-finite values
 *     give undefined results (they are not checked).
 *   - The caller owns all matrices. The library owns nothing it returns:
 *     temporary storage for a call is taken from the library's
 *     stream-ordered workspace pool of the current device (see
 *     ddg_workspace_reserve) on the call's stream and released on it before
 *     the call's work completes. The current device must be the one that
 *     `stream` and the matrices belong to.
 *   - Calls are asynchronous with respect to the host: work is queued on
 *     `stream` (a cudaStream_t, NULL = the legacy default stream) and may
 *     fork onto library-owned streams that join back into `stream`. Results
 *     are ready when `stream` reaches the point after the call.
 *   - Errors are returned as a status code, never by aborting; a
 *     human-readable message for the last failing call on the calling host
 *     thread is available from ddg_last_error(). A status other than DDG_OK
 *     means that no work, or not all of it, was queued.
 *   - Sizes of zero are valid and queue nothing (C := A B with l = 0 writes
 *     zeros for mode DDG_SET). Negative sizes, ld smaller than the column
 *     count, null planes of a non-empty matrix and C overlapping A or B are
 *     DDG_EINVAL.
 *   - The library keeps per-device state for the life of the process (its
 *     forked streams, its workspace pool, the address of the fixed array of
 *     dd_gemm_noalloc), made in the device's primary context: do not call
 *     it again in a process after cudaDeviceReset.
 */
#ifndef DDGEMM_H
#define DDGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DDG_OK = 0,
  DDG_EINVAL = 1,    /* invalid argument */
  DDG_ENOMEM = 2,    /* device memory for temporaries could not be had */
  DDG_ECUDA = 3,     /* a CUDA call failed; see ddg_last_error() */
  DDG_ESINGULAR = 4, /* LU: an exactly zero pivot */
  DDG_ETIMEOUT = 5,  /* a bounded device-side wait ran out */
  DDG_ENOTSUP = 6    /* combination not supported */
} ddg_status;

/* Section 2: the four algorithms the paper compares. */
typedef enum {
  DDG_SIMPLE = 0,   /* Eq. 1, one thread per c_ij, k ascending: bit-exact
                       reference order (the DD/QD multiply then add of each
                       term is the pinned sequence documented with the
                       kernels) */
  DDG_BLOCK = 1,    /* C_ij = sum_k A_ik B_kj over register/shared tiles
                       (for n <= 8 columns: one warp per c_ij, its lanes
                       splitting k, same arithmetic) */
  DDG_STRASSEN = 2, /* Strassen 1969: 7 products, 18 quadrant sums per level */
  DDG_WINOGRAD = 3, /* Winograd's variant: 7 products, 15 quadrant sums */
  DDG_OZAKI = 4     /* not in the paper (the Ozaki scheme): A and B split
                       exactly into `slices` INT8 digit matrices per row /
                       column scale (balanced base 128), slice products on the
                       INT8 tensor cores with INT32 accumulation, recombined
                       exactly and rounded to DD / QD. Error <= l (s + 3)
                       2^-7s max|a_i.| max|b_.j| per entry (normwise, not
                       elementwise, DD / QD accuracy); slices * l < 2^19,
                       m <= 65535 */,
  DDG_OZAKI2 = 5    /* not in the paper (Ozaki scheme II, Ozaki, Uchino and
                       Imamura 2025), DD only: rows of A / columns of B scaled
                       and rounded to integers of P bits, one INT8 product of
                       their residues per modulus (`slices` = the number N of
                       pairwise-coprime moduli <= 256), the integer product
                       recovered exactly by the Chinese remainder theorem and
                       rounded to DD. Error <= l 2^-P max|a_i.| max|b_.j| per
                       entry plus the DD rounding, P from
                       ddg_ozaki2_precision (N = 32, l = 4096: P = 113);
                       l <= 65536, m <= 65535; QD gives DDG_ENOTSUP */,
  DDG_OZAKI2_TC = 6 /* DDG_OZAKI2 with its residue products on the
                       fifth-generation tensor cores (not in the paper):
                       residues as BF16 (exact for |r| <= 128), tcgen05.mma
                       with FP32 accumulation in tensor memory, drained into
                       integers every 256 terms (exact: partial sums stay
                       integers below 2^22), operands staged by TMA. The
                       residues of the product, hence C, are the same bits
                       as DDG_OZAKI2; same limits (DD only, l <= 65536,
                       m <= 65535). The residue planes take 2 bytes per
                       element per modulus (twice DDG_OZAKI2's). */
} ddg_algo;

/* How C is written: C := A B, C := C + A B or C := C - A B. */
typedef enum { DDG_SET = 0, DDG_ADD = 1, DDG_SUB = 2 } ddg_mode;

typedef struct {
  double* hi;
  double* lo;
  int64_t ld;
} dd_mat;

typedef struct {
  double* x[4];
  int64_t ld;
} qd_mat;

typedef struct {
  int32_t algo;    /* ddg_algo */
  int32_t cutoff;  /* n_min (Section 3): a Strassen/Winograd level splits the
                      problem while min(m, l, n) > cutoff; >= 1 */
  int32_t pad;     /* odd dimensions: 0 = peel the last row/column and fix up
                      with Block products (default), 1 = zero-pad to a
                      multiple of 2^depth before recursing */
  int32_t streams; /* 1 = the 7 sub-products of the top level run in order on
                      `stream`; 7 (default, also for 0) = on 7 concurrent
                      streams (the paper's 7 OpenMP sections, Figs. 1-2) */
  int32_t accum;   /* Block multiply-add: 0 (default) = exact fixed-point
                      window accumulation on the integer pipe (operands as
                      multiword integers, no FP64 in the inner loop); larger
                      Block products first convert each operand once into
                      library workspace (about 20 B per DD element, 36 per
                      QD, of A and of B; where that workspace cannot be
                      allocated, tiles are converted as they are staged,
                      as with 2); 2 = the same arithmetic and bits,
                      every tile converted as it is staged (no operand
                      workspace); 1 = TwoSum accumulation on the FP64 pipe
                      (12 FP64 instructions per DD multiply-add, 113 per QD) */
  int32_t slices;  /* DDG_OZAKI: number of INT8 slices s, DD in [2, 18]
                      (0 = 16, about 2^-110 of the row / column maxima), QD
                      in [2, 32] (0 = 32, about 2^-222); DDG_OZAKI2: number
                      of moduli N in [2, 40] (0 = 32) */
  int32_t reserved[2]; /* must be zero */
} ddg_opts;

/* Fill *opts with the defaults: Winograd, cutoff 512, peeling, 7 streams,
 * fixed-point accumulation. */
void ddg_opts_default(ddg_opts* opts);

/*
 * dd_gemm: C (mode) A B in double-double, A m x l, B l x n, C m x n.
 * opts NULL = defaults. Accuracy: DDG_SIMPLE follows the pinned sequence
 * exactly; DDG_BLOCK stays within |C - C^| <= (2 l + 4) 2^-106 |A||B|
 * elementwise for every input, like the DD arithmetic of Section 2's Block
 * (each output's fixed-point window is set from the largest exponents of
 * its row of A and column of B; operands are shifted once to that scale
 * and an output whose window sum keeps fewer than 142 bits is recomputed
 * with every product at its own scale, and one that still keeps fewer
 * than 106 significant bits, as when those maxima sit at different k far
 * apart, with the window at its own largest term); products of small
 * integers (within 64 bits of their row / column maxima) are exact;
 * Strassen/Winograd within the normwise bound 8 l^log2(12) 2^-104
 * ||A|| ||B|| (these recursions are only normwise stable).
 */
ddg_status dd_gemm(int64_t m, int64_t l, int64_t n, dd_mat A, dd_mat B, dd_mat C, int32_t mode,
                   const ddg_opts* opts, void* stream);

/* qd_gemm: as dd_gemm for quad-double: Block within (2 l + 4) 2^-209 |A||B|
 * elementwise (operands shifted once to their row / column maximum; an
 * output keeping fewer than 245 window bits recomputed with every product
 * at its own scale, and one keeping fewer than 212 at its largest term),
 * Strassen / Winograd within 8 l^log2(12) 2^-208 ||A|| ||B||. */
ddg_status qd_gemm(int64_t m, int64_t l, int64_t n, qd_mat A, qd_mat B, qd_mat C, int32_t mode,
                   const ddg_opts* opts, void* stream);

/*
 * dd_getrf: in-place LU decomposition P A = L U of an n x n DD matrix
 * (Section 4, steps 1-3): right-looking blocked LU with block columns of K
 * (1 <= K <= 512; the paper takes K = alpha n_min) whose trailing update
 * A22 := A22 - L21 U12 is the DD product of `opts` (algo, cutoff, ...;
 * NULL = defaults, Winograd; DDG_OZAKI / DDG_OZAKI2 / DDG_OZAKI2_TC give
 * the residue and slice products' normwise accuracy for the updates) in
 * mode DDG_SUB. On return A holds L
 * (unit lower, below the diagonal) and U.
 *   pivot = 1: partial pivoting, pivot of column j = the first row i >= j
 *              with the largest |a_ij| compared as DD; pivot = 0: none (the
 *              paper's setting, Section 4).
 *   ipiv: device array of n int64: row j was interchanged with row ipiv[j]
 *         (0-based) at step j (ipiv[j] = j without pivoting).
 *   info: device pointer to one int64 or NULL. Non-NULL: the call is fully
 *         asynchronous and *info receives 0, or 1 + the first column with an
 *         exactly zero pivot (the factorisation continues past it, leaving
 *         that column's quotients untouched). NULL: the call waits for the
 *         stream and returns DDG_ESINGULAR for a zero pivot.
 * Temporary storage (partial arg-maxes, n/32 entries) comes from the
 * stream-ordered allocator.
 */
ddg_status dd_getrf(int64_t n, dd_mat A, int64_t* ipiv, int32_t K, int32_t pivot, const ddg_opts* opts,
                    int64_t* info, void* stream);

/*
 * dd_getrs: solve A X = B (Section 4, Eq. 2) with the factors of dd_getrf:
 * the row interchanges of ipiv applied to B, forward substitution with the
 * unit lower factor, back substitution with the upper factor (DD quotients
 * by the diagonal). B (n x nrhs) is overwritten by X. Recursive blocked
 * triangular solves: 32-row triangles in one kernel, off-diagonal updates by
 * the Block product. Temporary storage (a copy of B and the permutation)
 * comes from the stream-ordered allocator. Asynchronous.
 */
ddg_status dd_getrs(int64_t n, int64_t nrhs, dd_mat LU, const int64_t* ipiv, dd_mat B, void* stream);

/* qd_getrf / qd_getrs: the same LU and solve in quad-double (the paper's
 * QD LU with Winograd updates, Section 4), same arguments with qd_mat; the
 * quotients use one QD reciprocal of each pivot (the DD reciprocal refined
 * by one Newton step in QD, relative error about 2^-209). */
ddg_status qd_getrf(int64_t n, qd_mat A, int64_t* ipiv, int32_t K, int32_t pivot, const ddg_opts* opts,
                    int64_t* info, void* stream);
ddg_status qd_getrs(int64_t n, int64_t nrhs, qd_mat LU, const int64_t* ipiv, qd_mat B, void* stream);

/*
 * dd_gemm_noalloc: dd_gemm without any device allocation at call time.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot allocate device memory when they multiply: a service whose device
 * memory is handed out once at start-up and then fixed, a host framework
 * whose own allocator owns all free device memory, or a latency-bound loop
 * where an allocation could stall or fail under memory pressure.
 * Same arguments, modes and results as dd_gemm (Simple, Block, Strassen,
 * Winograd; peel or pad), except that the seven sub-products always run in
 * order on `stream` (opts->streams is ignored), so no streams or events are
 * created either. Recursion temporaries live in one fixed 64 MiB array
 * compiled into the library: every GPU that loads the library holds those
 * 64 MiB until the process exits. A product whose temporaries do not fit
 * (about 80 n^2 bytes for a square Winograd n, so n up to ~900 at any
 * cutoff) returns DDG_EINVAL with the needed size in ddg_last_error(), and
 * nothing is queued. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture. All calls on a device share the one
 * array: calls whose work overlaps on the GPU (different streams, or
 * different host threads) race on it and give wrong results, so order them.
 * Nothing has to start at zero: every temporary is written before it is read.
 */
ddg_status dd_gemm_noalloc(int64_t m, int64_t l, int64_t n, dd_mat A, dd_mat B, dd_mat C,
                           int32_t mode, const ddg_opts* opts, void* stream);

/*
 * Batched products (grouped launches). The paper has no batched form; this
 * runs many independent C (mode) A B problems of uneven shapes, DD and QD
 * mixed, as a few grouped persistent launches: every problem's Strassen /
 * Winograd recursion is expanded breadth-first, the fused passes of one
 * depth share a launch, and every base-case Block product of the batch
 * shares one launch per limb count (tiles taken from a global counter).
 * Problems must write disjoint C; A and B may be shared. A problem whose C
 * overlaps its own A or B is DDG_EINVAL; C overlapping another problem's
 * matrices is not checked (undefined results).
 */
typedef struct {
  int32_t limbs;   /* 2 (DD) or 4 (QD) */
  int32_t mode;    /* ddg_mode */
  int64_t m, l, n;
  double* A[4];    /* limb planes (device); unused entries ignored */
  int64_t lda;
  double* B[4];
  int64_t ldb;
  double* C[4];
  int64_t ldc;
  int32_t algo;    /* DDG_BLOCK, DDG_STRASSEN or DDG_WINOGRAD */
  int32_t cutoff;  /* recursion cutoff n_min, >= 1 */
} ddg_problem;

typedef struct {
  int64_t problems;
  int64_t leaf_tasks;       /* base-case products */
  int64_t leaf_tiles;       /* CTA tiles over all grouped Block launches */
  int64_t pass_tasks;       /* fused quadrant passes */
  int64_t launches_per_run; /* kernels per ddg_batch_run */
  uint64_t workspace_bytes;
  double leaf_macs;         /* multiply-adds of the base-case products (sum of m l n) */
} ddg_batch_stats;

typedef struct ddg_batch_s* ddg_batch;

/* Plan a batch on the current device: validates every problem, expands the
 * recursions, takes all temporaries in one block from the stream-ordered
 * allocator on `stream` and queues the upload of the task lists there (the
 * host copy is staged before the call returns). The plan keeps the pointers
 * of the problems; their matrices must stay valid while the plan is run.
 * Runs on other streams must be ordered after `stream`.
 * use_graph = 1: ddg_batch_run captures the launches into a CUDA graph on
 * its first call and replays the graph afterwards. */
ddg_status ddg_batch_create(ddg_batch* out, int32_t count, const ddg_problem* probs, int32_t use_graph,
                            void* stream);
/* ddg_batch_create with plan flags: DDG_BATCH_ONE_LEAF_LAUNCH runs every
 * base-case Block product of the batch, DD and QD together, in one
 * persistent grouped launch with tiles converted as they are staged (the
 * same bits as the default plan, which converts the operands of larger
 * products once in separate launches); a batch of Block problems (or of
 * problems no larger than their cutoff) then runs as a single kernel.
 * Unknown flags: DDG_EINVAL. */
#define DDG_BATCH_ONE_LEAF_LAUNCH 1
ddg_status ddg_batch_create_ex(ddg_batch* out, int32_t count, const ddg_problem* probs, int32_t use_graph,
                               int32_t flags, void* stream);
/* Queue one execution of the plan on `stream` (allocation-free). Runs of
 * one plan must not overlap on the GPU (they share the temporaries). */
ddg_status ddg_batch_run(ddg_batch b, void* stream);
ddg_status ddg_batch_get_stats(ddg_batch b, ddg_batch_stats* stats);
/* Free the plan: its memory is released in order on `stream` (after the
 * runs queued there); a plan that used a graph first waits for the device. */
ddg_status ddg_batch_destroy(ddg_batch b, void* stream);
/* One-shot: create, run and release on `stream` (asynchronous). */
ddg_status dd_gemm_batched(int32_t count, const ddg_problem* probs, void* stream);

/* FP64 instructions per DD (limbs = 2) or QD (limbs = 4) multiply-add in
 * the Block kernel's inner loop for accumulation scheme `accum` (0, 1 or 2, as
 * in ddg_opts), counted from its source (for rooflines): 0 for the
 * fixed-point scheme, whose inner loop runs on the integer pipe; -1 if
 * invalid. */
int32_t ddg_block_fp64_ops_per_mac(int32_t limbs, int32_t accum);

/* DDG_OZAKI2: the bits P of the integer scaling used with N moduli at inner
 * dimension l, min(120, floor((bitlen(M) - 2 - ceil(log2 l)) / 2)) with M
 * the product of the moduli (so that l 2^(2P) < M / 2 and the recovered
 * integer product is exact); -1 if N is outside [2, 40], l < 1 or P < 1. */
int32_t ddg_ozaki2_precision(int32_t moduli, int64_t l);

/* Launch profiling. Between ddg_profile_begin() and ddg_profile_end() every
 * product and pass launch of the library is bracketed by CUDA events on its
 * stream. ddg_profile_end() waits for those events and fills out[k] for
 * kernel kinds k = 0 (Simple), 1 (Block), 2 (quadrant passes), 3 (INT8
 * products), 4 (Block products with at most 8 columns, one warp per
 * output), 5 (operand conversions of the Block products), 6 (tcgen05
 * residue products of DDG_OZAKI2_TC), k < nkinds:
 * launches, sum of launch durations, busy time (union of the launch
 * intervals), and the algorithmic work and bytes of those launches.
 * For measurement only: it adds two event records per launch. */
typedef struct {
  uint64_t launches;
  double sum_ms;
  double busy_ms;
  double ops;   /* FP64 instructions (kind 0), multiply-adds (kinds 1 and 4),
                   DD / QD sums (kind 2), INT8 operations, 2 per
                   multiply-add (kind 3, the INT8 products), BF16
                   operations, 2 per multiply-add (kind 6) or converted
                   elements (kind 5) */
  double bytes;
} ddg_kernel_prof;
ddg_status ddg_profile_begin(void);
ddg_status ddg_profile_end(ddg_kernel_prof* out, int32_t nkinds);

/* Workspace pool (no counterpart in the paper; for services). The
 * temporaries of every call come from one stream-ordered memory pool per
 * device owned by the library. By default it keeps no memory between calls
 * (unused memory returns to the device at the next synchronisation).
 *
 * ddg_workspace_reserve(device, bytes): keep up to `bytes` of unused pool
 * memory mapped between calls and grow the pool to `bytes` now (blocking
 * until done), so that calls needing at most that much in total are served
 * without mapping memory. bytes = 0 only sets the threshold back to 0.
 * DDG_EINVAL for a device index that does not exist, DDG_ENOMEM if the
 * memory cannot be had (the threshold is then 0 again).
 * ddg_workspace_release(device): threshold 0 and return every unused byte
 * of the pool to the device now (memory of calls still in flight stays
 * until they complete).
 * ddg_workspace_stats(device, out): the pool's current mapped and used
 * bytes, its threshold and the largest used size so far. */
typedef struct {
  uint64_t reserved_bytes;  /* memory mapped by the pool */
  uint64_t used_bytes;      /* of which held by calls in flight */
  uint64_t threshold_bytes; /* unused memory kept between calls */
  uint64_t used_high_bytes; /* high-water mark of used_bytes */
} ddg_workspace_info;
ddg_status ddg_workspace_reserve(int32_t device, uint64_t bytes);
ddg_status ddg_workspace_release(int32_t device);
ddg_status ddg_workspace_stats(int32_t device, ddg_workspace_info* out);

/* Number of CUDA kernels this library has launched in this process, all
 * threads and devices together (monotonic; for launch accounting). */
uint64_t ddg_kernel_launches(void);

/* Bounded device waits that ran out on the current device since the last
 * reset: the tensor-core kernel of DDG_OZAKI2_TC waits on shared-memory
 * barriers with an iteration limit; a CTA whose wait runs out counts here,
 * finishes its copies and MMAs in flight, frees its tensor memory and
 * returns (its part of C is then wrong). Synchronous: waits for the device.
 * reset != 0 sets the count back to 0. -1 if it cannot be read. */
int32_t ddg_device_timeouts(int32_t reset);

/* Test support (no counterpart in the paper): run one of the library's
 * bounded device waits on a barrier that nothing completes, so that a test
 * can check that the wait gives up, the kernel returns and the host reads
 * the status, with no GPU fault, trap or hang. Synchronous (waits for the
 * device; about a second).
 *   which = 0: one CTA of the DDG_OZAKI2_TC tensor-core kernel with its TMA
 *              producer idle: the MMA thread's wait on the first stage runs
 *              out; ddg_device_timeouts() then counts it.
 *   which = 1: one LU panel launch whose grid barrier expects one arrival
 *              more than there are CTAs: every CTA's wait runs out and the
 *              factorisation status (info) becomes -1.
 * Returns DDG_ETIMEOUT when the wait ran out as intended, DDG_OK if it did
 * not, DDG_EINVAL for another `which`, DDG_ECUDA / DDG_ENOMEM on errors. */
ddg_status ddg_test_bounded_wait(int32_t which);

/* Message describing the last failure on this host thread ("" if none). */
const char* ddg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DDGEMM_H */
