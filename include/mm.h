/*
 * mm.h -- C ABI of the GB300 (sm_103a) dense FP64 matrix-product library.
 *
 * The operation is the square product C = A.B in double precision, as
 * defined by the sequential triple loop of Hasta and Mutiara (2010), Alg. 1
 * in Sec. 3.1: c(i,k) = sum over j of a(i,j) * b(j,k), accumulated from 0.0
 * (Alg. 3 and Alg. 4 reset c to 0.0 the same way).  The paper times it for
 * N from 10 to 2000 (Sec. 1.1, Sec. 4.1) and counts N^2 (2N - 1) operations
 * per product (Sec. 3.1, Alg. 2).
 *
 * Three forms compute it on the GPU:
 *   MM_NATIVE_FP64  FP64 tensor-core MMA (mma.sync f64), one rounding per
 *                   fused multiply-add, in an order other than the paper's.
 *   MM_EMU_BF16     split-precision emulation: A is scaled per row and B per
 *                   column by powers of two, each value is split into s
 *                   base-2^8 integer digits held exactly in bf16, the digit
 *                   products run on the tcgen05 tensor cores with exact
 *                   integer accumulation, and the exact sum is rounded once
 *                   to FP64.  Nothing in the paper corresponds to it.
 *   MM_EMU_MODULAR  modular emulation: A (per row) and B (per column) are
 *                   rounded to beta-bit fixed-point integers, their residues
 *                   modulo k pairwise coprime moduli <= 256 (held exactly in
 *                   bf16) are multiplied on the tcgen05 tensor cores, the
 *                   exact integer product is recovered by the Chinese
 *                   remainder theorem and rounded once to FP64 (after Ozaki,
 *                   Uchino and Imamura's "Ozaki scheme II", 2025): k products
 *                   instead of the s(s+1)/2 of the digit form.  Nothing in
 *                   the paper corresponds to it either.  Its tiles 256
 *                   columns wide run on CTA pairs (paired tcgen05.mma, 256 x
 *                   256 tiles), measured faster on GB300; the environment
 *                   variable MM_PAIR_MMA=0 runs them on single CTAs instead
 *                   (same results, bit for bit).
 *   MM_EMU_INT8     INT8 slice emulation: as MM_EMU_BF16 with s digits of
 *                   the (8s - 2)-bit fixed-point value, every digit a signed
 *                   byte (Ozaki-style slices with int32 accumulation), the
 *                   digit products on the integer tensor path (mma.sync
 *                   m16n8k32 s8, the only 8-bit integer MMA of sm_103a) and
 *                   recombined as the digit form is.  Far slower than the
 *                   bf16 forms on GB300; never chosen by MM_AUTO.
 * MM_AUTO picks one per problem (see mm_config).
 *
 * Conventions for every call:
 *   - Matrices are square, row-major, leading dimension N, FP64, 16-byte
 *     aligned device pointers, owned by the caller -- except in mm_gemm_ex
 *     and mm_gemm_grouped_ex, which take rectangular shapes, leading
 *     dimensions, transposed storage and 8-byte alignment.  C is overwritten
 *     (beta = 0) and must not overlap A or B.
 *   - A handle's workspace serves one call at a time: concurrent calls on
 *     different streams need one handle each.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL is the legacy default stream).  The return value covers argument
 *     checks and launch errors only; errors found on the device (a timed-out
 *     wait, non-finite input to the emulation) are kept in a status word
 *     read by mm_status_get, which synchronises the stream.
 *   - A handle is not thread safe: use one per host thread.  It owns a
 *     device workspace that grows on demand and is freed by mm_destroy.
 *   - Failed calls leave a message for mm_last_error.
 */
#ifndef MM_H_
#define MM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_handle_s* mm_handle;

typedef enum {
  MM_OK = 0,
  MM_ERR_INVALID = 1,      /* bad argument: NULL, negative size, misaligned pointer */
  MM_ERR_CUDA = 2,         /* a CUDA runtime or driver call failed */
  MM_ERR_NOMEM = 3,        /* workspace allocation failed */
  MM_ERR_UNSUPPORTED = 4,  /* size or slice count outside what the kernels support */
  MM_ERR_TIMEOUT = 5,      /* a device-side wait ran out of time (kernel wound down) */
  MM_ERR_NONFINITE = 6     /* emulation met an Inf or NaN input */
} mm_status;

typedef enum {
  MM_NATIVE_FP64 = 0,
  MM_EMU_BF16 = 1,
  MM_EMU_INT8 = 2,
  MM_AUTO = 3,
  MM_EMU_MODULAR = 4
} mm_mode;

/* Flags of mm_config.flags. */
#define MM_FLAG_NO_GRAPH 1u /* grouped calls launch directly instead of replaying a CUDA graph */
#define MM_FLAG_PROFILE 2u  /* bracket every kernel with CUDA events (implies MM_FLAG_NO_GRAPH) */
#define MM_FLAG_NO_GUARD 4u /* emulated forms skip the accuracy certificate (see mm_guard_read) */

typedef struct {
  mm_mode mode;          /* default MM_AUTO */
  int slices;            /* digit count s in 1..8 (MM_EMU_BF16, MM_EMU_INT8), moduli k in
                            2..16 (MM_EMU_MODULAR); 0 = chosen per problem */
  unsigned flags;        /* MM_FLAG_* */
  const char* tune_path; /* optional autotune table (text file); NULL = built-in table */
} mm_config;

/* Creates a handle on the current CUDA device.  cfg may be NULL (MM_AUTO,
 * automatic slice count).  *out receives the handle. */
mm_status mm_create(mm_handle* out, const mm_config* cfg);

/* Releases the handle and its workspace.  Waits for the device first. */
mm_status mm_destroy(mm_handle h);

/* C = A.B for one N x N problem (Alg. 1).  N = 0 is a no-op.
 * A, B, C: device pointers (see conventions). */
mm_status mm_gemm(mm_handle h, int N, const double* A, const double* B, double* C, void* stream);

/* `count` independent products C_p = A_p.B_p of uneven sizes Ns[p] in one
 * grouped launch per kernel.  Ns, As, Bs, Cs are HOST arrays of length
 * count, read during the call; the matrices they point to are device
 * memory.  Problems with N = 0 are skipped.  The first call with a given
 * (count, Ns, pointers) signature builds a CUDA graph; later identical calls
 * replay it (unless MM_FLAG_NO_GRAPH). */
mm_status mm_gemm_grouped(mm_handle h, int count, const int* Ns, const double* const* As,
                          const double* const* Bs, double* const* Cs, void* stream);

/* Rectangular product C (M x N) = op(A) (M x K) . op(B) (K x N): the sum of
 * Alg. 1 over the three dimensions the master/worker program of Alg. 2 names
 * separately (NRA = M, NCA = K, NCB = N; the paper's experiments are square).
 *   - transa = 0: A is stored M x K, op(A)(i,j) = A[i*lda + j], lda >= K;
 *     transa = 1: A is stored K x M (op(A) = A^T), op(A)(i,j) = A[j*lda + i],
 *     lda >= M.  Likewise transb = 0: B stored K x N, ldb >= N; transb = 1:
 *     B stored N x K, ldb >= K.  C is always M x N, C[i*ldc + j], ldc >= N.
 *     Sub-matrices of larger arrays are passed with their parents' row
 *     strides.  All device pointers, 8-byte aligned (not 16).
 *   - M = 0 or N = 0: no-op.  K = 0: C = 0.  Negative sizes, flags other than
 *     0 and 1, leading dimensions below the stored row length, null or
 *     misaligned pointers, and a C whose span overlaps A's or B's:
 *     MM_ERR_INVALID, nothing launched.
 *   - The plan (form, slice or moduli count, tile width) is the one for size
 *     max(M, N, K); the emulated forms' exponents run over the K entries of
 *     each row of op(A) and column of op(B), and the modular form's
 *     fixed-point width follows the rule of mm_modular_params with N = K.
 *   - Asynchronous on `stream`; device-side errors via mm_status_get. */
mm_status mm_gemm_ex(mm_handle h, int transa, int transb, int M, int N, int K, const double* A, int lda,
                     const double* B, int ldb, double* C, int ldc, void* stream);

/* `count` such products in one grouped launch per kernel, as
 * mm_gemm_grouped: every argument array is a HOST array of length count with
 * each problem's arguments as in mm_gemm_ex; transas / transbs may be NULL
 * (no transposes).  The graph signature covers every size, flag, leading
 * dimension and pointer. */
mm_status mm_gemm_grouped_ex(mm_handle h, int count, const int* transas, const int* transbs, const int* Ms,
                             const int* Ns, const int* Ks, const double* const* As, const int* ldas,
                             const double* const* Bs, const int* ldbs, double* const* Cs, const int* ldcs,
                             void* stream);

/* End-to-end form of mm_gemm on HOST buffers: copies A and B to the device,
 * computes, copies C back, and returns when C is on the host (the span the
 * paper times with MPI_Wtime, Alg. 2).  Host buffers are best pinned. */
mm_status mm_gemm_host(mm_handle h, int N, const double* A_host, const double* B_host, double* C_host,
                       void* stream);

/* End-to-end form of mm_gemm_grouped on HOST buffers: Ns, As, Bs, Cs as in
 * mm_gemm_grouped but the matrices are host memory (best pinned).  Returns
 * when every C_p is on the host.  The problems are cut into chunks (those
 * below N = 768 together, the larger ones in up to four chunks by size,
 * the smallest of those last); the copies of one chunk overlap the
 * computation of its neighbours (inputs on an upload stream, results on a
 * download stream, the products on `stream` as a grouped call).  The device
 * copies live in a grow-only handle buffer. */
mm_status mm_gemm_grouped_host(mm_handle h, int count, const int* Ns, const double* const* As_host,
                               const double* const* Bs_host, double* const* Cs_host, void* stream);

/* Synchronises `stream` and returns the first error recorded on the device
 * since the last call (and clears it), else MM_OK. */
mm_status mm_status_get(mm_handle h, void* stream);

/* Message of the last failed call on this handle (never NULL). */
const char* mm_last_error(mm_handle h);

/* Accuracy certificate of the emulated forms.  The product guaranteed is
 * Alg. 1's c(i,k) (Sec. 3.1); the guarantee is that every element is within
 * gamma_K (|A||B|)(i,k) of the exact product, gamma_K = K u / (1 - K u),
 * u = 2^-53, K the inner dimension -- the bound the paper's own recursive sum
 * obeys -- so that any two such results differ by at most 2 gamma_K |A||B|.
 * Unless the handle has MM_FLAG_NO_GUARD, every emulated launch also
 *   - writes one more plane per operand: the magnitude digits
 *     M = floor-ish(|v| 2^(7 - e)) in [0, 127] of every entry,
 *   - multiplies the two magnitude planes exactly on the tensor cores
 *     (S = sum_j M_A M_B, so (|A||B|)(i,k) >= S 2^(e_i + f_k - 14)),
 *   - tests for each element a bound of its own error (fixed-point rounding
 *     of both operands, the digit pairs the digit form leaves out, the final
 *     rounding) against gamma_K times that lower bound, and
 *   - recomputes every element that fails in native FP64 (fused
 *     multiply-adds, within gamma_K |A||B|); when more than a quarter of a
 *     problem's elements fail, the whole problem is recomputed natively.
 * Zero rows of A and columns of B are exact in every form and never fail.
 * On typical inputs nothing fails (uniform entries) or a few elements in
 * 10^4 (entries of magnitude 2^U(-20,20)); inputs whose rows mix magnitudes
 * far apart fail more and cost more.  Results in the subnormal range are not
 * covered (nor is the paper's loop there).
 * mm_guard_read synchronises `stream` and returns how many elements
 * (*elements) and whole problems (*problems, their elements included in
 * *elements) were recomputed natively since the last read, then clears the
 * counts.  Either pointer may be NULL. */
mm_status mm_guard_read(mm_handle h, void* stream, long long* elements, long long* problems);

/* Form and slice count the handle would use for an N x N problem (after
 * AUTO): form 0 = native FP64, 1 = digit emulation (slices = digits s),
 * 2 = modular emulation (slices = moduli k), 3 = INT8 slice emulation
 * (slices = digits s). */
mm_status mm_plan(mm_handle h, int N, int* form, int* slices);

/* Parameters of the modular form with k moduli at size N, computed on the
 * host (no handle, no GPU): *beta receives the fixed-point width, the
 * largest beta <= 62 with 514 N 2^(2 beta) <= 256 m_1 m_2 ... m_k, so that the
 * exact product of two beta-bit operands (at most N 2^(2 beta) in magnitude)
 * lies within half the modulus of zero with a margin of 1/514 of it and is
 * recovered from its residues; 0 when k is too small for N.  moduli (may be
 * NULL) receives m_1..m_k.
 * MM_ERR_INVALID for k outside 1..16 or N < 1. */
mm_status mm_modular_params(int k, int N, int* beta, int* moduli);

/* Device time of the last call made on this handle with MM_FLAG_PROFILE set,
 * in milliseconds, by kernel kind (events recorded on the call's stream):
 *   out_ms[0] scale and split (including zeroing of the row/column maxima)
 *   out_ms[1] slice products (with the digit form's fused recombination)
 *   out_ms[2] native FP64 kernels (including the certificate's recomputation)
 *   out_ms[3] recombination run as its own pass (small problems, the modular
 *             form, mm_recombine)
 *   out_ms[4] the accuracy certificate's product of the magnitude planes, when
 *             it has a launch of its own (with CTA pairs its units run in the
 *             slice-product launch, out_ms[1])
 * and launches[0..4] the number of kernel launches of each kind (may be
 * NULL).  Both arrays hold MM_PROFILE_KINDS entries.  Synchronises on the
 * recorded events.  MM_ERR_INVALID without the flag. */
#define MM_PROFILE_KINDS 5
mm_status mm_profile_read(mm_handle h, double out_ms[MM_PROFILE_KINDS], int launches[MM_PROFILE_KINDS]);

/* Measures the FP64 throughput of this GPU with two calibration kernels
 * (independent chains of mma.sync m16n8k4 f64, and of scalar FP64 FMA),
 * in TFLOP/s: the roof of the native form.  Blocks for a few milliseconds. */
mm_status mm_probe_fp64_peak(mm_handle h, double* dmma_tflops, double* dfma_tflops);

/* Measures the 8-bit integer MMA throughput of this GPU with a calibration
 * kernel (independent chains of mma.sync m16n8k32 s8, the instruction of the
 * INT8 slice form), in tera-operations per second (2 per multiply-add): the
 * roof of MM_EMU_INT8.  Blocks for a few milliseconds. */
mm_status mm_probe_int8_peak(mm_handle h, double* tops);

/* Failure-detection self-test: enqueues a kernel that waits on an mbarrier
 * nothing ever arrives on, through the same time-bounded wait every pipeline
 * of the library uses.  After timeout_ms (1..60000) the wait gives up, the
 * kernel records MM_ERR_TIMEOUT in the handle's status word and returns; the
 * CUDA context stays usable.  mm_status_get then reports MM_ERR_TIMEOUT.
 * The paper has no counterpart (its programs have no failure detection). */
mm_status mm_selftest_wait(mm_handle h, int timeout_ms, void* stream);

/* ---------------------------------------------------------------------
 * Steps of the emulation, exposed for testing each one on its own.
 * They use caller-provided device buffers with the layouts stated here.
 * --------------------------------------------------------------------- */

/* Scale and split (row/column scaling, then integer digits).
 * by_columns = 0: operand A, exponent e_i of row i; by_columns = 1: operand
 * B, exponent f_k of column k.  e_i is the smallest integer with
 * max_j |a_ij| < 2^e_i (0 for a zero row).  Each value v is turned into the
 * integer D = round-half-even(v * 2^(8s - 1 - e)) and D is written as s
 * balanced base-256 digits D = sum_t d_t 2^(8(s-t)), d_2..d_s in [-128,127],
 * d_1 in [-128,128] (Ozaki, Ogita, Oishi, Rump 2012 split, fixed-point form).
 * Outputs (device): exps[N] int32; digits: bf16 bit patterns, s planes of
 * rows x ld elements, plane t at digits + t*rows*ld.  For A, element (i,j)
 * sits at row i, column j; for B, (j,k) sits at row k, column j (B^T).
 * rows >= N a multiple of 128, ld >= N a multiple of 64, digits 16-byte
 * aligned; the padding is written with 0. */
mm_status mm_split(mm_handle h, int N, const double* M, int by_columns, int slices, int* exps,
                   uint16_t* digits, int rows, int ld, void* stream);

/* Scale and split without allocating: the same computation and output
 * layout as mm_split, for callers that may not allocate device memory at all
 * (code living inside another framework's memory pool, services that forbid
 * allocation after start-up, code that must avoid the device-wide
 * synchronisation of cudaFree).  It needs no handle.  The paper has no
 * counterpart; this is an interface convenience of the library.
 *   - Its only scratch (one 64-bit maximum per row or column) is a static
 *     device array of MM_SPLIT_NOALLOC_MAX_N entries (512 KiB) that exists on
 *     every GPU that loads the library, until the process exits or the
 *     device is reset.
 *   - N > MM_SPLIT_NOALLOC_MAX_N returns MM_ERR_UNSUPPORTED; bad arguments
 *     return MM_ERR_INVALID; nothing is launched in either case.
 *   - Every call made while `stream` is not being captured looks up the
 *     array's device address (cudaGetSymbolAddress) with the calling device
 *     current, so a device reset, which may move the array, is picked up by
 *     the next such call.  A call made during stream capture reuses the
 *     address found by the last uncaptured call on that device: make one
 *     call on the device before capturing (MM_ERR_CUDA otherwise).
 *   - Every call uses the same array: calls that overlap on the GPU (on
 *     different streams, or from several threads) race and corrupt each
 *     other's exponents.  Serialise them on one stream.
 *   - status: optional device int (may be NULL); the first error found on the
 *     device (MM_ERR_NONFINITE for an Inf or NaN input) is stored there if it
 *     holds 0.  Returns after enqueueing the work on `stream`. */
#define MM_SPLIT_NOALLOC_MAX_N 65536
mm_status mm_split_noalloc(int N, const double* M, int by_columns, int slices, int* exps, uint16_t* digits,
                           int rows, int ld, int* status, void* stream);

/* Exact level sums of digit products: for L = 2..s+1,
 *   S_L(i,k) = sum_j sum_{t+u=L} d_t(a_ij) d_u(b_jk)
 * written as int32 to levels[(L-2)*N*N + i*N + k].  Inputs are the digit
 * planes of mm_split (A: rows = a_rows; B: rows = b_rows, multiples of 128;
 * both with ld).  Requires s * N * 2^14 < 2^31. */
mm_status mm_level_sums(mm_handle h, int N, int slices, const uint16_t* a_digits, int a_rows,
                        const uint16_t* b_digits, int b_rows, int ld, int32_t* levels, void* stream);

/* Recombination: c_ik = RN( sum_L S_L(i,k) 2^(8(s+1-L)) ) * 2^(e_i + f_k - 8s - 6),
 * one round-to-nearest-even of the exact integer sum, then exact scaling. */
mm_status mm_recombine(mm_handle h, int N, int slices, const int32_t* levels, const int* a_exps,
                       const int* b_exps, double* C, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MM_H_ */
