/*
 * gbfft - batched one-dimensional complex-to-complex FFTs on GB300 (sm_103a).
 *
 * The library computes, for every row x of a batch,
 *
 *     y = DFT_N x,   DFT_N[m][k] = w_N^(m*k),   w_N = exp(-2*pi*i/N)
 *
 * (the DFT matrix of the FFTc paper, Sec. II), by a factorised Stockham
 * schedule: stages built from the factor types of the general-radix
 * Cooley-Tukey factorisation (Eq. 2) - a small DFT_r Kronecker-multiplied with
 * an identity, a diagonal of twiddle factors and a stride permutation - with
 * the whole schedule of one transform fused into one kernel for N <= 4096 and
 * Eq. 2's outer split into two passes for larger N.
 *
 * Conventions shared by every entry point:
 *   - Data: interleaved complex64, i.e. (float re, float im) pairs.  Row i of
 *     a batch starts at complex element i*N.  Pointers passed to execute calls
 *     are device pointers (unless the name says _host) that the caller owns;
 *     they must be 16-byte aligned.
 *   - Direction: GBFFT_FORWARD uses w_N = exp(-2*pi*i/N); GBFFT_INVERSE uses
 *     exp(+2*pi*i/N) and is unnormalised, so inverse(forward(x)) = N*x.
 *   - Errors: every call returns a gbfft_status; nothing throws across this
 *     boundary.  Execute calls are asynchronous on the caller's stream: launch
 *     errors come back at once, device-side problems are read with
 *     gbfft_plan_device_status() after the stream has been synchronised.
 *   - Plans are created on, and must be executed on, the CUDA device that was
 *     current at creation.  A plan owns its device tables and workspace; one
 *     plan must not run concurrently on two streams.
 */
#ifndef GBFFT_H
#define GBFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbfft_plan_s *gbfft_plan; /* opaque; owned by the library */

typedef enum {
    GBFFT_OK = 0,
    GBFFT_ERR_INVALID_ARG = 1,      /* null pointer, n < 1, batch < 0, bad enum */
    GBFFT_ERR_UNSUPPORTED_SIZE = 2, /* n has a prime factor the planner does not handle */
    GBFFT_ERR_ALIGNMENT = 3,        /* a data pointer is not 16-byte aligned */
    GBFFT_ERR_OVERLAP = 4,          /* in and out overlap without being identical */
    GBFFT_ERR_OOM = 5,              /* device allocation failed */
    GBFFT_ERR_BUDGET = 6,           /* request exceeds a memory budget */
    GBFFT_ERR_CUDA = 7,             /* a CUDA runtime call or launch failed */
    GBFFT_ERR_TIMEOUT = 8,          /* a bounded wait ran out */
    GBFFT_ERR_DEVICE_STATUS = 9,    /* a kernel reported an error in its status word */
    GBFFT_ERR_NOT_FOUND = 10        /* unknown ticket / variant */
} gbfft_status;

#define GBFFT_FORWARD (-1)
#define GBFFT_INVERSE (+1)

typedef enum {
    GBFFT_C2C_F32 = 0,           /* complex64 in/out, FP32 arithmetic, FP64-generated twiddles */
    GBFFT_C2C_F32_TC_FP16X2 = 1, /* complex64 in/out; every DFT_16 block as FP16 hi+lo tensor-core products */
    GBFFT_C2C_F32_TC_BF16X2 = 2, /* complex64 in/out; every DFT_16 block as BF16 hi+lo tensor-core products */
    GBFFT_C2C_F64 = 3            /* complex128 in/out (interleaved double re, im; 16 bytes per point), FP64
                                    arithmetic and FP64 twiddles, the paper's own precision (Sec. VI);
                                    single pass, n = 2^a 3^b 5^c 7^d <= 4096 with at most one odd factor
                                    (2^k, 3*2^k, 5*2^k, 7*2^k); relative L2 error ~1e-16*log2(n) */
} gbfft_dtype;

/* Human-readable name of a status code (static storage; never NULL). */
const char *gbfft_status_string(gbfft_status s);

/* Library version as major*10000 + minor*100 + patch. */
int gbfft_version(void);

/*
 * Create a plan for `batch` transforms of length `n` (Sec. II DFT_N) in
 * direction `direction` (GBFFT_FORWARD / GBFFT_INVERSE) and arithmetic `dtype`.
 * The planner factorises n into a radix schedule (Eq. 2 factor types) and
 * generates the twiddle table w_N^j, j < n, in FP64 on the device, rounded to
 * float32.  For FP32 n <= 4096 runs in one pass; above, the default is Eq. 2
 * as two passes (two HBM round trips), except n = 8192, where the one-pass
 * kernel on a pair of CTAs of a thread-block cluster (variant kind 4) is the
 * default because it measured faster.  batch may be 0 (execute is then a
 * no-op).  On success *out holds a
 * new plan that the caller releases with gbfft_destroy().  Errors:
 * INVALID_ARG, UNSUPPORTED_SIZE, OOM, CUDA.  *out is set to NULL on error.
 *
 * Tensor-core dtypes (GBFFT_C2C_F32_TC_*): n must be 16, 256 or 4096 (an
 * all-radix-16 schedule) or, FP16x2 only, a multiple of 8 up to 64 (the
 * direct DFT below); BF16x2 only 256 and 4096, because its error in a single
 * dense product, 4-6e-6 relative L2, exceeds the 1e-6*log2(N) accuracy
 * contract of the tensor-core path at smaller N.  Each stage's DFT_16 - the
 * dense DFT(16) block of the factorisation (Table I), multiplied as a matrix -
 * runs as a 32x32 real product on the tensor cores with both operands split
 * into high and low half-precision parts (Mh Xh + Mh Xl + Ml Xh, FP32
 * accumulation); FP16 columns are scaled by exact powers of two first.  Stage
 * twiddles stay FP32.  gbfft_plan_create_variant with a tensor-core dtype
 * selects the engine: variant 1 (N = 256, 4096; the default there) issues
 * tcgen05.mma from shared-memory operands into tensor memory and reads results
 * back with tcgen05.ld; variant 0 (N = 16, 256, 4096) issues warp-level
 * mma.sync.m16n8k16 on register fragments; variants 2 and 3 (N = 8, 16, 24,
 * ..., 64; FP16x2 only) are the direct DFT: y = F_N x as ONE split-precision
 * real product [yr yi] = [xr xi] [[Fr, Fi], [-Fi, Fr]] per 128 transforms on
 * tcgen05 (M = 128, K = N_out = 2N), no factorisation (the paper's direct-DFT
 * variant, Sec. VI).  Variant 2 (the default at N = 16 ... 64) is warp-
 * specialised: producer warps split rows into tensor memory, one thread issues
 * the MMAs and epilogue warps read the results back, on consecutive tiles at
 * once; variant 3 (the default at N = 8) runs each tile's phases one after the
 * other in every thread of a CTA.  The two-pass form is FP32-only (INVALID_ARG
 * otherwise).
 */
gbfft_status gbfft_plan_create(gbfft_plan *out, int64_t n, int64_t batch, int direction, int dtype);

/*
 * As gbfft_plan_create, but with the single-pass kernel variant forced to
 * index `variant` of gbfft_variant_info(n, ...) (used by the autotuner and by
 * tests that cover every variant).  NOT_FOUND if there is no such variant.
 */
gbfft_status gbfft_plan_create_variant(gbfft_plan *out, int64_t n, int64_t batch, int direction, int dtype,
                                       int variant);

/*
 * As gbfft_plan_create, but forcing the two-pass form of Eq. 2,
 *     DFT_N = (DFT_K (x) I_M) D^N_M (I_K (x) DFT_M) Pi^N_K,   N = K*M,
 * with outer factor K = k_outer (0 = the planner's choice).  Pass 1 gathers
 * the K stride-K columns of each row (Pi^N_K), transforms them (I_K (x) DFT_M)
 * and scales by D^N_M = diag(w_N^(k*j)) at position k*M + j on the way into a
 * plan-owned workspace of batch*n complex64; pass 2 applies DFT_K across the
 * workspace columns (DFT_K (x) I_M) and writes `out` in natural order.  This is
 * the default for lengths with no single-pass kernel (n > 4096).  Both K and M
 * must be lengths of the column kernels (32, 48, 64, 80, 96, 112, 128, 256,
 * 512).  Errors as gbfft_plan_create; NOT_FOUND when k_outer does not give a
 * supported split.
 */
gbfft_status gbfft_plan_create_twopass(gbfft_plan *out, int64_t n, int64_t batch, int direction, int dtype,
                                       int64_t k_outer);

/*
 * Run the plan: out = DFT_N in (row by row), asynchronously on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  `in` and `out` are
 * device pointers to batch*n complex64 values, 16-byte aligned; in == out
 * (in place) is allowed, partial overlap is not.  Errors: INVALID_ARG,
 * ALIGNMENT, OVERLAP, CUDA.
 */
gbfft_status gbfft_execute(gbfft_plan p, const void *in, void *out, void *cuda_stream);

/*
 * Host-buffer form of gbfft_execute: `in` and `out` are HOST pointers to
 * batch*n complex64 values (in == out allowed).  When both buffers are
 * addressable by the device (page-locked host memory mapped into its address
 * space - on a Grace-Blackwell node the GPU reaches it over NVLink-C2C - or
 * device memory) and 16-byte aligned, the plan's kernels read and write them
 * directly, with no staging.  Otherwise the batch is streamed through
 * a ring of three device staging buffers of about 32 MiB each (allocated by
 * the plan on the first call and kept until gbfft_destroy): the host-to-device
 * copy of one chunk, the transform of the previous chunk and the
 * device-to-host copy of the one before run concurrently on two internal
 * streams and `cuda_stream`.  The call is asynchronous like gbfft_execute: all
 * of its work is ordered after earlier work on `cuda_stream`, and later work on
 * `cuda_stream` (including a synchronise) sees `out` complete.  Page-locked
 * host memory (cudaHostAlloc / torch pin_memory) is needed for the copies to
 * overlap; pageable memory works but serialises them.  Errors: INVALID_ARG,
 * OVERLAP, OOM, CUDA.
 */
gbfft_status gbfft_execute_host(gbfft_plan p, const void *in, void *out, void *cuda_stream);

/* Release a plan and its device memory.  NULL is accepted (no-op). */
gbfft_status gbfft_destroy(gbfft_plan p);

/*
 * Describe a plan: length, batch, direction, number of stages and their
 * radices (up to 8 written to `radices`; may be NULL), the single-pass variant
 * index (-1 if the plan is multi-pass) and the device workspace it holds, in
 * bytes.  Any output pointer may be NULL.
 */
gbfft_status gbfft_plan_info(gbfft_plan p, int64_t *n, int64_t *batch, int *direction, int *nstages,
                             int *radices, int *variant, size_t *workspace_bytes);

/*
 * The Eq. 2 split of a plan: *k_outer = K and *m_inner = M for a two-pass
 * plan, (1, n) for a single-pass plan.  Output pointers may be NULL.
 */
gbfft_status gbfft_plan_factors(gbfft_plan p, int64_t *k_outer, int64_t *m_inner);

/*
 * Number of compiled single-pass kernel variants for length n (0 when n is
 * only reachable through the multi-pass path or not supported).
 */
int gbfft_num_variants(int64_t n);

/*
 * Variant `index` for length n: its radix schedule (stage count + up to 8
 * radices), transforms per CTA, threads per CTA and dynamic shared memory.
 * NOT_FOUND for an index out of range.  Output pointers may be NULL.
 */
gbfft_status gbfft_variant_info(int64_t n, int index, int *nstages, int *radices, int *rows_per_cta,
                                int *threads_per_cta, int *smem_bytes);

/*
 * Grid bound of a plan's persistent kernel (resident CTAs on the device at
 * plan creation); 0 for one-tile-per-CTA kernels, -1 for NULL.  Diagnostic.
 */
int gbfft_plan_grid_cap(gbfft_plan p);

/*
 * Kernel shape of variant `index` for length n: 0 one tile per CTA, 1
 * persistent with register prefetch, 2 one row per thread staged through
 * shared memory, 3 persistent with the next tile prefetched by TMA bulk copy
 * into shared memory (bounded mbarrier waits), 4 one row per thread-block
 * cluster (N > 4096, Eq. 2 on chip), 5 Pease's constant-geometry
 * factorisation of N = R^t (stride-R reads, stride-N/R writes at every stage,
 * digit-reversed input; one tile per CTA).  -1 for an index out of range.
 */
int gbfft_variant_kind(int64_t n, int index);

/*
 * Read (and clear) the plan's device status word after the stream that ran it
 * has been synchronised.  GBFFT_OK when no kernel reported a problem, else
 * DEVICE_STATUS / TIMEOUT.
 */
gbfft_status gbfft_plan_device_status(gbfft_plan p);

/*
 * Planner autotuner and wisdom (FFTW-style runtime planning, which the paper
 * lists as future work).  gbfft_autotune times, on scratch device buffers of
 * `batch` rows (allocated and freed inside the call; synchronous), every way
 * the library can run length n in direction/dtype: each compiled single-pass
 * variant, each two-pass split N = K*M (FP32), each tensor-core engine; it
 * returns the fastest (*best_variant >= 0 a variant/engine index, or -1 with
 * *best_k_outer = K for two-pass; *best_ms its median time over `reps`) and
 * records it as wisdom.  gbfft_plan_create uses wisdom for (n, dtype,
 * direction) when it has some.  gbfft_wisdom_export writes the table to a
 * text file (one line per entry, tagged with the GPU name);
 * gbfft_wisdom_import merges a file (with require_same_gpu != 0, entries from
 * other GPU models are skipped; INVALID_ARG on a malformed file, NOT_FOUND if
 * it cannot be opened); gbfft_wisdom_lookup queries one entry (NOT_FOUND if
 * none); gbfft_wisdom_forget clears it.  GBFFT_WISDOM=<file> in the
 * environment is imported once at the first plan creation.
 */
gbfft_status gbfft_autotune(int64_t n, int64_t batch, int direction, int dtype, int reps, int *best_variant,
                            int64_t *best_k_outer, float *best_ms);
gbfft_status gbfft_wisdom_lookup(int64_t n, int dtype, int direction, int *variant, int64_t *k_outer);
gbfft_status gbfft_wisdom_export(const char *path);
gbfft_status gbfft_wisdom_import(const char *path, int require_same_gpu);
gbfft_status gbfft_wisdom_forget(void);

/*
 * Multi-dimensional transforms: `batch` row-major complex64 arrays of shape
 * dims[0] x ... x dims[rank-1] (rank 1..3, the last axis contiguous, array i
 * at element i * prod(dims)), each transformed by DFT_{dims[0]} ⊗ ... ⊗
 * DFT_{dims[rank-1]} (the Kronecker product of Table I applied to whole
 * transforms; direction and scaling as gbfft_plan_create).  Execution: the
 * last axis by the single-pass row kernel, then every other axis, last to
 * first, by the column kernel of Eq. 2's second pass, in place in `out`.
 * Sizes: dims[rank-1] a single-pass length and a multiple of 16; the other
 * axes column lengths (8, 16, 32, 48, 64, 80, 96, 112, 128, 256, 512); else
 * UNSUPPORTED_SIZE.  FP32 only (INVALID_ARG otherwise).  Executed with
 * gbfft_execute / gbfft_execute_host; gbfft_plan_info reports n = prod(dims)
 * and the last axis' radix schedule.
 */
gbfft_status gbfft_plan_create_nd(gbfft_plan *out, int rank, const int64_t *dims, int64_t batch, int direction,
                                  int dtype);

/* Shape of a plan: *rank (1 for one-dimensional plans) and dims[0..rank-1]
 * (dims may be NULL; room for 3). */
gbfft_status gbfft_plan_dims(gbfft_plan p, int *rank, int64_t *dims);

/*
 * Factorisation-formula front end (the operator vocabulary of Table I, the
 * paper's own input language, Sec. IV-A): DFT(n), I(n), A ⊗ B (or `A kron B`),
 * A · B (or `A * B`, `A . B`), twiddle(N, M) = D^N_M, Permute(N, K) =
 * Pi^N_K, parentheses; ⊗ and · are right-associative at one precedence level
 * (the paper's grammar); UTF-8 text.  A program line such as Listing 1's
 * `var result = (DFT(2) ⊗ I(2)) · twiddle(4,2) · (I(2) ⊗ DFT(2)) · Permute(4,2)
 * · InputComplex;` is accepted: the `var name =` prefix, a trailing input
 * identifier and `;` are ignored.
 *
 * gbfft_formula_check: parses `formula` and checks symbolically that it
 * denotes DFT_N through Eq. 2, (DFT_K ⊗ I_M) · twiddle(N, M) · (I_K ⊗ DFT_M) ·
 * Permute(N, K) with N = K*M, or its transpose Permute(N, M) · (I_K ⊗ DFT_M) ·
 * twiddle(N, M) · (DFT_K ⊗ I_M) (the decimation-in-frequency order: DFT_N is
 * symmetric), recursively (each DFT factor may be such a product; Eq. 1 is
 * N = 4); or Pease's constant-geometry form for N = R^t, t >= 2 (Eq. 2 with
 * K = R unrolled over the digits),
 *     G_t · ... · G_1 · Rev_N,
 *     G_s = (DFT(R) ⊗ I(N/R)) · (twiddle(R^s, R^(s-1)) ⊗ I(R^(t-s))) · Permute(N, R),
 *     Rev_N = (I(R) ⊗ Rev_(N/R)) · Permute(N, R),  Rev_R = I(R)
 * (G_t's twiddle factor may be written twiddle(N, N/R) alone; Rev_(R^2) may be
 * written Permute(R^2, R)).  On success writes N, the outermost K (0 when the
 * formula is a single DFT(N) or Pease's form), and the DFT leaf sizes in the order the product
 * applies them (rightmost first; at most `max_leaves` written, *nleaves = the
 * full count).  Host only: no CUDA call.  Errors: INVALID_ARG (syntax,
 * dimension mismatch, or not a DFT factorisation), with a message in `err`
 * (`err_len` bytes, may be NULL/0).
 */
gbfft_status gbfft_formula_check(const char *formula, int64_t *n, int *leaves, int max_leaves, int *nleaves,
                                 int64_t *k_outer, char *err, size_t err_len);

/*
 * The factorisation a formula (Table I vocabulary) states at its top level:
 * 0 Eq. 2 (or a single DFT(N)), 1 Eq. 2's transpose (decimation in
 * frequency), 2 Pease's constant-geometry form (named in Sec. II; written out
 * above); -1 when gbfft_formula_check rejects it (NULL or malformed text
 * included).  `formula` is caller-owned UTF-8 text, only read.  Host only: no
 * CUDA call.
 */
int gbfft_formula_form(const char *formula);

/*
 * A plan for the transform a checked formula denotes, following the formula
 * as literally as the compiled kernels allow.  *match (may be NULL): 2 = the
 * formula's own factorisation (a single-pass plan whose Stockham radix
 * sequence is the formula's leaf sequence, the Pease kernel for a Pease
 * formula of a compiled length (variant kind 5), or Eq. 2's two-pass plan with the
 * formula's outermost split K x M over plain DFT(K), DFT(M) factors); 1 = the
 * same radices in another stage order (a Pease formula without a compiled
 * Pease kernel runs its radices as Stockham stages), or the outermost split with the inner
 * factors on the column kernels' own schedules; 0 = the default plan for N.
 * Errors as gbfft_formula_check (INVALID_ARG) and gbfft_plan_create.
 */
gbfft_status gbfft_plan_create_formula(gbfft_plan *out, const char *formula, int64_t batch, int direction, int dtype,
                                       int *match);

/*
 * Ragged batches: `count` independent transforms of uneven lengths n[i]
 * (any 1 <= n[i] <= 8192 whose prime factors are 2, 3, 5 and 7; others give
 * UNSUPPORTED_SIZE), transform i occupying complex elements
 * [offsets[i], offsets[i] + n[i]) of both the input and the output buffer
 * (typically packed back to back).  Transforms must not overlap each other
 * (OVERLAP).  Each is DFT_{n[i]} of Sec. II in direction `direction`.  The
 * plan groups the transforms by length, gives each length a Stockham radix
 * schedule over the radices 2, 3, 4, 5, 7, 8, 16 (read by the kernel at run
 * time), cuts each group into work items of a tile shape (rows per item, at
 * most 8192 elements and 512 rows) and uploads an item queue;
 * gbfft_execute_ragged then runs ONE persistent kernel launch in which every
 * CTA claims items from the queue until it is empty, replayed from a CUDA
 * graph (the counter reset and the launch, captured on the first execute and
 * patched when the buffers change).  The arrays n/offsets are copied; the
 * caller keeps ownership.  gbfft_plan_info reports n = elements spanned and
 * batch = count.
 */
gbfft_status gbfft_plan_ragged(gbfft_plan *out, const int64_t *n, const int64_t *offsets, int64_t count,
                               int direction, int dtype);

/* Run a ragged plan on device buffers `in`/`out` (16-byte aligned, in == out
 * allowed) asynchronously on `cuda_stream` (one graph launch).  INVALID_ARG if
 * the plan is not a ragged plan. */
gbfft_status gbfft_execute_ragged(gbfft_plan p, const void *in, void *out, void *cuda_stream);

/*
 * Autotuner for a ragged plan: tries the three queue orders, then for each length,
 * heaviest first, the compiled or the run-time engine (gbfft_ragged_set_engine),
 * the tile split 1, 2, 4, 8 (rows per item = (rows of the engine's tile)/split),
 * and, on the run-time engine, each candidate radix schedule of the length,
 * timing the whole persistent launch on `in`/`out` (median of
 * `reps` after one warm-up; `out` is overwritten), keeping each change that
 * makes it faster.  *best_ms (may be NULL) receives the best median time.
 * Synchronous.
 */
gbfft_status gbfft_ragged_autotune(gbfft_plan p, const void *in, void *out, int reps, float *best_ms);

/* Queue order of a ragged plan.  0: one queue, all items by work, heaviest
 * first.  1 (default): one queue, the items of one length together, heaviest
 * length first.  2: one sub-queue per length (in the order of 1), each SM
 * starting on a home sub-queue (SMs dealt to lengths in proportion to their
 * elements) and moving on to the next sub-queue when its own is exhausted, so
 * that an SM runs few distinct lengths.  Every order computes the same
 * results.  gbfft_ragged_set_queue_order sets it and rebuilds the queue
 * (INVALID_ARG for another value or plan kind); gbfft_ragged_queue_order
 * returns it (-1 if not a ragged plan).  The autotuner tries all three. */
gbfft_status gbfft_ragged_set_queue_order(gbfft_plan p, int order);
int gbfft_ragged_queue_order(gbfft_plan p);

/* Radix schedule the plan uses for length n: its stage count (0 if n is not in
 * the plan, -1 if not a ragged plan), radices written to `radices` (up to 8;
 * may be NULL).  The autotuner may switch a length to an alternative schedule. */
int gbfft_ragged_schedule(gbfft_plan p, int64_t n, int *radices);

/* Number of work items in the plan's queue (-1 if not a ragged plan). */
int64_t gbfft_ragged_num_items(gbfft_plan p);

/* The tile split the plan uses for length n (rows per item = (rows of the
 * tile)/split; the run-time engine's tile holds min(8192/n, 512) rows, a
 * compiled schedule's its own), 0 if n is not in this plan. */
int gbfft_ragged_tile_split(gbfft_plan p, int64_t n);

/*
 * Engine of a length in a ragged plan.  Lengths n = p * 2^k (p = 1, 3, 5, 7,
 * 8 <= n <= 8192) have a compiled schedule inside the persistent kernel (the
 * single-pass stage engine with the schedule and the tile fixed at compile
 * time; the default for those lengths); every length can also run the
 * run-time engine, which reads its radix schedule from the length's
 * descriptor.  gbfft_ragged_set_engine switches length n (n = 0: every length
 * of the plan; lengths without a compiled schedule then keep the run-time
 * engine) to the compiled (1) or run-time (0) engine and rebuilds the queue;
 * NOT_FOUND if n is not in the plan or has no compiled schedule (compiled =
 * 1), INVALID_ARG for other values.  gbfft_ragged_engine returns 1 / 0 for
 * length n, -1 if n is not in the plan or p is not a ragged plan.  The
 * autotuner may switch either way.
 */
gbfft_status gbfft_ragged_set_engine(gbfft_plan p, int64_t n, int compiled);
int gbfft_ragged_engine(gbfft_plan p, int64_t n);

/*
 * Failure injection and its bound (host side; never faults the GPU): mark
 * queue item `item` ready (nonzero) or not ready (0).  A CTA that claims an
 * item that is not ready waits for it at most the wait limit
 * (gbfft_ragged_set_wait_limit, default 200 ms, 1 us .. 10 s), then records
 * GBFFT_ERR_TIMEOUT in the plan's status word (gbfft_plan_device_status),
 * leaves that item's output untouched and continues with the queue.
 */
gbfft_status gbfft_ragged_set_item_ready(gbfft_plan p, int64_t item, int ready);
gbfft_status gbfft_ragged_set_wait_limit(gbfft_plan p, int64_t nanoseconds);

/*
 * Serving loop (native, one worker thread per server): continuous batching of
 * FFT requests under a device-memory budget.
 *
 * gbfft_server_create: `mem_budget_bytes` of device memory is reserved once
 * (one cudaMalloc) as the arena every admitted request's slot comes from;
 * `n_streams` (1..64) streams carry the groups.  Flags: GBFFT_SERVER_SERIAL
 * turns batching off (one request in flight, one stream: the naive queue);
 * GBFFT_SERVER_PHASES records timing events around every group's copies in,
 * transform and copies out (gbfft_server_phases); GBFFT_SERVER_PER_LENGTH
 * groups requests by (n, direction) only, without ragged launches;
 * GBFFT_SERVER_STAGED always copies rows through the arena (see below).
 * gbfft_server_submit queues a request - `batch` rows of length n (any length
 * gbfft_plan_create supports), direction, input and output buffers of
 * 8*n*batch bytes each, in host memory (page-locked for overlap) or device
 * memory (the copies use the unified address space: cudaMemcpyDefault); they
 * must stay valid until the request completes - stamps its arrival time and
 * returns a ticket.  BUDGET if the request alone exceeds the arena,
 * UNSUPPORTED_SIZE for lengths with no plan.  The worker admits queued
 * requests in FIFO order while their slots fit in the arena.  Admitted
 * requests of lengths n <= 8192 with prime factors 2, 3, 5, 7 are batched
 * across lengths: per direction, one slot holds all of them and ONE launch of
 * the persistent ragged kernel (gbfft_plan_ragged's kernel, its queue of
 * (length, rows) items built on the host and uploaded with one copy)
 * transforms every row.  When a request's input and output are both
 * device-visible (device memory, or page-locked host memory mapped into the
 * device's address space, which on a Grace-Blackwell node the GPU reaches
 * over NVLink-C2C) the launch reads and writes them in place where they are,
 * with no copies and no arena bytes for its rows; otherwise its rows are
 * copied into the slot, transformed there and copied back.  Input and output
 * must then not overlap partially (the same buffer is fine).  The other
 * lengths (and every length with GBFFT_SERVER_PER_LENGTH) are grouped by
 * (n, direction): device-visible, 16-byte aligned requests are transformed
 * where they are (the group's slot holds only a two-pass workspace), others
 * are copied into one slot and transformed there by one launch.  Each group
 * runs on the stream with the fewest bytes in flight: requests arriving
 * while earlier groups run are
 * admitted as memory frees up and overlap them.  Schedules, ragged length
 * descriptors and twiddle tables are built once per length and stay resident
 * (gbfft_server_prepare builds them ahead).  An event recorded after each
 * group's copies back, polled by the worker, stamps completion; latency is
 * completion - arrival.
 * gbfft_server_poll: *done = 1 finished, 0 pending, -1 failed/cancelled;
 * *latency_s once finished.  gbfft_server_timing splits a finished request's
 * latency: *queued_s = admission - arrival (waiting in the server's queue),
 * *latency_s as gbfft_server_poll (INVALID_ARG until finished).
 * gbfft_server_phases fills out8 for a finished request (INVALID_ARG until
 * then) with the phases of its service in seconds: {queued (admission -
 * arrival), host (the worker issuing the group's copies and launches), device
 * wait (start of the group's first copy on the device - end of that issue),
 * copies in, transform, copies out, observe (the worker seeing the completion
 * - end of the copies back on the device), latency}; device-side phases are
 * placed on the host clock through an event recorded at server creation, and
 * are NaN unless the server was created with GBFFT_SERVER_PHASES.
 * gbfft_server_wait blocks up to timeout_s
 * (TIMEOUT otherwise).  gbfft_server_release forgets a finished ticket.
 * gbfft_server_replay submits `count` requests at arrival offsets arrival_s[i]
 * (seconds after the call, non-decreasing) from the calling thread - an open
 * loop generator - and returns their tickets.
 * gbfft_server_stats fills out10 = {completed, p50 latency s, p99 latency s,
 * max latency s, requests/s, GB/s (16*n*batch bytes per request), groups
 * launched, max requests in flight, max arena bytes in use, window s}; the
 * window runs from the last reset/replay to the last completion.
 * gbfft_server_destroy cancels queued requests, waits for running ones and
 * frees everything.
 */
typedef struct gbfft_server_s *gbfft_server;
#define GBFFT_SERVER_SERIAL 1
#define GBFFT_SERVER_PHASES 2
#define GBFFT_SERVER_PER_LENGTH 4
#define GBFFT_SERVER_STAGED 8

gbfft_status gbfft_server_create(gbfft_server *out, size_t mem_budget_bytes, int n_streams, int flags);
gbfft_status gbfft_server_prepare(gbfft_server srv, int64_t n, int direction);
gbfft_status gbfft_server_submit(gbfft_server srv, int64_t n, int64_t batch, int direction, const void *host_or_dev_in,
                                 void *host_or_dev_out, uint64_t *ticket);
gbfft_status gbfft_server_poll(gbfft_server srv, uint64_t ticket, int *done, double *latency_s);
gbfft_status gbfft_server_timing(gbfft_server srv, uint64_t ticket, double *queued_s, double *latency_s);
gbfft_status gbfft_server_phases(gbfft_server srv, uint64_t ticket, double *out8);
gbfft_status gbfft_server_wait(gbfft_server srv, uint64_t ticket, double timeout_s);
gbfft_status gbfft_server_release(gbfft_server srv, uint64_t ticket);
gbfft_status gbfft_server_replay(gbfft_server srv, int64_t count, const int64_t *n, const int64_t *batch,
                                 const int *direction, const void *const *host_in, void *const *host_out,
                                 const double *arrival_s, uint64_t *tickets);
gbfft_status gbfft_server_stats(gbfft_server srv, double *out10);
gbfft_status gbfft_server_reset_stats(gbfft_server srv);
gbfft_status gbfft_server_destroy(gbfft_server srv);

/*
 * Allocation-free two-pass transform (the paper has no counterpart: this is
 * a deployment convenience of this library).  For callers that cannot
 * allocate device memory at the time of the call - hosts that own all device
 * memory through their own fixed arena and forbid further cudaMalloc, or
 * real-time loops that must not allocate after start-up - this computes
 * out = DFT_N in for `batch` rows exactly like a two-pass plan from
 * gbfft_plan_create_twopass(..., 0), without a plan: the workspace and the
 * twiddle tables live in one static device array of 64 MiB that is part of
 * the library image, so every GPU that loads the library holds those 64 MiB
 * until the process exits.  The tables are regenerated on the stream by each
 * call; `in`/`out` are caller-owned device pointers as for gbfft_execute.
 * Limits: 8*n*batch bytes of workspace plus the tables (8*n bytes and the
 * stage blocks, each rounded up to 256 bytes) must fit in the 64 MiB, else
 * GBFFT_ERR_BUDGET (checked before any byte count is formed, so a huge batch
 * cannot wrap it); n must have a two-pass split (UNSUPPORTED_SIZE).  The
 * array's device address belongs to the CUDA context that loaded the library's
 * module: the first call on a device looks it up in the current context, and
 * every later call whose stream is not capturing looks it up again, so a
 * device reset or another current context never leaves a stale address in
 * use.  Make the first call on each device before any stream capture.  All
 * calls share the array and it keeps the last call's contents: calls that
 * overlap on the GPU race and corrupt each other, so serialise them.  The call
 * makes no cudaMalloc/cudaFree.  Errors: INVALID_ARG, ALIGNMENT, OVERLAP,
 * UNSUPPORTED_SIZE, BUDGET, CUDA.
 */
gbfft_status gbfft_execute_twopass_noalloc(int64_t n, int64_t batch, int direction, const void *in, void *out,
                                           void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GBFFT_H */
