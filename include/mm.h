/*
 * mm.h -- C ABI of libmm, a single-GPU GB300 (sm_103a) library for the dense
 * matrix product C = A*B.
 *
 * The operation is the paper's matrix product (Sec. III): A is m x k, B is
 * k x n, C is m x n and C[i][j] = sum_p A[i][p] * B[p][j], the dot product of
 * row i of A with column j of B. All matrices are row-major, as in the paper's
 * C program (Sec. III, row-major storage), with leading dimensions
 * lda >= k, ldb >= n, ldc >= n counted in elements. (The paper names the
 * shapes m x n and n x p; here n -> k and p -> n.) Inputs and outputs are IEEE
 * binary64 (double) in every precision mode.
 *
 * Precision modes (mm_precision):
 *   MM_FP64      plain FP64 arithmetic on the FP64 pipe (the paper's
 *                computation, Sec. V). Inf and NaN propagate as in IEEE.
 *   MM_FP64_EMU  FP64-accuracy emulation: per-row (A) and per-column (B)
 *                power-of-two scaling, each entry rounded to t*s bits and split
 *                into s signed 8-bit integer slices held in bfloat16, slice
 *                products on the tcgen05 tensor cores with exact FP32 partial
 *                sums, exact integer recombination, one rounding to double
 *                (Ozaki, Ogita, Oishi, Rump 2012; Ootomo, Ozaki, Yokota 2024).
 *                The slice count s is chosen on the device for each product
 *                from the spread of its rows and columns (mm_slice_count_rule)
 *                so that the error stays near half of the componentwise
 *                bound 4k*2^-53 * (|A||B|); where no s <= 7 would, the product
 *                runs on the plain FP64 kernel instead (see mm_gemm).
 *                Products take the modular form instead where it fits
 *                (Ozaki, Uchino, Imamura 2025, "Ozaki scheme II"): the same
 *                scaled integers, b bits each, reduced modulo N <= 14 pairwise
 *                coprime moduli <= 256 (residues held in bfloat16), one
 *                residue product per modulus on tcgen05, each product reduced
 *                modulo its modulus, the exact integer product rebuilt by the
 *                Chinese remainder theorem and rounded once: N products
 *                instead of s(s+1)/2 (12 against 15 at M = N = K = 8192 on
 *                the benchmark inputs) for products with m*n*k >= 2^33; see
 *                mm_crt_rule and MM_OPT_FP64_SCHEME.
 *   MM_FP32_EMU  FP32-accuracy emulation: three bfloat16 slices per scaled
 *                entry and the six slice products with index sum <= 2, FP32
 *                accumulation on tcgen05. Bound 4k*2^-24 * (|A||B|).
 *
 * Status codes: every entry point returns an int status (MM_OK = 0 on
 * success); mm_status_string() gives a static English description.
 *
 * Ownership: the caller owns A, B, C and any stream it passes; the library owns
 * every workspace it allocates (from a per-handle stream-ordered pool, charged
 * against the handle's memory budget) and frees it with the handle.
 *
 * Threading: mm_gemm / mm_gemm_grouped may be called from several host threads
 * on distinct streams; the serving calls are thread-safe. A handle must not be
 * used after mm_destroy.
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ types */

typedef struct mm_handle_s *mm_handle;

typedef enum {
    MM_FP64 = 0,
    MM_FP64_EMU = 1,
    MM_FP32_EMU = 2
} mm_precision;

enum {
    MM_OK = 0,
    MM_PENDING = 1,          /* serve: request not finished yet */
    MM_ERR_INVALID_ARG = 2,  /* null pointer, negative size, ld too small, C overlapping A or B, unknown mode */
    MM_ERR_BUDGET = 3,       /* the request needs more device memory than the handle's budget */
    MM_ERR_NONFINITE = 4,    /* emulated mode met Inf or NaN in A or B */
    MM_ERR_CUDA = 5,         /* a CUDA runtime or driver call failed */
    MM_ERR_TIMEOUT = 6,      /* a bounded device-side wait ran out; the kernel returned early */
    MM_ERR_NOT_FOUND = 7,    /* serve: unknown or already collected ticket; tune: no entry, no file */
    MM_ERR_SHUTDOWN = 8,     /* serve: handle is being destroyed; request cancelled */
    MM_ERR_UNSUPPORTED = 9   /* no sm_100-family GPU (tcgen05) present */
};

/* One product C = A*B of the grouped and serving calls. Device pointers. */
typedef struct {
    int64_t m, n, k;
    const double *A; int64_t lda;
    const double *B; int64_t ldb;
    double *C;       int64_t ldc;
} mm_problem;

/* A serving request: the product, its accuracy class and a caller tag. The
 * operands are caller-owned device memory that must stay valid and unchanged
 * until the request completes. */
typedef struct {
    mm_problem prob;
    int precision;           /* an mm_precision */
    uint64_t user_tag;
} mm_request;

/* Completion record of a serving request. Times are microseconds on the
 * host's steady clock, measured from mm_create. */
typedef struct {
    int status;              /* MM_OK, MM_PENDING or the request's error */
    uint64_t user_tag;
    double t_submit_us;      /* mm_serve_submit returned */
    double t_admit_us;       /* admitted: memory reserved, queued for a batch */
    double t_launch_us;      /* its batch was launched */
    double t_done_us;        /* its batch finished on the GPU (host saw the event) */
    int32_t stream;          /* the serving stream its batch ran on (0 .. MM_OPT_SERVE_STREAMS-1) */
    double t_gpu_start_us;   /* its batch's work began on the GPU (device clock, CUDA events, */
    double t_gpu_end_us;     /*   from a reference event recorded when serving started) and ended */
} mm_req_status;

/* -------------------------------------------------------------- lifecycle */

/* Create a handle on CUDA device `device`. mem_budget_bytes caps the device
 * memory the handle may hold for workspaces and serving (0 = 40 GiB). Starts
 * the serving thread lazily (first mm_serve_submit).
 * Errors: MM_ERR_INVALID_ARG (out == NULL), MM_ERR_CUDA (no such device),
 * MM_ERR_UNSUPPORTED (device is not compute capability 10.x). */
int mm_create(mm_handle *out, int device, size_t mem_budget_bytes);

/* Finish or cancel every pending serving request (pending ones complete with
 * MM_ERR_SHUTDOWN), wait for the handle's GPU work, free everything. */
int mm_destroy(mm_handle h);

const char *mm_status_string(int status);

/* -------------------------------------------------------------------- GEMM */

/* C <- A*B (overwrite; no alpha or beta), Sec. III definition, row-major.
 * Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream):
 * returns once the kernels are queued. A, B, C are device pointers.
 * m == 0 or n == 0: nothing is done. k == 0: C is set to zero.
 * Argument errors (checked on the host before any launch): MM_ERR_INVALID_ARG
 * for NULL pointers with nonzero sizes, negative sizes, lda < k, ldb < n,
 * ldc < n, C overlapping A or B, or an unknown precision.
 * Device-side errors go to the error word of `stream` (each stream the handle
 * sees has its own), which mm_sync(h, stream) reports and clears: in the
 * emulated modes non-finite inputs make the affected rows/columns of C NaN
 * and report MM_ERR_NONFINITE; a device wait that ran out reports
 * MM_ERR_TIMEOUT (C is then incomplete).
 * MM_FP64_EMU slice count: with MM_OPT_SLICES = 0 (default) it is decided on
 * the device, after the exponent scan, from alpha = min over rows of
 * mean|a_ik| / 2^E_i and beta (the same over columns of B): the smallest s in
 * 3..7 with 0.3 * 6.5 * 2^(53-8s) <= 0.5 * 4 k sqrt(k) alpha beta (an estimate
 * of the largest error against half the bound; mm_slice_count_rule), else
 * the product runs on the plain FP64 kernel. The estimate takes the rows' and
 * columns' magnitudes as independent of each other; inputs built so that a
 * row's large entries meet a column's tiny ones can still exceed the bound.
 * The kernels for every candidate count are queued, and each returns at once
 * unless the count decided on the device is its own. For k <= 4 MM_FP64_EMU
 * computes with the FP64 kernel (per-row scaling to <= 56 bits cannot meet
 * the FP64 bound for such short sums). */
int mm_gemm(mm_handle h, int64_t m, int64_t n, int64_t k,
            const double *A, int64_t lda, const double *B, int64_t ldb,
            double *C, int64_t ldc, int precision, void *stream);

/* Same product with HOST operands (pageable or pinned): copies A and B to
 * device workspace, computes, copies C back, and synchronises. Returns the
 * device-side status of `stream` (including MM_ERR_NONFINITE /
 * MM_ERR_TIMEOUT). */
int mm_gemm_host(mm_handle h, int64_t m, int64_t n, int64_t k,
                 const double *A, int64_t lda, const double *B, int64_t ldb,
                 double *C, int64_t ldc, int precision, void *stream);

/* Wait for `stream` and return (and clear) the device status of the work the
 * handle queued on that stream: MM_OK, MM_ERR_NONFINITE or MM_ERR_TIMEOUT.
 * Streams are told apart by their cudaStream_t value; beyond 255 distinct
 * streams per handle the rest share one word. */
int mm_sync(mm_handle h, void *stream);

/* `count` independent products in one persistent launch per stage (the split
 * kernels, then the slice GEMM, for the emulated modes; one FP64 kernel for
 * MM_FP64), replayed from a CUDA graph. The graph is captured once per
 * (precision, stream, launch configuration) and again only when a call needs
 * more problems, tiles or workspace than the captured capacities; every call
 * copies its descriptors into it first. The launch configuration comes from
 * the autotuner's table (MM_OPT_AUTOTUNE) or the defaults. Each problem's
 * result equals mm_gemm on that problem: bit-identical for MM_FP64_EMU (the
 * same decision from the same spreads, the modular form's exact rebuild or
 * the digit form's exact recombination, whatever the tiles) and for
 * MM_FP64 when both use the same FP64 tile kernel; within its bound for
 * MM_FP32_EMU. Problems may have any shapes; their C must not overlap any A
 * or B. Errors as for mm_gemm, checked for every problem. The call blocks only
 * while it tunes, or when both graph slots are still running earlier calls. */
int mm_gemm_grouped(mm_handle h, int count, const mm_problem *probs,
                    int precision, void *stream);

/* ----------------------------------------------------------------- serving */

/* Queue a request (non-blocking); *ticket identifies it. The serving thread
 * admits queued requests while their workspace fits the memory budget and a
 * batch slot is free, groups admitted requests into grouped launches on two
 * or more streams so batches overlap, and records a completion event per
 * batch. Errors: MM_ERR_INVALID_ARG (bad problem), MM_ERR_BUDGET (one request
 * larger than the whole budget), MM_ERR_SHUTDOWN. */
int mm_serve_submit(mm_handle h, const mm_request *r, uint64_t *ticket);

/* Non-blocking poll: MM_OK (done; C is complete and *st filled; the ticket is
 * released), MM_PENDING (not yet), MM_ERR_NOT_FOUND (unknown ticket) or the
 * request's own error (also released): MM_ERR_NONFINITE when its own operands
 * held Inf/NaN (other requests of its batch are not affected), MM_ERR_TIMEOUT
 * when a device wait of its batch ran out (every request of that batch),
 * MM_ERR_CUDA on a launch failure. st may be NULL. */
int mm_serve_poll(mm_handle h, uint64_t ticket, mm_req_status *st);

/* Block until every submitted request has completed (or failed). */
int mm_serve_drain(mm_handle h);

/* ---------------------------------------------------------- configuration */

/* Options (mm_set_option / mm_get_option). */
enum {
    MM_OPT_SLICES = 1,        /* FP64-accuracy slice count s (0 = decided on the device for each
                                 product, see mm_gemm; else 3..7 for every product; the environment
                                 variable MM_SLICES sets it at mm_create) */
    MM_OPT_TIMEOUT_MS = 2,    /* bound on every device-side wait (default 2000) */
    MM_OPT_AUTOTUNE = 3,      /* 1 = on the first product (or group) of a shape bucket, time every
                                 candidate launch configuration on the caller's stream (blocking
                                 that call) and keep the fastest; see mm_tune_save */
    MM_OPT_SERVE_MAX_BATCH = 4,   /* requests per grouped launch (default 32) */
    MM_OPT_SERVE_STREAMS = 5,     /* serving streams (default 4) */
    MM_OPT_FP64_KERNEL = 6,       /* 0 = automatic, 1 = DFMA tiles, 2 = DMMA (mma.sync f64) tiles */
    MM_OPT_PROFILE = 7,           /* 1 = time every kernel launch with CUDA events (see mm_profile_read) */
    MM_OPT_CTA_PAIR = 8,          /* emulated products: 0 = automatic, 1 = one CTA per 128-row tile,
                                     2 = CTA pairs (cta_group::2) on 256-row tiles, 3 = CTA pairs in
                                     clusters of two on adjacent 256-wide tiles sharing A (each CTA
                                     loads half of its A rows for both pairs; single products whose
                                     tile-column count is even, else pairs) */
    MM_OPT_TILE_N = 9,            /* FP64-accuracy tile width: 0 = automatic, 128, 192, 240 or 256
                                     columns. Every choice gives the same bits. */
    MM_OPT_INT8_SLICES = 11,      /* 1 = FP64-accuracy single products (mm_gemm, mm_gemm_host) on
                                     signed-byte digits with the legacy integer tensor path
                                     (mma.sync m16n8k32 s8, int32 sums): scale exponent one larger
                                     (E = floor(log2 max) + 3, every digit in [-128, 127]), the
                                     automatic count from halved spreads, the same exact
                                     recombination. Slower on GB300 than the default bfloat16
                                     digits on tcgen05; kept for comparison. Grouped and served
                                     products always use the default. */
    MM_OPT_FP64_SCHEME = 12       /* FP64-accuracy products with the automatic slice count
                                     (MM_OPT_SLICES = 0), single, grouped and served: 0 = the
                                     modular form where mm_crt_rule fits and m*n*k >= 2^33, else
                                     the digit form (default: smaller products run faster on the
                                     digit form, whose split is shorter and whose epilogue a CTA
                                     with few tiles need not overlap); 1 = the digit form only;
                                     2 = the modular form wherever mm_crt_rule fits. */
};

/* Kernel classes for mm_profile_read. */
enum {
    MM_KERNEL_SLICE_GEMM = 0,     /* tcgen05 slice products + recombination (emulated modes) */
    MM_KERNEL_SPLIT = 1,          /* exponent scan and slicing of both operands */
    MM_KERNEL_FP64_GEMM = 2,      /* plain FP64 tile kernel */
    MM_KERNEL_REBUILD = 3         /* the modular form's rebuild of C from the residue bytes (single
                                     products; grouped launches rebuild inside the slice GEMM) */
};
int mm_set_option(mm_handle h, int option, int64_t value);
int mm_get_option(mm_handle h, int option, int64_t *value);

/* The automatic FP64-accuracy slice count for inner dimension k when the
 * smallest row spread of A is alpha_min and that of B's columns beta_min
 * (spread = mean |entry| / 2^E, E = floor(log2 max |entry|) + 2, so spreads
 * lie in (0, 1/2); +inf for no constraint). Error estimate: one term a_ik b_kj
 * carries an error of standard deviation at most 0.3 * 2^(E_i+F_j-8s) (digit
 * rounding plus the dropped level s+2 with independent uniform digits), k terms
 * grow it by sqrt(k), the largest output stays within 6.5 deviations, and the
 * bound is about 4k 2^-53 * k alpha beta 2^(E_i+F_j). Returns the smallest s
 * in 3..7 whose estimate is at most half the bound, 8 when none is (the
 * product then runs on the plain FP64 kernel), -1 for k < 1. The same function
 * runs on the device; the decision is evaluated in double. */
int mm_slice_count_rule(int64_t k, float alpha_min, float beta_min);

/* The modular form's parameters for inner dimension k and the smallest
 * spreads (as for mm_slice_count_rule). Its error comes only from rounding
 * each scaled entry to a b-bit integer (the residue products and the rebuild
 * are exact): one term carries an error of standard deviation at most
 * 0.21 * 2^(E_i+F_j-b). b0 is the smallest b in 24..53 with
 * 0.21 * 6.5 * 2^(53-b) <= 0.5 * 4 k sqrt(k) alpha beta (double arithmetic);
 * N the fewest moduli, taken in the order 256, 255, 253, 251, 247, 241, 239,
 * 233, 229, 227, 223, 217, 211, 199, whose product M_N exceeds k 2^(2 b0 - 1)
 * (so every output's integer sum lies inside (-M_N/2, M_N/2)); b then the
 * largest bit count, at most 53, those N moduli still hold. Returns N and
 * *bits = b, or 0 when no b in range qualifies or 14 moduli do not hold it
 * (the product then takes the digit form); -1 for k < 1 or bits == NULL. */
int mm_crt_rule(int64_t k, float alpha_min, float beta_min, int *bits);

/* ---------------------------------------------------------------- autotuner */

/* The tuning table maps shape buckets to launch configurations. Buckets:
 * single products by (precision, ceil(log2 m), ceil(log2 n), ceil(log2 k));
 * grouped calls by (precision, ceil(log2 count), ceil(log2 d)) where d is the
 * mean over the group of (m*n*k)^(1/3). Configurations: tile width (128, 192,
 * 240, 256) and CTAs per tile (1, 2) for the emulated modes, the FP64 tile
 * kernel (1 = DFMA, 2 = DMMA) for the plain mode. Entries are filled by
 * MM_OPT_AUTOTUNE or loaded from a file; explicit tile options
 * (MM_OPT_TILE_N, MM_OPT_CTA_PAIR, MM_OPT_FP64_KERNEL) take precedence. The
 * FP64-accuracy result never depends on the configuration.
 *
 * mm_tune_save writes the table as text (a header line, then one entry per
 * line: kind precision b0 b1 b2 bn cg kern ms); MM_ERR_INVALID_ARG if the
 * file cannot be written. mm_tune_load merges a saved table into the handle's;
 * MM_ERR_NOT_FOUND if the file does not exist, MM_ERR_INVALID_ARG (and nothing
 * merged) if any line is malformed or names a configuration the library
 * cannot launch. */
int mm_tune_save(mm_handle h, const char *path);
int mm_tune_load(mm_handle h, const char *path);

/* The configuration tuned for a bucket: grouped = 0 looks up the single
 * product (a, b, c) = (m, n, k); grouped = 1 the group bucket of a problems of
 * mean dimension b (c unused). MM_ERR_NOT_FOUND if the bucket has no entry. */
int mm_tune_lookup(mm_handle h, int grouped, int precision, int64_t a, int64_t b, int64_t c,
                   int *bn, int *cg, int *kern);

/* --------------------------------------------------- inputs and diagnostics */

/* Fill a rows x cols row-major device matrix (leading dimension ld) with the
 * seeded SplitMix64 counter-based uniform[-1,1) values (element (r,c) draws
 * counter r*cols+c of stream `stream_id`), optionally times 2^e with one
 * integer e uniform on [-20,20] per row (scale_mode 1) or per column
 * (scale_mode 2). Same definition as the Python input module. */
int mm_fill_uniform(double *X, int64_t rows, int64_t cols, int64_t ld,
                    uint64_t seed, uint64_t stream_id, int scale_mode,
                    uint64_t exp_stream_id, void *stream);

/* Exponents and slices as the emulated modes compute them, for checking the
 * integer work bit for bit. mode: MM_FP64_EMU or MM_FP32_EMU. For A (rows of
 * an m x k matrix, which = 0) or B (columns of a k x n matrix, which = 1):
 * exps[rows or cols] (int32) and slices[s][rows or cols][k] as bfloat16 bit
 * patterns (uint16; B's slices are transposed, K contiguous). s is the slice
 * count (FP64_EMU) or 3 (FP32_EMU). Device pointers; synchronous. */
int mm_debug_slices(mm_handle h, int which, int mode, int s,
                    int64_t rows, int64_t cols, const double *X, int64_t ldx,
                    int32_t *exps, uint16_t *slices, void *stream);

/* The automatic slice count of the product A*B as the device decides it
 * (scan, spreads, rule), with the smallest row and column spreads it used.
 * Device operands; synchronous. */
int mm_debug_slice_count(mm_handle h, int64_t m, int64_t n, int64_t k,
                         const double *A, int64_t lda, const double *B, int64_t ldb,
                         int *s, float *alpha_min, float *beta_min, void *stream);

/* The modular form's centred residues as the splitting kernel computes them,
 * for N moduli and b-bit scaled integers (given, not decided): for A (which =
 * 0, rows of an m x k matrix) or B (which = 1, columns of a k x n matrix),
 * exps[rows or cols] (int32, floor(log2 max) + 2) and planes[N][rows or
 * cols][k] as bfloat16 bit patterns (residue modulo the l-th modulus of
 * round-half-even(x 2^(b - E)), in [-floor(m/2), ceil(m/2) - 1]). Device
 * pointers; synchronous. */
int mm_debug_crt_residues(mm_handle h, int which, int N, int bits, int64_t rows, int64_t cols,
                          const double *X, int64_t ldx, int32_t *exps, uint16_t *planes, void *stream);

/* The modular form's rebuild pass alone, as it follows the slice GEMM of a
 * single product (Ozaki scheme II, the Chinese-remainder step): C[i][j] =
 * round-to-nearest(Y_ij 2^(E_i + F_j - 2 bits)), Y_ij the integer in
 * [-M_N/2, M_N/2) congruent to res's byte of (i, j) modulo the l-th modulus
 * for l < N (any byte value; it is taken modulo its modulus). res: the slice
 * GEMM's layout, plane l at res + l * m * 8 * ceil(n/8), within a plane
 * ceil(n/8) blocks of 8 columns, each block the m rows' 8-byte records in row
 * order. E (m), F (n): int32 exponents; an exponent of -1000000 marks a
 * non-finite row or column (NaN out). Device pointers; synchronous.
 * MM_ERR_INVALID_ARG for N outside 1..14, bits outside 1..53, m or n <= 0,
 * null pointers or ldc < n. */
int mm_debug_crt_rebuild(mm_handle h, int64_t m, int64_t n, int N, int bits, const uint8_t *res,
                         const int32_t *E, const int32_t *F, double *C, int64_t ldc, void *stream);

/* One automatic FP64-accuracy product (k > 4) as mm_gemm runs it, with the
 * device's decision: *code = SLICE count 3..7 (digit form), 8 (plain FP64
 * kernel) or 16 + N (modular form with N moduli and *bits = b), the smallest
 * spreads it used, and for the modular form the products' residues modulo
 * their moduli (bytes, [N][m][n], to res when res != NULL; capacity
 * 14*m*n). Device pointers; synchronous. */
int mm_debug_fp64_product(mm_handle h, int64_t m, int64_t n, int64_t k,
                          const double *A, int64_t lda, const double *B, int64_t ldb,
                          double *C, int64_t ldc, uint8_t *res, int *code, int *bits,
                          float *alpha_min, float *beta_min, void *stream);

/* The level products L_d (d = 2..s+1) of the FP64-accuracy mode as the
 * tensor-core kernel accumulates them (exact integers), written as int64
 * [s][m][n] to `levels` (device). Synchronous. */
int mm_debug_level_products(mm_handle h, int64_t m, int64_t n, int64_t k,
                            const double *A, int64_t lda, const double *B, int64_t ldb,
                            int s, int64_t *levels, void *stream);

/* The level products of the INT8 digit form (E = floor(log2 max) + 3,
 * digits as signed bytes) as the mma.sync s8 kernel accumulates them (exact
 * integers), int64 [s][m][n] to `levels` (device). Synchronous. */
int mm_debug_level_products_int8(mm_handle h, int64_t m, int64_t n, int64_t k,
                                 const double *A, int64_t lda, const double *B, int64_t ldb,
                                 int s, int64_t *levels, void *stream);

/* Failure-detection check of the device-side waits: launches one thread
 * that waits, with the same bounded wait every kernel of the library uses, on
 * an mbarrier that nothing arrives at, for timeout_ms (1..10000). The wait
 * gives up, the kernel returns and the call reports MM_ERR_TIMEOUT; the
 * context stays usable. Synchronous. */
int mm_debug_wait_timeout(mm_handle h, int64_t timeout_ms, void *stream);

/* Device peak microbenchmarks: FP64 DFMA and DMMA (mma.sync f64) rates in
 * TFLOP/s, each from a fixed-length register-resident loop on every SM. */
int mm_peak_fp64(mm_handle h, double *dfma_tflops, double *dmma_tflops);

/* Library counters since mm_create: kernels launched (all kinds). */
int mm_stats(mm_handle h, uint64_t *kernel_launches);

/* With MM_OPT_PROFILE on, every launch of a kernel class is bracketed by CUDA
 * events recorded on the stream it runs on. This waits for the recorded
 * events and returns the summed device time (ms) and the launch count of
 * `kernel` (an MM_KERNEL_* class) since the last reset; reset != 0 clears. */
int mm_profile_read(mm_handle h, int kernel, double *total_ms, uint64_t *launches, int reset);

/* ------------------------------------------------------ serving benchmark */

/* A seeded synthetic request stream for mm_serve_bench. Request i has M, N, K
 * each drawn log-uniform on [dim_lo, dim_hi] (round(exp(U(ln lo, ln hi)))),
 * the FP64-accuracy class with probability fp64_share (else FP32-accuracy),
 * and arrives at the i-th point of a Poisson process of rate rate_per_s
 * (rate_per_s <= 0: closed loop, every request is due at once). Operands live
 * in `slots` resident slots (dim_hi x dim_hi A, B and C each, A and B filled
 * once by mm_fill_uniform with seed*1000003 + slot on streams 1 and 2); request
 * i uses slot i % slots (its top-left m x k, k x n, m x n corners, leading
 * dimension dim_hi) and waits for the slot's previous request to finish. */
typedef struct {
    int64_t count;
    int64_t dim_lo, dim_hi;
    double fp64_share;
    double rate_per_s;
    uint64_t seed;
    int slots;
    int64_t sample_every;     /* copy every n-th request's C to the host (0 = none) */
} mm_serve_load;

typedef struct {
    int64_t completed, failed;
    double wall_s;            /* first arrival to last completion */
    double req_per_s;
    double tflops;            /* sum of 2mnk over wall_s */
    double p50_ms, p90_ms, p99_ms, max_ms, mean_ms;   /* scheduled arrival -> completion */
    double fp64_p99_ms, fp32_p99_ms;
} mm_serve_load_result;

typedef struct {
    int64_t index, m, n, k;
    int precision, slot;
    int64_t host_offset;      /* element offset of its C (m x n, row-major) in sample_host */
} mm_serve_sample;

/* Run the stream through mm_serve_submit / mm_serve_poll on h (blocking).
 * Latency is measured from each request's scheduled arrival to the completion
 * time the serving engine records. Every sample_every-th request's C is copied
 * to sample_host (capacity sample_cap doubles) and described in samples
 * (capacity max_samples); *n_samples receives the count. Sampled outputs are
 * gathered in a device buffer of sample_cap doubles during the run and copied
 * to sample_host after it (MM_ERR_BUDGET if that buffer cannot be had). Slots
 * are allocated for the run and freed after it. */
int mm_serve_bench(mm_handle h, const mm_serve_load *load, mm_serve_load_result *res,
                   mm_serve_sample *samples, int64_t max_samples, int64_t *n_samples,
                   double *sample_host, int64_t sample_cap);

/* ---------------------------------------------------- allocation-free call */

/* The emulated product (MM_FP64_EMU or MM_FP32_EMU) with no device
 * allocation at all, for callers that cannot call cudaMalloc: code running in
 * a host callback or inside an allocator's own hooks, latency-critical loops
 * that must never pay cudaMalloc's implicit device synchronisation, or
 * processes that reserve their device memory up front and allow no later
 * allocation. The paper has no counterpart; this is a library service.
 *
 * Same product, layout and results as mm_gemm with the same precision on a
 * handle whose slice count is automatic (MM_OPT_SLICES = 0 and MM_SLICES
 * unset): the FP64-accuracy result is bit-identical. No handle: it runs on the calling
 * thread's current device, asynchronously on `stream` (NULL = legacy default
 * stream). A, B, C are caller-owned device pointers.
 * Scratch: one fixed 32 MiB array inside the library image, held by every GPU
 * that loads it until the process exits. The first call on a device looks up
 * that array's device address (do it before any stream capture). Every call
 * on a device shares the array, so calls whose GPU work overlaps race; each
 * call clears what must start at zero itself.
 * Errors: MM_ERR_INVALID_ARG (as mm_gemm, or another precision),
 * MM_ERR_BUDGET (the problem's split operands need more than the fixed
 * scratch: about 14*(m+n)*k bytes for FP64-accuracy, 6*(m+n)*k for
 * FP32-accuracy), MM_ERR_CUDA. The call does not wait for its kernels, so
 * their device-side status (Inf/NaN inputs, which give NaN in the affected
 * rows/columns of C; a device wait that ran out after 2 s, which leaves C
 * incomplete) is read afterwards with mm_gemm_emu_static_status. */
int mm_gemm_emu_static(int64_t m, int64_t n, int64_t k,
                       const double *A, int64_t lda, const double *B, int64_t ldb,
                       double *C, int64_t ldc, int precision, void *stream);

/* The device-side status of the last mm_gemm_emu_static call on the calling
 * thread's current device (each call clears the scratch's status word when it
 * starts, in stream order): synchronises `stream` (the stream that call ran
 * on), reads the word and clears it. MM_OK; MM_ERR_NONFINITE (A or B held Inf
 * or NaN); MM_ERR_TIMEOUT (a device wait ran out, C is incomplete);
 * MM_ERR_CUDA. Calls on other streams that overlap race on the same word,
 * as they do on the scratch. */
int mm_gemm_emu_static_status(void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
