/*
 * btas.h -- C ABI of the GB300 (sm_103a) Basic Tropical Algebra Subroutines.
 *
 * Tropical semirings (Sec. I): max-plus, x (+) y = max(x, y), x (.) y = x + y
 * (Eq. 1-2), and min-plus, x (+) y = min(x, y), x (.) y = x + y (Eq. 3-4).
 * The library offers the "standard vector and matrix operations" of the
 * abstract and Sec. III in the BLAS style the paper takes as its model
 * (Related Work), plus all-pairs shortest paths by repeated squaring of the
 * weighted adjacency matrix (Sec. III).
 *
 * Conventions shared by every entry point
 *  - Matrices are dense and row-major (the paper indexes a[x][y] and
 *    a*M+b, Algorithms 2 and 3); leading dimensions are in elements.
 *  - Every array argument is a DEVICE pointer owned by the caller, unless the
 *    argument's description says "host".  The library never frees a caller's
 *    pointer.  Temporary device workspace is taken stream-ordered (on
 *    `stream`) from a memory pool the library owns per device, and released
 *    on the same stream; see btas_workspace_reserved.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All work is enqueued asynchronously on it; a call returns once
 *    the work is enqueued, except where an out-parameter needs a device
 *    result (documented per call), in which case the call synchronises
 *    `stream`.
 *  - Argument errors are detected on the host before anything is enqueued
 *    and return BTAS_ERR_ARG (nothing is written).  A failed CUDA call returns
 *    BTAS_ERR_CUDA.  btas_last_error_string() describes the most recent
 *    failure of the calling thread.
 *  - Tracing: every level-2/3 and APSP entry point is an NVTX range named
 *    after it (visible to Nsight tools).  BTAS_LOG=1 in the environment
 *    (read once per process) prints each call's execution choices -- the
 *    product kernel and where its choice came from, the APSP size regime and
 *    representations -- to stderr.
 *
 * Integer encoding of "no edge" / the semiring zero
 *  The paper marks a missing edge with 0 (Algorithm 2) or -1 (Algorithm 3);
 *  this library uses a dedicated value instead:
 *    BTAS_INF_I32  = 0x3FFFFFFF   min-plus (+)-identity, absorbing for (.)
 *    BTAS_NINF_I32 = -0x3FFFFFFF  max-plus (+)-identity, absorbing for (.)
 *  Finite int32 operands must lie in [-BTAS_I32_FINITE_MAX, BTAS_I32_FINITE_MAX]
 *  (2^28).  Then every sum of two operands fits in int32, and a result equal
 *  to or beyond BTAS_INF_I32 - 2^28 (resp. below -(BTAS_INF_I32 - 2^28)) can
 *  only come from an INF term and is stored as BTAS_INF_I32
 *  (BTAS_NINF_I32).  Finite results are exact.
 *  The 16-bit storage type (BTAS_U16) holds min-plus values in [0, 0x7FFF];
 *  BTAS_INF_U16 = 0x7FFF is INF and every result saturates at it.
 *  FP32 uses IEEE +inf (min-plus) / -inf (max-plus); each term a + b is one
 *  round-to-nearest-even add, so results are independent of summation order
 *  and bit-exact.  NaN, -inf in min-plus and +inf in max-plus operands are
 *  outside the domain.
 */
#ifndef BTAS_H
#define BTAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BTAS_INF_I32 0x3FFFFFFF
#define BTAS_NINF_I32 (-0x3FFFFFFF)
#define BTAS_I32_FINITE_MAX (1 << 28)
#define BTAS_INF_U16 0x7FFF

/* Semiring selector; may be OR-ed with the BTAS_GEMM_* flags below. */
typedef enum {
    BTAS_MINPLUS = 0, /* Eq. 3-4 */
    BTAS_MAXPLUS = 1  /* Eq. 1-2 */
} btas_semiring;

/* Flags OR-ed into the semiring argument of btas_gemm. */
#define BTAS_GEMM_ACCUMULATE 0x100 /* C <- C (+) A (.) B, the paper's Z <- Z (+) X (.) Y */
#define BTAS_GEMM_TRANS_B 0x200    /* B is given transposed: an n x k row-major matrix */
#define BTAS_GEMM_NO_CARRIER 0x400 /* accepted and ignored: btas_gemm changes representation only
                                       with BTAS_GEMM_PACKED (the APSP entry points have their own
                                       switches) */
#define BTAS_GEMM_PACKED 0x800     /* int32: exact packed 16-bit path when the operand ranges allow */
#define BTAS_GEMM_CHECKED 0x1000   /* int32/fp32: check the operand domain on the device (btas_sync_status) */

typedef enum {
    BTAS_I32 = 0, /* int32, encoding above */
    BTAS_F32 = 1, /* IEEE binary32 */
    BTAS_U16 = 2  /* uint16 min-plus values in [0, 0x7FFF], packed two per 32-bit lane */
} btas_dtype;

typedef enum {
    BTAS_OK = 0,
    BTAS_ERR_ARG = 1,         /* invalid argument; nothing enqueued */
    BTAS_ERR_BOUND = 2,       /* a requested exact reduced-precision path is not provably exact */
    BTAS_ERR_NOMEM = 3,       /* device workspace allocation failed */
    BTAS_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    BTAS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (batched/server scheduler,
                                 grid barriers of the cooperative APSP and SSSP kernels) */
    BTAS_ERR_BUDGET = 6,      /* request exceeds the configured device-memory budget */
    BTAS_ERR_UNSUPPORTED = 7  /* semiring/dtype combination not offered */
} btas_status;

/* Workspace pool.  Temporary device memory comes from a stream-ordered
 * memory pool the library creates for each device (cudaMemPoolCreate).
 * Freed blocks stay cached for later calls up to a release threshold, set
 * by the environment variable BTAS_POOL_KEEP_MB when the pool is created
 * (default 4096 MiB).  Without the cache, blocks would go back to the
 * driver at every synchronisation and each small call would pay for a
 * fresh mapping.
 * btas_workspace_reserved: bytes the current device's pool holds now.
 * btas_workspace_trim    : synchronises the device and releases every
 *                          cached block of its pool. */
int64_t btas_workspace_reserved(void);
btas_status btas_workspace_trim(void);

/* Library version as 10000*major + 100*minor + patch. */
int btas_version(void);

/* Human-readable description of the calling thread's most recent error. */
const char *btas_last_error_string(void);

/* Number of CUDA kernels this library has enqueued in this process so far
 * (all threads, all devices).  Diagnostic counter; never reset. */
int64_t btas_kernel_launches(void);

/* Diagnostic: measured issue ceiling of the current device for one inner-loop
 * instruction mix, in tropical terms (one (i,j,k) add-then-min) per clock per
 * SM, from a register-only kernel with one CTA per SM (synchronises the
 * device).  mix: 0 = int32 DPX fused add-min, 1 = fp32 add.f32x2 + 3-input
 * min, 2 = packed u16x2 DPX add-min, 3 = FFMA (multiply-adds, reference),
 * 4 = int32 IADD + 3-input min, 5 = int32 IMAD (x*1+y) + 3-input min,
 * 6 = int32 column split (mix 5 on 5 of 8 columns, DPX on 3),
 * 7 = fp32 two scalar adds + 3-input min. */
btas_status btas_measure_issue_rate(int mix, double *terms_per_clock_per_sm);

/* Diagnostic: the same probe with ctas_per_sm (1 or 2) CTAs of 256 threads
 * per SM, and the diagnostic mixes that separate pipe throughput from
 * register-operand reads:
 *   8  = FFMA x2 with the multiplier an immediate (two register operands),
 *   9  = fp32 two adds of an immediate + 3-input min,
 *   10 = int32 two IADD of an immediate + 3-input min,
 *   11 = int32 DPX add-min with an immediate addend,
 *   12 = int32 three-pipe split (DPX on 3 of 8 columns, IMAD + 3-input min
 *        on 3, FADD + 3-input min on 2),
 *   13 = DPX on 3 of 8 columns, add.f32x2 + 3-input min on 5,
 *   14 = int32 two IMAD of an immediate addend + 3-input min,
 *   15 = mix 0 with a different A register in every consecutive
 *        instruction (the other mixes keep a row's A across 8 of them).
 * The rate of an SM is taken from its first CTA's start to its last CTA's
 * end; the slowest SM is reported.  Errors: BTAS_ERR_ARG for a mix outside
 * 0..15 or ctas_per_sm outside {1, 2}. */
btas_status btas_measure_issue_rate_ex(int mix, int ctas_per_sm, double *terms_per_clock_per_sm);

/* ------------------------------------------------------------------------
 * Level 3: tropical matrix product (the product listing of Sec. IV, titled
 * "Matrix-Matrix Multiplication for Floyd-Warshall": replace + by min (or
 * max) and x by +).
 *
 *   C[i][j] = (+)_{0<=l<k} A[i][l] (.) B[l][j]           (default)
 *   C[i][j] = C[i][j] (+) (+)_l A[i][l] (.) B[l][j]      (BTAS_GEMM_ACCUMULATE)
 *
 * semiring : BTAS_MINPLUS or BTAS_MAXPLUS, optionally OR BTAS_GEMM_* flags.
 * dtype    : BTAS_I32, BTAS_F32, or BTAS_U16 (min-plus only).
 * m, n, k  : sizes, each >= 0.  k == 0 writes the (+)-identity (or leaves C
 *            unchanged with ACCUMULATE).  m == 0 or n == 0 is a no-op.
 * A        : m x k, leading dimension lda >= max(1, k).
 * B        : k x n with ldb >= max(1, n); with BTAS_GEMM_TRANS_B it is the
 *            n x k matrix B^T with ldb >= max(1, k).
 * C        : m x n, ldc >= max(1, n).  C must not overlap A or B.
 * Errors   : BTAS_ERR_ARG for negative sizes, short leading dimensions,
 *            NULL pointers with non-empty extents, unknown semiring/dtype;
 *            BTAS_ERR_UNSUPPORTED for max-plus with BTAS_U16.
 * Results are bit-exact with the definition for every tiling.
 *
 * BTAS_GEMM_PACKED (int32 only; ignored for other dtypes): both semirings
 * commute with a shift of each operand (min-plus: subtract the operand's
 * smallest finite entry; max-plus: subtract each entry from the largest),
 * after which every finite operand of A lies in [0, R_A] and of B in
 * [0, R_B].  When every entry of A and B is finite (|v| <= 2^28) or the
 * (+)-identity, and R_A + R_B < 0x7FFF, the product is computed exactly on
 * the packed u16x2 kernel (two terms per instruction) and shifted back;
 * otherwise on the int32 kernel.  The ranges are scanned and the choice is
 * made on the device: the call stays asynchronous, the results are
 * bit-identical either way, and it costs a few passes over A, B and C plus
 * device workspace of about 4mk + 2kn + 2mn bytes.
 *
 * BTAS_GEMM_CHECKED (BTAS_I32 and BTAS_F32; BTAS_ERR_UNSUPPORTED with
 * BTAS_U16): without it, operands outside the domain above are not detected
 * (an int32 entry beyond 2^28 that is not the (+)-identity can be clamped to
 * INF without notice).  With it, the call scans A, B (and C with
 * BTAS_GEMM_ACCUMULATE) on the device before the product: int32 entries must
 * satisfy |v| <= 2^28 or equal the semiring's (+)-identity; fp32 entries must
 * not be NaN or the other semiring's infinity.  A call that finds any entry
 * outside leaves C unwritten and adds the count to the device's status
 * words; the call itself stays asynchronous and returns BTAS_OK.
 * btas_sync_status reports (and clears) the words.  Cost: one extra read of
 * the operands (HBM-bound).  The first checked product (or btas_sync_status
 * call) on a device allocates its 256-byte status words with cudaMalloc:
 * make it outside stream capture.
 * ------------------------------------------------------------------------ */
btas_status btas_gemm(int semiring, int dtype, int64_t m, int64_t n, int64_t k,
                      const void *A, int64_t lda, const void *B, int64_t ldb,
                      void *C, int64_t ldc, void *stream);

/* Device-side errors of asynchronous calls.  Reads the current device's
 * status words after the work enqueued on `stream` (synchronises `stream`)
 * and clears them.  The words accumulate, across calls and streams, the
 * operand entries outside the domain that BTAS_GEMM_CHECKED products found;
 * synchronise other streams that ran checked products first.
 * out_of_domain, calls: HOST pointers or NULL; entries found and checked
 * calls that found any (each of those left its C unwritten).
 * Returns BTAS_ERR_ARG if any entry was found, else BTAS_OK (BTAS_ERR_CUDA on
 * a CUDA failure).  Calls that synchronise on their own report device-side
 * errors themselves (btas_apsp, btas_sssp and the other APSP entry points
 * return BTAS_ERR_ARG for a weight outside the domain and BTAS_ERR_TIMEOUT
 * when a bounded grid-barrier wait expires; btas_batch_wait and the server
 * report theirs); btas_apsp_noalloc has btas_apsp_noalloc_status. */
btas_status btas_sync_status(void *stream, int64_t *out_of_domain, int64_t *calls);

/* Diagnostic: number of products the current device has computed through
 * the packed path of BTAS_GEMM_PACKED since the library was loaded
 * (synchronises the device; -1 on a CUDA error). */
int64_t btas_packed_products(void);

/* ------------------------------------------------------------------------
 * Level 2: tropical matrix-vector product (the "standard vector and matrix
 * operations" of the abstract / Sec. III between levels 1 and 3).
 *   trans == 0: y[i] = (+)_j A[i][j] (.) x[j]    x: n, y: m
 *   trans == 1: y[j] = (+)_i x[i] (.) A[i][j]    x: m, y: n  (y = x^T A)
 * semiring may carry BTAS_GEMM_ACCUMULATE (y (+)= ...).  A: m x n device,
 * row-major, lda >= max(1, n); x, y contiguous device vectors.  dtype
 * BTAS_I32 or BTAS_F32.  An empty reduction writes the (+)-identity.
 * HBM-bound: A is streamed once.  Results are exact (order-independent).
 * ------------------------------------------------------------------------ */
btas_status btas_gemv(int semiring, int dtype, int trans, int64_t m, int64_t n, const void *A, int64_t lda,
                      const void *x, void *y, void *stream);

/* btas_sssp: single-source shortest paths from `src` by repeated min-plus
 * vector-matrix products d_{t+1} = d_t (x) W (Bellman-Ford; W[j][j] = 0
 * keeps d_t[j]) until d stops changing, at most n-1 products.  W: n x n int32
 * device matrix (domain as btas_apsp, checked); dist: n int32 device vector
 * (INF = unreachable) = row `src` of btas_apsp's result; not written if the
 * domain check fails (BTAS_ERR_ARG).  iterations: HOST pointer or NULL,
 * receives the number of products that changed d.  All products run in one
 * cooperative launch with one bounded grid barrier each (BTAS_ERR_TIMEOUT if
 * a wait expires; the first product also checks the domain), and the call
 * synchronises `stream` once.  Where a cooperative launch is refused (or
 * with BTAS_SSSP_NO_COOP=1 in the environment) it launches the products in
 * gated groups of 8 and synchronises once per group. */
btas_status btas_sssp(int64_t n, const int32_t *W, int64_t src, int32_t *dist, int *iterations, void *stream);

/* ------------------------------------------------------------------------
 * Level 1: tropical vector operations ("standard vector operations",
 * abstract and Sec. III).  Strides may be negative only where stated; here
 * they must be >= 1.
 *
 * btas_dot : *result = (+)_{i<n} x[i*incx] (.) y[i*incy].  `result` is a
 *            DEVICE pointer to one element of `dtype`.  n == 0 writes the
 *            (+)-identity.
 * btas_axpy: y[i*incy] <- y[i*incy] (+) (alpha (.) x[i*incx]).  `alpha` is a
 *            HOST pointer to one element of `dtype`.
 * btas_add : z[i] = x[i] (+) y[i]   (contiguous vectors of length n)
 * btas_mul : z[i] = x[i] (.) y[i]   (int32 result saturates to INF as above)
 * dtype    : BTAS_I32 or BTAS_F32.
 * ------------------------------------------------------------------------ */
btas_status btas_dot(int semiring, int dtype, int64_t n, const void *x, int64_t incx,
                     const void *y, int64_t incy, void *result, void *stream);
btas_status btas_axpy(int semiring, int dtype, int64_t n, const void *alpha,
                      const void *x, int64_t incx, void *y, int64_t incy, void *stream);
btas_status btas_add(int semiring, int dtype, int64_t n, const void *x, const void *y,
                     void *z, void *stream);
btas_status btas_mul(int semiring, int dtype, int64_t n, const void *x, const void *y,
                     void *z, void *stream);

/* ------------------------------------------------------------------------
 * All-pairs shortest paths by repeated squaring (Sec. III): D_0 = W,
 * D_{s+1} = D_s (x) D_s in min-plus, for S = ceil(log2(n-1)) squarings
 * (S = 0 for n <= 2).  After s squarings D_s holds the shortest walks of at
 * most 2^s edges; a shortest path has at most n-1 edges, so D_S is the APSP
 * distance matrix -- the same matrix Floyd-Warshall (Algorithm 2) computes.
 *
 * n : number of vertices, >= 0.
 * W : n x n int32 weighted adjacency matrix (row-major, leading dimension n):
 *     W[i][i] == 0, W[i][j] in [0, BTAS_I32_FINITE_MAX] for an edge,
 *     BTAS_INF_I32 for no edge.  Weights are non-negative (Sec. IV states
 *     the algorithm for non-negative edge weights).
 * D : n x n int32 output; D == W (in place) is allowed, any other overlap is
 *     not.
 * btas_apsp checks the domain on the device (one synchronisation of
 * `stream`; BTAS_ERR_ARG if violated), enables the early exit, and picks the
 * exact representation per squaring as btas_apsp_ex does without FORCE
 * flags.
 *
 * Execution by size (same results and the same squarings count in every
 * regime; FORCE_U16 / FORCE_CARRIER always take the tiled path):
 *   n <= 64         one thread block holds D in shared memory and runs the
 *                   domain check and every squaring (int32): one launch, one
 *                   read-back;
 *   64 < n <= 1792  one cooperative launch runs every squaring as split-k
 *                   pieces merged with atomicMin, one grid barrier (bounded
 *                   wait; BTAS_ERR_TIMEOUT if it expires) per squaring; each
 *                   squaring packed 16-bit while every finite entry of its
 *                   operand is <= 16383 (a bound the previous squaring
 *                   reports), else int32 (always int32 with FORCE_I32); from
 *                   n = 1408 with 128 x 128 tiles and warp-specialised
 *                   staging.  From n = 384 the launch also builds edge lists
 *                   of W: when every row has at most min(256, max(32, n / 4))
 *                   edges (rounded to 32) the first squaring runs as sparse
 *                   products over them, and after a squaring that lowered
 *                   few entries a closure certificate (X (x) W >= X, checked
 *                   at the lowered entries) can stop the solve without the
 *                   squaring that would only confirm the fixpoint (early exit
 *                   only); D and the squarings count are the same;
 *   1792 < n <= 4096  the same launch for graphs whose rows fit the edge
 *                   lists; it declines any other graph after the domain check
 *                   (D untouched), which then takes the tiled kernels;
 *   larger n        the tiled product kernels, one launch per squaring, with
 *                   the per-squaring exact representation described below.
 * BTAS_APSP_SMALL_MAX_N=m (0 .. 128) and BTAS_APSP_MID_MAX_N=m (0 .. 4096) in
 * the environment move the two boundaries (the latter as a plain size
 * limit); BTAS_APSP_NO_SMALL=1 / BTAS_APSP_NO_MID=1 send the first two
 * regimes to the tiled path.  The cooperative regime keeps, per calling host
 * thread, 64 bytes of mapped host memory for its status words and (for
 * workspaces up to 32 MiB, on the first device the thread uses) a 32 MiB
 * device workspace, both released when the thread exits; other workspace
 * comes from the pool of btas_workspace_*.
 * ------------------------------------------------------------------------ */
btas_status btas_apsp(int64_t n, const int32_t *W, int32_t *D, void *stream);

/* Flags for btas_apsp_ex. */
#define BTAS_APSP_EARLY_EXIT 0x1   /* stop squaring once D_{s+1} == D_s (result unchanged) */
#define BTAS_APSP_FORCE_I32 0x2    /* always run the plain int32 kernels */
#define BTAS_APSP_FORCE_U16 0x4    /* require the packed 16-bit path; BTAS_ERR_BOUND if not exact */
#define BTAS_APSP_FORCE_CARRIER 0x8 /* require the FP32-carrier path; BTAS_ERR_BOUND if not exact */

/* btas_apsp_ex: as btas_apsp, with
 *  flags           : BTAS_APSP_* bits.
 *                    Without FORCE bits the representation is chosen per
 *                    squaring from m = the largest finite entry of D_s (every
 *                    finite entry of D_{s+1} and every pairwise sum is <= 2m):
 *                    packed 16-bit if 2m < 0x7FFF, exact FP32 carrier if
 *                    2m < 2^24, else int32.  Each squaring's epilogue reports
 *                    the next m, so this mode synchronises `stream` once per
 *                    squaring.  FORCE_U16 / FORCE_CARRIER pin one
 *                    representation and require the static bound
 *                    B = (n-1) * max w to be below 0x7FFF / 2^23
 *                    (BTAS_ERR_BOUND otherwise).  FORCE_I32 with
 *                    bound == NULL runs int32 squarings without any host
 *                    synchronisation (the early exit is then decided on the
 *                    device: a converged squaring copies its input through).
 *  squarings_done  : HOST pointer or NULL; receives the number of squarings
 *                    that changed D (<= S).
 *  bound           : HOST pointer or NULL; receives B (or -1 if W has a
 *                    negative or out-of-domain entry, in which case the call
 *                    returns BTAS_ERR_ARG after synchronising).
 *  path            : HOST pointer or NULL; receives the set of
 *                    representations used, as bits: 1 = int32, 2 = FP32
 *                    carrier, 4 = packed 16-bit, 8 = the first squaring as
 *                    sparse products over edge lists (cooperative regime).
 * The domain scan (zero diagonal, weights in [0, 2^28] or INF) runs on the
 * device and synchronises `stream` once, except in the FORCE_I32 mode above.
 */
btas_status btas_apsp_ex(int64_t n, const int32_t *W, int32_t *D, int flags,
                         int *squarings_done, int64_t *bound, int *path, void *stream);

/* btas_apsp_u16: APSP on 16-bit storage (BTAS_U16 encoding, INF = 0x7FFF).
 * W and D are n x n uint16 device matrices, D == W allowed.  The caller
 * asserts max_w, the largest finite weight; the call returns BTAS_ERR_BOUND
 * unless (n-1) * max_w < 0x7FFF, which makes every intermediate distance
 * exact.  flags: BTAS_APSP_EARLY_EXIT or 0. */
btas_status btas_apsp_u16(int64_t n, const uint16_t *W, uint16_t *D, int max_w, int flags,
                          void *stream);

/* btas_closure: tropical closure (Kleene star) A* = E (+) A (+) A^2 (+) ...,
 * the shortest (min-plus) or longest (max-plus) walk weights of the matrix
 * graph A, computed as (E (+) A) squared until it stops changing (at most
 * ceil(log2(n-1)) squarings suffice when A* exists, Sec. III), E being the
 * tropical identity (0 on the diagonal).  Unlike btas_apsp, entries may be
 * negative (min-plus) or positive (max-plus) and the diagonal is arbitrary;
 * with non-negative weights and dtype BTAS_F32 this is FP32 APSP, bit-exact
 * with the same squaring sequence (fp32 results are those of repeated
 * squaring, not of Floyd-Warshall's evaluation order).
 * semiring/dtype: BTAS_MINPLUS or BTAS_MAXPLUS; BTAS_I32 or BTAS_F32.
 * A, Astar     : n x n device matrices, leading dimension n; may alias.
 * flags        : BTAS_APSP_EARLY_EXIT or 0 (the result is the same).
 * squarings_done: HOST pointer or NULL: squarings that changed the matrix.
 * The result is D_S, S = ceil(log2(n-1)) squarings of E (+) A (the loop
 * stops early at a fixpoint, which does not change it).  The call
 * synchronises `stream` once per squaring.  If all S squarings changed the
 * matrix, one more squaring is checked: a negative (min-plus) or positive
 * (max-plus) diagonal entry there proves a cycle of that sign, A* does not
 * exist, and the call returns BTAS_ERR_ARG.  int32: finite entries and
 * every walk weight must stay in [-2^28, 2^28]. */
btas_status btas_closure(int semiring, int dtype, int64_t n, const void *A, void *Astar, int flags,
                         int *squarings_done, void *stream);

/* btas_apsp_paths: APSP by repeated squaring (Sec. III) with path
 * reconstruction.  D receives the distances (as btas_apsp) and Next the
 * next-hop matrix: Next[i][j] = the vertex after i on a shortest path from i
 * to j, Next[i][i] = i, -1 if j is unreachable.  Ties are broken by one fixed
 * rule, so Next is reproducible: each squaring
 * D'[i][j] = min_k D[i][k] + D[k][j] takes the SMALLEST minimising k = k*,
 * and Next'[i][j] = Next[i][j] if k* == i, else Next[i][k*].  With positive
 * weights, following Next from i reaches j with total weight D[i][j].
 * W, D, Next: n x n int32 device matrices, leading dimension n (W must not
 * overlap D or Next).  Domain as btas_apsp (checked: BTAS_ERR_ARG).
 * flags: BTAS_APSP_EARLY_EXIT stops once a squaring changes neither D nor
 * Next (same result).  squarings_done: HOST pointer or NULL.  The call
 * synchronises `stream` once per squaring.  int32 only: while every
 * distance is <= 49151 and n <= 8192 a squaring is one int32 min-plus
 * product of the keys (D << 13) | k (minimum key = minimum distance with
 * the smallest k), else an argmin kernel; BTAS_PATHS_NO_KEYED=1 forces the
 * latter. */
btas_status btas_apsp_paths(int64_t n, const int32_t *W, int32_t *D, int32_t *Next, int flags, int *squarings_done,
                            void *stream);

/* btas_apsp_paths_f32: the same squaring with successors on binary32 weights
 * (the squaring APSP of Sec. III on real weights).  Each term is one
 * round-to-nearest-even add, and the SMALLEST k whose rounded sum attains the
 * minimum is kept, so D and Next are reproducible bit for bit; a tie that
 * only the rounding creates is broken like any other.  D equals
 * ceil(log2(n-1)) repeated fp32 min-plus squarings of W (stopped early, same
 * result, with BTAS_APSP_EARLY_EXIT).  Because of rounding, the weight of
 * the walk Next describes may differ from D[i][j] in the last bits.
 * W, D: n x n float device matrices, leading dimension n; Next: n x n int32
 * as in btas_apsp_paths (W must not overlap D or Next).  Domain (checked,
 * BTAS_ERR_ARG): zero diagonal, every other entry >= 0 or +inf (no edge);
 * no NaN, no -inf.  flags, squarings_done and synchronisation as
 * btas_apsp_paths; every squaring runs on the argmin kernel. */
btas_status btas_apsp_paths_f32(int64_t n, const float *W, float *D, int32_t *Next, int flags, int *squarings_done,
                                void *stream);

/* btas_apsp_fw: the same APSP distance matrix by blocked Floyd-Warshall --
 * Algorithm 2's pivot loop reorganised in 128 x 128 tiles: per pivot block,
 * the diagonal tile and its row and column panels relax in order, and every
 * other tile is updated by a tropical product with accumulate over the
 * block's pivots (the semiring GEMM kernel).  n^3 terms instead of
 * ceil(log2(n-1)) * n^3; int32 results identical to btas_apsp.  W, D as
 * btas_apsp (D == W allowed, any other overlap not); domain checked
 * (synchronises `stream` once).  With three or more pivot blocks, phases
 * 1-2 of the next block run on an internal stream of higher priority,
 * forked from and joined back to `stream` with events, so the call's work
 * is still ordered after earlier work on `stream` and before later work
 * (stream capture included); BTAS_FW_NO_LOOKAHEAD=1 keeps everything on
 * `stream`. */
btas_status btas_apsp_fw(int64_t n, const int32_t *W, int32_t *D, void *stream);

/* Number of squarings btas_apsp performs for n vertices: ceil(log2(n-1)). */
int btas_apsp_squarings(int64_t n);

/* ------------------------------------------------------------------------
 * btas_apsp_noalloc: the same APSP as btas_apsp (int32 or exact packed
 * 16-bit squarings as btas_apsp chooses them, early exit),
 * for callers that cannot allocate device memory when they call -- e.g. a
 * process whose own memory pool already holds the device's free memory, or
 * latency-critical code that must not allocate (an allocation can block or
 * synchronise) inside its loop.  The paper has no counterpart: it is an
 * interface addition of this library.
 *
 * It allocates nothing.  Its scratch is one fixed array of
 * BTAS_NOALLOC_SCRATCH_BYTES in device global memory that every GPU loading
 * this library holds until the process exits; hence n <= BTAS_NOALLOC_MAX_N
 * (larger n returns BTAS_ERR_ARG, nothing enqueued).  The caller still passes
 * W and D (device pointers, n x n int32, row-major, D == W allowed).
 * The smallest n run on the one-block kernel and the others on the
 * cooperative kernel, as in btas_apsp (the same size boundary); only if a
 * cooperative launch is not possible on the device do they take the tiled
 * int32 squarings.  Nothing is read back: the call does not synchronise
 * `stream`.
 * Every call looks up the array's device address in the current context
 * (a host-side lookup that does not synchronise), so it stays valid after a
 * context is torn down and recreated.  The first call on a device may load
 * the library's device code there: make it before any stream capture.  All
 * calls share the array and it keeps the last call's contents; the status
 * words are cleared on `stream` at the start of each call.  Calls whose work
 * overlaps on the GPU race on the array: order them (one stream, or events).
 * The one-block and cooperative kernels check the weight domain (zero
 * diagonal, weights in [0, 2^28] or BTAS_INF_I32) and leave D unwritten when
 * it fails, and so does the cooperative kernel when a bounded grid-barrier
 * wait expires; the call itself cannot see either (it reads nothing back):
 * btas_apsp_noalloc_status reports them.  The tiled fallback assumes the
 * domain.
 * ------------------------------------------------------------------------ */
#define BTAS_NOALLOC_MAX_N 1024
#define BTAS_NOALLOC_SCRATCH_BYTES \
    (256 + 3 * 4 * BTAS_NOALLOC_MAX_N * BTAS_NOALLOC_MAX_N + 2048 + 4 * BTAS_NOALLOC_MAX_N + 8 * 256 * BTAS_NOALLOC_MAX_N)
btas_status btas_apsp_noalloc(int64_t n, const int32_t *W, int32_t *D, void *stream);

/* Outcome of the most recent btas_apsp_noalloc call on the current device,
 * read from the status words that call left in the fixed array.  The read is
 * enqueued on `stream` (so it follows that call's work when both use the same
 * stream) and the stream is synchronised; it copies into host memory of the
 * call's own and allocates nothing.  Returns BTAS_OK (D holds the result),
 * BTAS_ERR_ARG (W outside the weight domain, D not written; also when no call
 * has been made on this device), BTAS_ERR_TIMEOUT (a grid-barrier wait of the
 * cooperative kernel expired, D not written) or BTAS_ERR_CUDA.
 * squarings_done: HOST pointer or NULL; squarings that changed D.  Another
 * btas_apsp_noalloc call enqueued in between overwrites the words. */
btas_status btas_apsp_noalloc_status(void *stream, int *squarings_done);

/* ------------------------------------------------------------------------
 * Autotuner for the tropical product kernels (the product of Eq. 1-4, and
 * the squarings of the Sec. III APSP that call it).  The paper fixes one
 * GPU kernel shape; this library has several compiled tile shapes and
 * inner-loop variants, all with identical results, and picks among them by
 * measurement on the device at hand.
 *
 * Key: (compute capability, SM count, semiring, dtype, size buckets of m, n
 * and k), where the bucket of x is ceil(log2(x)).  Value: the fastest kernel
 * (inner-loop variant, IMAD-path column count ns, tile configuration) and
 * the tile raster group (a schedule parameter).
 *
 * Kernel choice in btas_gemm, btas_apsp/_ex, btas_closure, btas_apsp_paths
 * and btas_apsp_fw, in this order: explicit environment overrides
 * (BTAS_CFG, BTAS_I32_VARIANT, BTAS_I32_NS, BTAS_F32_VARIANT, BTAS_U16_NS);
 * then a table entry for the key; then, if the environment sets BTAS_TUNE=1
 * and the stream is not being captured, a tuning run on the spot (it
 * synchronises the stream once and allocates scratch); then the built-in
 * defaults.  BTAS_TUNE_CACHE=<path> loads that file into the table on first
 * use, and an on-the-spot tuning run appends the table back to it.
 * btas_apsp_noalloc and the batched/server paths do not consult the table.
 *
 * btas_tune_gemm : times every compiled candidate for (semiring, dtype) at
 *                  m x n x k on `stream` (device scratch operands with
 *                  seeded values in the dtype's domain, INF entries
 *                  included; the caller's memory is not touched), checks
 *                  that every candidate's result equals the first one's bit
 *                  for bit (BTAS_ERR_INTERNAL otherwise), then times the
 *                  winner's raster groups, stores the best in the table and
 *                  fills *out (may be NULL).  Synchronises `stream`; takes
 *                  about 20 ms per candidate plus four products each.
 *                  semiring: BTAS_MINPLUS/BTAS_MAXPLUS; dtype: BTAS_I32,
 *                  BTAS_F32, or BTAS_U16 (min-plus only).  m, n, k >= 1.
 * btas_tune_lookup: 1 and *out filled if the table has an entry for the
 *                  key of the current device, else 0.
 * btas_tune_save : writes the whole table (every device's entries) to
 *                  `path`, one JSON object per line.
 * btas_tune_load : reads such a file and adds its entries (replacing equal
 *                  keys).  A malformed line, or a kernel this build does
 *                  not have, returns BTAS_ERR_ARG and adds nothing.
 *                  *loaded (may be NULL) receives the number of entries.
 * btas_tune_clear / btas_tune_entries: empty / count the table.
 * Thread safety: the table is guarded by a lock; tuning itself runs
 * unlocked, so two threads tuning the same key both measure and the later
 * store wins.
 * ------------------------------------------------------------------------ */
#define BTAS_ERR_INTERNAL 8 /* a self-check failed (tuning candidates disagree) */

typedef struct {
    int variant;             /* inner loop: 0 int32 DPX, 1 int32 IMAD/3-input-min mix,
                                2 fp32 add.f32x2, 3 fp32 scalar, 4 fp32 two adds + 3-input min,
                                16 packed u16x2 */
    int ns;                  /* columns (of 8) on the IMAD path; 0 if not applicable */
    int cfg;                 /* tile configuration id (u16: 0) */
    int tile_m, tile_n;      /* CTA output tile */
    int group_m;             /* tile-raster group height */
    int candidates;          /* kernels timed */
    double seconds;          /* best time of one product */
    double terms_per_second; /* m*n*k / seconds */
} btas_tune_result;

btas_status btas_tune_gemm(int semiring, int dtype, int64_t m, int64_t n, int64_t k, btas_tune_result *out,
                           void *stream);
int btas_tune_lookup(int semiring, int dtype, int64_t m, int64_t n, int64_t k, btas_tune_result *out);
btas_status btas_tune_save(const char *path);
btas_status btas_tune_load(const char *path, int *loaded);
void btas_tune_clear(void);
int btas_tune_entries(void);

/* ------------------------------------------------------------------------
 * Batched execution: many independent tropical products and APSP solves of
 * uneven sizes in ONE persistent kernel launch (captured once in a CUDA
 * graph and replayed).  Same arithmetic and bit-identical results as the
 * single calls; the batch only changes scheduling: output tile tasks
 * (128 x 128, or 64 x 64 for instances the tile autotuner gives the small
 * tile) are ordered by level (transposes, then squaring 1, 2, ...) and,
 * within a level, largest instance first; persistent CTAs claim tasks from a
 * global counter and wait (bounded) for the previous level of their own
 * instance.
 *
 * btas_batch_create  : *out receives a new empty batch.  flags:
 *                      BTAS_BATCH_NO_GRAPH launches the kernel directly
 *                      instead of replaying a captured graph.
 * btas_batch_add_apsp: APSP by repeated squaring of W into D (device, n x n
 *                      int32, leading dimension n), as btas_apsp with int32
 *                      kernels and the early exit.  D must not overlap W.
 *                      The domain (zero diagonal, weights in [0, 2^28] or
 *                      INF) is assumed, not checked.
 * btas_batch_add_gemm: C = A (x) B as btas_gemm (int32 or fp32, min-plus or
 *                      max-plus, optional BTAS_GEMM_TRANS_B; m, n, k >= 1).
 * btas_batch_launch  : enqueues the whole batch on `stream`.  The first
 *                      launch after an add builds the plan: it allocates the
 *                      device workspace (cudaMalloc; not stream-ordered) and
 *                      captures the graph, so it must not itself be inside a
 *                      stream capture.  Later launches replay the graph.
 *                      The caller's buffers must stay valid until the work
 *                      completes.
 * btas_batch_wait    : synchronises `stream` and returns the device status
 *                      word: BTAS_ERR_TIMEOUT if a bounded wait expired
 *                      (every CTA then stops; results are incomplete).
 * btas_batch_destroy : frees the plan and the batch (call after the work has
 *                      completed).
 * btas_batch_workspace_bytes / btas_batch_tasks: plan size diagnostics.
 * btas_batch_profile : tracing.  With BTAS_BATCH_PROFILE at create, every
 *                      CTA adds, per task, the SM clock cycles its first
 *                      thread spent on the task to a per-kind slot
 *                      (BTAS_BATCH_SLOT_*), and the cycles it spent in the
 *                      dependency wait to BTAS_BATCH_SLOT_WAIT.  Sums run
 *                      over all launches since the plan was built.  Fills
 *                      cycles[i] and counts[i] for i < min(slots,
 *                      BTAS_BATCH_PROFILE_SLOTS) after synchronising the
 *                      device; BTAS_ERR_ARG if the batch was created without
 *                      the flag or has not been launched.
 * ------------------------------------------------------------------------ */
typedef struct btas_batch_t btas_batch_t;
#define BTAS_BATCH_NO_GRAPH 0x1
#define BTAS_BATCH_PROFILE 0x2
#define BTAS_BATCH_PROFILE_SLOTS 12
#define BTAS_BATCH_SLOT_TRANSPOSE 0   /* level-0 transposes (and 16-bit forms) */
#define BTAS_BATCH_SLOT_COPY 1        /* n <= 2 APSP: D = W */
#define BTAS_BATCH_SLOT_APSP_U16 2    /* APSP squaring tile, packed u16x2 */
#define BTAS_BATCH_SLOT_APSP_I32 3    /* APSP squaring tile, int32 */
#define BTAS_BATCH_SLOT_APSP_DONE 4   /* APSP squaring tile after convergence (copy through) */
#define BTAS_BATCH_SLOT_GEMM_I32 5    /* product tile, int32 */
#define BTAS_BATCH_SLOT_GEMM_F32 6    /* product tile, fp32 */
#define BTAS_BATCH_SLOT_SQUARE_U16 7  /* server single-squaring tile, u16x2 */
#define BTAS_BATCH_SLOT_SQUARE_I32 8  /* server single-squaring tile, int32 */
#define BTAS_BATCH_SLOT_WAIT 9        /* waiting for the previous level */
#define BTAS_BATCH_SLOT_LISTS 10      /* APSP edge lists of W (level 0) */
#define BTAS_BATCH_SLOT_CERT 11       /* APSP closure certificate after a squaring */
btas_status btas_batch_create(btas_batch_t **out, int flags);
btas_status btas_batch_add_apsp(btas_batch_t *b, int64_t n, const int32_t *W, int32_t *D);
btas_status btas_batch_add_gemm(btas_batch_t *b, int semiring, int dtype, int64_t m, int64_t n, int64_t k,
                                const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc);
btas_status btas_batch_launch(btas_batch_t *b, void *stream);
btas_status btas_batch_wait(btas_batch_t *b, void *stream);
btas_status btas_batch_destroy(btas_batch_t *b);
int64_t btas_batch_workspace_bytes(btas_batch_t *b);
int btas_batch_tasks(btas_batch_t *b);
btas_status btas_batch_profile(btas_batch_t *b, uint64_t *cycles, uint64_t *counts, int slots);

/* Autotuner of the batched launch's output tile shape (the "tile shapes ...
 * picked by an autotuner" of the batched form).  For each instance kind
 * (0: APSP, 1: int32 min-plus product, 2: fp32 max-plus product) and each
 * size bucket of 32 up to n_max (1 .. 2048), it times one synthetic batch of
 * that bucket (three sizes, enough instances for about 1.5e10 terms; best of
 * 3 graph-captured launches after a warm-up) with the 128 x 128 tile and with
 * the 64 x 64 tile (4 x 4 outputs per thread) and records the 64 x 64 tile
 * where it is at least 3 % faster.  Plans built afterwards on the current
 * device use the table (an instance takes the entry of its larger output
 * side); BTAS_BATCH_TILE=64|128 in the environment overrides it.  Both tiles
 * compute bit-identical results.  Synchronises `stream`; allocates its
 * inputs with cudaMalloc (call it outside stream capture).  ms_out: HOST
 * array or NULL; entry 2*(kind*B + b) (+1) receives the 128 (64) tile's time
 * in ms of bucket b of kind, B = ceil(n_max / 32), for entries < max_entries.
 * btas_batch_tile: the table's tile for (kind, n) on the current device,
 * 128 or 64, or 0 if it has no entry.  btas_batch_tune_clear empties it. */
btas_status btas_batch_tune(int64_t n_max, void *stream, double *ms_out, int max_entries);
int btas_batch_tile(int kind, int64_t n);
void btas_batch_tune_clear(void);

/* Tile choice tuned on one batch itself: times the batch (best of 3
 * launches after a warm-up, on `stream`, synchronising) planned three ways
 * -- mode 0: each instance's tile from the table above (and
 * BTAS_BATCH_TILE); mode 1: 128 x 128 for every instance; mode 2: 64 x 64
 * for every instance -- and keeps the fastest for the batch's later
 * launches.  Results are bit-identical in every mode.  The batch's buffers
 * are read and written by the timing launches.  mode: HOST, receives the
 * choice; ms_out: HOST array of 3 or NULL, the three times in ms. */
btas_status btas_batch_select_tiles(btas_batch_t *b, void *stream, int *mode, double *ms_out);

/* ------------------------------------------------------------------------
 * Continuous-batching server: requests with HOST buffers (contiguous
 * row-major; pinned memory gives asynchronous copies) are admitted in
 * arrival order while the device-memory footprint of admitted requests stays
 * within `hbm_budget_bytes`.  An executor thread runs steps: each step runs
 * the next unit of every admitted request (a whole product, or one APSP
 * squaring) in one persistent launch; requests arriving meanwhile join the
 * next step.  A product completes after its step; an APSP solve after its
 * last squaring or as soon as a squaring changed nothing.  An APSP request
 * with n <= 1792 is instead solved whole in one unit, by the one-block or
 * the cooperative kernel of btas_apsp (the same size boundary), launched in the step
 * after the persistent kernel (BTAS_SERVER_NO_WHOLE=1 in the environment at
 * creation turns this off).  Results are bit-identical to btas_gemm /
 * btas_apsp.  Buffers must stay valid until the request is done.
 *
 * btas_server_create      : budget in bytes (> 0); flags must be 0.  The
 *                           current device is the server's device.
 * btas_server_submit_apsp : n x n int32 W (host) -> D (host); *ticket
 *                           receives the request id.  The domain (zero
 *                           diagonal, weights in [0, 2^28] or INF) is
 *                           checked on the device in the request's first
 *                           step (whole solve or first squaring); a
 *                           violation ends the request in state 3, failed,
 *                           with D not written.  BTAS_ERR_BUDGET if the
 *                           request alone exceeds the budget.
 * btas_server_submit_gemm : C (m x n) = A (m x k) (x) B (k x n), host,
 *                           int32 or fp32, min-plus or max-plus.
 * btas_server_poll        : state (0 queued, 1 running, 2 done, 3 failed)
 *                           and seconds since server creation at submit,
 *                           admission and completion (result in host
 *                           memory); any out-pointer may be NULL.
 * btas_server_wait_all    : blocks until no request is queued or running,
 *                           at most timeout_s (BTAS_ERR_TIMEOUT).
 * btas_server_stats       : steps run, units executed, requests completed,
 *                           device bytes currently admitted.
 * btas_server_destroy     : drains outstanding work, then frees the server.
 * ------------------------------------------------------------------------ */
typedef struct btas_server_t btas_server_t;
btas_status btas_server_create(btas_server_t **out, int64_t hbm_budget_bytes, int flags);
btas_status btas_server_submit_apsp(btas_server_t *s, int64_t n, const int32_t *W, int32_t *D, int64_t *ticket);
btas_status btas_server_submit_gemm(btas_server_t *s, int semiring, int dtype, int64_t m, int64_t n, int64_t k,
                                    const void *A, const void *B, void *C, int64_t *ticket);
btas_status btas_server_poll(btas_server_t *s, int64_t ticket, int *state, double *t_submit, double *t_admit,
                             double *t_done);
btas_status btas_server_wait_all(btas_server_t *s, double timeout_s);
btas_status btas_server_stats(btas_server_t *s, int64_t *steps, int64_t *units, int64_t *completed,
                              int64_t *bytes_in_use);
btas_status btas_server_destroy(btas_server_t *s);

#ifdef __cplusplus
}
#endif
#endif /* BTAS_H */
