// Internal interface between the C-ABI layer (btas_api.cu) and the kernel
// translation units.  Host-side declarations only.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "tgemm_args.h"

namespace btas {

// Process-wide count of kernels this library has enqueued (btas_kernel_launches).
void note_launch(int n = 1);
// Sets the calling thread's message returned by btas_last_error_string.
void record_error(const char *msg);
// BTAS_LOG level (read once from the environment) and a printf-style line
// to stderr when it is >= 1.
int log_level();
void log_event(const char *fmt, ...);
// Device facts queried once per device (some attribute queries cost
// hundreds of microseconds): compute capability major*10+minor, SM count,
// SM clock in kHz.  Returns false if the device cannot be queried.
struct DeviceInfo {
    int arch, sms, clock_khz;
};
bool current_device_info(DeviceInfo *out, int *device = nullptr);
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (function, device).
cudaError_t set_smem_once(const void *func, int bytes);
// Stream-ordered workspace from the library's pool of the current device.
cudaError_t ws_alloc(void **p, size_t bytes, cudaStream_t st);
cudaError_t ws_free(void *p, cudaStream_t st);
// Raise the current device pool's release threshold to at least `bytes`
// (memory freed to the pool stays cached up to it).
cudaError_t ws_keep_at_least(uint64_t bytes);

// ---- tropical GEMM kernel registry (tgemm_*.cu)
struct GemmKernel {
    int var;      // Variant
    int sr;       // Semiring
    int ns;       // kI32Mix: columns on the IMAD path
    int cfg;      // tile configuration id
    int bm, bn, threads, smem;
    cudaError_t (*launch)(const GemmArgs &, cudaStream_t);
};
const GemmKernel *find_gemm_kernel(int var, int sr, int ns, int cfg);
int gemm_kernel_count();
const GemmKernel *gemm_kernel_at(int i);

// ---- autotuner (tune.cu)
struct TuneChoice {
    int var, ns, cfg, group_m;  // var 16: packed u16x2 kernel (ns = its IMAD split)
};
// Tuned kernel for (sr, dtype, m, n, k) on the current device: a table entry,
// or -- when BTAS_TUNE=1 and `st` is not capturing -- a tuning run on the
// spot.  false: no choice (use the defaults).
bool tune_choice(int sr, int dtype, long long m, long long n, long long k, cudaStream_t st, TuneChoice *out);

// ---- auxiliary kernels (aux.cu)
// Per-device status words of asynchronous checks (allocated on first use):
// [0] entries outside the domain found by BTAS_GEMM_CHECKED products,
// [1] checked products that found any.  Read and cleared by btas_sync_status.
unsigned long long *device_status_words();
// BTAS_GEMM_CHECKED: count the entries of X outside the product's domain into
// *count and status[0].
cudaError_t launch_domain_check(const void *X, long long ld, int rows, int cols, int is_float, int sr, int *count,
                                unsigned long long *status, cudaStream_t st);
// *skip = (*count != 0) || packed path chosen (pack_state may be null); a
// violation counts the call in status[1].
cudaError_t launch_checked_gate(const int *count, const int *pack_state, int *skip, unsigned long long *status,
                                cudaStream_t st);
// dst (cols x rows, ldd) = transpose of src (rows x cols, lds); 4-byte elements.
// mode: 0 = copy, 1 = int32 -> fp32 carrier (INF -> +inf, -INF -> -inf),
// 2 = fp32 carrier -> int32 (inverse).
cudaError_t launch_transpose4(const void *src, long long lds, int rows, int cols, void *dst,
                              long long ldd, int mode, const int *skip, cudaStream_t st);
// Element-wise conversion of a rows x cols matrix (mode as above, 0 = copy).
cudaError_t launch_convert4(const void *src, long long lds, int rows, int cols, void *dst,
                            long long ldd, int mode, cudaStream_t st);
// Fill a rows x cols matrix of 4-byte elements with `bits`.
cudaError_t launch_fill4(void *dst, long long ldd, int rows, int cols, uint32_t bits, cudaStream_t st);
// dst = E (+) src for an n x n matrix of 4-byte elements (diagonal (+) 0).
cudaError_t launch_ident_oplus(const void *src, long long lds, int n, void *dst, long long ldd, int sr, int is_float,
                               cudaStream_t st);
// APSP domain scan of an n x n int32 matrix: out[0] = max finite weight,
// out[1] = number of entries out of the domain (negative, > 2^28 and not INF,
// or a non-zero diagonal).  out must be zeroed first.
cudaError_t launch_apsp_scan(const int *W, long long n, int *out, cudaStream_t st, long long ldw = 0);  // ldw 0: n

// ---- APSP with next-hop matrix (paths.cu)
// Keyed path squaring (paths.cu): while every finite entry of D is <=
// paths_key_max() and n <= paths_key_max_n(), one int32 min-plus product of
// A' = D << 13 and B' = (D << 13) | k gives distances and smallest
// minimising k together.  encode: A' (pitch n) and B'^T (pitch ldt);
// decode: keys -> D', N' (K may be Dn), change flag, largest finite entry.
int paths_key_max();
int paths_key_max_n();
cudaError_t launch_paths_encode(const int *D, int n, int *Ak, int *BkT, long long ldt, cudaStream_t st);
cudaError_t launch_paths_decode(const int *K, const int *D, const int *N, long long n, int *Dn, int *Nn, int *changed,
                                int *maxfin, cudaStream_t st);
cudaError_t launch_next_init(const int *W, long long n, int *N, cudaStream_t st);
// binary32 forms: successors of W (+inf = no edge), the weight-domain count
// (zero diagonal, entries >= 0 or +inf; *bad must be zeroed first) and the
// argmin squaring with one round-to-nearest add per term.
cudaError_t launch_next_init_f32(const float *W, long long n, int *N, cudaStream_t st);
cudaError_t launch_paths_scan_f32(const float *W, long long n, int *bad, cudaStream_t st);
cudaError_t launch_paths_square_f32(int n, const float *D, long long ldd, const float *Dt, long long ldt,
                                    const int *N, float *D2, int *N2, int *changed, cudaStream_t st);
cudaError_t launch_paths_square(int n, const int *D, long long ldd, const int *Dt, long long ldt, const int *N,
                                int *D2, int *N2, int *changed, cudaStream_t st);

// ---- level 2 (gemv.cu): trans 0: y_i = (+)_j A[i][j] (.) x_j; trans 1:
// y_j = (+)_i x_i (.) A[i][j]; accumulate keeps y as a (+) start value;
// changed (trans 1, optional) is set when some y entry changes; skip
// (trans 1 with accumulate, optional): *skip == 0 makes the launch a no-op.
cudaError_t launch_gemv(int sr, int dtype, int trans, int m, int n, const void *A, long long lda, const void *x,
                        void *y, int accumulate, int *changed, cudaStream_t st, const int *skip = nullptr);

// ---- Bellman-Ford SSSP in one cooperative launch (gemv.cu): W n x n
// (pitch n), dist (n ints, device); ws: sssp_coop_workspace(n) bytes; info
// (device, 4 ints, zeroed by the caller): [0] products that changed d, [1]
// status (BTAS_ERR_TIMEOUT), [2] entries of W outside the domain (checked
// during the first product; dist is then not written), [3] scratch.
size_t sssp_coop_workspace(long long n);
cudaError_t launch_sssp_coop(const int *W, long long n, int src, int *dist, void *ws, int *info, cudaStream_t st);

// ---- APSP in one thread block for n <= apsp_small_max_n() (small.cu).
// info (device, 3 ints): entries outside the domain, largest finite weight,
// squarings that changed D.  Nothing is written to D if the domain check
// fails.
int apsp_small_max_n();
int apsp_small_limit();  // the size up to which callers use it (<= apsp_small_max_n())
cudaError_t launch_apsp_small(const int *W, long long ldw, int n, int S, bool early, int *D, long long ldd,
                              int *info, cudaStream_t st);

// ---- APSP in one cooperative launch for apsp_small_limit() < n <=
// apsp_mid_max_n() (mid.cu).  ws: ws_bytes >= apsp_mid_workspace_min(n)
// bytes; with apsp_mid_workspace(n, S) bytes the launch also builds edge
// lists of W, which give the first squaring by sparse products (when every
// row has at most apsp_mid_list_cap(n) edges) and the closure certificate
// that saves the squaring which would only confirm the fixpoint.  info
// (device, 5 ints zeroed by the caller; or null: the words at
// apsp_mid_info(ws, n), zeroed by the launch): [0] entries outside the
// domain, [1] largest finite weight, [2] squarings that changed D, [3]
// status, [4] representations used (1 int32, 4 packed 16-bit, 8 the first
// squaring from the edge lists).  packed_ok =
// false keeps every squaring on int32 (so does BTAS_MID_NO_U16=1 in the
// environment).  From n = 1408 (BTAS_MID_WIDE_MIN_N) the launch takes the
// warp-specialised form with 128 x 128 tiles.  mailbox (optional, a
// host-mapped pointer the device can write): info[0 .. 4] are copied there
// as the launch ends, so the caller reads them after synchronising the
// stream, without a device-to-host copy.  bail_dense (with the full
// workspace): if some row of W has more edges than the lists hold, the
// launch stops after the domain check with D untouched and info[4] =
// kMidDeclined, and the caller solves on the tiled kernels.
constexpr int kMidDeclined = 16;
constexpr long long kMidSparseMaxN = 4096;  // largest n btas_apsp offers the cooperative kernel with bail_dense
int apsp_mid_max_n();
// Whether btas_apsp offers n to the cooperative kernel: every n <=
// apsp_mid_max_n(), and (unless BTAS_APSP_MID_MAX_N is set) every n <=
// kMidSparseMaxN with bail_dense, so that only graphs sparse enough for the
// edge lists stay there.  With the first squaring from the lists and the
// closure certificate it beats the tiled kernels on such graphs at every
// size measured up to 4096 (GB300, p = 0.02 and 0.05: 1.38 vs 1.62 ms at
// n = 2048, 4.95 vs 5.31 ms at 3072, 10.9 vs 13.7 ms at 4096); on dense
// graphs neither applies and the tiled kernels are faster above 1792.
bool apsp_mid_takes(long long n, int sms);
int apsp_mid_list_cap(long long n);
size_t apsp_mid_workspace_min(long long n);
size_t apsp_mid_workspace(long long n, int S);
int *apsp_mid_info(void *ws, long long n);
cudaError_t launch_apsp_mid(const int *W, long long ldw, int n, int S, bool early, bool packed_ok, int *D,
                            long long ldd, void *ws, size_t ws_bytes, int *info, cudaStream_t st,
                            int *mailbox = nullptr, bool bail_dense = false);

// ---- blocked Floyd-Warshall (fw.cu): phases 1 and 2 of pivot block kb
// pmax (optional): atomicMax of the largest finite value the phases store
// (the pivot row and column panels).
// Lookahead update: pivot block kb's phase-3 terms applied to block row and
// column kb + 1 only (nothing when kb is the last block).
cudaError_t launch_fw_cross(int *D, long long n, int kb, cudaStream_t st);
cudaError_t launch_fw_phase12(int *D, long long n, int kb, int *pmax, cudaStream_t st);
// int32 phase 3 of pivot block (offset o, width bw) over every tile outside
// tile rows and columns [x0, x1), in one launch; skipped when *bypass != 0.
cudaError_t launch_fw_phase3_i32(int *D, long long n, long long o, int bw, const int *RPT, int x0, int x1,
                                 const int *bypass, cudaStream_t st);
// Packed phase 3 set-up for pivot block kb: state[0] = 1 if 2 * *pmax <
// 0x7FFF (state[1] = !state[0]); when set, the column panel goes to Ad
// (duplicated words, n x ldad) and the row panel to Bu (uint16, bw x ldbu).
cudaError_t launch_fw_pack(int *D, long long n, int kb, const int *pmax, int *state, uint32_t *Ad, long long ldad,
                           uint16_t *Bu, long long ldbu, cudaStream_t st);
int fw_block();

// ---- vector kernels (tvec.cu)
cudaError_t launch_dot(int sr, int dtype, long long n, const void *x, long long incx, const void *y,
                       long long incy, void *result, void *partials, int nblocks, cudaStream_t st);
cudaError_t launch_axpy(int sr, int dtype, long long n, uint32_t alpha_bits, const void *x,
                        long long incx, void *y, long long incy, cudaStream_t st);
cudaError_t launch_ewise(int op, int sr, int dtype, long long n, const void *x, const void *y,
                         void *z, cudaStream_t st);

// ---- packed 16-bit GEMM (tgemm_u16.cu)
struct U16Args {
    int m, n, k;
    const uint16_t *A; long long lda;
    const uint16_t *B; long long ldb;   // k x n row-major (not transposed)
    uint16_t *C; long long ldc;
    const uint16_t *prev; long long ldp;
    int *changed;
    const int *skip;
    int one;
    int *maxfin;  // optional: atomicMax of the largest output below INF16
    const int *gate;    // optional: *gate == 0 => the launches do nothing
    bool adup_ready;    // `adup` already holds A's duplicated words (no pre-pass)
    int *Ci;            // optional: int32 accumulate target, Ci = min(Ci, result); C is then not written
    long long ldci;
    int xr0, xr1, xc0, xc1;  // with Ci: rows [xr0, xr1) and columns [xc0, xc1) of Ci are left untouched
};
// Duplicates A into `adup` (m x round4(k) 32-bit words, caller workspace;
// with adup_ready the caller has filled it, with that pitch) and runs the
// packed product; ns = number of the 8 column pairs per thread that
// take the IMAD + 3-input-min path (the rest use DPX).
cudaError_t launch_tgemm_u16_ws(const U16Args &a, uint32_t *adup, int ns, cudaStream_t st);
// ---- exact packed path for int32 products (pack.cu).  Device state words:
// [0] packed? [1] offset of A [2] offset of B [3] !packed [4..7] ranges
// and out-of-domain count.  All launches are stream-ordered; the choice is
// made on the device.  extra_bad (optional, device): a count of entries
// outside the domain from the caller's own check; non-zero withdraws the
// packed path.
constexpr int kPackStateInts = 16;
constexpr int kPackStateUse = 0, kPackStateNotUse = 3;
cudaError_t launch_pack_prepare(int sr, int m, int n, int k, const int *A, long long lda, const int *B, long long ldb,
                                bool trans_b, int *state, uint32_t *adup, uint16_t *bu, long long ldbu,
                                cudaStream_t st, const int *extra_bad = nullptr);
cudaError_t launch_pack_finish(int sr, int m, int n, const uint16_t *cu, long long ldcu, const int *state, int *C,
                               long long ldc, bool accumulate, cudaStream_t st);
long long packed_products(int device);
cudaError_t launch_narrow_u16(const int *src, long long total, uint16_t *dst, cudaStream_t st);
cudaError_t launch_widen_u16_i32(const uint16_t *src, long long total, int *dst, cudaStream_t st);

}  // namespace btas
