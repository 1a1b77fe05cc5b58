// Persistent tile-task kernel shared by the batched launch (batch.cu) and
// the continuous-batching server (server.cu).  Host code sees only the
// descriptor structs and the launcher.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace btas {

constexpr int kBT = 128;  // task tile edge (level-0 transposes, and the default output tile)
constexpr int kBTSmall = 64;  // the smaller output tile an instance can take instead

enum TaskType : int {
    kTaskTranspose = 0,
    kTaskApsp = 1,
    kTaskGemm = 2,
    kTaskCopy = 3,
    kTaskSquare = 4,
    kTaskLists = 5,  // APSP level 0: the edge lists of 32 rows of W
    kTaskCert = 6    // APSP after squaring s (its level): the closure certificate over a block of rows
};
enum InstKind : int { kInstApsp = 0, kInstGemm = 1, kInstSquare = 2 };

// One problem of a launch.  kInstApsp: a whole APSP solve (levels = S
// squarings); kInstGemm: one product; kInstSquare: ONE squaring
// C = A (x) A with prev = A, B operand A^T in Q0 (level 0 transposes A into
// Q0 when t0_rows > 0), optional transposed output into Q1 and a change flag
// at changed_ptr.
struct BInst {
    int kind, sr, dtype;
    int tile;             // output tile edge of the level >= 1 tasks: kBT or kBTSmall (0 = kBT)
    int m, n, k;
    int levels;           // APSP: S (>= 1); GEMM / square: 1
    int tiles_m, tiles_n; // output tiles
    int t0_rows, t0_cols; // level-0 transpose source shape (0 x 0: none)
    int done_base;        // done[done_base + level]
    int flag_base;        // changed[flag_base + level]
    int trans_b;
    const void *A;        // GEMM A / APSP W / square input
    long long lda;
    const void *B;        // GEMM B (k x n, or n x k if trans_b)
    long long ldb;
    void *C;              // GEMM C / APSP D / square output
    long long ldc;
    void *X0, *X1;        // APSP intermediate D_s (n x n, pitch ldx)
    long long ldx;
    void *Q0, *Q1;        // APSP transposes / GEMM B^T (Q0) / square B operand and transposed output
    long long ldq;
    int *changed_ptr;     // square: change flag
    // packed 16-bit operand forms of D (set 0 / set 1): duplicated words
    // (pitch ldq) and uint16 values (pitch ldu); APSP: D_s lives in set s & 1;
    // square: input in set 0, output in set 1
    uint32_t *Ad0, *Ad1;
    uint16_t *U0, *U1;
    long long ldu;
    int use_u16;          // APSP: packed squarings allowed; square: 1 = run this one packed,
                          // 2 = decide on the device from *maxfin_in (packed when
                          // 2 * max < 0x7FFF; level-0 transposes then also write the
                          // 16-bit forms of the input into Ad0 / U0)
    int *maxfin_ptr;      // square: atomicMax of the largest finite output
    const int *maxfin_in; // square with use_u16 == 2: largest finite entry of the input,
                          // written before the launch
    // APSP closure certificate (cert = 1): edge lists of W built at level 0
    // (row i: (j + 1, W[i][j]) for its edges j != i in lists[i * cap ..],
    // then zeros; deg[i] edges), and after each squaring s < levels a
    // certificate over blocks of cert_rows rows; when it holds, squaring s + 1
    // copies D_s forward instead of computing it
    int cert;
    int cap;
    int cert_rows;
    int2 *lists;
    int *deg;
};

struct BatchParams {
    const int4 *tasks;  // (type, inst, level, tile)
    int total;
    int *next;
    int *done;
    int *changed;
    int *maxfin;        // per (instance, level): largest finite entry of D_level
    int *certfail;      // per (instance, level): [0] a row has more edges than the lists hold;
                        // [s] the certificate after squaring s failed
    int *status;
    const BInst *insts;
    long long timeout_cycles;
    int withhold_inst;  // fault injection for tests: this instance's level-1+ tasks never become ready
    unsigned long long *prof;  // optional: (cycles, count) per BTAS_BATCH_SLOT_*
};

// Dynamic shared memory and CTAs per SM of the persistent kernel.
int batch_kernel_smem();
int batch_kernel_threads();
cudaError_t batch_kernel_prepare(int *ctas_per_sm);
cudaError_t launch_batch_kernel(const BatchParams &p, int grid, cudaStream_t st);
long long batch_timeout_cycles(int device);

}  // namespace btas
