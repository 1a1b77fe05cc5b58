/*
 * btas_oracle.c -- plain, slow, obviously-correct CPU reference for the
 * tropical-algebra hot path.  TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the benchmark's CPU-baseline leg may call it; the library's own
 * product path never does.  It shares no code, header or constant table with
 * the CUDA implementation.
 *
 * Every routine is the textbook definition written out:
 *   - semiring operations: max-plus (Eq. 1-2) and min-plus (Eq. 3-4), Sec. I;
 *   - tropical matrix product Z <- Z (+) X (.) Y, "Matrix-Matrix
 *     Multiplication for Floyd-Warshall" (the second listing titled
 *     Algorithm 3), obtained from the linear-algebra product by replacing
 *     + with min (or max) and x with +;
 *   - APSP by repeated squaring of the weighted adjacency matrix, Sec. III;
 *   - sequential Floyd-Warshall, Algorithm 2 (Sec. IV), with a dedicated
 *     INF for "no edge" instead of the paper's 0 sentinel;
 *   - Dijkstra from one source and brute-force enumeration of simple paths
 *     (textbook routines, used only to pin the above).
 *
 * Integer encoding (a reading of the paper, which uses 0 or -1 for "no
 * edge"): INF = 0x3FFFFFFF is the min-plus (+)-identity and is absorbing for
 * (.); -INF = -0x3FFFFFFF plays the same role in max-plus.  Finite values lie
 * in [-2^28, 2^28].  The 16-bit path stores values in [0, 0x7FFF] with
 * INF16 = 0x7FFF and saturates every result at INF16.  FP32 uses IEEE +inf
 * (min-plus) / -inf (max-plus) and one round-to-nearest add per term.
 *
 * Loops over independent output rows carry an OpenMP pragma; the arithmetic
 * of every output element is the plain sequential k-loop.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define O_INF32 ((int32_t)0x3FFFFFFF)
#define O_NINF32 ((int32_t)-0x3FFFFFFF)
#define O_INF16 ((int32_t)0x7FFF)

enum { O_MINPLUS = 0, O_MAXPLUS = 1 };

static int o_threads = 1;

void oracle_set_threads(int t) { o_threads = t > 0 ? t : 1; }
int oracle_get_threads(void) { return o_threads; }

/* ---------- scalar semiring operations (Eq. 1-4) ---------- */

/* x (.) y in the integer encoding: INF (or -INF) absorbs, otherwise x + y. */
static int32_t otimes_i32(int sr, int32_t x, int32_t y) {
    int32_t absorb = (sr == O_MINPLUS) ? O_INF32 : O_NINF32;
    if (x == absorb || y == absorb) return absorb;
    return x + y;
}

/* x (+) y: min (Eq. 3) or max (Eq. 1). */
static int32_t oplus_i32(int sr, int32_t x, int32_t y) {
    if (sr == O_MINPLUS) return x < y ? x : y;
    return x > y ? x : y;
}

/* One IEEE binary32 round-to-nearest add: the file is compiled with
 * -ffp-contract=off and no fast-math, and both targets evaluate float
 * expressions in float (FLT_EVAL_METHOD == 0). */
static float otimes_f32(float x, float y) {
    float s = x + y;
    return s;
}

static float oplus_f32(int sr, float x, float y) {
    if (sr == O_MINPLUS) return y < x ? y : x;
    return y > x ? y : x;
}

/* ---------- tropical matrix product (Eq. 1-4; product listing, Sec. IV) ----------
 * C[i][j] = (+)_{k<K} A[i][k] (.) B[k][j]; with accumulate != 0 the old
 * C[i][j] enters the (+) as in Z <- Z (+) X (.) Y.  Row-major, leading
 * dimensions in elements.  K = 0 yields the (+)-identity (or leaves C). */
void oracle_tgemm_i32(int sr, int accumulate, int64_t m, int64_t n, int64_t k,
                      const int32_t *A, int64_t lda, const int32_t *B, int64_t ldb,
                      int32_t *C, int64_t ldc) {
    int32_t ident = (sr == O_MINPLUS) ? O_INF32 : O_NINF32;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1) num_threads(o_threads)
    for (i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            int32_t acc = accumulate ? C[i * ldc + j] : ident;
            for (int64_t kk = 0; kk < k; ++kk)
                acc = oplus_i32(sr, acc, otimes_i32(sr, A[i * lda + kk], B[kk * ldb + j]));
            C[i * ldc + j] = acc;
        }
    }
}

void oracle_tgemm_f32(int sr, int accumulate, int64_t m, int64_t n, int64_t k,
                      const float *A, int64_t lda, const float *B, int64_t ldb,
                      float *C, int64_t ldc) {
    float ident = (sr == O_MINPLUS) ? INFINITY : -INFINITY;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1) num_threads(o_threads)
    for (i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            float acc = accumulate ? C[i * ldc + j] : ident;
            for (int64_t kk = 0; kk < k; ++kk)
                acc = oplus_f32(sr, acc, otimes_f32(A[i * lda + kk], B[kk * ldb + j]));
            C[i * ldc + j] = acc;
        }
    }
}

/* 16-bit min-plus with saturation at INF16: a term with an INF16 operand is
 * INF16, any finite sum is exact, and the result is min(INF16, min_k term). */
void oracle_tgemm_u16(int accumulate, int64_t m, int64_t n, int64_t k,
                      const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb,
                      uint16_t *C, int64_t ldc) {
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1) num_threads(o_threads)
    for (i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            int32_t acc = accumulate ? (int32_t)C[i * ldc + j] : O_INF16;
            for (int64_t kk = 0; kk < k; ++kk) {
                int32_t a = A[i * lda + kk], b = B[kk * ldb + j];
                int32_t s = (a >= O_INF16 || b >= O_INF16) ? O_INF16 : a + b;
                if (s < acc) acc = s;
            }
            if (acc > O_INF16) acc = O_INF16;
            C[i * ldc + j] = (uint16_t)acc;
        }
    }
}

/* ---------- APSP ---------- */

/* Number of squarings S = ceil(log2(n-1)) for n >= 3, 0 otherwise: after s
 * squarings D holds the shortest walks of at most 2^s edges (Sec. III), and a
 * shortest path has at most n-1 edges. */
int oracle_apsp_squarings(int64_t n) {
    int s = 0;
    int64_t reach = 1;
    while (reach < n - 1) { reach *= 2; ++s; }
    return s;
}

/* APSP by repeated squaring (Sec. III): D_0 = W, D_{s+1} = D_s (x) D_s in
 * min-plus, S times.  Out of place; D receives D_S. */
void oracle_apsp_squaring_i32(int64_t n, const int32_t *W, int32_t *D, int squarings) {
    size_t bytes = (size_t)n * (size_t)n * sizeof(int32_t);
    int32_t *cur = (int32_t *)malloc(bytes ? bytes : 1);
    int32_t *nxt = (int32_t *)malloc(bytes ? bytes : 1);
    if (bytes) memcpy(cur, W, bytes);
    for (int s = 0; s < squarings; ++s) {
        oracle_tgemm_i32(O_MINPLUS, 0, n, n, n, cur, n, cur, n, nxt, n);
        int32_t *t = cur; cur = nxt; nxt = t;
    }
    if (bytes) memcpy(D, cur, bytes);
    free(cur);
    free(nxt);
}

void oracle_apsp_squaring_u16(int64_t n, const uint16_t *W, uint16_t *D, int squarings) {
    size_t bytes = (size_t)n * (size_t)n * sizeof(uint16_t);
    uint16_t *cur = (uint16_t *)malloc(bytes ? bytes : 1);
    uint16_t *nxt = (uint16_t *)malloc(bytes ? bytes : 1);
    if (bytes) memcpy(cur, W, bytes);
    for (int s = 0; s < squarings; ++s) {
        oracle_tgemm_u16(0, n, n, n, cur, n, cur, n, nxt, n);
        uint16_t *t = cur; cur = nxt; nxt = t;
    }
    if (bytes) memcpy(D, cur, bytes);
    free(cur);
    free(nxt);
}

/* APSP by repeated squaring with next-hop (successor) tracking.  N_0[i][j] =
 * j for an edge i->j (i != j), i on the diagonal, -1 for no edge.  One
 * squaring: D'[i][j] = min_k D[i][k] + D[k][j] with k* the SMALLEST minimising
 * k (all k in 0..n-1, including i and j); N'[i][j] = -1 if D'[i][j] is INF,
 * else the first hop of the walk (i -> k*) + (k* -> j): N[i][j] when k* == i
 * (the first leg is empty), N[i][k*] otherwise.  Exactly `squarings` steps. */
void oracle_apsp_paths_i32(int64_t n, const int32_t *W, int32_t *D, int32_t *Next, int squarings) {
    size_t nn = (size_t)n * (size_t)n;
    int32_t *d = (int32_t *)malloc(nn ? nn * 4 : 4), *d2 = (int32_t *)malloc(nn ? nn * 4 : 4);
    int32_t *x = (int32_t *)malloc(nn ? nn * 4 : 4), *x2 = (int32_t *)malloc(nn ? nn * 4 : 4);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            d[i * n + j] = W[i * n + j];
            x[i * n + j] = (i == j) ? (int32_t)i : (W[i * n + j] == O_INF32 ? -1 : (int32_t)j);
        }
    for (int s = 0; s < squarings; ++s) {
        int64_t i;
#pragma omp parallel for schedule(dynamic, 1) num_threads(o_threads)
        for (i = 0; i < n; ++i) {
            for (int64_t j = 0; j < n; ++j) {
                int32_t best = O_INF32;
                int64_t kbest = -1;
                for (int64_t k = 0; k < n; ++k) {
                    int32_t t = otimes_i32(O_MINPLUS, d[i * n + k], d[k * n + j]);
                    if (t < best) { best = t; kbest = k; }
                }
                d2[i * n + j] = best;
                if (best == O_INF32) x2[i * n + j] = -1;
                else if (kbest == i) x2[i * n + j] = x[i * n + j];
                else x2[i * n + j] = x[i * n + kbest];
            }
        }
        int32_t *t = d; d = d2; d2 = t;
        t = x; x = x2; x2 = t;
    }
    memcpy(D, d, nn * 4);
    memcpy(Next, x, nn * 4);
    free(d); free(d2); free(x); free(x2);
}

/* The same next-hop squaring on binary32 weights (+inf = no edge, weights
 * >= 0): each term is one round-to-nearest add (otimes_f32), and the SMALLEST
 * k whose rounded sum attains the minimum is kept, so a tie that only the
 * rounding creates is broken towards the smaller k like any other tie.
 * N_0 and the successor rule are those of oracle_apsp_paths_i32.  Exactly
 * `squarings` steps. */
void oracle_apsp_paths_f32(int64_t n, const float *W, float *D, int32_t *Next, int squarings) {
    size_t nn = (size_t)n * (size_t)n;
    float *d = (float *)malloc(nn ? nn * 4 : 4), *d2 = (float *)malloc(nn ? nn * 4 : 4);
    int32_t *x = (int32_t *)malloc(nn ? nn * 4 : 4), *x2 = (int32_t *)malloc(nn ? nn * 4 : 4);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            d[i * n + j] = W[i * n + j];
            x[i * n + j] = (i == j) ? (int32_t)i : (isinf(W[i * n + j]) ? -1 : (int32_t)j);
        }
    for (int s = 0; s < squarings; ++s) {
        int64_t i;
#pragma omp parallel for schedule(dynamic, 1) num_threads(o_threads)
        for (i = 0; i < n; ++i) {
            for (int64_t j = 0; j < n; ++j) {
                float best = INFINITY;
                int64_t kbest = -1;
                for (int64_t k = 0; k < n; ++k) {
                    float t = otimes_f32(d[i * n + k], d[k * n + j]);
                    if (t < best) { best = t; kbest = k; }
                }
                d2[i * n + j] = best;
                if (isinf(best)) x2[i * n + j] = -1;
                else if (kbest == i) x2[i * n + j] = x[i * n + j];
                else x2[i * n + j] = x[i * n + kbest];
            }
        }
        float *tf = d; d = d2; d2 = tf;
        int32_t *t = x; x = x2; x2 = t;
    }
    memcpy(D, d, nn * 4);
    memcpy(Next, x, nn * 4);
    free(d); free(d2); free(x); free(x2);
}

/* Sequential Floyd-Warshall (Algorithm 2): pivot z outermost, relax
 * D[x][y] through z when both legs exist.  In place; row z and column z do
 * not change while z is the pivot, so the in-place update is exact. */
void oracle_fw_i32(int64_t n, int32_t *D) {
    for (int64_t z = 0; z < n; ++z) {
        int64_t x;
#pragma omp parallel for schedule(static) num_threads(o_threads)
        for (x = 0; x < n; ++x) {
            int32_t dxz = D[x * n + z];
            if (dxz == O_INF32) continue;
            for (int64_t y = 0; y < n; ++y) {
                int32_t dzy = D[z * n + y];
                if (dzy == O_INF32 || x == y) continue;
                if (dxz + dzy < D[x * n + y]) D[x * n + y] = dxz + dzy;
            }
        }
    }
}

/* Dijkstra from `src` on the dense adjacency matrix W (non-negative weights,
 * INF = no edge), the O(n^2) array form.  dist receives one row of APSP. */
void oracle_dijkstra_i32(int64_t n, const int32_t *W, int64_t src, int32_t *dist) {
    char *done = (char *)calloc((size_t)(n ? n : 1), 1);
    for (int64_t v = 0; v < n; ++v) dist[v] = O_INF32;
    dist[src] = 0;
    for (int64_t it = 0; it < n; ++it) {
        int64_t u = -1;
        int32_t best = O_INF32;
        for (int64_t v = 0; v < n; ++v)
            if (!done[v] && dist[v] < best) { best = dist[v]; u = v; }
        if (u < 0) break;
        done[u] = 1;
        for (int64_t v = 0; v < n; ++v) {
            int32_t w = W[u * n + v];
            if (w == O_INF32 || done[v]) continue;
            if (best + w < dist[v]) dist[v] = best + w;
        }
    }
    free(done);
}

/* Dijkstra from several sources; rows[s] = distances from srcs[s]. */
void oracle_dijkstra_rows_i32(int64_t n, const int32_t *W, int64_t nsrc,
                              const int64_t *srcs, int32_t *rows) {
    int64_t s;
#pragma omp parallel for schedule(dynamic, 1) num_threads(o_threads)
    for (s = 0; s < nsrc; ++s) oracle_dijkstra_i32(n, W, srcs[s], rows + s * n);
}

/* Brute force: the minimum weight over every simple path, by depth-first
 * enumeration.  Only for n <= 8. */
static void bf_dfs(int64_t n, const int32_t *W, int64_t src, int64_t u, int64_t len,
                   unsigned visited, int32_t *row) {
    if (len < row[u]) row[u] = (int32_t)len;
    for (int64_t v = 0; v < n; ++v) {
        if (visited & (1u << v)) continue;
        int32_t w = W[u * n + v];
        if (w == O_INF32) continue;
        bf_dfs(n, W, src, v, len + w, visited | (1u << v), row);
    }
}

int oracle_bruteforce_apsp_i32(int64_t n, const int32_t *W, int32_t *D) {
    if (n > 8) return -1;
    for (int64_t s = 0; s < n; ++s) {
        int32_t *row = D + s * n;
        for (int64_t v = 0; v < n; ++v) row[v] = O_INF32;
        bf_dfs(n, W, s, s, 0, 1u << s, row);
    }
    return 0;
}

/* ---------- level 2: tropical matrix-vector products ----------
 * trans == 0: y[i] = (+)_j A[i][j] (.) x[j]   (i < m, j < n)
 * trans == 1: y[j] = (+)_i x[i] (.) A[i][j]   (j < n, i < m)
 * accumulate: the old y entry enters the (+). */
void oracle_gemv_i32(int sr, int trans, int accumulate, int64_t m, int64_t n, const int32_t *A, int64_t lda,
                     const int32_t *x, int32_t *y) {
    int32_t ident = (sr == O_MINPLUS) ? O_INF32 : O_NINF32;
    int64_t outer = trans ? n : m, inner = trans ? m : n;
    for (int64_t o = 0; o < outer; ++o) {
        int32_t acc = accumulate ? y[o] : ident;
        for (int64_t q = 0; q < inner; ++q) {
            int32_t a = trans ? A[q * lda + o] : A[o * lda + q];
            acc = oplus_i32(sr, acc, otimes_i32(sr, trans ? x[q] : x[q], a));
        }
        y[o] = acc;
    }
}

void oracle_gemv_f32(int sr, int trans, int accumulate, int64_t m, int64_t n, const float *A, int64_t lda,
                     const float *x, float *y) {
    float ident = (sr == O_MINPLUS) ? INFINITY : -INFINITY;
    int64_t outer = trans ? n : m, inner = trans ? m : n;
    for (int64_t o = 0; o < outer; ++o) {
        float acc = accumulate ? y[o] : ident;
        for (int64_t q = 0; q < inner; ++q) {
            float a = trans ? A[q * lda + o] : A[o * lda + q];
            acc = oplus_f32(sr, acc, otimes_f32(x[q], a));
        }
        y[o] = acc;
    }
}

/* Single-source shortest paths by repeated vector-matrix products
 * (Bellman-Ford in min-plus form): d_0 = e_src (0 at src, INF elsewhere),
 * d_{t+1} = d_t (x) W (row vector times matrix; W[j][j] = 0 keeps d_t[j]),
 * until d stops changing, at most n-1 products.  Returns the number of
 * products that changed d. */
int oracle_sssp_i32(int64_t n, const int32_t *W, int64_t src, int32_t *dist) {
    int32_t *nxt = (int32_t *)malloc((size_t)(n ? n : 1) * 4);
    for (int64_t v = 0; v < n; ++v) dist[v] = O_INF32;
    dist[src] = 0;
    int changed_steps = 0;
    for (int64_t t = 0; t + 1 < n; ++t) {
        oracle_gemv_i32(O_MINPLUS, 1, 0, n, n, W, n, dist, nxt);
        int changed = 0;
        for (int64_t v = 0; v < n; ++v) changed |= nxt[v] != dist[v];
        memcpy(dist, nxt, (size_t)n * 4);
        if (!changed) break;
        ++changed_steps;
    }
    free(nxt);
    return changed_steps;
}

/* ---------- tropical vector operations ("standard vector operations", Abstract / Sec. III) ---------- */

/* dot: (+)_i x_i (.) y_i */
int32_t oracle_dot_i32(int sr, int64_t n, const int32_t *x, int64_t incx,
                       const int32_t *y, int64_t incy) {
    int32_t acc = (sr == O_MINPLUS) ? O_INF32 : O_NINF32;
    for (int64_t i = 0; i < n; ++i)
        acc = oplus_i32(sr, acc, otimes_i32(sr, x[i * incx], y[i * incy]));
    return acc;
}

float oracle_dot_f32(int sr, int64_t n, const float *x, int64_t incx,
                     const float *y, int64_t incy) {
    float acc = (sr == O_MINPLUS) ? INFINITY : -INFINITY;
    for (int64_t i = 0; i < n; ++i)
        acc = oplus_f32(sr, acc, otimes_f32(x[i * incx], y[i * incy]));
    return acc;
}

/* axpy-like: y_i <- y_i (+) (alpha (.) x_i) */
void oracle_axpy_i32(int sr, int64_t n, int32_t alpha, const int32_t *x, int64_t incx,
                     int32_t *y, int64_t incy) {
    for (int64_t i = 0; i < n; ++i)
        y[i * incy] = oplus_i32(sr, y[i * incy], otimes_i32(sr, alpha, x[i * incx]));
}

void oracle_axpy_f32(int sr, int64_t n, float alpha, const float *x, int64_t incx,
                     float *y, int64_t incy) {
    for (int64_t i = 0; i < n; ++i)
        y[i * incy] = oplus_f32(sr, y[i * incy], otimes_f32(alpha, x[i * incx]));
}

/* element-wise z_i = x_i (+) y_i and z_i = x_i (.) y_i */
void oracle_add_i32(int sr, int64_t n, const int32_t *x, const int32_t *y, int32_t *z) {
    for (int64_t i = 0; i < n; ++i) z[i] = oplus_i32(sr, x[i], y[i]);
}

void oracle_mul_i32(int sr, int64_t n, const int32_t *x, const int32_t *y, int32_t *z) {
    for (int64_t i = 0; i < n; ++i) z[i] = otimes_i32(sr, x[i], y[i]);
}

void oracle_add_f32(int sr, int64_t n, const float *x, const float *y, float *z) {
    for (int64_t i = 0; i < n; ++i) z[i] = oplus_f32(sr, x[i], y[i]);
}

void oracle_mul_f32(int sr, int64_t n, const float *x, const float *y, float *z) {
    (void)sr;
    for (int64_t i = 0; i < n; ++i) z[i] = otimes_f32(x[i], y[i]);
}
