/*
 * CSR assembly of the 3D Taylor-Hood Q2-Q1 Stokes operator from per-cell
 * blocks (input generator; none of the patch-relaxation arithmetic).
 *
 * Every cell has 89 element DOFs: 3 x 27 velocity (component-blocked, tensor
 * order) then 8 pressure vertices; edofs[c][a] is the global DOF of element
 * DOF a, or -1 when it was eliminated (Dirichlet velocity).  The element
 * matrix is
 *     E[27k + a][27k + b] = K[c][a][b]                  (velocity, same component)
 *     E[81 + q][27k + a]  = E[27k + a][81 + q] = Bd[c][k][q][a]   (divergence)
 * and zero elsewhere; those zeros are still stored (the symbolic pattern of
 * the cell couples all its DOFs).  Row and column `pin` are dropped and the
 * pin row gets a unit diagonal.  Every entry is the sum of its cell
 * contributions in increasing cell order, starting from 0.0, so the result
 * does not depend on the thread count.
 *
 * Build: gcc -O2 -fPIC -shared [-fopenmp] (no architecture-specific flags).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NE 89

static int cmp_i32(const void* a, const void* b) {
    const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static double entry(const double* K, const double* Bd, int64_t c, int a, int b) {
    if (a < 81 && b < 81) {
        if (a / 27 != b / 27) return 0.0;
        return K[(c * 27 + a % 27) * 27 + b % 27];
    }
    if (a >= 81 && b >= 81) return 0.0;
    if (a >= 81) return Bd[((c * 3 + b / 27) * 8 + (a - 81)) * 27 + b % 27];
    return Bd[((c * 3 + a / 27) * 8 + (b - 81)) * 27 + a % 27];
}

/* Row -> (cell, local DOF) lists in increasing cell order.  Returns 0 or -1
 * (allocation failure).  *start gets n+1 offsets, *item the pairs packed as
 * cell * NE + a. */
static int row_lists(int64_t n, int64_t nc, const int64_t* edofs, int64_t pin, int64_t** start_out,
                     int64_t** item_out) {
    int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!start) return -1;
    for (int64_t c = 0; c < nc; ++c)
        for (int a = 0; a < NE; ++a) {
            const int64_t r = edofs[c * NE + a];
            if (r >= 0 && r != pin) start[r + 1]++;
        }
    for (int64_t r = 0; r < n; ++r) start[r + 1] += start[r];
    int64_t* item = (int64_t*)malloc(sizeof(int64_t) * (size_t)(start[n] > 0 ? start[n] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!item || !fill) { free(start); free(item); free(fill); return -1; }
    memcpy(fill, start, sizeof(int64_t) * (size_t)n);
    for (int64_t c = 0; c < nc; ++c)
        for (int a = 0; a < NE; ++a) {
            const int64_t r = edofs[c * NE + a];
            if (r >= 0 && r != pin) item[fill[r]++] = c * NE + a;
        }
    free(fill);
    *start_out = start;
    *item_out = item;
    return 0;
}

/* Pass 1: row lengths (rowptr, n+1 entries, int64).  Returns 0 or -1. */
int stokes3d_pattern_count(int64_t n, int64_t nc, const int64_t* edofs, int64_t pin, int64_t* rowptr) {
    int64_t *start = NULL, *item = NULL;
    if (row_lists(n, nc, edofs, pin, &start, &item)) return -1;
    int fail = 0;
#pragma omp parallel
    {
        int32_t* stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!stamp) {
#pragma omp atomic write
            fail = 1;
        } else {
            for (int64_t i = 0; i < n; ++i) stamp[i] = -1;
#pragma omp for schedule(dynamic, 256)
            for (int64_t r = 0; r < n; ++r) {
                int64_t len = 0;
                if (r == pin) len = 1;
                for (int64_t t = start[r]; t < start[r + 1]; ++t) {
                    const int64_t c = item[t] / NE;
                    for (int b = 0; b < NE; ++b) {
                        const int64_t col = edofs[c * NE + b];
                        if (col < 0 || col == pin) continue;
                        if (stamp[col] != (int32_t)r) { stamp[col] = (int32_t)r; ++len; }
                    }
                }
                rowptr[r + 1] = len;
            }
            free(stamp);
        }
    }
    free(start);
    free(item);
    if (fail) return -1;
    rowptr[0] = 0;
    for (int64_t r = 0; r < n; ++r) rowptr[r + 1] += rowptr[r];
    return 0;
}

/* Pass 2: sorted columns and summed values.  rowptr from pass 1; colidx and
 * vals have rowptr[n] entries.  K: nc x 27 x 27, Bd: nc x 3 x 8 x 27.
 * Returns 0 or -1. */
int stokes3d_fill(int64_t n, int64_t nc, const int64_t* edofs, int64_t pin, const int64_t* rowptr,
                  const double* K, const double* Bd, int32_t* colidx, double* vals) {
    int64_t *start = NULL, *item = NULL;
    if (row_lists(n, nc, edofs, pin, &start, &item)) return -1;
    int fail = 0;
#pragma omp parallel
    {
        int32_t* stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!stamp) {
#pragma omp atomic write
            fail = 1;
        } else {
            for (int64_t i = 0; i < n; ++i) stamp[i] = -1;
#pragma omp for schedule(dynamic, 256)
            for (int64_t r = 0; r < n; ++r) {
                int32_t* cols = colidx + rowptr[r];
                double* v = vals + rowptr[r];
                const int64_t len = rowptr[r + 1] - rowptr[r];
                if (r == pin) {
                    if (len == 1) { cols[0] = (int32_t)pin; v[0] = 1.0; }
                    continue;
                }
                int64_t k = 0;
                for (int64_t t = start[r]; t < start[r + 1]; ++t) {
                    const int64_t c = item[t] / NE;
                    for (int b = 0; b < NE; ++b) {
                        const int64_t col = edofs[c * NE + b];
                        if (col < 0 || col == pin) continue;
                        if (stamp[col] != (int32_t)r) {
                            stamp[col] = (int32_t)r;
                            if (k < len) cols[k] = (int32_t)col;
                            ++k;
                        }
                    }
                }
                if (k != len) {
#pragma omp atomic write
                    fail = 1;
                    continue;
                }
                qsort(cols, (size_t)len, sizeof(int32_t), cmp_i32);
                for (int64_t j = 0; j < len; ++j) v[j] = 0.0;
                /* cell contributions in increasing cell order */
                for (int64_t t = start[r]; t < start[r + 1]; ++t) {
                    const int64_t c = item[t] / NE;
                    const int a = (int)(item[t] % NE);
                    for (int b = 0; b < NE; ++b) {
                        const int64_t col = edofs[c * NE + b];
                        if (col < 0 || col == pin) continue;
                        int64_t lo = 0, hi = len - 1;
                        while (lo < hi) {
                            const int64_t mid = (lo + hi) >> 1;
                            if (cols[mid] < col) lo = mid + 1; else hi = mid;
                        }
                        v[lo] += entry(K, Bd, c, a, b);
                    }
                }
            }
            free(stamp);
        }
    }
    free(start);
    free(item);
    return fail ? -1 : 0;
}
