/*
 * cpu_mttkrp.c — multithreaded FP64 CPU MTTKRP, the all-cores CPU baseline
 * timed beside the GPU library.
 *
 * It computes what the single-threaded oracle computes (paper Sec. 3
 * elementwise computation: every nonzero adds val * Hadamard product of the
 * other modes' factor rows into row i_d of a zero-initialised output,
 * generalised to N modes as in Alg. 2), but over a copy of the nonzeros
 * ordered by the output coordinate, so that OpenMP threads can own whole
 * output rows: each thread takes rows dynamically, accumulates a row in FP64
 * registers and stores it once (no atomics, no reduction).  Separate code:
 * it shares nothing with the oracle or with the GPU library.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Order of the nonzeros by coordinate `mode` (counting sort, stable):
 * perm[rowptr[i] .. rowptr[i+1]) are the nonzeros with i_mode = i.
 * rowptr has dims[mode] + 1 entries.  Returns 0, or -1 on allocation failure. */
int cpu_order(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int mode, int32_t* perm,
              int64_t* rowptr) {
    const int64_t I = dims[mode];
    memset(rowptr, 0, (size_t)(I + 1) * sizeof(int64_t));
    for (int64_t k = 0; k < nnz; ++k) ++rowptr[idx[k * nmodes + mode] + 1];
    for (int64_t i = 0; i < I; ++i) rowptr[i + 1] += rowptr[i];
    int64_t* next = (int64_t*)malloc((size_t)I * sizeof(int64_t));
    if (!next) return -1;
    memcpy(next, rowptr, (size_t)I * sizeof(int64_t));
    for (int64_t k = 0; k < nnz; ++k) perm[next[idx[k * nmodes + mode]]++] = (int32_t)k;
    free(next);
    return 0;
}

/* out[i][r] = sum over the nonzeros of row i of val * prod_{n != mode} A_n(i_n, r), FP64,
 * for every row (rows without nonzeros become 0).  factors: nmodes pointers to fp32
 * [dims[n]][R] (factors[mode] unused); out: fp64 [dims[mode]][R].  threads <= 0: all. */
int cpu_mttkrp(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, const float* vals,
               const float* const* factors, int R, int mode, const int32_t* perm, const int64_t* rowptr,
               double* out, int threads) {
    (void)nnz;
    if (R < 1 || R > 1024 || mode < 0 || mode >= nmodes) return -1;
    const int64_t I = dims[mode];
    const int T = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel num_threads(T)
    {
        double acc[1024], prod[1024];
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < I; ++i) {
            for (int r = 0; r < R; ++r) acc[r] = 0.0;
            for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
                const int64_t k = perm[j];
                const double v = (double)vals[k];
                for (int r = 0; r < R; ++r) prod[r] = v;
                for (int n = 0; n < nmodes; ++n) {
                    if (n == mode) continue;
                    const float* a = factors[n] + (int64_t)idx[k * nmodes + n] * R;
                    for (int r = 0; r < R; ++r) prod[r] *= (double)a[r];
                }
                for (int r = 0; r < R; ++r) acc[r] += prod[r];
            }
            double* o = out + i * R;
            for (int r = 0; r < R; ++r) o[r] = acc[r];
        }
    }
    return 0;
}

int cpu_threads(void) { return omp_get_max_threads(); }
