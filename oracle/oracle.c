/*
 * oracle.c — FP64 CPU oracle for sparse MTTKRP and the sampled CP model.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The GPU library
 * never calls, links or includes anything from this directory, and this
 * file includes nothing from the GPU library.
 *
 * Every routine is a plain, single-threaded loop over the nonzeros in the
 * order the caller gives them, accumulating in double precision.  Factor
 * entries are read in their storage type (fp32, bf16, fp16, or fp64 for the
 * ALS oracle) and widened exactly to double.
 *
 * What is computed (paper, Sec. 3 "Elementwise computation" and Alg. 2):
 *   for output mode d and each nonzero x at (i_0, ..., i_{N-1}),
 *     M(i_d, r) += val(x) * prod_{w != d} Y_w(i_w, r),   r = 0..R-1,
 *   with M starting at zero.  Over all nonzeros this is the mode-d MTTKRP
 *   X_(d) (Khatri-Rao product of the other factors) of Sec. 2.1 Eq. 1.
 * The sampled CP model (Sec. 2.1, CPD) at a nonzero is
 *     m = sum_r prod_n Y_n(i_n, r).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_F32 = 0, ORC_BF16 = 1, ORC_F16 = 2, ORC_F64 = 3 };

/* exact widening of one stored factor entry to double */
static double widen(const void* base, int dtype, int64_t i) {
    if (dtype == ORC_F32) return (double)((const float*)base)[i];
    if (dtype == ORC_F64) return ((const double*)base)[i];
    uint16_t h = ((const uint16_t*)base)[i];
    if (dtype == ORC_BF16) {
        /* bfloat16 is the upper half of an IEEE binary32 */
        uint32_t b = (uint32_t)h << 16;
        float f;
        memcpy(&f, &b, 4);
        return (double)f;
    }
    /* IEEE binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits */
    int sign = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0)
        v = (double)m * (1.0 / 16777216.0); /* subnormal: m * 2^-24 */
    else if (e == 31)
        v = m ? (0.0 / 0.0) : (1.0 / 0.0);
    else {
        v = (double)(1024 + m);
        int p = e - 25; /* (1024 + m) * 2^(e - 15 - 10) */
        while (p > 0) { v *= 2.0; --p; }
        while (p < 0) { v *= 0.5; ++p; }
    }
    return sign ? -v : v;
}

static int check(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int R) {
    if (nnz < 0 || nmodes < 1 || R < 1) return -1;
    for (int n = 0; n < nmodes; ++n)
        if (dims[n] < 1) return -1;
    for (int64_t k = 0; k < nnz; ++k)
        for (int n = 0; n < nmodes; ++n)
            if (idx[k * nmodes + n] < 0 || idx[k * nmodes + n] >= dims[n]) return -2;
    return 0;
}

/*
 * Mode-`mode` MTTKRP.  idx: [nnz][nmodes] 0-based; vals: fp32 (vals32) or
 * fp64 (vals64; used when vals32 is NULL); factors[n]: [dims[n]][R] row-major
 * in `dtype` (factors[mode] is not read); out: [dims[mode]][R] fp64,
 * overwritten.  Returns 0, -1 (bad argument) or -2 (index out of range).
 */
int oracle_mttkrp(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, const float* vals32,
                  const double* vals64, const void* const* factors, int dtype, int R, int mode, double* out) {
    int rc = check(nnz, nmodes, dims, idx, R);
    if (rc) return rc;
    if (mode < 0 || mode >= nmodes) return -1;
    memset(out, 0, sizeof(double) * (size_t)dims[mode] * (size_t)R);
    double* ell = (double*)malloc(sizeof(double) * (size_t)R);
    if (!ell) return -1;
    for (int64_t k = 0; k < nnz; ++k) {
        const int32_t* c = idx + k * nmodes;
        double v = vals32 ? (double)vals32[k] : vals64[k];
        for (int r = 0; r < R; ++r) ell[r] = v; /* l(r) starts at the nonzero's value */
        for (int w = 0; w < nmodes; ++w) {
            if (w == mode) continue;
            for (int r = 0; r < R; ++r) ell[r] *= widen(factors[w], dtype, (int64_t)c[w] * R + r);
        }
        double* row = out + (int64_t)c[mode] * R;
        for (int r = 0; r < R; ++r) row[r] += ell[r];
    }
    free(ell);
    return 0;
}

/*
 * The same sum restricted to a chosen set of output rows (values fp32 in vals32, or fp64 in
 * vals64 when vals32 is NULL): rows[0..nrows) is
 * a strictly increasing list of mode-`mode` indices and out is [nrows][R].
 * A bitmap screens the nonzeros and a binary search finds the row's slot,
 * so a full-size tensor can be checked on a sample of its output rows.
 */
int oracle_mttkrp_rows(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, const float* vals32,
                       const double* vals64, const void* const* factors, int dtype, int R, int mode, int64_t nrows,
                       const int64_t* rows, double* out) {
    if (nnz < 0 || nmodes < 1 || R < 1 || mode < 0 || mode >= nmodes || nrows < 0) return -1;
    for (int64_t j = 0; j < nrows; ++j)
        if (rows[j] < 0 || rows[j] >= dims[mode] || (j && rows[j] <= rows[j - 1])) return -1;
    memset(out, 0, sizeof(double) * (size_t)nrows * (size_t)R);
    int64_t I = dims[mode];
    uint8_t* bits = (uint8_t*)calloc((size_t)(I / 8 + 1), 1);
    double* ell = (double*)malloc(sizeof(double) * (size_t)R);
    if (!bits || !ell) { free(bits); free(ell); return -1; }
    for (int64_t j = 0; j < nrows; ++j) bits[rows[j] >> 3] |= (uint8_t)(1u << (rows[j] & 7));
    for (int64_t k = 0; k < nnz; ++k) {
        const int32_t* c = idx + k * nmodes;
        int64_t i = c[mode];
        if (i < 0 || i >= I) { free(bits); free(ell); return -2; }
        if (!(bits[i >> 3] & (1u << (i & 7)))) continue;
        int64_t lo = 0, hi = nrows - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (rows[mid] < i) lo = mid + 1; else hi = mid;
        }
        double v = vals32 ? (double)vals32[k] : vals64[k];
        for (int r = 0; r < R; ++r) ell[r] = v;
        for (int w = 0; w < nmodes; ++w) {
            if (w == mode) continue;
            if (c[w] < 0 || c[w] >= dims[w]) { free(bits); free(ell); return -2; }
            for (int r = 0; r < R; ++r) ell[r] *= widen(factors[w], dtype, (int64_t)c[w] * R + r);
        }
        for (int r = 0; r < R; ++r) out[lo * R + r] += ell[r];
    }
    free(bits);
    free(ell);
    return 0;
}

/* Sampled CP model m[k] = sum_r prod_n Y_n(i_n(k), r), fp64. */
int oracle_cp_sample(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, const void* const* factors,
                     int dtype, int R, double* m) {
    int rc = check(nnz, nmodes, dims, idx, R);
    if (rc) return rc;
    for (int64_t k = 0; k < nnz; ++k) {
        const int32_t* c = idx + k * nmodes;
        double s = 0.0;
        for (int r = 0; r < R; ++r) {
            double p = 1.0;
            for (int n = 0; n < nmodes; ++n) p *= widen(factors[n], dtype, (int64_t)c[n] * R + r);
            s += p;
        }
        m[k] = s;
    }
    return 0;
}

/*
 * Gradient of L = sum_k phi(m_k) with respect to every factor, given the
 * per-nonzero derivative g_k = dL/dm_k (fp64): dL/dY_n = MTTKRP_n with the
 * nonzero values replaced by g.  grads[n] is [dims[n]][R] fp64, overwritten.
 */
int oracle_cp_grad(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, const double* g,
                   const void* const* factors, int dtype, int R, double* const* grads) {
    for (int n = 0; n < nmodes; ++n) {
        int rc = oracle_mttkrp(nnz, nmodes, dims, idx, NULL, g, factors, dtype, R, n, grads[n]);
        if (rc) return rc;
    }
    return 0;
}
