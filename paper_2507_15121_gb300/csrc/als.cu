// als.cu — the dense steps of a CP-ALS sweep around the MTTKRP kernel.
//
// CP decomposition by alternating least squares (Sec. 2.1: ALS performs the
// mode-wise MTTKRPs of Eq. 1 in turn, iteratively).  After the mode-d MTTKRP
// M = X_(d) (Khatri-Rao of the other factors) the factor becomes the
// least-squares solution A_d = M V^-1, V the Hadamard product of the other
// factors' Gram matrices.  Per mode the library runs:
//
//   solve_kernel   one block, fp64: V = Hadamard of the other Grams,
//                  Cholesky V = L L^T, W = V^-1 (written as fp32)
//   apply_kernel   A_d = M W stored (fp32, 4x4 register tiles, packed f32x2
//                  FMA); the same pass accumulates the Gram of the stored
//                  A_d and ip_r = sum_i M(i,r) A_d(i,r)
//   finish_kernel  one block: commits the new Gram; the fit when asked (after a
//                  sweep's last mode, or after a single update)
//   gram_kernel    A^T A of the starting factors (first sweep only)
//   normalize      on request: unit-norm columns, lambda = product of the norms
//
// The factors are not normalised between modes.  Least-squares updates are
// covariant under column scaling (scaling a column of one factor scales the
// matching column of the next update inversely), so the sequence of models
// [[A_0, ..., A_{N-1}]] equals that of the per-step normalised algorithm; the
// Gram of every factor is the exact Gram of its stored values, so V stays
// consistent with what the MTTKRP reads.  The fit is that of the stored model:
//   <X, X^>  = sum_r ip_r                      (MTTKRP identity, last mode)
//   ||X^||^2 = sum_{r,s} prod_n G_n(r,s)
// Neither is derived from a quadratic form in V^-1, which cancels
// catastrophically when V is ill-conditioned (as it is for the small modes of
// power-law tensors).  Sums: fp32 over a tile, compensated (Kahan) fp32
// across tiles, fp64 across blocks.  Ranks up to kAlsMaxRank.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "amped_internal.h"

namespace amped {
namespace {

constexpr int kAlsMaxRank = 64;

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float lo2(unsigned long long v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi2(unsigned long long v) { return __uint_as_float((uint32_t)(v >> 32)); }
// (a.lo * b.lo + c.lo, a.hi * b.hi + c.hi), each rounded once
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Upper-triangle 4x4 tile k of an NT x NT tile grid, row-major: (ta, tb), ta <= tb.
__device__ __forceinline__ void tri_tile(int k, int NT, int& ta, int& tb) {
    ta = 0;
    while (k >= NT - ta) {
        k -= NT - ta;
        ++ta;
    }
    tb = ta + k;
}

// Copies rows [base, base + nr) of the row-major [rows][R] matrix A into
// tile[row * LD + col] (cols < R only; the padding columns are left alone).
__device__ __forceinline__ void stage_rows(const float* __restrict__ A, int64_t base, int nr, int R, float* tile,
                                           int LD) {
    const float* src = A + base * R;
    const int n = nr * R;
    if ((R & 3) == 0) {
        for (int e = threadIdx.x * 4; e < n; e += blockDim.x * 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(src + e));
            const int row = e / R, col = e - row * R;
            *reinterpret_cast<float4*>(tile + row * LD + col) = v;
        }
    } else {
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int row = e / R;
            tile[row * LD + e - row * R] = __ldg(src + e);
        }
    }
}

// Per-thread share of an R x R Gram accumulated over staged row tiles: the 4x4
// tiles on and above the diagonal, TILES threads per group, GROUPS groups per
// block taking every GROUPS-th row.  Sums: fp32 over one tile's rows, Kahan
// fp32 across tiles, fp64 across groups (fixed order) and blocks (atomics).
template <int RP>
struct GramAcc {
    static constexpr int NT = RP / 4;
    static constexpr int TILES = NT * (NT + 1) / 2;
    static constexpr int GROUPS = 256 / TILES;
    static_assert(GROUPS >= 1, "rank too large for one block");
    int g, k, ta, tb;
    float s[16], c[16];

    __device__ __forceinline__ void init() {
        g = threadIdx.x / TILES;
        k = threadIdx.x - g * TILES;
        tri_tile(k, NT, ta, tb);
#pragma unroll
        for (int j = 0; j < 16; ++j) s[j] = c[j] = 0.f;
    }
    // rows [0, nr) of tile (row stride LD floats, padding columns zero)
    __device__ __forceinline__ void add(const float* tile, int nr, int LD) {
        if (g >= GROUPS) return;
        unsigned long long acc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = 0ull;
        for (int i = g; i < nr; i += GROUPS) {
            const float4 a = *reinterpret_cast<const float4*>(tile + i * LD + ta * 4);
            const float4 b = *reinterpret_cast<const float4*>(tile + i * LD + tb * 4);
            const unsigned long long b01 = pack2(b.x, b.y), b23 = pack2(b.z, b.w);
            const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const unsigned long long aa = pack2(av[x], av[x]);
                acc[2 * x] = ffma2(aa, b01, acc[2 * x]);
                acc[2 * x + 1] = ffma2(aa, b23, acc[2 * x + 1]);
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {  // Kahan: s carries the sum, c its lost low part
            const float part[2] = {lo2(acc[j]), hi2(acc[j])};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = 2 * j + h;
                const float y = part[h] - c[q];
                const float t = s[q] + y;
                c[q] = (t - s[q]) - y;
                s[q] = t;
            }
        }
    }
    // G[a][b] += this block's sums (every thread of the block calls this)
    __device__ __forceinline__ void flush(double* red, double* __restrict__ G, int R) {
        __syncthreads();
        for (int gg = 0; gg < GROUPS; ++gg) {  // groups summed in a fixed order
            if (g == gg)
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    red[k * 16 + j] = (gg ? red[k * 16 + j] : 0.0) + ((double)s[j] - (double)c[j]);
            __syncthreads();
        }
        for (int e = threadIdx.x; e < TILES * 16; e += blockDim.x) {
            int ua, ub;
            tri_tile(e / 16, NT, ua, ub);
            const int a = ua * 4 + (e & 15) / 4, b = ub * 4 + (e & 3);
            if (a < R && b < R) {
                const double v = red[e];
                atomicAdd(G + a * R + b, v);
                if (ua != ub) atomicAdd(G + b * R + a, v);
            }
        }
    }
};

// Rows per tile of gram_kernel (static shared memory stays under 48 KB).
template <int RP>
struct GramTile {
    static constexpr int ROWS = RP == 64 ? 96 : 256;
    static constexpr int LD = RP + 4;
    static constexpr int V4 = ROWS * RP / 4 / 256;  // float4 per thread when R == RP
};

// G += A^T A for a row-major [rows][R] fp32 matrix.  RP = R rounded up to 8,
// 16, 32 or 64.  When R is a multiple of 4 the next tile is loaded into
// registers while the current one is summed.
template <int RP>
__global__ void __launch_bounds__(256, 2) gram_kernel(const float* __restrict__ A, int64_t rows, int R,
                                                      double* __restrict__ G) {
    using TL = GramTile<RP>;
    constexpr int LD = TL::LD;
    __shared__ __align__(16) float tile[TL::ROWS * LD];
    __shared__ double red[GramAcc<RP>::TILES * 16];
    GramAcc<RP> acc;
    acc.init();
    for (int e = threadIdx.x; e < TL::ROWS * LD; e += blockDim.x) tile[e] = 0.f;  // padding columns stay zero
    const int64_t step = (int64_t)gridDim.x * TL::ROWS;
    const bool vec = (R & 3) == 0;
    float4 nxt[TL::V4];
    auto fetch = [&](int64_t base) {
        const int n = (int)((rows - base < TL::ROWS ? rows - base : TL::ROWS) * R);
        const float* src = A + base * R;
#pragma unroll
        for (int j = 0; j < TL::V4; ++j) {
            const int e = (threadIdx.x + j * 256) * 4;
            if (e < n) nxt[j] = __ldg(reinterpret_cast<const float4*>(src + e));
        }
    };
    int64_t base = (int64_t)blockIdx.x * TL::ROWS;
    if (vec && base < rows) fetch(base);
    for (; base < rows; base += step) {
        const int nr = (int)(rows - base < TL::ROWS ? rows - base : TL::ROWS);
        __syncthreads();
        if (vec) {
#pragma unroll
            for (int j = 0; j < TL::V4; ++j) {
                const int e = (threadIdx.x + j * 256) * 4;
                if (e < nr * R) {
                    const int row = e / R;
                    *reinterpret_cast<float4*>(tile + row * LD + e - row * R) = nxt[j];
                }
            }
            if (base + step < rows) fetch(base + step);
        } else {
            stage_rows(A, base, nr, R, tile, LD);
        }
        __syncthreads();
        acc.add(tile, nr, LD);
    }
    acc.flush(red, G, R);
}

// One block of 256 threads; dynamic shared memory of 2 R (R+1) + 2 R doubles.
// V = Hadamard of the other modes' Grams; Cholesky V = L L^T (right-looking);
// Z = L^-1 (right-looking substitution); Y = V^-1 = Z^T Z, written as fp32 W.
// Every step spreads its entries over the block; the only divisions are the
// R reciprocals of the pivots.
__global__ void __launch_bounds__(256) solve_kernel(AlsParams p) {
    extern __shared__ double smem[];
    const int R = p.R, LD = R + 1, tid = threadIdx.x, nth = blockDim.x;
    double* V = smem;            // V, then L (lower)
    double* Z = V + R * LD;      // L^-1 (lower)
    double* dinv = Z + R * LD;   // [R] 1 / L_jj
    double* dg = dinv + R;       // [R] diagonal of V before the factorisation
    __shared__ int bad;
    if (tid == 0) bad = 0;
    for (int e = tid; e < R * R; e += nth) {
        const int a = e / R, b = e - a * R;
        double v = 1.0;
        for (int n = 0; n < p.N; ++n)
            if (n != p.mode) v *= p.grams[(int64_t)n * R * R + e];
        V[a * LD + b] = v;
        Z[a * LD + b] = a == b ? 1.0 : 0.0;
        if (a == b) dg[a] = v;
    }
    __syncthreads();
    // Cholesky: a pivot below 1e-12 of its original diagonal entry (or not
    // positive) marks V as singular and stops the update of this mode.
    for (int j = 0; j < R; ++j) {
        if (tid == 0) {
            double d = V[j * LD + j];
            if (!(d > 1e-12 * dg[j])) {
                if (!bad) bad = j + 1;
                d = dg[j] > 0.0 ? dg[j] : 1.0;  // keeps the arithmetic finite; the result is discarded
            }
            d = sqrt(d);
            V[j * LD + j] = d;
            dinv[j] = 1.0 / d;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < R; i += nth) V[i * LD + j] *= dinv[j];
        __syncthreads();
        const int n = R - j - 1;  // trailing block: rows/cols j+1 .. R-1, lower triangle
        for (int e = tid; e < n * n; e += nth) {
            const int i = j + 1 + e / n, k = j + 1 + e % n;
            if (k <= i) V[i * LD + k] -= V[i * LD + j] * V[k * LD + j];
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) *p.info = bad;
        return;
    }
    // Z = L^-1, one column of L at a time: scale row q, then eliminate below it
    for (int q = 0; q < R; ++q) {
        for (int c = tid; c <= q; c += nth) Z[q * LD + c] *= dinv[q];
        __syncthreads();
        const int n = R - q - 1, w = q + 1;
        for (int e = tid; e < n * w; e += nth) {
            const int i = q + 1 + e / w, c = e % w;
            Z[i * LD + c] -= V[i * LD + q] * Z[q * LD + c];
        }
        __syncthreads();
    }
    // W = Z^T Z (Z lower triangular: Y_ab = sum_{q >= max(a,b)} Z_qa Z_qb)
    for (int e = tid; e < R * R; e += nth) {
        const int a = e / R, b = e - a * R;
        const int lo = a > b ? a : b;
        double sum = 0.0;
        for (int q = lo; q < R; ++q) sum += Z[q * LD + a] * Z[q * LD + b];
        p.w[e] = (float)sum;
    }
    if (tid == 0) *p.info = 0;
}

// Asynchronous global -> shared copies (no registers in flight), in groups.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shape of apply_kernel for padded rank RP: CT column groups of 4, RG row
// groups, 4 rows per thread (rows rg, rg + RG, rg + 2 RG, rg + 3 RG of a tile,
// so the rows a warp reads together are consecutive and hit different banks).
template <int RP>
struct ApplyShape {
    static constexpr int CT = RP / 4;
    static constexpr int RG = 256 / CT;
    static constexpr int ROWS = 4 * RG;  // rows per tile
    static constexpr int LD = RP + 4;    // M tile row stride (floats)
    // two M tiles, the transposed A tile [RP][ROWS], W^T [RP][RP]
    static constexpr size_t smem_bytes() {
        return sizeof(float) * ((size_t)2 * ROWS * LD + (size_t)RP * ROWS + (size_t)RP * RP);
    }
};

// Row-major [n][RP] arrays whose row c has its 4-float chunks XOR-swizzled by
// the column group c / 4: the eight column groups of a warp that read the same
// k (or the same rows) land in eight different bank groups.
__device__ __forceinline__ int swz(int c, int k, int stride) { return c * stride + (k ^ (((c >> 2) & 7) << 2)); }

// Copies rows [base, base + nr) of M into a tile (row stride LD) without
// registers; columns >= R and rows >= nr are left as they are.
__device__ __forceinline__ void stage_async(const float* __restrict__ M, int64_t base, int nr, int R, float* tile,
                                            int LD) {
    const float* src = M + base * R;
    if ((R & 3) == 0) {
        const int q = R / 4, n = nr * q;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int row = e / q, c = (e - row * q) * 4;
            cp_async16(tile + row * LD + c, src + (int64_t)row * R + c);
        }
    } else {
        const int n = nr * R;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int row = e / R;
            cp_async4(tile + row * LD + e - row * R, src + e);
        }
    }
    cp_async_commit();
}

// A = M W for the MTTKRP output M (row-major [rows][R]) and the solve's
// W = V^-1 (fp32), stored; in the same pass ga += A^T A (of the fp32 values
// stored) and ip[r] += sum_i M(i,r) A(i,r).  Does nothing when the solve
// reported a singular V.  RP = R rounded up to 8, 16, 32 or 64.  Tiles of M
// are double-buffered with cp.async.  The product uses packed f32x2 FMA with
// the operand pairs loaded as 64-bit words: (M[i][k], M[i][k+1]) x
// (W[k][c], W[k+1][c]), W^T in shared memory.  The Gram reads A^T from shared
// memory, four rows of two columns per pair of 128-bit loads.
template <int RP>
__global__ void __launch_bounds__(256, 2) apply_kernel(const float* __restrict__ M, int64_t rows, AlsParams p,
                                                       float* __restrict__ A) {
    using SH = ApplyShape<RP>;
    constexpr int CT = SH::CT, RG = SH::RG, ROWS = SH::ROWS, LD = SH::LD;
    constexpr int NT = RP / 4, TILES = NT * (NT + 1) / 2, GROUPS = 256 / TILES;
    static_assert(GROUPS >= 1 && TILES * 16 * 2 <= 2 * ROWS * LD, "Gram reduction must fit in the M tiles");
    extern __shared__ __align__(16) float dsm[];
    float* buf0 = dsm;
    float* buf1 = dsm + ROWS * LD;
    float* at = dsm + 2 * ROWS * LD;  // A^T [RP][ROWS], swizzled
    float* wt = at + RP * ROWS;       // W^T [RP][RP], swizzled
    __shared__ double colr[RP];
    if (*p.info) return;
    const int R = p.R;
    const int tid = threadIdx.x, ct = tid % CT, rg = tid / CT, c0 = ct * 4;
    const int64_t step = (int64_t)gridDim.x * ROWS;
    int64_t base = (int64_t)blockIdx.x * ROWS;
    // zero the tiles (padding columns and rows must stay finite zeros), then W^T
    for (int e = tid; e < 2 * ROWS * LD + RP * ROWS; e += blockDim.x) dsm[e] = 0.f;
    for (int e = tid; e < RP * RP; e += blockDim.x) {
        const int c = e / RP, k = e - c * RP;
        wt[swz(c, k, RP)] = (k < R && c < R) ? p.w[k * R + c] : 0.f;
    }
    for (int e = tid; e < RP; e += blockDim.x) colr[e] = 0.0;
    __syncthreads();
    if (base < rows) stage_async(M, base, (int)(rows - base < ROWS ? rows - base : ROWS), R, buf0, LD);
    // Gram share of this thread: the 4x4 tile (ta, tb), ta <= tb, of group g
    const int g = tid / TILES, kt = tid - g * TILES;
    int ta = 0, tb = 0;
    tri_tile(kt, NT, ta, tb);
    float gs[16], gc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) gs[j] = gc[j] = 0.f;
    float is[4] = {0.f, 0.f, 0.f, 0.f}, ic[4] = {0.f, 0.f, 0.f, 0.f};
    int cur = 0;
    for (; base < rows; base += step, cur ^= 1) {
        const int nr = (int)(rows - base < ROWS ? rows - base : ROWS);
        const float* tile = cur ? buf1 : buf0;
        __syncthreads();  // the other buffer's and the A^T tile's last readers are done
        if (base + step < rows) {
            const int64_t nb = base + step;
            stage_async(M, nb, (int)(rows - nb < ROWS ? rows - nb : ROWS), R, cur ? buf0 : buf1, LD);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        // ---- product: acc[i][q] = (sum over even k, sum over odd k) of M[row_i][k] W[k][c0+q]
        unsigned long long acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = 0ull;
#pragma unroll 1
        for (int k = 0; k < RP; k += 4) {
            ulonglong2 mv[4], wv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) mv[i] = *reinterpret_cast<const ulonglong2*>(tile + (rg + i * RG) * LD + k);
#pragma unroll
            for (int q = 0; q < 4; ++q) wv[q] = *reinterpret_cast<const ulonglong2*>(wt + swz(c0 + q, k, RP));
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] = ffma2(mv[i].x, wv[q].x, acc[i][q]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] = ffma2(mv[i].y, wv[q].y, acc[i][q]);
        }
        float av[4][4];
        float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int q = 0; q < 4; ++q) av[i][q] = lo2(acc[i][q]) + hi2(acc[i][q]);
            if (rg + i * RG < nr) {
                const float4 m = *reinterpret_cast<const float4*>(tile + (rg + i * RG) * LD + c0);
                part[0] = fmaf(m.x, av[i][0], part[0]);
                part[1] = fmaf(m.y, av[i][1], part[1]);
                part[2] = fmaf(m.z, av[i][2], part[2]);
                part[3] = fmaf(m.w, av[i][3], part[3]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // Kahan across tiles
            const float y = part[q] - ic[q];
            const float t = is[q] + y;
            ic[q] = (t - is[q]) - y;
            is[q] = t;
        }
        // ---- store A (global, row-major) and A^T (shared, for the Gram); rows >= nr are zeros in A^T
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = rg + i * RG;
            const bool ok = row < nr;
#pragma unroll
            for (int q = 0; q < 4; ++q) at[swz(c0 + q, row, ROWS)] = ok ? av[i][q] : 0.f;
            if (!ok) continue;
            float* dst = A + (base + row) * R;
            if ((R & 3) == 0) {
                if (c0 < R) *reinterpret_cast<float4*>(dst + c0) = make_float4(av[i][0], av[i][1], av[i][2], av[i][3]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c0 + q < R) dst[c0 + q] = av[i][q];
            }
        }
        __syncthreads();
        // ---- Gram over the tile's 4-row chunks: G[a][b] += sum_r A[r][a] A[r][b]
        if (g < GROUPS) {
            float ga[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) ga[j] = 0.f;
            const int nq = (nr + 3) / 4;
            for (int qd = g; qd < nq; qd += GROUPS) {
                float4 a[4], b[4];
#pragma unroll
                for (int x = 0; x < 4; ++x) a[x] = *reinterpret_cast<const float4*>(at + swz(ta * 4 + x, qd * 4, ROWS));
#pragma unroll
                for (int y = 0; y < 4; ++y) b[y] = *reinterpret_cast<const float4*>(at + swz(tb * 4 + y, qd * 4, ROWS));
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        float v = ga[x * 4 + y];
                        v = fmaf(a[x].x, b[y].x, v);
                        v = fmaf(a[x].y, b[y].y, v);
                        v = fmaf(a[x].z, b[y].z, v);
                        v = fmaf(a[x].w, b[y].w, v);
                        ga[x * 4 + y] = v;
                    }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float yv = ga[j] - gc[j];
                const float t = gs[j] + yv;
                gc[j] = (t - gs[j]) - yv;
                gs[j] = t;
            }
        }
    }
    // block reduction of the Gram (groups in a fixed order), reusing the M tiles
    double* red = reinterpret_cast<double*>(dsm);
    __syncthreads();
    for (int gg = 0; gg < GROUPS; ++gg) {
        if (g == gg)
#pragma unroll
            for (int j = 0; j < 16; ++j) red[kt * 16 + j] = (gg ? red[kt * 16 + j] : 0.0) + ((double)gs[j] - (double)gc[j]);
        __syncthreads();
    }
    for (int e = tid; e < TILES * 16; e += blockDim.x) {
        int ua, ub;
        tri_tile(e / 16, NT, ua, ub);
        const int a = ua * 4 + (e & 15) / 4, b = ub * 4 + (e & 3);
        if (a < R && b < R) {
            const double v = red[e];
            atomicAdd(p.ga + a * R + b, v);
            if (ua != ub) atomicAdd(p.ga + b * R + a, v);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (c0 + q < R) atomicAdd(&colr[c0 + q], (double)is[q] - (double)ic[q]);
    __syncthreads();
    for (int e = tid; e < R; e += blockDim.x) atomicAdd(p.ip + e, colr[e]);
}

// One block: when the update succeeded, grams[mode] = the new Gram; after the
// last mode, the fit terms of the stored model.  On a singular V the counters
// are bumped and the old Gram stays.
__global__ void __launch_bounds__(256) finish_kernel(AlsParams p) {
    const int R = p.R, tid = threadIdx.x;
    __shared__ double red[2][8];
    const int info = *p.info;
    if (info == 0) {
        double* gout = p.grams + (int64_t)p.mode * R * R;
        for (int e = tid; e < R * R; e += blockDim.x) gout[e] = p.ga[e];
    } else if (tid == 0) {
        p.stats[5] += 1.0;
        if (p.stats[6] == 0.0) p.stats[6] = (double)(p.mode + 1);
    }
    if (!p.last) return;
    if (info != 0) {
        if (tid == 0)
            for (int q = 0; q < 5; ++q) p.stats[q] = NAN;
        return;
    }
    __syncthreads();  // the committed Gram is read back below
    double xy = 0.0, yy = 0.0;
    for (int e = tid; e < R * R; e += blockDim.x) {
        const int a = e / R, b = e - a * R;
        double v = 1.0;
        for (int n = 0; n < p.N; ++n) v *= p.grams[(int64_t)n * R * R + e];
        yy += v;
        if (a == b) xy += p.ip[a];
    }
    const int warp = tid >> 5, lane = tid & 31;
    for (int o = 16; o > 0; o >>= 1) {
        xy += __shfl_xor_sync(0xffffffffu, xy, o);
        yy += __shfl_xor_sync(0xffffffffu, yy, o);
    }
    if (lane == 0) {
        red[0][warp] = xy;
        red[1][warp] = yy;
    }
    __syncthreads();
    if (tid == 0) {
        double xs = 0.0, ys = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            xs += red[0][q];
            ys += red[1][q];
        }
        const double xx = p.xnorm2;
        const double res = xx - 2.0 * xs + ys;
        const double res_c = res > 0.0 ? res : 0.0;
        p.stats[0] = xx > 0.0 ? 1.0 - sqrt(res_c) / sqrt(xx) : 0.0;
        p.stats[1] = res_c;
        p.stats[2] = xx;
        p.stats[3] = xs;
        p.stats[4] = ys;
    }
}

// A[:, r] /= ||A[:, r]|| with the norms from the diagonal of the factor's Gram
// (columns of zeros stay zero).
__global__ void __launch_bounds__(256) normalize_kernel(float* __restrict__ A, int64_t rows, int R,
                                                        const double* __restrict__ G) {
    __shared__ float inv[kAlsMaxRank];
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const double d = G[r * R + r];
        inv[r] = d > 0.0 ? (float)(1.0 / sqrt(d)) : 0.f;
    }
    __syncthreads();
    const int64_t n = rows * R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        A[e] *= inv[e % R];
}

// lambda_r = prod_n ||A_n[:, r]||; every Gram scaled to the unit-norm factors.
// Runs after the normalize_kernel launches (which read the old diagonals).
__global__ void __launch_bounds__(256) lambda_kernel(double* __restrict__ grams, int N, int R,
                                                     float* __restrict__ lambda) {
    __shared__ double nrm[AMPED_MAX_MODES * kAlsMaxRank];
    for (int e = threadIdx.x; e < N * R; e += blockDim.x) {
        const double d = grams[(int64_t)(e / R) * R * R + (e % R) * (R + 1)];
        nrm[e] = d > 0.0 ? sqrt(d) : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        double l = 1.0;
        for (int n = 0; n < N; ++n) l *= nrm[n * R + r];
        lambda[r] = (float)l;
    }
    for (int e = threadIdx.x; e < N * R * R; e += blockDim.x) {
        const int n = e / (R * R), a = (e / R) % R, b = e % R;
        const double d = nrm[n * R + a] * nrm[n * R + b];
        grams[e] = d > 0.0 ? grams[e] / d : 0.0;
    }
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 152;
    return sms;
}

int grid_for(int64_t units, int per_block, int blocks_per_sm) {
    const int64_t cap = (int64_t)sm_count() * (blocks_per_sm > 0 ? blocks_per_sm : 1);
    int64_t g = (units + per_block - 1) / per_block;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// Blocks of `kernel` (256 threads, `dyn` bytes of dynamic shared memory) resident on one SM.
template <class K>
int resident(K kernel, size_t dyn = 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 256, dyn) != cudaSuccess || n < 1) n = 1;
    return n;
}

int padded_rank(int R) { return R <= 8 ? 8 : R <= 16 ? 16 : R <= 32 ? 32 : 64; }

}  // namespace

int als_max_rank() { return kAlsMaxRank; }

int launch_gram(const float* A, int64_t rows, int R, double* G, void* stream, int* launched) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (R < 1 || R > kAlsMaxRank) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * R * R, st);
    if (e != cudaSuccess) return (int)e;
    if (rows <= 0) return 0;
#define AMPED_GRAM_CASE(RP)                                                                                \
    case RP:                                                                                               \
        gram_kernel<RP><<<grid_for(rows, GramTile<RP>::ROWS, resident(gram_kernel<RP>)), 256, 0, st>>>(A, rows, R, G); \
        break;
    switch (padded_rank(R)) {
        AMPED_GRAM_CASE(8)
        AMPED_GRAM_CASE(16)
        AMPED_GRAM_CASE(32)
        default: AMPED_GRAM_CASE(64)
    }
#undef AMPED_GRAM_CASE
    ++*launched;
    return (int)cudaGetLastError();
}

int launch_als_solve(const AlsParams& p, void* stream, int* launched) {
    if (p.R < 1 || p.R > kAlsMaxRank) return (int)cudaErrorInvalidValue;
    const size_t bytes = sizeof(double) * ((size_t)2 * p.R * (p.R + 1) + 2 * (size_t)p.R);
    const cudaError_t attr = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (attr != cudaSuccess) return (int)attr;
    solve_kernel<<<1, 256, bytes, static_cast<cudaStream_t>(stream)>>>(p);
    ++*launched;
    return (int)cudaGetLastError();
}

int launch_als_apply(const AlsParams& p, const float* M, int64_t rows, float* A, void* stream, int* launched) {
    if (p.R < 1 || p.R > kAlsMaxRank) return (int)cudaErrorInvalidValue;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int R = p.R;
    cudaError_t e = cudaMemsetAsync(p.ga, 0, sizeof(double) * ((size_t)R * R + R), st);  // ga, then ip
    if (e != cudaSuccess) return (int)e;
    if (rows > 0 && als_apply_tc_supported(R)) {
        // A = M W and ip on the tensor cores, then the Gram of the stored A (when the solve
        // failed the product does nothing and finish_kernel ignores the Gram)
        e = (cudaError_t)launch_als_apply_tc(p, M, rows, A, stream, launched);
        if (e != cudaSuccess) return (int)e;
        e = (cudaError_t)launch_gram(A, rows, R, p.ga, stream, launched);
        if (e != cudaSuccess) return (int)e;
    } else if (rows > 0) {
#define AMPED_APPLY_CASE(RP)                                                                                    \
    case RP: {                                                                                                 \
        const size_t bytes = ApplyShape<RP>::smem_bytes();                                                     \
        e = cudaFuncSetAttribute(apply_kernel<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);   \
        if (e != cudaSuccess) return (int)e;                                                                   \
        apply_kernel<RP><<<grid_for(rows, ApplyShape<RP>::ROWS, resident(apply_kernel<RP>, bytes)), 256, bytes, st>>>( \
            M, rows, p, A);                                                                                    \
        break;                                                                                                 \
    }
        switch (padded_rank(R)) {
            AMPED_APPLY_CASE(8)
            AMPED_APPLY_CASE(16)
            AMPED_APPLY_CASE(32)
            default: AMPED_APPLY_CASE(64)
        }
#undef AMPED_APPLY_CASE
        ++*launched;
    }
    finish_kernel<<<1, 256, 0, st>>>(p);
    ++*launched;
    return (int)cudaGetLastError();
}

int launch_als_normalize(float* const* factors, const int64_t* dims, int N, int R, double* grams, float* lambda,
                         void* stream, int* launched) {
    if (R < 1 || R > kAlsMaxRank || N < 1 || N > AMPED_MAX_MODES) return (int)cudaErrorInvalidValue;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int n = 0; n < N; ++n) {
        const int64_t elems = dims[n] * R;
        normalize_kernel<<<grid_for(elems, 256 * 8, 8), 256, 0, st>>>(factors[n], dims[n], R,
                                                                        grams + (size_t)n * R * R);
        ++*launched;
    }
    lambda_kernel<<<1, 256, 0, st>>>(grams, N, R, lambda);
    ++*launched;
    return (int)cudaGetLastError();
}

}  // namespace amped
