// kernels.cuh — sm_103a kernels of the sparse MTTKRP library (templates).
//
// MTTKRP (paper Sec. 3 elementwise computation, Alg. 2), restated for one
// GB300:
//  * A "worker" is LPN consecutive lanes of a warp; lane q of a worker owns
//    ranks q*VEC .. q*VEC+VEC-1 of every factor row, so one factor row is one
//    coalesced LPN*VEC-element access (Alg. 2 gives one thread per rank of a
//    nonzero; here VEC ranks per thread for 128-bit accesses).
//  * Workers pull segments from a device-wide ticket counter (the single-GPU
//    form of the paper's idle-SM-takes-the-next-partition assignment,
//    Sec. 4.2) inside a persistent grid.
//  * A segment is a merge-path slice of the mode-ordered copy (rows +
//    nonzeros <= items).  The worker streams the segment's coordinate and
//    value arrays with 128-bit loads (4 nonzeros per lane, L2 evict-first),
//    broadcasts each nonzero inside the worker with one shuffle per array,
//    gathers the N-1 input factor rows, and accumulates the row in registers
//    while the output index is unchanged.  A completed row is stored once;
//    only rows that straddle a segment boundary leave a partial in the split
//    buffer, combined afterwards in a fixed order in fp64 (no atomics, so the
//    result does not depend on scheduling).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "amped_internal.h"

namespace amped {

// ------------------------------------------------------------------ loads
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 4 consecutive 32-bit stream words, read once: no L1 allocation, evict-first in L2
__device__ __forceinline__ int4 ld_stream_i4(const int32_t* ptr, uint64_t pol) {
    int4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(ptr), "l"(pol));
    return r;
}
__device__ __forceinline__ float4 ld_stream_f4(const float* ptr, uint64_t pol) {
    float4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(ptr), "l"(pol));
    return r;
}

// component c of a vector; with c known after unrolling this folds to a register move
__device__ __forceinline__ int comp_rt(const int4& v, int c) {
    return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}
__device__ __forceinline__ float comp_rt(const float4& v, int c) {
    return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}

// Factor-row gather: VEC consecutive entries of type T widened to fp32.
template <typename T, int VEC>
struct Row;

template <>
struct Row<float, 4> {
    static __device__ __forceinline__ void load(const void* base, int64_t off, float (&x)[4]) {
        const float* p = static_cast<const float*>(base) + off;
        asm("ld.global.nc.L1::evict_last.v4.f32 {%0,%1,%2,%3}, [%4];"
            : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3])
            : "l"(p));
    }
};
template <>
struct Row<float, 1> {
    static __device__ __forceinline__ void load(const void* base, int64_t off, float (&x)[1]) {
        x[0] = __ldg(static_cast<const float*>(base) + off);
    }
};
template <>
struct Row<__nv_bfloat16, 8> {
    static __device__ __forceinline__ void load(const void* base, int64_t off, float (&x)[8]) {
        const __nv_bfloat16* p = static_cast<const __nv_bfloat16*>(base) + off;
        uint32_t w[4];
        asm("ld.global.nc.L1::evict_last.v4.b32 {%0,%1,%2,%3}, [%4];"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
            : "l"(p));
#pragma unroll
        for (int i = 0; i < 4; ++i) {  // bf16 is the high half of an fp32
            x[2 * i] = __uint_as_float(w[i] << 16);
            x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
};
template <>
struct Row<__nv_bfloat16, 1> {
    static __device__ __forceinline__ void load(const void* base, int64_t off, float (&x)[1]) {
        const unsigned short* p = static_cast<const unsigned short*>(base) + off;
        x[0] = __uint_as_float((uint32_t)__ldg(p) << 16);
    }
};
template <>
struct Row<__half, 8> {
    static __device__ __forceinline__ void load(const void* base, int64_t off, float (&x)[8]) {
        const __half* p = static_cast<const __half*>(base) + off;
        uint32_t w[4];
        asm("ld.global.nc.L1::evict_last.v4.b32 {%0,%1,%2,%3}, [%4];"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
            : "l"(p));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h = *reinterpret_cast<__half2*>(&w[i]);
            float2 f = __half22float2(h);
            x[2 * i] = f.x;
            x[2 * i + 1] = f.y;
        }
    }
};
template <>
struct Row<__half, 1> {
    static __device__ __forceinline__ void load(const void* base, int64_t off, float (&x)[1]) {
        x[0] = __half2float(__ldg(static_cast<const __half*>(base) + off));
    }
};

template <int VEC>
__device__ __forceinline__ void store_row(float* dst, const float (&a)[VEC], bool streaming) {
    if constexpr (VEC % 4 == 0) {
#pragma unroll
        for (int i = 0; i < VEC; i += 4) {
            float4 v = make_float4(a[i], a[i + 1], a[i + 2], a[i + 3]);
            if (streaming)
                __stcs(reinterpret_cast<float4*>(dst + i), v);
            else
                *reinterpret_cast<float4*>(dst + i) = v;
        }
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) dst[i] = a[i];
    }
}

// ------------------------------------------------------------------ MTTKRP
// Steps staged per chunk: all gathers of a chunk are issued before any use.
template <int VEC>
struct Chunk {
    static constexpr int value = VEC >= 8 ? 4 : 8;
};

template <int NIN>
struct StreamBatch {
    int4 idx[NIN];
    float4 val;
};

template <int NIN>
__device__ __forceinline__ void load_batch(const MttkrpParams& p, int kl, uint64_t pol, StreamBatch<NIN>& b) {
#pragma unroll
    for (int n = 0; n < NIN; ++n) b.idx[n] = ld_stream_i4(p.idx[n] + kl, pol);
    if (p.perm == nullptr) {
        b.val = ld_stream_f4(p.val + kl, pol);
    } else {  // gradient path: values live in caller order
        const int4 pc = ld_stream_i4(p.perm + kl, pol);
        const int cap = p.nnz > 0 ? p.nnz - 1 : 0;  // slack entries of perm are clamped
        b.val.x = __ldg(p.gval + min(max(pc.x, 0), cap));
        b.val.y = __ldg(p.gval + min(max(pc.y, 0), cap));
        b.val.z = __ldg(p.gval + min(max(pc.z, 0), cap));
        b.val.w = __ldg(p.gval + min(max(pc.w, 0), cap));
    }
}

template <typename T, int VEC, int LPN, int NIN>
__device__ __forceinline__ void mttkrp_segment(const MttkrpParams& p, int s, int q, unsigned wmask, bool active,
                                               uint64_t pol) {
    static_assert(LPN >= 2, "the rowptr window needs at least two lanes");
    constexpr int NB = 4 * LPN;  // nonzeros per stream batch of a worker
    constexpr int CH = Chunk<VEC>::value < NB ? Chunk<VEC>::value : NB;
    const int R = p.R;
    const int row_s = __ldg(p.seg_row + s), nz_s = __ldg(p.seg_nz + s);
    const int row_e = __ldg(p.seg_row + s + 1), nz_e = __ldg(p.seg_nz + s + 1);

    // rowptr window: lane q holds rowptr[rwb + 4q .. rwb + 4q + 3]
    int rwb = row_s & ~3;
    int4 rw = __ldg(reinterpret_cast<const int4*>(p.rowptr + rwb) + q);
    auto rowptr_at = [&](int i) -> int {
        const int o = i - rwb;
        return __shfl_sync(wmask, comp_rt(rw, o & 3), o >> 2, LPN);
    };
    auto ensure_window = [&](int i) {  // make rows i and i+1 addressable
        if (i + 1 - rwb >= 4 * LPN) {
            rwb = i & ~3;
            rw = __ldg(reinterpret_cast<const int4*>(p.rowptr + rwb) + q);
        }
    };

    const bool cont = rowptr_at(row_s) < nz_s;  // the first row began in an earlier segment
    int i = row_s;
    int rend;  // end of row i's nonzeros inside this segment
    if (i < row_e) {
        ensure_window(i);
        rend = rowptr_at(i + 1);
    } else {
        rend = nz_e;
    }
    bool touched = false;  // row i received a nonzero in this segment

    float acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = 0.f;

    const int64_t rq = (int64_t)q * VEC;
    auto flush = [&](int row) {
        if (active) {
            float* dst;
            bool streaming = false;
            if (row == row_s && cont) {
                dst = p.part + ((int64_t)s * 2) * R + rq;  // head partial of a split row
            } else if (row < row_e) {
                dst = p.out + (int64_t)row * R + rq;  // complete row: written exactly once
                streaming = true;
            } else {
                dst = p.part + ((int64_t)s * 2 + 1) * R + rq;  // tail partial of a split row
            }
            store_row<VEC>(dst, acc, streaming);
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
        touched = false;
    };
    auto advance = [&]() {  // close row i, move to row i+1
        flush(i);
        ++i;
        if (i < row_e) {
            ensure_window(i);
            rend = rowptr_at(i + 1);
        } else {
            rend = nz_e;
        }
    };

    int kb = nz_s & ~3;
    StreamBatch<NIN> cur, nxt;
    if (kb < nz_e) load_batch<NIN>(p, kb + 4 * q, pol, cur);
    for (; kb < nz_e; kb += NB) {
        if (kb + NB < nz_e) load_batch<NIN>(p, kb + NB + 4 * q, pol, nxt);  // prefetch
#pragma unroll 1
        for (int j0 = 0; j0 < NB; j0 += CH) {
            if (kb + j0 >= nz_e) break;
            float t[CH][VEC];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int k = kb + j0 + u;
                const int src = (j0 + u) >> 2;  // lane holding nonzero j0+u; component u&3
                int c[NIN];
#pragma unroll
                for (int n = 0; n < NIN; ++n) c[n] = __shfl_sync(wmask, comp_rt(cur.idx[n], u & 3), src, LPN);
                const float v = __shfl_sync(wmask, comp_rt(cur.val, u & 3), src, LPN);
                const bool valid = active && k >= nz_s && k < nz_e;
#pragma unroll
                for (int e = 0; e < VEC; ++e) t[u][e] = valid ? v : 0.f;
                if (valid) {
#pragma unroll
                    for (int n = 0; n < NIN; ++n) {
                        float x[VEC];
                        Row<T, VEC>::load(p.fac[n], (int64_t)c[n] * R + rq, x);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) t[u][e] *= x[e];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int k = kb + j0 + u;
                if (k < nz_s || k >= nz_e) continue;
                while (k >= rend) advance();
#pragma unroll
                for (int e = 0; e < VEC; ++e) acc[e] += t[u][e];
                touched = true;
            }
        }
        cur = nxt;
    }
    // close the rows that end in this segment, then the last row if it continues
    while (i < row_e) advance();
    if (i < p.I && touched) flush(i);
}

template <typename T, int VEC, int LPN, int NIN>
__global__ void __launch_bounds__(256) mttkrp_kernel(const MttkrpParams p) {
    const int lane = threadIdx.x & 31;
    const int q = lane % LPN;
    const unsigned wmask = (LPN == 32 ? 0xffffffffu : ((1u << LPN) - 1u)) << (lane - q);
    const bool active = q * VEC < p.R;
    const uint64_t pol = policy_evict_first();
    int s = 0;
    if (q == 0) s = atomicAdd(p.queue, 1);
    s = __shfl_sync(wmask, s, 0, LPN);
    while (s < p.S) {
        int nxt = 0;
        if (q == 0) nxt = atomicAdd(p.queue, 1);  // next ticket, latency hidden by this segment
        mttkrp_segment<T, VEC, LPN, NIN>(p, s, q, wmask, active, pol);
        s = __shfl_sync(wmask, nxt, 0, LPN);
    }
}

// ------------------------------------------------------------------ sampled CP model
// m_k = sum_r prod_n A_n(i_n(k), r) for every nonzero k in caller order (the
// CP model of Sec. 2.1 evaluated at the coordinates).  Same worker layout as
// the MTTKRP kernel; the rank sum is a shuffle reduction inside the worker and
// each lane stores the results of its 4 stream positions as one float4.
template <typename T, int VEC, int LPN, int NM>
__global__ void __launch_bounds__(256) sample_kernel(const SampleParams p) {
    constexpr int NB = 4 * LPN;
    constexpr int CH = Chunk<VEC>::value < NB ? Chunk<VEC>::value : NB;
    const int lane = threadIdx.x & 31;
    const int q = lane % LPN;
    const unsigned wmask = (LPN == 32 ? 0xffffffffu : ((1u << LPN) - 1u)) << (lane - q);
    const bool active = q * VEC < p.R;
    const uint64_t pol = policy_evict_first();
    const int64_t rq = (int64_t)q * VEC;
    const int worker = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LPN);
    const int nworkers = (int)((gridDim.x * (int64_t)blockDim.x) / LPN);
    const int nbatch = (p.nnz + NB - 1) / NB;
    for (int b = worker; b < nbatch; b += nworkers) {
        const int kb = b * NB, kl = kb + 4 * q;
        int4 bi[NM];
#pragma unroll
        for (int n = 0; n < NM; ++n) bi[n] = ld_stream_i4(p.idx[n] + kl, pol);
        float res[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int j0 = 0; j0 < NB; j0 += CH) {
            if (kb + j0 >= p.nnz) break;
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int j = j0 + u;
                float prod[VEC];
#pragma unroll
                for (int e = 0; e < VEC; ++e) prod[e] = 1.f;
#pragma unroll
                for (int n = 0; n < NM; ++n) {
                    const int c = __shfl_sync(wmask, comp_rt(bi[n], u & 3), j >> 2, LPN);
                    float x[VEC];
                    if (active) {
                        Row<T, VEC>::load(p.fac[n], (int64_t)c * p.R + rq, x);
                    } else {
#pragma unroll
                        for (int e = 0; e < VEC; ++e) x[e] = 0.f;
                    }
#pragma unroll
                    for (int e = 0; e < VEC; ++e) prod[e] *= x[e];
                }
                float sum = 0.f;
#pragma unroll
                for (int e = 0; e < VEC; ++e) sum += prod[e];
#pragma unroll
                for (int o = LPN / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(wmask, sum, o, LPN);
                if (q == (j >> 2)) res[u & 3] = sum;
            }
        }
        if (kl + 3 < p.nnz) {
            __stcs(reinterpret_cast<float4*>(p.m + kl), make_float4(res[0], res[1], res[2], res[3]));
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (kl + e < p.nnz) p.m[kl + e] = res[e];
        }
    }
}

}  // namespace amped
