// kernels.cuh — sm_103a kernels of the sparse MTTKRP library (templates).
//
// MTTKRP (paper Sec. 3 elementwise computation, Alg. 2), restated for one
// GB300:
//  * A "lane group" is LPN consecutive lanes of a warp; lane q of a group owns
//    ranks q*VEC .. q*VEC+VEC-1 of every factor row, so one factor row is one
//    coalesced 256-bit load per lane (Alg. 2 gives one thread per rank of a
//    nonzero; here 8 fp32 or 16 16-bit ranks per lane).
//  * Warps pull segments from a device-wide ticket counter (the single-GPU
//    form of the paper's idle-SM-takes-the-next-partition assignment,
//    Sec. 4.2) inside a persistent grid.
//  * A segment is a merge-path slice of the mode-ordered copy (rows +
//    nonzeros <= items).  The warp streams the segment's coordinate and value
//    arrays with 128-bit evict-first loads and stages them as one record per
//    nonzero in shared memory.  A staged batch that lies inside one row takes
//    the factored path (fiber_batch: each group walks 16 consecutive nonzeros
//    and gathers the outer slots' rows only at run starts); other chunks take
//    the interleaved chunk path (group g takes every G-th nonzero).  The row
//    is accumulated in registers while the output index is unchanged and
//    stored once; only rows that straddle a segment boundary leave a partial
//    in the split buffer, combined afterwards in a fixed order in fp64 (no
//    atomics, so the result does not depend on scheduling).
//  * Rows with few nonzeros go to short segments (one row per lane group).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "amped_internal.h"

namespace amped {

// ------------------------------------------------------------------ checked builds
// With AMPED_CHECKS an index outside its array records the first failure in
// the error word ({code, index, slot}) and is replaced by an in-bounds one (0);
// without it these helpers are the plain index and the bound is never read.
__device__ __forceinline__ void check_fail(int32_t* err, int32_t code, int64_t index, int32_t slot) {
    if (atomicCAS(err, 0, code) == 0) {
        err[1] = (int32_t)index;
        err[2] = slot;
    }
}
__device__ __forceinline__ int checked_index(int32_t* err, int32_t code, int c, int bound, int slot) {
#if AMPED_CHECKS
    if ((uint32_t)c >= (uint32_t)bound) {
        check_fail(err, code, c, slot);
        return 0;
    }
#endif
    return c;
}
// coordinate c of input slot n, as a factor row index
__device__ __forceinline__ uint64_t frow(const MttkrpParams& p, int n, int c) {
    return (uint64_t)(uint32_t)checked_index(p.err, kCheckCoord, c, p.fdim[n], n);
}
// an output row id read from the row tables
__device__ __forceinline__ int out_row(const MttkrpParams& p, int id) {
    return checked_index(p.err, kCheckOutRow, id, p.out_rows, -1);
}

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

// ------------------------------------------------------------------ packed fp32 helpers
// fp32 pairs in one 64-bit register for the sm_100-family packed instructions.
__device__ __forceinline__ unsigned long long pk(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(unsigned long long r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// exact fp32 product of two bf16 / fp16 halves of 32-bit words (lo*lo, hi*hi)
__device__ __forceinline__ void prod_bf16(uint32_t a, uint32_t b, float& lo, float& hi) {
    asm("{ .reg .b16 al, ah, bl, bh; mov.b32 {al, ah}, %2; mov.b32 {bl, bh}, %3;\n\t"
        "fma.rn.f32.bf16 %0, al, bl, 0f00000000; fma.rn.f32.bf16 %1, ah, bh, 0f00000000; }"
        : "=f"(lo), "=f"(hi) : "r"(a), "r"(b));
}
__device__ __forceinline__ void prod_f16(uint32_t a, uint32_t b, float& lo, float& hi) {
    asm("{ .reg .b16 al, ah, bl, bh; mov.b32 {al, ah}, %2; mov.b32 {bl, bh}, %3;\n\t"
        "fma.rn.f32.f16 %0, al, bl, 0f00000000; fma.rn.f32.f16 %1, ah, bh, 0f00000000; }"
        : "=f"(lo), "=f"(hi) : "r"(a), "r"(b));
}

// Raw row slices as loaded: 32 bytes per lane for the vector shapes (one
// 256-bit load; four lanes cover a 128-byte row of 32 fp32 or 64 16-bit values).
__device__ __forceinline__ void ld_v8(const void* p, uint32_t (&w)[8]) {
    asm("ld.global.nc.L1::evict_last.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
        : "l"(p));
}
template <typename T, int VEC>
struct Raw;
template <>
struct Raw<float, 8> {
    uint32_t w[8];
    __device__ __forceinline__ void load(const float* p) { ld_v8(p, w); }
};
template <>
struct Raw<__nv_bfloat16, 16> {
    uint32_t w[8];
    __device__ __forceinline__ void load(const __nv_bfloat16* p) { ld_v8(p, w); }
};
template <>
struct Raw<__half, 16> {
    uint32_t w[8];
    __device__ __forceinline__ void load(const __half* p) { ld_v8(p, w); }
};
template <>
struct Raw<float, 1> {
    float f;
    __device__ __forceinline__ void load(const float* p) { f = __ldg(p); }
};
template <>
struct Raw<__nv_bfloat16, 1> {
    float f;
    __device__ __forceinline__ void load(const __nv_bfloat16* p) {
        f = __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p)) << 16);
    }
};
template <>
struct Raw<__half, 1> {
    float f;
    __device__ __forceinline__ void load(const __half* p) { f = __half2float(__ldg(p)); }
};

__device__ __forceinline__ float lo_f(uint32_t w, const __nv_bfloat16*) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi_f(uint32_t w, const __nv_bfloat16*) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float lo_f(uint32_t w, const __half*) {
    return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
}
__device__ __forceinline__ float hi_f(uint32_t w, const __half*) {
    return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
}

// acc[e] += v * prod_n x_n[e] for the vector shapes (no staging, no masks).
template <typename T, int VEC, int NIN>
struct Mac;
template <int NIN>
struct Mac<float, 8, NIN> {  // packed f32x2: four pairs per lane
    static __device__ __forceinline__ void run(float (&acc)[8], float v, const Raw<float, 8> (&x)[NIN]) {
        const unsigned long long vv = pk(v, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            unsigned long long pr = pk(__uint_as_float(x[0].w[2 * k]), __uint_as_float(x[0].w[2 * k + 1]));
#pragma unroll
            for (int n = 1; n < NIN; ++n)
                pr = mul2(pr, pk(__uint_as_float(x[n].w[2 * k]), __uint_as_float(x[n].w[2 * k + 1])));
            unsigned long long a = fma2(vv, pr, pk(acc[2 * k], acc[2 * k + 1]));
            upk(a, acc[2 * k], acc[2 * k + 1]);
        }
    }
};
template <typename H, int NIN>
struct Mac16 {  // 16-bit factors: exact fp32 products of the first two, fp32 for the rest
    static __device__ __forceinline__ void run(float (&acc)[16], float v, const Raw<H, 16> (&x)[NIN]) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float lo, hi;
            if constexpr (NIN == 1) {
                lo = lo_f(x[0].w[i], (const H*)nullptr);
                hi = hi_f(x[0].w[i], (const H*)nullptr);
            } else {
                if constexpr (std::is_same<H, __nv_bfloat16>::value)
                    prod_bf16(x[0].w[i], x[1].w[i], lo, hi);
                else
                    prod_f16(x[0].w[i], x[1].w[i], lo, hi);
#pragma unroll
                for (int n = 2; n < NIN; ++n) {
                    lo *= lo_f(x[n].w[i], (const H*)nullptr);
                    hi *= hi_f(x[n].w[i], (const H*)nullptr);
                }
            }
            acc[2 * i] = fmaf(v, lo, acc[2 * i]);
            acc[2 * i + 1] = fmaf(v, hi, acc[2 * i + 1]);
        }
    }
};
template <int NIN>
struct Mac<__nv_bfloat16, 16, NIN> : Mac16<__nv_bfloat16, NIN> {};
template <int NIN>
struct Mac<__half, 16, NIN> : Mac16<__half, NIN> {};

// Scalar (VEC = 1) shapes: one rank per lane, any R <= 32.
template <typename T, int NIN>
struct Mac<T, 1, NIN> {
    static __device__ __forceinline__ void run(float (&acc)[1], float v, const Raw<T, 1> (&x)[NIN]) {
        float pr = x[0].f;
#pragma unroll
        for (int n = 1; n < NIN; ++n) pr *= x[n].f;
        acc[0] = fmaf(v, pr, acc[0]);
    }
};

// Widen a raw row slice to fp32.
__device__ __forceinline__ void widen(const Raw<float, 8>& r, float (&x)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = __uint_as_float(r.w[i]);
}
template <typename H>
__device__ __forceinline__ void widen(const Raw<H, 16>& r, float (&x)[16]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        x[2 * i] = lo_f(r.w[i], (const H*)nullptr);
        x[2 * i + 1] = hi_f(r.w[i], (const H*)nullptr);
    }
}
template <typename T>
__device__ __forceinline__ void widen(const Raw<T, 1>& r, float (&x)[1]) {
    x[0] = r.f;
}

// Reduce-scatter of VEC-wide partial rows over the G groups of a warp (lanes
// q, q+LPN, q+2LPN, ... hold the same ranks): after log2(G) halving rounds
// each lane holds VEC/G summed ranks starting at the returned offset.
template <int VEC, int G, int LPN>
__device__ __forceinline__ int reduce_scatter(float (&a)[VEC], int g) {
    int e0 = 0;
#pragma unroll
    for (int k = 0; (1 << k) < G; ++k) {
        const int c = VEC >> k;
        const int bit = (g >> k) & 1;
#pragma unroll
        for (int i = 0; i < c / 2; ++i) {
            const float keep = bit ? a[c / 2 + i] : a[i];
            const float send = bit ? a[i] : a[c / 2 + i];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, LPN << k);
        }
        e0 += bit * (c / 2);
    }
    return e0;
}

template <int M, int VEC>
__device__ __forceinline__ void store_part(float* dst, const float (&a)[VEC], bool streaming) {
    if constexpr (M >= 4) {
#pragma unroll
        for (int i = 0; i < M; i += 4) {
            const float4 v = make_float4(a[i], a[i + 1], a[i + 2], a[i + 3]);
            if (streaming)
                __stcs(reinterpret_cast<float4*>(dst + i), v);
            else
                *reinterpret_cast<float4*>(dst + i) = v;
        }
    } else if constexpr (M == 2) {
        const float2 v = make_float2(a[0], a[1]);
        if (streaming)
            __stcs(reinterpret_cast<float2*>(dst), v);
        else
            *reinterpret_cast<float2*>(dst) = v;
    } else {
        if (streaming)
            __stcs(dst, a[0]);
        else
            *dst = a[0];
    }
}

// ------------------------------------------------------------------ residual (completion) helpers
// t[e] = prod_n x_n[e] in fp32 (the Khatri-Rao row of one nonzero, without its value).
template <typename T, int VEC, int NIN>
__device__ __forceinline__ void kr_row(float (&t)[VEC], const Raw<T, VEC> (&x)[NIN]) {
    if constexpr (std::is_same<T, float>::value && VEC == 8) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            unsigned long long pr = pk(__uint_as_float(x[0].w[2 * k]), __uint_as_float(x[0].w[2 * k + 1]));
#pragma unroll
            for (int n = 1; n < NIN; ++n)
                pr = mul2(pr, pk(__uint_as_float(x[n].w[2 * k]), __uint_as_float(x[n].w[2 * k + 1])));
            upk(pr, t[2 * k], t[2 * k + 1]);
        }
    } else if constexpr (VEC == 16) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float lo, hi;
            if constexpr (NIN == 1) {
                lo = lo_f(x[0].w[i], (const T*)nullptr);
                hi = hi_f(x[0].w[i], (const T*)nullptr);
            } else {
                if constexpr (std::is_same<T, __nv_bfloat16>::value)
                    prod_bf16(x[0].w[i], x[1].w[i], lo, hi);
                else
                    prod_f16(x[0].w[i], x[1].w[i], lo, hi);
#pragma unroll
                for (int n = 2; n < NIN; ++n) {
                    lo *= lo_f(x[n].w[i], (const T*)nullptr);
                    hi *= hi_f(x[n].w[i], (const T*)nullptr);
                }
            }
            t[2 * i] = lo;
            t[2 * i + 1] = hi;
        }
    } else {
        float pr = x[0].f;
#pragma unroll
        for (int n = 1; n < NIN; ++n) pr *= x[n].f;
        t[0] = pr;
    }
}

// Sum over the group's LPN lanes of sum_e a[e] * b[e]: the sampled model value
// of one nonzero (a = its Khatri-Rao row, b = the output-mode factor row).
template <int VEC, int LPN>
__device__ __forceinline__ float group_dot(const float (&a)[VEC], const float (&b)[VEC]) {
    float d = 0.f;
#pragma unroll
    for (int e = 0; e < VEC; ++e) d = fmaf(a[e], b[e], d);
#pragma unroll
    for (int o = 1; o < LPN; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    return d;
}

// The lane's slice of output-mode factor row `row` (zeros for lanes beyond R).
template <typename T, int VEC>
__device__ __forceinline__ void load_out_row(const MttkrpParams& p, int row, int q, float (&a)[VEC]) {
    if (q * VEC < p.R) {
        Raw<T, VEC> r;
        r.load(static_cast<const T*>(p.fout) + (int64_t)row * p.R + q * VEC);
        widen(r, a);
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) a[e] = 0.f;
    }
}

// ------------------------------------------------------------------ MTTKRP
// Steps per chunk (nonzeros per group per fast-path chunk): all gathers of a
// chunk are issued before any use.  The 256-bit vector shapes hold a 32-byte
// slice of every gathered row in registers, so they take 2 steps at 64
// registers (4 blocks of 256 threads per SM); on GB300 at R = 32 that beat 4
// steps at 3 blocks per SM by 3-4 %.  Scalar shapes take 4; 5+ input modes
// take half as many (registers).
template <int VEC, int NIN>
struct Chunk {
    static constexpr int value = VEC >= 8 ? (NIN >= 5 ? 1 : 2) : (NIN >= 5 ? 2 : 4);
};

constexpr int kBatch = 128;  // nonzeros per stream batch of a warp (32 lanes x 4)

template <int NIN>
struct StreamBatch {
    int4 idx[NIN];
    float4 val;
};

template <int NIN>
__device__ __forceinline__ void load_batch(const MttkrpParams& p, int kl, StreamBatch<NIN>& b) {
    const uint64_t pol = policy_evict_first();
    kl = checked_index(p.err, kCheckStream, kl, (int)(p.stride - 3), -1);
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

// L2 prefetch of one stream batch (NIN + 1 arrays of kBatch words = 4 lines each);
// no registers are held, so the batch's own loads later hit L2.
template <int NIN>
__device__ __forceinline__ void prefetch_batch(const MttkrpParams& p, int kb, int lane) {
    if (lane < 4 * (NIN + 1)) {
        const int a = lane >> 2, line = lane & 3;
        const int32_t* base = a < NIN ? p.idx[a] : (p.perm ? p.perm : reinterpret_cast<const int32_t*>(p.val));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + kb + 32 * line));
    }
}

// Shared-memory staging of one stream batch per warp, one record per nonzero:
// the NIN input coordinates and the value's bit pattern, 16 bytes for up to
// three input modes ({i0, i1, i2, v}), 32 bytes for four ({i0..i3}, {v, -, -, -}).
// Record j lives in slot j ^ ((j >> 3) & 7) of each 16-byte array: with that
// swizzle the staging stores (lane l writes records 4l..4l+3) and the per-step
// loads (G consecutive records) both touch every 16-byte bank group at most
// once per 128 bytes.
__device__ __forceinline__ int swz(int j) { return j ^ ((j >> 3) & 7); }

template <int NIN, bool WIDE = (NIN > 3)>
struct Rec {  // up to three input coordinates and the value: 16 bytes
    int4 a;
    __device__ __forceinline__ int idx(int n) const { return n == 0 ? a.x : n == 1 ? a.y : a.z; }
    __device__ __forceinline__ float val() const { return __int_as_float(a.w); }
};
template <int NIN>
struct Rec<NIN, true> {  // four to seven input coordinates, then the value: 32 bytes
    int4 a, b;
    __device__ __forceinline__ int idx(int n) const { return n < 4 ? comp_rt(a, n) : comp_rt(b, n - 4); }
    __device__ __forceinline__ float val() const { return __int_as_float(comp_rt(b, NIN - 4)); }
};

template <int NIN, bool WIDE = (NIN > 3)>
struct WarpStage {
    int4 a[kBatch];
    __device__ __forceinline__ Rec<NIN> get(int j) const { return Rec<NIN>{a[swz(j)]}; }
};
template <int NIN>
struct WarpStage<NIN, true> {
    int4 a[kBatch];
    int4 b[kBatch];
    __device__ __forceinline__ Rec<NIN> get(int j) const { return Rec<NIN>{a[swz(j)], b[swz(j)]}; }
};

template <int NIN>
__device__ __forceinline__ void stage_batch(WarpStage<NIN>& st, int lane, const StreamBatch<NIN>& b) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int slot = swz(4 * lane + c);
        if constexpr (NIN <= 3) {
            int4 r;
            r.x = comp_rt(b.idx[0], c);
            r.y = NIN > 1 ? comp_rt(b.idx[NIN > 1 ? 1 : 0], c) : 0;
            r.z = NIN > 2 ? comp_rt(b.idx[NIN > 2 ? 2 : 0], c) : 0;
            r.w = __float_as_int(comp_rt(b.val, c));
            st.a[slot] = r;
        } else {
            st.a[slot] = make_int4(comp_rt(b.idx[0], c), comp_rt(b.idx[1], c), comp_rt(b.idx[2], c),
                                   comp_rt(b.idx[3], c));
            int w[4];
#pragma unroll
            for (int n = 4; n < 8; ++n)  // coordinates 4.., then the value, then zeros
                w[n - 4] = n < NIN ? comp_rt(b.idx[n < NIN ? n : 0], c)
                                   : (n == NIN ? __float_as_int(comp_rt(b.val, c)) : 0);
            st.b[slot] = make_int4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Factored path (the fiber factorisation of compressed-sparse-fiber MTTKRP,
// done per lane group) for a staged batch of kBatch nonzeros that lies inside
// one row and inside the segment.  Group g walks the RUN = kBatch/G
// consecutive nonzeros g*RUN .. g*RUN+RUN-1.  The copy orders a row
// lexicographically by the input slots, so along the walk slot 0 changes
// least often, then slot 1, and so on: a "run" at level l is a stretch of
// nonzeros with equal slots 0..l.  The product of a nonzero factors as
//   val * A_0(c0) * ... * A_{L-1}(c_{L-1}) * A_L(c_L)      (L = NIN - 1)
// so the row sum is, per level-0 run, A_0 times the sum over its level-1
// runs of A_1 times ... times the sum of val * A_L over the level-(L-1) run.
// t[l] holds the open level-l run's inner sum; when slot l changes, the run
// closes (t[l-1] += x[l] * t[l], or acc for l = 0) and the new run's row x[l]
// is gathered.  That row is needed only when its run closes, so its latency
// is hidden behind the run, while the innermost slot's rows (needed by every
// nonzero) are gathered ZA nonzeros ahead.  Rows delivered to the lanes per
// nonzero: one for slot L plus one per run start of the outer slots, instead
// of NIN; on power-law tensors that is 1.5-2 instead of 3 at four modes.
template <typename T, int VEC, int LPN, int NIN, int ZA>
__device__ __forceinline__ void fiber_batch(const MttkrpParams& p, const WarpStage<NIN>& st, int g,
                                            const T* const (&fl)[NIN], uint32_t R, float (&acc)[VEC]) {
    static_assert(std::is_same<T, float>::value && VEC == 8, "fp32 rows of 8 ranks per lane");
    constexpr int G = 32 / LPN, RUN = kBatch / G, L = NIN - 1;
    static_assert(L >= 1 && RUN % ZA == 0, "factored path shape");
    Raw<T, VEC> x[L];  // the open run's row, per level
    unsigned long long t[L][VEC / 2];  // open run's inner sums, as fp32 pairs
    int cur[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        cur[l] = -1;
#pragma unroll
        for (int e = 0; e < VEC; ++e) x[l].w[e] = 0u;
#pragma unroll
        for (int e = 0; e < VEC / 2; ++e) t[l][e] = 0ull;
    }
    auto close_into = [&](const Raw<T, VEC>& xr, unsigned long long (&tt)[VEC / 2], unsigned long long* dst) {
#pragma unroll
        for (int e = 0; e < VEC / 2; ++e) {
            dst[e] = fma2(pk(__uint_as_float(xr.w[2 * e]), __uint_as_float(xr.w[2 * e + 1])), tt[e], dst[e]);
            tt[e] = 0ull;
        }
    };
    unsigned long long a2[VEC / 2];  // acc as pairs while the batch runs
#pragma unroll
    for (int e = 0; e < VEC / 2; ++e) a2[e] = pk(acc[2 * e], acc[2 * e + 1]);
    const int j0 = g * RUN;
#pragma unroll 1
    for (int u = 0; u < RUN; u += ZA) {
        Rec<NIN> r[ZA];
        Raw<T, VEC> z[ZA];
#pragma unroll
        for (int a = 0; a < ZA; ++a) {
            r[a] = st.get(j0 + u + a);
            z[a].load(fl[L] + frow(p, L, r[a].idx(L)) * R);
        }
#pragma unroll
        for (int a = 0; a < ZA; ++a) {
            bool ch[L];
#pragma unroll
            for (int l = 0; l < L; ++l) ch[l] = (l > 0 && ch[l - 1]) || r[a].idx(l) != cur[l];
            // close the runs that end here, innermost first
#pragma unroll
            for (int l = L - 1; l >= 1; --l)
                if (ch[l]) close_into(x[l], t[l], t[l - 1]);
            if (ch[0]) close_into(x[0], t[0], a2);
            // open the new runs
#pragma unroll
            for (int l = 0; l < L; ++l)
                if (ch[l]) {
                    cur[l] = r[a].idx(l);
                    x[l].load(fl[l] + frow(p, l, cur[l]) * R);
                }
            const unsigned long long vv = pk(r[a].val(), r[a].val());
#pragma unroll
            for (int e = 0; e < VEC / 2; ++e)
                t[L - 1][e] = fma2(vv, pk(__uint_as_float(z[a].w[2 * e]), __uint_as_float(z[a].w[2 * e + 1])), t[L - 1][e]);
        }
    }
#pragma unroll
    for (int l = L - 1; l >= 1; --l) close_into(x[l], t[l], t[l - 1]);
    close_into(x[0], t[0], a2);
#pragma unroll
    for (int e = 0; e < VEC / 2; ++e) upk(a2[e], acc[2 * e], acc[2 * e + 1]);
}

// Shapes that take the factored path (fp32 rows of 8 ranks per lane, 3- and
// 4-mode tensors: register room for the open runs at 64 registers) and how
// many nonzeros ahead the innermost rows are gathered.  On GB300 it is 9-12 %
// faster than the chunk path on the 4-mode power-law tensor and equal on the
// 3-mode one; deeper look-ahead and L1 prefetch of the next rows measured no
// better or slower.
template <typename T, int VEC, int NIN>
struct Factored {
    static constexpr bool value = std::is_same<T, float>::value && VEC == 8 && (NIN == 2 || NIN == 3);
    static constexpr int ahead = NIN == 2 ? 2 : 1;
};

// One warp processes one segment.  The warp holds G = 32/LPN groups; at
// step u of a chunk, group g takes nonzero base + u*G + g, so all control
// flow (batches, chunks, row ends) is uniform across the warp.  A chunk that
// lies inside one row and inside the segment takes the fast path (no masks:
// gathers and multiply-adds straight into the row accumulator); other chunks
// stage their products and close rows that end inside a step with a
// butterfly sum over the groups.
template <typename T, int VEC, int LPN, int NIN, bool RES>
__device__ __forceinline__ void mttkrp_segment(const MttkrpParams& p, int s, WarpStage<NIN>& st, int lane,
                                               const T* const (&fl)[NIN], double& lsum) {
    constexpr int G = 32 / LPN;
    constexpr int CH = Chunk<VEC, NIN>::value;
    constexpr int CHN = CH * G;  // nonzeros per chunk
    static_assert(kBatch % CHN == 0, "a chunk must tile the batch");
    const int g = lane / LPN, q = lane % LPN;
    const bool active = q * VEC < p.R;
    const uint32_t R = (uint32_t)p.R;
    const int row_s = __ldg(p.seg_row + s), nz_s = __ldg(p.seg_nz + s);
    const int row_e = __ldg(p.seg_row + s + 1), nz_e = __ldg(p.seg_nz + s + 1);

    // rowptr window of 64 rows in two registers per lane: w0 = rowptr[rwb + lane], w1 = rowptr[rwb + 32 + lane]
    int rwb = row_s;
    int w0 = __ldg(p.rowptr + checked_index(p.err, kCheckRowptr, rwb + lane, p.I + 1 + kPad, -1));
    int w1 = __ldg(p.rowptr + checked_index(p.err, kCheckRowptr, rwb + 32 + lane, p.I + 1 + kPad, -1));
    auto rowptr_at = [&](int r) -> int { return __shfl_sync(0xffffffffu, w0, r - rwb); };
    auto ensure_window = [&](int r) {  // keep rows r and r+1 in w0; slide by 32 (next half prefetched)
        if (r + 1 - rwb >= 32) {
            rwb += 32;
            w0 = w1;
            w1 = __ldg(p.rowptr + checked_index(p.err, kCheckRowptr, rwb + 32 + lane, p.I + 1 + kPad, -1));
        }
    };

    const bool cont = rowptr_at(row_s) < nz_s;  // the first row began in an earlier segment
    int i = row_s;
    int rstart = nz_s;  // first nonzero of row i inside this segment
    int rend = i < row_e ? rowptr_at(i + 1) : nz_e;  // end of row i's nonzeros inside this segment

    float acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
    float ao[RES ? VEC : 1];  // residual mode: output-mode factor row of row i
    if constexpr (RES) {
        if (i < p.I) load_out_row<T, VEC>(p, out_row(p, __ldg(p.rows_L + i)), q, ao);
    }

    auto flush = [&](int row) {
        const int64_t rq = (int64_t)(lane % LPN) * VEC;
        float* dst;
        bool streaming = false;
        if (row == row_s && cont) {
            dst = p.part + ((int64_t)s * 2) * R + rq;  // head partial of a split row
        } else if (row < row_e) {
            dst = p.out + (int64_t)out_row(p, __ldg(p.rows_L + row)) * R + rq;  // complete row: written exactly once
            streaming = true;
        } else {
            dst = p.part + ((int64_t)s * 2 + 1) * R + rq;  // tail partial of a split row
        }
        const int cnt = rend - rstart;  // nonzeros of the row inside this segment
        if (cnt > 1 && G > 1 && G <= VEC) {
            // reduce-scatter over the G groups: each lane ends with VEC/G summed ranks
            const int e0 = reduce_scatter<VEC, G, LPN>(acc, g);
            if (active) store_part<VEC / G>(dst + e0, acc, streaming);
        } else {
            int owner = 0;  // group holding the row's complete sum
            if (cnt == 1) {
                // one contribution, already the sum; nonzero k is always processed by group (k - (nz_s & ~3)) % G
                owner = (rstart - (nz_s & ~3)) & (G - 1);
            } else if (cnt > 1) {
#pragma unroll
                for (int o = LPN; o < 32; o <<= 1)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
            }
            if (g == owner && active) store_row<VEC>(dst, acc, streaming);
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
    };
    auto advance = [&]() {  // close row i, move to row i+1
        flush(i);
        ++i;
        rstart = rend;
        if (i < row_e) {
            ensure_window(i);
            rend = rowptr_at(i + 1);
        } else {
            rend = nz_e;
        }
        if constexpr (RES) {
            if (i < p.I && rend > rstart) load_out_row<T, VEC>(p, out_row(p, __ldg(p.rows_L + i)), q, ao);
        }
    };

    int kb = nz_s & ~3;
    for (; kb < nz_e; kb += kBatch) {
        {
            StreamBatch<NIN> cur;
            load_batch<NIN>(p, kb + 4 * lane, cur);
            __syncwarp();
            stage_batch<NIN>(st, lane, cur);
            __syncwarp();
        }
        if (kb + kBatch < nz_e) prefetch_batch<NIN>(p, kb + kBatch, lane);  // next batch into L2
        if constexpr (!RES && Factored<T, VEC, NIN>::value) {
            if (kb >= nz_s && kb + kBatch <= nz_e && kb + kBatch <= rend) {  // the batch lies inside row i
                if (active) fiber_batch<T, VEC, LPN, NIN, Factored<T, VEC, NIN>::ahead>(p, st, g, fl, R, acc);
                continue;
            }
        }
#pragma unroll 1
        for (int c0 = 0; c0 < kBatch; c0 += CHN) {
            const int base = kb + c0;
            if (base >= nz_e) break;
            if (base + CHN <= nz_s) continue;
            if (base >= nz_s && base + CHN <= nz_e && base + CHN <= rend) {
                // fast path: every nonzero of the chunk is valid and in row i
                if constexpr (!RES) {
                    if (active) {
#pragma unroll
                        for (int u = 0; u < CH; ++u) {
                            const Rec<NIN> r = st.get(c0 + u * G + g);
                            Raw<T, VEC> x[NIN];
#pragma unroll
                            for (int n = 0; n < NIN; ++n)
                                x[n].load(fl[n] + frow(p, n, r.idx(n)) * R);
                            Mac<T, VEC, NIN>::run(acc, r.val(), x);
                        }
                    }
                } else {
                    // residual mode: value r = (model at the nonzero) - x, contribution r * KR row
#pragma unroll
                    for (int u = 0; u < CH; ++u) {
                        const Rec<NIN> r = st.get(c0 + u * G + g);
                        float t[VEC];
                        if (active) {
                            Raw<T, VEC> x[NIN];
#pragma unroll
                            for (int n = 0; n < NIN; ++n)
                                x[n].load(fl[n] + frow(p, n, r.idx(n)) * R);
                            kr_row<T, VEC, NIN>(t, x);
                        } else {
#pragma unroll
                            for (int e = 0; e < VEC; ++e) t[e] = 0.f;
                        }
                        const float res = group_dot<VEC, LPN>(t, ao) - r.val();
#pragma unroll
                        for (int e = 0; e < VEC; ++e) acc[e] = fmaf(res, t[e], acc[e]);
                        if (q == 0) lsum += (double)res * (double)res;
                    }
                }
                continue;
            }
            // slow path, in halves of SH steps: stage masked products, then walk rows
            constexpr int SH = CH > 4 ? 4 : CH;
#pragma unroll
            for (int h = 0; h < CH; h += SH) {
                float t[SH][VEC];
                float vv[RES ? SH : 1];  // residual mode: the staged products omit the value
#pragma unroll
                for (int u = 0; u < SH; ++u) {
                    const int j = c0 + (h + u) * G + g;
                    const int k = kb + j;
                    const bool valid = active && k >= nz_s && k < nz_e;
                    const Rec<NIN> r = st.get(j);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) t[u][e] = 0.f;
                    if constexpr (RES) vv[u] = r.val();
                    if (valid) {
                        Raw<T, VEC> x[NIN];
#pragma unroll
                        for (int n = 0; n < NIN; ++n)
                            x[n].load(fl[n] + frow(p, n, r.idx(n)) * R);
                        if constexpr (RES)
                            kr_row<T, VEC, NIN>(t[u], x);
                        else
                            Mac<T, VEC, NIN>::run(t[u], r.val(), x);
                    }
                }
#pragma unroll
                for (int u = 0; u < SH; ++u) {
                    const int kstep = base + (h + u) * G;
                    if (kstep >= nz_e) break;
                    const int klast = min(kstep + G, nz_e) - 1;
                    if (klast < nz_s) continue;
                    if constexpr (!RES) {
                        if (kstep >= rstart && klast < rend) {  // the whole step lies in row i
#pragma unroll
                            for (int e = 0; e < VEC; ++e) acc[e] += t[u][e];
                            continue;
                        }
                    }
                    const int kg = kstep + g;
                    while (true) {
                        const bool in = kg >= rstart && kg < rend && kg >= nz_s && kg < nz_e;
                        if constexpr (RES) {
                            // the model value needs the output-mode row of the nonzero's own row
                            const float res = group_dot<VEC, LPN>(t[u], ao) - vv[u];
#pragma unroll
                            for (int e = 0; e < VEC; ++e) acc[e] = in ? fmaf(res, t[u][e], acc[e]) : acc[e];
                            if (in && q == 0) lsum += (double)res * (double)res;
                        } else {
#pragma unroll
                            for (int e = 0; e < VEC; ++e) acc[e] += in ? t[u][e] : 0.f;
                        }
                        if (klast < rend) break;
                        advance();
                    }
                }
            }
        }
    }
    // close the rows that end in this segment, then the last row if it continues
    while (i < row_e) advance();
    if (i < p.I && rend > rstart) flush(i);
}

// One short segment: at most kShortRows rows (sorted by length, so rows of a
// round have similar lengths) whose nonzeros fit one staged batch.  Group g
// accumulates row r0+g by itself and stores it: no cross-group reduction.
template <typename T, int VEC, int LPN, int NIN, bool RES>
__device__ __forceinline__ void mttkrp_short(const MttkrpParams& p, int t, WarpStage<NIN>& st, int lane,
                                             const T* const (&fl)[NIN], double& lsum) {
    constexpr int G = 32 / LPN;
    const int g = lane / LPN, q = lane % LPN;
    const bool active = q * VEC < p.R;
    const uint32_t R = (uint32_t)p.R;
    const int a = __ldg(p.seg_short + t), nr = __ldg(p.seg_short + t + 1) - a;  // nr <= 31
    const int my_rp = __ldg(p.rowptr_S + a + min(lane, nr));  // lane l: start of short row a+l; lane nr: end
    const int my_id = lane < nr ? out_row(p, __ldg(p.rows_S + a + lane)) : 0;
    const int k0 = __shfl_sync(0xffffffffu, my_rp, 0), k1 = __shfl_sync(0xffffffffu, my_rp, nr);
    const int kb = k0 & ~3;  // k1 - kb < kBatch by construction of the short segments
#if AMPED_CHECKS
    if (k1 - kb > kBatch || k0 > k1) {  // warp-uniform: the whole warp skips the segment
        if (lane == 0) check_fail(p.err, kCheckShort, t, -1);
        return;
    }
#endif
    if (k1 > k0) {
        StreamBatch<NIN> cur;
        load_batch<NIN>(p, kb + 4 * lane, cur);
        __syncwarp();
        stage_batch<NIN>(st, lane, cur);
        __syncwarp();
    }
    for (int r0 = 0; r0 < nr; r0 += G) {
        const int rr = r0 + g;
        const int start = __shfl_sync(0xffffffffu, my_rp, min(rr, nr));
        const int end = __shfl_sync(0xffffffffu, my_rp, min(rr + 1, nr));
        const int len = rr < nr ? end - start : 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        float acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
        const int id = __shfl_sync(0xffffffffu, my_id, rr & 31);
        if constexpr (!RES) {
            for (int k = 0; k < maxlen; k += 2) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (active && k + u < len) {
                        const Rec<NIN> r = st.get(start + k + u - kb);
                        Raw<T, VEC> x[NIN];
#pragma unroll
                        for (int n = 0; n < NIN; ++n)
                            x[n].load(fl[n] + frow(p, n, r.idx(n)) * R);
                        Mac<T, VEC, NIN>::run(acc, r.val(), x);
                    }
                }
            }
        } else {
            float ao[VEC];
            if (rr < nr) {
                load_out_row<T, VEC>(p, id, q, ao);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) ao[e] = 0.f;
            }
            for (int k = 0; k < maxlen; ++k) {
                const bool in = k < len;
                const Rec<NIN> r = st.get(in ? start + k - kb : 0);
                float tt[VEC];
                if (active && in) {
                    Raw<T, VEC> x[NIN];
#pragma unroll
                    for (int n = 0; n < NIN; ++n) x[n].load(fl[n] + frow(p, n, r.idx(n)) * R);
                    kr_row<T, VEC, NIN>(tt, x);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) tt[e] = 0.f;
                }
                const float res = group_dot<VEC, LPN>(tt, ao) - r.val();
                if (in) {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) acc[e] = fmaf(res, tt[e], acc[e]);
                    if (q == 0) lsum += (double)res * (double)res;
                }
            }
        }
        if (rr < nr && active) store_row<VEC>(p.out + (int64_t)id * R + q * VEC, acc, true);
    }
    __syncwarp();  // the stage is reused by the warp's next segment
}

// Resident blocks per SM the residual-mode kernel is compiled for: as many as
// fit without heavy spilling (it needs the output-mode row, the gathered
// Khatri-Rao row and the accumulator per lane).
template <typename T, int VEC, int NIN>
constexpr int res_blocks() {
    return VEC == 1 ? 4 : (sizeof(T) == 2 ? 2 : (NIN <= 2 ? 4 : 3));
}

template <typename T, int VEC, int LPN, int NIN, bool RES>
__global__ void __launch_bounds__(256, RES ? res_blocks<T, VEC, NIN>() : 4) mttkrp_kernel(const MttkrpParams p) {
    __shared__ __align__(16) WarpStage<NIN> stage[8];
    const int lane = threadIdx.x & 31;
    WarpStage<NIN>& st = stage[threadIdx.x >> 5];
    const int q = lane % LPN;
    const T* fl[NIN];  // this lane's first rank in every input factor
#pragma unroll
    for (int n = 0; n < NIN; ++n) fl[n] = static_cast<const T*>(p.fac[n]) + q * VEC;
    const int total = p.S + p.S_S;  // long segments first, then short segments
    double lsum = 0.0;  // residual mode: this lane's share of sum (m - x)^2
    int s = 0;
    if (lane == 0) s = atomicAdd(p.queue, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    while (s < total) {
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(p.queue, 1);  // next ticket, latency hidden by this segment
        if (s < p.S)
            mttkrp_segment<T, VEC, LPN, NIN, RES>(p, s, st, lane, fl, lsum);
        else
            mttkrp_short<T, VEC, LPN, NIN, RES>(p, s - p.S, st, lane, fl, lsum);
        s = __shfl_sync(0xffffffffu, nxt, 0);
    }
    if constexpr (RES) {
        if (p.loss != nullptr) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            if (lane == 0 && lsum != 0.0) atomicAdd(p.loss, 0.5 * lsum);
        }
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
    constexpr int CH = 4;  // a multiple of 4: step u of a chunk is component u of its lane's int4
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
        for (int n = 0; n < NM; ++n)
            bi[n] = ld_stream_i4(p.idx[n] + checked_index(p.err, kCheckStream, kl, (int)(p.stride - 3), n), pol);
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
                        Raw<T, VEC> raw;
                        raw.load(static_cast<const T*>(p.fac[n]) +
                                 (int64_t)checked_index(p.err, kCheckCoord, c, p.fdim[n], n) * p.R + rq);
                        widen(raw, x);
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
