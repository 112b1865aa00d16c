// als_tc.cu — the CP-ALS apply's contraction on the 5th-generation tensor
// cores (sm_103a).
//
// After the mode-d MTTKRP M and the solve's W = V^-1 (Sec. 2.1: ALS performs
// the mode-wise MTTKRPs in turn, with the standard least-squares update), the
// apply needs, for rank R = 32,
//   A  = M W                      stored (fp32, row-major [rows][R])
//   ip += sum_i M(i,:) * A(i,:)   per column (fp64)
//   ga  = A^T A                   the Gram of the stored A (fp64)
// A = M W is a dense contraction ([rows x 32] x [32 x 32]): it runs here on
// tcgen05.mma with its fp32 accumulator in tensor memory, at fp32 accuracy
// from TF32 inputs by the three-term split x = hi + lo (hi = x rounded to
// TF32, lo = the rest rounded to TF32):
//   M W ~ Mhi Whi + Mhi Wlo + Mlo Whi            (relative error about 2^-21)
// The Gram follows in gram_kernel (als.cu): compensated fp32 sums over tiles
// and fp64 across them keep it within 1e-6 of the exact Gram of the stored
// values, which the next modes' normal equations rely on; a tensor-core Gram
// (M padded from 32 to the 128-row MMA shape) measured 1.2e-6 low (the
// accumulator's rounding over 128 rows) and was slower.
//
// One CTA of 128 threads (4 warps, one per 32 tensor-memory lanes), 3 per SM,
// walks 128-row tiles of M: a bulk TMA copy brings the raw tile into shared
// memory (two stages in flight), all threads split it into hi / lo K-major
// operands in the 128-byte swizzle, thread 0 issues the 12 MMAs (K = 32 in 4
// steps of 8, 3 terms) and commits them to an mbarrier, and every warp reads
// its 32 rows of A back from tensor memory (tcgen05.ld), stores them and adds
// its rows' M * A into fp32 column sums (folded into per-warp fp64 sums every
// 16 tiles).  Every wait is bounded; a wait that gives up sets the status word
// (AlsParams.info = -2) and the CTA frees its tensor memory and stops.
#include <cuda_runtime.h>

#include <cstdint>

#include "amped_internal.h"

namespace amped {
namespace {

constexpr int kR = 32;            // rank of this kernel (a K-major row is 128 bytes: one swizzle row)
constexpr int kTile = 128;        // rows per tile = the MMA's M
constexpr int kStages = 2;        // raw M tiles in flight
constexpr uint32_t kTileBytes = kTile * kR * 4;  // 16 KB
constexpr int kThreads = 128;
constexpr long kWaitLimit = 1l << 26;  // mbarrier polls before a wait gives up (seconds)

// Shared-memory layout (offsets from a 1024-byte aligned base).
constexpr uint32_t kOffMh = 0;                         // M hi [128][128 B], 128-byte swizzle
constexpr uint32_t kOffMl = kOffMh + kTileBytes;       // M lo
constexpr uint32_t kOffWh = kOffMl + kTileBytes;       // W^T hi [32][128 B]
constexpr uint32_t kOffWl = kOffWh + 4096;             // W^T lo
constexpr uint32_t kOffRaw = kOffWl + 4096;            // raw M tiles [kStages][16 KB]
constexpr uint32_t kSmemUsed = kOffRaw + kStages * kTileBytes;
constexpr uint32_t kSmemBytes = kSmemUsed + 1024;      // + alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Byte offset of element (row, k) of a K-major [rows][32] fp32 operand in the
// 128-byte swizzle: 16-byte chunk k/4 of row r sits at chunk (k/4) ^ (r % 8).
__device__ __forceinline__ uint32_t sw128(int row, int k) {
    return (uint32_t)(row * 128 + ((((k >> 2) ^ (row & 7)) & 7) << 4) + (k & 3) * 4);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::tf32: fp32 accumulator, TF32 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    for (long it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
          "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]),
          "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]),
          "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Bulk copy of one raw tile (rows [base, base + nr) of M, contiguous) into a stage.
__device__ __forceinline__ void load_tile(const float* M, int64_t base, int nr, uint32_t dst, uint32_t bar) {
    const uint32_t bytes = (uint32_t)nr * kR * 4;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(M + base * kR), "r"(bytes), "r"(bar)
                 : "memory");
}

__global__ void __launch_bounds__(kThreads, 3) apply_tc_kernel(const float* __restrict__ M, int64_t rows, AlsParams p,
                                                               float* __restrict__ A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full[kStages];  // raw tile s has landed
    __shared__ uint64_t mma_bar;        // the last committed MMA group is done
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    __shared__ double ipw[kThreads / 32][kR];  // per-warp fp64 column sums of M * A
    if (*p.info) return;  // singular V: nothing to apply (the whole grid returns before any allocation)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s0 = smem_u32(sm);
    const int64_t ntiles = (rows + kTile - 1) / kTile;

    // W^T hi / lo: B operand of the product, row c = output column, K = k
    for (int e = tid; e < kR * kR; e += kThreads) {
        const int c = e / kR, k = e % kR;
        const float x = p.w[k * kR + c], h = tf32_rn(x), l = tf32_rn(x - h);
        *reinterpret_cast<float*>(sm + kOffWh + sw128(c, k)) = h;
        *reinterpret_cast<float*>(sm + kOffWl + sw128(c, k)) = l;
    }
    if (warp == 0) {
        // 32 columns: the product's accumulator (128 lanes x 32 fp32)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        failed = 0;
        for (int s = 0; s < kStages; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t t_prod = tmem;
    const uint32_t bar_mma = smem_u32(&mma_bar);
    uint32_t ph_full[kStages] = {0u, 0u};
    uint32_t ph_mma = 0u;
    constexpr uint32_t kIdesc = idesc_tf32(kTile, kR);

    // prefetch the first kStages tiles of this CTA
    if (tid == 0)
        for (int s = 0; s < kStages; ++s) {
            const int64_t t = blockIdx.x + (int64_t)s * gridDim.x;
            if (t < ntiles) {
                const int64_t b = t * kTile;
                load_tile(M, b, (int)(rows - b < kTile ? rows - b : kTile), s0 + kOffRaw + s * kTileBytes,
                          smem_u32(&full[s]));
            }
        }

    // Column sums of M * A: this thread's rows since the last flush in fp32 (at most
    // kIpFlush rows per column), then a warp reduction into per-warp fp64 sums.
    constexpr int kIpFlush = 16;
    float ipf[kR];
#pragma unroll
    for (int c = 0; c < kR; ++c) ipf[c] = 0.f;
    if (tid < kThreads / 32 * kR) (&ipw[0][0])[tid] = 0.0;  // read after the loop's barriers
    const int my_tiles = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
    auto flush_ip = [&]() {
#pragma unroll
        for (int c = 0; c < kR; ++c) {
            float v = ipf[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) ipw[warp][c] += (double)v;
            ipf[c] = 0.f;
        }
    };
    int it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int s = it % kStages;
        const int64_t base = t * kTile;
        const int nr = (int)(rows - base < kTile ? rows - base : kTile);
        const unsigned char* raw = sm + kOffRaw + s * kTileBytes;  // rows [base, base + nr) of M
        // ---- wait for the raw tile, split it into hi / lo operands (rows >= nr are zero)
        const bool got = bar_wait(smem_u32(&full[s]), ph_full[s]);
        ph_full[s] ^= 1u;
        if (!got) failed = 1;
#pragma unroll
        for (int j = 0; j < kTileBytes / 16 / kThreads; ++j) {
            const int f = tid + j * kThreads;  // float4 index: row f / 8, chunk f % 8
            const int row = f >> 3, ch = f & 7;
            float4 v = row < nr ? *reinterpret_cast<const float4*>(raw + f * 16) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 h, l;
            h.x = tf32_rn(v.x); l.x = tf32_rn(v.x - h.x);
            h.y = tf32_rn(v.y); l.y = tf32_rn(v.y - h.y);
            h.z = tf32_rn(v.z); l.z = tf32_rn(v.z - h.z);
            h.w = tf32_rn(v.w); l.w = tf32_rn(v.w - h.w);
            const uint32_t off = (uint32_t)(row * 128 + (((ch ^ (row & 7)) & 7) << 4));
            *reinterpret_cast<float4*>(sm + kOffMh + off) = h;
            *reinterpret_cast<float4*>(sm + kOffMl + off) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(failed)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const int64_t tn = t + (int64_t)kStages * gridDim.x;  // raw stage s is free: refill it
            if (tn < ntiles) {
                const int64_t b = tn * kTile;
                load_tile(M, b, (int)(rows - b < kTile ? rows - b : kTile), s0 + kOffRaw + s * kTileBytes,
                          smem_u32(&full[s]));
            }
            // ---- product: D_prod = Mhi Whi + Mhi Wlo + Mlo Whi over K = 32 (4 steps of 8)
#pragma unroll
            for (int kk = 0; kk < kR / 8; ++kk) {
                const uint32_t off = kk * 32;
                const uint64_t mh = smem_desc(s0 + kOffMh + off), ml = smem_desc(s0 + kOffMl + off);
                const uint64_t wh = smem_desc(s0 + kOffWh + off), wl = smem_desc(s0 + kOffWl + off);
                mma_tf32(t_prod, mh, wh, kIdesc, kk > 0);
                mma_tf32(t_prod, mh, wl, kIdesc, 1);
                mma_tf32(t_prod, ml, wh, kIdesc, 1);
            }
            mma_commit(bar_mma);
        }
        const bool done_p = bar_wait(bar_mma, ph_mma);
        ph_mma ^= 1u;
        if (__syncthreads_or(!done_p)) {
            failed = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- epilogue: row `tid` of the tile
        float a[kR];
        tmem_ld32(t_prod + ((uint32_t)(32 * warp) << 16), a);
        const int row = tid;
        if (row < nr) {
            // M row `row` as hi + lo from the swizzled operands (a quarter-warp's eight rows hit
            // eight different bank groups); hi + lo is M to 2^-22
#pragma unroll
            for (int j = 0; j < kR / 4; ++j) {
                const uint32_t off = (uint32_t)(row * 128 + (((j ^ (row & 7)) & 7) << 4));
                const float4 h = *reinterpret_cast<const float4*>(sm + kOffMh + off);
                const float4 l = *reinterpret_cast<const float4*>(sm + kOffMl + off);
                ipf[4 * j + 0] = fmaf(h.x + l.x, a[4 * j + 0], ipf[4 * j + 0]);
                ipf[4 * j + 1] = fmaf(h.y + l.y, a[4 * j + 1], ipf[4 * j + 1]);
                ipf[4 * j + 2] = fmaf(h.z + l.z, a[4 * j + 2], ipf[4 * j + 2]);
                ipf[4 * j + 3] = fmaf(h.w + l.w, a[4 * j + 3], ipf[4 * j + 3]);
            }
            float4* dst = reinterpret_cast<float4*>(A + (base + row) * kR);
#pragma unroll
            for (int c = 0; c < kR; c += 4) dst[c / 4] = make_float4(a[c], a[c + 1], a[c + 2], a[c + 3]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // M hi / lo and the accumulator are free again
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if ((it + 1) % kIpFlush == 0 || it + 1 == my_tiles) flush_ip();  // uniform over the block
    }
    if (failed) {
        if (tid == 0) atomicExch(p.info, -2);
    } else {
        __syncthreads();
        if (tid < kR) {  // the warps' column sums in a fixed order, one atomic per column
            double v = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) v += ipw[w][tid];
            atomicAdd(p.ip + tid, v);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

}  // namespace

bool als_apply_tc_supported(int R) { return R == kR; }

// Launch of the tensor-core product for R = 32: 3 CTAs per SM, persistent.
int launch_als_apply_tc(const AlsParams& p, const float* M, int64_t rows, float* A, void* stream, int* launched) {
    cudaError_t e = cudaFuncSetAttribute(apply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return (int)e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    const int64_t ntiles = (rows + kTile - 1) / kTile;
    int64_t grid = 3 * (int64_t)sms;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    apply_tc_kernel<<<(unsigned)grid, kThreads, kSmemBytes, static_cast<cudaStream_t>(stream)>>>(M, rows, p, A);
    ++*launched;
    return (int)cudaGetLastError();
}

}  // namespace amped
