// combine.cu — deterministic combine of split-row partials.
//
// A row longer than a segment is cut across segments (paper Sec. 3.2: equal
// partitions with atomics between SMs).  Here each segment leaves the partial
// of such a row in its own slot (head slot for a row that began earlier, tail
// slot for a row that continues), and these kernels add the slots of every
// split row in segment order in fp64, so the result is independent of the
// order in which segments ran.  Level 1: one warp per task (at most
// kCombineSlots consecutive slots of one split row).  Level 2: one block per
// split row that has more than one task, adding its task sums in a fixed order.
#include <cuda_runtime.h>

#include "amped_internal.h"

namespace amped {

__global__ void __launch_bounds__(256) combine_tasks_kernel(const CombineParams p) {
    const int task = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (task >= p.ntask) return;
    const int j = p.tasks[4 * task], lo = p.tasks[4 * task + 1], hi = p.tasks[4 * task + 2];
    const bool first_tail = p.tasks[4 * task + 3] != 0;
    const int row = p.split_info[2 * j];
    const bool single = p.split_info[2 * j + 3] - p.split_info[2 * j + 1] == 1;
    for (int r = lane; r < p.R; r += 32) {
        double s = 0.0;
#pragma unroll 8
        for (int seg = lo; seg < hi; ++seg) {
            const int64_t slot = (seg == lo && first_tail) ? 2 * (int64_t)seg + 1 : 2 * (int64_t)seg;
            s += (double)p.part[slot * p.R + r];
        }
        if (single)
            p.out[(int64_t)row * p.R + r] = (float)s;
        else
            p.tsum[(int64_t)task * p.R + r] = s;
    }
}

// One block per split row with several tasks: warp w adds tasks t0+w, t0+w+8, ...
// in order, then warp 0 adds the eight warp sums in order (fixed association).
__global__ void __launch_bounds__(256) combine_multi_kernel(const CombineParams p) {
    __shared__ double part[8][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = p.multi[blockIdx.x];
    const int row = p.split_info[2 * j], t0 = p.split_info[2 * j + 1], t1 = p.split_info[2 * j + 3];
    for (int r0 = 0; r0 < p.R; r0 += 32) {
        const int r = r0 + lane;
        double s = 0.0;
        if (r < p.R) {
#pragma unroll 4
            for (int t = t0 + w; t < t1; t += 8) s += p.tsum[(int64_t)t * p.R + r];
        }
        part[w][lane] = s;
        __syncthreads();
        if (w == 0 && r < p.R) {
            double tot = 0.0;
#pragma unroll
            for (int x = 0; x < 8; ++x) tot += part[x][lane];
            p.out[(int64_t)row * p.R + r] = (float)tot;
        }
        __syncthreads();
    }
}

int launch_combine(const CombineParams& p, void* stream, int* launched) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *launched = 0;
    if (p.ntask == 0) return 0;
    combine_tasks_kernel<<<(p.ntask + 7) / 8, 256, 0, st>>>(p);
    ++*launched;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || p.nmulti == 0) return (int)e;
    combine_multi_kernel<<<p.nmulti, 256, 0, st>>>(p);
    ++*launched;
    return (int)cudaGetLastError();
}

}  // namespace amped
