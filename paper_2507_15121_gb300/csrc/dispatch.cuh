// dispatch.cuh — picks the kernel shape (vector width VEC, lanes per worker
// LPN, input-mode count) for one factor dtype and launches it.  Included by
// one translation unit per dtype so the three instantiation sets compile in
// parallel.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "kernels.cuh"

namespace amped {

constexpr int kMaxDevices = 64;

// Launch state of one kernel instantiation, kept per device: the grid size
// (resident blocks x SMs of that device) and whether the carveout attribute
// has been set there.  Threads racing on the first launch compute the same
// value, so a relaxed atomic store is enough.
struct PerDeviceGrid {
    std::atomic<int> grid[kMaxDevices];
    template <class Init>
    int get(Init init) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return init();
        int g = grid[dev].load(std::memory_order_relaxed);
        if (g == 0) {
            g = init();
            grid[dev].store(g, std::memory_order_relaxed);
        }
        return g;
    }
};

constexpr int kCarveoutPercentWide = 60;  // 32-byte records (4+ input modes): 4 blocks x 32 KB
constexpr int kCarveoutPercent = 30;  // ~68 KB of the 228 KB shared-memory maximum: 4 blocks x 16 KB

template <typename K>
static int blocks_per_sm(K kernel) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, 256, 0) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

static int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Vector width for a (dtype, R): 32-byte row slices when R allows, else scalar.
template <typename T>
struct Shape {
    static constexpr int kVec = 32 / (int)sizeof(T);
    static int vec(int R) { return (R % kVec == 0 && R <= 32 * kVec) ? kVec : (R <= 32 ? 1 : 0); }
    // Lanes per worker: a power of two >= 2 (the rowptr window of a worker
    // must hold rows i and i+1 after a reload at i & ~3, which needs 8 entries).
    static int lpn(int R, int vec) {
        int need = (R + vec - 1) / vec, l = 2;
        while (l < need) l <<= 1;
        return vec == 1 ? 32 : l;
    }
};

template <typename T, int VEC, int LPN, int NIN, bool RES>
static int launch_mttkrp_shape(const MttkrpParams& p, int grid_cap, cudaStream_t st) {
    auto k = mttkrp_kernel<T, VEC, LPN, NIN, RES>;
    static PerDeviceGrid grid;  // persistent grid: every resident block slot on every SM
    int g = grid.get([&] {
        // The kernel needs little shared memory (the staged stream batches);
        // ask for the smallest carveout so the rest of the SM's 256 KB stays L1
        // cache for the factor-row gathers.  The attribute is per device.
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             NIN > 3 ? kCarveoutPercentWide : kCarveoutPercent);
        return blocks_per_sm(k) * device_sms();
    });
    if (grid_cap > 0 && g > grid_cap) g = grid_cap;
    k<<<g, 256, 0, st>>>(p);
    return (int)cudaGetLastError();
}

template <typename T, int VEC, int NIN, bool RES>
static int launch_mttkrp_lpn(int lpn, const MttkrpParams& p, int grid_cap, cudaStream_t st) {
    if constexpr (VEC == 1) {
        return launch_mttkrp_shape<T, 1, 32, NIN, RES>(p, grid_cap, st);
    } else {
        switch (lpn) {
            case 2: return launch_mttkrp_shape<T, VEC, 2, NIN, RES>(p, grid_cap, st);
            case 4: return launch_mttkrp_shape<T, VEC, 4, NIN, RES>(p, grid_cap, st);
            case 8: return launch_mttkrp_shape<T, VEC, 8, NIN, RES>(p, grid_cap, st);
            case 16: return launch_mttkrp_shape<T, VEC, 16, NIN, RES>(p, grid_cap, st);
            default: return launch_mttkrp_shape<T, VEC, 32, NIN, RES>(p, grid_cap, st);
        }
    }
}

template <typename T, int VEC, bool RES>
static int launch_mttkrp_nin(int nin, int lpn, const MttkrpParams& p, int grid_cap, cudaStream_t st) {
    switch (nin) {
        case 1: return launch_mttkrp_lpn<T, VEC, 1, RES>(lpn, p, grid_cap, st);
        case 2: return launch_mttkrp_lpn<T, VEC, 2, RES>(lpn, p, grid_cap, st);
        case 3: return launch_mttkrp_lpn<T, VEC, 3, RES>(lpn, p, grid_cap, st);
        case 4: return launch_mttkrp_lpn<T, VEC, 4, RES>(lpn, p, grid_cap, st);
        case 5: return launch_mttkrp_lpn<T, VEC, 5, RES>(lpn, p, grid_cap, st);
        case 6: return launch_mttkrp_lpn<T, VEC, 6, RES>(lpn, p, grid_cap, st);
        case 7: return launch_mttkrp_lpn<T, VEC, 7, RES>(lpn, p, grid_cap, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

template <typename T, bool RES>
static int launch_mttkrp_t(int nin, const MttkrpParams& p, int grid_cap, cudaStream_t st) {
    const int vec = Shape<T>::vec(p.R);
    const int lpn = Shape<T>::lpn(p.R, vec);
    if (vec == Shape<T>::kVec) return launch_mttkrp_nin<T, Shape<T>::kVec, RES>(nin, lpn, p, grid_cap, st);
    if (vec == 1) return launch_mttkrp_nin<T, 1, RES>(nin, lpn, p, grid_cap, st);
    return (int)cudaErrorInvalidValue;
}

template <typename T, int VEC, int LPN, int NM>
static int launch_sample_shape(const SampleParams& p, cudaStream_t st) {
    auto k = sample_kernel<T, VEC, LPN, NM>;
    static PerDeviceGrid grids;
    const int grid = grids.get([&] { return blocks_per_sm(k) * device_sms(); });
    const int64_t workers_needed = ((int64_t)p.nnz + 4 * LPN - 1) / (4 * LPN);
    int64_t g = (workers_needed * LPN + 255) / 256;
    if (g > grid) g = grid;
    if (g < 1) g = 1;
    k<<<(int)g, 256, 0, st>>>(p);
    return (int)cudaGetLastError();
}

template <typename T, int VEC, int NM>
static int launch_sample_lpn(int lpn, const SampleParams& p, cudaStream_t st) {
    if constexpr (VEC == 1) {
        return launch_sample_shape<T, 1, 32, NM>(p, st);
    } else {
        switch (lpn) {
            case 2: return launch_sample_shape<T, VEC, 2, NM>(p, st);
            case 4: return launch_sample_shape<T, VEC, 4, NM>(p, st);
            case 8: return launch_sample_shape<T, VEC, 8, NM>(p, st);
            case 16: return launch_sample_shape<T, VEC, 16, NM>(p, st);
            default: return launch_sample_shape<T, VEC, 32, NM>(p, st);
        }
    }
}

template <typename T, int VEC>
static int launch_sample_nm(int lpn, const SampleParams& p, cudaStream_t st) {
    switch (p.nmodes) {
        case 2: return launch_sample_lpn<T, VEC, 2>(lpn, p, st);
        case 3: return launch_sample_lpn<T, VEC, 3>(lpn, p, st);
        case 4: return launch_sample_lpn<T, VEC, 4>(lpn, p, st);
        case 5: return launch_sample_lpn<T, VEC, 5>(lpn, p, st);
        case 6: return launch_sample_lpn<T, VEC, 6>(lpn, p, st);
        case 7: return launch_sample_lpn<T, VEC, 7>(lpn, p, st);
        case 8: return launch_sample_lpn<T, VEC, 8>(lpn, p, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

template <typename T>
static int launch_sample_t(const SampleParams& p, cudaStream_t st) {
    const int vec = Shape<T>::vec(p.R);
    const int lpn = Shape<T>::lpn(p.R, vec);
    if (vec == Shape<T>::kVec) return launch_sample_nm<T, Shape<T>::kVec>(lpn, p, st);
    if (vec == 1) return launch_sample_nm<T, 1>(lpn, p, st);
    return (int)cudaErrorInvalidValue;
}

}  // namespace amped

// Two translation units per dtype (compiled in parallel): the MTTKRP and
// sampled-model launchers, and the residual (completion-gradient) launcher.
#define AMPED_DEFINE_DTYPE_LAUNCHERS(T, SUFFIX)                                                               \
    namespace amped {                                                                                       \
    int launch_mttkrp_##SUFFIX(int nin, const MttkrpParams& p, int grid_cap, void* st) {                    \
        return launch_mttkrp_t<T, false>(nin, p, grid_cap, static_cast<cudaStream_t>(st));                 \
    }                                                                                                       \
    int launch_sample_##SUFFIX(const SampleParams& p, void* st) {                                           \
        return launch_sample_t<T>(p, static_cast<cudaStream_t>(st));                                        \
    }                                                                                                       \
    int vec_##SUFFIX(int R) { return Shape<T>::vec(R); }                                                    \
    }
#define AMPED_DEFINE_DTYPE_RESIDUAL_LAUNCHER(T, SUFFIX)                                                       \
    namespace amped {                                                                                       \
    int launch_residual_##SUFFIX(int nin, const MttkrpParams& p, int grid_cap, void* st) {                  \
        return launch_mttkrp_t<T, true>(nin, p, grid_cap, static_cast<cudaStream_t>(st));                  \
    }                                                                                                       \
    }
