// amped_internal.h — structures shared by the host reorder, the C ABI and the
// CUDA kernels of the GB300 sparse MTTKRP library.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/amped.h"

namespace amped {

constexpr int kMaxIn = AMPED_MAX_MODES - 1;  // input modes of one MTTKRP
constexpr int kPad = 256;                    // elements of slack after every stream array
constexpr int kCombineSlots = 32;            // partial slots summed by one combine task

// ---------------------------------------------------------------------------
// Host side: one mode-ordered copy, as built by the reorder (reorder.cpp).
// ---------------------------------------------------------------------------
template <class T>
struct HostBuf {  // malloc-backed array without value-initialisation
    T* p = nullptr;
    size_t n = 0;
    HostBuf() = default;
    HostBuf(const HostBuf&) = delete;
    HostBuf& operator=(const HostBuf&) = delete;
    ~HostBuf() { release(); }
    bool alloc(size_t count);
    void release();
    T& operator[](size_t i) { return p[i]; }
    const T& operator[](size_t i) const { return p[i]; }
};

struct SplitRow {
    int32_t row;   // output row straddling segment boundaries s_a..s_b
    int32_t s_a;   // first straddled boundary (the row starts in segment s_a-1)
    int32_t s_b;   // last straddled boundary (the row ends in segment s_b)
};

struct HostMode {
    int mode = 0;
    int64_t I = 0;                 // rows of this mode
    int64_t nnz = 0;
    HostBuf<int32_t> perm;         // [nnz]  caller index of the k-th nonzero in mode order
    HostBuf<int32_t> rowptr;       // [I+1]  row i owns nonzeros rowptr[i]..rowptr[i+1]-1
    HostBuf<int32_t> seg_row;      // [S+1]  merge-path split points: rows completed before segment s
    HostBuf<int32_t> seg_nz;       // [S+1]  nonzeros consumed before segment s
    int32_t S = 0;                 // segments
    HostBuf<SplitRow> splits;      // rows that straddle a segment boundary
    int32_t nsplit = 0;
    HostBuf<int32_t> tasks;        // [ntask][4] {split id, s_lo, s_hi (exclusive), first-slot-is-tail}
    int32_t ntask = 0;
    HostBuf<int32_t> split_info;   // [nsplit+1][2] {row, first task}; sentinel holds ntask
    HostBuf<int32_t> multi;        // split ids with more than one task
    int32_t nmulti = 0;
};

// Validates coordinates; returns the first offending nonzero or -1.
int64_t find_bad_index(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int threads);

// Stable order of the nonzeros by coordinate `mode` (two-level counting sort,
// parallel) into hm.perm / hm.rowptr.  The sequence sorted is the caller
// order, or `order[0..nnz)` when given (so sorting by a secondary key first
// gives a lexicographic order).  Returns false on allocation failure.
bool sort_mode(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int mode, int threads,
               HostMode& hm, const int32_t* order = nullptr);

// The other mode whose coordinate orders nonzeros inside a row (largest dim), or -1.
int inner_mode(int nmodes, const int64_t* dims, int mode);
// Mode order: by i_mode, and inside a row by the inner mode's coordinate when
// inner_sort is set (caller order otherwise); both stable.
bool order_mode(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int mode, bool inner_sort,
                int threads, HostMode& hm);

// Cuts the mode-ordered copy into merge-path segments of at most `items`
// work items (nonzeros + row ends) and derives the split-row combine tasks.
bool cut_segments(HostMode& hm, int items);

// Struct-of-arrays columns of a mode-ordered copy:
//   dst[k] = idx[perm[k]][src_mode]   and   dst[k] = vals[perm[k]]
void gather_column(const HostMode& hm, int nmodes, const int32_t* idx, int src_mode, int32_t* dst, int threads);
void gather_values(const HostMode& hm, const float* vals, float* dst, int threads);
// Caller-order column: dst[k] = idx[k][mode].
void caller_column(int64_t nnz, int nmodes, const int32_t* idx, int mode, int32_t* dst, int threads);

// ---------------------------------------------------------------------------
// Device side.
// ---------------------------------------------------------------------------
struct MttkrpParams {
    const int32_t* rowptr;       // [I+1] (+ slack)
    const int32_t* idx[kMaxIn];  // input-mode coordinate streams in mode order (+ slack)
    const void* fac[kMaxIn];     // input-mode factors [dims][R]
    const float* val;            // values in mode order (+ slack); unused when perm != nullptr
    const int32_t* perm;         // gradient path: mode order -> caller order (+ slack)
    const float* gval;           // gradient path: per-nonzero values in caller order
    const int32_t* seg_row;      // [S+1]
    const int32_t* seg_nz;       // [S+1]
    float* out;                  // [I][R]
    float* part;                 // [S][2][R] head/tail partials of split rows
    int* queue;                  // segment ticket counter, zero at launch
    int32_t I, S, R, nnz;
};

struct CombineParams {
    const int32_t* tasks;       // [ntask][4]
    const int32_t* split_info;  // [nsplit+1][2]
    const int32_t* multi;       // [nmulti]
    const float* part;          // [S][2][R]
    double* tsum;               // [ntask][R]
    float* out;                 // [I][R]
    int32_t ntask, nmulti, R;
};

struct SampleParams {
    const int32_t* idx[AMPED_MAX_MODES];  // caller-order coordinates (+ slack)
    const void* fac[AMPED_MAX_MODES];
    float* m;                             // [nnz] (+ slack for the vector store)
    int32_t nnz, R, nmodes;
};

// Split-row combine launcher (combine.cu).  Returns a cudaError_t value as
// int, counts the kernels it launched, never synchronises.
int launch_combine(const CombineParams& p, void* stream, int* launched);

}  // namespace amped
