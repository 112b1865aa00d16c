// amped_internal.h — structures shared by the host reorder, the C ABI and the
// CUDA kernels of the GB300 sparse MTTKRP library.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/amped.h"

// Checked builds (nvcc -DAMPED_CHECKS=1): the MTTKRP and sampled-model kernels
// check every gather coordinate, output row id, stream position and row-table
// window against its array, record the first failed check in the handle's
// device error word and clamp the access in bounds; the entry point then waits
// for the stream and returns AMPED_ERR_INDEX.  Off (0) in the default build.
#ifndef AMPED_CHECKS
#define AMPED_CHECKS 0
#endif

namespace amped {

constexpr int kMaxIn = AMPED_MAX_MODES - 1;  // input modes of one MTTKRP

// Failed-check codes in err[0] (err[1] = the offending index, err[2] = slot or mode).
enum CheckCode : int32_t {
    kCheckCoord = 1,    // gather coordinate outside its factor's rows
    kCheckOutRow = 2,   // output row id outside the output mode's rows
    kCheckStream = 3,   // stream position beyond the copy's arrays
    kCheckRowptr = 4,   // row-table window beyond the long rows' table
    kCheckShort = 5,    // short segment wider than one staged batch
};
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
    HostBuf<int32_t> perm;         // [nnz]  caller index of the k-th nonzero of the copy
    HostBuf<int32_t> rowptr;       // [I+1]  before classify_rows: row i owns perm[rowptr[i] .. rowptr[i+1])
    // After classify_rows the copy holds the long rows (>= threshold nonzeros, by
    // increasing row id) first and then the short rows (by decreasing length).
    int32_t L = 0;                 // long rows
    int64_t nnz_L = 0;             // their nonzeros (copy positions 0 .. nnz_L)
    HostBuf<int32_t> rows_L;       // [L]    row ids
    HostBuf<int32_t> rowptr_L;     // [L+1]  copy positions of long row j: rowptr_L[j] .. rowptr_L[j+1]
    int32_t Sr = 0;                // short rows (including rows without nonzeros)
    HostBuf<int32_t> rows_S;       // [Sr]   row ids
    HostBuf<int32_t> rowptr_S;     // [Sr+1] copy positions (rowptr_S[0] = nnz_L)
    HostBuf<int32_t> seg_short;    // [S_S+1] short-row index where short segment t starts
    int32_t S_S = 0;               // short segments
    HostBuf<int32_t> seg_row;      // [S+1]  long merge path: long rows completed before segment s
    HostBuf<int32_t> seg_nz;       // [S+1]  nonzeros consumed before segment s
    int32_t S = 0;                 // long segments
    HostBuf<SplitRow> splits;      // long rows (long-row index) that straddle a segment boundary
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

// Priority of the coordinates in the inner order: modes by decreasing
// dimension (by increasing dimension when `ascending`), ties by increasing mode
// index (prio[0] is the most significant).
void mode_priority(int nmodes, const int64_t* dims, int* prio, bool ascending = false);
// Caller indices in lexicographic order of all N coordinates, most significant
// (highest priority) first; ties keep caller order.  One stable counting sort
// per mode, least significant first.  Returns false on allocation failure.
bool lex_order(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int threads, HostBuf<int32_t>& out,
               bool ascending = false);
// Mode order: by i_mode; inside a row in the order of `lex` (the lexicographic
// order from lex_order, which orders a row by the other coordinates in priority
// order), or in caller order when lex is null.  Stable.
bool order_mode(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int mode, const int32_t* lex,
                int threads, HostMode& hm);

// Splits the rows into long rows (at least `threshold` nonzeros; threshold
// <= 0 makes every non-empty row long) and short rows, and rebuilds hm.perm as
// [long rows in row-id order][short rows by decreasing length, ties by id].
bool classify_rows(HostMode& hm, int threshold, int threads);

// Most rows and nonzeros in one short segment: a short segment's nonzeros are
// staged in one 128-entry batch, which starts up to 3 entries early.
constexpr int kShortRows = 31;
constexpr int kShortNnz = 124;

// Cuts the long part into merge-path segments of at most `items` work items
// (nonzeros + row ends) with the split-row combine tasks, and the short part
// into segments of at most kShortRows rows and kShortNnz nonzeros.
bool cut_segments(HostMode& hm, int items);

// Struct-of-arrays columns of a mode-ordered copy:
//   dst[k] = idx[perm[k]][src_mode]   and   dst[k] = vals[perm[k]]
void gather_column(const HostMode& hm, int nmodes, const int32_t* idx, int src_mode, int32_t* dst, int threads);
void gather_values(const HostMode& hm, const float* vals, float* dst, int threads);
// Every input slot's column and the values of a mode-ordered copy in one pass
// over the nonzeros (one visit of each nonzero's coordinate record):
// cols[s][k] = idx[perm[k]][slot_mode[s]], dvals[k] = vals[perm[k]].
void gather_copy(const HostMode& hm, int nmodes, const int32_t* idx, const float* vals, int nin, const int* slot_mode,
                 int32_t* const* cols, float* dvals, int threads);
// Caller-order column: dst[k] = idx[k][mode].
void caller_column(int64_t nnz, int nmodes, const int32_t* idx, int mode, int32_t* dst, int threads);

// ||X||^2 with repeated coordinates summed into one entry, from a copy ordered
// by order_mode (before classify_rows).  With lex_sorted (the copy follows the
// lexicographic order) repeated coordinates are adjacent inside a row;
// otherwise each row is sorted by the full coordinate first.  fp64, the same
// result for any thread count.  Returns a negative value on allocation failure.
double norm2_merged(const HostMode& hm, int nmodes, const int32_t* idx, const float* vals, bool lex_sorted,
                    int threads);

// ---------------------------------------------------------------------------
// Device side.
// ---------------------------------------------------------------------------
struct MttkrpParams {
    const int32_t* rowptr;       // [L+1] copy positions of the long rows (+ slack)
    const int32_t* rows_L;       // [L]   row ids of the long rows
    const int32_t* rowptr_S;     // [Sr+1] copy positions of the short rows (+ slack)
    const int32_t* rows_S;       // [Sr]  row ids of the short rows (+ slack)
    const int32_t* seg_short;    // [S_S+1] first short row of every short segment
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
    const void* fout;            // residual mode: the output mode's factor [rows][R]
    double* loss;                // residual mode: accumulates 1/2 sum (m - x)^2 (may be null)
    int32_t I, S, R, nnz;        // I: long rows; S: long segments
    int32_t S_S;                 // short segments (tickets S .. S+S_S-1)
    // used by checked builds only (AMPED_CHECKS)
    int32_t* err;                // [4] first failed check {code, index, slot, 0}
    int32_t fdim[kMaxIn];        // rows of each input slot's factor
    int32_t out_rows;            // rows of the output mode
    int64_t stride;              // elements per stream array
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
    // used by checked builds only (AMPED_CHECKS)
    int32_t* err;                         // [4] first failed check
    int32_t fdim[AMPED_MAX_MODES];        // rows of each factor
    int64_t stride;                       // elements per coordinate array
};

// One CP-ALS mode update (als.cu).
struct AlsParams {
    double* grams;       // [N][R][R] Grams of the current factors; row `mode` is replaced on success
    float* w;            // [R][R] V^-1, fp32 (workspace)
    double* ga;          // [R][R] Gram of the stored update, then (contiguous) ...
    double* ip;          // [R] ... sum_i M(i,r) A(i,r) of the stored update (workspace)
    int* info;           // 0, or the first failed Cholesky pivot + 1
    double* stats;       // [8] fit terms (written when `last` is set), failure counters
    double xnorm2;       // ||X||^2
    int32_t N, mode, R, last;  // last: compute the fit terms of the model after this update
};
int als_max_rank();
// G = A^T A (fp64; G is zeroed first) of a row-major [rows][R] fp32 matrix.
int launch_gram(const float* A, int64_t rows, int R, double* G, void* stream, int* launched);
// Cholesky solve: w = V^-1, info.
int launch_als_solve(const AlsParams& p, void* stream, int* launched);
// A = M W with its Gram and ip unless the solve failed, then the commit of the
// Gram and, after the last mode, the fit.
int launch_als_apply(const AlsParams& p, const float* M, int64_t rows, float* A, void* stream, int* launched);
// The tensor-core apply (als_tc.cu, tcgen05 3xTF32): the ranks it is built for,
// and its launch (same contract as launch_als_apply without the finish).
bool als_apply_tc_supported(int R);
int launch_als_apply_tc(const AlsParams& p, const float* M, int64_t rows, float* A, void* stream, int* launched);
// Unit-norm columns for every factor, lambda = product of the norms, Grams rescaled.
int launch_als_normalize(float* const* factors, const int64_t* dims, int N, int R, double* grams, float* lambda,
                         void* stream, int* launched);

// Split-row combine launcher (combine.cu).  Returns a cudaError_t value as
// int, counts the kernels it launched, never synchronises.
int launch_combine(const CombineParams& p, void* stream, int* launched);

}  // namespace amped
