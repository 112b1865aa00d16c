// reorder.cpp — host preprocessing: per-mode output-row order and the
// segment table (paper Sec. 3.1 tensor sharding, Sec. 3.2 inter-shard
// partitioning, Sec. 4.2 partition-to-threadblock mapping).
//
// The paper groups all nonzeros sharing an output index into one shard so no
// two GPUs update the same row, and cuts each shard into equal-size
// partitions, one per threadblock, with atomics between them.  On one GPU the
// whole tensor is one shard; it is ordered by the output coordinate (a stable
// counting sort) and cut into segments of equal *work*: the merge-path split
// of the sequence "nonzeros of row 0, end of row 0, nonzeros of row 1, ..."
// into pieces of `items` items.  A segment therefore holds at most `items`
// nonzeros and at most `items` row ends, so empty rows (which must still be
// written as zero) and rows longer than a segment are both balanced.  Rows
// that straddle a segment boundary are the only ones written by more than one
// segment; they are listed as split rows and combined deterministically.
#include <omp.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "amped_internal.h"

namespace amped {

template <class T>
bool HostBuf<T>::alloc(size_t count) {
    release();
    p = static_cast<T*>(std::malloc(std::max<size_t>(count, 1) * sizeof(T)));
    n = p ? count : 0;
    return p != nullptr;
}
template <class T>
void HostBuf<T>::release() {
    std::free(p);
    p = nullptr;
    n = 0;
}
template struct HostBuf<int32_t>;
template struct HostBuf<int64_t>;
template struct HostBuf<SplitRow>;
template struct HostBuf<float>;

static int nthreads(int threads) { return threads > 0 ? threads : omp_get_max_threads(); }

int64_t find_bad_index(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int threads) {
    int64_t first = -1;
    const int T = nthreads(threads);
#pragma omp parallel num_threads(T)
    {
        int64_t mine = -1;
#pragma omp for schedule(static)
        for (int64_t k = 0; k < nnz; ++k) {
            if (mine >= 0) continue;
            for (int n = 0; n < nmodes; ++n) {
                int32_t c = idx[k * nmodes + n];
                if (c < 0 || c >= dims[n]) {
                    mine = k;
                    break;
                }
            }
        }
#pragma omp critical
        if (mine >= 0 && (first < 0 || mine < first)) first = mine;
    }
    return first;
}

bool sort_mode(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int mode, int threads,
               HostMode& hm, const int32_t* order) {
    const int64_t I = dims[mode];
    hm.mode = mode;
    hm.I = I;
    hm.nnz = nnz;
    if (!hm.perm.alloc((size_t)nnz) || !hm.rowptr.alloc((size_t)I + 1)) return false;
    const int T = nthreads(threads);

    // the sequence being sorted (caller indices 0..nnz-1, or `order` when given) and its
    // keys, gathered once so that every later pass reads them contiguously
    HostBuf<int32_t> key, tkey, tmp;
    if (!key.alloc((size_t)nnz) || !tkey.alloc((size_t)nnz) || !tmp.alloc((size_t)nnz)) return false;
#pragma omp parallel for schedule(static) num_threads(T)
    for (int64_t j = 0; j < nnz; ++j) key[(size_t)j] = idx[(order ? (int64_t)order[j] : j) * nmodes + mode];

    // level 1: bucket by the high bits of the key, at most 2^16 buckets
    int bits = 0;
    while ((int64_t(1) << bits) < I) ++bits;
    const int shift = bits > 16 ? bits - 16 : 0;
    const int64_t B = ((I - 1) >> shift) + 1;
    std::vector<int64_t> hist((size_t)T * (size_t)B, 0);
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const int64_t lo = nnz * t / T, hi = nnz * (t + 1) / T;
        int64_t* h = hist.data() + (size_t)t * B;
        for (int64_t j = lo; j < hi; ++j) ++h[key[(size_t)j] >> shift];
    }
    // exclusive scan in (bucket, thread) order keeps the scatter stable
    std::vector<int64_t> bstart((size_t)B + 1);
    int64_t run = 0;
    for (int64_t b = 0; b < B; ++b) {
        bstart[b] = run;
        for (int t = 0; t < T; ++t) {
            int64_t c = hist[(size_t)t * B + b];
            hist[(size_t)t * B + b] = run;
            run += c;
        }
    }
    bstart[B] = run;
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const int64_t lo = nnz * t / T, hi = nnz * (t + 1) / T;
        int64_t* off = hist.data() + (size_t)t * B;
        for (int64_t j = lo; j < hi; ++j) {
            const int32_t kv = key[(size_t)j];
            const int64_t dst = off[kv >> shift]++;
            tmp[(size_t)dst] = order ? order[j] : (int32_t)j;
            tkey[(size_t)dst] = kv;
        }
    }
    // level 2: stable counting sort of each bucket by the low bits; fills rowptr
    const int64_t span = int64_t(1) << shift;
#pragma omp parallel num_threads(T)
    {
        std::vector<int64_t> cnt((size_t)span + 1);
#pragma omp for schedule(dynamic, 16)
        for (int64_t b = 0; b < B; ++b) {
            const int64_t k0 = bstart[b], k1 = bstart[b + 1];
            const int64_t key0 = b << shift, nkeys = std::min(span, I - key0);
            std::fill(cnt.begin(), cnt.begin() + nkeys + 1, 0);
            for (int64_t j = k0; j < k1; ++j) ++cnt[(size_t)(tkey[(size_t)j] - key0) + 1];
            for (int64_t x = 0; x < nkeys; ++x) {
                cnt[(size_t)x + 1] += cnt[(size_t)x];
                hm.rowptr[(size_t)(key0 + x)] = (int32_t)(k0 + cnt[(size_t)x]);
            }
            for (int64_t j = k0; j < k1; ++j)
                hm.perm[(size_t)(k0 + cnt[(size_t)(tkey[(size_t)j] - key0)]++)] = tmp[(size_t)j];
        }
    }
    hm.rowptr[(size_t)I] = (int32_t)nnz;
    return true;
}

void mode_priority(int nmodes, const int64_t* dims, int* prio, bool ascending) {
    for (int n = 0; n < nmodes; ++n) prio[n] = n;
    if (ascending)
        std::stable_sort(prio, prio + nmodes, [&](int a, int b) { return dims[a] < dims[b]; });
    else
        std::stable_sort(prio, prio + nmodes, [&](int a, int b) { return dims[a] > dims[b]; });
}

bool lex_order(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int threads, HostBuf<int32_t>& out,
               bool ascending) {
    int prio[AMPED_MAX_MODES];
    mode_priority(nmodes, dims, prio, ascending);
    // least significant key first; every pass is stable, so ties keep the earlier passes' order
    HostMode cur, prev;
    for (int p = nmodes - 1; p >= 0; --p) {
        if (!sort_mode(nnz, nmodes, dims, idx, prio[p], threads, cur, p == nmodes - 1 ? nullptr : prev.perm.p))
            return false;
        std::swap(cur.perm.p, prev.perm.p);
        std::swap(cur.perm.n, prev.perm.n);
    }
    std::swap(out.p, prev.perm.p);
    std::swap(out.n, prev.perm.n);
    return true;
}

bool order_mode(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int mode, const int32_t* lex,
                int threads, HostMode& hm) {
    return sort_mode(nnz, nmodes, dims, idx, mode, threads, hm, lex);
}

bool classify_rows(HostMode& hm, int threshold, int threads) {
    const int64_t I = hm.I;
    const int32_t* rp = hm.rowptr.p;
    const int T = nthreads(threads);
    const int64_t thr = threshold > 0 ? threshold : 1;
    // count classes and short-row lengths (short lengths are < thr)
    int64_t L = 0, nnz_L = 0;
    std::vector<int64_t> cnt((size_t)thr, 0);
    for (int64_t i = 0; i < I; ++i) {
        const int64_t len = (int64_t)rp[i + 1] - rp[i];
        if (len >= thr) {
            ++L;
            nnz_L += len;
        } else {
            ++cnt[(size_t)len];
        }
    }
    const int64_t Sr = I - L;
    hm.L = (int32_t)L;
    hm.nnz_L = nnz_L;
    hm.Sr = (int32_t)Sr;
    if (!hm.rows_L.alloc((size_t)L) || !hm.rowptr_L.alloc((size_t)L + 1) || !hm.rows_S.alloc((size_t)Sr) ||
        !hm.rowptr_S.alloc((size_t)Sr + 1))
        return false;
    // short rows by decreasing length, ties by increasing id (counting sort)
    std::vector<int64_t> start((size_t)thr, 0);
    int64_t run = 0;
    for (int64_t len = thr - 1; len >= 0; --len) {
        start[(size_t)len] = run;
        run += cnt[(size_t)len];
    }
    int64_t jl = 0;
    hm.rowptr_L[0] = 0;
    for (int64_t i = 0; i < I; ++i) {
        const int64_t len = (int64_t)rp[i + 1] - rp[i];
        if (len >= thr) {
            hm.rows_L[(size_t)jl] = (int32_t)i;
            hm.rowptr_L[(size_t)jl + 1] = (int32_t)(hm.rowptr_L[(size_t)jl] + len);
            ++jl;
        } else {
            hm.rows_S[(size_t)start[(size_t)len]++] = (int32_t)i;
        }
    }
    hm.rowptr_S[0] = (int32_t)nnz_L;
    for (int64_t j = 0; j < Sr; ++j) {
        const int32_t r = hm.rows_S[(size_t)j];
        hm.rowptr_S[(size_t)j + 1] = hm.rowptr_S[(size_t)j] + (rp[r + 1] - rp[r]);
    }
    // the copy's order: long rows, then short rows
    HostBuf<int32_t> np;
    if (!np.alloc((size_t)hm.nnz)) return false;
#pragma omp parallel for schedule(dynamic, 4096) num_threads(T)
    for (int64_t j = 0; j < L; ++j) {
        const int32_t r = hm.rows_L[(size_t)j];
        std::memcpy(np.p + hm.rowptr_L[(size_t)j], hm.perm.p + rp[r], (size_t)(rp[r + 1] - rp[r]) * 4);
    }
#pragma omp parallel for schedule(dynamic, 4096) num_threads(T)
    for (int64_t j = 0; j < Sr; ++j) {
        const int32_t r = hm.rows_S[(size_t)j];
        if (rp[r + 1] > rp[r])
            std::memcpy(np.p + hm.rowptr_S[(size_t)j], hm.perm.p + rp[r], (size_t)(rp[r + 1] - rp[r]) * 4);
    }
    std::swap(hm.perm.p, np.p);
    std::swap(hm.perm.n, np.n);
    return true;
}

bool cut_segments(HostMode& hm, int items) {
    // ---- long part: merge path over the long rows
    const int64_t I = hm.L, nnz = hm.nnz_L, total = I + nnz;
    const int64_t S = (total + items - 1) / items;
    hm.S = (int32_t)S;
    if (!hm.seg_row.alloc((size_t)S + 1) || !hm.seg_nz.alloc((size_t)S + 1)) return false;
    const int32_t* rp = hm.rowptr_L.p;
    // Boundary d = s*items on the merge path: the end of long row i sits at position
    // rowptr_L[i+1] + i; the rows completed before d are those whose end lies
    // before d, found by binary search; the rest of d counts consumed nonzeros.
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s <= S; ++s) {
        const int64_t d = std::min(total, s * (int64_t)items);
        int64_t lo = 0, hi = I;  // first row whose end position is >= d
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if ((int64_t)rp[mid + 1] + mid < d) lo = mid + 1; else hi = mid;
        }
        hm.seg_row[(size_t)s] = (int32_t)lo;
        hm.seg_nz[(size_t)s] = (int32_t)(d - lo);
    }
    // split rows: boundary s is straddled when its row started before it
    std::vector<SplitRow> sp;
    for (int64_t s = 1; s < S; ++s) {
        const int32_t r = hm.seg_row[(size_t)s];
        if (r >= I || hm.seg_nz[(size_t)s] <= rp[r]) continue;
        if (!sp.empty() && sp.back().row == r && sp.back().s_b == s - 1)
            sp.back().s_b = (int32_t)s;
        else
            sp.push_back({r, (int32_t)s, (int32_t)s});
    }
    hm.nsplit = (int32_t)sp.size();
    if (!hm.splits.alloc(sp.size())) return false;
    if (!sp.empty()) std::memcpy(hm.splits.p, sp.data(), sp.size() * sizeof(SplitRow));
    // combine tasks: the slots of split row j are T[s_a-1], H[s_a], ..., H[s_b],
    // cut into runs of at most kCombineSlots consecutive segments; split_info
    // carries the output row id
    std::vector<int32_t> tasks, info, multi;
    for (int32_t j = 0; j < hm.nsplit; ++j) {
        const SplitRow& r = sp[(size_t)j];
        info.push_back(hm.rows_L[(size_t)r.row]);
        info.push_back((int32_t)(tasks.size() / 4));
        int32_t nt = 0;
        for (int32_t lo = r.s_a - 1; lo <= r.s_b; lo += kCombineSlots, ++nt) {
            tasks.push_back(j);
            tasks.push_back(lo);
            tasks.push_back(std::min(lo + kCombineSlots, r.s_b + 1));
            tasks.push_back(lo == r.s_a - 1 ? 1 : 0);
        }
        if (nt > 1) multi.push_back(j);
    }
    info.push_back(0);
    info.push_back((int32_t)(tasks.size() / 4));
    hm.ntask = (int32_t)(tasks.size() / 4);
    hm.nmulti = (int32_t)multi.size();
    if (!hm.tasks.alloc(tasks.size()) || !hm.split_info.alloc(info.size()) || !hm.multi.alloc(multi.size()))
        return false;
    if (!tasks.empty()) std::memcpy(hm.tasks.p, tasks.data(), tasks.size() * 4);
    std::memcpy(hm.split_info.p, info.data(), info.size() * 4);
    if (!multi.empty()) std::memcpy(hm.multi.p, multi.data(), multi.size() * 4);

    // ---- short part: greedy runs of short rows
    std::vector<int32_t> ss;
    int64_t j = 0;
    while (j < hm.Sr) {
        ss.push_back((int32_t)j);
        const int64_t k0 = hm.rowptr_S[(size_t)j];
        int64_t e = j;
        while (e < hm.Sr && e - j < kShortRows && hm.rowptr_S[(size_t)e + 1] - k0 <= kShortNnz) ++e;
        j = e;
    }
    ss.push_back((int32_t)hm.Sr);
    hm.S_S = (int32_t)ss.size() - 1;
    if (!hm.seg_short.alloc(ss.size())) return false;
    std::memcpy(hm.seg_short.p, ss.data(), ss.size() * 4);
    return true;
}

void gather_column(const HostMode& hm, int nmodes, const int32_t* idx, int src_mode, int32_t* dst, int threads) {
    const int T = nthreads(threads);
#pragma omp parallel for schedule(static) num_threads(T)
    for (int64_t k = 0; k < hm.nnz; ++k) dst[k] = idx[(int64_t)hm.perm[(size_t)k] * nmodes + src_mode];
}

void gather_copy(const HostMode& hm, int nmodes, const int32_t* idx, const float* vals, int nin, const int* slot_mode,
                 int32_t* const* cols, float* dvals, int threads) {
    const int T = nthreads(threads);
#pragma omp parallel for schedule(static) num_threads(T)
    for (int64_t k = 0; k < hm.nnz; ++k) {
        const int64_t src = hm.perm[(size_t)k];
        const int32_t* rec = idx + src * nmodes;
        for (int s = 0; s < nin; ++s) cols[s][k] = rec[slot_mode[s]];
        dvals[k] = vals[src];
    }
}

void gather_values(const HostMode& hm, const float* vals, float* dst, int threads) {
    const int T = nthreads(threads);
#pragma omp parallel for schedule(static) num_threads(T)
    for (int64_t k = 0; k < hm.nnz; ++k) dst[k] = vals[hm.perm[(size_t)k]];
}

void caller_column(int64_t nnz, int nmodes, const int32_t* idx, int mode, int32_t* dst, int threads) {
    const int T = nthreads(threads);
#pragma omp parallel for schedule(static) num_threads(T)
    for (int64_t k = 0; k < nnz; ++k) dst[k] = idx[k * nmodes + mode];
}

double norm2_merged(const HostMode& hm, int nmodes, const int32_t* idx, const float* vals, bool lex_sorted,
                    int threads) {
    const int T = nthreads(threads);
    constexpr int64_t kRowsPerChunk = 4096;
    const int64_t nch = (hm.I + kRowsPerChunk - 1) / kRowsPerChunk;
    std::vector<double> part;
    try {
        part.assign((size_t)nch, 0.0);
    } catch (...) {
        return -1.0;
    }
    auto same = [&](int32_t x, int32_t y) {
        for (int n = 0; n < nmodes; ++n)
            if (idx[(int64_t)x * nmodes + n] != idx[(int64_t)y * nmodes + n]) return false;
        return true;
    };
    auto less = [&](int32_t x, int32_t y) {
        for (int n = 0; n < nmodes; ++n) {
            const int32_t a = idx[(int64_t)x * nmodes + n], b = idx[(int64_t)y * nmodes + n];
            if (a != b) return a < b;
        }
        return false;
    };
    bool failed = false;
#pragma omp parallel num_threads(T)
    {
        std::vector<int32_t> run;
#pragma omp for schedule(dynamic, 1)
        for (int64_t c = 0; c < nch; ++c) {
            double s = 0.0;
            const int64_t i_end = std::min<int64_t>(hm.I, (c + 1) * kRowsPerChunk);
            for (int64_t i = c * kRowsPerChunk; i < i_end; ++i) {
                const int64_t a = hm.rowptr[(size_t)i], b = hm.rowptr[(size_t)i + 1];
                if (lex_sorted) {  // repeated coordinates are adjacent: sum each run in copy order
                    for (int64_t j = a; j < b;) {
                        double v = 0.0;
                        int64_t q = j;
                        while (q < b && same(hm.perm[(size_t)q], hm.perm[(size_t)j])) v += vals[hm.perm[(size_t)q++]];
                        s += v * v;
                        j = q;
                    }
                    continue;
                }
                if (b - a == 1) {
                    const double v = vals[hm.perm[(size_t)a]];
                    s += v * v;
                    continue;
                }
                if (b == a) continue;
                try {
                    run.assign(hm.perm.p + a, hm.perm.p + b);
                } catch (...) {
#pragma omp atomic write
                    failed = true;
                    continue;
                }
                std::stable_sort(run.begin(), run.end(), less);  // equal coordinates keep copy order
                for (size_t j = 0; j < run.size();) {
                    double v = 0.0;
                    size_t q = j;
                    while (q < run.size() && same(run[q], run[j])) v += vals[run[q++]];
                    s += v * v;
                    j = q;
                }
            }
            part[(size_t)c] = s;
        }
    }
    if (failed) return -1.0;
    double total = 0.0;
    for (double v : part) total += v;  // fixed chunk order
    return total;
}

}  // namespace amped
