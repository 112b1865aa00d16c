// api.cu — the C ABI (include/amped.h): handle construction, argument
// checking, scratch management and kernel dispatch.  Host code only; the
// kernels live in kernels.cuh (instantiated per dtype) and combine.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <omp.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "amped_internal.h"

namespace amped {
int launch_mttkrp_f32(int nin, const MttkrpParams& p, int grid_cap, void* st);
int launch_mttkrp_bf16(int nin, const MttkrpParams& p, int grid_cap, void* st);
int launch_mttkrp_f16(int nin, const MttkrpParams& p, int grid_cap, void* st);
int launch_residual_f32(int nin, const MttkrpParams& p, int grid_cap, void* st);
int launch_residual_bf16(int nin, const MttkrpParams& p, int grid_cap, void* st);
int launch_residual_f16(int nin, const MttkrpParams& p, int grid_cap, void* st);
int launch_sample_f32(const SampleParams& p, void* st);
int launch_sample_bf16(const SampleParams& p, void* st);
int launch_sample_f16(const SampleParams& p, void* st);
int vec_f32(int R);
int vec_bf16(int R);
int vec_f16(int R);
}  // namespace amped

using namespace amped;

namespace {

thread_local std::string g_err;
thread_local int64_t g_call_allocs = 0;  // device allocations made by the current entry-point call
std::atomic<int64_t> g_launches{0};

// Start of every entry point: clear the thread's error message and restart
// the per-call allocation count the fault injector uses.
void begin_call() {
    g_err.clear();
    g_call_allocs = 0;
}

amped_status fail(amped_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

amped_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? AMPED_ERR_OOM : AMPED_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// NVTX range over a host-side phase (the reorder, the uploads, each mode's
// launches), shown by Nsight Systems and Nsight Compute; without an attached
// tool the push and pop do nothing.
struct Range {
    explicit Range(const char* fmt, ...) {
        char buf[96];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        nvtxRangePushA(buf);
    }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// Host-side fault injection for testing clean-up paths: AMPED_FAULT=alloc:K
// makes the K-th device allocation (1-based) inside each entry-point call
// report failure, as cudaMalloc does when the device is out of memory.  The
// variable is read at every allocation, so a test can arm and disarm it
// between calls.
int64_t fault_alloc_at() {
    const char* s = std::getenv("AMPED_FAULT");
    if (!s || std::strncmp(s, "alloc:", 6) != 0) return 0;
    return (int64_t)std::atoll(s + 6);
}

// Scratch of amped_mttkrp_noalloc: one static device array per GPU.  Host
// code must not use this name as an address (on the host it is only a
// stand-in); the device address comes from cudaGetSymbolAddress, looked up
// once per device by noalloc_resolve with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[AMPED_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};
cudaError_t g_noalloc_err[kMaxDevices] = {};

// Looks up the array's address on `dev` (the current device) once.  Called by
// amped_tensor_create, so the array's module is loaded, and its memory
// reserved, when the first handle on a device is built rather than inside an
// allocation-free call.  A failed lookup is remembered and reported by
// amped_mttkrp_noalloc; it does not fail the handle.
void noalloc_resolve(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_addr[dev]) return;
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e == cudaSuccess && ptr) {
        g_noalloc_addr[dev] = ptr;
        g_noalloc_err[dev] = cudaSuccess;
    } else {
        g_noalloc_err[dev] = e == cudaSuccess ? cudaErrorInvalidSymbol : e;
        cudaGetLastError();  // the failure is reported by the allocation-free call, not left pending
    }
}

size_t esize(amped_dtype dt) { return dt == AMPED_F32 ? 4 : 2; }

int kernel_vec(amped_dtype dt, int R) {
    switch (dt) {
        case AMPED_F32: return vec_f32(R);
        case AMPED_BF16: return vec_bf16(R);
        case AMPED_F16: return vec_f16(R);
    }
    return 0;
}

struct DevMode {
    int64_t I = 0;      // rows of the mode
    int32_t L = 0;      // long rows
    int32_t S_S = 0;    // short segments
    int32_t S = 0, nsplit = 0, ntask = 0, nmulti = 0;
    int32_t* rowptr = nullptr;     // [L+1] copy positions of the long rows
    int32_t* rows_L = nullptr;     // [L] their row ids
    int32_t* rowptr_S = nullptr;   // [Sr+1] copy positions of the short rows
    int32_t* rows_S = nullptr;     // [Sr] their row ids
    int32_t* seg_short = nullptr;  // [S_S+1]
    int32_t* idx = nullptr;  // N-1 streams of `stride` elements
    float* val = nullptr;
    int32_t* perm = nullptr;
    int32_t* seg = nullptr;   // seg_row [S+1], then seg_nz [S+1]
    int32_t* table = nullptr; // tasks [4*ntask], split_info [2*(nsplit+1)], multi [nmulti]
    int slot_mode[AMPED_MAX_MODES] = {};  // input slot -> tensor mode; slot 0 is the inner-order mode
};

// Input slots of a mode copy.  With the lexicographic inner order: the other
// modes in priority order (decreasing dimension), which is the order the copy
// sorts a row by, so slot 0 changes least often along a row and the kernel's
// cached factor rows are reused longest.  Otherwise: increasing mode index.
int input_slots(int nmodes, const int64_t* dims, int mode, bool inner_sort, bool ascending, int* slot_mode) {
    int prio[AMPED_MAX_MODES];
    if (inner_sort) {
        mode_priority(nmodes, dims, prio, ascending);
    } else {
        for (int n = 0; n < nmodes; ++n) prio[n] = n;
    }
    int nin = 0;
    for (int p = 0; p < nmodes; ++p)
        if (prio[p] != mode) slot_mode[nin++] = prio[p];
    return nin;
}

}  // namespace

struct amped_tensor {
    int N = 0;
    int64_t nnz = 0;
    int64_t dims[AMPED_MAX_MODES] = {};
    int device = 0;
    int64_t stride = 0;  // elements per stream array, slack included
    DevMode m[AMPED_MAX_MODES];
    int32_t* coo = nullptr;  // caller-order coordinates, N streams of `stride`
    float* part = nullptr;   // [maxS][2][rcap]
    double* tsum = nullptr;  // [maxTask][rcap]
    int* queue = nullptr;
    int32_t* err = nullptr;  // checked builds: the kernels' failed-check word [4]
    int32_t maxS = 0, maxTask = 0, rcap = 0;
    void* ev_start = nullptr;
    void* ev_stop = nullptr;
    void* stage_fac[AMPED_MAX_MODES] = {};
    size_t stage_fac_bytes[AMPED_MAX_MODES] = {};
    float* stage_out[AMPED_MAX_MODES] = {};
    size_t stage_out_bytes[AMPED_MAX_MODES] = {};
    double xnorm2 = 0.0;        // ||X||^2, repeated coordinates summed
    float* als_m = nullptr;     // CP-ALS: MTTKRP output [max dim][als_rcap]
    double* als_gm = nullptr;   // CP-ALS: the update's Gram [R][R], then ip [R]
    float* als_w = nullptr;     // CP-ALS: solve output [R][R]
    int* als_info = nullptr;    // CP-ALS: solve status
    int als_rcap = 0;
    bool host_streams = false;      // per-nonzero streams in mapped pinned host memory
    void* up_stream = nullptr;      // amped_mttkrp_all_host: upload and download streams and events
    void* down_stream = nullptr;
    void* copy_ev[AMPED_MAX_MODES + 4] = {};
    std::vector<void*> allocs;
    std::vector<void*> host_allocs;

    cudaError_t dalloc(void** p, size_t bytes) {
        *p = nullptr;
        const int64_t n = ++g_call_allocs;
        const int64_t f = fault_alloc_at();
        if (f > 0 && n == f) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) allocs.push_back(*p);
        return e;
    }
    void dfree(void* p) {
        if (!p) return;
        auto it = std::find(allocs.begin(), allocs.end(), p);
        if (it != allocs.end()) allocs.erase(it);
        cudaFree(p);
    }
    // A per-nonzero stream: device memory, or mapped pinned host memory read over the host link.
    cudaError_t salloc(void** p, size_t bytes) {
        if (!host_streams) return dalloc(p, bytes);
        *p = nullptr;
        const int64_t n = ++g_call_allocs;
        const int64_t f = fault_alloc_at();
        if (f > 0 && n == f) return cudaErrorMemoryAllocation;
        void* h = nullptr;
        cudaError_t e = cudaHostAlloc(&h, bytes ? bytes : 16, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) return e;
        host_allocs.push_back(h);
        std::memset(h, 0, bytes ? bytes : 16);  // slack included; also touches every page once
        return cudaHostGetDevicePointer(p, h, 0);
    }
    ~amped_tensor() {
        for (void* e : copy_ev)
            if (e) cudaEventDestroy(static_cast<cudaEvent_t>(e));
        if (up_stream) cudaStreamDestroy(static_cast<cudaStream_t>(up_stream));
        if (down_stream) cudaStreamDestroy(static_cast<cudaStream_t>(down_stream));
        for (void* p : allocs) cudaFree(p);
        for (void* p : host_allocs) cudaFreeHost(p);
    }
};

namespace {

template <class T>
cudaError_t upload(amped_tensor* t, T** dst, const T* src, size_t n, size_t cap) {
    cudaError_t e = t->dalloc(reinterpret_cast<void**>(dst), cap * sizeof(T));
    if (e != cudaSuccess) return e;
    if (cap > n) e = cudaMemset(*dst + n, 0, (cap - n) * sizeof(T));
    if (e == cudaSuccess && n) e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

// upload() for a per-nonzero stream (device or mapped host memory; cudaMemcpyDefault
// resolves either through unified addressing).
template <class T>
cudaError_t upload_stream(amped_tensor* t, T** dst, const T* src, size_t n, size_t cap) {
    cudaError_t e = t->salloc(reinterpret_cast<void**>(dst), cap * sizeof(T));
    if (e != cudaSuccess) return e;
    if (n) e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyDefault);
    if (e == cudaSuccess && cap > n && !t->host_streams)  // host streams start zeroed
        e = cudaMemset(*dst + n, 0, (cap - n) * sizeof(T));
    return e;
}

// Streams and events for the overlapped copies of amped_mttkrp_all_host, created on first use.
cudaError_t ensure_copy_streams(amped_tensor* t) {
    if (t->up_stream) return cudaSuccess;
    cudaStream_t a = nullptr, b = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking);
    for (int i = 0; e == cudaSuccess && i < AMPED_MAX_MODES + 4; ++i) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        t->copy_ev[i] = ev;
    }
    if (e != cudaSuccess) {
        if (a) cudaStreamDestroy(a);
        if (b) cudaStreamDestroy(b);
        return e;
    }
    t->up_stream = a;
    t->down_stream = b;
    return cudaSuccess;
}

// Scratch for the split-row partials, sized for rank R.
amped_status ensure_scratch(amped_tensor* t, int R) {
    if (R <= t->rcap && t->queue) return AMPED_OK;
    const int rc = std::max(R, t->rcap);
    cudaError_t e;
    if (!t->queue && (e = t->dalloc(reinterpret_cast<void**>(&t->queue), 64 * sizeof(int))) != cudaSuccess)
        return cuda_fail(e, "scratch allocation");
    cudaDeviceSynchronize();  // scratch may still be in use by earlier work on any stream
    t->dfree(t->part);
    t->dfree(t->tsum);
    t->part = nullptr;
    t->tsum = nullptr;
    t->rcap = 0;
    if ((e = t->dalloc(reinterpret_cast<void**>(&t->part), (size_t)t->maxS * 2 * rc * sizeof(float))) !=
        cudaSuccess)
        return cuda_fail(e, "scratch allocation");
    if ((e = t->dalloc(reinterpret_cast<void**>(&t->tsum), (size_t)t->maxTask * rc * sizeof(double))) !=
        cudaSuccess)
        return cuda_fail(e, "scratch allocation");
    t->rcap = rc;
    return AMPED_OK;
}

// CP-ALS workspace for rank R: the MTTKRP output of the largest mode, its Gram,
// the solve output and status.
amped_status ensure_als(amped_tensor* t, int R) {
    if (R <= t->als_rcap) return AMPED_OK;
    int64_t rows = 0;
    for (int n = 0; n < t->N; ++n) rows = std::max<int64_t>(rows, t->dims[n]);
    cudaDeviceSynchronize();  // the old workspace may still be in use on any stream
    t->dfree(t->als_m);
    t->dfree(t->als_gm);
    t->dfree(t->als_w);
    t->dfree(t->als_info);
    t->als_m = nullptr;
    t->als_gm = nullptr;
    t->als_w = nullptr;
    t->als_info = nullptr;
    t->als_rcap = 0;
    cudaError_t e;
    if ((e = t->dalloc(reinterpret_cast<void**>(&t->als_m), (size_t)rows * R * sizeof(float))) != cudaSuccess ||
        (e = t->dalloc(reinterpret_cast<void**>(&t->als_gm), ((size_t)R * R + R) * sizeof(double))) != cudaSuccess ||
        (e = t->dalloc(reinterpret_cast<void**>(&t->als_w), (size_t)R * R * sizeof(float))) != cudaSuccess ||
        (e = t->dalloc(reinterpret_cast<void**>(&t->als_info), 16)) != cudaSuccess)
        return cuda_fail(e, "CP-ALS workspace allocation");
    t->als_rcap = R;
    return AMPED_OK;
}

// Default segment size: large segments (fewer split rows, fewer tickets) but at
// least ~8 segments per resident warp of the persistent grid, so the ticket
// queue can still balance the load.
int default_segment_items(int64_t nnz, int nmodes, const int64_t* dims, int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) sms = 152;
    int64_t rows = 0;
    for (int n = 0; n < nmodes; ++n) rows = std::max<int64_t>(rows, dims[n]);
    const int64_t warps = (int64_t)sms * 32;  // 4 blocks of 8 warps per SM
    const int64_t per = (nnz + rows) / (8 * warps);
    return (int)std::min<int64_t>(4096, std::max<int64_t>(256, per));
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

amped_status check_call(amped_tensor* t, const void* const* factors, amped_dtype fdtype, int R, int skip_mode,
                        int* vec) {
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (!factors) return fail(AMPED_ERR_INVALID, "factor pointer array is NULL");
    if (fdtype != AMPED_F32 && fdtype != AMPED_BF16 && fdtype != AMPED_F16)
        return fail(AMPED_ERR_INVALID, "unknown factor dtype %d", (int)fdtype);
    if (R < 1) return fail(AMPED_ERR_INVALID, "rank R=%d must be >= 1", R);
    *vec = kernel_vec(fdtype, R);
    if (*vec == 0)
        return fail(AMPED_ERR_UNSUPPORTED, "no kernel for rank R=%d with %s factors", R,
                    fdtype == AMPED_F32 ? "fp32" : "16-bit");
    const size_t al = (size_t)*vec * esize(fdtype);
    for (int n = 0; n < t->N; ++n) {
        if (n == skip_mode) continue;
        if (!factors[n]) return fail(AMPED_ERR_INVALID, "factor %d is NULL", n);
        if (!aligned(factors[n], al)) return fail(AMPED_ERR_INVALID, "factor %d is not %zu-byte aligned", n, al);
    }
    if (t->N < 2 && skip_mode >= 0) return AMPED_OK;
    if (t->N - 1 > kMaxIn && skip_mode >= 0)
        return fail(AMPED_ERR_UNSUPPORTED, "MTTKRP kernels are built for 2 to %d modes, tensor has %d", kMaxIn + 1,
                    t->N);
    return AMPED_OK;
}

// One mode: reset the ticket counter, run the persistent kernel, combine split rows.
// Checked builds: waits for the stream and reports (then clears) the first
// bounds check the kernels failed since the last look.  Default builds: no-op.
amped_status check_device(amped_tensor* t, cudaStream_t st, const char* what) {
#if AMPED_CHECKS
    if (!t->err) return AMPED_OK;
    int32_t w[4] = {0, 0, 0, 0};
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(w, t->err, sizeof w, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (w[0] != 0) {
        static const char* names[] = {"?", "gather coordinate", "output row id", "stream position", "row-table window",
                                      "short segment width"};
        cudaMemset(t->err, 0, sizeof w);
        return fail(AMPED_ERR_INDEX, "%s: device bounds check failed: %s %d (slot %d)", what,
                    names[(w[0] > 0 && w[0] <= kCheckShort) ? w[0] : 0], w[1], w[2]);
    }
#else
    (void)t;
    (void)st;
    (void)what;
#endif
    return AMPED_OK;
}

// The fields of MttkrpParams that checked builds use.
void set_bounds(const amped_tensor* t, const DevMode& dm, MttkrpParams& p) {
    p.err = t->err;
    for (int slot = 0; slot < t->N - 1; ++slot) p.fdim[slot] = (int32_t)t->dims[dm.slot_mode[slot]];
    p.out_rows = (int32_t)dm.I;
    p.stride = t->stride;
}

amped_status run_mode(amped_tensor* t, int mode, const void* const* factors, amped_dtype fdtype, int R, int vec,
                      float* out, const float* gval, cudaStream_t st, bool residual = false, double* loss = nullptr) {
    const DevMode& dm = t->m[mode];
    if (!out) return fail(AMPED_ERR_INVALID, "output for mode %d is NULL", mode);
    if (!aligned(out, vec > 1 ? 16 : 4)) return fail(AMPED_ERR_INVALID, "output for mode %d is misaligned", mode);
    Range range("amped mttkrp mode %d%s", mode, residual ? " (residual)" : (gval ? " (gradient)" : ""));
    amped_status s = ensure_scratch(t, R);
    if (s != AMPED_OK) return s;
    if (t->N == 1) {  // no input modes: the product is empty, out(i,r) = sum of the row's values
        return fail(AMPED_ERR_UNSUPPORTED, "single-mode tensors have no MTTKRP kernel");
    }
    cudaError_t e = cudaMemsetAsync(t->queue, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    MttkrpParams p{};
    p.rowptr = dm.rowptr;
    p.rows_L = dm.rows_L;
    p.rowptr_S = dm.rowptr_S;
    p.rows_S = dm.rows_S;
    p.seg_short = dm.seg_short;
    p.S_S = dm.S_S;
    const int nin = t->N - 1;
    for (int slot = 0; slot < nin; ++slot) {
        p.idx[slot] = dm.idx + (size_t)slot * t->stride;
        p.fac[slot] = factors[dm.slot_mode[slot]];
    }
    p.val = dm.val;
    p.perm = gval ? dm.perm : nullptr;
    p.gval = gval;
    p.seg_row = dm.seg;
    p.seg_nz = dm.seg + dm.S + 1;
    p.out = out;
    p.part = t->part;
    p.queue = t->queue;
    p.I = dm.L;
    p.S = dm.S;
    p.R = R;
    p.nnz = (int32_t)t->nnz;
    p.fout = residual ? factors[mode] : nullptr;
    p.loss = residual ? loss : nullptr;
    set_bounds(t, dm, p);
    if (t->ev_start) cudaEventRecord(static_cast<cudaEvent_t>(t->ev_start), st);
    int rc;
    if (residual) {
        switch (fdtype) {
            case AMPED_F32: rc = launch_residual_f32(nin, p, 0, st); break;
            case AMPED_BF16: rc = launch_residual_bf16(nin, p, 0, st); break;
            default: rc = launch_residual_f16(nin, p, 0, st); break;
        }
    } else {
        switch (fdtype) {
            case AMPED_F32: rc = launch_mttkrp_f32(nin, p, 0, st); break;
            case AMPED_BF16: rc = launch_mttkrp_bf16(nin, p, 0, st); break;
            default: rc = launch_mttkrp_f16(nin, p, 0, st); break;
        }
    }
    if (t->ev_stop) cudaEventRecord(static_cast<cudaEvent_t>(t->ev_stop), st);
    t->ev_start = t->ev_stop = nullptr;
    if (rc != 0) return cuda_fail((cudaError_t)rc, "MTTKRP kernel launch");
    ++g_launches;
    CombineParams c{};
    c.tasks = dm.table;
    c.split_info = dm.table + 4 * (size_t)dm.ntask;
    c.multi = c.split_info + 2 * ((size_t)dm.nsplit + 1);
    c.part = t->part;
    c.tsum = t->tsum;
    c.out = out;
    c.ntask = dm.ntask;
    c.nmulti = dm.nmulti;
    c.R = R;
    int launched = 0;
    rc = launch_combine(c, st, &launched);
    g_launches += launched;
    if (rc != 0) return cuda_fail((cudaError_t)rc, "split-row combine launch");
    return check_device(t, st, "MTTKRP kernel");
}

}  // namespace

extern "C" {

const char* amped_version(void) { return AMPED_CHECKS ? "amped-gb300 0.1 (sm_103a, checked)" : "amped-gb300 0.1 (sm_103a)"; }

const char* amped_last_error(void) { return g_err.c_str(); }

int64_t amped_kernel_launches(void) { return g_launches.load(); }

amped_status amped_tensor_create(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx,
                                 const float* vals, const amped_opts* opts, amped_tensor_t* out) {
    begin_call();
    if (!out) return fail(AMPED_ERR_INVALID, "output handle pointer is NULL");
    *out = nullptr;
    if (nmodes < 1 || nmodes > AMPED_MAX_MODES)
        return fail(AMPED_ERR_INVALID, "nmodes=%d outside 1..%d", nmodes, AMPED_MAX_MODES);
    if (nnz < 0 || nnz > (int64_t)INT32_MAX - 4 * kPad)
        return fail(AMPED_ERR_INVALID, "nnz=%lld outside 0..2^31-%d", (long long)nnz, 4 * kPad);
    if (!dims) return fail(AMPED_ERR_INVALID, "dims is NULL");
    for (int n = 0; n < nmodes; ++n)
        if (dims[n] < 1 || dims[n] > (int64_t)INT32_MAX - 4 * kPad)
            return fail(AMPED_ERR_INVALID, "dims[%d]=%lld outside 1..2^31-%d", n, (long long)dims[n], 4 * kPad);
    if (nnz > 0 && (!idx || !vals)) return fail(AMPED_ERR_INVALID, "idx or vals is NULL");
    int items = 0, threads = 0, max_rank = 64, short_thr = 32;
    bool keep_perm = true, keep_coo = true, inner_sort = true, ascending = false, host_streams = false;
    if (opts) {
        if (opts->segment_items < 0 || opts->max_rank < 0 || opts->host_threads < 0)
            return fail(AMPED_ERR_INVALID, "negative option");
        if (opts->segment_items > 0) items = opts->segment_items;
        if (opts->max_rank > 0) max_rank = opts->max_rank;
        threads = opts->host_threads;
        keep_perm = opts->keep_perm != 2;
        keep_coo = opts->keep_coo != 2;
        if (opts->inner_order < 0 || opts->inner_order > 3)
            return fail(AMPED_ERR_INVALID, "inner_order=%d is not 0, 1, 2 or 3", opts->inner_order);
        inner_sort = opts->inner_order != 1;
        ascending = opts->inner_order == 3;
        if (opts->short_rows > 0) short_thr = std::min(opts->short_rows, kShortNnz + 1);
        if (opts->short_rows < 0) short_thr = 1;  // every non-empty row takes the long path
        if (opts->stream_memory < 0 || opts->stream_memory > 2)
            return fail(AMPED_ERR_INVALID, "stream_memory=%d is not 0, 1 or 2", opts->stream_memory);
        host_streams = opts->stream_memory == 2;
    }
    const int64_t bad = find_bad_index(nnz, nmodes, dims, idx, threads);
    if (bad >= 0) {
        std::string c;
        for (int n = 0; n < nmodes; ++n) c += (n ? "," : "") + std::to_string(idx[bad * nmodes + n]);
        return fail(AMPED_ERR_INDEX, "nonzero %lld has coordinate (%s) outside dims", (long long)bad, c.c_str());
    }

    Range range("amped_tensor_create (%lld nonzeros, %d modes)", (long long)nnz, nmodes);
    amped_tensor* t = new (std::nothrow) amped_tensor;
    if (!t) return fail(AMPED_ERR_OOM, "host allocation failed");
    cudaGetDevice(&t->device);
    noalloc_resolve(t->device);
    if (items == 0) items = default_segment_items(nnz, nmodes, dims, t->device);
    t->N = nmodes;
    t->nnz = nnz;
    t->host_streams = host_streams;
    for (int n = 0; n < nmodes; ++n) t->dims[n] = dims[n];
    t->stride = ((nnz + kPad) + 63) / 64 * 64;
    const size_t stride = (size_t)t->stride;

    auto bail = [&](amped_status s) {
        delete t;
        return s;
    };
    HostBuf<int32_t> col;  // [N-1][stride]: the input slots' columns of one copy
    HostBuf<float> fcol;
    if (!col.alloc(stride * (size_t)std::max(1, nmodes - 1)) || !fcol.alloc(stride))
        return bail(fail(AMPED_ERR_OOM, "host allocation failed"));
    cudaError_t e;
    HostBuf<int32_t> lex;  // lexicographic order of all coordinates; every mode's copy is a stable sort of it
    {
        Range lex_range("lexicographic order");
        if (inner_sort && !lex_order(nnz, nmodes, dims, idx, threads, lex, ascending))
            return bail(fail(AMPED_ERR_OOM, "host allocation failed in the lexicographic order"));
    }
    for (int mode = 0; mode < nmodes; ++mode) {
        Range mode_range("mode %d copy: reorder, plan, upload", mode);
        HostMode hm;
        if (!order_mode(nnz, nmodes, dims, idx, mode, inner_sort ? lex.p : nullptr, threads, hm))
            return bail(fail(AMPED_ERR_OOM, "host allocation failed in the reorder of mode %d", mode));
        if (mode == 0) {
            t->xnorm2 = norm2_merged(hm, nmodes, idx, vals, inner_sort, threads);
            if (t->xnorm2 < 0.0) return bail(fail(AMPED_ERR_OOM, "host allocation failed computing the tensor norm"));
        }
        if (!classify_rows(hm, short_thr, threads) || !cut_segments(hm, items))
            return bail(fail(AMPED_ERR_OOM, "host allocation failed in the reorder of mode %d", mode));
        DevMode& dm = t->m[mode];
        dm.I = hm.I;
        dm.L = hm.L;
        dm.S_S = hm.S_S;
        dm.S = hm.S;
        dm.nsplit = hm.nsplit;
        dm.ntask = hm.ntask;
        dm.nmulti = hm.nmulti;
        if ((e = upload(t, &dm.rowptr, hm.rowptr_L.p, (size_t)hm.L + 1, (size_t)hm.L + 1 + kPad)) != cudaSuccess ||
            (e = upload(t, &dm.rows_L, hm.rows_L.p, (size_t)hm.L, (size_t)hm.L + kPad)) != cudaSuccess ||
            (e = upload(t, &dm.rowptr_S, hm.rowptr_S.p, (size_t)hm.Sr + 1, (size_t)hm.Sr + 1 + kPad)) != cudaSuccess ||
            (e = upload(t, &dm.rows_S, hm.rows_S.p, (size_t)hm.Sr, (size_t)hm.Sr + kPad)) != cudaSuccess ||
            (e = upload(t, &dm.seg_short, hm.seg_short.p, (size_t)hm.S_S + 1, (size_t)hm.S_S + 1)) != cudaSuccess)
            return bail(cuda_fail(e, "device copy of the row tables"));
        const int nin = nmodes > 1 ? input_slots(nmodes, dims, mode, inner_sort, ascending, dm.slot_mode) : 0;
        {
            int32_t* cols[AMPED_MAX_MODES];
            for (int slot = 0; slot < nin; ++slot) cols[slot] = col.p + (size_t)slot * stride;
            gather_copy(hm, nmodes, idx, vals, nin, dm.slot_mode, cols, fcol.p, threads);
            for (int slot = 0; slot < nin; ++slot) std::memset(cols[slot] + nnz, 0, (stride - (size_t)nnz) * 4);
            std::memset(fcol.p + nnz, 0, (stride - (size_t)nnz) * 4);
#if AMPED_CHECKS
            // Checked builds only: AMPED_FAULT=coord:K corrupts the slot-0 coordinate of copy
            // position K of mode 0 after validation, so a test can watch a kernel's bounds check
            // catch it (the access is clamped; the call reports AMPED_ERR_INDEX).
            if (mode == 0 && nin > 0 && nnz > 0) {
                const char* f = std::getenv("AMPED_FAULT");
                if (f && std::strncmp(f, "coord:", 6) == 0)
                    cols[0][(size_t)(std::atoll(f + 6) % nnz)] = (int32_t)dims[dm.slot_mode[0]] + 3;
            }
#endif
        }
        if (nin > 0) {
            if ((e = t->salloc(reinterpret_cast<void**>(&dm.idx), (size_t)nin * stride * 4)) != cudaSuccess)
                return bail(cuda_fail(e, "copy of the coordinates"));
            if ((e = cudaMemcpy(dm.idx, col.p, (size_t)nin * stride * 4, cudaMemcpyDefault)) != cudaSuccess)
                return bail(cuda_fail(e, "copy of the coordinates"));
        }
        if ((e = upload_stream(t, &dm.val, fcol.p, stride, stride)) != cudaSuccess)
            return bail(cuda_fail(e, "copy of the values"));
        if (keep_perm && (e = upload_stream(t, &dm.perm, hm.perm.p, (size_t)nnz, stride)) != cudaSuccess)
            return bail(cuda_fail(e, "copy of the permutation"));
        std::vector<int32_t> seg((size_t)2 * (hm.S + 1));
        std::memcpy(seg.data(), hm.seg_row.p, (size_t)(hm.S + 1) * 4);
        std::memcpy(seg.data() + hm.S + 1, hm.seg_nz.p, (size_t)(hm.S + 1) * 4);
        if ((e = upload(t, &dm.seg, seg.data(), seg.size(), seg.size())) != cudaSuccess)
            return bail(cuda_fail(e, "device copy of the segment table"));
        std::vector<int32_t> table((size_t)4 * hm.ntask + 2 * ((size_t)hm.nsplit + 1) + hm.nmulti);
        if (hm.ntask) std::memcpy(table.data(), hm.tasks.p, (size_t)4 * hm.ntask * 4);
        std::memcpy(table.data() + 4 * (size_t)hm.ntask, hm.split_info.p, 2 * ((size_t)hm.nsplit + 1) * 4);
        if (hm.nmulti)
            std::memcpy(table.data() + 4 * (size_t)hm.ntask + 2 * ((size_t)hm.nsplit + 1), hm.multi.p,
                        (size_t)hm.nmulti * 4);
        if ((e = upload(t, &dm.table, table.data(), table.size(), table.size())) != cudaSuccess)
            return bail(cuda_fail(e, "device copy of the combine table"));
        t->maxS = std::max(t->maxS, hm.S);
        t->maxTask = std::max(t->maxTask, hm.ntask);
    }
    if (keep_coo) {
        if ((e = t->salloc(reinterpret_cast<void**>(&t->coo), (size_t)nmodes * stride * 4)) != cudaSuccess)
            return bail(cuda_fail(e, "copy of the caller-order coordinates"));
        for (int n = 0; n < nmodes; ++n) {
            caller_column(nnz, nmodes, idx, n, col.p, threads);
            std::memset(col.p + nnz, 0, (stride - (size_t)nnz) * 4);
            if ((e = cudaMemcpy(t->coo + (size_t)n * stride, col.p, stride * 4, cudaMemcpyDefault)) != cudaSuccess)
                return bail(cuda_fail(e, "copy of the caller-order coordinates"));
        }
    }
    amped_status s = ensure_scratch(t, max_rank);
    if (s != AMPED_OK) return bail(s);
#if AMPED_CHECKS
    if ((e = t->dalloc(reinterpret_cast<void**>(&t->err), 4 * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMemset(t->err, 0, 4 * sizeof(int32_t))) != cudaSuccess)
        return bail(cuda_fail(e, "error word of the bounds checks"));
#endif
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(cuda_fail(e, "tensor create"));
    *out = t;
    return AMPED_OK;
}

amped_status amped_tensor_destroy(amped_tensor_t t) {
    begin_call();
    if (!t) return AMPED_OK;
    cudaDeviceSynchronize();
    delete t;
    return AMPED_OK;
}

amped_status amped_tensor_info(amped_tensor_t t, int64_t* nnz, int* nmodes, int64_t* dims) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (nnz) *nnz = t->nnz;
    if (nmodes) *nmodes = t->N;
    if (dims)
        for (int n = 0; n < t->N; ++n) dims[n] = t->dims[n];
    return AMPED_OK;
}

amped_status amped_mttkrp(amped_tensor_t t, int mode, const void* const* factors, amped_dtype fdtype, int R,
                          float* out, void* stream) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (mode < 0 || mode >= t->N) return fail(AMPED_ERR_INVALID, "mode %d outside 0..%d", mode, t->N - 1);
    int vec = 0;
    amped_status s = check_call(t, factors, fdtype, R, mode, &vec);
    if (s != AMPED_OK) return s;
    return run_mode(t, mode, factors, fdtype, R, vec, out, nullptr, static_cast<cudaStream_t>(stream));
}

amped_status amped_mttkrp_all(amped_tensor_t t, const void* const* factors, amped_dtype fdtype, int R,
                              float* const* outs, void* stream) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (!outs) return fail(AMPED_ERR_INVALID, "output pointer array is NULL");
    int vec = 0;
    amped_status s = check_call(t, factors, fdtype, R, -1, &vec);
    if (s != AMPED_OK) return s;
    if (t->N - 1 > kMaxIn) return fail(AMPED_ERR_UNSUPPORTED, "MTTKRP kernels are built for 2 to %d modes", kMaxIn + 1);
    for (int n = 0; n < t->N; ++n)
        if (!outs[n]) return fail(AMPED_ERR_INVALID, "output for mode %d is NULL", n);
    for (int n = 0; n < t->N; ++n) {
        s = run_mode(t, n, factors, fdtype, R, vec, outs[n], nullptr, static_cast<cudaStream_t>(stream));
        if (s != AMPED_OK) return s;
    }
    return AMPED_OK;
}

amped_status amped_mttkrp_all_host(amped_tensor_t t, const void* const* factors, amped_dtype fdtype, int R,
                                   float* const* outs, void* stream) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (!outs || !factors) return fail(AMPED_ERR_INVALID, "factor or output pointer array is NULL");
    Range range("amped mttkrp_all_host");
    int vec = 0;
    // host pointers: check everything except device alignment, which the staging provides
    const void* dummy[AMPED_MAX_MODES];
    for (int n = 0; n < t->N; ++n) {
        if (!factors[n] || !outs[n]) return fail(AMPED_ERR_INVALID, "host buffer %d is NULL", n);
        dummy[n] = reinterpret_cast<const void*>(uintptr_t(256));
    }
    amped_status s = check_call(t, dummy, fdtype, R, -1, &vec);
    if (s != AMPED_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const void* dfac[AMPED_MAX_MODES];
    float* dout[AMPED_MAX_MODES];
    for (int n = 0; n < t->N; ++n) {
        const size_t fb = (size_t)t->dims[n] * R * esize(fdtype), ob = (size_t)t->dims[n] * R * 4;
        if (t->stage_fac_bytes[n] < fb) {
            cudaStreamSynchronize(st);
            t->dfree(t->stage_fac[n]);
            t->stage_fac_bytes[n] = 0;
            if ((e = t->dalloc(&t->stage_fac[n], fb)) != cudaSuccess) return cuda_fail(e, "staging allocation");
            t->stage_fac_bytes[n] = fb;
        }
        if (t->stage_out_bytes[n] < ob) {
            cudaStreamSynchronize(st);
            t->dfree(t->stage_out[n]);
            t->stage_out_bytes[n] = 0;
            if ((e = t->dalloc(reinterpret_cast<void**>(&t->stage_out[n]), ob)) != cudaSuccess)
                return cuda_fail(e, "staging allocation");
            t->stage_out_bytes[n] = ob;
        }
        dfac[n] = t->stage_fac[n];
        dout[n] = t->stage_out[n];
    }
    // Copies overlap the kernels: the factors mode 0 needs go first, factor 0 is uploaded
    // while mode 0 runs, and the outputs are downloaded while the later modes run.  The
    // downloads start once the uploads are done, so they do not share the host link with the
    // upload of factor 0, which every mode after the first waits for.
    if ((e = ensure_copy_streams(t)) != cudaSuccess) return cuda_fail(e, "copy streams");
    cudaStream_t up = static_cast<cudaStream_t>(t->up_stream), down = static_cast<cudaStream_t>(t->down_stream);
    cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(t->copy_ev);  // [0] entry, [1] rest in, [2] factor 0 in,
                                                                  // [3 + m] output m ready, [3 + N] outputs out
    auto upload = [&](int n) {
        const size_t fb = (size_t)t->dims[n] * R * esize(fdtype);
        return cudaMemcpyAsync(t->stage_fac[n], factors[n], fb, cudaMemcpyHostToDevice, up);
    };
    if ((e = cudaEventRecord(ev[0], st)) != cudaSuccess || (e = cudaStreamWaitEvent(up, ev[0], 0)) != cudaSuccess)
        return cuda_fail(e, "copy ordering");
    for (int n = 1; n < t->N; ++n)
        if ((e = upload(n)) != cudaSuccess) return cuda_fail(e, "factor upload");
    if ((e = cudaEventRecord(ev[1], up)) != cudaSuccess || (e = upload(0)) != cudaSuccess ||
        (e = cudaEventRecord(ev[2], up)) != cudaSuccess || (e = cudaStreamWaitEvent(st, ev[1], 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(down, ev[2], 0)) != cudaSuccess)
        return cuda_fail(e, "factor upload");
    for (int n = 0; n < t->N; ++n) {
        if (n == 1 && (e = cudaStreamWaitEvent(st, ev[2], 0)) != cudaSuccess) return cuda_fail(e, "copy ordering");
        s = run_mode(t, n, dfac, fdtype, R, vec, dout[n], nullptr, st);
        if (s != AMPED_OK) return s;
        if ((e = cudaEventRecord(ev[3 + n], st)) != cudaSuccess || (e = cudaStreamWaitEvent(down, ev[3 + n], 0)) != cudaSuccess)
            return cuda_fail(e, "copy ordering");
        const size_t ob = (size_t)t->dims[n] * R * 4;
        if ((e = cudaMemcpyAsync(outs[n], dout[n], ob, cudaMemcpyDeviceToHost, down)) != cudaSuccess)
            return cuda_fail(e, "output download");
    }
    if (t->N == 1 && (e = cudaStreamWaitEvent(st, ev[2], 0)) != cudaSuccess) return cuda_fail(e, "copy ordering");
    if ((e = cudaEventRecord(ev[3 + t->N], down)) != cudaSuccess || (e = cudaStreamWaitEvent(st, ev[3 + t->N], 0)) != cudaSuccess)
        return cuda_fail(e, "copy ordering");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "host MTTKRP");
    return AMPED_OK;
}

amped_status amped_cp_sample(amped_tensor_t t, const void* const* factors, amped_dtype fdtype, int R, float* m_out,
                             void* stream) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (!t->coo) return fail(AMPED_ERR_INVALID, "handle was created without caller-order coordinates (keep_coo)");
    int vec = 0;
    amped_status s = check_call(t, factors, fdtype, R, -1, &vec);
    if (s != AMPED_OK) return s;
    if (t->N < 2 || t->N > AMPED_MAX_MODES)
        return fail(AMPED_ERR_UNSUPPORTED, "sampled-model kernels are built for 2 to %d modes", AMPED_MAX_MODES);
    if (t->nnz == 0) return AMPED_OK;
    if (!m_out || !aligned(m_out, 16)) return fail(AMPED_ERR_INVALID, "m_out is NULL or not 16-byte aligned");
    SampleParams p{};
    for (int n = 0; n < t->N; ++n) {
        p.idx[n] = t->coo + (size_t)n * t->stride;
        p.fac[n] = factors[n];
    }
    p.m = m_out;
    p.nnz = (int32_t)t->nnz;
    p.R = R;
    p.nmodes = t->N;
    p.err = t->err;
    for (int n = 0; n < t->N; ++n) p.fdim[n] = (int32_t)t->dims[n];
    p.stride = t->stride;
    Range range("amped cp_sample");
    int rc;
    switch (fdtype) {
        case AMPED_F32: rc = launch_sample_f32(p, stream); break;
        case AMPED_BF16: rc = launch_sample_bf16(p, stream); break;
        default: rc = launch_sample_f16(p, stream); break;
    }
    if (rc != 0) return cuda_fail((cudaError_t)rc, "sampled-model kernel launch");
    ++g_launches;
    return check_device(t, static_cast<cudaStream_t>(stream), "sampled-model kernel");
}

amped_status amped_cp_grad(amped_tensor_t t, const void* const* factors, amped_dtype fdtype, int R,
                           const float* gvals, float* const* grads, void* stream) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (!grads) return fail(AMPED_ERR_INVALID, "gradient pointer array is NULL");
    if (t->nnz > 0 && !gvals) return fail(AMPED_ERR_INVALID, "gvals is NULL");
    if (t->N > 1 && !t->m[0].perm && t->nnz > 0)
        return fail(AMPED_ERR_INVALID, "handle was created without permutations (keep_perm)");
    int vec = 0;
    amped_status s = check_call(t, factors, fdtype, R, -1, &vec);
    if (s != AMPED_OK) return s;
    if (t->N - 1 > kMaxIn) return fail(AMPED_ERR_UNSUPPORTED, "MTTKRP kernels are built for 2 to %d modes", kMaxIn + 1);
    for (int n = 0; n < t->N; ++n)
        if (!grads[n]) return fail(AMPED_ERR_INVALID, "gradient %d is NULL", n);
    for (int n = 0; n < t->N; ++n) {
        s = run_mode(t, n, factors, fdtype, R, vec, grads[n], t->nnz ? gvals : nullptr,
                     static_cast<cudaStream_t>(stream));
        if (s != AMPED_OK) return s;
    }
    return AMPED_OK;
}

amped_status amped_plan_mode(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int mode,
                             int segment_items, int inner_order, int short_rows, amped_plan_sizes* sizes,
                             int32_t* perm, int32_t* rows_long, int32_t* rowptr_long, int32_t* seg_row,
                             int32_t* seg_nz, int32_t* splits, int32_t* rows_short, int32_t* rowptr_short,
                             int32_t* seg_short) {
    begin_call();
    if (nmodes < 1 || nmodes > AMPED_MAX_MODES || !dims || nnz < 0 || nnz > (int64_t)INT32_MAX - 4 * kPad)
        return fail(AMPED_ERR_INVALID, "bad tensor shape");
    if (mode < 0 || mode >= nmodes) return fail(AMPED_ERR_INVALID, "mode %d outside 0..%d", mode, nmodes - 1);
    for (int n = 0; n < nmodes; ++n)
        if (dims[n] < 1 || dims[n] > (int64_t)INT32_MAX - 4 * kPad)
            return fail(AMPED_ERR_INVALID, "dims[%d]=%lld out of range", n, (long long)dims[n]);
    if (nnz > 0 && !idx) return fail(AMPED_ERR_INVALID, "idx is NULL");
    const int items = segment_items > 0 ? segment_items : 1024;  // host-only query: no device to size for
    const int thr = short_rows > 0 ? std::min(short_rows, kShortNnz + 1) : short_rows < 0 ? 1 : 32;
    const int64_t bad = find_bad_index(nnz, nmodes, dims, idx, 0);
    if (bad >= 0) return fail(AMPED_ERR_INDEX, "nonzero %lld has a coordinate outside dims", (long long)bad);
    HostMode hm;
    HostBuf<int32_t> lex;
    if (inner_order < 0 || inner_order > 3) return fail(AMPED_ERR_INVALID, "inner_order=%d is not 0..3", inner_order);
    const bool inner_sort = inner_order != 1;
    if ((inner_sort && !lex_order(nnz, nmodes, dims, idx, 0, lex, inner_order == 3)) ||
        !order_mode(nnz, nmodes, dims, idx, mode, inner_sort ? lex.p : nullptr, 0, hm) ||
        !classify_rows(hm, thr, 0) || !cut_segments(hm, items))
        return fail(AMPED_ERR_OOM, "host allocation failed");
    if (sizes) {
        sizes->nnz = nnz;
        sizes->rows = hm.I;
        sizes->long_rows = hm.L;
        sizes->long_nnz = hm.nnz_L;
        sizes->short_rows = hm.Sr;
        sizes->long_segments = hm.S;
        sizes->short_segments = hm.S_S;
        sizes->split_rows = hm.nsplit;
    }
    if (perm && nnz) std::memcpy(perm, hm.perm.p, (size_t)nnz * 4);
    if (rows_long && hm.L) std::memcpy(rows_long, hm.rows_L.p, (size_t)hm.L * 4);
    if (rowptr_long) std::memcpy(rowptr_long, hm.rowptr_L.p, ((size_t)hm.L + 1) * 4);
    if (seg_row) std::memcpy(seg_row, hm.seg_row.p, ((size_t)hm.S + 1) * 4);
    if (seg_nz) std::memcpy(seg_nz, hm.seg_nz.p, ((size_t)hm.S + 1) * 4);
    if (splits)
        for (int32_t j = 0; j < hm.nsplit; ++j) {
            splits[3 * j] = hm.splits[(size_t)j].row;
            splits[3 * j + 1] = hm.splits[(size_t)j].s_a;
            splits[3 * j + 2] = hm.splits[(size_t)j].s_b;
        }
    if (rows_short && hm.Sr) std::memcpy(rows_short, hm.rows_S.p, (size_t)hm.Sr * 4);
    if (rowptr_short) std::memcpy(rowptr_short, hm.rowptr_S.p, ((size_t)hm.Sr + 1) * 4);
    if (seg_short) std::memcpy(seg_short, hm.seg_short.p, ((size_t)hm.S_S + 1) * 4);
    return AMPED_OK;
}

amped_status amped_norm2_host(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, const float* vals,
                              int inner_order, double* norm2) {
    begin_call();
    if (!norm2) return fail(AMPED_ERR_INVALID, "norm2 is NULL");
    if (nmodes < 1 || nmodes > AMPED_MAX_MODES || !dims || nnz < 0 || nnz > (int64_t)INT32_MAX - 4 * kPad)
        return fail(AMPED_ERR_INVALID, "bad tensor shape");
    for (int n = 0; n < nmodes; ++n)
        if (dims[n] < 1 || dims[n] > (int64_t)INT32_MAX - 4 * kPad)
            return fail(AMPED_ERR_INVALID, "dims[%d]=%lld out of range", n, (long long)dims[n]);
    if (nnz > 0 && (!idx || !vals)) return fail(AMPED_ERR_INVALID, "idx or vals is NULL");
    const int64_t bad = find_bad_index(nnz, nmodes, dims, idx, 0);
    if (bad >= 0) return fail(AMPED_ERR_INDEX, "nonzero %lld has a coordinate outside dims", (long long)bad);
    HostMode hm;
    HostBuf<int32_t> lex;
    if (inner_order < 0 || inner_order > 3) return fail(AMPED_ERR_INVALID, "inner_order=%d is not 0..3", inner_order);
    const bool inner_sort = inner_order != 1;
    if ((inner_sort && !lex_order(nnz, nmodes, dims, idx, 0, lex, inner_order == 3)) ||
        !order_mode(nnz, nmodes, dims, idx, 0, inner_sort ? lex.p : nullptr, 0, hm))
        return fail(AMPED_ERR_OOM, "host allocation failed");
    const double v = norm2_merged(hm, nmodes, idx, vals, inner_sort, 0);
    if (v < 0.0) return fail(AMPED_ERR_OOM, "host allocation failed");
    *norm2 = v;
    return AMPED_OK;
}

amped_status amped_cp_completion_grad(amped_tensor_t t, const void* const* factors, amped_dtype fdtype, int R,
                                      float* const* grads, double* loss, void* stream) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (!grads) return fail(AMPED_ERR_INVALID, "gradient pointer array is NULL");
    Range range("amped cp_completion_grad");
    int vec = 0;
    amped_status s = check_call(t, factors, fdtype, R, -1, &vec);
    if (s != AMPED_OK) return s;
    if (t->N < 2 || t->N - 1 > kMaxIn)
        return fail(AMPED_ERR_UNSUPPORTED, "completion kernels are built for 2 to %d modes", kMaxIn + 1);
    for (int n = 0; n < t->N; ++n)
        if (!grads[n]) return fail(AMPED_ERR_INVALID, "gradient %d is NULL", n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (loss) {
        cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), st);
        if (e != cudaSuccess) return cuda_fail(e, "loss reset");
    }
    for (int n = 0; n < t->N; ++n) {
        // the loss is accumulated once, in the pass over mode 0
        s = run_mode(t, n, factors, fdtype, R, vec, grads[n], nullptr, st, true, n == 0 ? loss : nullptr);
        if (s != AMPED_OK) return s;
    }
    return AMPED_OK;
}

amped_status amped_tensor_norm2(amped_tensor_t t, double* norm2) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (!norm2) return fail(AMPED_ERR_INVALID, "norm2 is NULL");
    *norm2 = t->xnorm2;
    return AMPED_OK;
}

}  // extern "C"

namespace {

// Argument checks shared by the CP-ALS entry points; fills cf and vec.
amped_status als_check(amped_tensor* t, float* const* factors, int R, const double* grams, const double* stats,
                       int flags, const void** cf, int* vec) {
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (!factors || !grams || !stats) return fail(AMPED_ERR_INVALID, "factors, grams or stats is NULL");
    if (flags & ~AMPED_ALS_INIT) return fail(AMPED_ERR_INVALID, "unknown flags 0x%x", flags);
    if (R < 1) return fail(AMPED_ERR_INVALID, "rank R=%d must be >= 1", R);
    if (R > als_max_rank()) return fail(AMPED_ERR_UNSUPPORTED, "CP-ALS is built for ranks up to %d", als_max_rank());
    if (t->N < 2 || t->N - 1 > kMaxIn) return fail(AMPED_ERR_UNSUPPORTED, "CP-ALS is built for 2 to %d modes", kMaxIn + 1);
    for (int n = 0; n < t->N; ++n) cf[n] = factors[n];
    amped_status s = check_call(t, cf, AMPED_F32, R, -1, vec);
    if (s != AMPED_OK) return s;
    for (int n = 0; n < t->N; ++n)
        if (!aligned(factors[n], 16)) return fail(AMPED_ERR_INVALID, "factor %d is not 16-byte aligned", n);
    if (!aligned(grams, 8) || !aligned(stats, 8)) return fail(AMPED_ERR_INVALID, "grams or stats is misaligned");
    return ensure_als(t, R);
}

// Optional starting Grams, then the failure counters reset.
amped_status als_begin(amped_tensor* t, float* const* factors, int R, double* grams, double* stats, int flags,
                       cudaStream_t st) {
    int launched = 0, rc = 0;
    if (flags & AMPED_ALS_INIT)
        for (int n = 0; n < t->N && rc == 0; ++n)
            rc = launch_gram(factors[n], t->dims[n], R, grams + (size_t)n * R * R, st, &launched);
    if (rc == 0) rc = (int)cudaMemsetAsync(stats + 5, 0, 2 * sizeof(double), st);
    g_launches += launched;
    return rc ? cuda_fail((cudaError_t)rc, "CP-ALS initial Grams") : AMPED_OK;
}

// One mode: MTTKRP, fp64 solve, apply with the Gram fused, commit; the fit
// terms of the resulting model when `fit` is set.
amped_status als_mode(amped_tensor* t, int m, float* const* factors, const void* const* cf, int R, int vec,
                      double* grams, double* stats, bool fit, cudaStream_t st) {
    amped_status s = run_mode(t, m, cf, AMPED_F32, R, vec, t->als_m, nullptr, st);
    if (s != AMPED_OK) return s;
    int launched = 0;
    AlsParams p{};
    p.grams = grams;
    p.ga = t->als_gm;
    p.ip = p.ga + (size_t)R * R;
    p.w = t->als_w;
    p.info = t->als_info;
    p.stats = stats;
    p.xnorm2 = t->xnorm2;
    p.N = t->N;
    p.mode = m;
    p.R = R;
    p.last = fit;
    int rc = launch_als_solve(p, st, &launched);
    if (rc == 0) rc = launch_als_apply(p, t->als_m, t->dims[m], factors[m], st, &launched);
    g_launches += launched;
    return rc ? cuda_fail((cudaError_t)rc, "CP-ALS kernel launch") : AMPED_OK;
}

}  // namespace

extern "C" {

amped_status amped_cp_als_sweep(amped_tensor_t t, float* const* factors, int R, double* grams, double* stats,
                                int flags, void* stream) {
    begin_call();
    const void* cf[AMPED_MAX_MODES];
    int vec = 0;
    amped_status s = als_check(t, factors, R, grams, stats, flags, cf, &vec);
    if (s != AMPED_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Range range("amped cp_als_sweep (rank %d)", R);
    if ((s = als_begin(t, factors, R, grams, stats, flags, st)) != AMPED_OK) return s;
    for (int m = 0; m < t->N; ++m)
        if ((s = als_mode(t, m, factors, cf, R, vec, grams, stats, m == t->N - 1, st)) != AMPED_OK) return s;
    return AMPED_OK;
}

amped_status amped_cp_als_update(amped_tensor_t t, int mode, float* const* factors, int R, double* grams,
                                 double* stats, int flags, void* stream) {
    begin_call();
    const void* cf[AMPED_MAX_MODES];
    int vec = 0;
    amped_status s = als_check(t, factors, R, grams, stats, flags, cf, &vec);
    if (s != AMPED_OK) return s;
    if (mode < 0 || mode >= t->N) return fail(AMPED_ERR_INVALID, "mode %d outside 0..%d", mode, t->N - 1);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((s = als_begin(t, factors, R, grams, stats, flags, st)) != AMPED_OK) return s;
    return als_mode(t, mode, factors, cf, R, vec, grams, stats, true, st);
}

amped_status amped_cp_als_normalize(amped_tensor_t t, float* const* factors, int R, double* grams, float* lambda,
                                    void* stream) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (!factors || !grams || !lambda) return fail(AMPED_ERR_INVALID, "factors, grams or lambda is NULL");
    if (R < 1 || R > als_max_rank())
        return fail(AMPED_ERR_UNSUPPORTED, "CP-ALS is built for ranks 1 to %d", als_max_rank());
    for (int n = 0; n < t->N; ++n)
        if (!factors[n] || !aligned(factors[n], 4)) return fail(AMPED_ERR_INVALID, "factor %d is NULL or misaligned", n);
    if (!aligned(grams, 8) || !aligned(lambda, 4)) return fail(AMPED_ERR_INVALID, "grams or lambda is misaligned");
    int launched = 0;
    const int rc = launch_als_normalize(factors, t->dims, t->N, R, grams, lambda, stream, &launched);
    g_launches += launched;
    if (rc != 0) return cuda_fail((cudaError_t)rc, "CP-ALS normalisation launch");
    return AMPED_OK;
}

amped_status amped_set_kernel_events(amped_tensor_t t, void* start, void* stop) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    t->ev_start = start;
    t->ev_stop = stop;
    return AMPED_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free MTTKRP: the same kernels, with their scratch in the fixed
// static device array g_noalloc_scratch instead of the handle's allocations.
// ---------------------------------------------------------------------------
extern "C" amped_status amped_mttkrp_noalloc(amped_tensor_t t, int mode, const void* const* factors,
                                             amped_dtype fdtype, int R, float* out, void* stream) {
    begin_call();
    if (!t) return fail(AMPED_ERR_INVALID, "tensor handle is NULL");
    if (mode < 0 || mode >= t->N) return fail(AMPED_ERR_INVALID, "mode %d outside 0..%d", mode, t->N - 1);
    int vec = 0;
    amped_status s = check_call(t, factors, fdtype, R, mode, &vec);
    if (s != AMPED_OK) return s;
    if (t->N == 1) return fail(AMPED_ERR_UNSUPPORTED, "single-mode tensors have no MTTKRP kernel");
    if (!out) return fail(AMPED_ERR_INVALID, "output for mode %d is NULL", mode);
    if (!aligned(out, vec > 1 ? 16 : 4)) return fail(AMPED_ERR_INVALID, "output for mode %d is misaligned", mode);
    const DevMode& dm = t->m[mode];
    // layout inside the static array: ticket counter, split partials [S][2][R] fp32, task sums [tasks][R] fp64
    const size_t part_off = 256;
    const size_t part_bytes = (size_t)dm.S * 2 * (size_t)R * sizeof(float);
    const size_t tsum_off = (part_off + part_bytes + 255) / 256 * 256;
    const size_t need = tsum_off + (size_t)dm.ntask * (size_t)R * sizeof(double);
    if (need > AMPED_NOALLOC_SCRATCH_BYTES)
        return fail(AMPED_ERR_UNSUPPORTED,
                    "mode %d at rank %d needs %zu bytes of scratch, more than the %u-byte static buffer; "
                    "use amped_mttkrp or a larger segment_items",
                    mode, R, need, (unsigned)AMPED_NOALLOC_SCRATCH_BYTES);
    int dev = -1;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return cuda_fail(de, "cudaGetDevice");
    if (dev != t->device)
        return fail(AMPED_ERR_INVALID, "device %d is current but the handle lives on device %d", dev, t->device);
    void* base = nullptr;
    cudaError_t lookup = cudaErrorInvalidSymbol;
    if (dev >= 0 && dev < kMaxDevices) {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        base = g_noalloc_addr[dev];
        lookup = g_noalloc_err[dev];
    }
    if (!base && lookup == cudaSuccess) lookup = cudaErrorInvalidSymbol;
    if (!base) return cuda_fail(lookup, "static scratch of the allocation-free MTTKRP unavailable on this device");
    unsigned char* b = static_cast<unsigned char*>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(b, 0, sizeof(int), st);  // the ticket counter must start at zero
    if (e != cudaSuccess) return cuda_fail(e, "ticket reset");
    MttkrpParams p{};
    p.rowptr = dm.rowptr;
    p.rows_L = dm.rows_L;
    p.rowptr_S = dm.rowptr_S;
    p.rows_S = dm.rows_S;
    p.seg_short = dm.seg_short;
    p.S_S = dm.S_S;
    const int nin = t->N - 1;
    for (int slot = 0; slot < nin; ++slot) {
        p.idx[slot] = dm.idx + (size_t)slot * t->stride;
        p.fac[slot] = factors[dm.slot_mode[slot]];
    }
    p.val = dm.val;
    p.perm = nullptr;
    p.gval = nullptr;
    p.seg_row = dm.seg;
    p.seg_nz = dm.seg + dm.S + 1;
    p.out = out;
    p.part = reinterpret_cast<float*>(b + part_off);
    p.queue = reinterpret_cast<int*>(b);
    p.I = dm.L;
    p.S = dm.S;
    p.R = R;
    p.nnz = (int32_t)t->nnz;
    set_bounds(t, dm, p);
    if (t->ev_start) cudaEventRecord(static_cast<cudaEvent_t>(t->ev_start), st);
    int rc;
    switch (fdtype) {
        case AMPED_F32: rc = launch_mttkrp_f32(nin, p, 0, st); break;
        case AMPED_BF16: rc = launch_mttkrp_bf16(nin, p, 0, st); break;
        default: rc = launch_mttkrp_f16(nin, p, 0, st); break;
    }
    if (t->ev_stop) cudaEventRecord(static_cast<cudaEvent_t>(t->ev_stop), st);
    t->ev_start = t->ev_stop = nullptr;
    if (rc != 0) return cuda_fail((cudaError_t)rc, "MTTKRP kernel launch");
    ++g_launches;
    CombineParams c{};
    c.tasks = dm.table;
    c.split_info = dm.table + 4 * (size_t)dm.ntask;
    c.multi = c.split_info + 2 * ((size_t)dm.nsplit + 1);
    c.part = p.part;
    c.tsum = reinterpret_cast<double*>(b + tsum_off);
    c.out = out;
    c.ntask = dm.ntask;
    c.nmulti = dm.nmulti;
    c.R = R;
    int launched = 0;
    rc = launch_combine(c, st, &launched);
    g_launches += launched;
    if (rc != 0) return cuda_fail((cudaError_t)rc, "split-row combine launch");
    return check_device(t, st, "MTTKRP kernel");
}
