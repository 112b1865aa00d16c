/*
 * amped.h — C ABI of the GB300 sparse MTTKRP library.
 *
 * The library computes sparse MTTKRP along every mode of an N-mode COO
 * tensor (paper Sec. 2.1 Eq. 1: X_(d) times the Khatri-Rao product of the
 * other factors), which is the bottleneck of CP decomposition, together with
 * the sampled CP model and its gradient for gradient-based CP completion, and
 * CP decomposition by alternating least squares around the MTTKRP.  Everything
 * runs on one GPU.  There is no CPU fallback: a call either enqueues CUDA
 * kernels or returns an error (amped_plan_mode and amped_norm2_host are
 * host-only queries).
 *
 * Conventions shared by all entry points
 *  - Indices are 0-based int32; nnz < 2^31; 1 <= nmodes <= AMPED_MAX_MODES;
 *    every dims[n] >= 1 and < 2^31.
 *  - Factors are dense row-major [dims[n]][R] device arrays in fp32, bf16 or
 *    fp16 (`amped_dtype`), base address aligned to 16 bytes (32 bytes when R
 *    is a multiple of 8 (fp32) or 16 (16-bit)).  Products and sums are always
 *    fp32; outputs are fp32.
 *  - Device buffers passed in (factors, outputs, values) are owned by the
 *    caller and must stay valid until the work enqueued on `stream` is done.
 *    The handle owns every device copy it builds and frees it in
 *    amped_tensor_destroy.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream).  Argument errors are detected on the host before
 *    anything is enqueued and return without side effects; launch errors
 *    return AMPED_ERR_CUDA.  amped_last_error() describes the last failure
 *    of the calling thread.
 *  - A handle may be used from one host thread at a time; calls on the same
 *    handle that overlap on the GPU (different streams) race on the
 *    handle's scratch buffers, so serialise them on one stream.
 */
#ifndef AMPED_H
#define AMPED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMPED_MAX_MODES 8

typedef enum {
    AMPED_OK = 0,
    AMPED_ERR_INVALID = -1,     /* bad argument (null pointer, size, mode, alignment) */
    AMPED_ERR_INDEX = -2,       /* a coordinate lies outside its mode's range (in a build compiled
                                   with -DAMPED_CHECKS=1 also: a kernel's device bounds check failed;
                                   the access was clamped and the message names the check) */
    AMPED_ERR_OOM = -3,         /* host or device allocation failed */
    AMPED_ERR_CUDA = -4,        /* a CUDA runtime call or kernel launch failed */
    AMPED_ERR_UNSUPPORTED = -5, /* rank / dtype / mode count this build has no kernel for */
    AMPED_ERR_TIMEOUT = -6      /* reserved: a bounded device wait gave up (no kernel waits today) */
} amped_status;

typedef enum { AMPED_F32 = 0, AMPED_BF16 = 1, AMPED_F16 = 2 } amped_dtype;

/* Options for amped_tensor_create.  Zero-initialise and set what you need;
 * a field left at 0 takes its default. */
typedef struct {
    int32_t segment_items; /* work items (nonzeros + output rows) per long-row segment; default:
                              (nnz + rows) / (8 x resident warps), clamped to 256..4096 */
    int32_t keep_perm;     /* 1 = keep each copy's nonzero permutation on the device (needed by
                              amped_cp_grad); 2 = do not keep it; 0 = default (keep) */
    int32_t keep_coo;      /* 1 = keep the coordinates in caller order on the device (needed by
                              amped_cp_sample); 2 = do not keep; 0 = default (keep) */
    int32_t max_rank;      /* rank the scratch is first sized for (grown on demand); default 64 */
    int32_t host_threads;  /* threads for the host reorder; 0 = all available */
    int32_t inner_order;   /* order of the nonzeros inside an output row: 1 = caller order (stable);
                              2 = lexicographic in the other coordinates, the mode with the largest
                              dimension most significant (ties: lower mode index), so consecutive
                              nonzeros share factor rows the kernel keeps in registers; 3 = the same
                              with the smallest dimension most significant; 0 = default (2); other
                              values are AMPED_ERR_INVALID */
    int32_t short_rows;    /* rows with fewer nonzeros than this (at most 125) are "short": they are
                              sorted by length and processed one row per lane group; longer rows are
                              processed by whole warps along the merge path.  0 = default (32);
                              negative = every row with a nonzero is long */
    int32_t stream_memory; /* where the per-nonzero streams of the copies live (coordinates, values,
                              permutations, caller-order coordinates): 1 = device memory; 2 = pinned
                              host memory mapped into the device's address space, read by the
                              kernels over the host link (out-of-core: the tensor may exceed HBM;
                              factors, outputs, row tables and scratch stay on the device);
                              0 = default (1) */
} amped_opts;

typedef struct amped_tensor* amped_tensor_t;

/*
 * Build the per-mode copies of a COO tensor (paper Sec. 3: one copy of the
 * tensor per output mode, Sec. 3.1 tensor sharding, Sec. 3.2 inter-shard
 * partitioning; here the whole tensor is one shard on one GPU).
 *   nnz      number of nonzeros, 0 <= nnz < 2^31
 *   nmodes   N, 1..AMPED_MAX_MODES
 *   dims     host array [N], each >= 1
 *   idx      host array [nnz][N] int32, 0-based (array-of-structs, caller order)
 *   vals     host array [nnz] fp32
 *   opts     NULL for defaults
 *   out      receives the handle
 * For every mode d the nonzeros are grouped by output row i_d (inside a row as opts.inner_order
 * says) and stored as struct-of-arrays (the N-1 other coordinates and the value).  Rows with at
 * least opts.short_rows nonzeros ("long") come first and are cut into merge-path segments of at
 * most `segment_items` work items (one per nonzero and one per row end), so a row longer than a
 * segment is split across segments; the other rows follow, sorted by length, in small segments.
 * Returns AMPED_ERR_INDEX (and names the first bad nonzero in
 * amped_last_error) when a coordinate is out of range.  The copies live on
 * the device that is current when this is called, and every later call on
 * the handle must run with that device current.  Synchronous: the copies are
 * on the device when it returns.  Host memory is borrowed only for the
 * duration of the call.
 */
amped_status amped_tensor_create(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx,
                                 const float* vals, const amped_opts* opts, amped_tensor_t* out);

/* Free every device and host buffer of the handle (synchronises the device first). NULL is a no-op. */
amped_status amped_tensor_destroy(amped_tensor_t t);

/* Shape queries (host only). */
amped_status amped_tensor_info(amped_tensor_t t, int64_t* nnz, int* nmodes, int64_t* dims /* [N] or NULL */);

/*
 * Mode-`mode` MTTKRP (paper Sec. 3 elementwise computation, Alg. 2):
 *   out(i, r) = sum over nonzeros x with i_mode = i of val(x) * prod_{n != mode} A_n(i_n, r)
 *   factors  host array of N device pointers; factors[n] is [dims[n]][R] in `fdtype`;
 *            factors[mode] is not read and may be NULL
 *   R        rank, 1..256 for fp32 and 1..512 for bf16/fp16 (R > 32 needs R % 8 == 0 for fp32,
 *            R % 16 == 0 for 16-bit); tensors of 2 to 8 modes
 *   out      device [dims[mode]][R] fp32, fully overwritten (rows without nonzeros become 0)
 * Enqueues a scratch reset, the persistent MTTKRP kernel and the split-row combine on `stream`.
 */
amped_status amped_mttkrp(amped_tensor_t t, int mode, const void* const* factors, amped_dtype fdtype, int R,
                          float* out, void* stream);

/* All modes back to back with the same input factors (paper Alg. 1 on one GPU, without the
 * all-gather): outs[d] receives the mode-d MTTKRP.  outs is a host array of N device pointers. */
amped_status amped_mttkrp_all(amped_tensor_t t, const void* const* factors, amped_dtype fdtype, int R,
                              float* const* outs, void* stream);

/*
 * amped_mttkrp_all on HOST buffers: copies the factors host->device into staging owned by the
 * handle, runs every mode, copies the outputs device->host, and returns when the outputs are on
 * the host.  factors: host array of N host pointers ([dims[n]][R] in fdtype); outs: host array
 * of N host pointers ([dims[n]][R] fp32).  Page-locked host memory gives full copy bandwidth.
 */
amped_status amped_mttkrp_all_host(amped_tensor_t t, const void* const* factors, amped_dtype fdtype, int R,
                                   float* const* outs, void* stream);

/*
 * Sampled CP model (paper Sec. 2.1, CPD) at every nonzero, in caller order:
 *   m_out[k] = sum_r prod_n A_n(i_n(k), r)        (device [nnz] fp32, overwritten)
 * Needs the handle's caller-order coordinates (opts.keep_coo).
 */
amped_status amped_cp_sample(amped_tensor_t t, const void* const* factors, amped_dtype fdtype, int R,
                             float* m_out, void* stream);

/*
 * Gradient of a loss L(m) of the sampled model (the CP model of paper Sec. 2.1 read at the
 * nonzeros), given gvals[k] = dL/dm_k in caller order (device [nnz] fp32).  By the chain rule
 * dm_k/dA_n(i, r) is the product of the other modes' factor entries at nonzero k, so the gradient
 * is the elementwise computation of paper Sec. 3 (Alg. 2) with each nonzero's value replaced by
 * gvals[k]:
 *   grads[n](i, r) = sum over nonzeros k with i_n(k) = i of gvals[k] * prod_{w != n} A_w(i_w(k), r)
 * i.e. the mode-n MTTKRP with the values replaced by gvals, for every n.  grads: host array of N
 * device pointers [dims[n]][R] fp32, overwritten.  Needs opts.keep_perm.
 */
amped_status amped_cp_grad(amped_tensor_t t, const void* const* factors, amped_dtype fdtype, int R,
                           const float* gvals, float* const* grads, void* stream);

/*
 * Fused gradient of the CP completion loss over the tensor's own values x (the values given to
 * amped_tensor_create), without materialising the sampled model or the residuals:
 *   r_k = m_k - x_k,  m_k = sum_r prod_n A_n(i_n(k), r)          (CP model, paper Sec. 2.1)
 *   grads[n](i, r) = sum_{k: i_n(k) = i} r_k * prod_{w != n} A_w(i_w(k), r)   (Sec. 3 EC with r_k)
 *   *loss = 1/2 sum_k r_k^2                                      (fp64, device; may be NULL)
 * One pass per mode over that mode's copy: each nonzero's model value is rebuilt from the
 * output mode's factor row and the gathered Khatri-Rao row.  grads: host array of N device
 * pointers [dims[n]][R] fp32, overwritten.  Equal to amped_cp_grad with gvals = m - x.
 */
amped_status amped_cp_completion_grad(amped_tensor_t t, const void* const* factors, amped_dtype fdtype, int R,
                                      float* const* grads, double* loss, void* stream);

/*
 * ||X||^2 of the tensor given to amped_tensor_create, with repeated coordinates summed into one
 * entry (fp64, computed on the host at create time).  *norm2 is a host double.
 */
amped_status amped_tensor_norm2(amped_tensor_t t, double* norm2);

/*
 * Host-only: the same ||X||^2 computed from host arrays without a GPU (the norm amped_tensor_create
 * stores).  inner_order as in amped_opts (0 = default); *norm2 is a host double.
 */
amped_status amped_norm2_host(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, const float* vals,
                              int inner_order, double* norm2);

/* amped_cp_als_sweep flag: compute grams[n] = A_n^T A_n of the given factors before the sweep. */
#define AMPED_ALS_INIT 1

/*
 * One sweep of CP decomposition by alternating least squares (paper Sec. 2.1: ALS performs the
 * mode-wise MTTKRPs of Eq. 1 in turn; the least-squares update after each MTTKRP is the standard
 * CP-ALS normal-equation step, which the paper does not spell out).  For d = 0 .. N-1, each step
 * seeing the factors updated before it:
 *   M        = MTTKRP_d(X; A_n, n != d)                         (amped_mttkrp, fp32)
 *   V        = Hadamard product over n != d of grams[n]         (fp64)
 *   A_d      = M V^-1                                           (fp64 Cholesky of V; the product
 *                                                                in fp32, on the tensor cores
 *                                                                with a 3-term TF32 split at R = 32)
 *   grams[d] = A_d^T A_d of the stored fp32 values              (fp64)
 * The columns are NOT normalised between modes: least-squares updates are covariant under column
 * scaling, so the models [[A_0, ..., A_{N-1}]] equal those of the per-step normalised algorithm.
 * Call amped_cp_als_normalize for unit-norm factors and lambda.  After the sweep, for the model
 * X^ = [[A_0, ..., A_{N-1}]]:
 *   stats[0] = 1 - ||X - X^|| / ||X||        stats[1] = ||X - X^||^2 (clamped at 0)
 *   stats[2] = ||X||^2                       stats[3] = <X, X^>      stats[4] = ||X^||^2
 *   stats[5] = modes whose V was singular in this sweep (their factor and Gram are left
 *              unchanged; a singular last mode sets stats[0..4] to NaN)
 *   stats[6] = first such mode + 1, or 0
 * factors: host array of N device pointers [dims[n]][R] fp32, 16-byte aligned (32-byte when R is
 *          a multiple of 8), updated in place.
 * grams:   device [N][R][R] fp64; on entry the Grams of the factors (or pass AMPED_ALS_INIT to
 *          compute them), on return those of the updated factors.
 * stats:   device [8] fp64.  1 <= R <= 64 (R > 32 a multiple of 8); 2 to 8 modes.
 * The MTTKRP output and the solve's result live in workspace the handle allocates on first use
 * (dims_max x R fp32).  Asynchronous: read stats after synchronising the stream.
 */
amped_status amped_cp_als_sweep(amped_tensor_t t, float* const* factors, int R, double* grams, double* stats,
                                int flags, void* stream);

/*
 * One CP-ALS mode update (the step amped_cp_als_sweep repeats for d = 0 .. N-1): the mode-`mode`
 * MTTKRP, the fp64 solve against the Hadamard product of the other Grams, factors[mode] replaced by
 * the unnormalised least-squares update and grams[mode] by its Gram; stats as for a sweep, for the
 * model after this update (stats[5..6] count this update only).  Same arguments and flags as
 * amped_cp_als_sweep, plus the mode.
 */
amped_status amped_cp_als_update(amped_tensor_t t, int mode, float* const* factors, int R, double* grams,
                                 double* stats, int flags, void* stream);

/*
 * Normalised form of a CP model [[A_0, ..., A_{N-1}]] = [[lambda; B_0, ..., B_{N-1}]]: every
 * factor's columns scaled to unit 2-norm in place (a zero column stays zero), lambda_r = product
 * over n of the column norms (device [R] fp32), and grams (device [N][R][R] fp64, the Grams of the
 * factors on entry) rescaled to the unit-norm factors.  One pass over every factor.
 */
amped_status amped_cp_als_normalize(amped_tensor_t t, float* const* factors, int R, double* grams, float* lambda,
                                    void* stream);

/* Sizes of a mode's plan (amped_plan_mode). */
typedef struct {
    int64_t nnz, rows;                    /* nonzeros; rows of the mode (dims[mode]) */
    int64_t long_rows, long_nnz;          /* long rows and their nonzeros (copy positions 0 .. long_nnz) */
    int64_t short_rows;                   /* short rows, including rows without nonzeros */
    int64_t long_segments, short_segments, split_rows;
} amped_plan_sizes;

/*
 * Host-only planning query: the reorder, row classes and segment tables that amped_tensor_create
 * builds for mode `mode`, without touching the GPU (for inspection and tests).  segment_items,
 * inner_order and short_rows as in amped_opts (0 = defaults, except segment_items 0 = 1024 here).  Call once with every array NULL to
 * read `sizes`, then again with buffers of these lengths (any may be NULL to skip it):
 *   perm          [nnz]               caller index of the k-th nonzero of the mode's copy
 *   rows_long     [long_rows]         row ids of the long rows (increasing)
 *   rowptr_long   [long_rows+1]       copy positions of long row j: rowptr_long[j] .. rowptr_long[j+1]
 *   seg_row       [long_segments+1]   long rows completed before long segment s (merge path)
 *   seg_nz        [long_segments+1]   nonzeros consumed before long segment s
 *   splits        [split_rows][3]     {long-row index, s_a, s_b}: the row straddles boundaries s_a..s_b
 *   rows_short    [short_rows]        row ids of the short rows (by decreasing length)
 *   rowptr_short  [short_rows+1]      copy positions of short row j (rowptr_short[0] = long_nnz)
 *   seg_short     [short_segments+1]  first short row of short segment t
 * Coordinates are validated as in create.
 */
amped_status amped_plan_mode(int64_t nnz, int nmodes, const int64_t* dims, const int32_t* idx, int mode,
                             int segment_items, int inner_order, int short_rows, amped_plan_sizes* sizes,
                             int32_t* perm, int32_t* rows_long, int32_t* rowptr_long, int32_t* seg_row,
                             int32_t* seg_nz, int32_t* splits, int32_t* rows_short, int32_t* rowptr_short,
                             int32_t* seg_short);

/*
 * Size of the library's fixed device scratch buffer used by amped_mttkrp_noalloc (32 MiB).
 * It is reserved on a device when the first handle is created there (amped_tensor_create looks
 * up the buffer's device address, which loads the module that holds it) and stays reserved
 * until the process exits.
 */
#define AMPED_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/*
 * amped_mttkrp without any device memory allocation.  (Not from the paper: the paper has no
 * counterpart; this is a deployment convenience of this library.)
 *
 * Who needs it: callers that must not allocate device memory while they run, for example code
 * that hands every byte of the GPU to its own memory pool or arena, code with a fixed memory
 * budget reserved up front, or a latency-sensitive loop where cudaMalloc's implicit device
 * synchronisation is not acceptable.  amped_mttkrp may allocate (or grow) the handle's scratch
 * on a call with a larger rank than before; this entry point never does.  It computes exactly
 * what amped_mttkrp computes for the same arguments.
 *
 * Scratch: the split-row partials, their fp64 task sums and the segment ticket counter live in
 * one static device array of AMPED_NOALLOC_SCRATCH_BYTES that the library defines.  A call whose
 * mode needs more (4*2*S*R + 8*tasks*R bytes plus 256 for S segments and the mode's combine
 * tasks) returns AMPED_ERR_UNSUPPORTED without launching anything; use amped_mttkrp then, or a
 * larger segment_items at create time (fewer segments).
 *
 * Set-up: amped_tensor_create looks up the array's address on its device (cudaGetSymbolAddress,
 * with that device current), once per device, so this call itself only reads the cached address.
 * The device current at the call must be the handle's device (else AMPED_ERR_INVALID).  If that
 * lookup failed at create time, this call returns AMPED_ERR_CUDA.  The array is shared by every
 * handle and every call on the device and keeps the last call's contents (the ticket counter is
 * cleared on the call's stream before each launch): calls that may overlap on the GPU (different
 * streams, other threads) race on it, so serialise them.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  Honours amped_set_kernel_events like amped_mttkrp.
 */
amped_status amped_mttkrp_noalloc(amped_tensor_t t, int mode, const void* const* factors, amped_dtype fdtype,
                                  int R, float* out, void* stream);

/* Profiling hook: record `start` / `stop` (cudaEvent_t, may be NULL) on the call's stream
 * immediately before and after the next MTTKRP kernel launch of this handle; cleared after use. */
amped_status amped_set_kernel_events(amped_tensor_t t, void* start, void* stop);

/* Number of CUDA kernels this library has launched in this process (all handles). */
int64_t amped_kernel_launches(void);

/* Message describing the last error returned to the calling thread ("" if none).
 * Fault injection for testing clean-up paths (host side only): with the environment variable
 * AMPED_FAULT=alloc:K, the K-th device allocation (1-based) inside each entry-point call fails as
 * if the device were out of memory; the call then frees what it built and returns AMPED_ERR_OOM.
 * The variable is read at every allocation. */
const char* amped_last_error(void);

/* Library version string. */
const char* amped_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AMPED_H */
