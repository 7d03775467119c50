/*
 * bed.h -- C ABI of the batched divide-and-conquer symmetric eigensolver for mini-batches of small
 * FP32 matrices (1 <= n <= 64) on NVIDIA GB300 (sm_103a).
 *
 * Method: Y. Song, "A Short Note on Batch-efficient Divide-and-Conquer Algorithm for
 * EigenDecomposition" (arXiv 2604.27325), Sec. 2. Each matrix is reduced to tridiagonal form by
 * Householder reflections (Sec. 2 defers this stage to the authors' earlier work), torn into
 * rank-one-coupled blocks (Sec. 2.1, Eq. (1)-(3)) down to leaves of at most 8 rows (Sec. 2.2: 1x1 and
 * 2x2 leaves in closed form, larger ones by the implicit QL iteration), merged back through
 * the secular equation (Sec. 2.3, Eq. (4)-(22)) with Gu-Eisenstat eigenvectors (Eq. (23)-(25)), and
 * back-transformed. One launch runs the whole path for every matrix of the batch; each matrix lives
 * in one thread block's shared memory.
 *
 * Conventions shared by every entry point:
 *   - Matrices are dense, row-major, contiguous FP32: A[b][i][j] at A + (b*n + i)*n + j.
 *   - Only the lower triangle (i >= j) of A is read (the upper triangle may hold anything).
 *   - W[b][j] (b*n + j) receives the eigenvalues in ascending order; V[b][i][j] receives component i
 *     of the eigenvector of W[b][j] (eigenvectors are the COLUMNS of V[b]), so that
 *     A[b] = V[b] diag(W[b]) V[b]^T. Each eigenvector is scaled to unit length and signed so that
 *     its entry of largest magnitude (first such index on ties) is positive.
 *   - info[b] receives a bit set of BED_INFO_* flags (0 = success); info may be NULL.
 *   - All data pointers are DEVICE pointers owned by the caller; the library allocates no device
 *     memory per call, never synchronizes, and returns as soon as the work is enqueued on `stream`
 *     (0 = the legacy default stream). Results are ready when `stream` reaches that point.
 *   - Argument errors are returned before anything is enqueued. A launch failure returns
 *     BED_ERR_CUDA (the CUDA error string is available through bed_last_cuda_error()).
 *   - Numerical outcomes never fail the call: they are reported per matrix through info.
 */
#ifndef BED_H
#define BED_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BED_OK = 0,
    BED_ERR_INVALID_ARG = 1,   /* null pointer, negative batch, misaligned pointer, bad params */
    BED_ERR_UNSUPPORTED_N = 2, /* n outside [1, bed_max_n()] */
    BED_ERR_CUDA = 3,          /* the CUDA runtime refused the launch or an attribute call */
    BED_ERR_TOO_LARGE = 4,     /* the batch exceeds a fixed capacity (bed_eigh_ragged_f32_noalloc, servers) */
    BED_ERR_TIMEOUT = 5        /* bed_server_wait: the request did not complete in time */
} bed_status;

/* per-matrix outcome flags written to info[b] */
enum {
    BED_INFO_OK = 0,
    BED_INFO_NOT_CONVERGED = 1, /* a secular root hit the iteration cap; its last iterate is kept */
    BED_INFO_NONFINITE = 2,     /* A[b] held a NaN or an infinity: W[b] and V[b] are set to NaN */
    BED_INFO_TIMEOUT = 4,       /* the staging copy of A[b] did not complete within stage_wait_us: W[b], V[b]
                                   NaN; the team goes on once the copy has landed (a second wait of at most
                                   2 s), and stops taking matrices if it never does */
    BED_INFO_BAD_N = 8          /* ragged batches: ns[b] outside [1, 64]; the matrix was skipped */
};

/*
 * Constants of the method. The paper leaves all of them unnamed; bed_default_params() gives the
 * defaults below. Passing NULL wherever a `const bed_params*` is taken means the defaults.
 */
typedef struct {
    int leaf_size;           /* divide (Sec. 2.1) until blocks have <= leaf_size rows, 1..8, or 0 (default):
                                automatic, a built-in per-n choice of 4 or 8 (and 2 for n = 2) measured by the
                                autotuner on a GB300; blocks of 3..8 rows are solved by the implicit QL
                                iteration (Sec. 2.2) */
    int k_multisection;      /* k of Eq. (16), >= 2 (default 4) */
    int max_section_iters;   /* cap on multi-section steps per root, 0..256 (default 24) */
    int max_halley_iters;    /* cap on Halley steps per root, 1..256 (default 32) */
    float section_rel_eps;   /* Eq. (17): sectioning stops when U - L < eps * (initial bracket), (0,1) (default 2^-1) */
    float stop_c;            /* Halley stops when |f| <= stop_c * u * (1 + rho sum|z^2/(d - lambda)|), u = 2^-24 (default 8) */
    float deflation_tol_scale; /* deflation tolerance = scale * u * max(max|d|, rho |z|^2) (default 8) */
    int threads_per_matrix;  /* 0 = automatic (nmax the smallest of {16, 32, 48, 64} that holds n; 4*nmax
                                threads, except 2*nmax = 128 for nmax = 64 unless merge_tensor_cores = 1);
                                otherwise 2*nmax or 4*nmax for an nmax of that set with nmax >= n, the
                                smallest such nmax when two match (64 = 4*16 or 2*32; 128 = 4*32 or 2*64) */
    int retire_by_vote;      /* 1 (default): a warp stops iterating secular roots as soon as all of its lanes
                                have converged (the recast of the paper's progressive batch shrinkage,
                                Eq. (22)); 0: every warp runs to the iteration caps with converged lanes
                                idle. Results are bitwise identical either way. */
    int merge_tensor_cores;  /* 0 (default): the merge products of Eq. (4) on the FP32 FMA pipes; 1: on the
                                tensor cores as split-3xTF32 (each operand split into two TF32 parts, three
                                mma.sync m16n8k8 per product, FP32 accumulation). Applies to launches of
                                bed_eigh_f32* with teams of 4*nmax threads; a merge level with more 16 x 8
                                tiles than the registers hold, 2*nmax teams, the ragged kernel and the
                                server use the FP32 products. Results agree with the FP32 path to the
                                same tolerance, not bitwise. */
    int stage_wait_us;       /* limit in microseconds of a team's wait for the bulk copy that stages a matrix
                                in shared memory, 0..60,000,000 (default 2,000,000); a matrix whose copy has
                                not landed by then gets BED_INFO_TIMEOUT. 0 gives up without waiting, which
                                exercises that path deterministically (the copy is still drained). */
    int matrices_per_cta;    /* uniform launches (bed_eigh_f32*): 0 (default) one thread block per matrix; k
                                in 1..2^20: ceil(batch / k) blocks, block i solving matrices i, i + blocks,
                                ... in turn (about k each) in its shared memory. Results are bitwise the same
                                whatever k; the ragged kernel and the server hand out their own units. */
    int n_bisect_first;      /* bisection steps per secular root (Eq. (13)-(15)) before the multi-section
                                steps of Eq. (16), 1..64 (default 1, the paper's single bisection); the
                                steps after the first count toward max_section_iters, and the switch to
                                Halley (Eq. (17)) may come before they are all taken */
} bed_params;

/* Fills *p with the defaults listed above. */
void bed_default_params(bed_params* p);

/*
 * Eigendecomposition of `batch` symmetric n x n FP32 matrices (Sec. 2, whole path).
 *   A     [batch][n][n] device, read-only, 4-byte aligned (16-byte alignment and even n enable the
 *         bulk-copy staging path).
 *   W     [batch][n]    device, written.
 *   V     [batch][n][n] device, written (may not alias A).
 *   info  [batch]       device int32, written; may be NULL.
 *   batch >= 0 (0: nothing is enqueued, BED_OK).
 *   n     in [1, bed_max_n()].
 *   p     NULL or parameters (validated; BED_ERR_INVALID_ARG if out of range).
 *   stream CUDA stream to enqueue on.
 */
bed_status bed_eigh_f32(const float* A, float* W, float* V, int32_t* info, int64_t batch, int n,
                        const bed_params* p, cudaStream_t stream);

/* Work counters a launch can accumulate (device memory, caller-owned, caller-zeroed). */
typedef struct {
    unsigned long long matrices;  /* matrices solved */
    unsigned long long roots;     /* secular roots solved (non-deflated eigenvalues of all merges) */
    unsigned long long evals;     /* evaluations of f (Eq. (8)) spent on those roots */
    unsigned long long deflated;  /* eigenpairs deflated in merges */
} bed_counters;

/*
 * Same as bed_eigh_f32, and additionally adds this launch's work counts to *counters (a DEVICE
 * pointer to one bed_counters, updated with atomics; may not be NULL). Used to measure the mean
 * number of secular iterations that enters the FLOP count.
 */
bed_status bed_eigh_f32_counted(const float* A, float* W, float* V, int32_t* info, int64_t batch,
                                int n, const bed_params* p, bed_counters* counters,
                                cudaStream_t stream);

/*
 * End-to-end solve of a uniform batch held in HOST memory (no counterpart in the paper: the
 * copy-in / solve / copy-out pipeline of a caller whose matrices live on the host).
 *   A_host, W_host, V_host, info_host  host buffers in the layouts of bed_eigh_f32 (info_host may be
 *            NULL); they must be page-locked (cudaHostAlloc / cudaHostRegister) for the copies to run
 *            asynchronously and overlap
 *   A_dev [batch*n*n], W_dev [batch*n], V_dev [batch*n*n], info_dev [batch] (may be NULL)
 *            caller-owned device scratch; the library allocates nothing
 *   chunks   the batch is cut into this many pieces (0: automatic, two from 256 matrices on, else one);
 *            piece c is copied in, solved and copied out on stream s[c % 2], so that the copies of one
 *            piece overlap the solve of another. s0 and s1 may be the same stream (no overlap).
 * Returns after enqueuing everything (argument errors before anything is enqueued, as bed_eigh_f32);
 * the results are in host memory once both streams have reached this call's work. The host buffers
 * must stay valid until then.
 */
bed_status bed_eigh_f32_host(const float* A_host, float* W_host, float* V_host, int32_t* info_host,
                             int64_t batch, int n, const bed_params* p, float* A_dev, float* W_dev,
                             float* V_dev, int32_t* info_dev, int chunks, cudaStream_t s0,
                             cudaStream_t s1);

/*
 * Zero-copy solve of a uniform batch held in PAGE-LOCKED HOST memory (no counterpart in the paper:
 * the input/output path of a caller whose matrices live on the host). The kernel reads every matrix
 * straight from A_host and writes W_host, V_host, info_host over the host-device link through the
 * unified address space, so that each matrix's transfers overlap the solve of the others and no
 * device buffer or copy is involved.
 *   A_host, W_host, V_host, info_host  host buffers in the layouts of bed_eigh_f32 (info_host may be
 *            NULL); each must lie inside one page-locked allocation of the current CUDA context
 *            (cudaHostAlloc, cudaMallocHost or cudaHostRegister), checked with cudaPointerGetAttributes
 *            on its first and last byte: BED_ERR_INVALID_ARG otherwise, before anything is enqueued.
 * Returns after enqueuing the launch on `stream`; the results are in host memory once the stream has
 * reached it. The buffers must stay valid and untouched by the host until then.
 */
bed_status bed_eigh_f32_pinned(const float* A_host, float* W_host, float* V_host, int32_t* info_host,
                               int64_t batch, int n, const bed_params* p, cudaStream_t stream);

/*
 * Several uniform batches of different n in page-locked host memory, solved by one call (the
 * zero-copy path of bed_eigh_f32_pinned for each batch, with the stream fork and join done here).
 *   count            number of batches (0: nothing is enqueued)
 *   ns[k], batches[k] size and matrix count of batch k (a batch of 0 matrices is skipped)
 *   A_host[k], W_host[k], V_host[k], info_host[k]  its buffers, as in bed_eigh_f32_pinned; info_host
 *                    may be NULL (no info for any batch) or hold NULL entries
 *   origin           the batches start after the work already enqueued on `origin`, and `origin` waits
 *                    for all of them (through two events the library keeps per calling thread)
 *   side, nside      streams the launches run on, largest n first, batch j of that order on
 *                    side[j % nside], so that batches of different n run side by side
 *   p                NULL or parameters for every batch. When more than one stream is used and
 *                    threads_per_matrix is 0 (automatic), batches of 17..32 rows run 64-thread teams
 *                    rather than 128: half the registers per matrix, so that more of them fit beside the
 *                    larger sizes' blocks (alone, such a batch is faster with 128 threads)
 * Every argument of every batch is checked before anything is enqueued (BED_ERR_UNSUPPORTED_N,
 * BED_ERR_INVALID_ARG); after a CUDA error (BED_ERR_CUDA) earlier launches of the call may stay
 * enqueued, still joined to `origin`.
 * The results are in host memory once `origin` has reached this call's work.
 */
bed_status bed_eigh_many_f32_pinned(int count, const int* ns, const int64_t* batches, const float* const* A_host,
                                    float* const* W_host, float* const* V_host, int32_t* const* info_host,
                                    const bed_params* p, cudaStream_t origin, const cudaStream_t* side, int nside);

/*
 * Ragged batches: matrices of mixed size in one persistent launch (Sec. 2.1 notes that dividing turns a
 * batch of B matrices into B*R blocks; here blocks of all sizes share the GPU in one launch).
 *
 * Work is handed out in units of one thread block (256 threads) split into teams, one matrix per team:
 *   team type 0: 1 team of 256 threads, any n <= 64;   type 1: 2 teams of 128 threads, n <= 32;
 *   type 2: 4 teams of 64 threads, n <= 16;            type 3: 8 teams of 32 threads, n <= 16;
 *   type 4: 1 team of 192 threads (the block's other 64 threads idle), n <= 48.
 * bed_ragged_tuning chooses the team type and the leaf size of the divide tree for every n (entries
 * 1..64 are used; an autotuner fills it by measurement).
 */
typedef struct {
    unsigned char team[65]; /* team type for each n */
    unsigned char leaf[65]; /* leaf size (1..8) for each n */
} bed_ragged_tuning;

/* Fills *t with the built-in choice: type 2 for n <= 16, type 1 for n <= 32, type 4 for n <= 48, type 0
 * above; for each n the automatic leaf size of bed_params.leaf_size = 0. */
void bed_ragged_default_tuning(bed_ragged_tuning* t);

/* Bytes of device workspace bed_eigh_ragged_f32 needs for `count` matrices (a multiple of 256). */
size_t bed_eigh_ragged_workspace_size(int64_t count);

/*
 * Eigendecomposition of `count` symmetric FP32 matrices of mixed size, in one stream-ordered pair of
 * launches (a one-block ordering pass, then the persistent kernel). All arrays are DEVICE memory:
 *   A         packed matrices; matrix b is ns[b] x ns[b] row-major at A + offsets[b] (lower triangle read)
 *   offsets   [count] int64 element offsets of each matrix in A, also used for V
 *   ns        [count] int32 sizes; a size outside [1, 64] sets info[b] = BED_INFO_BAD_N and skips b
 *   W         eigenvalues of matrix b (ascending) at W + w_offsets[b]
 *   w_offsets [count] int64 element offsets into W
 *   V         eigenvectors of matrix b (columns) at V + offsets[b]; V may not alias A
 *   info      [count] int32 flags (may be NULL)
 *   p         NULL or parameters (leaf_size and threads_per_matrix are ignored: the tuning decides)
 *   tuning    NULL (built-in choice) or a host-side table, validated (a team type must fit its n)
 *   workspace device memory of at least bed_eigh_ragged_workspace_size(count) bytes, 16-byte aligned,
 *             owned by the caller; it must not be used by another call until this one completes
 *   counters  NULL or a device bed_counters that the launch adds its work counts to
 * The first call on a device performs a one-time setup of that device (it uploads the divide trees of
 * every size, synchronously); make that first call before capturing calls into a CUDA graph. The calls
 * themselves enqueue only kernel launches and can be captured and replayed.
 */
bed_status bed_eigh_ragged_f32(const float* A, const int64_t* offsets, const int32_t* ns, int64_t count,
                               float* W, const int64_t* w_offsets, float* V, int32_t* info,
                               const bed_params* p, const bed_ragged_tuning* tuning, void* workspace,
                               size_t workspace_bytes, bed_counters* counters, cudaStream_t stream);

/*
 * Allocation-free variant of bed_eigh_ragged_f32 (the paper has no counterpart; this is a convenience
 * of this library). Some callers cannot obtain device memory for the workspace: code that runs inside
 * a host framework whose allocator owns all of the device memory it may use, plugins handed only the
 * input and output buffers, or services that must not call cudaMalloc once they are running (it may
 * fail under memory pressure and it synchronizes the device). This entry point takes no workspace:
 * it uses a scratch array compiled into the library, of fixed size, that every GPU which loads the
 * library keeps for the life of the process.
 *   - At most BED_NOALLOC_MAX_COUNT matrices per call; a larger count returns BED_ERR_TOO_LARGE
 *     before anything is enqueued. The scratch holds BED_NOALLOC_SCRATCH_BYTES bytes.
 *   - The first call on a device looks up the scratch's device address (and performs the same
 *     one-time device setup as bed_eigh_ragged_f32); make that first call before any stream capture.
 *   - Every call on a device uses the same scratch, and it keeps what the last call left there: the
 *     launches reset everything they read before reading it. Two calls whose work overlaps on the
 *     GPU (different streams without ordering between them) race on the scratch and give undefined
 *     results; order such calls or use bed_eigh_ragged_f32 with separate workspaces.
 *   - It calls no allocation routine. Arguments otherwise as for bed_eigh_ragged_f32.
 *   - The looked-up address and the device setup are cached per device for the life of the process;
 *     after cudaDeviceReset the library must be reloaded before it is used on that device again.
 */
#define BED_NOALLOC_MAX_COUNT 65536
#define BED_NOALLOC_SCRATCH_BYTES ((64 + 4 * BED_NOALLOC_MAX_COUNT + 255) / 256 * 256)
bed_status bed_eigh_ragged_f32_noalloc(const float* A, const int64_t* offsets, const int32_t* ns, int64_t count,
                                       float* W, const int64_t* w_offsets, float* V, int32_t* info,
                                       const bed_params* p, const bed_ragged_tuning* tuning,
                                       bed_counters* counters, cudaStream_t stream);

/*
 * Backward of the eigendecomposition layer (the paper's introduction motivates ED as a differentiable
 * layer of a network): given the outputs W [batch][n], V [batch][n][n] of bed_eigh_f32 and the
 * gradients of a loss with respect to them, gW (same shape as W) and gV (same shape as V), writes
 *     gA = (G + G^T)/2,  G = V (diag(gW) + F o (V^T gV)) V^T,
 * F_ij = 1/(W_j - W_i) when |W_j - W_i| > gap_eps (i != j) and 0 otherwise (pairs that close are not
 * separable eigenvectors), into gA [batch][n][n]. gA is the gradient over symmetric perturbations of A
 * (torch.linalg.eigh's convention). All pointers DEVICE memory; gW or gV may be NULL (zero gradient);
 * gA may not alias V. gap_eps >= 0 and finite. Same ownership, error and stream rules as bed_eigh_f32.
 * gap_eps = 0 masks exact ties only. FP32 eigenvalues closer than about n * 2^-24 * max|W| cannot be
 * told apart, and 1/(W_j - W_i) for such a pair is rounding noise of size up to 2^24 / (n max|W|):
 * for inputs that may have (nearly) repeated eigenvalues pass a gap_eps of at least that size, e.g.
 * 1e-6 * max|W| (the differentiation workload, with gaps >= 1e-3, needs none).
 */
bed_status bed_eigh_backward_f32(const float* W, const float* V, const float* gW, const float* gV, float* gA,
                                 int64_t batch, int n, float gap_eps, cudaStream_t stream);

/*
 * Request loop (continuous batching) for serving eigendecompositions on the current device (no
 * counterpart in the paper, whose introduction motivates the method by training and inference).
 * A request is b matrices of one size n in host memory (row-major, lower triangle read). The server
 * admits requests in arrival order while their results fit `host_result_bytes` of pinned host memory
 * and whatever they stage in the device arena fits `device_budget_bytes`; everything admitted since
 * the previous launch is solved by one ragged launch (the persistent kernel of bed_eigh_ragged_f32) on
 * a free one of `streams` streams, so requests that arrive while others run are admitted as slots and
 * memory free up and their work overlaps on the device. A launch that carries a single request uses
 * the uniform kernel with the ragged kernel's team shape and leaf size for its n, so a request's results
 * are the same whether or not it shared a launch. With zero_copy = 1 (default) a page-locked input is
 * read by the kernels in place and the results are written straight into the pinned result memory
 * (inputs that are not page-locked are copied into the device arena first); with zero_copy = 0 inputs
 * and results pass through the device arena with copies. A completion thread polls every launch in
 * flight and retires each as soon as it is done. mode 1 instead runs one uniform-size launch (default
 * parameters) per request, first come first served, on one stream (the plain per-request baseline,
 * with the same data path). The server allocates its device and pinned host memory once, in
 * bed_server_create, and owns two threads; every entry point below is thread-safe.
 */
typedef struct bed_server bed_server;

typedef struct {
    size_t device_budget_bytes; /* device arena (default 4 GB) */
    size_t host_result_bytes;   /* pinned host memory for results held until released (default 2 GB) */
    int streams;                /* launches that may be in flight at once (default 3; 1 in mode 1) */
    int max_launch_matrices;    /* cap on the matrices of one launch (default 16384) */
    int mode;                   /* 0: continuous batching (default); 1: one launch per request */
    int zero_copy;              /* 1 (default): page-locked inputs read in place, results written in place;
                                   0: inputs and results copied through the device arena */
} bed_server_config;

typedef struct {
    int64_t requests, matrices, launches; /* completed since creation or the last reset */
    int64_t peak_device_bytes;            /* largest arena footprint admitted */
    double p50_s, p99_s, mean_s, max_s;   /* request latency: submit to results in host memory */
    double span_s;                        /* first submit to last completion */
    /* where the slowest requests spent their time, each the largest since creation or the last reset:
       submit to admission into a launch (waiting for a slot, or for memory that releases free), the
       host enqueueing one launch, and a launch's enqueue to the completion thread seeing it done */
    double max_admit_wait_s, max_enqueue_s, max_inflight_s;
} bed_server_stats;

void bed_server_default_config(bed_server_config* c);

/* Creates a server on the current device. p, t: NULL or parameters / ragged tuning (as for
 * bed_eigh_ragged_f32). Returns BED_ERR_CUDA if the device or pinned memory cannot be allocated. */
bed_status bed_server_create(const bed_server_config* cfg, const bed_params* p, const bed_ragged_tuning* t,
                             bed_server** out);

/* Queues b x n x n FP32 matrices at A_host (host memory that must stay unchanged until the request
 * completes; page-locked memory is read in place by the kernels under zero_copy, other memory is copied
 * to the device arena). *request_id identifies it. A request that alone exceeds the budgets or has more
 * than max_launch_matrices matrices is refused with BED_ERR_TOO_LARGE (it still gets an id to release). */
bed_status bed_server_submit(bed_server* s, const float* A_host, int32_t b, int32_t n, int64_t* request_id);

/* Waits up to timeout_s seconds (< 0: without limit) for a request; on BED_OK, *V ([b][n][n], columns
 * are eigenvectors), *W ([b][n], ascending) and *info ([b]) point into the server's pinned result
 * memory, valid until bed_server_release. Returns the request's status (BED_ERR_TOO_LARGE for a refused
 * request) or BED_ERR_TIMEOUT. Any pointer argument may be NULL. */
bed_status bed_server_wait(bed_server* s, int64_t id, double timeout_s, const float** W, const float** V,
                           const int32_t** info);

/* Returns a completed request's result memory to the server and forgets the id. */
bed_status bed_server_release(bed_server* s, int64_t id);

bed_status bed_server_get_stats(bed_server* s, bed_server_stats* out);
bed_status bed_server_reset_stats(bed_server* s);

/* Stops the threads after the queued requests are launched, waits for the device, frees everything. */
void bed_server_destroy(bed_server* s);

/*
 * FP32 FMA throughput probe (no counterpart in the paper: it measures the denominator of the
 * eigensolver's FP32 ALU roofline). Launches `blocks` x `threads` threads (threads a multiple of 32,
 * at most 256), each running bed_fma_peak_chains() independent FMA chains for `iters` rounds, and
 * writes one float per thread to out [blocks * threads] (device memory) so the work is kept. The caller
 * times the launch: it performs 2 * bed_fma_peak_chains() * iters * blocks * threads FP32 FLOPs.
 */
int bed_fma_peak_chains(void);
bed_status bed_fma_peak_launch(float* out, int blocks, int threads, int iters, cudaStream_t stream);

/* Largest supported n (64). */
int bed_max_n(void);

/* Static string naming a status code. */
const char* bed_status_string(bed_status s);

/* Text of the last CUDA error seen by a failing call on this thread ("" if none). */
const char* bed_last_cuda_error(void);

/*
 * Host-side description of the divide tree the kernels follow for size n (Sec. 2.1: split at
 * floor(s/2) until blocks have <= leaf_size rows; leaf_size 0 = the automatic choice for n). Pure host
 * logic, no CUDA call.
 *   merges  [3*64] receives (lo, mid, hi) of each merge, deepest level first (may be NULL)
 *   level_of[64]   receives the merge level (0 = deepest) of each merge (may be NULL)
 * Returns the number of merges (n - number of leaves), or -1 for an unsupported n / leaf_size.
 */
int bed_plan_describe(int n, int leaf_size, int* merges, int* level_of);

#ifdef __cplusplus
}
#endif

#endif /* BED_H */
