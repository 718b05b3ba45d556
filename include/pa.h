/*
 * pa.h — C ABI of the GB300 (sm_103a) Toeplitz-hash library for length-compatible
 * privacy amplification (Wang, Zhang, Yu, Guo, arXiv 1805.02372).
 *
 * The operation (Sec. 2.1 Eq. 1; Sec. 2.3 Steps 1-2): an m x n binary Toeplitz
 * matrix T, fixed by an (n+m-1)-bit seed s through
 *
 *        T[i][j] = s[n-1+i-j]        0 <= i < m, 0 <= j < n,
 *
 * compresses the n-bit corrected key x into the m-bit final key
 *
 *        y[i] = XOR_j ( x[j] AND s[n-1+i-j] )  =  (T x mod 2)[i].
 *
 * Equivalently (Sec. 3, Step 3) y[i] is coefficient n-1+i of the product of the
 * polynomials s(z) and x(z), reduced mod 2. The paper's r = u T with T of size
 * n x l is the transpose of this m x n form: the same bits, with l = m.
 *
 * Bit buffers: bit j of a string is bit (j & 63) of uint64_t word (j >> 6).
 *   key  : ceil(n/64) words; bits at positions >= n are ignored.
 *   seed : ceil((n+m-1)/64) words; bits at positions >= n+m-1 are ignored.
 *   out  : ceil(m/64) words; fully overwritten, bits at positions >= m set to 0.
 * Device buffers must be 16-byte aligned (PA_ERR_ALIGN otherwise). The caller owns
 * every bit buffer; a plan owns its device workspace. Calls that take a stream
 * are asynchronous on it; no call synchronises the device unless it says so.
 * No C++ exception crosses this interface: every call returns a pa_status.
 * Several plans may be used concurrently on different streams; a single plan must
 * not be used by two calls that overlap on the GPU (its workspace is shared).
 */
#ifndef PA_H
#define PA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (0 = success, negative = error). */
#define PA_OK 0
#define PA_ERR_INVALID (-1)     /* n == 0, m == 0, null pointer, bad option or size   */
#define PA_ERR_ALIGN (-2)       /* a device bit buffer is not 16-byte aligned          */
#define PA_ERR_NOMEM (-3)       /* device or host allocation failed                    */
#define PA_ERR_CUDA (-4)        /* a CUDA runtime call failed (see pa_last_cuda_error) */
#define PA_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up                  */
#define PA_ERR_UNSUPPORTED (-6) /* the requested path cannot run these sizes           */
#define PA_ERR_PRECISION (-7)   /* FFT tile whose proven rounding bound is not < 1/2   */
#define PA_ERR_TOO_LARGE (-8)   /* sizes exceed pa_hash_direct_static's fixed scratch  */

/* Interchangeable kernels. Every path returns the same bits. */
typedef enum {
    PA_PATH_AUTO = 0,       /* planner / autotuner choice                                */
    PA_PATH_DIRECT = 1,     /* bit-packed AND + popcount parity (Sec. 2.1 definition)    */
    PA_PATH_NTT64 = 2,      /* exact NTT modulo 2^64-2^32+1 (Sec. 3, FFT route, exact)  */
    PA_PATH_NTT31 = 3,      /* exact NTT modulo a prime below 2^31 (5*2^25+1, 7*2^26+1 or
                               15*2^27+1: see pa_opts.ntt_prime; sums grouped so every
                               coefficient count stays below p)                          */
    PA_PATH_FFT = 4,        /* FP32 FFT sub-blocks under a proven rounding bound; FP64
                               butterflies on the tile lengths where the FP32 bound fails */
    PA_PATH_BLOCK_INT8 = 5, /* block-Toeplitz Y = sum_d T_d X_d, INT8 tensor cores,
                               INT32 accumulation, then mod 2                            */
    PA_PATH_BLOCK_FP8 = 6   /* the same block-Toeplitz contraction on the tcgen05 tensor
                               cores: bits as e4m3 0 / 2^-6, FP32 accumulation in tensor
                               memory (exact: at most 2^15 products per partial sum,
                               a multiple of 2^-12 below 8),
                               then mod 2; tile edge b = 128                             */
} pa_path;

/* Planner options; zero-initialise and set what you need (0 / -1 = choose). */
typedef struct {
    int32_t path;              /* pa_path                                                 */
    int32_t device;            /* CUDA device ordinal, -1 = current device                */
    uint32_t log2_transform;   /* transform paths: log2 of the transform size N           */
    uint32_t block_b;          /* block paths: tile edge b, INT8 in {128, 256, 512}, FP8 128 */
    uint64_t tile_in;          /* key sub-block length L (the paper's batch length); block
                                  FP8: contraction positions per CTA chunk, a multiple of
                                  128 up to 32768                                         */
    uint64_t tile_out;         /* output sub-block length M (column split of Sec. 3). An
                                  NTT geometry that would need more than 2^22 tile pairs
                                  without transform-domain sums is PA_ERR_UNSUPPORTED     */
    uint32_t force_fp64;       /* FFT path: use FP64 butterflies even where FP32 is proven */
    uint32_t max_slots;        /* batches: at most this many transform spectra resident at
                                  once (reused round-robin, >= 4); 0 = automatic         */
    uint32_t fd_mode;          /* NTT paths with several key and output sub-blocks: sum the
                                  products of an output sub-block in the transform domain
                                  (each key and seed-window spectrum computed once, one
                                  inverse per output sub-block). 0 = when the planner
                                  estimates it faster, 1 = never, 2 = whenever possible   */
    uint32_t ntt_prime;        /* PA_PATH_NTT31: 28 = 5*2^25+1, 29 = 7*2^26+1, 31 =
                                  15*2^27+1; 0 = 28 when n < 5*2^25+1 (no count exceeds
                                  n), else 29 (the lazily reduced 28-bit field's
                                  transforms take fewer reduction steps). Any n:
                                  a tile pair's counts are at most L < p, and a transform-
                                  domain sum covers at most (p-1)/L key sub-blocks (longer
                                  keys take several sums per output sub-block, their bits
                                  XOR-merged as Eq. finalkey merges sub-blocks)           */
    uint32_t fd_group;         /* transform-domain sums: at most this many key sub-blocks
                                  per sum; 0 = the prime's exactness limit (p-1)/L. Like
                                  fd_mode it also binds an autotuned batch's NTT blocks  */
    uint32_t seg_in;           /* transform-domain sums run in segments (the paper's blocks
                                  run serially through a fixed workspace, Sec. 3): key
                                  sub-blocks per segment; 0 = automatic (segments only when
                                  the resident spectra would exceed 96 GiB)               */
    uint32_t seg_out;          /* segments: output sub-blocks per slice; 0 = automatic     */
    uint32_t seg_cap_gib;      /* segments: GiB of spectra one segment may hold; 0 = 32    */
    uint32_t outer_mode;       /* transform-domain sums with equal key and output sub-blocks
                                  are, bin by bin, convolutions over the sub-block index
                                  (the window of (I, J) depends on I - J); computed with
                                  transforms over that index instead of one product per
                                  (I, J): 0 = when the planner estimates it faster,
                                  1 = never, 2 = whenever possible                        */
    uint32_t reserved[3];
} pa_opts;

/* What a plan decided (pa_plan_query / pa_plan_describe). */
typedef struct {
    uint64_t n, m;
    int32_t path;              /* resolved pa_path                                        */
    uint32_t log2_transform;   /* transform size N = 2^log2_transform (transform paths)   */
    uint64_t tile_in;          /* key sub-block length L (block FP8: contraction positions
                                  per CTA chunk)                                          */
    uint64_t tile_out;         /* output sub-block length M (block FP8: outputs per tile)  */
    uint64_t tiles_in;         /* p: number of key sub-blocks (block FP8: chunks per tile) */
    uint64_t tiles_out;        /* q: number of output sub-blocks (block FP8: output tiles) */
    uint32_t block_b;          /* block path tile edge                                    */
    uint32_t fp64;             /* FFT path runs FP64 butterflies                          */
    double rounding_bound;     /* FFT path: proven bound on |v - rint(v)|, else 0         */
    uint64_t workspace_bytes;  /* device workspace owned by the plan                      */
    uint32_t kernels_per_call; /* kernel launches one pa_hash enqueues                    */
    uint32_t fd;               /* NTT: transform-domain accumulation (see pa_opts.fd_mode) */
    uint64_t windows;          /* with fd: seed-window spectra computed (distinct offsets) */
    uint32_t prime_bits;       /* NTT paths: bits of the prime (28, 29, 31 or 64), else 0 */
    uint32_t sum_groups;       /* with fd: transform-domain sums per output sub-block     */
    uint32_t seg_in;           /* segmented fd: key sub-blocks per segment, else 0        */
    uint32_t seg_out;          /* segmented fd: output sub-blocks per slice, else 0       */
    uint64_t segments;         /* segmented fd: launches run in order (slices x segments) */
    uint32_t outer_log2;       /* fd sums by transforms over the sub-block index: log2 of
                                  their size, else 0                                      */
    uint32_t outer_slice;      /* ... output sub-blocks per such convolution              */
} pa_plan_desc;

typedef struct pa_plan_s *pa_plan_t;

/* Plan the hash of an n-bit key into m bits with the default (fastest known) path
 * (Sec. 3 Step 2: the sub-block lengths p and q are chosen from the sizes and the device
 * memory before any product runs; Eq. Ti / Eq. Tij split the key and the output). The
 * planner picks the path, the key and output sub-block lengths (L, M), the transform size
 * N or the block tile b. Allocates the plan's device workspace on the current device.
 * out: receives the plan handle (NULL on failure). PA_ERR_INVALID for n = 0, m = 0 or a
 * null out; PA_ERR_NOMEM if the workspace cannot be allocated. */
int pa_plan(uint64_t n, uint64_t m, pa_plan_t *out);

/* Same with options (Sec. 3 Step 2 with the caller fixing some of the choices; opts may
 * be NULL). PA_ERR_UNSUPPORTED if a forced path cannot handle (n, m), including an NTT
 * plan without transform-domain sums whose work list would exceed 2^28 items or 2^22 tile
 * pairs (refused before anything is allocated); PA_ERR_PRECISION if a forced FFT tile has
 * no proven bound. */
int pa_plan_ex(uint64_t n, uint64_t m, const pa_opts *opts, pa_plan_t *out);

/* Resolve a plan on the host only: no GPU and no device memory are touched. An NTT plan
 * is laid out as pa_plan_ex would (its work list is built in host memory and freed before
 * the call returns; a key of 1e10 bits takes a few seconds). Same status codes as
 * pa_plan_ex; out is written only on PA_OK. */
int pa_plan_query(uint64_t n, uint64_t m, const pa_opts *opts, pa_plan_desc *out);

/* Describe a created plan. PA_ERR_INVALID for a null plan or out. */
int pa_plan_describe(pa_plan_t plan, pa_plan_desc *out);

/* Release the plan and its workspace (synchronises the plan's last stream). */
void pa_plan_destroy(pa_plan_t plan);

/* y = T x mod 2 (Sec. 2.3 Step 1/2 with the decomposition of Sec. 3).
 * seed_bits, key_bits, out_bits: device pointers, 16-byte aligned.
 * stream: a cudaStream_t (NULL = legacy default stream). Asynchronous: kernel-side
 * errors (a bounded wait that gave up) are read afterwards with pa_plan_status.
 * PA_ERR_INVALID for a null plan or buffer; PA_ERR_ALIGN for a buffer not 16-byte
 * aligned; PA_ERR_CUDA if a launch fails; PA_ERR_NOMEM if the first call on a device
 * cannot build its twiddle tables. */
int pa_hash(pa_plan_t plan, const uint64_t *seed_bits, const uint64_t *key_bits,
            uint64_t *out_bits, void *stream);

/* The same hash from and to HOST buffers: copies the key and seed to the plan's
 * device staging (allocated on the first call), hashes, copies the result back and
 * synchronises the stream. Host buffers need no alignment. Errors as pa_hash, plus
 * PA_ERR_NOMEM if the staging cannot be allocated. */
int pa_hash_host(pa_plan_t plan, const uint64_t *seed_host, const uint64_t *key_host,
                 uint64_t *out_host, void *stream);

/* Worst |v - rint(v)| seen in the plan's last call, with the proven bound (synchronises the
 * plan's stream): the FFT path's rounded convolution values, and the block FP8 path's
 * tensor-core sums scaled to counts (proven exact, bound 0, measured every run). The
 * integer paths report 0. The residual is cleared for the next call. bound may be NULL.
 * PA_ERR_INVALID for a null plan or residual; PA_ERR_CUDA if the read fails. */
int pa_last_residual(pa_plan_t plan, double *residual, double *bound);

/* The proven bound on |v - rint(v)| used by the FFT path for a tile of transform
 * size 2^log2_transform, key sub-block tile_in and output sub-block tile_out, for
 * FP32 (fp64 = 0) or FP64 butterflies. A tile is used only if its bound is < 1/2.
 * Host only. PA_ERR_INVALID for a null bound or log2_transform outside 1..40. */
int pa_fft_rounding_bound(uint32_t log2_transform, uint64_t tile_in, uint64_t tile_out, int fp64,
                          double *bound);

/* Device-side status of the plan's last call: PA_OK, or PA_ERR_TIMEOUT if a
 * bounded wait in a kernel gave up (synchronises the plan's stream). PA_ERR_INVALID for a
 * null plan; PA_ERR_CUDA if the read fails. */
int pa_plan_status(pa_plan_t plan);

/* y = T x mod 2 on the direct path WITHOUT allocating anything. The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc (a pipeline that reserved
 * its device memory once and forbids allocation later, a process whose device memory
 * belongs to another framework's allocator, code that must not meet out-of-memory
 * mid-key). The kernel's scratch (reversed key, status word) is a static device array of
 * about 4 MiB that every GPU loading this library holds until the process exits.
 *   n <= 2^25 (33,554,432) key bits, else PA_ERR_TOO_LARGE; m as for pa_hash.
 *   seed_bits, key_bits, out_bits: device pointers, 16-byte aligned, same layout as
 *   pa_hash; stream: cudaStream_t (NULL = legacy default stream); asynchronous.
 * Outside stream capture every call looks the array's device address up
 * (cudaGetSymbolAddress) with the current device, so the address is never stale after a
 * device reset. Under stream capture the address cached by an earlier uncaptured call on
 * that device is used; a call under capture with none cached returns PA_ERR_INVALID, so
 * make the first call on each device before any capture. Every call shares the one array
 * and leaves its contents behind (the status word is cleared at each call, the reversed
 * key is rewritten in full): calls that overlap on the GPU race, so serialise them (one
 * stream, or events). Calls no cudaMalloc, cudaFree or allocating library routine. A
 * bounded device wait that gives up leaves the output incomplete and records
 * PA_ERR_TIMEOUT in the array's status word: read it with pa_direct_static_status. */
int pa_hash_direct_static(uint64_t n, uint64_t m, const uint64_t *seed_bits,
                          const uint64_t *key_bits, uint64_t *out_bits, void *stream);

/* Device status of the last pa_hash_direct_static call on the current device: synchronises
 * `stream` (the stream that call used; NULL = legacy default stream), reads the status
 * word of the static array (PA_OK, or PA_ERR_TIMEOUT if a bounded wait in the kernel gave
 * up), clears it, and returns it; PA_ERR_CUDA if a CUDA call fails, PA_ERR_INVALID under
 * stream capture before any uncaptured call on the device. Allocates nothing. */
int pa_direct_static_status(void *stream);

/* The seed of the square matrix of Eq. 1 (Sec. 2.1): Eq. 1 writes an n x n Toeplitz matrix
 * with the 2n-1 parameters t_0 .. t_{2n-2} (t_0 .. t_{n-1} down the first column, t_n ..
 * t_{2n-2} along the first row after t_0). In this library's form T[i][j] = s[n-1+i-j] that
 * is s[n-1+d] = t_d for d >= 0 and s[n-1-e] = t_{n-1+e} for e >= 1.
 *   n       : matrix size, >= 1 (hash it with m = n).
 *   t_bits  : host, ceil((2n-1)/64) words, bit d = t_d (LSB-first); bits >= 2n-1 ignored.
 *   seed_bits: host, ceil((2n-1)/64) words, fully written, bits >= 2n-1 set to 0.
 * Host only (no GPU, no allocation); PA_ERR_INVALID for n = 0 or a null pointer. */
int pa_seed_from_eq1(uint64_t n, const uint64_t *t_bits, uint64_t *seed_bits);

/* ---- Many independent blocks in one launch (Sec. 3: batches run in parallel) ---- */

typedef struct {
    uint64_t n, m;
    const uint64_t *seed_bits; /* device, 16-byte aligned                               */
    const uint64_t *key_bits;  /* device, 16-byte aligned                               */
    uint64_t *out_bits;        /* device, 16-byte aligned                               */
} pa_block;

typedef struct {
    double max_residual;       /* worst |v - rint(v)| over FP tiles (0 if none ran)       */
    double bound;              /* largest proven bound among the FP tiles                 */
    uint32_t blocks_per_path[8]; /* indexed by pa_path                                    */
    uint64_t work_items;       /* tiles in the persistent launch's work list              */
    uint32_t graph_replayed;   /* 1 if a captured CUDA graph was replayed                 */
    uint32_t reserved[5];
} pa_report;

typedef struct pa_batch_s *pa_batch_t;

/* Plan a batch for these (n_i, m_i) shapes: path and tiles per block chosen by the
 * autotuner, one persistent work list, workspace allocated once. Only the
 * shapes are read from blocks[]; pointers may be NULL at planning time. opts may be NULL
 * (autotuned); a forced path applies to every block. PA_ERR_INVALID for a null blocks
 * or out, count 0 or above 2^24, or a block with n or m of 0 or above 2^40 bits (all
 * checked before the autotuner's calibration); a block's planning status
 * (PA_ERR_UNSUPPORTED, PA_ERR_PRECISION) if a forced path cannot take it; PA_ERR_NOMEM or
 * PA_ERR_CUDA if the workspace cannot be set up. */
int pa_batch_plan(const pa_block *blocks, size_t count, const pa_opts *opts, pa_batch_t *out);

/* Run a planned batch with these buffers (same shapes, in the same order). The
 * launch sequence is captured once in a CUDA graph and replayed when the buffer
 * pointers and stream are unchanged. rep may be NULL; when it is not, the call
 * synchronises the stream to fill it and returns the device status (PA_ERR_TIMEOUT if a
 * bounded wait gave up). PA_ERR_INVALID for a null batch or blocks, a count or a shape
 * that differs from the plan's, or a null buffer; PA_ERR_ALIGN for a buffer not 16-byte
 * aligned; PA_ERR_CUDA if a launch fails. */
int pa_batch_run(pa_batch_t batch, const pa_block *blocks, size_t count, void *stream,
                 pa_report *rep);

/* Same as pa_batch_run with HOST bit buffers: copies every key and seed to device
 * staging owned by the batch (allocated on the first call), runs, copies the outputs
 * back, synchronises. Host buffers need no alignment. PA_ERR_INVALID for a mismatched
 * block list or a null buffer; PA_ERR_NOMEM if the staging cannot be allocated; otherwise
 * as pa_batch_run. */
int pa_batch_run_host(pa_batch_t batch, const pa_block *host_blocks, size_t count, void *stream,
                      pa_report *rep);

/* Same as pa_batch_run_host without synchronising: enqueues on `stream` the copies of every
 * key and seed into the batch's device staging, the batch's kernels and the copies of the
 * outputs back to host_blocks[i].out_bits, all copies by cudaMemcpyAsync (the copy engines,
 * no SM time). With page-locked host buffers the call returns once everything is enqueued
 * and the copies can overlap kernels running on other streams: two batches planned for the
 * same blocks, run alternately on two streams, move one step's keys in and outputs out
 * while the other step computes (the paper's blocks streamed through the GPU with copies
 * hidden, Sec. 3). Pageable buffers work but the runtime stages them synchronously.
 * The host buffers must stay valid, and the outputs are not ready, until the stream has
 * passed this call's work. One call per batch in flight: the staging is the batch's, so
 * a second call on the same batch must be ordered after the first (same stream, or an event).
 * PA_ERR_INVALID for a mismatched block list; kernel-side errors are read afterwards with
 * pa_batch_get_report. */
int pa_batch_run_host_async(pa_batch_t batch, const pa_block *host_blocks, size_t count, void *stream);

/* The report of the batch's last run, read after the work enqueued on `stream`: copies the
 * batch's device header on that stream and synchronises it. rep as in pa_batch_run; returns
 * the device status (PA_OK, or e.g. PA_ERR_TIMEOUT from a bounded wait that gave up). */
int pa_batch_get_report(pa_batch_t batch, void *stream, pa_report *rep);

/* What the batch plan chose for each block (path, tiles, transform size); count must be
 * the batch's block count. workspace_bytes of a block in its prime field's shared
 * persistent launch counts only a header: that launch's tables and spectra belong to the
 * batch as a whole. */
int pa_batch_describe(pa_batch_t batch, pa_plan_desc *out, size_t count);

void pa_batch_destroy(pa_batch_t batch);

/* One-shot batched hash: plans (cached by shape list), runs, optionally reports. */
int pa_hash_batched(const pa_block *blocks, size_t count, void *stream, pa_report *rep);

/* ---- Serving: continuous batching of requests arriving by device memory ----
 * (Sec. 3: the corrected keys come from reconciliation already in device memory, and
 * blocks are hashed in parallel batches.)
 * A server owns `slots` CUDA streams and a device-memory budget. Submitted requests
 * queue in FIFO order; each poll retires finished waves and, for every free slot, plans
 * the requests waiting at that moment as one batch (one persistent launch for the
 * transform blocks) and launches it on the slot's stream, so waves overlap on the GPU.
 * A wave whose workspace does not fit the budget next to the waves in flight waits.
 * Request buffers are the caller's (device, 16-byte aligned) and must stay valid until
 * the request completes. Batches of a server allocate and free in stream order. */

typedef struct {
    uint32_t slots;               /* concurrent waves (streams), default 2                 */
    uint32_t max_blocks_per_wave; /* default 64                                            */
    uint64_t memory_budget_bytes; /* 0 = unlimited                                         */
    uint32_t reserved[4];
} pa_server_opts;

typedef struct {
    uint64_t tag;                 /* the tag given at submit                               */
    int32_t status;               /* PA_OK or the wave's error                             */
    uint32_t reserved;
} pa_completion;

typedef struct pa_server_s *pa_server_t;

/* Creates the streams and calibrates the autotuner (synchronous, once per device). opts
 * may be NULL (defaults). PA_ERR_INVALID for a null out; PA_ERR_NOMEM; PA_ERR_CUDA if a
 * stream cannot be created; the autotuner's status if its calibration fails. */
int pa_server_create(const pa_server_opts *opts, pa_server_t *out);
/* Queues one request; thread-safe; does not launch (poll does). The request is copied;
 * its buffers are not read until its wave runs. PA_ERR_INVALID for a null server or
 * request, n or m of 0 or above 2^40 bits, or a null buffer; PA_ERR_NOMEM if the queue
 * cannot grow. */
int pa_server_submit(pa_server_t server, const pa_block *request, uint64_t tag);
/* Retires finished waves into done[0..max) (count = entries written; a wave is reported
 * whole or not at all), then admits waiting requests into free slots. Each completion
 * carries its wave's status. A wave that cannot be planned leaves its requests queued,
 * in order, and poll returns the plan's status (the next poll tries again).
 * PA_ERR_INVALID for a null server or count, or done = NULL with max > 0. */
int pa_server_poll(pa_server_t server, pa_completion *done, size_t max, size_t *count);
/* Requests waiting and requests in flight; either pointer may be NULL. PA_ERR_INVALID
 * for a null server. */
int pa_server_pending(pa_server_t server, uint64_t *queued, uint64_t *in_flight);
/* Counters of a server since its creation. */
typedef struct {
    uint64_t waves;               /* waves launched                                         */
    uint64_t requests_done;       /* requests retired by poll                               */
    double plan_s_total;          /* host seconds spent forming, planning and enqueuing the
                                     launched waves (the batch plan is on the latency path)  */
    double plan_s_max;            /* the longest of those, one wave                          */
    uint64_t waves_held_back;     /* wave formations undone by the memory budget             */
    uint64_t reserved[4];
} pa_server_stats;
/* PA_ERR_INVALID for a null server or out. */
int pa_server_get_stats(pa_server_t server, pa_server_stats *out);
/* Waits for the waves in flight, then releases everything. */
void pa_server_destroy(pa_server_t server);

/* ---- Per-kernel timing: CUDA events recorded around every launch on the
 * launching stream while enabled (tracing for roofline measurements). ---- */

typedef struct {
    char name[40];             /* kernel name                                             */
    uint32_t launches;         /* launches timed since profiling was enabled              */
    uint32_t reserved;
    double total_ms;           /* summed event-to-event device time                       */
} pa_kernel_time;

/* enable != 0 clears previous records and starts recording; 0 stops. PA_ERR_INVALID for a
 * null plan. */
int pa_plan_profile(pa_plan_t plan, int enable);

/* Per-kernel totals (synchronises on the recorded events). count = entries written (at
 * most max; out may be NULL with max = 0). PA_ERR_INVALID for a null plan or max < 0;
 * PA_ERR_CUDA if an event cannot be read. The batch forms behave the same. */
int pa_plan_kernel_times(pa_plan_t plan, pa_kernel_time *out, int max, int *count);

int pa_batch_profile(pa_batch_t batch, int enable);
int pa_batch_kernel_times(pa_batch_t batch, pa_kernel_time *out, int max, int *count);

/* ---- Diagnostics ---- */

/* Failure-detection self-test: runs a kernel whose bounded wait can never be satisfied
 * (which = 1: a dependency counter of the persistent launch that nothing signals;
 * which = 2: an mbarrier expecting bytes that never arrive) and stores the kernel's
 * device status in *device_status; PA_ERR_TIMEOUT is the expected value. Every bounded
 * device wait gives up after 4 s (plus 0.5 s for copies in flight), so this takes about
 * four to five seconds; synchronises the device. The GPU context remains usable.
 * PA_ERR_INVALID for another `which` or a null device_status. */
int pa_selftest(int which, int *device_status);

/* Measured issue-rate peaks for the roofline of the integer paths (no counterpart in the
 * paper: a measurement of this GPU). The NTT and direct kernels are bound by integer
 * arithmetic, not by memory, so their roofline is the rate at which this GPU executes the
 * operations they are built from. The probe runs one such operation on independent
 * register chains in every thread of every SM (no memory traffic, no barriers, two CTAs of
 * 512 threads per SM like the NTT kernel) and times it with CUDA events:
 *   which = PA_PEAK_NTT_BUTTERFLY: the lazy Gentleman-Sande butterfly of the 29-bit field
 *           (one operation = one butterfly, Sec. 3 Step 1's transform);
 *   which = PA_PEAK_NTT_MULADD: acc += x y in the 29-bit field (Montgomery product plus lazy
 *           addition: the pointwise products and transform-domain sums of Sec. 3 Step 2);
 *   which = PA_PEAK_SHIFT_AND: acc ^= x & funnel_shift(lo, hi, k), the direct kernel's step
 *           (one operation = one shift-and-accumulate of 32 bit products, Sec. 2.1 Eq. 1);
 *   which = PA_PEAK_MMA_S8: warp-level mma.sync m16n8k32 s8 -> s32, the INT8 block path's
 *           instruction (one operation = one multiply-accumulate);
 *   which = PA_PEAK_MMA_B1: warp-level mma.sync m16n8k256 b1 AND + POPC -> s32, the binary
 *           form of the block contraction (one operation = one 1-bit AND product summed).
 *   which = PA_PEAK_NTT_GROUP28, PA_PEAK_NTT_GROUP29: radix-16 butterfly groups of the
 *           28-bit (5*2^25+1) or 29-bit field as the NTT kernel's rounds run them (lazy
 *           reduction schedule, twiddles read from shared memory), forward and inverse
 *           groups alike (one operation = one butterfly).
 * *ops_per_s: the fastest of three launches of about 20 ms (after a warm-up);
 * *ms (nullable): that launch's device time. Synchronous; allocates at most 4 KB of device
 * memory for the duration of the call. PA_ERR_INVALID for another `which` or a null
 * ops_per_s. */
#define PA_PEAK_NTT_BUTTERFLY 1
#define PA_PEAK_NTT_MULADD 2
#define PA_PEAK_SHIFT_AND 3
#define PA_PEAK_MMA_S8 4
#define PA_PEAK_MMA_B1 5
#define PA_PEAK_NTT_GROUP28 6
#define PA_PEAK_NTT_GROUP29 7
int pa_probe_peak(int which, double *ops_per_s, double *ms);

const char *pa_strerror(int status);

/* The last CUDA error code seen by this thread (0 if none). */
int pa_last_cuda_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int pa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PA_H */
