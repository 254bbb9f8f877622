/*
 * optigpu.h -- C ABI of the GB300 (sm_103a) transpose and sum-reduction
 * library.
 *
 * The two operations are the case studies of the thesis "Source-to-Source
 * Transformations for GPU Code Generation" (arxiv 2605.13864):
 *
 *   transpose   Listing 3.5, Sec. 3.1:  out[x][y] = in[y][x]  for x < W, y < H.
 *               Here H = rows, W = cols, `src` is rows x cols and `dst` is
 *               cols x rows, both dense row-major, so
 *               dst[c * rows + r] = src[r * cols + c].  The thesis's problem
 *               is out-of-place (Listings 3.5, 3.11), so src and dst must not
 *               overlap.  Elements are copied bit for bit.
 *
 *   reduce_sum  Listing 2.1, Sec. 2.1:  the result is reduce_sum(N, A), the
 *               sum of A(0) .. A(N-1).  Listing 2.2 (Sec. 2.2.1) splits it
 *               into per-chunk partial sums followed by a sum of the partials;
 *               this library computes the partials on the GPU and finishes
 *               them on the GPU too (the thesis's benchmark finishes them on
 *               the host, Sec. 7.1).
 *
 * Conventions for every entry point:
 *   - Pointers named src/dst/out are DEVICE pointers owned by the caller
 *     (allocate them with cudaMalloc, torch, ...); the library never frees
 *     them.  The library owns its internal workspaces.
 *   - `stream` is a cudaStream_t passed as an opaque pointer (NULL = the
 *     legacy default stream).  Calls are asynchronous: they validate the
 *     arguments, enqueue kernels on `stream` and return without waiting.
 *   - A call that returns anything but OPTIGPU_OK has enqueued nothing
 *     (argument errors are found before any launch).  Errors raised while
 *     the kernels run are reported by optigpu_stream_status().
 *   - Calls are thread-safe.  Calls on one stream are ordered by the stream;
 *     calls on different streams use different workspaces.
 */
#ifndef OPTIGPU_H
#define OPTIGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OPTIGPU_VERSION 100 /* 1.0.0 */

/* A cudaStream_t. */
typedef void *optigpu_stream_t;

/* Element types.  The transpose copies 4-byte (INT32, FLOAT32) or 2-byte
 * (BFLOAT16, FLOAT16) elements bit for bit; the sum interprets them. */
typedef enum {
    OPTIGPU_INT32 = 0,
    OPTIGPU_FLOAT32 = 1,
    OPTIGPU_BFLOAT16 = 2,
    OPTIGPU_FLOAT16 = 3
} optigpu_dtype;

typedef enum {
    OPTIGPU_OK = 0,
    OPTIGPU_ERR_INVALID_ARG = 1,      /* null pointer with nonzero size, negative or too large size, bad flag */
    OPTIGPU_ERR_UNSUPPORTED_DTYPE = 2,/* dtype outside optigpu_dtype */
    OPTIGPU_ERR_OVERLAP = 3,          /* transpose src and dst byte ranges overlap */
    OPTIGPU_ERR_CUDA = 4,             /* a CUDA runtime call failed; see optigpu_last_error() */
    OPTIGPU_ERR_OOM = 5,              /* a workspace or budget allocation failed */
    OPTIGPU_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up */
    OPTIGPU_ERR_BUSY = 7,             /* serving: no slot or memory budget left right now */
    OPTIGPU_ERR_NOT_FOUND = 8         /* unknown ticket or handle */
} optigpu_status;

/* Operations, for batch descriptors and the autotuner. */
typedef enum {
    OPTIGPU_OP_TRANSPOSE = 0,
    OPTIGPU_OP_REDUCE = 1,
    OPTIGPU_OP_BATCH = 2, /* autotuner only: the batch kernel's configurations */
    OPTIGPU_OP_SCAN = 3   /* tuner: form of the inclusive scan (0 .. 3; see optigpu_scan_inclusive) */
} optigpu_op;

/* ------------------------------------------------------------------------ */
/* Transpose (Listing 3.5, Sec. 3.1)                                        */
/* ------------------------------------------------------------------------ */

/* Transpose kernels.  AUTO picks the fastest eligible one for the shape. */
typedef enum {
    OPTIGPU_TRANSPOSE_AUTO = 0,
    /* 32x32 shared-memory tile padded by one 4-byte bank per row, one
     * barrier, 8 rows of threads moving 4 elements each: the classic
     * bank-conflict-free form of the thesis's Listing 3.6 kernel (Sec. 7.1
     * compares against this form).  Any shape, any alignment. */
    OPTIGPU_TRANSPOSE_TILE32 = 1,
    /* Persistent kernel: TMA 2-D tile loads into a multi-stage shared-memory
     * ring (mbarrier completion), 16-byte micro-block transposes in
     * registers, TMA 2-D tile stores.  Needs 16-byte aligned src/dst and
     * rows, cols multiples of 16 / element size.  Launched with
     * programmatic stream serialisation: it may be launched while the
     * previous kernel on the stream runs, and waits for it to finish (and
     * its writes to be visible) before any tile moves. */
    OPTIGPU_TRANSPOSE_TMA = 2
} optigpu_transpose_kernel;

/* dst (cols x rows) = transpose of src (rows x cols).
 *   src, dst  device pointers, dense row-major, esize(dtype) bytes/element;
 *             must not overlap.  May be NULL only if rows * cols == 0.
 *   rows, cols >= 0; rows * cols * esize < 2^62.  rows == 0 or cols == 0 is
 *             a no-op that returns OPTIGPU_OK.
 * Returns INVALID_ARG, UNSUPPORTED_DTYPE, OVERLAP or CUDA (launch failure). */
optigpu_status optigpu_transpose(const void *src, void *dst, int64_t rows,
                                 int64_t cols, optigpu_dtype dtype,
                                 optigpu_stream_t stream);

/* Same, with an explicit kernel choice.  Asking for TMA on an ineligible
 * shape or alignment returns INVALID_ARG. */
optigpu_status optigpu_transpose_ex(const void *src, void *dst, int64_t rows,
                                    int64_t cols, optigpu_dtype dtype,
                                    optigpu_transpose_kernel kernel,
                                    optigpu_stream_t stream);

/* Pitched transpose: dst[c * ldd + r] = src[r * lds + c] for r < rows,
 * c < cols (row pitches lds >= cols and ldd >= rows, in elements), so either
 * matrix may be a sub-block of a larger row-major array.  Same kernels (TMA
 * when pointers are 16-byte aligned and rows, cols, lds, ldd are multiples of
 * 16 / element size), same errors (OVERLAP on the touched byte spans). */
optigpu_status optigpu_transpose_strided(const void *src, int64_t lds, void *dst, int64_t ldd,
                                         int64_t rows, int64_t cols, optigpu_dtype dtype,
                                         optigpu_stream_t stream);

/* A stack of equal transposes: for b < batch,
 *   dst[b * stride_dst + c * rows + r] = src[b * stride_src + r * cols + c].
 * Each matrix is dense; strides (elements) must be >= rows * cols.  One
 * launch: the TMA kernel with 3-D tensor maps (the batch index is the third
 * coordinate) when pointers, shapes and strides allow, else the padded tile
 * kernel.  Errors as optigpu_transpose (OVERLAP on the touched byte spans). */
optigpu_status optigpu_transpose_batched(const void *src, int64_t stride_src, void *dst,
                                         int64_t stride_dst, int64_t batch, int64_t rows,
                                         int64_t cols, optigpu_dtype dtype,
                                         optigpu_stream_t stream);

/* In-place transpose of the square n x n matrix `a` (dense row-major):
 * a[j][i] <- a[i][j] for all i, j.  Each CTA swaps one pair of 64 x 64 tiles
 * through shared memory.  n in [0, 2^30]; errors as optigpu_transpose. */
optigpu_status optigpu_transpose_inplace(void *a, int64_t n, optigpu_dtype dtype,
                                         optigpu_stream_t stream);

/* 1 if the TMA kernel accepts this shape and these pointers, else 0. */
int optigpu_transpose_tma_eligible(const void *src, const void *dst,
                                   int64_t rows, int64_t cols,
                                   optigpu_dtype dtype);

/* Index (see optigpu_tune_config_name) of the concrete transpose
 * configuration AUTO launches for a rows x cols matrix of dtype, assuming
 * 16-byte aligned pointers: the selected configuration, with the default
 * "by size" entry resolved by the bytes the call moves.  -1 for a bad dtype
 * or a negative size. */
int optigpu_transpose_config_for(int64_t rows, int64_t cols, optigpu_dtype dtype);

/* ------------------------------------------------------------------------ */
/* Sum reduction (Listing 2.1, Sec. 2.1; partial-sum form Listing 2.2)      */
/* ------------------------------------------------------------------------ */

/* Accumulation modes for FLOAT32 / BFLOAT16 / FLOAT16 input (INT32 input is
 * always exact in int64).  The chunk partition and the combine order depend
 * only on (n, dtype, flags), so repeated calls give bit-identical results. */
#define OPTIGPU_REDUCE_PLAIN 0u       /* FP32 per-thread sums and FP32 trees */
#define OPTIGPU_REDUCE_COMPENSATED 1u /* FP32 Neumaier per-thread sums, TwoSum trees */

/* Elements per chunk: one partial sum per OPTIGPU_REDUCE_CHUNK elements
 * (the role of the 128-element tiles of Listing 2.2). */
#define OPTIGPU_REDUCE_CHUNK 16384

/* *out = sum of src[0 .. n).
 *   src   device pointer to n elements of dtype (any alignment; 16-byte
 *         aligned input takes the vector path).  May be NULL if n == 0.
 *   out   device pointer to ONE 8-byte value: int64_t for INT32 input,
 *         double for float input.  Float partials are combined in FP64 on
 *         the GPU (no float atomics); the FP32 value is (float)*out.
 *   n     >= 0 and < 2^62.  n == 0 writes 0.
 * Uses a per-stream library workspace of 8 * ceil(n / CHUNK) + 256 bytes,
 * allocated with cudaMalloc on first use, so the first call on a stream must
 * not happen during stream capture.  A later, larger sum on the stream gets a
 * new, larger workspace; the old one is retired but stays allocated until
 * optigpu_release_workspaces(), so a CUDA graph captured with it stays valid.
 * The kernel is launched with programmatic stream serialisation: it may be
 * launched while the previous kernel on the stream is still running, and
 * every CTA waits for that kernel to finish (and its writes to be visible)
 * before touching memory, so stream order is kept; back-to-back sums overlap
 * a launch with the previous sum's tail.
 * Returns INVALID_ARG, UNSUPPORTED_DTYPE, OOM or CUDA. */
optigpu_status optigpu_reduce_sum(const void *src, int64_t n,
                                  optigpu_dtype dtype, void *out,
                                  optigpu_stream_t stream);

/* Same, with accumulation flags (OPTIGPU_REDUCE_*).  Unknown flag bits
 * return INVALID_ARG. */
optigpu_status optigpu_reduce_sum_ex(const void *src, int64_t n,
                                     optigpu_dtype dtype, void *out,
                                     uint32_t flags, optigpu_stream_t stream);

/* Segmented sums: out[s] = sum of src[offsets[s] .. offsets[s+1]) for
 * s < nseg, each bit-identical to optigpu_reduce_sum_ex on that segment.
 *   offsets  HOST array of nseg + 1 non-decreasing element offsets (< 2^40).
 *   out      device array of nseg 8-byte results (int64 / double); empty
 *            segments give 0.
 * The offsets are staged in pinned host memory; one small kernel reads them
 * there (or from one asynchronous upload, where the device cannot address
 * pinned memory) and builds the batch tables, then all segments run in one
 * launch of the batch kernel (one work item per 16384-element chunk of every
 * segment).  The call returns without waiting for the device, except to
 * reuse a staging buffer of two calls before.  Uses a per-stream library
 * workspace (allocated on first use).  Errors as optigpu_reduce_sum_ex. */
optigpu_status optigpu_reduce_segmented(const void *src, const int64_t *offsets, int32_t nseg,
                                        optigpu_dtype dtype, void *out, uint32_t flags,
                                        optigpu_stream_t stream);

/* Inclusive prefix sums: dst[i] = src[0] + ... + src[i] (the thesis names
 * parallel prefix sum as future work, Sec. 9).
 *   int32 input    -> dst holds int64 values (exact).
 *   float input    -> dst holds float32 values (fp32, bf16 and fp16 input):
 *                     FP32 inside each 4096-element chunk (8192 for 16-bit
 *                     input in forms 0 and 2), carries between chunks in
 *                     FP64 (forms 0-2) or FP32 hi + lo pairs (form 3);
 *                     within 1e-6 of the sum of |x| over the prefix.
 * Every form fixes the expression of each output by its index alone, so the
 * result is bit-identical from run to run (device waits bounded; a wait that
 * gives up is reported by optigpu_stream_status).  Tuner configurations
 * (OPTIGPU_OP_SCAN), kept per input class (int32; the float types together):
 *   0  one pass over chunks claimed in order; block (k, m) is the sum of the
 *      totals of chunks [m 32^k, (m+1) 32^k), formed by a fixed butterfly
 *      over its 32 children, and the carry of chunk c adds, level by level
 *      from the top, the complete blocks before c inside its parent group
 *      (the base-32 digits of c); each carry is used one chunk after it is
 *      fetched.  The default for int32 input.
 *   1  three launches (chunk sums, carries, chunk scans).
 *   2  form 0 reading each carry at once (the same bits as 0).
 *   3  one pass over slices of 2 (fp32), 3 (16-bit) or 1 (int32) chunks,
 *      slice s taken by CTA s mod G of a cooperative launch of one CTA per
 *      SM; the carry of slice s is a fixed butterfly over 32 running sums,
 *      sum l adding the totals of the slices j < s with j = l (mod 32) left
 *      to right.  The default for float input.
 * src and dst must not overlap; n in [0, 2^40].  Uses a per-stream library
 * workspace of about 4 bytes per 1024 elements.  Errors as
 * optigpu_reduce_sum_ex, plus OVERLAP. */
optigpu_status optigpu_scan_inclusive(const void *src, void *dst, int64_t n,
                                      optigpu_dtype dtype, optigpu_stream_t stream);

/* Histogram of int32 values (the thesis names histograms as future work,
 * Sec. 9): counts[b] = number of i with lo + b*width <= src[i] <
 * lo + (b+1)*width, for b < nbins; values outside are not counted.
 *   counts  device array of nbins int64, overwritten (zeroed, then counted).
 *   width >= 1, 1 <= nbins <= 2^26, |lo| and width <= 2^40.
 * Per-CTA shared-memory counters (nbins <= 12288) merged with integer
 * atomics; exact, so bit-exact against any correct count. */
optigpu_status optigpu_histogram_i32(const int32_t *src, int64_t n, int64_t lo, int64_t width,
                                     int32_t nbins, int64_t *counts, optigpu_stream_t stream);

/* Allocates (or grows) the workspace `stream` needs for sums of up to n
 * elements, so that later sums on that stream -- for example inside a CUDA
 * graph capture -- allocate nothing.  Growing never frees a workspace that a
 * captured graph may still use (see optigpu_release_workspaces).
 * INVALID_ARG for n < 0, OOM on allocation failure. */
optigpu_status optigpu_reduce_reserve(int64_t n, optigpu_stream_t stream);

/* Allocation-free sum.  The thesis has no counterpart to this entry point:
 * it exists for callers that must not have the library allocate device
 * memory -- applications that own all device memory through their own pool,
 * loops that must not reach the driver's allocator after start-up, or
 * processes held to a hard memory budget.
 *   Same arguments, result and bit-identical summation order as
 *   optigpu_reduce_sum_ex, but the per-chunk partials and the completion
 *   counter live in one fixed device array of 256 KiB + 256 bytes that every
 *   GPU loading the library holds until the process exits.  The call itself
 *   allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 *   routine); it clears the counter with cudaMemsetAsync and launches.
 *   n is limited to 32768 * OPTIGPU_REDUCE_CHUNK = 2^29 elements; larger n
 *   returns INVALID_ARG with that limit in optigpu_last_error().
 *   The first call on a device looks up the array's device address (set-up,
 *   once per device, with that device current); make that first call before
 *   any stream capture.  cudaDeviceReset() invalidates that address: after a
 *   reset, call optigpu_release_workspaces() (which forgets it) before the
 *   next call on that device.
 *   All calls share the one array: calls whose kernels overlap on the GPU
 *   (for example on two streams at once) race and give wrong sums.  Order
 *   them, e.g. by issuing them on one stream. */
optigpu_status optigpu_reduce_sum_noalloc(const void *src, int64_t n,
                                          optigpu_dtype dtype, void *out,
                                          uint32_t flags,
                                          optigpu_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Host buffers: the same operations with the copies pipelined              */
/* ------------------------------------------------------------------------ */
/* The thesis's host code copies the whole input in, launches and copies the
 * result back (Listings 3.6, 3.11).  These entry points take HOST pointers
 * and cut the work into row bands (transpose) or chunk bands (sum) that
 * alternate between two internal streams, so copies in, kernels and copies
 * out overlap.  Results are identical to the device-buffer calls (the sum is
 * bit-identical to optigpu_reduce_sum_ex).  Pinned host memory
 * (cudaHostAlloc / cudaHostRegister) makes the copies asynchronous; pageable
 * memory works but copies synchronously.  The calls are asynchronous on
 * `stream`: host buffers must stay valid and untouched until it completes.
 * Device staging buffers (2 x 2 x ~64 MiB) are library-owned, cudaMalloc'd on
 * first use per device and reused; do not call during stream capture. */

/* host_dst (cols x rows) = transpose of host_src (rows x cols), both dense
 * row-major in host memory.  Errors as optigpu_transpose (OVERLAP for
 * overlapping host ranges). */
optigpu_status optigpu_transpose_host(const void *host_src, void *host_dst, int64_t rows,
                                      int64_t cols, optigpu_dtype dtype,
                                      optigpu_stream_t stream);

/* *host_out (8 bytes: int64 or double) = sum of host_src[0 .. n).  Errors as
 * optigpu_reduce_sum_ex. */
optigpu_status optigpu_reduce_sum_host(const void *host_src, int64_t n, optigpu_dtype dtype,
                                       void *host_out, uint32_t flags,
                                       optigpu_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batches: many uneven transposes and sums in one persistent launch        */
/* ------------------------------------------------------------------------ */
/* The thesis launches one kernel per problem (Listings 3.6, 6.21).  A batch
 * plan runs thousands of independent instances of both problems in one
 * persistent kernel fed by a device work queue (an integer atomic counter).
 * Each instance computes exactly what the single calls compute: transposes
 * are bit copies and every sum is bit-identical to optigpu_reduce_sum_ex with
 * the same flags (same chunks, same combine order), whatever the mix. */

/* One instance of a batch. */
typedef struct {
    int32_t op;      /* OPTIGPU_OP_TRANSPOSE or OPTIGPU_OP_REDUCE */
    int32_t dtype;   /* optigpu_dtype */
    const void *src; /* device input: rows x cols (transpose) or rows elements (sum) */
    void *dst;       /* transpose: cols x rows output; sum: the 8-byte result (int64 or double) */
    int64_t rows;    /* transpose rows, or the sum's length n */
    int64_t cols;    /* transpose cols; ignored for sums */
} optigpu_desc;

typedef struct optigpu_batch_plan optigpu_batch_plan;

/* Plan flags (OPTIGPU_REDUCE_COMPENSATED applies to every float sum). */
#define OPTIGPU_BATCH_NO_GRAPH 2u /* launch directly instead of replaying a CUDA graph */

/* Validates the `count` descriptors, flattens them into work items (tiles of
 * the transposes, 16384-element chunks of the sums), uploads the tables to a
 * plan-owned device workspace (cudaMalloc; freed by _destroy) and captures
 * one run -- queue reset and kernel launch -- into a CUDA graph.  Every
 * descriptor is checked like the single calls (INVALID_ARG,
 * UNSUPPORTED_DTYPE, OVERLAP within an instance).  Instances must not write
 * to memory that another instance of the plan reads or writes.  The plan
 * keeps the pointers: the buffers must stay valid while it is used.
 * Synchronous; must not run during stream capture. */
optigpu_status optigpu_batch_plan_create(const optigpu_desc *descs, int32_t count,
                                         uint32_t flags, optigpu_batch_plan **plan);

/* Enqueues one run of the plan on `stream` (one graph launch).  Runs of one
 * plan share its workspace: order them (one stream, or events). */
optigpu_status optigpu_batch_run(optigpu_batch_plan *plan, optigpu_stream_t stream);

/* Work items, algorithmic bytes of one run (2*esize*rows*cols per
 * transpose, esize*n per sum) and persistent grid size of the last run. */
optigpu_status optigpu_batch_plan_info(const optigpu_batch_plan *plan, int64_t *items,
                                       int64_t *bytes, int32_t *grid);

/* Times every batch configuration (transpose tile 32 or 64, CTAs per SM) on
 * this plan's own buffers -- the instances are really computed, so outputs
 * are overwritten with the same values -- selects the fastest for the plan
 * and as the default of later plans, and re-captures the graph.
 * Synchronises `stream`. */
optigpu_status optigpu_batch_autotune(optigpu_batch_plan *plan, int reps,
                                      optigpu_stream_t stream, int *best_config,
                                      float *best_ms);

/* Frees the plan's workspace and graph (wait for its runs first). */
void optigpu_batch_plan_destroy(optigpu_batch_plan *plan);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of transpose and sum requests               */
/* ------------------------------------------------------------------------ */
/* The thesis runs each problem once from host code (Listings 3.6, 3.11:
 * allocate, copy in, launch, copy out, free).  The server keeps that flow per
 * request but shares the device among many requests: it admits queued
 * requests while slots and a device-memory budget allow, keeps their buffers
 * in a device arena, copies their inputs in, runs each step's admitted
 * requests as one persistent batch kernel (the batch plans' kernel), copies
 * results out and frees the buffers when the step's completion event fires.
 * Requests that arrive while earlier steps run go into the next step on
 * another stream, so their copies and kernels overlap on the device.  Each
 * result equals the single call's (transposes bit for bit, sums bit-identical
 * to optigpu_reduce_sum_ex with the server's flags). */

typedef struct optigpu_server optigpu_server;

/* One request: the data lives in HOST memory (pinned memory makes the copies
 * asynchronous).  host_dst receives cols x rows elements for a transpose, or
 * one 8-byte value (int64 / double) for a sum.  Both buffers must stay valid
 * until the request is done. */
typedef struct {
    int32_t op;           /* OPTIGPU_OP_TRANSPOSE or OPTIGPU_OP_REDUCE */
    int32_t dtype;        /* optigpu_dtype */
    int64_t rows;         /* transpose rows, or the sum's length n */
    int64_t cols;         /* transpose cols; ignored for sums */
    const void *host_src; /* rows x cols (or n) elements */
    void *host_dst;
} optigpu_request;

typedef struct {
    int64_t submitted, completed, pending, in_flight, max_in_flight;
    int64_t steps;    /* launched steps (stream submissions) */
    int64_t launches; /* kernel launches, copy kernels included (per batched step: gather, batch
                         kernel, scatter; per request in per-call mode: the plain kernel, plus a
                         gather and a scatter with OPTIGPU_SERVER_COPY_KERNELS) */
    int64_t bytes_in_use, peak_bytes; /* device arena */
    int64_t replay_max_loop_gap_ns;   /* last optigpu_server_replay: longest time between two
                                         rounds of its serving loop (a host-side stall) */
} optigpu_server_stats;

/* Server flags (OPTIGPU_REDUCE_COMPENSATED applies to every float sum). */
#define OPTIGPU_SERVER_PER_CALL 4u /* baseline: one plain kernel per request, one request per stream */
/* Copy path, held fixed to compare the modes.  By default a batched step
 * moves pinned request buffers with two SM copy kernels (a gather and a
 * scatter through the device's mapping of the host memory) and per-call mode
 * uses one copy-engine call (cudaMemcpyAsync) per buffer; pageable buffers
 * always go through the copy engines. */
#define OPTIGPU_SERVER_COPY_ENGINES 8u  /* every buffer by a copy-engine call, batched mode too */
#define OPTIGPU_SERVER_COPY_KERNELS 16u /* per-call mode: pinned buffers by one gather and one
                                           scatter copy kernel per request */

/* Creates a server with a device arena of mem_budget_bytes (one cudaMalloc,
 * >= 1 MiB), at most max_slots requests on the device at once and n_streams
 * streams (1..1024; at most n_streams steps in flight).  INVALID_ARG for bad
 * sizes or flags (COPY_ENGINES with COPY_KERNELS), OOM if the budget cannot
 * be allocated. */
optigpu_status optigpu_server_create(size_t mem_budget_bytes, int32_t max_slots,
                                     int32_t n_streams, uint32_t flags,
                                     optigpu_server **server);

/* Queues a request (validated now: INVALID_ARG / UNSUPPORTED_DTYPE, or
 * INVALID_ARG if it alone exceeds the budget); returns its ticket.  BUSY
 * when the queue holds 2^24 requests. */
optigpu_status optigpu_server_submit(optigpu_server *server, const optigpu_request *req,
                                     uint64_t *ticket);

/* One round of the loop: completes finished steps, admits queued requests in
 * arrival order into every free stream while slots and budget allow (one
 * step takes at most max_slots / n_streams requests, so steps overlap), and
 * launches them.  *launched (may be NULL) = number of steps launched.
 * If a step's launch fails, the call waits for that step's stream, returns
 * the step's requests to the head of the queue (their arena space and slots
 * are freed) and returns the error (CUDA or OOM); a later step retries them. */
optigpu_status optigpu_server_step(optigpu_server *server, int32_t *launched);

/* *done = 1 once the ticket's result is in its host buffer (the ticket is
 * then forgotten); NOT_FOUND for unknown or already-reported tickets. */
optigpu_status optigpu_server_poll(optigpu_server *server, uint64_t ticket, int32_t *done);

/* Steps until every queued request has completed. */
optigpu_status optigpu_server_drain(optigpu_server *server);

optigpu_status optigpu_server_get_stats(optigpu_server *server, optigpu_server_stats *stats);

/* Replays an open-loop trace: request i is submitted when arrival_s[i]
 * seconds (non-decreasing) have passed since the call started; the loop
 * steps until all have completed and writes latency_s[i] = completion time
 * (the host sees the step's event fire) - arrival time. */
optigpu_status optigpu_server_replay(optigpu_server *server, const optigpu_request *reqs,
                                     const double *arrival_s, int64_t count, double *latency_s);

/* Testing hook (the thesis has no counterpart): the nth step launch from now
 * on (1 = the next; 0 cancels) fails on the host part-way through (after any
 * copy-engine input copies are enqueued), as a failed CUDA call would, so
 * that the recovery described at optigpu_server_step can be exercised
 * without a device fault.
 * INVALID_ARG for a null server or nth < 0. */
optigpu_status optigpu_server_inject_step_failure(optigpu_server *server, int32_t nth);

/* Waits for the server's streams and frees everything it owns. */
void optigpu_server_destroy(optigpu_server *server);

/* ------------------------------------------------------------------------ */
/* Autotuning                                                               */
/* ------------------------------------------------------------------------ */
/* The thesis fixes its launch parameters by hand (the tile size 32 and the
 * 128-element chunk in its transformation scripts, Sec. 2.2.1 and 3.2); this
 * library compiles several configurations of each kernel (tile shape,
 * pipeline depth, output buffers; CTAs per SM for the sum) and picks among
 * them by measurement.  Selections are process-wide.  None of them changes a
 * result: transposes are bit copies and the sum's chunk partition is fixed. */



/* Number of configurations of `op` for `dtype` (-1 for a bad op or dtype).
 * Transpose: indices 0 .. n-2 are TMA kernels, n-1 the padded tile32 kernel;
 * index 0, the default, picks between indices 1 and 2 by the bytes a call
 * moves (optigpu_transpose_config_for tells which).
 * OPTIGPU_OP_BATCH ignores `dtype`; its selection is the default of new
 * plans.  OPTIGPU_OP_SCAN: 0 = single pass (radix-32 carries used one
 * chunk later), 1 = three passes, 2 = single pass (carries read at once),
 * 3 = windowed single pass; the choice is kept per input class (INT32; the
 * float types together). */
int optigpu_tune_num_configs(optigpu_op op, optigpu_dtype dtype);

/* Static name of configuration `config`, or NULL if out of range. */
const char *optigpu_tune_config_name(optigpu_op op, optigpu_dtype dtype, int config);

/* Selects the configuration AUTO uses from now on.  For the transpose the
 * choice is per element size (INT32 and FLOAT32 share one, BFLOAT16 and
 * FLOAT16 the other).  INVALID_ARG for an index out of range. */
optigpu_status optigpu_tune_select(optigpu_op op, optigpu_dtype dtype, int config);

/* Currently selected configuration index (-1 for a bad op or dtype). */
int optigpu_tune_selected(optigpu_op op, optigpu_dtype dtype);

/* Named integer parameters: "transpose.group_rows" (tile-rows the TMA
 * transpose walks before moving one tile-column right, 1..4096, default 16).
 * NOT_FOUND for an unknown name. */
optigpu_status optigpu_tune_set_param(const char *name, int64_t value);
int64_t optigpu_tune_get_param(const char *name); /* -1 if unknown */

/* Times every configuration of `op` on a rows x cols problem (the sum and
 * the scan use n = rows * cols) in library-owned scratch memory (cudaMalloc'd and freed
 * inside the call), `reps` timed launches each after two warm-ups, median of
 * CUDA-event times on `stream`; selects the fastest and returns its index
 * and time.  Transpose TMA configurations are skipped when the shape is not
 * TMA-eligible.  Synchronises `stream`.  Must not run during stream capture. */
optigpu_status optigpu_autotune(optigpu_op op, optigpu_dtype dtype, int64_t rows, int64_t cols,
                                int reps, optigpu_stream_t stream, int *best_config,
                                float *best_ms);

/* Writes / reads the current selections as a small text file.  A cache
 * named by the OPTIGPU_TUNE_CACHE environment variable is read when the
 * library is loaded. */
optigpu_status optigpu_tune_save(const char *path);
optigpu_status optigpu_tune_load(const char *path);

/* ------------------------------------------------------------------------ */
/* Status and housekeeping                                                  */
/* ------------------------------------------------------------------------ */

/* Waits for `stream`, then reports the first asynchronous CUDA error
 * (OPTIGPU_ERR_CUDA) or a device-side wait that gave up since the last call
 * (OPTIGPU_ERR_TIMEOUT; the device flag is per device and is cleared by this
 * call).  OPTIGPU_OK otherwise. */
optigpu_status optigpu_stream_status(optigpu_stream_t stream);

/* Failure-detection self-test (the thesis has no counterpart): enqueues a
 * kernel that waits, with the library's bounded device wait, on a barrier
 * phase nothing completes.  After limit_ns (in (0, 10 s]) it gives up and
 * records a timeout, so the next optigpu_stream_status on that stream returns
 * OPTIGPU_ERR_TIMEOUT and the CUDA context stays usable.  No fault, no hang. */
optigpu_status optigpu_selftest_wait_timeout(uint64_t limit_ns, optigpu_stream_t stream);

/* Static description of a status code; never NULL. */
const char *optigpu_status_string(optigpu_status status);

/* Text of the last error raised on the calling thread ("" if none). */
const char *optigpu_last_error(void);

/* Device-side wait limit in nanoseconds for kernels that spin on a barrier
 * (default 2e9, or the OPTIGPU_WAIT_LIMIT_NS environment variable). */
void optigpu_set_wait_limit_ns(uint64_t ns);

/* Frees every workspace the library holds for the current device, including
 * those retired when a stream needed a larger one.  Call it with no work in
 * flight on the library's streams, and only once no CUDA graph captured from
 * the library's calls will be replayed again (such graphs keep the
 * workspace addresses they were captured with). */
optigpu_status optigpu_release_workspaces(void);

/* OPTIGPU_VERSION of the loaded library. */
int optigpu_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OPTIGPU_H */
