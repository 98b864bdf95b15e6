/*
 * sketch.h -- C ABI of the GB300 random-sketch library.
 *
 * The library computes sketches of a dense FP32 matrix A by a dense random
 * matrix whose entries are regenerated on the GPU from a counter-based
 * generator instead of being stored or read from memory:
 *
 *   left  sketch  Y[k x n] = S[k x m] * A[m x n]
 *   right sketch  Y[m x k] = A[m x n] * Omega,   Omega = S^T, S[k x n]
 *
 * with S(r, c) = s * q(g(r, c)), s = fl32(1/sqrt(k)), g(r, c) a Gaussian
 * N(0,1), Rademacher +-1 or uniform [0,1) draw that is a pure function of
 * (seed, r, c), and q the storage precision of the generated operand.
 *
 * Paper: arXiv 2603.20966 (Al Daas et al., "Communication Lower Bounds and
 * Algorithms for Sketching with Random Dense Matrices").  The product is the
 * sketch B = A Omega of Sec. 1 and Sec. 3; the left form is the transposed
 * computation the paper notes after Theorem 2 (Omega^T A^T).  Generating the
 * random operand where it is consumed, with a shared seed, is the paper's
 * "generate Omega redundantly instead of communicating it" (Sec. 6.2 and
 * Alg. 1 GenRandom); on one GPU it becomes "generate S tiles in shared
 * memory instead of reading S from HBM".
 *
 * Conventions for every call:
 *  - Matrices are row-major with a leading dimension (elements between
 *    consecutive rows).  Pointers named A, Y, out are DEVICE pointers unless
 *    the function name ends in _host.  The caller owns every buffer it
 *    passes; the library never frees or retains them past the call.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *    work is asynchronous on that stream; a return of SK_OK means the work
 *    was validated and enqueued.
 *  - Host-detectable errors return immediately, enqueue nothing and leave
 *    outputs untouched: SK_EINVAL for a NULL handle/pointer, a size <= 0,
 *    a leading dimension smaller than the row length, or an index beyond
 *    2^32; SK_EUNSUPPORTED for a precision/size combination a form does not
 *    implement; SK_ECUDA when a CUDA call fails (cudaGetLastError is
 *    cleared).  Errors raised on the device (a bounded wait that gave up,
 *    a bounds check) are recorded in a per-handle status word that
 *    sk_stream_status() reads.
 *  - Determinism: identical (seed, dist, k, precision, A) give bit-identical
 *    Y on the same GPU model, independent of stream, batch or serving mix.
 *  - A handle may be used from one host thread at a time.
 */
#ifndef SKETCH_H_
#define SKETCH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SK_OK = 0,
  SK_EINVAL = 1,        /* bad argument */
  SK_ENOMEM = 2,        /* device or host allocation failed */
  SK_ECUDA = 3,         /* a CUDA runtime/driver call failed */
  SK_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
  SK_EBUDGET = 5,       /* request exceeds the serving memory budget */
  SK_EUNSUPPORTED = 6,  /* combination not implemented by the selected form */
  SK_EBUSY = 7,         /* result not ready yet (serving poll) */
  SK_ECANCELLED = 8     /* request cancelled before completion */
} sk_status;

/* Distribution of g(r, c).  Gaussian is the paper's theoretical choice
 * (Sec. 1, "Gaussian random matrices"); uniform is what its experiments
 * draw with Philox (Sec. 6.2); Rademacher +-1 is exact in every precision. */
typedef enum { SK_GAUSSIAN = 0, SK_RADEMACHER = 1, SK_UNIFORM = 2 } sk_dist;

/* Arithmetic form of the product.
 *  SK_FP32     FP32 generated operand, FP32 FMA on the CUDA cores.
 *  SK_BF16X2   generated operand rounded to BF16, A split into BF16 hi + lo
 *              parts (hi = bf16(a), lo = bf16(a - hi)), two tensor-core MMAs
 *              per tile with FP32 accumulation in tensor memory.
 *  SK_FP8E4M3  right sketch only: generated operand rounded to E4M3, A
 *              quantised to E4M3 with one power-of-two scale per row
 *              (sk_quantize_e4m3), one kind::f8f6f4 tensor-core MMA per
 *              tile with FP32 accumulation; the row scale is applied in the
 *              epilogue.  Low precision is not in the paper; the error
 *              against the exact product is a few percent (3-bit
 *              significands), reported rather than held to 1e-5.
 * The 1/sqrt(k) scale is one FP32 multiply in every form's epilogue. */
typedef enum { SK_FP32 = 0, SK_BF16X2 = 1, SK_FP8E4M3 = 2 } sk_precision;

typedef struct sk_sketch* sk_handle;

/* Create a sketch operator.  seed: the Philox key (low 32 bits -> key word
 * 0, high 32 bits -> key word 1).  dist: an sk_dist.  k: sketch size
 * (rows of S), 1 <= k <= 2^31.  *out receives the handle.  Allocates a few
 * bytes of device memory for the status word on the current device; all
 * later calls on the handle must run with that device current.
 * Errors: SK_EINVAL (bad dist/k/out), SK_ENOMEM, SK_ECUDA. */
sk_status sk_create(uint64_t seed, int dist, int64_t k, sk_handle* out);

/* Select the arithmetic form (an sk_precision) for later apply calls.
 * Default SK_FP32.  Errors: SK_EINVAL. */
sk_status sk_set_precision(sk_handle h, int precision);

/* Read back the handle's parameters (any pointer may be NULL). */
sk_status sk_get_info(sk_handle h, uint64_t* seed, int* dist, int64_t* k, int* precision,
                      float* scale);

/* Left sketch Y[k x n] = S[k x m] A[m x n] (A: m x n, leading dim lda >= n;
 * Y: k x n, leading dim ldy >= n; both device pointers, FP32).  S(r, c)
 * for r < k, c < m.  Requires m < 2^32.  The tensor-core forms additionally
 * require A and Y 16-byte aligned and lda, ldy multiples of 4 (SK_EINVAL
 * otherwise).  Y is fully overwritten.  A and Y must not overlap.
 * In the SK_FP32 form k is at most 65535 launch tiles of rows of S: 8,388,480
 * when n > 128 (tiles of 128 rows), 16,776,960 when n <= 128 (tiles of 256
 * rows); CUDA rejects the launch of a larger k and the call returns SK_ECUDA
 * (nothing runs). */
sk_status sk_apply_left(sk_handle h, const float* A, int64_t m, int64_t n, int64_t lda, float* Y,
                        int64_t ldy, void* stream);

/* Right sketch Y[m x k] = A[m x n] S^T (S: k x n, S(r, c) for r < k,
 * c < n).  Same conventions as sk_apply_left; requires n < 2^32.  In the
 * SK_FP8E4M3 form the call quantises A into the workspace first
 * (sk_quantize_e4m3) and then runs sk_apply_right_e4m3 (the left sketch
 * returns SK_EUNSUPPORTED in that form). */
sk_status sk_apply_right(sk_handle h, const float* A, int64_t m, int64_t n, int64_t lda,
                         float* Y, int64_t ldy, void* stream);

/* The two products of a Nystrom approximation (the paper's Sec. 5, Alg. 2
 * RandCompNys on one device): B[n x k] = A Omega and C[k x k] = Omega^T B,
 * Omega = S^T the handle's n x k random matrix (k = r), for a symmetric
 * A[n x n] (not checked).  Runs the right sketch of A into B, then the left
 * sketch of B into C, both regenerating the same S; the Nystrom
 * approximation is then B C^+ B^T.  Conventions of sk_apply_left /
 * sk_apply_right (B is the second product's input: the tensor-core form
 * needs it 16-byte aligned with ldb a multiple of 4).  Errors as those
 * calls; SK_EUNSUPPORTED in the SK_FP8E4M3 form. */
sk_status sk_nystrom(sk_handle h, const float* A, int64_t n, int64_t lda, float* B, int64_t ldb,
                     float* C, int64_t ldc, void* stream);

/* The left sketch of sk_apply_left in the SK_BF16X2 form with S read from
 * memory instead of generated: the "communicate Omega" side of the paper's
 * trade between generating the random matrix and moving it (Sec. 6.2,
 * generation versus communication), kept to measure that trade on one GPU.
 * S: device BF16 (raw 16-bit words), row r < k at S + r * lds, columns
 * c < m; sk_materialize(h, 0, 0, k, m, SK_BF16X2, 0, S, lds) writes the
 * handle's own S, for which Y equals sk_apply_left's bit for bit (Y is
 * s S A with s the handle's 1/sqrt(k), whatever S holds).  The
 * kernel reads S in 16-column slabs: columns m .. round_up(m, 16) - 1 of
 * every row are read too and must hold finite values (multiplied by zero).
 * Requires the handle in the SK_BF16X2 form (else SK_EUNSUPPORTED), k and
 * lds multiples of 8, lds >= round_up(m, 16), S 16-byte aligned, and the
 * alignment rules of sk_apply_left's tensor-core forms (else SK_EINVAL).
 * The caller owns S; it is read asynchronously on `stream`. */
sk_status sk_apply_left_stored(sk_handle h, const void* S, int64_t lds, const float* A, int64_t m,
                               int64_t n, int64_t lda, float* Y, int64_t ldy, void* stream);

/* E4M3 form of A for the FP8 right sketch: row_exp[i] = the smallest integer
 * e with max_j |A[i][j]| <= 448 * 2^e (0 for a row of zeros), and
 * Aq[i*ldq + j] = RNE_e4m3(A[i][j] * 2^-e) for j < n (OCP E4M3, largest 448,
 * no code saturates), 0 for n <= j < ldq.  A: device FP32, leading dim
 * lda >= n; Aq: device, 16-byte aligned, ldq >= n a multiple of 16; row_exp:
 * device int32[m].  Asynchronous on `stream`.  Errors: SK_EINVAL, SK_ECUDA. */
sk_status sk_quantize_e4m3(const float* A, int64_t m, int64_t n, int64_t lda, uint8_t* Aq,
                           int64_t ldq, int32_t* row_exp, void* stream);

/* FP8 right sketch of an already quantised A (as sk_quantize_e4m3 writes it,
 * e.g. a resident copy reused by many sketches): Y[m x k] =
 * s 2^row_exp[i] sum_c e4m3(Aq[i][c]) e4m3(g(j, c)), accumulated in FP32 on
 * the tensor cores.  The handle supplies seed, dist and k whatever its form.
 * Y: device FP32, 16-byte aligned, ldy >= k a multiple of 4.
 * Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
sk_status sk_apply_right_e4m3(sk_handle h, const uint8_t* Aq, const int32_t* row_exp, int64_t m,
                              int64_t n, int64_t ldq, float* Y, int64_t ldy, void* stream);

/* Left sketch that allocates no device memory, for callers that cannot let
 * a library call cudaMalloc: an application whose device memory belongs to
 * another allocator (a framework's caching allocator, a serving engine that
 * reserves HBM up front), or a latency-critical path that cannot absorb the
 * implicit synchronisation of cudaMalloc/cudaFree.  The paper has no
 * counterpart; this is a deployment convenience.
 *
 * Computes the same Y[k x n] = S[k x m] A[m x n] as sk_apply_left in the
 * FP32 form (the handle's precision must be SK_FP32, else
 * SK_EUNSUPPORTED), with the same argument meaning and layout.  Its split-K
 * partials live in a 16 MiB array compiled into the library, which every GPU
 * that loads the library holds until the process exits.  Problems whose
 * partials would exceed it -- splits * k * n * 4 bytes > 16 MiB, with
 * sk_workspace_size(h, 0, m, n) reporting that byte count -- are rejected
 * with SK_EUNSUPPORTED before anything is enqueued.  Every call looks up the
 * current device's address of the array (cudaGetSymbolAddress, which
 * allocates nothing), so the address stays right after a cudaDeviceReset;
 * on a device's first call the CUDA runtime may load the library's device
 * code, so make that first call before any stream capture.
 * All calls on a device share the array and each call writes every partial
 * it later reads, so nothing needs clearing between calls, but calls whose
 * work overlaps on the GPU (different streams, no ordering) race on it and
 * give undefined results: order them on one stream or with events.
 * Errors: SK_EINVAL, SK_EUNSUPPORTED, SK_ECUDA (sk_last_cuda_error then
 * describes the failing CUDA call, as for every other entry point). */
sk_status sk_apply_left_noalloc(sk_handle h, const float* A, int64_t m, int64_t n, int64_t lda,
                                float* Y, int64_t ldy, void* stream);

/* The same two products with HOST buffers: A is copied to the device, the
 * sketch computed, and Y copied back before the call returns (the call
 * synchronises `stream`).  Pinned host memory gives full copy bandwidth;
 * pageable memory works.  A (or Y) whose leading dimension equals its row
 * length, a multiple of 4, moves as one linear copy; other layouts as a
 * pitched copy.  Only the n (or output) columns of each row are read (or
 * written).  Device staging memory is owned by the handle and reused across
 * calls.  Errors as above plus SK_ENOMEM. */
sk_status sk_apply_left_host(sk_handle h, const float* A, int64_t m, int64_t n, int64_t lda,
                             float* Y, int64_t ldy, void* stream);
sk_status sk_apply_right_host(sk_handle h, const float* A, int64_t m, int64_t n, int64_t lda,
                              float* Y, int64_t ldy, void* stream);

/* Debugging: write the block S(row0 .. row0+rows-1, col0 .. col0+cols-1)
 * to the device buffer `out` (leading dim ld >= cols).  fmt selects the
 * stored value set and element type: SK_FP32 -> float g (or fl32(s*g)
 * when scaled != 0); SK_BF16X2 -> uint16 bf16(g); SK_FP8E4M3 -> uint8
 * e4m3(g).  scaled != 0 is valid only with SK_FP32.  row0+rows <= 2^32 and
 * col0+cols <= 2^32.  The fused kernels never call this; S never exists in
 * device memory on the apply paths. */
sk_status sk_materialize(sk_handle h, int64_t row0, int64_t col0, int64_t rows, int64_t cols,
                         int fmt, int scaled, void* out, int64_t ld, void* stream);

/* Scratch memory: bytes of device workspace an apply call with these sizes
 * needs in the handle's current form (side 0 = left, 1 = right), or 0.
 * sk_set_workspace lends the handle a caller-owned device buffer of `bytes`
 * (16-byte aligned; NULL/0 returns to handle-owned scratch, which the
 * handle allocates with cudaMalloc on first need and frees in sk_destroy).
 * A lent buffer must stay valid until every call that used it completed. */
sk_status sk_workspace_size(sk_handle h, int side, int64_t m, int64_t n, size_t* bytes);
sk_status sk_set_workspace(sk_handle h, void* ptr, size_t bytes);

/* Synchronise `stream`, then return and clear the handle's device status
 * word: SK_OK, SK_ETIMEOUT (a bounded wait gave up; outputs of the affected
 * call are undefined), or SK_ECUDA if the stream reported an error. */
sk_status sk_stream_status(sk_handle h, void* stream);

/* ---- Batches: many independent left sketches in one persistent launch ----
 *
 * A batch collects left sketches Y_i = S_i A_i (each with its own handle,
 * hence its own seed, distribution and k, and its own m, n) and runs them in
 * one launch of the persistent tensor-core kernel: the (problem, tile,
 * split) work items, ordered longest first on the host, are handed out on
 * the device by an atomic queue to whichever CTA pair is free; then one
 * launch reduces every problem's split partials in fixed order.  The two launches
 * are captured once into a CUDA graph and replayed by later sk_batch_run
 * calls on an unchanged batch (on a created stream; on the legacy default
 * stream, which cannot be captured, the two launches are issued directly).  Each member's result is bit-identical to
 * running it alone with the same work decomposition, and within 1e-5 of
 * the FP64 product in any case.  This is the batching the paper's problem
 * statement (Sec. 1: many sketches of matrices of different shapes) calls
 * for on one GPU; the paper itself runs one sketch at a time. */
typedef struct sk_batch* sk_batch_handle;

/* Create an empty batch.  Allocates a status word on the current device.
 * Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
sk_status sk_batch_create(sk_batch_handle* out);

/* Append the left sketch Y[k x n] = S[k x m] A[m x n] of handle `h` (which
 * must be in the SK_BF16X2 form; seed, dist and k are read now).  A and Y are
 * device pointers with the conventions of sk_apply_left (16-byte aligned,
 * lda and ldy multiples of 4); they must stay valid for every later run.
 * Invalidates the batch's plan and graph.  Errors: SK_EINVAL,
 * SK_EUNSUPPORTED (form other than SK_BF16X2). */
sk_status sk_batch_add(sk_batch_handle b, sk_handle h, const float* A, int64_t m, int64_t n,
                       int64_t lda, float* Y, int64_t ldy);

/* Run every sketch of the batch on `stream` (asynchronous).  The first run
 * after a change plans the work (with the configuration sk_batch_tune or
 * sk_batch_set_config chose, else one from the tuning cache file named by
 * the environment variable SK_TUNE_CACHE, else the default: items of 512
 * stages, 512-column tiles, 4-stage ring), allocates the batch's device
 * buffers and captures the graph; later runs replay it.
 * Errors: SK_EINVAL (empty batch), SK_ENOMEM, SK_ECUDA. */
sk_status sk_batch_run(sk_batch_handle b, void* stream);

/* Autotune the kernel configuration: time the batch (CUDA events on
 * `stream`, synchronising) for every candidate and keep the fastest.  The
 * candidates combine the tile shape (output tiles of at most 512 columns,
 * two MMA instructions per K step, or of at most 256), the pipeline depth
 * (operand ring of 4 stages, or of 8 half-width stages, which needs tiles of
 * at most 256 columns) and the item length (128 to 4096 stages of 16 rows of
 * m per work item).  *chosen (may be NULL) receives the item length;
 * sk_batch_config reports the whole choice.  When SK_TUNE_CACHE names a
 * writable file the choice is recorded there under a signature of the
 * batch's shapes.  Errors as sk_batch_run. */
sk_status sk_batch_tune(sk_batch_handle b, void* stream, int64_t* chosen);

/* Fix the configuration of later runs instead of tuning: item_stages >= 1
 * (16-row units of m per work item), tile_cols 512 or 256 (widest output
 * tile), ring_stages 4 or 8 (8 requires tile_cols 256).  Invalidates the
 * plan and graph.  Errors: SK_EINVAL. */
sk_status sk_batch_set_config(sk_batch_handle b, int64_t item_stages, int32_t tile_cols,
                              int32_t ring_stages);

/* The configuration the next plan uses (tuned, set, cached or default);
 * any output pointer may be NULL.  Errors: SK_EINVAL. */
sk_status sk_batch_config(sk_batch_handle b, int64_t* item_stages, int32_t* tile_cols,
                          int32_t* ring_stages);

/* Synchronise `stream`, return and clear the batch's device status word
 * (SK_OK or SK_ETIMEOUT). */
sk_status sk_batch_status(sk_batch_handle b, void* stream);

/* Number of sketches in the batch (in *count). */
sk_status sk_batch_size(sk_batch_handle b, int64_t* count);

/* Release the batch and its device buffers (not the members' handles). */
sk_status sk_batch_destroy(sk_batch_handle b);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of left sketches under an HBM budget.
 *
 * The paper sketches one matrix per call (Sec. 3 problem statement); a
 * server turns the same operation into a request stream.  A server owns one
 * device pool of `hbm_budget_bytes` (allocated at creation) and a host
 * scheduler thread.  sk_server_submit enqueues a request for the left sketch
 * Y[k x n] = S[k x m] A[m x n] of a handle; the request's arrival time is the
 * time of the call.  The scheduler:
 *  - admits pending requests strictly in arrival order while the next one
 *    fits in the pool and fewer than `max_slots` requests are resident; an
 *    admitted request receives pool memory for a copy of A (row stride n
 *    rounded up to 4), for Y (same stride) and for its split partials, and
 *    A is copied in on a copy stream;
 *  - at each step boundary (one of its two compute streams idle) launches
 *    every admitted request not yet launched as one step: the SK_BF16X2
 *    requests as one persistent batched launch plus one batched reduce
 *    (as sk_batch_run), the SK_FP32 requests as fused SIMT launches.  Steps
 *    on the two streams overlap on the device, so requests arriving while
 *    others run join the next step without waiting for the GPU to drain;
 *  - completes a step when its event is observed; the copy of A and the
 *    partials go back to the pool, Y stays there until fetched or released.
 * Latency = arrival to the observation of the completion (host steady
 * clock).  Work items have a fixed length (512 stages of 16 rows), so a
 * request's decomposition, its accumulation order and its result depend
 * only on its own (seed, dist, k, precision, A), never on the mix.
 * All server calls are thread-safe. */
typedef struct sk_server* sk_server_handle;

typedef struct {
  int64_t submitted;          /* requests accepted by sk_server_submit */
  int64_t completed;          /* finished without error */
  int64_t failed;             /* finished with a device error */
  int64_t pending;            /* waiting for admission */
  int64_t resident;           /* holding pool memory (admitted, running or done) */
  int64_t steps;              /* steps launched */
  int64_t max_step_requests;  /* most requests in one step */
  double p50_ms, p99_ms;      /* latency percentiles of completed requests */
  double mean_ms, max_ms;
  double mean_wait_ms;        /* arrival to launch, mean over completed */
  double flops;               /* 2 k m n summed over completed requests */
  double busy_s;              /* first arrival to last completion, seconds */
  uint64_t pool_bytes;        /* size of the pool */
  uint64_t peak_bytes;        /* most pool bytes in use at once */
} sk_server_stats;

/* Create a server on the current device with a pool of `hbm_budget_bytes`
 * (rounded up to 256) and at most `max_slots` resident requests (>= 1).
 * Errors: SK_EINVAL, SK_ENOMEM (pool allocation), SK_ECUDA. */
sk_status sk_server_create(uint64_t hbm_budget_bytes, int32_t max_slots,
                           sk_server_handle* out);

/* Submit Y = S A for handle `h` (form SK_BF16X2 or SK_FP32; seed, dist, k and
 * form are read now, the handle may be destroyed afterwards).  A[m x n] with
 * leading dimension lda is a host or device pointer (unified addressing).
 * The server records an event on `stream` (the stream that produces A; NULL
 * = the legacy default stream) and copies A only after it, so A may still be
 * in production on that stream; A must stay valid and unchanged until the
 * request completes or fails.  Device memory, managed memory and mapped
 * pinned host memory are read by a copy kernel, pageable host memory through
 * the copy engine.  On success *ticket identifies the request.  Errors:
 * SK_EINVAL, SK_EUNSUPPORTED (other forms), SK_EBUDGET (the request alone
 * needs more than the whole pool; nothing is enqueued), SK_ECANCELLED
 * (server shutting down), SK_ECUDA. */
sk_status sk_server_submit(sk_server_handle s, sk_handle h, const float* A, int64_t m,
                           int64_t n, int64_t lda, void* stream, int64_t* ticket);

/* Non-blocking: SK_OK when the request has completed (then *latency_ms, if
 * not NULL, receives its latency), SK_EBUSY while pending or running, the
 * device error (e.g. SK_ETIMEOUT) if it failed, SK_EINVAL for an unknown or
 * released ticket. */
sk_status sk_server_poll(sk_server_handle s, int64_t ticket, double* latency_ms);

/* As sk_server_poll, but blocks up to `timeout_s` seconds for completion;
 * SK_EBUSY when the time ran out. */
sk_status sk_server_wait(sk_server_handle s, int64_t ticket, double timeout_s,
                         double* latency_ms);

/* Copy the completed request's Y[k x n] into `Y` (host or device pointer,
 * leading dimension ldy >= n) on `stream`, after the work already enqueued
 * there, wait for the copy and release the request.  Errors: SK_EBUSY (not
 * complete), the request's device error (the request is released),
 * SK_EINVAL, SK_ECUDA (the result is kept; the call may be repeated). */
sk_status sk_server_fetch(sk_server_handle s, int64_t ticket, float* Y, int64_t ldy,
                          void* stream);

/* Release a request: its pool memory is returned now if it has finished,
 * else as soon as it finishes (its latency still counts).  SK_EINVAL for an
 * unknown ticket. */
sk_status sk_server_release(sk_server_handle s, int64_t ticket);

/* Snapshot of the server's counters and latency percentiles. */
sk_status sk_server_stats_get(sk_server_handle s, sk_server_stats* out);

/* Clear the latency samples and counters of finished requests (pending and
 * resident requests are kept). */
sk_status sk_server_reset_stats(sk_server_handle s);

/* Stop admitting, wait for launched steps to finish (pending requests are
 * cancelled), release the pool and the server. */
sk_status sk_server_destroy(sk_server_handle s);

/* Synchronise `stream` and copy the handle's four device status words
 * without clearing them: [0] the sk_status sk_stream_status would return,
 * [1] where the first bounded wait that gave up was waiting (role * 16 +
 * barrier: roles 1 TMA producer, 2 MMA issuer, 3 epilogue, 4 worker;
 * barriers 0 staging full, 1 staging empty, 2 operand full, 3 operand empty,
 * 4 accumulator full, 5 accumulator empty, 6 S rows received from another
 * CTA, 8 work-queue slot free, 9 work item published), [2] the pipeline stage (or
 * accumulation chain) it was waiting for, [3] the linear index of its CTA.
 * Words 1-3 are meaningful only when word 0 is SK_ETIMEOUT. */
sk_status sk_debug_status(sk_handle h, void* stream, int32_t out[4]);

/* Failure injection for tests of the bounded waits above (not in the paper;
 * it lets a test make a device wait run out without faulting anything).
 * limit_ns: the limit of every bounded wait of the handle's later tensor-
 * core launches, at least 1 ms; 0 restores the default of 2 s.
 * stall_stage >= 0: in later BF16 left sketches on this handle the TMA
 * producer issues no copy for that pipeline stage (stages counted from 0
 * over each CTA's, or CTA pair's, run of a launch), so every wait that
 * depends on it gives up after
 * limit_ns: the kernel records SK_ETIMEOUT and the waiting site (see
 * sk_debug_status), waits (again bounded) for the copies and MMAs already
 * in flight, frees its tensor memory and exits; Y is then undefined.
 * stall_stage < 0 turns the injection off.  Errors: SK_EINVAL. */
sk_status sk_debug_set_wait(sk_handle h, uint64_t limit_ns, int64_t stall_stage);

/* Release the handle and the device memory it owns.  Waits for nothing:
 * the caller must ensure no enqueued work still uses it. */
sk_status sk_destroy(sk_handle h);

/* Measurement hook: when both events are non-NULL (cudaEvent_t created by
 * the caller on the handle's device), every later apply call records
 * `start_event` on its stream immediately before the launch of its main
 * fused kernel and `stop_event` immediately after it, so the caller can
 * read that kernel's duration with cudaEventElapsedTime.  NULL, NULL turns
 * the hook off.  The events stay owned by the caller. */
sk_status sk_profile_events(sk_handle h, void* start_event, void* stop_event);

/* Number of kernels this library has launched in the calling process
 * (all handles, all devices), for launch accounting. */
uint64_t sk_launch_count(void);

/* Static human-readable name of a status code. */
const char* sk_status_string(int status);

/* Description of the CUDA error behind the most recent SK_ECUDA / SK_ENOMEM
 * returned to the calling host thread ("no error" if none). */
const char* sk_last_cuda_error(void);

/* Library version as an integer MAJOR*10000 + MINOR*100 + PATCH. */
int sk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SKETCH_H_ */
