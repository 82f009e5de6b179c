/*
 * qftfft.h -- C ABI of the GB300 QFT->FFT library (libqftfft.so).
 *
 * The library computes discrete Fourier transforms by executing the quantum
 * Fourier transform circuit on a 2^n-amplitude state vector, following
 * Markidis et al., "Not Your Usual FFT: QFT->FFT via Classical Quantum-Circuit
 * Simulation".  The problem statement it implements is Sec. 3 of that paper:
 *
 *   1. encode:  scale_in = ||x||_2, psi = x / scale_in, index k of the array is
 *               the basis state |b_{n-1} ... b_0>, qubit q_j = bit j (LSB q_0);
 *   2. build the n-qubit QFT circuit of Fig. 1 (H on each wire from the most
 *      significant down, each followed by the controlled phases R_{d+1}
 *      whose control lies d wires below, then the qubit-reversal swaps); the
 *      range-k approximate QFT keeps only the controlled phases with d <= k
 *      (Sec. 2, "Approximate QFT");
 *   3. evolve:  psi' = U psi with U = DFT_N / sqrt(N) (Sec. 3 step 3), where
 *      DFT_N = [omega^{kl}], omega = e^{-2 pi i / N} for the forward direction
 *      (Sec. 2) and e^{+2 pi i / N} for the inverse;
 *   4. decode:  rescale psi' to FFT units with scale_in (Sec. 3 step 4).
 *
 * Calls map onto those steps: qft_plan_create (step 2, host only),
 * qft_load (step 1: place the caller's array in the state buffer),
 * qft_execute (steps 1 and 3-4 on the GPU: the norm, the circuit and the
 * rescaling run inside the pass kernels), qft_read (copy the result out).
 *
 * Everything is asynchronous on the caller's CUDA stream unless stated.  No
 * call allocates device memory except qft_plan_create (small, plan-owned) and
 * the server calls; state buffers and workspaces are caller-owned.
 *
 * Data layout: a state is N = 2^n complex numbers, interleaved (re, im):
 * complex64 = 2 x float32 (8 bytes), complex128 = 2 x float64 (16 bytes) --
 * the memory layout of torch.complex64 / torch.complex128.  Device pointers
 * must be 256-byte aligned (what cudaMalloc and the torch caching allocator
 * return).
 *
 * Errors: every call returns QFT_OK (0) or a negative QFT_ERR_* code; no call
 * aborts, throws or traps.  A CUDA launch/runtime failure is reported as
 * QFT_ERR_CUDA (qft_last_cuda_error gives the cudaError_t value).  Faults that
 * happen asynchronously on the GPU surface at the caller's next synchronising
 * CUDA call.
 */
#ifndef QFTFFT_H
#define QFTFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque handles.  qft_stream_t is a cudaStream_t (NULL = legacy default stream). */
typedef struct qft_plan_s* qft_plan_t;
typedef struct qft_server_s* qft_server_t;
typedef struct CUstream_st* qft_stream_t;

enum qft_dtype { QFT_C64 = 0, QFT_C128 = 1 };

/* Sign of the exponent (Sec. 2: omega_N = e^{-2 pi i / N} is the forward transform). */
enum qft_direction { QFT_FORWARD = -1, QFT_INVERSE = +1 };

/* Output scaling (Sec. 3 step 4).  With psi' = DFT_N x / (scale_in sqrt N):
 *   STATE    psi'                       (the normalised simulator state)
 *   UNITARY  scale_in psi'  = DFT_N x / sqrt(N)
 *   UNNORM   scale_in sqrt(N) psi' = DFT_N x      (numpy.fft.fft for FORWARD)
 *   INV_N    scale_in psi' / sqrt(N) = DFT_N x / N (numpy.fft.ifft for INVERSE) */
enum qft_scale { QFT_SCALE_STATE = 0, QFT_SCALE_UNITARY = 1, QFT_SCALE_UNNORM = 2, QFT_SCALE_INV_N = 3 };

/* Output index order.  NATURAL applies the final qubit-reversal swaps (a drop-in
 * FFT); BITREV leaves them to the caller as an output index permutation, as the
 * paper does (Sec. 3 step 2): out[i] holds frequency bitrev_n(i). */
enum qft_order { QFT_ORDER_NATURAL = 0, QFT_ORDER_BITREV = 1 };

enum qft_status {
    QFT_OK = 0,
    QFT_ERR_BAD_ARG = -1,     /* NULL handle/pointer, n or k or enum out of range   */
    QFT_ERR_SIZE = -2,        /* length is zero or not a power of two                */
    QFT_ERR_BUDGET = -3,      /* request exceeds the server's HBM admission budget   */
    QFT_ERR_CUDA = -4,        /* a CUDA runtime/driver call failed                    */
    QFT_ERR_TIMEOUT = -5,     /* a bounded wait (host or device) ran out             */
    QFT_ERR_NOMEM = -6,       /* host or plan-owned device allocation failed         */
    QFT_ERR_UNSUPPORTED = -7, /* valid request the library does not implement       */
    QFT_ERR_STATE = -8,       /* call out of order (e.g. unknown ticket)             */
    QFT_ERR_CANCELED = -9     /* the request was withdrawn before it ran             */
};

/* Planner options; pass NULL for defaults.  Zero fields mean "choose". */
typedef struct {
    int order;          /* QFT_ORDER_NATURAL (default) or QFT_ORDER_BITREV                 */
    int tile_bits;      /* log2(amplitudes per CTA tile); 0 = default (complex64 natural
                           order from n = 23: the wide pass kernel, 14; else 13 c64, 12
                           c128).  14 (complex64, NATURAL order, no other shape field, no
                           precision tier, the whole register or a subset plan with w0
                           = 0) asks for the wide pass kernel: tiles of 2^14 amplitudes (4
                           coalescing batch bits and two register stages of up to 5
                           wires), so ceil(n / 10) passes; QFT_ERR_UNSUPPORTED where the
                           planner finds no wide shape.  Default plans take it, where
                           the planner finds a wide shape, for complex64 natural order
                           on arrays of >= 2^23 amplitudes (n >= 23, or w0 = 0 subsets
                           of n >= 14 wires).                                           */
    int coalesce_bits;  /* min log2(contiguous amplitudes per HBM run); 0 = default         */
    int max_stage_bits; /* max wires per register stage (1..5; 1..4 with 512 threads); 0 =
                           default.  With a tensor-core tier (precision 1..5) it is f, the
                           widest fused block (4..7; 0 = 6): one block of <= f wires per
                           pass, 2^12-amplitude tiles for f = 5, 6 and 2^11 for f = 4, 7
                           (QFT_ERR_BAD_ARG outside 4..7)                                   */
    int wait_limit_ms;  /* bound of every device-side wait; 0 = default (2000 ms)           */
    int test_skip_first_load; /* TEST HOOK, 0 in normal use: 1 = never issue the first
                                 tile load, so the kernel's bounded wait expires and
                                 reports QFT_ERR_TIMEOUT (exercises failure reporting
                                 without a fault; see also the test-hook section)       */
    int threads;        /* CTA size of the pass kernel: 256 (stages <= 5 wires) or 512
                           (stages <= 4 wires); 0 = default.  Double-float complex128 with
                           256 threads, tile_bits <= 11 and max_stage_bits <= 3 runs two
                           CTAs per SM (128 registers per thread).                         */
    int precision;      /* QFT_PREC_*: 0 = the default CUDA-core path (complex64 in FP32;
                           complex128 in double-float, see QFT_PREC_FP64); 6 = complex128 in
                           IEEE FP64 arithmetic; 1..5 = complex64 only, each pass's fused
                           block of <= f wires (max_stage_bits; default 6) as a dense
                           complex GEMM on the tensor cores
                           (see enum qft_precision).  The block matrices are built and
                           uploaded (plan-owned device memory) by the plan's first execute,
                           which should precede any capture. */
    int paired;         /* must be 0.  (Packed FP32x2 "paired" stages, one thread running two
                           groups, measured slower than one group per thread on GB300 in
                           every plan shape and were removed; 1 gives
                           QFT_ERR_UNSUPPORTED.  Passes whose tile is <= 2^12 complex64
                           amplitudes and whose blocks have <= 4 wires run two CTAs per
                           SM.)                                                            */
    int pass_split;     /* NATURAL order, 3 or more passes: how wires left over by an even
                           split are placed.  1 = on the middle passes, so the first pass
                           (whose HBM runs the natural-order input spreads over the whole
                           state) keeps more batch wires and so longer runs; 2 = on the
                           first passes; 0 = the planner's choice (1 for complex64 with
                           n >= 27 and default tiles, where it measured faster; else 2).
                           With all shape fields 0 the planner also picks 2^12-amplitude
                           tiles for complex64 n >= 27 and 512 threads for double-float
                           complex128 n >= 21 (the tuned shapes on GB300).                */
} qft_opts;

/* Precision tier (complex64 plans): the block matrix and the data are rounded to
 * the operand format, products accumulate in FP32.  The x3 tiers split each
 * operand into hi + lo and add hi*hi + lo*hi + hi*lo.
 *
 * complex128 plans compute by default in double-float arithmetic: every
 * amplitude is an unevaluated sum of two FP32 numbers (about 48 significant
 * bits) and all arithmetic runs on the FP32 pipe with error-free
 * transformations, because GB300 executes FP64 at 1/64 of its FP32 rate.  The
 * input and output stay IEEE complex128 in memory; the relative L2 error
 * against the exact transform stays far inside 1e-13 n.  Before the first pass
 * a pre-pass reads the state once for its largest binary exponent, and the
 * input is scaled by that power of two (exactly) so every FP64 magnitude is
 * handled; zero and subnormal FP64 components are read as zero.
 * QFT_PREC_FP64 runs the same passes in IEEE FP64 arithmetic instead.
 * Batches (qft_batch_*) run complex128 transforms in the plans' arithmetic
 * (all plans of one batch must agree). */
enum qft_precision { QFT_PREC_NATIVE = 0, QFT_PREC_TF32 = 1, QFT_PREC_BF16 = 2, QFT_PREC_BF16X3 = 3,
                     QFT_PREC_FP16 = 4, QFT_PREC_FP16X3 = 5, QFT_PREC_FP64 = 6 };

/* What the planner built (Sec. 3.1: the plan is defined by the qubit count,
 * the fused blocks and the pre-fusion gate counters). */
typedef struct {
    int n, k_eff, direction, dtype, order;
    long long n_h, n_cp, n_swap;     /* gate counts before fusion (Table 2)            */
    int passes;                      /* HBM sweeps per execute                          */
    int wires_per_pass[8];           /* transform wires fused into each pass            */
    int stages_per_pass[8];          /* register stages (fused blocks) in each pass     */
    int tile_bits[8];                /* log2(amplitudes per tile) of each pass          */
    int coalesce_bits[8];            /* log2(contiguous amplitudes per run) per pass   */
    size_t workspace_bytes;          /* qft_workspace_size()                            */
    long long bytes_per_execute;     /* algorithmic HBM bytes: passes * 2 * N * elem   */
    int n_addr, w0;                  /* array of 2^n_addr amplitudes; the transform acts
                                        on index bits [w0, w0 + n) (qft_plan_create:
                                        n_addr = n, w0 = 0)                            */
    int fused_blocks;                /* Sec. 3.1's plan (num_qubits, fused_blocks,
                                        max_fused_size): the fused gate blocks the
                                        circuit is cut into -- here the register stages
                                        of all passes, each one block of consecutive
                                        wires with its Hadamards and controlled phases */
    int max_fused_size;              /* qubits of the widest fused block               */
} qft_plan_info;

/* Step 2 (Sec. 3, Fig. 1): build the circuit for n qubits, cutoff k
 * (k < 0 or k >= n-1: exact QFT; 0 <= k < n-1: range-k AQFT, Sec. 2),
 * direction (QFT_FORWARD/QFT_INVERSE) and dtype (QFT_C64/QFT_C128), and plan its
 * passes.  Host work only, plus a small plan-owned device block.  1 <= n <= 34
 * (c64) or 33 (c128).  *out is set to NULL on failure. */
int qft_plan_create(qft_plan_t* out, int n, int k, int direction, int dtype, const qft_opts* opts);
int qft_plan_destroy(qft_plan_t plan);

/* A QFT on a subset of the index bits (multi-dimensional and strided batched
 * transforms as QFTs on qubit subsets): the array has 2^n_addr amplitudes,
 * and the n-wire (A)QFT of Sec. 3 acts on the qubits q_w0 .. q_{w0+n-1}
 * (index bits [w0, w0 + n)), independently for every value of the other
 * index bits.  A row-major 2^a x 2^b array transforms along its rows with
 * (n_addr = a + b, w0 = 0, n = b) and along its columns with (w0 = b, n = a);
 * both in turn give the 2-D DFT.  NATURAL order reverses only the n
 * transform bits.  Supported shapes: w0 = 0 (any n, the planner of
 * qft_plan_create with the upper bits as a batch index); the n wires plus
 * min(w0, 4) low batch bits fit one tile (one HBM pass); or w0 >= 4 (3 for
 * complex128) for any n (several passes).  Other shapes return
 * QFT_ERR_UNSUPPORTED, as do the tensor-core tiers.  Execution as for qft_plan_create plans (load, execute,
 * execute_oop, read with 2^n_addr amplitudes), except that QFT_SCALE_STATE is
 * rejected (QFT_ERR_BAD_ARG): there is no single state to normalise.  Subset
 * plans are not batched (qft_batch_create: QFT_ERR_UNSUPPORTED). */
int qft_plan_create_subset(qft_plan_t* out, int n_addr, int w0, int n, int k, int direction, int dtype,
                           const qft_opts* opts);
int qft_plan_get_info(qft_plan_t plan, qft_plan_info* info);

/* Bytes of caller-allocated device workspace qft_execute needs (always > 0:
 * it holds scale_in, the status word and the norm partial sums; NATURAL-order
 * plans of more than one pass also need an N-amplitude ping-pong buffer). */
size_t qft_workspace_size(qft_plan_t plan);

/* Step 1: copy len complex values from src into the device state buffer
 * d_state (N = 2^n amplitudes of the plan's dtype).  src is a host pointer
 * (src_on_device = 0; pinned memory gives an asynchronous copy) or a device
 * pointer (src_on_device = 1).  len must equal 2^n (QFT_ERR_SIZE otherwise).
 * The normalisation x / scale_in is deferred: qft_execute computes scale_in
 * while it reads the state and folds 1/scale_in into its last store. */
int qft_load(qft_plan_t plan, void* d_state, const void* src, size_t len, int src_on_device,
             qft_stream_t stream);

/* Step 1 for a length that is not a power of two: the register has
 * n = ceil(log2 len) qubits (Sec. 3 step 1), so the caller's len <= 2^n
 * values are copied to the start of d_state and the other 2^n - len
 * amplitudes are set to zero.  The transform is then the 2^n-point DFT of the
 * zero-padded sequence -- the paper's encoding, which is not the len-point
 * DFT of the data.  len > 2^n gives QFT_ERR_SIZE; len = 2^n is qft_load. */
int qft_load_padded(qft_plan_t plan, void* d_state, const void* src, size_t len, int src_on_device,
                    qft_stream_t stream);

/* Steps 1 and 3-4 on the GPU, in place on d_state: scale_in = ||x||_2,
 * psi' = U (x / scale_in), then the output scaling scale_mode (QFT_SCALE_*).
 * d_workspace: qft_workspace_size(plan) bytes of device memory, 256-byte
 * aligned, owned by the caller; after the call its first double holds
 * scale_in (see qft_get_scale_in).  d_scale_in: optional device pointer that
 * also receives scale_in (NULL = none).  A zero input gives a zero output and
 * scale_in = 0.  Concurrent executes must use distinct workspaces. */
int qft_execute(qft_plan_t plan, void* d_state, void* d_workspace, double* d_scale_in, int scale_mode,
                qft_stream_t stream);

/* qft_execute out of place: reads d_in (N amplitudes, 256-byte aligned,
 * not modified) and writes the result to d_out (N amplitudes, 256-byte
 * aligned).  Same steps, workspace, scale_in and errors as qft_execute; the
 * state is never copied: the first pass reads d_in and the last pass writes
 * d_out.  d_in == d_out is the in-place transform; buffers that overlap
 * otherwise give undefined results. */
int qft_execute_oop(qft_plan_t plan, const void* d_in, void* d_out, void* d_workspace, double* d_scale_in,
                    int scale_mode, qft_stream_t stream);

/* One pass of qft_execute: launches only pass `pass` (0 .. passes-1, see
 * qft_plan_get_info).  Calling it for pass = 0, 1, ..., passes-1 in order on
 * one stream is exactly qft_execute (pass 0 also clears the status word); it
 * lets a caller put events or other work between the HBM sweeps. */
int qft_execute_pass(qft_plan_t plan, int pass, void* d_state, void* d_workspace, double* d_scale_in,
                     int scale_mode, qft_stream_t stream);

/* ---------------------------------------------------------------- batches
 * Many transforms of different sizes and cutoffs in one call.  (Batching is
 * not in the paper, which times one transform at a time; it is the same
 * circuit per transform.)  All plans of a batch must share dtype and
 * direction.  Each transform's result, scale handling and accuracy are those
 * of qft_execute with the same plan, within the parity bounds of its
 * arithmetic (a transform may run on another pass shape than its plan's, see
 * qft_batch_execute).  Plans of the tensor-core precision tier
 * (qft_opts.precision != 0) are not batched: QFT_ERR_UNSUPPORTED; nor are
 * plans on 2^14-amplitude tiles (qft_opts.tile_bits = 14, and the default
 * complex64 natural-order plans from n = 23) outside 14 <= n <= 20. */
typedef struct qft_batch_s* qft_batch_t;

/* Bytes of caller-owned device workspace a batch of these plans needs
 * (per transform: scale_in and norm partial sums, plus the ping-pong buffer of
 * natural-order multi-pass plans).  0 on bad arguments. */
size_t qft_batch_workspace_size(const qft_plan_t* plans, int count);

/* Bind transform i = plans[i] on d_states[i] (2^n amplitudes each, 256-byte
 * aligned) for i < count.  d_workspace: qft_batch_workspace_size bytes,
 * 256-byte aligned, caller-owned.  d_scale_in: optional device array of count
 * doubles that receives each scale_in (NULL = none).  scale_mode: QFT_SCALE_*
 * for every transform.  Allocates the batch's small device tables (work list,
 * pass descriptors, tensor maps); the plans must outlive the batch. */
int qft_batch_create(qft_batch_t* out, const qft_plan_t* plans, void* const* d_states, int count, void* d_workspace,
                     size_t workspace_bytes, double* d_scale_in, int scale_mode);

/* Run every transform of the batch in place, asynchronously, on stream
 * (capturable into a CUDA graph).  Complex64 natural-order transforms of
 * 14 <= n <= 20 qubits whose plans leave the tile shape to the planner (or ask
 * for tile_bits = 14) run on the 2^14-amplitude-tile pass kernel: one launch
 * per pass for all transforms of one (n, k, direction), on the batch's side
 * streams, which wait for stream and which stream then waits for.  The rest
 * run in one persistent launch over a work list on stream itself.  Before
 * either, one memset clears the counters and the status word. */
int qft_batch_execute(qft_batch_t batch, qft_stream_t stream);

/* How a batch runs (qft_batch_execute). */
typedef struct {
    int transforms;        /* count given to qft_batch_create                        */
    int wide_groups;       /* (n, k, direction) groups on the 2^14-tile pass kernel   */
    int wide_transforms;   /* transforms in those groups                            */
    int persistent_items;  /* tile items of the persistent launch (0: no launch)      */
    int kernel_launches;   /* kernels one qft_batch_execute launches                 */
    int side_streams;      /* streams the groups run on                              */
} qft_batch_info;
int qft_batch_get_info(qft_batch_t batch, qft_batch_info* info);

/* Synchronise stream and read the batch's device status word (0 or QFT_ERR_TIMEOUT). */
int qft_batch_status(qft_batch_t batch, qft_stream_t stream);
int qft_batch_destroy(qft_batch_t batch);

/* ---------------------------------------------------------------- serving
 * A continuous-batching request loop for transforms of mixed n, cutoff,
 * direction and dtype (not in the paper; each request runs the circuit of
 * Sec. 3).  A worker thread admits requests in arrival order as soon as their
 * device bytes fit in the HBM budget next to everything in flight and an
 * in-flight slot is free.  Small requests (n <= the batching limit, 18 by
 * default, see qft_server_set_batching) join the batch forming for their
 * (dtype, direction, scale mode), and every pass of the worker launches each
 * forming batch whose slot is free as one batched persistent launch (the
 * qft_batch kernel) on a high-priority stream, so requests that arrive while
 * others run join the next batch as slots and memory free up.  Larger
 * requests run their own passes (copy in, qft_execute, copy out) on the
 * least-loaded of the normal-priority streams; the batches are scheduled
 * between those passes.  Server batches use one fixed kernel shape, so a
 * request's result is bit for bit the same alone and in any mix.  Each
 * request's latency is recorded from submit to completion.  The server
 * allocates and pools its own device buffers and caches one plan per (n, k,
 * direction, dtype, order). */
typedef struct {
    int n, k, direction, dtype, order, scale_mode; /* as qft_plan_create / qft_execute        */
    const void* input;                             /* 2^n complex values, host or device     */
    int input_on_device;
    void* output;                                  /* 2^n complex values, host or device     */
    int output_on_device;
    double* scale_in_out;                          /* optional host double receiving scale_in */
} qft_request;

typedef struct {
    long long completed, failed, pending, in_flight;
    size_t bytes_in_use, bytes_pooled;
    double p50_ms, p99_ms, max_ms;                 /* submit-to-completion latency           */
    double requests_per_s;                         /* completed / (last completion - first submit) */
    long long batches;                             /* batched launches since the last reset       */
    long long batched_requests;                    /* requests those launches carried              */
} qft_server_stats;

/* Start a server on the current device.  hbm_budget_bytes bounds the device
 * memory of admitted requests; streams (0 = 8) and max_inflight (0 = 64). */
int qft_server_create(qft_server_t* out, size_t hbm_budget_bytes, int streams, int max_inflight);
/* Queue a request (its buffers must stay valid until it completes); *ticket identifies it.
 * Requests larger than the budget fail with QFT_ERR_BUDGET. */
int qft_server_submit(qft_server_t server, const qft_request* request, uint64_t* ticket);
/* *done = 1 once finished; returns the request's status if finished, else QFT_OK. */
int qft_server_poll(qft_server_t server, uint64_t ticket, int* done);
/* Block until the request finishes (timeout_ms < 0: no limit; QFT_ERR_TIMEOUT when it
 * expires) and return its status; *latency_ms (optional) gets its latency.  Forgets the ticket. */
int qft_server_wait(qft_server_t server, uint64_t ticket, int timeout_ms, double* latency_ms);
int qft_server_get_stats(qft_server_t server, qft_server_stats* out);
int qft_server_reset_stats(qft_server_t server);
/* Withdraw a request that has not been admitted yet: QFT_OK, and the ticket
 * then reports QFT_ERR_CANCELED (poll / wait).  A request already running or
 * finished cannot be withdrawn: QFT_ERR_STATE. */
int qft_server_cancel(qft_server_t server, uint64_t ticket);
/* Requests with n <= max_n (0 <= max_n <= 34; 0 = none) are batched; the
 * default is 18.  Requests already admitted keep their path. */
int qft_server_set_batching(qft_server_t server, int max_n);
/* Finish every queued request, then stop the worker and free the server's memory. */
int qft_server_destroy(qft_server_t server);

/* qft_execute without a caller-provided workspace, for callers that cannot
 * allocate device memory: code that runs while a stream is being captured into
 * a CUDA graph (cudaMalloc is not allowed during capture), host runtimes that
 * own the device heap and give libraries no allocator, and latency-critical
 * loops that must never enter an allocator.  The paper has no counterpart;
 * this is a library convenience.
 *
 * The workspace comes from a fixed scratch array in the library's device image
 * (32 MiB + 4 KiB, held on every GPU that loads the library until the process
 * exits).  Plans whose qft_workspace_size() exceeds it are rejected with
 * QFT_ERR_SIZE: BITREV plans and single-pass plans always fit; NATURAL-order
 * multi-pass plans fit up to n = 22 (complex64) / n = 21 (complex128).
 * Allocates nothing.  The first call on a device looks up the scratch address
 * for that device (it must be the current device) and caches it, so make the
 * first call before any stream capture.  All calls share the scratch and it
 * keeps the last call's contents; calls whose kernels overlap on the GPU race.
 * scale_in is returned only through d_scale_in (device pointer, may be NULL).
 * Tensor-core tier plans (qft_opts.precision 1..5) allocate their block
 * matrices on their first qft_execute; before that has run, this entry point
 * returns QFT_ERR_UNSUPPORTED instead of allocating.  A device wait that
 * expired is reported by qft_noalloc_status, not by the return code. */
int qft_execute_noalloc(qft_plan_t plan, void* d_state, double* d_scale_in, int scale_mode, qft_stream_t stream);

/* The status word of the scratch used by qft_execute_noalloc on the current
 * device, after synchronising stream: 0, or QFT_ERR_TIMEOUT if a kernel of the
 * last such call gave up a bounded wait (its output is then incomplete).
 * Allocates nothing; a negative QFT_ERR_* on a CUDA failure. */
int qft_noalloc_status(qft_stream_t stream);

/* Read-back after Sec. 3 step 4 (the decode scaling, applied by qft_execute's
 * last pass): copy the N results from d_state to dst (host if dst_on_device =
 * 0, else device).  Asynchronous on stream; pinned host memory gives an
 * asynchronous copy.  QFT_ERR_BAD_ARG on null pointers; dst == d_state is a
 * no-op. */
int qft_read(qft_plan_t plan, const void* d_state, void* dst, int dst_on_device, qft_stream_t stream);

/* Synchronise stream, then return scale_in recorded in the workspace by the last execute. */
int qft_get_scale_in(qft_plan_t plan, const void* d_workspace, double* out, qft_stream_t stream);

/* Synchronise stream and read the device status word of the workspace
 * (0 = ok, QFT_ERR_TIMEOUT if a kernel's bounded wait expired). */
int qft_check_status(qft_plan_t plan, const void* d_workspace, qft_stream_t stream);

/* ---------------------------------------------------------------------------
 * Real-input transforms of N = 2^n real samples (2 <= n <= 34 for float32
 * data, QFT_C64; 2 <= n <= 33 for float64 data, QFT_C128).  They pack the
 * real samples into the N/2 amplitudes of an (n-1)-qubit state (sample 2m as
 * the real and 2m+1 as the imaginary part, the same bytes) and run the exact
 * (n-1)-qubit QFT (Sec. 3 steps 2-3) plus one sweep that separates or joins
 * the spectra of the even and odd samples.  This extends the paper's encode
 * step (Sec. 3 step 1), which takes complex input only.
 *
 *   FORWARD (R2C, numpy.fft.rfft):  d_in = N reals, d_out = N/2 + 1 complex
 *       X_k = f sum_j x_j e^{-2 pi i j k / N},  k = 0 .. N/2
 *   INVERSE (C2R, numpy.fft.irfft): d_in = N/2 + 1 complex (a Hermitian half
 *       spectrum; the imaginary parts of X_0 and X_{N/2} are ignored),
 *       d_out = N reals
 *       x_j = f sum_{k=0}^{N-1} X_k e^{+2 pi i j k / N},  X_{N-k} = conj X_k
 *
 * f is the scale mode's factor: QFT_SCALE_UNNORM 1, QFT_SCALE_UNITARY
 * 1/sqrt(N), QFT_SCALE_INV_N 1/N (numpy's rfft is FORWARD + UNNORM, its irfft
 * INVERSE + INV_N).  QFT_SCALE_STATE has no meaning here: QFT_ERR_BAD_ARG.
 * d_in and d_out are distinct, 256-byte aligned device buffers; d_in is not
 * modified.  The workspace is qft_rplan_workspace_size() bytes.  opts as for
 * qft_plan_create (order must be NATURAL; tensor-core tiers are not offered:
 * QFT_ERR_UNSUPPORTED).  qft_rplan_create allocates small plan-owned twiddle
 * tables (complex128 only). */
typedef struct qft_rplan_s* qft_rplan_t;
int qft_rplan_create(qft_rplan_t* out, int n, int direction, int dtype, const qft_opts* opts);
int qft_rplan_destroy(qft_rplan_t plan);
size_t qft_rplan_workspace_size(qft_rplan_t plan);
int qft_rplan_execute(qft_rplan_t plan, const void* d_in, void* d_out, void* d_workspace, int scale_mode,
                      qft_stream_t stream);

/* ---------------------------------------------------------------------------
 * Quantum phase estimation on the QFT engine (eigenvalue estimation, named in
 * the paper's conclusion, Sec. 6, as the next use of a QFT state-vector
 * simulator).  The operator U is given in its eigenbasis: d = 2^d_bits
 * eigenvectors u_j with eigenphases theta_j in turns (U u_j = e^{2 pi i
 * theta_j} u_j; theta_j is taken mod 1) and the input state's overlaps c_j
 * (complex, sum |c_j|^2 = 1 for a normalised input).  The joint register
 * holds m counting qubits in the low index bits and the system state in the
 * high bits: 2^(m + d_bits) amplitudes of the given dtype.
 *
 * qft_qpe_prepare writes the state after H on every counting qubit and the
 * controlled evolutions C-U^{2^k} (k = 0 .. m-1):
 *     psi[j 2^m + y] = c_j exp(2 pi i sum_k y_k frac(theta_j 2^k)) / sqrt(2^m)
 * (the phases of all controlled evolutions summed exactly as the 64-bit
 * fixed-point product frac(theta_j) 2^64 * y mod 2^64; only the final
 * sine/cosine rounds, in the dtype's precision).  d_theta: d
 * doubles, d_coef: d complex128 values, both device memory; d_workspace:
 * qft_qpe_workspace_size(m, d_bits) bytes of device memory, 16-byte aligned
 * (QFT_ERR_BAD_ARG otherwise), which the call fills with per-eigenvector
 * constants and must stay allocated until the prepare has run on the stream.
 * The Fourier
 * readout is then the transform of the counting qubits with omega =
 * e^{-2 pi i / 2^m} -- this library's QFT_FORWARD, the paper's convention,
 * which is the textbook inverse QFT of phase estimation: a subset plan
 * (qft_plan_create_subset(n_addr = m + d_bits, w0 = 0, n = m, k, QFT_FORWARD))
 * executed with QFT_SCALE_UNITARY.  qft_qpe_probabilities writes
 *     P(x) = sum_j |psi[j 2^m + x]|^2,   x = 0 .. 2^m - 1
 * (2^m doubles, device memory): the counting register's distribution, which
 * concentrates at x ~ theta_j 2^m.  Requires 1 <= m, 0 <= d_bits <= 20,
 * m + d_bits <= 34 (complex64) or 33 (complex128). */
size_t qft_qpe_workspace_size(int m, int d_bits);
int qft_qpe_prepare(void* d_state, int m, int d_bits, const double* d_theta, const void* d_coef, int dtype,
                    void* d_workspace, qft_stream_t stream);
int qft_qpe_probabilities(const void* d_state, int m, int d_bits, int dtype, double* d_prob, qft_stream_t stream);

/* ---------------------------------------------------------------------------
 * Monte Carlo backend (Sec. 6, "Monte Carlo simulation in the sum-over-
 * histories style"): estimates of single output bins of the range-k transform
 * (natural order) from importance-sampled input indices, at a cost set by the
 * number of samples M instead of the 2^n amplitudes.  The amplitude
 * <y|U_k|x> is the sum over input indices j of x_j exp(s 2 pi i phase(j, y) / N)
 * / sqrt(N), phase(j, y) = sum of j_a y_b 2^(a+b) over n-1-k <= a+b <= n-1
 * (j y mod N for the exact transform; s = direction).
 *
 * qft_mc_prepare builds the proposal from the input x (2^n amplitudes of the
 * dtype, device memory, 16-byte aligned): an integer weight per index,
 * q_j = floor(m_j 2^S / 2^(E+1)) + 1 (0 for x_j = 0) with
 * m_j = max(|Re x_j|, |Im x_j|), 2^E <= max m < 2^(E+1) and S = min(62 - n, 52),
 * formed by shifting the significand of m_j -- at least 1 for every nonzero
 * amplitude -- and their prefix sums, T = sum q, into
 * d_workspace (qft_mc_workspace_size(n) bytes of device memory, 256-byte
 * aligned; the workspace holds the proposal until the next prepare and also
 * the partial sums of qft_mc_sample and qft_mc_bins, so calls that overlap on
 * the device with the same workspace race; use one workspace per stream).
 *
 * qft_mc_sample draws M >= 1 indices: for uniform u_i in [0, 1) (d_uniforms,
 * M doubles in device memory, drawn by the caller; u_i 2^53 is truncated to
 * an integer) the target t = floor(u_i 2^53 T / 2^53) selects the index j
 * with C_{j-1} <= t < C_j (C the prefix sums of q), written to d_index (M
 * int64), and its weight w = x_j T / q_j to d_weight (M complex128, 2M
 * doubles, 16-byte aligned).  Every step is integer arithmetic or one correctly
 * rounded FP64 division and product.  A zero input gives index 0 and weight 0
 * everywhere.
 *
 * qft_mc_bins evaluates, for each of nbins (<= 65536) output bins d_bins
 * (int64, device memory), the mean of z_i = w_i exp(s 2 pi i phase(j_i, y) /
 * N) / sqrt(N) over the M samples (an unbiased estimate of <y|U_k|x>), the
 * unbiased estimate (|sum z|^2 - sum |z|^2) / (M (M - 1)) of |<y|U_k|x>|^2
 * and the standard error sqrt((sum |z|^2 / M - |mean|^2) / (M - 1)) of the
 * mean: d_out[4b .. 4b+3] = (Re mean, Im mean, power, standard error),
 * doubles in device memory.  The phase is exact (integers mod 2^n); its
 * sine and cosine and the products are FP32, summed in FP32 over runs of 32
 * samples and in FP64 beyond.  d_workspace must be the one the samples were
 * drawn with (it holds their sum of |w|^2).  k < 0 or k >= n - 1: exact.
 *
 * Sparse inputs (the backend's reach beyond a state vector): an input with K
 * nonzero amplitudes d_vals[j] (K values of the dtype, 16-byte aligned) at
 * input indices d_pos[j] (K int64, each < 2^n) of an n-wire register,
 * n <= 62.  qft_mc_prepare_sparse builds the proposal over the K entries
 * (S = min(62 - ceil(log2 K), 52); workspace qft_mc_sparse_workspace_size(K)
 * bytes) and qft_mc_sample_sparse draws entries exactly as above but writes
 * the drawn entry's input index d_pos[j] to d_index; qft_mc_bins then takes
 * the register's n.  1 <= K <= 2^34.
 *
 * All return QFT_ERR_BAD_ARG for null or misaligned pointers and out of range
 * sizes (dense: 1 <= n <= 34 complex64, 33 complex128; qft_mc_bins:
 * 1 <= n <= 62), and are asynchronous on the stream. */
size_t qft_mc_workspace_size(int n);
size_t qft_mc_sparse_workspace_size(int64_t K);
int qft_mc_prepare_sparse(int64_t K, int dtype, const void* d_vals, void* d_workspace, qft_stream_t stream);
int qft_mc_sample_sparse(int64_t K, int dtype, const int64_t* d_pos, const void* d_vals, const void* d_workspace,
                         const double* d_uniforms, int64_t m, int64_t* d_index, double* d_weight,
                         qft_stream_t stream);
int qft_mc_prepare(int n, int dtype, const void* d_x, void* d_workspace, qft_stream_t stream);
int qft_mc_sample(int n, int dtype, const void* d_x, const void* d_workspace, const double* d_uniforms, int64_t m,
                  int64_t* d_index, double* d_weight, qft_stream_t stream);
int qft_mc_bins(int n, int k, int direction, const int64_t* d_index, const double* d_weight, int64_t m,
                const int64_t* d_bins, int nbins, const void* d_workspace, double* d_out, qft_stream_t stream);

/* Diagnostics: write pass i of the plan as a flat integer record (tile bits,
 * register stages with their wires and lane maps, tile-index -> wire and
 * output-address maps, tile-coordinate segments, TMA box geometry, grid,
 * shared memory, buffers) into out[0..cap); returns the record length or a
 * negative error.  The record order is fixed by this library version and is
 * read by the test-suite's index checks; it is not a stable interface. */
int qft_plan_describe_pass(qft_plan_t plan, int i, long long* out, int cap);

/* ---------------------------------------------------------------- test hooks
 * For the test-suite's failure-reporting checks; not for normal use.  (The
 * other hook is qft_opts.test_skip_first_load.)
 *
 * The server's next `count` device allocations fail as if cudaMalloc had
 * failed.  A request that cannot get memory while others are running waits
 * for them; with nothing running it fails with QFT_ERR_NOMEM.  Used to check
 * that an allocation failure is reported and leaks nothing. */
int qft_server_inject_alloc_failures(qft_server_t server, int count);

/* Error description (static string). */
const char* qft_strerror(int code);
/* cudaError_t value behind the last QFT_ERR_CUDA returned on this thread. */
int qft_last_cuda_error(void);
/* Library version as major*10000 + minor*100 + patch. */
int qft_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QFTFFT_H */
