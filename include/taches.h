/*
 * taches.h -- C ABI of a GB300 (sm_103a) library for the taches-algorithm:
 * streaming, block-by-block time-domain convolution with an impulse response
 * (IR) that may change between input samples.
 *
 * Method: L. Millot and G. Pele, "An alternative approach for the convolution
 * in time-domain: the taches-algorithms", AES 125th Convention, 2008.
 *   - Every input sample x[n] spawns a "tache" x[n] * h[0..L-1] that is added
 *     to the output from sample n on (Sec. 3.2, Eq. 4):
 *         y[m] = sum_n x[n] * h_{v(n)}[m - n].
 *   - The IR used by sample n, h_{v(n)}, is the one in force when n arrived.
 *     Replacing the IR affects only later samples, even one sample apart
 *     (abstract and Sec. 6).
 *   - The input comes in blocks of Nb samples and each pushed block yields
 *     the output block of the same sample range at once (buffer algorithm,
 *     Sec. 4.2). A shorter last block is allowed.
 *   - The output is L-1 samples longer than the input. This "temporal
 *     overflow" (Sec. 4.1) is delivered by tc_flush.
 *
 * The GPU computes each output block as an output-side gather,
 *     y[t0+i] = sum_k h_{v(t0+i-k)}[k] * x[t0+i-k],
 * over the resident input history. This gives the same values as the
 * paper's scatter into a ring accumulator, up to float rounding.
 *
 * Conventions (all entry points):
 *   - Every call returns a tc_status. Nothing throws or aborts across the
 *     ABI. On error, tc_last_error() returns a message for the calling thread.
 *   - The library owns all device memory that it allocates. The caller owns
 *     the x, y and h buffers that it passes, and the library keeps no pointer
 *     to them after the call returns (device-pointer calls: after the
 *     enqueued work has run).
 *   - Samples are float32. A group with C channels takes x as [C][n] and
 *     returns y as [C][n], row-major with rows of exactly n floats.
 *   - Host-pointer calls are synchronous: they return once y holds the
 *     result. Page-locked host buffers (cudaHostAlloc, cudaHostRegister, a
 *     pinned torch tensor) are copied directly by the copy engines; pageable
 *     ones go through the stream's own pinned staging buffers. Device-pointer calls (the *_dev functions, or on_device = 1)
 *     enqueue work on the stream's CUDA stream and return at once.
 *   - Use one tc_stream from one thread at a time. Different tc_streams may
 *     be used from different threads.
 */
#ifndef TACHES_H
#define TACHES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_stream tc_stream; /* opaque, owned by the library */

typedef enum tc_status {
    TC_OK = 0,
    TC_EINVAL = 1,       /* bad argument: NULL pointer, zero size, n > max_push, IR longer than L, ... */
    TC_ENOMEM = 2,       /* device or pinned allocation failed, or every IR slot is still in use */
    TC_ESTATE = 3,       /* call not allowed now: push before any IR, push after the last (short) block or after flush */
    TC_ECUDA = 4,        /* a CUDA call or kernel launch failed; tc_last_error() has the CUDA message */
    TC_ETIMEOUT = 5,     /* a bounded device-side wait gave up; the results of that call are invalid */
    TC_EUNSUPPORTED = 6  /* the option is not available for this kind of stream */
} tc_status;

typedef enum tc_precision {
    TC_FP32 = 0,         /* FP32 FMA on CUDA cores (any stream kind) */
    TC_BF16 = 1,         /* BF16 tensor cores, FP32 accumulate (shared-IR groups and MIMO only) */
    TC_BF16_SPLIT = 2    /* BF16 hi/lo split of both operands, 3 tensor products, FP32 accumulate */
} tc_precision;

/* Describes a stream; filled by tc_get_info. */
typedef struct tc_info {
    size_t channels;     /* rows of x per push (MIMO: inputs) */
    size_t outputs;      /* rows of y per push (MIMO: outputs; otherwise = channels) */
    size_t L;            /* IR length (taps) */
    size_t block;        /* nominal block size Nb */
    size_t max_push;     /* largest n accepted by one push */
    uint64_t pushed;     /* input samples pushed so far, per channel */
    int shared_ir;       /* 1: one IR for every channel */
    int precision;       /* tc_precision */
    int state;           /* 0 open, 1 ended (short block pushed), 2 flushed */
    int max_versions;    /* IR versions that can be live at once, per IR set */
    uint64_t tensor_launches;  /* launches that ran on the tensor cores (BF16 modes) */
    uint64_t fp32_fallbacks;   /* BF16-mode launches that ran on the FP32 gather because
                                  their window straddled an IR switch */
} tc_info;

/* ---------------------------------------------------------------------- */
/* Opening and closing                                                     */
/* ---------------------------------------------------------------------- */

/* One mono stream, FP32, IR length L taps, block Nb = block samples: the
 * state that the buffer algorithm keeps from one block to the next (Sec. 4.2:
 * the residue ring r and its index), held here as the input history and the
 * IR versions. Allocates that state on the current CUDA device: the input
 * history, the IR slots and the scratch for the split tap sums.
 * Errors: TC_EINVAL if L == 0, block == 0 or out == NULL; TC_ENOMEM; TC_ECUDA. */
tc_status tc_open_stream(size_t L, size_t block, tc_stream **out);

/* One mono stream with a precision, on a device, with pushes of up to
 * max_push samples (0: block). device = -1: the current CUDA device;
 * otherwise the stream's memory and work are on that device (the calling
 * thread's current device is left as it was). precision TC_FP32 runs the
 * gather (K1); TC_BF16 and TC_BF16_SPLIT run the tensor-core contraction (K2)
 * with the output of a push cut into rows of 256 samples (K2's channels are
 * overlapping windows of the one input), falling back to K1 for windows that
 * straddle an IR switch. The tensor-core form is the matrix organisation that
 * Sec. 4.2 suggests for GPUs. Errors: as tc_open_group; TC_EINVAL for a bad
 * device or precision. */
tc_status tc_open_stream_ex(size_t L, size_t block, tc_precision precision, int device, size_t max_push,
                            tc_stream **out);

/* A group of `channels` streams pushed together: multichannel signals
 * (Sec. 6), each channel's data a row of a matrix (Sec. 4.2, the remark on
 * GPUs). With shared_ir = 1 all channels use one IR. The
 * BF16 modes then run on the tensor cores as a Toeplitz(h) x X contraction.
 * With shared_ir = 0 each channel has its own IR and its own IR versions
 * (FP32 only). max_push >= block is the largest n of one push. A push of
 * several blocks gives the same values as pushing them one at a time,
 * since Nb affects only timing (Sec. 5.2, Table 2). max_push = 0 means block.
 * Errors: TC_EINVAL (sizes 0, max_push < block); TC_EUNSUPPORTED (BF16
 * with per-channel IRs); TC_ENOMEM; TC_ECUDA. */
tc_status tc_open_group(size_t channels, size_t L, size_t block, int shared_ir,
                        tc_precision precision, size_t max_push, tc_stream **out);

/* nin inputs and nout outputs. Output o is sum_i h_{o,i} * x_i, each term
 * Eq. 4 with its own IR; the paper has no MIMO form beyond multichannel
 * signals (Sec. 6). The IR set is [nout][nin][L]. Pushes take x as [nin][n] and return y as [nout][n].
 * Errors as tc_open_group. */
tc_status tc_open_mimo(size_t nin, size_t nout, size_t L, size_t block,
                       tc_precision precision, size_t max_push, tc_stream **out);

/* Frees everything the stream owns (after its device work has finished),
 * then releases what the library's stream-ordered pool holds above 2 GiB on
 * the stream's device, so that the unmapping happens here and not at another
 * caller's next synchronisation. NULL is accepted. Library housekeeping, no
 * counterpart in the paper. */
tc_status tc_close(tc_stream *s);

/* Back to the state right after open: no IR, nothing pushed, the history
 * zeroed, as the buffer algorithm's initialisation of r and its index
 * (Sec. 4.2). Keeps all allocations. */
tc_status tc_reset(tc_stream *s);

/* Maximum number of IR versions live at once per IR set (default 4). A
 * version stays live while a future output still needs a sample that spawned
 * its tache with it (abstract, Sec. 6: taches keep the IR they were spawned
 * with), that is until L-1 samples after the next version
 * starts. Only allowed before the first tc_set_ir*. Reallocates the IR slots. */
tc_status tc_set_max_versions(tc_stream *s, int max_versions);

/* Use this CUDA stream (a cudaStream_t passed as void*; NULL = the library's
 * own stream) for all of this tc_stream's later device work. Library
 * plumbing, no counterpart in the paper. Errors: TC_EINVAL (s NULL). */
tc_status tc_set_cuda_stream(tc_stream *s, void *cuda_stream);

/* Fills *info (see tc_info). Errors: TC_EINVAL (NULL). */
tc_status tc_get_info(const tc_stream *s, tc_info *info);

/* ---------------------------------------------------------------------- */
/* IR versions (abstract, Sec. 6: update the IR "for next samples")        */
/* ---------------------------------------------------------------------- */

/* Sets the IR h[0..n-1], n <= L (zero-padded to L), for every channel. It
 * takes effect from the next input sample to be pushed (abstract: the IR is
 * updated for the next samples). Taches already
 * spawned keep their IR. h is a host pointer and is copied before the call
 * returns. Errors: TC_EINVAL (n == 0 or n > L, h NULL); TC_ENOMEM (no free
 * IR slot: too many versions still live); TC_ECUDA. */
tc_status tc_set_ir(tc_stream *s, const float *h, size_t n);

/* As tc_set_ir, but the IR is used from input sample index `sample` on (0 =
 * first sample of the stream). This gives the exact per-sample switch of
 * Sec. 6: the switch may fall inside a block. sample must be >= the number
 * of samples already pushed, and >= the start of the latest version. A
 * version set at the same sample replaces it. */
tc_status tc_set_ir_at(tc_stream *s, const float *h, size_t n, uint64_t sample);
/* Continuous time-varying IR (Sec. 6: the IR may also change progressively).
 * From this call on, each IR switch (tc_set_ir, tc_set_ir_at,
 * tc_set_ir_rows) at sample s is a crossfade over `ramp` samples: input
 * sample n spawns its tache with (1 - a) h_old + a h_new, where
 * a = clamp((n - s + 1) / ramp, 0, 1). ramp = 1 (the default, and after
 * tc_reset) is the hard switch. A switch may not start before the previous
 * crossfade has ended (TC_EINVAL). Windows that read a crossfade run on the
 * FP32 gather in every precision mode. Errors: TC_EINVAL for ramp outside
 * [1, 2^24]. */
tc_status tc_set_crossfade(tc_stream *s, size_t ramp);

/* One IR per IR set, all taking effect at `sample`. h is [sets][n]. sets is
 * 1 for a shared-IR group, channels for a per-channel group, and nout*nin
 * ([nout][nin][n]) for MIMO. h_on_device = 1: h is a device pointer; the copy
 * is enqueued on the stream and h must stay valid until it has run.
 * Errors as tc_set_ir_at. */
tc_status tc_set_ir_rows(tc_stream *s, const float *h, size_t n, uint64_t sample, int h_on_device);

/* ---------------------------------------------------------------------- */
/* Pushing input, receiving output (buffer algorithm, Sec. 4.2)            */
/* ---------------------------------------------------------------------- */

/* Pushes n <= block samples per channel (host x [channels][n]). Receives
 * the n output samples of the same sample range (host y [outputs][n]).
 * n < block marks the last block (Sec. 4.2, Nb <- min(Nb, size(pe))); only
 * tc_flush is allowed after it.
 * Errors: TC_EINVAL (NULL, n == 0, n > block); TC_ESTATE (no IR covers
 * the next sample, or stream ended); TC_ECUDA; TC_ETIMEOUT. */
tc_status tc_push_block(tc_stream *s, const float *x, size_t n, float *y);

/* As tc_push_block, for n <= max_push samples. n should be a multiple of
 * block; otherwise this is the last push. on_device:
 *   0 (TC_PUSH_HOST): host buffers, synchronous;
 *   1 (TC_PUSH_DEVICE): device pointers; the call enqueues the work on the
 *     stream's CUDA stream and returns without waiting (check with tc_sync);
 *   2 (TC_PUSH_PINNED_ASYNC): page-locked host buffers (TC_EINVAL otherwise);
 *     the call enqueues the copy of x to the device, the kernels and the copy
 *     of y back, and returns. The copies run on a second CUDA stream of the
 *     library through two device staging slots, so they overlap the kernels
 *     of the neighbouring pushes. x may be reused, and y read, after tc_sync
 *     or tc_flush. */
enum { TC_PUSH_HOST = 0, TC_PUSH_DEVICE = 1, TC_PUSH_PINNED_ASYNC = 2 };
tc_status tc_push(tc_stream *s, const float *x, size_t n, float *y, int on_device);

/* Temporal overflow (Sec. 4.1): the last L-1 output samples per output row,
 * as if L-1 zeros were pushed. Host y holds [outputs][cap], and row o gets
 * min(cap, L-1) samples. *n_out (optional) receives L-1. After this, only
 * tc_reset or tc_close is allowed.
 * Errors: TC_EINVAL (y NULL, cap < L-1); TC_ESTATE (already flushed). */
tc_status tc_flush(tc_stream *s, float *y, size_t cap, size_t *n_out);

/* Device version of tc_flush (Sec. 4.1, temporal overflow): y is a device
 * [outputs][L-1] buffer. Asynchronous. Errors as tc_flush. */
tc_status tc_flush_dev(tc_stream *s, float *y, size_t *n_out);

/* Waits for the stream's enqueued device work (library plumbing, no
 * counterpart in the paper). Returns TC_ETIMEOUT if a kernel reported a
 * bounded-wait failure, TC_ECUDA on a CUDA error. */
tc_status tc_sync(tc_stream *s);

/* ---------------------------------------------------------------------- */
/* Checkpoint / resume                                                     */
/* ---------------------------------------------------------------------- */

/* Checkpoint (no counterpart in the paper; what is saved is the state the
 * buffer algorithm carries between blocks, Sec. 4.2). Copies everything the
 * stream's future outputs depend on into a host blob:
 * shape, position and state, the live IR versions (start sample, crossfade
 * length, IR rows) and the input history from the stream's current base, plus
 * the tuning knobs. buf NULL: only *size is set (bytes needed). Waits for the
 * stream's device work. Errors: TC_EINVAL (NULL size, cap < needed). */
tc_status tc_stream_export(tc_stream *s, void *buf, size_t cap, size_t *size);
/* Restores a blob of tc_stream_export into s, which must have the same kind,
 * precision, channel counts, L, block and max_push (TC_EINVAL otherwise, or
 * for a blob that is not one). s's previous state is discarded. Pushes after
 * the import give the same bits as the exported stream would have: the
 * history keeps its layout, so the kernels split the taps the same way.
 * Waits for the copies. */
tc_status tc_stream_import(tc_stream *s, const void *buf, size_t size);

/* ---------------------------------------------------------------------- */
/* One-shot convolution (off-line use, Sec. 3.2)                           */
/* ---------------------------------------------------------------------- */

/* y[0..N+L-2] = x[0..N-1] * h[0..L-1], all device pointers, FP32. When
 * N < L the operands swap roles (Sec. 3.2: x * h = h * x; the gather's work is
 * (N + L - 1) L), unless TC_NO_ROLE_SWAP=1 is set in the environment. Runs on
 * cuda_stream (a cudaStream_t as void*; NULL = default stream) and waits
 * for it before returning. Its working memory (the input with zero margins,
 * about N + 6 L floats, and up to 256 MiB of split-sum partials) comes from
 * the library's stream-ordered memory pool on cuda_stream and goes back to it
 * before return; the pool keeps up to 2 GiB of freed memory mapped for the
 * next calls. Errors: TC_EINVAL (NULL or zero sizes, L > 2^30); TC_ENOMEM;
 * TC_ECUDA; TC_ETIMEOUT. */
tc_status tc_convolve(const float *x, size_t N, const float *h, size_t L, float *y, void *cuda_stream);

/* ---------------------------------------------------------------------- */
/* One-shot convolution without allocation                                 */
/* ---------------------------------------------------------------------- */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory where they call: a real-time audio callback
 * (cudaMalloc may block for an unbounded time and miss the block deadline),
 * or a host program whose own allocator owns the GPU's memory.
 *
 * Same result as tc_convolve, y[0..N+L-2] = x[0..N-1] * h[0..L-1] (device
 * pointers, FP32, the same role swap), but it calls no cudaMalloc, cudaFree or allocating
 * routine. Its working memory (input history with zero margins, shifted IR
 * copies, split-sum partials, counters) lives in one fixed 32 MiB device
 * array inside this library. Each GPU that loads the library holds that array
 * until the process exits.
 *   - Limit: the working set, about N + 13 L + 5e4 floats (N >= L after the
 *     role swap), must fit in
 *     32 MiB = 8388608 floats: for example N up to 8.2 million samples with
 *     L = 4096. A call beyond it returns TC_EINVAL and names the size it
 *     would need.
 *     N or L above 8388608 is rejected the same way before any other work.
 *   - The first call on a device looks up the array's device address with
 *     that device current. Make that first call before any CUDA stream
 *     capture. The address is kept for the life of the process: do not use
 *     the library across cudaDeviceReset.
 *   - Every call uses the same array and clears what must start at zero.
 *     Calls that overlap on the GPU (different streams, or threads without
 *     ordering) race and give wrong results, so serialise them.
 * Runs on cuda_stream (NULL = default stream) and waits for it before
 * returning. Errors: TC_EINVAL (NULL, zero or too large sizes); TC_ECUDA;
 * TC_ETIMEOUT. */
tc_status tc_convolve_noalloc(const float *x, size_t N, const float *h, size_t L, float *y, void *cuda_stream);

/* ---------------------------------------------------------------------- */
/* One signal on the tensor cores                                          */
/* ---------------------------------------------------------------------- */

/* y[0..N+L-2] = x[0..N-1] * h[0..L-1] (device pointers, FP32 in and out) with
 * the products on the tcgen05 tensor cores: the output is cut into rows of
 * 256 samples, and every row is a channel of the shared-IR contraction (K2),
 * whose histories are overlapping windows of the one input. precision:
 * TC_BF16 (BF16 operands, FP32 accumulation; about 2e-3 relative L2),
 * TC_BF16_SPLIT (hi/lo BF16 split of both operands, three products; about
 * 5e-6) or TC_FP32 (the same as tc_convolve). The shorter operand takes the
 * IR role (Sec. 3.2) unless TC_NO_ROLE_SWAP=1. The rows are written straight
 * into y (the last one stops at y's end). Working memory (the padded input as
 * BF16 hi and, for the split, lo; the IR's Toeplitz tiles; K-part partials and
 * their tickets) comes from the library's stream-ordered pool. Runs on
 * cuda_stream and waits for it. Errors: TC_EINVAL (NULL, zero sizes, unknown
 * precision, L > 2^26); TC_ENOMEM; TC_ECUDA; TC_ETIMEOUT. */
tc_status tc_convolve_tc(const float *x, size_t N, const float *h, size_t L, float *y, int precision,
                         void *cuda_stream);

/* ---------------------------------------------------------------------- */
/* Exact fixed-point convolution with one requantization (Sec. 5.4)      */
/* ---------------------------------------------------------------------- */

/* Q15 input and taps (int16, value = code / 2^15). Every product is summed
 * exactly, and each output sample is requantized once to Q15, after all of its
 * products are in (the ideal requantization of Sec. 5.4):
 *   acc[m] = sum_k x[m-k] h[k]                       (int64, Q30, exact)
 *   y[m]   = clamp(round_half_even(acc[m] / 2^15), -32768, 32767)
 * for m in [0, N+L-1). The result is bit-exact and independent of how the GPU
 * splits the work.
 *   - x: N codes; h: L codes; y: N+L-1 codes; acc: N+L-1 int64. All device
 *     pointers, owned by the caller. y or acc may be NULL (not both): NULL acc
 *     uses a temporary from the stream-ordered allocator; NULL y skips the
 *     requantization.
 *   - L <= 2^19 keeps |acc| < 2^49, far inside int64. When N < L the operands
 *     swap roles (Sec. 3.2) unless TC_NO_ROLE_SWAP=1; the result is bit-identical.
 *   - TC_Q15_INNER=imad in the environment selects the widening-multiply form
 *     of the kernel instead of the default dp2a form (same result).
 * Runs on cuda_stream (NULL = default stream) and waits for it before
 * returning. Errors: TC_EINVAL (NULL pointers, N == 0, L == 0 or L > 2^19);
 * TC_ENOMEM; TC_ECUDA. */
tc_status tc_convolve_q15(const int16_t *x, size_t N, const int16_t *h, size_t L, int16_t *y, int64_t *acc,
                          void *cuda_stream);

/* ---------------------------------------------------------------------- */
/* Failure detection check (library tooling; no counterpart in the paper)  */
/* ---------------------------------------------------------------------- */

/* Every device-side wait of the kernels is bounded (by %globaltimer and a
 * poll count); when a bound is reached the kernel reports into its error word
 * and returns, and the call returns TC_ETIMEOUT. This runs one kernel whose
 * wait (on an mbarrier that nothing completes) must run out after limit_ns
 * nanoseconds (1 <= limit_ns <= 1e10). Returns TC_ETIMEOUT, the expected
 * result, after about limit_ns; the CUDA context stays usable. TC_EINVAL for
 * a bad limit; TC_ECUDA if the wait did not report. Runs on cuda_stream
 * (NULL = default stream) and waits for it. */
tc_status tc_selftest_wait(unsigned long long limit_ns, void *cuda_stream);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of many independent streams               */
/* ---------------------------------------------------------------------- */
/*
 * A tc_server holds many mono FP32 streams on one device. Each has its own IR
 * length L, block size Nb and IR versions. Real time is Sec. 5.1's criterion
 * (the convolution computes faster than the stimulus plays), here per block:
 * its output is due one block period after its last input sample. Many
 * streams at once extend the multichannel outlook of Sec. 6; batching them is
 * this library's, not the paper's. The streams' blocks run in batches:
 *   - tc_server_submit queues one input block and returns at once. It never
 *     waits for the GPU.
 *   - A step takes the oldest pending block of every stream that has one. It
 *     runs all of them as ONE batch: one host-to-device copy, one scatter
 *     kernel into the streams' histories, one FP32 gather launch over a work
 *     list with one item per stream, and one device-to-host copy.
 *   - Blocks submitted while a step runs join the next step. The worker
 *     thread started by tc_server_start runs steps back to back while blocks
 *     are pending. tc_server_step runs one step on the calling thread
 *     instead.
 *   - A stream is admitted only while its device state (input history, IR
 *     slots, version table) fits the memory budget. Otherwise tc_server_add
 *     returns TC_ENOMEM and the caller retries once streams have left.
 *     tc_server_remove releases the state.
 *   - A group (tc_server_add_group) is C channels that share one IR: a
 *     multichannel source through one room response (multichannel signals,
 *     Sec. 6). Its blocks are [C][n]; each step runs them as one push of a
 *     shared-IR group stream on the group's own CUDA stream, beside the
 *     step's gather launch and ordered by events: K2 on the tensor cores in
 *     TC_BF16 and TC_BF16_SPLIT, the gather in TC_FP32.
 * Each stream gives the same output as a tc_stream opened with the same L and
 * block and fed the same calls (a group: as tc_open_group with shared_ir = 1
 * and the same precision). The output does not depend on which blocks of
 * other streams share its steps, up to FP32 rounding (BF16 modes: up to the
 * rounding of their products).
 * Thread safety: submit, poll and get_stats may be called from any thread at
 * any time. The other calls serialise on the server.
 */
typedef struct tc_server tc_server;

typedef struct tc_server_stats {
    size_t streams;      /* streams admitted and not removed */
    size_t mem_used;     /* device bytes held by those streams */
    size_t mem_budget;   /* budget given to tc_server_open */
    uint64_t steps;      /* batched steps run */
    uint64_t blocks;     /* blocks completed (flush tails included) */
    uint64_t rejected;   /* tc_server_add calls refused for memory */
    double busy_s;       /* wall time spent inside steps (seconds) */
    double tap_macs;     /* useful work done: input samples x L (x channels for a group), summed over
                            finished blocks (flush tails excluded) */
    uint64_t tensor_launches;  /* group pushes that ran on the tensor cores (BF16 modes) */
    uint64_t fp32_fallbacks;   /* BF16-mode group pushes that ran on the FP32 gather because their
                                  window straddled an IR switch */
    double k1_ms;        /* device time of the steps' K1 work-list launches (CUDA events, ms) */
    double k1_macs;      /* tap-MACs those launches computed (inputs x L, flush tails included) */
    uint64_t pool_admissions;  /* tc_server_add admissions whose state did not fit tc_server_reserve's
                                  reservation (allocated from the pool) */
    uint64_t grows;      /* growths of the steps' own buffers (allocations made inside a step) */
    double host_collect_s;  /* worker thread host time: taking queued blocks into steps (seconds) */
    double host_pack_s;     /* packing inputs and work items, enqueueing copies and kernels */
    double host_deliver_s;  /* delivering finished steps (outputs, latencies, positions) */
} tc_server_stats;

/* Opens a server on the current CUDA device. mem_budget_bytes bounds the
 * device memory of admitted streams. max_step_samples bounds the input
 * samples of one step (0: 4M). It sizes the pinned staging buffers; a block
 * that would overflow a step waits for the next one. */
tc_status tc_server_open(size_t mem_budget_bytes, size_t max_step_samples, tc_server **out);
/* Stops the worker, waits for the GPU and frees everything (trimming the
 * library's pool as tc_close does). NULL is a no-op. */
tc_status tc_server_close(tc_server *srv);
/* Reserves min(bytes, budget) bytes of device memory for the states of
 * later tc_server_add admissions: one allocation made now, carved up by the
 * server (first fit; a removed stream's range is reused once the steps that
 * read it have completed). Without it each admission allocates from the
 * server's memory pool, which maps new device memory when it has to grow, and
 * mapping memory while steps run stalled them: measured on the serving trace,
 * steps of about 1 ms (against 0.1 ms), and once 65 ms, coincided with
 * admissions. Admissions that do not fit the reservation still fall back to
 * the pool. Call it once, before serving; the memory stays with the server
 * until tc_server_close. Groups (tc_server_add_group) do not use it. The paper
 * has no counterpart (serving). Errors: TC_EINVAL (NULL); TC_ESTATE (called
 * before); TC_ENOMEM (the device has no room); TC_ECUDA. */
tc_status tc_server_reserve(tc_server *srv, size_t bytes);

/* Admits a stream with IR length L (1 <= L <= 2620792) and block size block,
 * with initial IR h[0..n) (n <= L; shorter IRs are zero-padded). *id names
 * the stream in later calls. flags: 0, or TC_SERVER_DISCARD_OUTPUT to keep no
 * output blocks (load generation: only the latency is recorded). TC_ENOMEM:
 * the budget (or the device) has no room now. */
enum { TC_SERVER_DISCARD_OUTPUT = 1 };
tc_status tc_server_add(tc_server *srv, size_t L, size_t block, const float *h, size_t n, int flags,
                        uint64_t *id);
/* Admits a group of `channels` rows sharing one IR (1 <= channels <= 4096,
 * channels x block <= max_step_samples), precision TC_FP32, TC_BF16 or
 * TC_BF16_SPLIT. Every call that takes or returns samples of a group uses
 * [channels][n] row-major buffers: submit (x holds channels x n floats),
 * attach_source (x is [channels][n]), poll (*n_out counts floats, channels x
 * the block's samples) and flush (channels x (L - 1) floats). IR switches
 * (tc_server_set_ir_at) apply to every channel; up to four versions are live.
 * Errors as tc_server_add; TC_EINVAL for a bad channel count or precision. */
tc_status tc_server_add_group(tc_server *srv, size_t channels, size_t L, size_t block, const float *h, size_t n,
                              int precision, int flags, uint64_t *id);
/* New IR version from input sample `sample` on (Eq. 4 with per-sample
 * versions, Sec. 6). sample must not be below the samples already submitted.
 * Up to three versions are live per stream; TC_ENOMEM when all three are
 * still needed by the input history. */
tc_status tc_server_set_ir_at(tc_server *srv, uint64_t id, const float *h, size_t n, uint64_t sample);
/* Queues input block x[0..n) (n <= block; a shorter block is the stream's
 * last). The library copies x before returning. The block's latency is
 * counted from the call. */
tc_status tc_server_submit(tc_server *srv, uint64_t id, const float *x, size_t n);
/* Queues count blocks at once (block i: stream ids[i], xs[i][0..ns[i])), in
 * order. t_ready[i] (t_ready may be NULL: now) is the time on
 * tc_server_clock() at which block i was complete; its latency is counted
 * from there. Checks every block first and queues none on an error. */
tc_status tc_server_submit_many(tc_server *srv, size_t count, const uint64_t *ids, const float *const *xs,
                                const size_t *ns, const double *t_ready);
/* Live input: the stream's next input is x[0..n), after any input already
 * submitted. It arrives at fs samples per second from time t0 on
 * tc_server_clock(), as from a capture device. Block b (b = 0, 1, ...) is
 * queued at its ready time t0 + min((b + 1) * block, n) / fs and its latency
 * counts from there; the last block may be short, and the input ends with
 * it. The library reads x in place when the block runs: the caller keeps x
 * alive and unchanged until the stream is removed. TC_ESTATE if the stream
 * already has a source, has blocks queued or its input has ended;
 * tc_server_submit is refused on the stream afterwards. */
tc_status tc_server_attach_source(tc_server *srv, uint64_t id, const float *x, size_t n, double t0, double fs);
/* *state: 0 input still open, 1 input ended with blocks still queued or
 * running, 2 drained (every block done: ready for flush or remove). */
tc_status tc_server_stream_state(tc_server *srv, uint64_t id, int *state);
/* Runs one batched step on the calling thread (TC_ESTATE while the worker
 * runs). *blocks_done (may be NULL) is the number of blocks it completed. */
tc_status tc_server_step(tc_server *srv, size_t *blocks_done);
/* Starts / stops the worker thread. tc_server_stop returns TC_ECUDA if the
 * worker stopped on an error; tc_last_error() then has its message. */
tc_status tc_server_start(tc_server *srv);
tc_status tc_server_stop(tc_server *srv);
/* Takes the stream's oldest finished output block, if any. *n_out = 0 if
 * none is ready yet. The block has as many samples as its input block and
 * goes to y[0..n) (cap >= n, else TC_EINVAL; a group's block is [channels][n]
 * and *n_out = channels x n). t_submit and t_done (may be
 * NULL) get the submit and completion times on tc_server_clock(). */
tc_status tc_server_poll(tc_server *srv, uint64_t id, float *y, size_t cap, size_t *n_out, double *t_submit,
                         double *t_done);
/* Ends the stream's input and returns the last L - 1 output samples (the
 * temporal overflow of Sec. 4.1) in y[0..L-1) (cap >= L - 1; a group:
 * [channels][L - 1], cap >= channels x (L - 1)). Runs steps on
 * the calling thread until they are done; stop the worker first
 * (TC_ESTATE otherwise). Poll the stream's finished blocks before or after. */
tc_status tc_server_flush(tc_server *srv, uint64_t id, float *y, size_t cap, size_t *n_out);
/* Removes the stream and frees its device state. TC_ESTATE while blocks of
 * the stream are still queued (its finished, unpolled outputs are dropped). */
tc_status tc_server_remove(tc_server *srv, uint64_t id);
/* Fills *st (see tc_server_stats). Errors: TC_EINVAL (NULL). */
tc_status tc_server_get_stats(tc_server *srv, tc_server_stats *st);
/* Moves up to cap recorded block latencies (seconds from ready to result on
 * the host, in completion order) into out, and the nominal block size of each
 * block's stream into block (may be NULL), then forgets them. Flush tails are
 * not recorded. */
tc_status tc_server_latencies(tc_server *srv, double *out, uint32_t *block, size_t cap, size_t *n_out);
/* As tc_server_latencies, and if parts is not NULL it also receives, per
 * block, three floats (seconds) that add up to its latency: ready -> taken
 * into a step by the worker, taken -> the step's copies and kernels enqueued,
 * enqueued -> results on the host. parts holds 3 * cap floats, kind cap bytes
 * (both caller-owned, may be NULL). kind[i] tags block i's stream: 0 a plain
 * stream (FP32 gather), 1 + precision (TC_FP32, TC_BF16, TC_BF16_SPLIT) a
 * group. The paper has no counterpart (tracing of the serving loop). */
tc_status tc_server_latencies_ex(tc_server *srv, double *out, uint32_t *block, float *parts, uint8_t *kind,
                                 size_t cap, size_t *n_out);
/* Monotonic clock of the poll timestamps (seconds). */
double tc_server_clock(void);
/* Options (value 0 or 1), set at any time:
 *   TC_SERVER_AUTOTUNE  (default 1) pick the gather's tap chunk per step class
 *                       (magnitudes of the step's work and longest IR) by
 *                       measured time: each chunk is tried twice per class,
 *                       then the fastest is used; 0 = fixed rule (largest
 *                       chunk with >= 4 waves and < 10 % padding).
 *   TC_SERVER_GRAPH     (default 0) replay each step as one CUDA graph
 *                       (copies, ingest, gather and its timing events) whose
 *                       node parameters are updated per step, instead of
 *                       separate stream operations. */
enum { TC_SERVER_AUTOTUNE = 0, TC_SERVER_GRAPH = 1 };
tc_status tc_server_set_option(tc_server *srv, int option, int value);
/* Step log (tracing): one record per step, the last 65536 steps kept. */
typedef struct tc_server_step_rec {
    double t_begin;      /* step start (tc_server_clock) */
    double t_launch;     /* host packing done, copies and kernels enqueued from here */
    double t_done;       /* results on the host */
    uint32_t blocks;     /* blocks in the step */
    uint32_t samples;    /* input samples in the step */
    uint32_t ctas;       /* CTAs of the gather launch */
    uint32_t variant;    /* tap chunk of the gather: 0 = 640, 1 = 2560, 2 = 7040 taps */
} tc_server_step_rec;
/* Moves the newest min(cap, logged) records (oldest first) into out and
 * clears the log. */
tc_status tc_server_step_log(tc_server *srv, tc_server_step_rec *out, size_t cap, size_t *n_out);

/* ---------------------------------------------------------------------- */
/* Diagnostics (library tooling; no counterpart in the paper)              */
/* ---------------------------------------------------------------------- */

/* Message of the calling thread's last failed call ("" if none). Valid until
 * that thread's next call into the library. */
const char *tc_last_error(void);

/* Static name of a status code. */
const char *tc_status_str(tc_status st);

/* Number of kernel launches this library has issued in this process. Counts
 * every launch, on every stream. */
uint64_t tc_kernel_launches(void);

/* Tuning knobs (autotuner and experiments); value -1 restores the default.
 *   TC_TUNE_K1_CHUNK     tap chunk of the FP32 gather: 0 = 640, 1 = 2560,
 *                        2 = 7040 taps per CTA (default: picked per launch)
 *   TC_TUNE_K2_RANGE     K blocks (of 32 samples in the BF16 split, of 64 in
 *                        plain BF16) accumulated serially on the
 *                        tensor cores before the pairwise reduction of
 *                        ranges (default 16 for the BF16 split, 4096 for
 *                        BF16; 1..4096; rounded up to an even count for
 *                        the split; MIMO streams: K blocks of 32, rounded
 *                        up to a multiple of 8)
 *   TC_TUNE_K2_PAIR      2 = pairs of CTAs on two SMs (tcgen05
 *                        cta_group::2) per 256 channels x 256 outputs, each
 *                        SM staging half the operands, persistent (one pair
 *                        per two SMs walks the units; default; a group of
 *                        at most 128 channels pairs two adjacent output
 *                        tiles instead, and the BF16 split takes the pairs
 *                        when it has two tiles of either kind, else one tile
 *                        per CTA); plain BF16 only: 3 = the
 *                        same pairs launched one per unit; 1 = two
 *                        128-channel tiles per CTA sharing each IR tile;
 *                        0 = one tile per CTA (the split: any value but 2)
 *   TC_TUNE_K2_SPLIT     K parts per tensor-core output tile, each a
 *                        contiguous range of the IR's K blocks on its own CTA
 *                        (or CTA pair), added by a fixed pairwise tree
 *                        (1..64, capped at the tile's K blocks; default:
 *                        the fewest parts that fill the GPU's waves to 90 %)
 *   TC_TUNE_K2_FOLD      1 = the K parts of a tile are added inside the
 *                        tensor-core kernel, by the warp that stores the last
 *                        part of its slice (default; up to 16 parts, on the
 *                        persistent CTA pairs and the one-tile kernel);
 *                        0 = by a separate reduction launch. Both add the
 *                        parts by the same tree: the results are identical
 *   TC_TUNE_K2_ORDER     order in which the persistent CTA pairs take their
 *                        units (channel tile pair, output tile, K part):
 *                        0 = K part fastest, then output tile; 1 = output
 *                        tile fastest, then K part; 2 = output tile, then
 *                        channel tile, K part slowest (default: the pairs
 *                        running at a time share one K range of the IR
 *                        tiles in L2). Changes no result bit
 *   TC_TUNE_ZERO_SKIP    1 = zero gating on the FP32 gather (the zero-skip of
 *                        Sec. 3.2 and 4.2 at block level, threshold 0): a
 *                        staged stretch of input that is all zero skips its
 *                        taps. Exact (the skipped products are zeros); saves
 *                        time on silent input. 0 / -1 = off (default).
 * Errors: TC_EINVAL for an unknown knob or value out of range. */
typedef enum tc_tune_knob {
    TC_TUNE_K1_CHUNK = 0,
    TC_TUNE_K2_RANGE = 1,
    TC_TUNE_K2_PAIR = 2,
    TC_TUNE_ZERO_SKIP = 3,
    TC_TUNE_K2_SPLIT = 4,
    TC_TUNE_K2_FOLD = 5,
    TC_TUNE_K2_ORDER = 6
} tc_tune_knob;
tc_status tc_set_tuning(tc_stream *s, int knob, long long value);

/* TC_CHECK_LAUNCH=1 in the environment (read at each launch): before every
 * FP32-gather launch of a tc_stream, the host checks the ranges the kernel
 * will touch (staged input windows 16-byte aligned and inside the history
 * rows, tap chunks inside the IR slot, version slots, scratch) and returns
 * TC_EINVAL with the offending range instead of launching. Off by default. */

/* Test hook: host-side failure injection. With nth > 0, the nth next time
 * the library reaches `site` it reports a failure there instead of making the
 * call (no CUDA call fails and no GPU fault is made); nth = 0 disarms.
 *   TC_INJECT_PUSH_COPY    a push's input copy (tc_push_block, tc_push): the
 *                          push returns TC_ECUDA before the stream's position
 *                          moves, so the same push may be retried.
 *   TC_INJECT_SERVER_STEP  a server step's launch: tc_server_step returns
 *                          TC_ECUDA; the worker thread stops, and
 *                          tc_server_stop returns TC_ECUDA. The step's blocks
 *                          are dropped and their streams can be removed.
 * Errors: TC_EINVAL for an unknown site or nth < 0. */
enum { TC_INJECT_PUSH_COPY = 1, TC_INJECT_SERVER_STEP = 2 };
tc_status tc_test_inject(int site, int nth);

/* Kernel timing (tracing aid). With enable = 1, each later convolution kernel
 * launch of this stream is bracketed by CUDA events on the stream that runs
 * it. tc_profile_read waits for the stream, then returns the summed event
 * time in ms, the number of timed launches and the useful multiply-adds they
 * did. The useful multiply-adds count one per (output sample, in-range tap,
 * input row). It then clears the totals. Timing adds a little overhead per
 * launch. */
tc_status tc_profile(tc_stream *s, int enable);
tc_status tc_profile_read(tc_stream *s, double *ms, uint64_t *launches, double *useful_macs);

#ifdef __cplusplus
}
#endif

#endif /* TACHES_H */
