/*
 * fnt.h -- C ABI of libfnt: Fermat-number-transform chromatic dispersion
 * compensation (FNT-CDC) and adaptive equalisation (FNT-AEQ) on one GB300 GPU.
 *
 * Method: S. Chen et al., "Fermat Number Transform Based Chromatic Dispersion
 * Compensation and Adaptive Equalization Algorithm", arXiv 2405.04253.
 *   eq. (1)/(2)  length-N transform pair over Z_F, F = 2^16 + 1
 *   eq. (3)/(4)  conditions on F and the radix alpha
 *   eq. (5)      overflow constraint that makes the integer result exact
 *   eq. (6)      RDE tap update of the 4x4 real-valued MIMO equaliser
 *   eq. (7)/(8)  complex convolution from two real products
 *   CDC: F = 65537, alpha = sqrt(2) (= 4080), N = 64, 5-bit signal, 6-bit taps
 *   AEQ: F = 65537, alpha = 2, N = 32, 5-bit signal, 14-bit taps in two 7-bit groups
 *
 * Conventions for every call:
 *   - Nothing throws.  Every call returns an fnt_status; fnt_last_error() gives
 *     the detail text of the last failure on the calling thread.
 *   - Sample buffers are int8 / int16 arrays owned by the caller.  Unless a call
 *     says otherwise they are DEVICE pointers on the current CUDA device.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that take a stream only enqueue work on it and return; results are
 *     ready when the stream reaches that point.
 *   - Host arrays passed in (frame tables, taps, tap state) are read before the
 *     call returns and may be reused right after.
 *   - All results are bit-exact integers: the same on every run and every launch
 *     shape.
 */
#ifndef FNT_H
#define FNT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FNT_API __attribute__((visibility("default")))
#else
#define FNT_API
#endif

typedef enum fnt_status {
    FNT_OK = 0,
    FNT_ERR_INVALID = 1,   /* bad argument, shape or pointer */
    FNT_ERR_BOUND = 2,     /* parameters violate eq. (4) or constraint (5) */
    FNT_ERR_NOMEM = 3,     /* device or host allocation failed */
    FNT_ERR_BUSY = 4,      /* session admission refused: memory cap or slots full */
    FNT_ERR_TIMEOUT = 5,   /* poll timed out with nothing completed */
    FNT_ERR_CUDA = 6,      /* a CUDA runtime call failed (detail in fnt_last_error) */
    FNT_ERR_NOT_FOUND = 7, /* unknown link or ticket */
    FNT_ERR_CANCELLED = 8  /* the request was cancelled before it was launched */
} fnt_status;

/* Copies the calling thread's last error text into buf (always NUL-terminated).
 * Returns the full length of the message. */
FNT_API size_t fnt_last_error(char *buf, size_t len);

/* Library version, e.g. "fnt 1.0 sm_103a". */
FNT_API const char *fnt_version(void);

/* ------------------------------------------------------------------ plan ---- */

/*
 * Parameters of one CDC -> resample -> AEQ configuration.
 *
 * n_cdc, alpha_cdc   CDC transform length and radix.  Supported: 64 with 4080
 *                    (sqrt 2 mod 65537, section "Proposed FNT-CDC&AEQ structure").
 * cdc_step           overlap-save step S (new samples per 64-sample block).
 *                    0 = N - L + 1 for each frame's tap count L.  Must satisfy
 *                    32 <= S <= N - L + 1 for every frame (the zero padding that
 *                    turns circular into linear convolution, text after eq. (5)).
 * n_aeq, alpha_aeq   AEQ transform length and radix: 32 with 2 (the paper's AEQ)
 *                    or 64 with 4080.
 * aeq_taps           K, taps per real filter of the 4x4 MIMO: must be 16.
 *                    The AEQ step is n_aeq - K symbols per block.
 * mu_shift           m: the update of eq. (6) is applied as floor(G / 2^m);
 *                    0 <= m <= 62, or 63 for mu = 0 (taps held fixed).
 * rde_a              A: the 16QAM ring radii of the RDE error are sqrt(2, 10, 18) A,
 *                    1 <= A <= 4096.
 * tap_init           w0: initial taps are w0 (Q1.13) at centre tap K/2 of the four
 *                    diagonal filters XI->XI, XQ->XQ, YI->YI, YQ->YQ, 0 elsewhere.
 * aeq_segment        symbols per AEQ segment for long streams; 0 = one serial run
 *                    per frame.  With segments, output segment s covers symbols
 *                    [s*seg, (s+1)*seg) and its AEQ run starts aeq_warmup symbols
 *                    earlier (not before 0) from the frame's initial taps (its
 *                    state, or the plan's taps), reading the K = 16 symbols of
 *                    the frame before its start as input history (zero before
 *                    the frame); only the segment's own outputs are kept.  With
 *                    fixed taps the segments reproduce the serial outputs
 *                    exactly.  Segments run in parallel.
 * aeq_warmup         symbols of adaptation each segment runs before its own
 *                    outputs (ignored without segments; 0 is allowed).
 * aeq_update_period  P, AEQ blocks per tap update, 0..64 (0 and 1: every block,
 *                    the paper's eq. (6) schedule).  For P > 1 the gradient G of
 *                    eq. (6) is summed over P blocks of a run (a frame, or a
 *                    segment counted from its warm-up start) and applied as
 *                    floor(sum / 2^m) after every P-th block and after the
 *                    run's last block; the taps are fixed in between.
 * aeq_freq_sum       0 (default): one inverse FNT per (input, output, tap
 *                    group), exact for every input (constraint (5) holds per
 *                    pair).  1: the four inputs' products are summed in Z_F
 *                    before one inverse FNT per (output, group); outputs are
 *                    the centred residues of the summed convolutions, which
 *                    wrap where a sum leaves [-32768, 32768].  2: summed only
 *                    for a block and polarisation where 16 times the sum of
 *                    |tap group values| over the inputs is at most 32767 (so
 *                    no output wraps), per pair otherwise: results equal 0's.
 */
typedef struct fnt_plan_desc {
    int32_t n_cdc;
    int32_t alpha_cdc;
    int32_t cdc_step;
    int32_t n_aeq;
    int32_t alpha_aeq;
    int32_t aeq_taps;
    int32_t mu_shift;
    int32_t rde_a;
    int32_t tap_init;
    int32_t aeq_update_period;
    int64_t aeq_segment;
    int64_t aeq_warmup;
    int32_t aeq_freq_sum;
    int32_t reserved;
} fnt_plan_desc;

/* Fills *desc with the defaults: N=64/4080, S = N-L+1, AEQ N=32/2, K=16, m=10,
 * A=64, w0=2048, no segments, an update every block. */
FNT_API void fnt_plan_desc_default(fnt_plan_desc *desc);

typedef struct fnt_plan fnt_plan;

/* Validates desc (eq. (4): alpha^N = 1 with order exactly N, N invertible mod F;
 * supported (N, alpha) pairs; ranges above) and creates a plan on the current
 * device.  A plan holds no per-call state and may be used from several threads
 * and streams at once; calls with it must be made with its device current
 * (FNT_ERR_INVALID otherwise).  The one-shot calls take their work memory (tables and
 * intermediate buffers) from a memory pool of the plan that keeps up to 1 GiB
 * mapped between calls.  Errors: FNT_ERR_INVALID, FNT_ERR_BOUND,
 * FNT_ERR_NOMEM, FNT_ERR_CUDA. */
FNT_API fnt_status fnt_plan_create(const fnt_plan_desc *desc, fnt_plan **out);
/* Waits for the device, then frees the plan and its memory pool. */
FNT_API fnt_status fnt_plan_destroy(fnt_plan *plan);

/* Multiplication counts of the kernels for a plan description (no device
 * needed), in the units of Tab. 1
 * (real multiplications per symbol; twiddle products by powers of the radix
 * are not counted, as in the paper, since they are shifts in its hardware).
 *   cdc_mults_per_symbol  pointwise products of the CDC per symbol and
 *                         polarisation, for a frame with cd_len taps
 *                         (2 N per block, S / 2 symbols per block at 2 sps)
 *   aeq_mults_per_symbol  pointwise products of the 4x4 AEQ per symbol
 *                         (32 N_aeq per block of N_aeq - 16 symbols) on the
 *                         warp-per-chain kernel
 *   aeq_cta_mults_per_symbol  the same on the CTA-per-chain kernel
 * The products are counted from the kernels' own product stages: the library
 * runs the templates those kernels execute, on the host, with an arithmetic
 * policy that counts instead of computing; power-of-two multiplications
 * (eq. (8)'s -2^8) count as shifts.  At the operating point of Tab. 1 (CDC
 * N = 64 with 50 % overlap, i.e. cdc_step = 32; AEQ N = 32) these are 8, 64
 * and 64. */
typedef struct fnt_op_counts {
    double cdc_mults_per_symbol;
    double aeq_mults_per_symbol;
    double cdc_butterflies_per_symbol;
    double aeq_cta_mults_per_symbol;
} fnt_op_counts;

FNT_API fnt_status fnt_op_counts_for(const fnt_plan_desc *desc, int32_t cd_len, fnt_op_counts *out);

/* ---------------------------------------------------------------- frames ---- */

/*
 * One independent frame.
 *   in        samples.  CDC and chain: int8 [n][n_pol][2] (I, Q), 5-bit signed
 *             [-16, 15], 2 samples per symbol.  AEQ alone: int8 [n][4]
 *             (XI, XQ, YI, YQ), 5-bit signed, 1 sample per symbol.
 *   out       results.  CDC: int16 [n][n_pol][2], the exact complex convolution
 *             z[t] = sum_k h[k] x[t-k] (zero history, no delay compensation).
 *             Chain: int16 [n_sym][4] AEQ output at 1 sample per symbol with
 *             n_sym = ceil((n - phase) / 2), phase = ((L - 1) / 2) mod 2.
 *             AEQ alone: int16 [n][4].
 *   cd_taps   HOST int8 [cd_len][2] (re, im), 6-bit signed [-32, 31]; CDC and
 *             chain only (ignored by the AEQ alone).
 *   aeq_state DEVICE int32 [4 (S2)][4 (S1)][K] master taps of the AEQ
 *             (tap = state >> 16), read at the start and overwritten with the
 *             adapted taps at the end; NULL = start from the plan's initial taps
 *             and keep nothing.  With AEQ segments every segment starts from the
 *             state as it was when the call began (the library copies it first)
 *             and the state then receives the final taps of the last segment.
 *             Ignored by the CDC.
 *   n         samples (CDC, chain) or symbols (AEQ alone); 0 is allowed.
 *   n_pol     1 or 2 for the CDC; 2 for the chain; ignored by the AEQ alone.
 *   cd_len    L, 1..31 (31 * 2 * 16 * 32 = 31744 keeps every output inside int16
 *             and inside constraint (5)); with n_pol = 2 both polarisations use
 *             the same taps.
 */
typedef struct fnt_frame {
    const void *in;
    void *out;
    const int8_t *cd_taps;
    int32_t *aeq_state;
    int64_t n;
    int32_t n_pol;
    int32_t cd_len;
} fnt_frame;

/*
 * A batch of frames processed by one call.  `frames` is a HOST array.
 * host_buffers = 0: in/out of every frame are device pointers.
 * host_buffers = 1: in/out are host pointers.  Page-locked buffers are read
 *                   and written in place by the kernels through their device
 *                   mapping (on GB300, Grace memory over NVLink-C2C); pageable
 *                   ones are copied in and back through device memory of the
 *                   library's own.  The call returns only after the outputs
 *                   are in host memory.
 */
typedef struct fnt_frame_batch {
    int32_t n_frames;
    int32_t host_buffers;
    const fnt_frame *frames;
} fnt_frame_batch;

/* FNT-CDC alone (sections "Fermat number transform" and "Proposed FNT-CDC&AEQ
 * structure": eqs. (1), (2), (5), (7), (8)).  Errors: FNT_ERR_INVALID (shapes,
 * tap values outside 6 bits), FNT_ERR_BOUND (cd_len or step beyond eq. (5) /
 * the zero padding), FNT_ERR_NOMEM, FNT_ERR_CUDA. */
FNT_API fnt_status fnt_cdc_run(const fnt_plan *plan, const fnt_frame_batch *batch, void *stream);

/* FNT-AEQ alone on 1-sample/symbol 5-bit PDM input (eq. (6) and the 4x4
 * RV-MIMO with two 7-bit tap groups).  Each frame is one serial run, or
 * segmented when the plan says so.  Errors as fnt_cdc_run. */
FNT_API fnt_status fnt_aeq_run(const fnt_plan *plan, const fnt_frame_batch *batch, void *stream);

/* The receiver chain of the experimental section: FNT-CDC on both
 * polarisations, requantisation of the CDC output to 5 bits
 * (x = sat[-16,15](floor((z + 2^(s-1)) / 2^s)), s the smallest shift with
 * 4^s >= 2 E, E = sum_k |h[k]|^2: the AEQ input keeps at most the CDC input's
 * loading), resampling to 1 sample/symbol (times t = phase mod 2),
 * then FNT-AEQ.  Errors as fnt_cdc_run. */
FNT_API fnt_status fnt_cdc_aeq_run(const fnt_plan *plan, const fnt_frame_batch *batch, void *stream);

/* ------------------------------------------------------ prepared batches ---- */

typedef enum fnt_op { FNT_OP_CDC = 0, FNT_OP_AEQ = 1, FNT_OP_CHAIN = 2 } fnt_op;

typedef struct fnt_batch fnt_batch;

/*
 * Prepared batches, launch knobs and the serving session below are execution
 * machinery.  The paper defines none of them (it describes a hardware
 * datapath); they schedule the operations of eqs. (1)-(8) and (6) defined
 * above, and change no result.
 *
 * Prepares a batch once for repeated launches: validates it, builds the work
 * lists (frames split into 32-block CDC items; AEQ chains or segments sorted
 * longest first), uploads them and allocates the intermediate buffers, all in
 * device memory owned by the fnt_batch.  Buffers are device memory
 * (host_buffers = 0) or page-locked host memory (host_buffers = 1), which the
 * kernels read and write in place; pageable host memory is rejected with
 * FNT_ERR_INVALID.  Launches do not wait for the device; the caller
 * synchronises the stream before reading host outputs.  use_graph = 1 records
 * the launch into a CUDA graph on the first fnt_batch_launch and replays it
 * afterwards.
 */
FNT_API fnt_status fnt_batch_create(const fnt_plan *plan, const fnt_frame_batch *batch, int32_t op,
                            int32_t use_graph, fnt_batch **out);

/* Enqueues the prepared work on `stream`.  Launches of one fnt_batch must not
 * overlap on the device (they share its intermediate buffers). */
FNT_API fnt_status fnt_batch_launch(fnt_batch *b, void *stream);

/* Host-buffer batches (host_buffers = 1): with on = 1, every launch first
 * copies each frame's page-locked input into device memory of the batch's own,
 * by DMA on a stream of the batch's own, and the kernels read that copy instead
 * of reading the input across the host link (outputs are still written in
 * place).  The copy does not wait for `stream`: it starts when
 * fnt_batch_launch is called, as soon as this batch's previous launch has
 * consumed its inputs, so it overlaps work queued before it (the previous step
 * of a stream, say).  The input must therefore hold the frame's data when
 * fnt_batch_launch is called, not only once the stream reaches the launch.
 * One copy per frame and launch.  on = 0 returns to the in-place reads.  Waits
 * for the device to be idle; FNT_ERR_INVALID for a batch without host inputs. */
FNT_API fnt_status fnt_batch_set_input_copy(fnt_batch *b, int32_t on);

/* Enqueues one stage of the prepared work: stage 0 = the CDC kernel, stage 1 =
 * the AEQ kernel (a stage the op does not have enqueues nothing).  Running
 * stage 0 then stage 1 on one stream equals fnt_batch_launch without a graph;
 * it lets a caller time or overlap the two kernels separately. */
FNT_API fnt_status fnt_batch_launch_stage(fnt_batch *b, int32_t stage, void *stream);

/* Number of kernel launches one fnt_batch_launch enqueues. */
FNT_API int32_t fnt_batch_kernel_count(const fnt_batch *b);

FNT_API fnt_status fnt_batch_destroy(fnt_batch *b);

/* Sets the warps per CTA of the CDC and AEQ kernels used by later launches of
 * this plan (autotuner hook).  0 keeps the current value. */
FNT_API fnt_status fnt_plan_set_launch(fnt_plan *plan, int32_t cdc_warps, int32_t aeq_warps);

/* Prepared chain batches created after this call split their work into
 * `chunks` pieces (1..16; default 1 = off): the CDC of piece k runs on the
 * caller's stream and the AEQ of piece k on a side stream of the batch as soon
 * as the CDC items it reads are done, so CDC and AEQ can overlap.  Results do
 * not depend on it.  (On one 2^21-sample stream it measured slower: each AEQ
 * piece is a latency-bound set of serial chains.) */
FNT_API fnt_status fnt_plan_set_pipeline(fnt_plan *plan, int32_t chunks);

/* Caps the AEQ warps resident per SM for later launches of this plan
 * (autotuner hook): each AEQ CTA then reserves enough shared memory that at
 * most max(1, max_warps_per_sm / aeq warps per CTA) CTAs share an SM.  0
 * (default) lets resources decide.  Long serial AEQ chains (frames with fresh
 * taps and no segments) finish sooner when fewer share an SM, which can
 * shorten a batch whose longest chain sets its time.  Results do not depend on
 * it.  FNT_ERR_INVALID outside [0, 64]. */
FNT_API fnt_status fnt_plan_set_aeq_occupancy(fnt_plan *plan, int32_t max_warps_per_sm);

/* Picks the AEQ kernel of later launches of this plan: 1 = one warp per (chain,
 * polarisation), the throughput layout for many chains; 2 = one CTA per (chain,
 * polarisation), which spreads each block of the serial recurrence of eq. (6)
 * (section "Proposed FNT-CDC&AEQ structure") over 288 threads and cuts the time
 * per block of a lone chain; 0 (default) = 2 when the launch's chains fit one
 * CTA per SM and its longest chain has at least 256 AEQ blocks, else 1 (short
 * chains, such as the segments of served frames, do better in 1 when several
 * launches share the GPU, as each CTA of 2 holds a whole SM).  Plans with
 * aeq_freq_sum != 0 always use 1.  Results do not depend on it.
 * FNT_ERR_INVALID outside [0, 2]. */
FNT_API fnt_status fnt_plan_set_aeq_kernel(fnt_plan *plan, int32_t kind);

/* Picks the CDC kernel of later launches of this plan: 1 = one overlap-save
 * block per lane (each 64-point transform in one thread's registers), the
 * throughput layout; 2 = one block per 8 threads, each transform run as a
 * four-step 8 x 8 transform over them (eqs. (1)/(2) split by index, section
 * "Fermat number transform"), for work too small to fill the GPU one block per
 * lane; 0 (default) = 2 when a launch has fewer 32-block work items than twice
 * the SM count, else 1.  Results do not depend on it.  FNT_ERR_INVALID
 * outside [0, 2]. */
FNT_API fnt_status fnt_plan_set_cdc_kernel(fnt_plan *plan, int32_t kind);

/* The one-block-per-lane CDC kernel fetches the 32 input windows of a PDM work
 * item of one polarisation (items of both polarisations use 4-byte copies),
 * one contiguous span of the frame, with a single TMA bulk copy
 * (cp.async.bulk) into shared memory when the span, widened to 16-byte
 * boundaries, lies inside the frame and the input is 16-byte aligned; other
 * items use 4-byte asynchronous copies.  The copy's completion is awaited on an
 * mbarrier for at most about 5 ms.  A wait that runs out sets bit 1
 * (FNT_FAULT_CDC_WINDOW_WAIT) of the current device's fault word, and that
 * warp stops (its blocks' outputs are not written); nothing else waits on the
 * device.  fnt_device_faults returns the fault word of the current device and,
 * with clear != 0, resets it.  It reads the word with a synchronous copy on
 * the legacy default stream: synchronise the streams whose kernels it should
 * cover first.  Errors: FNT_ERR_INVALID (null faults), FNT_ERR_CUDA. */
#define FNT_FAULT_CDC_WINDOW_WAIT 1u
FNT_API fnt_status fnt_device_faults(int32_t clear, uint32_t *faults);

/* Test hook: with mode 1, later one-shot calls and prepared batches of this
 * plan arm the CDC's window barrier without issuing the bulk copy, so the
 * bounded wait runs out and sets FNT_FAULT_CDC_WINDOW_WAIT: a way to test that
 * path without faulting anything.  0 (default) is normal operation.
 * FNT_ERR_INVALID for other modes. */
FNT_API fnt_status fnt_plan_set_test_inject(fnt_plan *plan, int32_t mode);

/* The CDC kernel (1 or 2, as above) a launch of `n_items` CDC work items (32
 * overlap-save blocks of one polarisation, or of both) of this plan takes; 0
 * for a null plan. */
FNT_API int32_t fnt_plan_cdc_kernel_for(const fnt_plan *plan, int64_t n_items);

/* The AEQ kernel (1 or 2, as above) a launch of `n_chains` AEQ chains of this
 * plan, the longest of `longest_symbols` symbols, takes; 0 for a null plan.
 * A chain is a frame, or one AEQ segment of a frame with its warm-up. */
FNT_API int32_t fnt_plan_aeq_kernel_for(const fnt_plan *plan, int64_t n_chains, int64_t longest_symbols);

/* The plan's initial AEQ taps (the state a frame without aeq_state, or a newly
 * configured serving link, starts from): HOST int32 [4 (S2)][4 (S1)][16],
 * zero except the centre tap of the four diagonal filters, tap_init << 16.
 * The paper leaves the initial taps open; this is the usual centre-spike start.
 * Copying it into a frame's aeq_state starts that state's adaptation there. */
FNT_API fnt_status fnt_plan_initial_taps(const fnt_plan *plan, int32_t *state);

/* CDC work items created after this call cover 32 overlap-save blocks of one
 * polarisation (pols = 1) or of both polarisations of a PDM frame (pols = 2);
 * 0 (default) picks 2 when the work fills the GPU at least twice over and 1
 * otherwise.  Results do not depend on it. */
FNT_API fnt_status fnt_plan_set_cdc_items(fnt_plan *plan, int32_t pols);

/* on = 1: later AEQ launches of this plan compute the gradient of eq. (6) on the
 * tensor cores instead of the integer pipes (default 0).  Results are
 * bit-identical: e z (|e z| <= 2^46) is split into four balanced 12-bit limbs,
 * which, like the 5-bit input, are exact in f16, and every per-block sum of
 * limb x input products stays below 2^24, so the f32 accumulation is exact and
 * the limb sums are recombined in int64.  Off by default because the paper's
 * path is integer arithmetic throughout. */
FNT_API fnt_status fnt_plan_set_tensor_gradient(fnt_plan *plan, int32_t on);

/* ------------------------------------------------- allocation-free chain ---- */

/* Largest frame (samples) and AEQ segment count fnt_cdc_aeq_run_noalloc takes. */
#define FNT_NOALLOC_MAX_SAMPLES (1 << 21)
#define FNT_NOALLOC_MAX_SEGMENTS 4096

/*
 * The receiver chain of fnt_cdc_aeq_run for ONE frame, without allocating any
 * memory.  The paper has no counterpart: this exists for callers that cannot
 * allocate device memory where they process a frame (a latency-critical receive
 * loop that cannot afford an allocation's synchronisation or latency, or an
 * application that owns all device memory through its own allocator).
 *
 * The caller passes the frame as for fnt_cdc_aeq_run (device in / out / state,
 * host taps).  The work tables and the intermediate CDC -> AEQ symbols live in
 * a fixed array of about 4.3 MiB in device memory that belongs to the library
 * image: every GPU that loads libfnt holds it until the process exits.  The
 * first call on a device, with that device current, sets up: it looks up the
 * array's address, creates the events that guard the library's host copies of
 * the work tables, and (once per process) page-locks those host copies; make
 * that first call outside any stream capture.  Each call uploads its tables
 * with one asynchronous copy and does not wait for the stream (a host copy is
 * reused four calls later, after its last upload has run).  The call cannot be
 * captured in a CUDA graph: on a capturing stream it returns FNT_ERR_INVALID
 * and enqueues nothing.  All calls on a device share the array and overwrite
 * it, so calls whose work overlaps on the GPU race: keep them on one stream or
 * wait between them.  Frames longer than
 * FNT_NOALLOC_MAX_SAMPLES, or plans that cut one into more than
 * FNT_NOALLOC_MAX_SEGMENTS AEQ segments, are rejected with FNT_ERR_BOUND before
 * anything is enqueued.  Results equal fnt_cdc_aeq_run's bit for bit.
 */
FNT_API fnt_status fnt_cdc_aeq_run_noalloc(const fnt_plan *plan, const fnt_frame *frame, void *stream);

/* ---------------------------------------------------------------- serving ---- */

/*
 * Continuous-batching session over n_links links.  Each link has fixed CD taps
 * and an AEQ tap state that stays in device memory and carries from one of the
 * link's frames to the next (frames of a link run in submission order; the
 * delay line does not carry).  Requests are admitted while the session's device
 * memory for them (intermediate CDC -> AEQ symbols, state copies) stays within
 * mem_cap_bytes.  The scheduler packs admitted frames into waves (at most one
 * frame per link).  The oldest frame of every link with nothing on the device
 * goes into a wave on one of n_streams main streams, so waves of unrelated links
 * run concurrently.  While a link's previous frame is still on the device, its
 * next frame goes into a chained wave (with the next frames of the other links
 * whose latest frame is in that same wave) on one of 4 * n_streams further
 * streams, which waits on the device for that one wave: the host never has to
 * observe a completion before launching a link's next frame, and a waiting frame
 * holds no main stream.  A plan with AEQ
 * segments cuts a long frame into segments that start from the link's taps as
 * the frame began (as fnt_cdc_aeq_run does with a frame state); the last
 * segment writes the link's taps.
 */
typedef struct fnt_session fnt_session;

typedef struct fnt_completion {
    uint64_t ticket;
    int32_t link;
    int32_t status;          /* fnt_status of this request */
    int64_t n_sym;           /* symbols written */
    double submit_us;        /* host steady-clock times, microseconds */
    double start_us;         /* its wave was launched */
    double done_us;          /* completion was observed */
} fnt_completion;

FNT_API fnt_status fnt_session_create(const fnt_plan *plan, int32_t n_links, size_t mem_cap_bytes,
                              int32_t n_streams, fnt_session **out);

/* Fixed CD taps of a link (HOST int8 [L][2]); resets its AEQ state to the plan's
 * initial taps.  Not allowed while the link has requests in the session. */
FNT_API fnt_status fnt_session_set_link(fnt_session *s, int32_t link, const int8_t *cd_taps, int32_t L);

/* Submits one PDM frame: in = int8 [n][2][2], out = int16 [n_sym][4] (as for
 * fnt_cdc_aeq_run).  Each is device memory or page-locked host memory, which
 * the kernels read and write in place through its device mapping (no staging
 * copies); pageable host memory is rejected with FNT_ERR_INVALID.  The buffers must stay valid until
 * the request completes.  Returns FNT_ERR_BUSY, admitting nothing, when the
 * request does not fit under the memory cap right now. */
FNT_API fnt_status fnt_session_submit(fnt_session *s, int32_t link, const void *in, int64_t n, void *out,
                              uint64_t *ticket);

/* One request of fnt_session_submit_many: the arguments of fnt_session_submit. */
typedef struct fnt_request {
    int32_t link;
    int32_t reserved;        /* must be 0 */
    const void *in;          /* int8 [n][2][2] */
    int64_t n;               /* samples per polarisation */
    void *out;               /* int16 [n_sym][4] */
} fnt_request;

/* Admits reqs[0..n_reqs) in order, each exactly as fnt_session_submit would,
 * then runs the scheduler once, so a burst of requests forms full waves with
 * one call.  Stops at the first request that is not admitted and returns its
 * status (FNT_ERR_BUSY when the memory cap refuses it: poll, then submit the
 * rest); FNT_OK when all were admitted.  *n_admitted is the number admitted and
 * tickets[0..*n_admitted) their tickets (HOST arrays of n_reqs entries). */
FNT_API fnt_status fnt_session_submit_many(fnt_session *s, const fnt_request *reqs, int32_t n_reqs,
                                   uint64_t *tickets, int32_t *n_admitted);

/* Cancels an admitted request that has not been launched yet: it completes
 * (through fnt_session_poll) with status FNT_ERR_CANCELLED, its memory is
 * released, and its link's later frames run as if it had never been
 * submitted.  FNT_ERR_NOT_FOUND when the ticket is unknown, already launched or
 * already complete (a launched frame always runs to completion). */
FNT_API fnt_status fnt_session_cancel(fnt_session *s, uint64_t ticket);

/* Counters of a session since its creation (a snapshot). */
typedef struct fnt_session_stats {
    uint64_t admitted;        /* requests admitted */
    uint64_t completed;       /* requests completed OK */
    uint64_t failed;          /* requests completed with an error (not cancelled) */
    uint64_t cancelled;       /* requests cancelled before launch */
    uint64_t waves;           /* waves launched */
    uint64_t chained_waves;   /* of which waited on the device for an earlier wave */
    uint64_t wave_frames;     /* frames in all launched waves */
    uint64_t max_wave;        /* largest wave, frames */
    uint64_t arena_used;      /* bytes of the memory cap held now */
    uint64_t arena_peak;      /* most bytes ever held */
    int32_t queued;           /* admitted, not launched */
    int32_t in_flight;        /* launched, not complete */
} fnt_session_stats;

FNT_API fnt_status fnt_session_get_stats(fnt_session *s, fnt_session_stats *out);

/* Drives the scheduler and collects finished requests (at most max_done).  Waits
 * up to timeout_us for at least one completion (0 = do not wait); returns
 * FNT_ERR_TIMEOUT when nothing completed in that time. */
FNT_API fnt_status fnt_session_poll(fnt_session *s, int32_t timeout_us, fnt_completion *done,
                            int32_t max_done, int32_t *n_done);

/* Requests admitted and not yet returned by fnt_session_poll. */
FNT_API int32_t fnt_session_pending(const fnt_session *s);

/* Checkpoint / resume of a link's AEQ state (HOST int32 [4][4][K]).  The link
 * must have no request in the session.  Resuming with a saved state gives the
 * same results, bit for bit, as never having stopped. */
FNT_API fnt_status fnt_session_get_link_state(fnt_session *s, int32_t link, int32_t *state);
FNT_API fnt_status fnt_session_set_link_state(fnt_session *s, int32_t link, const int32_t *state);

/* Fault injection for tests of the serving loop (host side only): the next
 * n_waves wave launches fail before anything is enqueued, as a failed CUDA call
 * would; their requests complete with status FNT_ERR_CUDA, their memory is
 * released and their links' tap states are left as they were. */
FNT_API fnt_status fnt_session_inject_failures(fnt_session *s, int32_t n_waves);

/* Runs every admitted request to completion, then frees the session. */
FNT_API fnt_status fnt_session_destroy(fnt_session *s);

#ifdef __cplusplus
}
#endif

#endif /* FNT_H */
