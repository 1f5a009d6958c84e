/*
 * rx.h -- C ABI of the GB300 coherent-receiver DSP library.
 *
 * The library runs the receiver chain of arXiv 2108.07004 (Sec. 2) in the
 * dual-polarisation form: overlap-save chromatic-dispersion compensation
 * (CDC) -> 2x2 butterfly FIR equaliser adapted block-wise (CMA, then
 * decision-directed LMS) -> blind phase search (BPS) -> exact log-sum-exp
 * bit LLRs with BER / GMI counting.  Every step runs in the library's own
 * CUDA kernels on the calling process's current device.
 *
 * Conventions shared by every entry point
 *   - Return value: RX_OK (0) or a negative RX_E* code; the message of the
 *     last failure on the calling thread is returned by rx_last_error().
 *   - Complex samples are interleaved float32 (re, im) ("c64").  A stream's
 *     samples are polarisation-major: [2][n_samples] (X then Y).  A handle
 *     processes S independent streams of equal length at once ("streams"
 *     parameter, default 1); buffers then carry a leading [S] dimension.
 *   - Pointers documented as "device" must be CUDA device (or managed)
 *     memory; "host" pointers are ordinary host memory.  The caller owns
 *     every buffer it passes; the library owns the handle, its tables, its
 *     per-stream state and its scratch memory (allocated with cudaMalloc on
 *     first use and freed by rx_destroy).
 *   - Work is enqueued on the handle's CUDA stream (rx_set_stream; the
 *     default is the legacy default stream).  Calls returning statistics
 *     synchronise that stream.
 *   - LLR sign: positive means bit 0.  Bit order of a label: MSB first.
 *   - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef RX_H
#define RX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RX_OK         0
#define RX_EINVAL    (-1)   /* bad argument or unsupported configuration   */
#define RX_ENOMEM    (-2)   /* device or host allocation failed            */
#define RX_ECUDA     (-3)   /* a CUDA runtime call failed                  */
#define RX_ETIMEDOUT (-4)   /* a bounded device wait gave up               */
#define RX_EBUSY     (-5)   /* handle in use / parameter locked            */
#define RX_ESTATE    (-6)   /* call out of order (e.g. no reference set)   */

/* built-in formats: Gray-mapped square QAM on each polarisation (1-3) and
 * the 4D 64-ary geometrically shaped format (4: the library's design by the
 * paper's Sec. 5 optimiser, frozen in data/gs4d64_v1.json and compiled in;
 * the paper prints no 4D table) */
#define RX_FMT_CUSTOM   0
#define RX_FMT_DP_QPSK  1
#define RX_FMT_DP_16QAM 2
#define RX_FMT_DP_64QAM 3
#define RX_FMT_GS4D64   4

typedef struct rx_handle rx_handle;

/* Constellation description.  Sec. 2 of the paper uploads the points and
 * their bit mapping to the GPU and assumes no symmetry of the format; the
 * phase search here uses the rotational symmetry sym_order (1, 2 or 4) and
 * the library verifies it exactly at creation.
 *   kind      RX_FMT_*; for built-ins the other fields are ignored.
 *   dims      2: one 2D table used on each polarisation (m_bits per pol);
 *             4: one joint 4D table over both polarisations.
 *   m_bits    bits per table entry (table size 2^m_bits; dims 2: 2 .. 7,
 *             i.e. 4 to 128 points per polarisation, the paper's 4- to
 *             64-QAM, GS-8 and GS-128 (Sec. 5); dims 4: 6), with at most
 *             32 (dims 2) / 16 (dims 4) orbits under the rotation by
 *             2 pi / sym_order.
 *   points    host, [2^m_bits][dims] float32 (re, im [, re_y, im_y]),
 *             copied at creation.
 *   labels    host, [2^m_bits] bit label of each row, a permutation of
 *             0 .. 2^m_bits - 1. */
typedef struct {
    int kind;
    int dims;
    int m_bits;
    int sym_order;
    const float *points;
    const uint32_t *labels;
} rx_format;

/* Per-stream statistics (host struct, filled by rx_process / rx_get_stats).
 * Counting covers symbols skip_head .. N - skip_tail - 1 of the stream and
 * needs a reference (rx_set_reference); Sec. 3 counts errors offline over
 * many buffers. */
typedef struct {
    uint64_t n_sym;        /* symbols counted                                  */
    uint64_t n_bits;       /* bits counted (n_sym * m)                         */
    uint64_t bit_errors;   /* hard decisions (LLR < 0 -> 1) != reference bits  */
    double   gmi_sum;      /* sum of log2(1 + exp(-(1 - 2b) LLR)) over bits    */
    double   gmi;          /* m - gmi_sum / n_sym  (bits per 4D symbol)        */
    double   ber;          /* bit_errors / n_bits                              */
    double   evm_num;      /* sum |z - d|^2 (d: nearest point)                 */
    double   evm_den;      /* sum |d|^2                                        */
    double   sigma2_last;  /* noise variance used for the last block           */
    uint64_t n_out;        /* LLR rows written for this stream (rx_push /      */
                           /* rx_flush: valid rows handed out so far)          */
    uint32_t blocks;       /* blocks processed                                 */
    uint32_t reserved;
    uint64_t first_valid;  /* rx_push: index in this call's llr_out of the     */
                           /* first row that holds a symbol (the rows before   */
                           /* it are the stream delay's zeros); otherwise 0    */
} rx_stats;

/* ---- lifetime ---------------------------------------------------------- */

/* Create a receiver for one format and link.  symbol_rate in Bd, sps must
 * be 2, cd_ps_per_nm is the accumulated dispersion D*L to undo, taps the
 * odd FIR length per butterfly branch (7, 15 or 31), bps_phases the number
 * of BPS test phases B (8 .. 64).  Returns NULL on error (rx_last_error()). */
rx_handle *rx_create(const rx_format *format, double symbol_rate, int sps,
                     double cd_ps_per_nm, int taps, int bps_phases);
void rx_destroy(rx_handle *h);                      /* NULL-safe */

/* Set / read a numeric parameter.  Keys (defaults in brackets):
 *   "fft" [1024] (1024 or 4096), "overlap" [256] (even, < fft/2),
 *   "mu" [1e-3], "bps_window" [64] (even, 2..64), "block" [4096] symbols,
 *   "n_upd" [1024] (<= block - bps_window/2), "lag" [1] (1..4),
 *   "n_pre" [2048], "cma_passes" [1], "n_cma" [0], "n_train" [1024]
 *   (<= 20000), "train_passes" [3],
 *   "sigma2" [0 = estimate per block], "skip_head" [4096],
 *   "skip_tail" [512], "streams" [1], "rolloff" [0.1],
 *   "cd_ps_per_nm" [the value given to rx_create]: the dispersion to undo,
 *   "matched_filter" [1]: 0 leaves the root-raised-cosine matched filter
 *   out of the CDC's spectral multiply, for input that an earlier stage has
 *   already filtered (the static equaliser after the KK front-end, Sec. 2;
 *   with cd_ps_per_nm = 0 the CDC is then the identity),
 *   "widely_linear" [0]: 1 makes the butterfly widely linear, y_q =
 *   sum_p sum_t conj(h_qp[t]) x_p[2k+D-t] + conj(g_qp[t]) conj(x_p[2k+D-t])
 *   (the paper's equaliser acts on the signal and its conjugate, Sec. 2);
 *   every tap array of the handle and of the stage entries (rx_fir, rx_lms,
 *   rx_train) is then [S][2][2][2T] with h_qp[0..T-1] then g_qp[0..T-1],
 *   "lms_block" [1]: the block-wise (blind) tap updates in groups of this
 *   many (1..64) whose outputs and errors all use the taps at the group's
 *   start (block LMS, a parallel variant beside the exact recursion; also
 *   rx_lms modes 0-2; the start-up training stays sequential),
 *   "lms_start" [0]: where the update over block n starts: 0 from U_{n-1}
 *   (one chain through all blocks), 1 from W_n = U_{n-lag}, the taps that
 *   equalised block n (Sec. 2's "part of a buffer updates the taps for
 *   later buffers" read per buffer), so the blocks n = r (mod lag) form lag
 *   independent chains that run concurrently on lag streams,
 *   "wavelength_nm" [1550], "profile" [0] (1: time every launch group and
 *   every block, 2: time the BPS launches only),
 *   "precision" [0]: storage of the chain's CDC and FIR outputs, 0 float32,
 *   1 half (FP16), 2 bfloat16; arithmetic, LMS taps and the phase unwrap
 *   stay float32 (the precision variant; rx_get_state / rx_set_state need 0),
 *   "bps_tc" [0]: 1 forms the phase search's orbit correlations on the
 *   tensor cores (4D tables of 16 orbits; reads 0 where unsupported),
 *   "lms_exact" [0]: 1 runs the DD-LMS's warp-wide nearest-point search on
 *   every update; 0 takes each decision a sub-block ahead on the update's
 *   partial output and keeps it while the corrections added since stay
 *   inside half its margin (the same decisions and taps, bit for bit),
 *   "sm_reserve" [0]: SMs the handle leaves to other work on the GPU (e.g.
 *   another handle's frame in flight) when it sizes the phase search and
 *   FIR grids to one wave; the phase search's range split, and with it the
 *   summation order of the block's sigma^2, follows the grid,
 *   "issue" [0]: how rx_process / rx_process_blocks issue their work: 0
 *   each stage group on its own stream (start-up and LMS chains, demap)
 *   with events between them, so a handle alone overlaps its own stages; 1
 *   every launch on the handle's stream, no event operations (for handles
 *   that run beside many others, whose work fills the device: the host
 *   issues about a third of the operations); 2 as 1, and a call that
 *   continues a stream (b0 > 0) is captured as a CUDA graph and launched
 *   as one, the handle's instantiated graph updated in place when only
 *   kernel arguments changed.  Results are the same in every mode; the
 *   host entry (rx_process_host) and the streaming entry always use 0,
 *   "fir_tma" [1]: the FIR stages each tile's input window with the tensor
 *   memory accelerator (3D tensor copies of the [2S][n_samples] rows in
 *   64-byte groups, zero-filled outside them) where the rows are 16-byte
 *   aligned whole groups (N a multiple of 4 for float32 storage, of 8 for
 *   16-bit storage), else, and with 0, with cp.async; the outputs are the
 *   same bits.
 * Changing a parameter resets the stream state (rx_reset). */
int rx_set_param(rx_handle *h, const char *key, double value);
int rx_get_param(const rx_handle *h, const char *key, double *value);

/* Use cuda_stream (a cudaStream_t) for all later work of this handle. */
int rx_set_stream(rx_handle *h, void *cuda_stream);

/* Known transmitted bits, device, [S][n_sym][m] uint8 (0/1), m bits per 4D
 * symbol (dims 2: X bits then Y bits).  Enables the start-up training
 * alignment (Sec. 2: the equaliser first converges on a training sequence)
 * over the first n_train symbols and BER/GMI counting.  Copied. */
int rx_set_reference(rx_handle *h, const uint8_t *bits, size_t n_sym);

/* rx_set_reference with the bits left in host memory ([S][n_sym][m] uint8,
 * as above): the next rx_process_host copies them in group by group beside
 * the samples (rows a group's blocks count with, and for the first group
 * the training span), so that the copy overlaps the chain.  Any other entry
 * point that needs the reference first copies it whole on the handle's
 * stream.  `bits` must stay valid and unchanged until that call returns;
 * pinned memory keeps the copies asynchronous.  Device memory for the bits
 * (S * n_sym * m bytes) and the labels is kept by the handle. */
int rx_set_reference_host(rx_handle *h, const uint8_t *bits, size_t n_sym);

/* Forget the stream state (taps, phase, counters): the next rx_process
 * starts a new stream. */
int rx_reset(rx_handle *h);

/* ---- the chain ---------------------------------------------------------- */

/* Run the whole chain over S complete streams.
 *   samples   device, [S][2][n_samples] c64, n_samples = 2 * N.
 *   llr_out   device, [S][N][m] float32, caller-allocated.
 *   stats     host, [S] rx_stats or NULL; when non-NULL the call waits for
 *             the device and fills it.
 * Block schedule (Sec. 2: part of one buffer updates the equaliser taps used
 * for later buffers): start-up CMA and training alignment, then for every
 * block of "block" symbols: FIR with the taps from "lag" blocks back, BPS,
 * unwrap, LLRs, then LMS over the block's first n_upd symbols. */
int rx_process(rx_handle *h, const void *samples, size_t n_samples,
               float *llr_out, rx_stats *stats);

/* rx_process with host buffers: samples (host, [S][2][n_samples] c64) in,
 * LLRs (host, [S][N][m]) out; results identical to rx_process.  The blocks
 * run in groups of two: the input samples a group's CDC frames read are
 * copied in on one copy stream and its LLR rows copied out on another, so
 * the copies overlap the chain of the neighbouring groups (asynchronously
 * when the host buffers are pinned; pageable buffers also work); from the
 * second group on, a group's CDC runs on a stream of its own as soon as
 * its samples are in.  Device
 * copies of the input and output are kept by the handle (allocated on first
 * use).  Returns when the LLRs are in llr_out. */
int rx_process_host(rx_handle *h, const void *samples, size_t n_samples,
                    float *llr_out, rx_stats *stats);

/* Statistics of the last rx_process (host [S]); synchronises. */
int rx_get_stats(rx_handle *h, rx_stats *stats);

/* ---- streaming: one call per buffer of a continuous stream ---------------
 * Sec. 2 of the paper processes the ADC's DMA buffers one after another in
 * real time, the equaliser taps learned on part of one buffer serving the
 * buffers after it.  rx_push takes the next n_samples samples per
 * polarisation of each of the S streams (device or host memory,
 * [S][2][n_samples] c64; any even count, 0 included) and writes exactly
 * n_samples / 2 LLR rows per stream into llr_out (device, [S][n_samples/2]
 * [m] float32): output row r of a stream (counted over all its pushes)
 * holds symbol r - d, where d is the fixed stream delay of rx_stream_delay;
 * rows r < d are zeros, and stats.first_valid gives the first row of this
 * call that holds a symbol.  rx_flush ends the stream: the samples pushed so
 * far are the whole stream (zeros after its end, as in rx_process), and the
 * symbols not yet handed out come out: r = min(N, d) rows per stream,
 * written packed as [S][r][m] into llr_out (N = the stream's symbols, the
 * samples pushed / 2); *n_rows receives r.  The pushed rows after
 * the delay followed by the flushed rows are bit for bit the LLRs of one
 * rx_process over the concatenated samples, and the counters equal its
 * counters when the reference (rx_set_reference, set before the first push)
 * holds exactly the stream's N symbols: counting covers symbols skip_head
 * .. ref_n - skip_tail - 1, since the stream's end is not known before the
 * flush.
 *
 * The delay: the chain is block-wise (the noise variance and the LMS span
 * of a block use the whole block), so the symbols of block n leave once the
 * samples of every CDC frame the block reads are in.  With
 * need(n) = ceil((2 max((n+1) block, max(n_pre, n_train)) + D) / hop) hop
 * + overlap/2 samples (hop = fft - overlap, D = (taps-1)/2) for blocks
 * 0 .. n and C(n) = n block - bps_window/2 symbols done after blocks
 * 0 .. n-1, d = max over n of (floor((need(n) - 1) / 2) - C(n)), about
 * block + bps_window/2 + (hop + overlap/2 + D)/2 symbols; at the
 * benchmark's settings (block 2^16, FFT 4096 / overlap 1024, 31 taps,
 * window 64) d = 67 359.
 *
 * The handle keeps a window of about (3 + hop / gcd(2 block, hop)) blocks
 * of the stream (input samples and LLR rows twice each), allocated by the
 * first push; a push of many samples is taken in pieces of one block.  A
 * parameter change, rx_set_reference, rx_reset or a whole-stream call
 * (rx_process, rx_process_blocks, rx_process_host, rx_set_state) ends the
 * stream without output; the next push starts a new one.  Symbol outputs
 * (rx_set_symbol_output) are not available while streaming (RX_EINVAL).
 * Both calls return after queuing the work when stats is NULL; with stats
 * they synchronise and fill it ([S]).  Errors: RX_EINVAL (odd n_samples,
 * NULL buffers), RX_ESTATE (rx_flush without a stream). */
int rx_stream_delay(rx_handle *h, size_t *delay);
int rx_push(rx_handle *h, const void *samples, size_t n_samples, float *llr_out, rx_stats *stats);
int rx_flush(rx_handle *h, float *llr_out, size_t *n_rows, rx_stats *stats);

/* Wait at most timeout_ms (>= 0) of host time for the work queued on the
 * handle's CUDA stream: RX_OK when it is done, RX_ETIMEDOUT (the work goes
 * on; wait again later) when the time ran out first.  For callers that may
 * not block without a bound, e.g. a real-time loop that must take the next
 * DMA buffer in time. */
int rx_wait(rx_handle *h, double timeout_ms);

/* Device time of the last rx_process per stage, from CUDA events recorded
 * around every launch on its own stream when the parameter "profile" is 1
 * (2: the "bps" stage only)
 * (launch counts are kept always).  stage: "cdc", "fir", "bps", "unwrap",
 * "demap", "lms", "startup" or "all".  ms_total may be NULL; synchronises
 * the device when it is not. */
int rx_get_profile(rx_handle *h, const char *stage, double *ms_total, uint64_t *launches);

/* Per-block latency of the last rx_process (profile = 1): device time from
 * the start of a block's FIR to the end of its demapping, in ms, for up to
 * cap blocks; *n receives the number of blocks.  ms may be NULL to query. */
int rx_get_block_latency(rx_handle *h, double *ms, size_t cap, size_t *n);

/* Run blocks b0 .. b1-1 of S streams whose complete samples are at
 * `samples` (device, [S][2][n_samples] c64, n_samples = 2 N), the block
 * schedule of rx_process cut at block boundaries (Sec. 2: the taps an LMS
 * span produces serve later buffers, so the state carried from block to
 * block is the taps, the phase unwrap carry and the counters).
 *   b0 == 0   starts the stream: start-up CMA and training, then block 0.
 *   b0 >  0   continues the stream: the handle must hold the state after
 *             block b0 - 1 of a stream of the same N, left by an earlier
 *             call or restored by rx_set_state; RX_ESTATE otherwise.
 *   b1        <= ceil(N / block); b1 > b0.
 * llr_out (device, [S][N][m]) receives rows a(b0) .. e(b1-1) - 1, where
 * a(n) = max(0, n*block - W/2), e(n) = (n+1)*block - W/2 (N for the last
 * block), W = "bps_window"; other rows are not touched.  Only the CDC
 * frames these blocks read are filtered.  stats as in rx_process (counters
 * accumulate over the calls of one stream).  Calls for b0 = 0 .. B-1 in
 * order give the same output as one rx_process over the stream. */
int rx_process_blocks(rx_handle *h, const void *samples, size_t n_samples, size_t b0,
                      size_t b1, float *llr_out, rx_stats *stats);

/* Checkpoint / resume of the stream state between blocks (what block n of
 * the schedule needs from blocks before it).  A state is a host byte
 * buffer: one rx_state_header, then, for n = blocks_done, L = lag,
 * S = streams, T = taps per butterfly branch (the filter length, 2x it when
 * "widely_linear" is 1; the header's taps field holds this number),
 * W = bps_window, K = n*block:
 *   taps     [L][S][2][2][T] c64: U_{n-L+j}, j = 0 .. L-1, the LMS results
 *            blocks n .. n+L-1 equalise with (block n+j uses entry j);
 *            U_{n-1} (entry L-1) is where the LMS of block n starts;
 *            U_i = W_0 (start-up result) for i < 0.  Tap layout h[q][p][t]
 *            of rx_fir.
 *   carry    [S][2] int32: unwrap carry (m, b) of the last symbol before
 *            a(n), as in rx_unwrap.
 *   y_tail   [S][2][W] c64: FIR output of symbols K-W .. K-1 (zeros before
 *            symbol 0), the phase-search window halo of block n.
 *   counters [S] rx_state_counters.
 * Nothing else carries from block to block: a state restored into a handle
 * with the same create arguments and parameters continues the stream as
 * the handle that saved it would (rx_process_blocks with b0 = n).  The
 * layout is public so that a state can be built from outside (a test
 * injects a model receiver's state). */
#define RX_STATE_MAGIC   0x31535852u   /* "RXS1" */
#define RX_STATE_VERSION 1u
typedef struct {
    uint32_t magic;        /* RX_STATE_MAGIC                                   */
    uint32_t version;      /* RX_STATE_VERSION                                 */
    int32_t  streams;      /* S      must match the handle                     */
    int32_t  taps;         /* T      must match                                */
    int32_t  lag;          /* L      must match                                */
    int32_t  bps_window;   /* W      must match                                */
    int32_t  bps_phases;   /* B      must match                                */
    int32_t  m_bits;       /* m      must match                                */
    int64_t  block;        /* block length, must match                         */
    int64_t  n_sym;        /* N of the stream (symbols)                        */
    int64_t  blocks_done;  /* n >= 1: the next block to run                    */
    int64_t  lms_updates;  /* LMS updates so far (CMA -> DD switch at n_cma)   */
} rx_state_header;
typedef struct {
    uint64_t bit_errors, n_sym;
    double   gmi_sum, evm_num, evm_den, sigma2;
} rx_state_counters;

/* Serialise the state after the last processed block into buf (host).
 * *len in: capacity, out: bytes used; buf NULL queries the size.
 * RX_ESTATE before the first block of a stream has run; RX_EINVAL when
 * the capacity is too small (*len then holds the size).  Synchronises. */
int rx_get_state(rx_handle *h, void *buf, size_t *len);
/* Restore a state (host buf of exactly len bytes, layout above).  RX_EINVAL
 * on a bad magic, version or length, or a header that does not match the
 * handle's parameters; nothing is changed then.  blocks_done must be >= 1
 * (block 0 also needs the start-up's training phases, which are not part
 * of a state).  Synchronises. */
int rx_set_state(rx_handle *h, const void *buf, size_t len);

/* ---- learned demapper -------------------------------------------------- */

/* An MLP 4 -> 128 -> 128 -> 6 (GELU) as a learned alternative to the exact
 * log-sum-exp demapper (the paper designs its constellations with the GMI of
 * exact bitwise demapping, Sec. 5; the learned form is judged by its GMI gap
 * to it).  Input x = (Re z_X, Im z_X, Re z_Y, Im z_Y) of a de-rotated 4D
 * symbol; output o = sigma^2 * LLR (LLR > 0 means bit 0, MSB first), so
 * LLR = o / sigma^2 with the block's noise variance.  Layers compute with
 * bfloat16-rounded weights (round to nearest even) of float32 master
 * weights, float32 activations and accumulation; training minimises the mean
 * binary cross-entropy over the bits with Adam (beta 0.9 / 0.999, eps 1e-8).
 * Parameters, float32, in this order: W1 [128][4], b1 [128], W2 [128][128],
 * b2 [128], W3 [6][128], b3 [6].  Device buffers below: x [n][4] float32,
 * sigma2 [n] float32, bits [n][6] uint8 (0/1), llr [n][6] float32.  Work
 * goes on the MLP's stream (rx_mlp_set_stream).  Batch reductions are in a
 * fixed order: results do not depend on timing. */
#define RX_MLP_PARAMS 17926
typedef struct rx_mlp rx_mlp;
/* params: host [RX_MLP_PARAMS] float32, copied; NULL gives zeros.  NULL on error. */
rx_mlp *rx_mlp_create(const float *params);
void rx_mlp_destroy(rx_mlp *m);                     /* NULL-safe */
int rx_mlp_set_stream(rx_mlp *m, void *cuda_stream);
/* float32 master parameters to / from host memory; setting resets Adam. */
int rx_mlp_get_params(rx_mlp *m, float *params);
int rx_mlp_set_params(rx_mlp *m, const float *params);
/* Gradient of the mean BCE over a batch of n samples into grad (device
 * [RX_MLP_PARAMS]) and the loss into loss (device [1], may be NULL). */
int rx_mlp_grad(rx_mlp *m, const float *x, const float *sigma2, const uint8_t *bits, size_t n,
                float *grad, float *loss);
/* One Adam step on a batch of n samples with learning rate lr; the batch's
 * loss (before the step) into loss (device [1], may be NULL). */
int rx_mlp_train_step(rx_mlp *m, const float *x, const float *sigma2, const uint8_t *bits,
                      size_t n, float lr, float *loss);
/* LLRs of n samples. */
int rx_mlp_infer(rx_mlp *m, const float *x, const float *sigma2, size_t n, float *llr);
/* Kernel paths (results equal within the tolerances stated above):
 *   "train_tc"  1 (default): the three 128-wide GEMMs of a training step on
 *               the tcgen05 tensor cores, float32 operands split into three
 *               bfloat16 terms (bfloat16 weights enter exactly), float32
 *               accumulation; 0: float32 SIMT GEMMs.
 *   "infer"     2 (default): fused inference with the 128 x 128 layer on the
 *               tcgen05 tensor cores (accumulators in tensor memory); 1: the
 *               same layer as mma.sync.
 * The tensor-core kernels' waits are bounded: a wait that gave up is
 * reported as RX_ETIMEDOUT by the next rx_mlp_get_params (or rx_get_stats of
 * a handle using the MLP).  RX_EINVAL for another key or value. */
int rx_mlp_set_param(rx_mlp *m, const char *key, double value);
int rx_mlp_get_param(const rx_mlp *m, const char *key, double *value);

/* The chain's demapper: m (not owned; must outlive its use) replaces the
 * exact log-sum-exp LLRs of rx_process with the MLP's (counting unchanged);
 * NULL restores the exact demapper.  RX_EINVAL unless the format is a
 * 64-point 4D table. */
int rx_set_demapper(rx_handle *h, rx_mlp *m);
/* Symbol outputs of later rx_process calls (device, caller-owned, sized for
 * the streams' N): x4 [S][N][4] float32, the de-rotated 4D symbols as the
 * learned demapper takes them, and sigma2 [S][N] float32, each symbol's
 * block noise variance; either may be NULL (not written).  Used to make the
 * learned demapper's training data from the chain. */
int rx_set_symbol_output(rx_handle *h, float *x4, float *sigma2);

/* ---- serving: continuous batching over streams ---------------------------- */

/* One request = one stream with its own format, link and receiver settings.
 * Device buffers are caller-owned and must stay valid until the request is
 * done: samples [2][n_samples] c64, llr_out [N][m] float32, ref_bits
 * [N][m] uint8 (may be NULL: no training stage, no counting).  fft,
 * overlap, block, n_pre: 0 keeps the handle default.  Custom tables are
 * copied at submission. */
typedef struct {
    rx_format format;
    double symbol_rate;
    int sps;
    double cd_ps_per_nm;
    int taps;
    int bps_phases;
    int fft, overlap, block, n_pre;
    const void *samples;
    size_t n_samples;
    float *llr_out;
    const uint8_t *ref_bits;
} rx_request;

/* A server admits queued requests in arrival order while fewer than
 * max_slots run and the running ones' device-memory estimates (about 53 B
 * per symbol plus 1 MiB) leave room in mem_budget_bytes; each admitted
 * request gets a handle and CUDA stream (a finished request's, kept idle for
 * the next request with the same format, symbol rate, sps, taps and test
 * phases, so that no device memory is freed while others run; idle handles
 * count against the budget and are destroyed when room is needed), and
 * every step issues (from up to "issue_threads" host threads of the library,
 * one request's blocks always from one thread) the next
 * "blocks_per_step" blocks of every running request, so requests that arrived at different
 * times overlap on the device (the paper's multiple processing streams,
 * Sec. 2); by default a request's launches all go on its own stream
 * without event operations (issue mode 1, rx_server_set_param).  A finished request frees its slot and memory at the next step.
 * Results of a request equal those of a handle processing it alone.  Every
 * entry point takes the server's lock, so submit / poll / info and the
 * settings may be called from any thread; steps come from one place at a
 * time (the caller's rx_server_step / rx_server_run, or the server's own loop
 * of rx_server_start).  Errors: rx_server_last_error() (per thread). */
typedef struct rx_server rx_server;
#define RX_REQ_QUEUED  0
#define RX_REQ_RUNNING 1
#define RX_REQ_DONE    2
#define RX_REQ_FAILED  3
rx_server *rx_server_create(size_t mem_budget_bytes, int max_slots);
void rx_server_destroy(rx_server *s);               /* NULL-safe; waits for running work */
/* Queue a request (RX_EINVAL if it alone exceeds the budget); *id names it. */
int rx_server_submit(rx_server *s, const rx_request *r, uint64_t *id);
/* Retire finished requests, admit what fits, issue the next blocks_per_step
 * blocks of each running request; *n_left (may be NULL) = running + queued.
 * Does not wait. */
int rx_server_step(rx_server *s, int *n_left);
/* Step until every submitted request is done. */
int rx_server_run(rx_server *s);
/* The server's own loop: a host thread of the library, on the device current
 * at the call, that steps while requests run or wait (waiting up to 100 us
 * between steps that issue nothing, and sleeping while none are submitted),
 * so requests submitted from any thread are admitted and issued without the
 * caller stepping; rx_server_step and rx_server_run return RX_ESTATE while it
 * runs.  rx_server_stop ends it after its current step (requests still
 * running then finish by rx_server_step / rx_server_run); rx_server_destroy
 * stops it first.  RX_ESTATE if already running / not running. */
int rx_server_start(rx_server *s);
int rx_server_stop(rx_server *s);
/* State (RX_REQ_*) of a request and, once done, its statistics. */
int rx_server_poll(rx_server *s, uint64_t id, int *state, rx_stats *stats);
/* Server settings: "issue" [1], the issue mode of the requests' handles
 * (rx_set_param "issue"); "issue_threads" (1 .. 64), the host threads that
 * issue a step's blocks; "blocks_per_step" (1 .. 2^20), the blocks of each
 * running request issued per step (one rx_process_blocks call: fewer calls
 * and CDC launches, coarser interleaving).  Their defaults follow the
 * environment's CUDA_DEVICE_MAX_CONNECTIONS (the CUDA context's hardware
 * work queues, which the requests' streams share; 8 unless set before the
 * context is created): 4 threads and 4 blocks at 32 or more queues, else 2
 * threads (at most the host's cores) and 2 blocks at 16, 1 block below.
 * "block_latency" [0]: 1 times every issue call of every request (an event
 * pair on the request's stream around the call's launches; turning it on
 * clears the times kept), read by rx_server_get_block_latency.  Many concurrent
 * requests run best with CUDA_DEVICE_MAX_CONNECTIONS=32.  RX_EINVAL
 * otherwise. */
int rx_server_set_param(rx_server *s, const char *key, double value);
/* Reads a setting above, "running" (1 while the server's loop runs) or a
 * counter: "handles_created",
 * "handles_destroyed", "handle_regrows" (pooled handles reused for a request
 * longer than their buffers, which then grow).  RX_EINVAL for other keys. */
int rx_server_get_param(const rx_server *s, const char *key, double *value);
/* With "block_latency" on: the device time (ms) from the start of each issue
 * call's first launch to the end of its last (one call covers
 * blocks_per_step blocks of a request, and includes the time other requests'
 * work held the device), for the requests retired since it was turned on, in
 * retirement order.  *n = how many are kept; the first min(cap, *n) go to ms
 * (may be NULL when cap = 0). */
int rx_server_get_block_latency(const rx_server *s, double *ms, size_t cap, size_t *n);
/* Memory in use, the most requests ever running at once, steps taken. */
int rx_server_info(rx_server *s, size_t *mem_used, int *max_active, long *steps);
const char *rx_server_last_error(void);

/* Format facts: dims, m (bits per 4D symbol), M (table size). */
int rx_format_info(const rx_handle *h, int *dims, int *m, int *M);

const char *rx_last_error(void);

/* ---- measurement aid -------------------------------------------------------
 * The paper has no counterpart: this measures the denominator of the phase
 * search's roofline.  Issue rate of one FP32 instruction kind on the current
 * device, in lane-instructions per second: kind 0 fma.rn.f32 (FFMA), 1
 * fma.rn.f32x2 (FFMA2, two multiply-adds per lane-instruction), 2 min.f32
 * (FMNMX).  Two blocks of 1024 threads per SM run 8 independent chains per
 * thread for iters x 16 x 8 instructions (one warm-up launch first); *ms
 * (may be NULL) receives the timed launch's device time.  Synchronises its
 * own stream; RX_EINVAL for a bad kind or iters < 1. */
int rx_issue_rate(int kind, int iters, double *lane_instr_per_s, double *ms);

/* ---- single stages (the steps rx_process chains; for tests and custom
 *      pipelines).  All arrays are device memory with a leading [S]. ----- */

/* A1 CDC: overlap-save FFT filtering with conj(H_CD) * H_MF, global
 * framing from sample 0.  in, out: [S][2][n_samples] c64 (out != in).
 * With "precision" 1 or 2, out holds half or bfloat16 (re, im) pairs
 * (4 bytes per sample), as the chain stores its CDC output. */
int rx_cdc(rx_handle *h, const void *in, void *out, size_t n_samples);

/* A2 FIR: y_q[k] = sum_p sum_t conj(h_qp[t]) x_p[2k + D - t], D = (T-1)/2,
 * for k0 <= k < k1.  x: [S][2][n_samples], taps: [S][2][2][T] c64
 * (index [q][p][t]), y: [S][2][k1 - k0].  With "precision" 1 or 2, x and y
 * are half or bfloat16 pairs (the chain's storage); arithmetic is float32. */
int rx_fir(rx_handle *h, const void *x, size_t n_samples, const void *taps,
           size_t k0, size_t k1, void *y);

/* A3 LMS: sequential updates over symbols k0 .. k0 + n_upd - 1 of x,
 * in place on taps [S][2][2][T].  mode 0: CMA; 1: DD-LMS using the phase
 * codes pcode [S][N] (uint16: b | (m mod S) << 8, see rx_unwrap);
 * 2: CMA for updates u0 + i < n_cma, DD after; 3: data-aided LMS with the
 * reference symbols (rx_set_reference) in place of the decisions.
 * passes > 1 repeats the span (start-up). */
int rx_lms(rx_handle *h, const void *x, size_t n_samples, void *taps,
           size_t k0, size_t n_upd, const uint16_t *pcode, int mode,
           int passes, uint64_t u0);

/* A3 training stage on taps [S][2][2][T] (in place), the start-up step of
 * rx_process after CMA: output order and phases from the correlation of the
 * equalised first n_train symbols with the reference, data-aided phase codes
 * (written to pcode, [S][n_train] uint16) and train_passes passes of
 * data-aided LMS.  Needs rx_set_reference. */
int rx_train(rx_handle *h, const void *x, size_t n_samples, void *taps, uint16_t *pcode);

/* A4 BPS: test-phase index b_k for a <= k < e from y [S][2][n_y] (symbols
 * 0 .. n_y - 1 of the stream), windows truncated at n_valid.  b_out:
 * [S][e - a] uint8. */
int rx_bps(rx_handle *h, const void *y, size_t n_y, size_t a, size_t e,
           size_t n_valid, uint8_t *b_out);

/* A4 unwrap + de-rotation: from b [S][e - a] and the carry (m_prev, b_prev)
 * carry_in [S][2] int32, compute the integer unwrap m_k, z_k = y_k *
 * exp(-j phi_k) into z [S][2][e - a], phase codes into pcode [S][e - a],
 * the carry after the range into carry_out [S][2] and the decision-directed
 * noise variance of the range into sigma2 [S] (float64). */
int rx_unwrap(rx_handle *h, const void *y, size_t n_y, const uint8_t *b,
              size_t a, size_t e, const int32_t *carry_in, void *z,
              uint16_t *pcode, int32_t *carry_out, double *sigma2);

/* rx_unwrap without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * while they process -- a real-time thread on which cudaMalloc / cudaFree
 * (which can synchronise the whole device and take unbounded time) is not
 * allowed, or an application whose device memory is owned by another
 * allocator or a fixed budget.  Arguments, layouts and results are those of
 * rx_unwrap; the caller still passes every input and output buffer.
 * Scratch (per-block unwrap increments, noise partial sums, completion
 * tickets) lives in one static device array of 64 KiB compiled into the
 * library; every GPU that loads the library keeps it until the process
 * exits.  S streams x n_blocks blocks need about 12 bytes per (stream,
 * block) plus 4 bytes per stream; a call that would need more than the
 * 64 KiB returns RX_EINVAL without launching anything.  The first call on
 * a device looks up the array's device address with that device current
 * (once per device; make that first call before any stream capture).  The
 * address is kept for the life of the process: after cudaDeviceReset on a
 * device, or under another context than the device's primary one, it is
 * stale, so such a program must not call this entry point again.  All
 * calls share the array and it keeps the last call's contents: the tickets
 * are cleared at the start of every call, so calls that are ordered on the
 * GPU are independent, but calls that overlap on the GPU (different streams,
 * different handles, different host threads) race on the scratch. */
int rx_unwrap_static(rx_handle *h, const void *y, size_t n_y, const uint8_t *b, size_t a,
                     size_t e, const int32_t *carry_in, void *z, uint16_t *pcode,
                     int32_t *carry_out, double *sigma2);

/* A5 LLRs: llr [S][K][m] from z [S][2][K] with noise variance sigma2 [S]
 * (float64, device). */
int rx_demap(rx_handle *h, const void *z, size_t K, const double *sigma2,
             float *llr);

/* ---- Kramers-Kronig front-end (Sec. 2) ------------------------------------
 * The paper's receiver detects a carrier-assisted single-polarisation
 * signal with one photodiode and recovers the field by the Kramers-Kronig
 * relation: ADC codes are converted to floating point with the DC term that
 * the AC-coupled detector lost added back, square root and logarithm give
 * ln|E|, and an overlap-save pair of 1024-point FFTs applies the
 * frequency-domain Hilbert transform that yields the phase; the field is
 * then downconverted.  Format-agnostic: no table is involved.
 *
 * Readings of the steps the paper leaves open (the signal below the
 * carrier: E = A + s e^{-j 2 pi fc n}):
 *   phase      phi = IFFT(G FFT(ln|E|)) per frame, G = +j on the positive
 *              bins, -j on the negative bins, 0 at DC and N/2;
 *   carrier    A = exp(frame mean of ln|E|), subtracted from the field;
 *   output     s[n] = (sqrt(I[n]) e^{j phi[n]} - A) e^{+j 2 pi u / 2^32},
 *              u = fc_step * n mod 2^32, n counted from the stream start;
 *   frames     1024 samples starting at f*(1024 - n_ov) - n_ov/2, the
 *              centre 1024 - n_ov kept; outside the stream the codes are 0
 *              (intensity = the DC term);
 *   clamp      I = max(scale * code + dc, floor) before sqrt and log. */
typedef struct rx_kk rx_kk;
typedef struct {
    int n_ov;            /* frame overlap, even, 0 < n_ov < 1024 (512: the paper's 100 % overlap-save) */
    float floor;         /* intensity clamp (> 0) */
    uint32_t fc_step;    /* carrier offset from the signal centre, cycles per sample * 2^32 */
} rx_kk_params;
/* NULL on error (rx_last_error).  The parameters are copied. */
rx_kk *rx_kk_create(const rx_kk_params *p);
void rx_kk_destroy(rx_kk *k);                       /* NULL-safe; synchronises its stream */
int rx_kk_set_stream(rx_kk *k, void *cuda_stream);
/* codes      device, [n_streams][n] int16 ADC codes (12-bit values or any
 *            int16), 1 <= n_streams <= 256.
 * levels     host, [n_streams][2] float32: photocurrent per code and the DC
 *            term of each stream; copied by value into the launch.
 * field_out  device, [n_streams][n] complex64 (interleaved float pairs),
 *            caller-allocated; every sample is written.
 * Asynchronous on the object's stream.  RX_EINVAL for NULL pointers, n = 0
 * or n_streams out of range. */
int rx_kk_field(rx_kk *k, const int16_t *codes, size_t n_streams, size_t n, const float *levels,
                float *field_out);

/* ---- static frequency-domain equaliser with resampling (Sec. 2) ----------
 * The paper's second FFT pair: a static equaliser of 203 taps, optimised
 * offline from a training sequence whenever acquisition starts, applied in
 * the frequency domain together with the resampling from 4 to 2 samples
 * per symbol.  Readings of what the paper leaves open:
 *   taps       h[t], t < T, at the input rate, centred: z[n] = sum_t h[t] x[n + D - t], D = (T-1)/2;
 *   training   regularised least squares on the symbol instants:
 *              (R + lam I) h = U^H d, R = U^H U, U[i][t] = x[sps*i + D - t]
 *              (0 outside the stream), lam = delta * trace(R) / T, in float64;
 *   applying   overlap-save frames of 1024 input samples starting at
 *              f*(1024 - n_ov) - n_ov/2, spectrum times
 *              H[k] = sum_t h[t] e^{-j 2 pi k (t - D)/1024} on |f| < fs/4
 *              (k < 256 or k >= 768) and 0 elsewhere, inverse FFT, centre
 *              1024 - n_ov samples kept, every second one output. */
typedef struct rx_fde rx_fde;
/* taps odd, 1 <= taps <= n_ov + 1; n_ov a multiple of 4, 0 < n_ov < 1024.  NULL on error. */
rx_fde *rx_fde_create(int taps, int n_ov);
void rx_fde_destroy(rx_fde *e);                     /* NULL-safe; synchronises its stream */
int rx_fde_set_stream(rx_fde *e, void *cuda_stream);
/* x      device, [n] complex64, one stream at the input rate (sps samples per symbol).
 * d      device, [K] complex64, the known symbols; symbol i sits at input sample sps*i.
 * Asynchronous; the taps replace the previous ones.  Scratch of T*T*16
 * bytes is kept by the object. */
int rx_fde_train(rx_fde *e, const float *x, size_t n, const float *d, size_t K, int sps, double delta);
/* taps: host, [T][2] float64 (re, im).  set: replaces the taps (and the
 * response); get: synchronises and copies them out. */
int rx_fde_set_taps(rx_fde *e, const double *taps);
int rx_fde_get_taps(rx_fde *e, double *taps);
/* x  device, [n_streams][n] complex64 (n even); y device, [n_streams][n/2]
 * complex64, caller-allocated.  RX_ESTATE before any taps were set or
 * trained.  Asynchronous. */
int rx_fde_apply(rx_fde *e, const float *x, size_t n_streams, size_t n, float *y);

#ifdef __cplusplus
}
#endif
#endif /* RX_H */
