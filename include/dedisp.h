/*
 * dedisp.h - C ABI of a GB300 (sm_103a) library for incoherent
 * dedispersion, after Barsdell, Bailes, Barnes & Fluke, "Accelerating
 * incoherent dedispersion" (arXiv:1201.5380).
 *
 * What it computes
 *   Direct transform, Sec. 2.1 Eq. 2:
 *       D[d][t] = sum_{c < N_nu} mask[c] * A[c][t + delay(d, c)],
 *   with the per-channel delay of Eq. 3-4:
 *       Delta T(c)   = (k_DM / dtau) * ((nu0 + c*dnu)^-2 - nu0^-2),
 *       delay(d, c)  = round(DM(d) * Delta T(c)),   k_DM = 4.148808e3,
 *   where round() is round-half-up (floor(x + 0.5)) evaluated in IEEE double
 *   on the host, and the kill mask is applied arithmetically (Sec. 2.3).
 *   Sub-band variant, Sec. 4.1 with Eq. (eq:combining_subbands):
 *       S[g][n][t] = sum_{c' < N'} A[nN'+c'][t + delay(gn, nN'+c') - delay(gn, nN')]
 *       D[d][t]    = sum_{n < N_SB} S[g(d)][n][t + delay(d, nN')]
 *   with trials grouped consecutively N'_DM per group and gn the group's
 *   first (lowest) trial, the early-edge alignment of Appendix B.
 *
 * Data layouts
 *   Input: a time-major filterbank.  Row t (t = 0 .. nsamps_out + max_delay
 *   - 1) starts at byte t * in_row_stride_bytes and holds channels
 *   0 .. nchans-1.  For in_nbits = 1, 2 or 4, channel c occupies bits
 *   [(c*nbits) mod 8, +nbits) of byte (c*nbits)/8 of the row, least
 *   significant bits first; in_nbits = 8 is one unsigned byte per channel;
 *   in_nbits = DD_IN_F32 is one little-endian float per channel.
 *   Channel 0 is at frequency nu0 (f0_mhz); channel c at f0_mhz + c*df_mhz.
 *   Output: DM-major, row d (one per trial) of nsamps_out samples starting
 *   at element d * out_row_stride_elems.  Integer input gives uint32 sums
 *   (exact); float input gives float sums (FP32 accumulation).
 *
 * Ownership and threading
 *   Handles are created and destroyed by the library.  Input and output
 *   buffers always belong to the caller; the library never keeps a caller
 *   pointer after a call returns.  A plan binds to the CUDA device that is
 *   current when it is created and must be used with that device current.
 *   A plan, stream or batch handle may be used by one host thread at a time.
 *
 * Errors
 *   Every call returns a dd_status; nothing is thrown across the ABI.  On
 *   an error the output buffer's contents are unspecified (its size is never
 *   exceeded).  Device-side bound checks never trap: they record a flag that
 *   dd_plan_get_device_status returns.
 */
#ifndef GB300_DEDISP_H
#define GB300_DEDISP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DD_ABI_VERSION 1

typedef enum dd_status {
    DD_OK = 0,
    DD_ERR_INVALID_ARG = 1,       /* null handle/pointer, bad size, bad band */
    DD_ERR_NO_DM_LIST = 2,        /* execute before a DM list was set */
    DD_ERR_UNSUPPORTED_NBITS = 3, /* in_nbits not in {1, 2, 4, 8, 32} */
    DD_ERR_INPUT_TOO_SHORT = 4,   /* fewer than nsamps_out + max_delay rows */
    DD_ERR_OOM = 5,               /* device or host allocation failed */
    DD_ERR_CUDA = 6,              /* a CUDA runtime call failed */
    DD_ERR_TIMEOUT = 7,           /* a bounded wait expired */
    DD_ERR_DEVICE_BOUNDS = 8,     /* a kernel clamped an out-of-range index */
    DD_ERR_OVERFLOW = 9,          /* nchans * max sample could exceed uint32 */
    DD_ERR_NOT_READY = 10,        /* request not finished yet */
    DD_ERR_REJECTED = 11          /* admission control refused the request */
} dd_status;

/* in_nbits value for 32-bit float samples */
#define DD_IN_F32 32

/* dd_execute / dd_stream_push flags */
#define DD_DEVICE_PTRS 0x1u /* in and out are device pointers; the call is
                               asynchronous on cuda_stream.  Otherwise they
                               are host pointers and the call copies in,
                               computes, copies out and synchronises. */
#define DD_SUBBAND 0x2u     /* use the two-stage sub-band method (needs
                               dd_plan_set_subband) instead of direct */
#define DD_SCRUNCH 0x4u     /* direct with time-scrunching (needs
                               dd_plan_set_scrunch; device pointers) */
#define DD_TREE 0x8u        /* the piecewise linear tree method (needs
                               dd_plan_set_tree; integer input) */

typedef struct dd_plan_s *dd_plan;
typedef struct dd_stream_s *dd_stream;
typedef struct dd_batch_s *dd_batch;

/* Human-readable name of a status code (static string). */
const char *dd_status_string(dd_status status);

/* ---- plan: the problem statement of Sec. 2.1 (nu0, dnu, dtau, N_nu, DM(d)) */

/* Create a plan for nchans channels sampled every dt_s seconds, channel 0
 * at f0_mhz and channel spacing df_mhz (must be < 0: a descending band with
 * channel 0 the highest frequency, so that every delay of Eq. 3-4 is >= 0;
 * the lowest channel f0_mhz + (nchans-1)*df_mhz must stay > 0).
 * Binds the plan to the current CUDA device (no device memory is touched
 * until the first execute). */
dd_status dd_plan_create(dd_plan *plan, int nchans, double dt_s, double f0_mhz,
                         double df_mhz);

/* Release the plan and every device buffer it owns.  NULL is a no-op. */
void dd_plan_destroy(dd_plan plan);

/* Set the trial DMs (pc cm^-3): ndm >= 1 values, non-negative and
 * non-decreasing.  Copied; rebuilds the delay table of Eq. 4. */
dd_status dd_plan_set_dm_list(dd_plan plan, const double *dms, int ndm);

/* Generate trial DMs on [dm_lo, dm_hi) by the bounded-smearing rule read
 * from Sec. 5.2 (the paper gives only its outcome: 1196 trials for
 * 0 <= DM < 1000 with the HTRU band).  With t_s = dt in us, w =
 * pulse_width_us, nu_c the mean channel frequency in GHz,
 * a = 2 k_DM |dnu| / nu_c^3 * 1e-3 (us per unit DM) and b = a * nchans / 4,
 * DM_0 = dm_lo and DM_{i+1} is the larger root x of
 *   t_s^2 + w^2 + a^2 x^2 + b^2 (x - DM_i)^2 = tol^2 (t_s^2 + w^2 + a^2 DM_i^2).
 * tol > 1 (1.25 in the benchmarks). */
dd_status dd_plan_generate_dm_list(dd_plan plan, double dm_lo, double dm_hi,
                                   double pulse_width_us, double tol);

/* Channel kill mask of Sec. 2.3: nchans bytes, 0 = drop, nonzero = keep.
 * NULL keeps every channel.  Copied. */
dd_status dd_plan_set_killmask(dd_plan plan, const uint8_t *mask);

/* Largest nsamps_out the plan will be executed with; sizes the device
 * workspace up front (execute grows it on demand otherwise). */
dd_status dd_plan_set_gulp(dd_plan plan, int64_t gulp_samples);

/* Enable the sub-band method of Sec. 4.1: chans_per_subband (N') must
 * divide nchans; dms_per_nominal (N'_DM) >= 1.  0, 0 disables it.
 * The stage-1 sums are kept on the device in 8-bit lanes for 1- and 2-bit
 * input when N' * (2^nbits - 1) < 128 and nchans * (2^nbits - 1) < 2^16
 * under the default tiling (dms_per_block 32, words per lane chosen per
 * format), else in 16-bit lanes when N' * max sample < 2^16, else in 32-bit
 * words.  Results are exact in every case. */
dd_status dd_plan_set_subband(dd_plan plan, int chans_per_subband,
                              int dms_per_nominal);

/* Nominal DM of each group of N'_DM trials in the sub-band method: 0 (the
 * default) takes the group's lowest trial, the early-edge alignment App. B
 * analyses; 1 takes its middle trial, which halves the largest DM error
 * between a trial and its nominal DM (App. B) and with it the smearing.
 * Nominal trials stay exact either way. */
dd_status dd_plan_set_subband_alignment(dd_plan plan, int centred);

/* Enable the piecewise linear tree method of Sec. 3.1.1 (execute with
 * DD_TREE): chans_per_subband (N') a power of two from 2 to 128 dividing
 * nchans; 0 disables it.  Stage 1 runs the tree of Sec. 3.1 (Eq.
 * tree_algorithm_first .. last, Theta of Eq. tree_integer_delay, the
 * shuffle Phi of Eq. shuffle) on every sub-band of N' channels, giving the
 * linear trails d' = 0 .. N'-1 of Eq. subband_result; stage 2 combines them
 * by Eq. combining_subbands:
 *     D[d][t] = sum_n S[n][d'_n(d)][t + delay(d, nN')],
 *     d'_n(d) = delay(d, (n+1)N') - delay(d, nN'),
 * with delay(d, N_nu), one channel past the band, from Eq. 3-4 at the band
 * edge (so the band edge f0 + nchans*df must be > 0).  Every trial must
 * satisfy d'_n(d) < N' in every sub-band, i.e. lie below the piecewise
 * diagonal DM of Eq. tree_dm_limit (dd_plan_get_tree_dm_limit); an execute
 * with a trial beyond it returns DD_ERR_INVALID_ARG.  Integer input (1, 2, 4
 * or 8 bits), uint32 output; the input holds nsamps_out + the rows that
 * dd_plan_get_input_rows reports with DD_TREE (the largest stage-2 shift
 * plus N' - 1, the tree's own reach).  Results are approximate by design:
 * the trails are piecewise linear (App. A bounds the smear). */
dd_status dd_plan_set_tree(dd_plan plan, int chans_per_subband);
/* Eq. (tree_dm_limit): (N' - 1/2) / (Delta T(N_nu) - Delta T(N_nu - N')),
 * the DM up to which the basic piecewise linear tree reaches, for
 * N' = chans_per_subband. */
dd_status dd_plan_get_tree_dm_limit(dd_plan plan, int chans_per_subband, double *dm_diag);

/* Bits per output sample of dd_execute: 32 (exact uint32 sums, the
 * default), or 16 / 8 for the scaled low-bit output of Sec. 4.3.  The paper
 * gives no scaling rule; here a scaled sample is
 *   min(sum >> shift, 2^bits - 1),  shift = max(0, bitlen(N_nu * max) - bits),
 * with max the largest input sample (2^nbits - 1) and bitlen(x) the number
 * of bits of x: the top bits of the range the sum can reach, a plain
 * integer operation.  Rows are then uint16 / uint8 with out_row_stride_elems
 * in those elements.  Integer input only; not with DD_SCRUNCH, streams,
 * batches, the server or dd_execute_noalloc (they take uint32 plans). */
dd_status dd_plan_set_output_bits(dd_plan plan, int bits);

/* Time-scrunching (Sec. 2.2): trials beyond twice the diagonal DM (where
 * the top two channels' delays differ by one sample) are dedispersed at
 * half the time resolution, at a quarter beyond four times it, and so on up
 * to max_factor (a power of two, at most 16; 0 turns it off).  A trial of
 * factor s sums s adjacent input samples and uses Eq. 3-4 at s*dt; its output
 * row holds nsamps_out / s samples (the rest of the row is not written).
 * Input of 1, 2 or 4 bits per sample only.  Execute with DD_SCRUNCH. */
dd_status dd_plan_set_scrunch(dd_plan plan, int max_factor);
/* Factor of every trial (1 when scrunching is off). */
dd_status dd_plan_get_scrunch_factors(dd_plan plan, int32_t *factors);
/* Input rows an execute of nsamps_out samples reads with these flags
 * (DD_SUBBAND / DD_SCRUNCH / DD_TREE): nsamps_out + max_delay for direct. */
dd_status dd_plan_get_input_rows(dd_plan plan, int64_t nsamps_out, unsigned flags,
                                 int64_t *rows);

/* Kernel tiling: trials per thread block (16, 32 or 64), the most channels
 * staged per pass (4, 8, 16 or 32; default 32: each trial block stages as
 * many as its windows leave room for in shared memory, a power of two, or
 * for 4- and 8-bit input any multiple of 4) and output words per
 * lane (2, 4, 8 or 16; compiled shapes: 32x4, 64x2, 16x4, 32x2, 32x8 and
 * 32x16 trials x words, the last only where the staged image holds one or
 * two samples a word: float input and the sub-band method's second stage;
 * an execute whose staged format lacks the shape returns DD_ERR_INVALID_ARG).  0
 * keeps the current value.  words_per_lane < 0 (the default) picks it per
 * staged format: 16 for one or two samples a word (float input, 16-bit
 * lanes), 8 for 4- and 8-bit input (8- and 10-bit lanes), 4 for 1- and
 * 2-bit input.
 * The autotuner below sets all three for the format it is given.
 * dd_plan_get_tuning reports 0 words per lane while it is chosen per
 * format. */
dd_status dd_plan_set_tuning(dd_plan plan, int dms_per_block, int chans_per_chunk,
                             int words_per_lane);
dd_status dd_plan_get_tuning(dd_plan plan, int *dms_per_block, int *chans_per_chunk,
                             int *words_per_lane);

/* The chunk geometry of the direct kernel for in_nbits input under the
 * plan's tiling, from its host-built staging tables (no device work): the
 * number of trial blocks, and per block the channels staged per chunk and
 * the window width in 32-bit words, then the launch's dynamic shared
 * memory (its widest block's).  Each block stages as many channels (a power
 * of two, 4 to the tiling's chunk cap; for 4- and 8-bit input any multiple
 * of 4, evened out over the chunks it takes) as its two staging buffers
 * allow in shared memory; when all blocks get the same number they share
 * one width.
 * Pass null arrays to get n_blocks only; the arrays hold n_blocks entries. */
dd_status dd_plan_get_chunk_geometry(dd_plan plan, int in_nbits, int32_t *n_blocks,
                                     int32_t *chans_per_chunk, int32_t *window_words,
                                     size_t *smem_bytes);

/* Time every tiling candidate on nsamps_out synthetic samples of in_nbits
 * and keep the fastest (Sec. 2.3 and 4.3 tuned block shape by hand; this
 * searches the same kind of knobs).  Allocates temporary device buffers;
 * synchronises cuda_stream. */
dd_status dd_plan_autotune(dd_plan plan, int in_nbits, int64_t nsamps_out,
                           void *cuda_stream);

dd_status dd_plan_get_dm_count(dd_plan plan, int32_t *ndm);
/* Copies ndm doubles. */
dd_status dd_plan_get_dm_list(dd_plan plan, double *dms);
/* Largest delay(d, c) of Eq. 4: the input needs nsamps_out + max_delay rows. */
dd_status dd_plan_get_max_delay(dd_plan plan, int32_t *max_delay);
/* Rows beyond nsamps_out that the sub-band path reads:
 * max_{d,c} delay(gn(d), c) - delay(gn(d), n0(c)) + delay(d, n0(c)). */
dd_status dd_plan_get_subband_max_delay(dd_plan plan, int32_t *max_delay);
/* Copies the int32 delay table, ndm x nchans, row d = trial d. */
dd_status dd_plan_get_delay_table(dd_plan plan, int32_t *delays);
/* Synchronises the plan's device and returns (then clears) the OR of the
 * device-side bound flags of every launch since the last call; 0 = clean. */
dd_status dd_plan_get_device_status(dd_plan plan, uint32_t *flags);

/* Kernel timing (tracing): while enabled, every kernel the plan launches is
 * bracketed by CUDA events on its own stream.  get_kernel_timing synchronises
 * on those events and returns the device time (ms) and launch count of one
 * kernel kind since the last reset: kind 0 = corner turn (unpack/transpose
 * into the staged image), 1 = dedispersion kernel (direct, or the first
 * stage of the sub-band and tree methods), 2 = the second stage of the
 * sub-band and tree methods.  reset clears all. */
#define DD_KERNEL_CORNER_TURN 0
#define DD_KERNEL_DEDISP 1
#define DD_KERNEL_STAGE2 2
dd_status dd_plan_set_kernel_timing(dd_plan plan, int enable);
dd_status dd_plan_get_kernel_timing(dd_plan plan, int kind, double *total_ms,
                                    int64_t *launches);
dd_status dd_plan_reset_kernel_timing(dd_plan plan);

/* ---- execute: one gulp */

/* Dedisperse nsamps_out output samples per trial.  The input must hold
 * nsamps_out + max_delay rows (sub-band: + subband max_delay).  out gets
 * ndm rows of nsamps_out samples, row stride out_row_stride_elems
 * (>= nsamps_out).  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  See DD_DEVICE_PTRS for host vs device pointers. */
dd_status dd_execute(dd_plan plan, int64_t nsamps_out, const void *in, int in_nbits,
                     int64_t in_row_stride_bytes, void *out,
                     int64_t out_row_stride_elems, void *cuda_stream, unsigned flags);

/* ---- fixed-scratch execution */

/* Bytes of the fixed device scratch array used by dd_execute_noalloc. */
#define DD_NOALLOC_SCRATCH_BYTES (64u << 20)

/* The direct transform of dd_execute (device pointers, asynchronous on
 * cuda_stream) for callers that must not allocate GPU memory: for example a
 * real-time pipeline that reserves all of its device memory when it starts
 * and cannot let a call allocate (or free, which synchronises the device)
 * in the middle of an observation, or a host framework that owns all of the
 * GPU's memory.  The paper has no counterpart to this call.
 * Everything the kernels need besides the caller's input and output (staged
 * image, trial-block and staging tables, kill mask, status word) lives in one
 * file-scope device array of DD_NOALLOC_SCRATCH_BYTES, which every GPU that
 * loads the library holds until the process exits; the call itself allocates
 * and frees nothing.  The first call on a device looks up the array's device
 * address (set-up).  No call may be captured in a CUDA graph: each copies
 * its tables and kill mask from pageable host memory.
 * Returns DD_ERR_OOM, before launching anything, when the staged image and
 * tables need more than the array (the image takes about nchans *
 * (nsamps_out + max_delay) times the bytes per staged sample: half a byte
 * for 1- and 2-bit input, 1 for 4-bit, 4/3 for 8-bit (three samples a
 * word), 4 for float input).  The output rows are uint32 (float for float
 * input): a plan with scaled output (dd_plan_set_output_bits below 32) is
 * rejected with DD_ERR_INVALID_ARG.
 * All calls share the array and each starts by reloading it: calls whose work
 * overlaps on the GPU (other streams or threads) race, so the caller must
 * serialise them.  Its device-side bound flags are read with
 * dd_noalloc_get_device_status, not dd_plan_get_device_status. */
dd_status dd_execute_noalloc(dd_plan plan, int64_t nsamps_out, const void *in_dev,
                             int in_nbits, int64_t in_row_stride_bytes, void *out_dev,
                             int64_t out_row_stride_elems, void *cuda_stream);
/* The device-side bound flags (the dd_plan_get_device_status bits) of the
 * latest dd_execute_noalloc call on the current device: waits for
 * cuda_stream (the stream that call used; NULL = the legacy default stream)
 * to finish, then copies the 4-byte status word out of the scratch array.
 * It allocates and frees nothing and does not clear the word (the next
 * call resets it); 0 = clean.  DD_ERR_INVALID_ARG when flags is NULL;
 * CUDA errors of the wait or the copy are returned as their dd_status. */
dd_status dd_noalloc_get_device_status(void *cuda_stream, uint32_t *flags);

/* ---- streaming: consecutive gulps of one beam (the overlap of Eq. 2) */

/* A stream keeps the last max_delay input rows of its beam resident on the
 * device, so that pushed gulps are dedispersed as one continuous series:
 * the concatenation of every push's output equals dd_execute over the
 * concatenated input.  Output sample k of the series needs input rows up
 * to k + max_delay, so outputs lag the input by max_delay samples.
 * max_gulp bounds nsamps_in per push.  The plan must outlive the stream. */
dd_status dd_stream_create(dd_stream *stream, dd_plan plan, int in_nbits,
                           int64_t max_gulp);
void dd_stream_destroy(dd_stream stream);

/* Append nsamps_in input rows and write every output sample that became
 * computable (*nsamps_out of them, nsamps_in once the stream is primed) to
 * out (row stride out_row_stride_elems, capacity >= nsamps_in per row). */
dd_status dd_stream_push(dd_stream stream, const void *in, int64_t nsamps_in,
                         int64_t in_row_stride_bytes, void *out,
                         int64_t out_row_stride_elems, int64_t *nsamps_out,
                         void *cuda_stream, unsigned flags);

/* Samples pushed and produced so far. */
dd_status dd_stream_position(dd_stream stream, int64_t *samples_in,
                             int64_t *samples_out);

/* Checkpoint: the stream state is (samples in, samples out, resident tail
 * rows).  snapshot_size gives the bytes needed; snapshot copies the state
 * into a host buffer (synchronising); restore loads one written by a stream
 * of the same plan shape and nbits. */
dd_status dd_stream_snapshot_size(dd_stream stream, int64_t *bytes);
dd_status dd_stream_snapshot(dd_stream stream, void *host_buf, int64_t bytes);
dd_status dd_stream_restore(dd_stream stream, const void *host_buf, int64_t bytes);

/* ---- batch: pushes of several streams in one persistent launch */

/* Collects stream pushes (device pointers only) and runs the transform of
 * all of them in a single launch: the work of every beam - different
 * channel counts, gulp lengths and DM lists, same in_nbits - is one list
 * of (beam, trial block, time tile) items.  Results equal per-stream
 * dd_stream_push bit for bit. */
dd_status dd_batch_create(dd_batch *batch);
void dd_batch_destroy(dd_batch batch);
dd_status dd_batch_clear(dd_batch batch);
dd_status dd_batch_add(dd_batch batch, dd_stream stream, const void *in_dev,
                       int64_t nsamps_in, int64_t in_row_stride_bytes, void *out_dev,
                       int64_t out_row_stride_elems);
/* Launch everything added since the last clear on cuda_stream
 * (asynchronous); nsamps_out[i] receives the outputs of the i-th add. */
dd_status dd_batch_launch(dd_batch batch, void *cuda_stream, int64_t *nsamps_out);

/* ---- graph: a batch's launch captured once, replayed gulp after gulp
 *
 * In steady-state streaming every gulp of a batch does the same GPU work
 * (appends, corner turns, one persistent launch, tail moves) on the same
 * buffers, apart from each stream's two tail buffers, which swap roles every
 * push.  dd_batch_graph_create records the batch's current adds as two CUDA
 * graphs (one per tail-buffer role) and dd_batch_graph_launch replays the
 * one that matches, then advances the streams as dd_batch_launch would, so
 * a gulp costs one graph launch instead of dozens of calls.
 * Requirements: every stream of the batch is primed (its overlap tail is
 * full: it has taken at least max_delay input rows), the same adds (the
 * same device buffers and gulp sizes) were launched once with
 * dd_batch_launch, which sizes the buffers the capture reuses, and neither
 * the batch, its streams, their plans nor the buffers change while the
 * graph is used; the caller refills the input buffers between replays.
 * Returns DD_ERR_INVALID_ARG when a stream is not primed. */
typedef struct dd_batch_graph_s *dd_batch_graph;
dd_status dd_batch_graph_create(dd_batch_graph *graph, dd_batch batch);
/* Replay on cuda_stream (asynchronous); nsamps_out[i] receives the outputs
 * of the i-th add. */
dd_status dd_batch_graph_launch(dd_batch_graph graph, void *cuda_stream, int64_t *nsamps_out);
void dd_batch_graph_destroy(dd_batch_graph graph);

/* ---- serving: gulps of many beams as they arrive (continuous batching)
 *
 * The paper processes fixed blocks one at a time and has no serving layer;
 * this engine applies the streaming transform above to many beams at once.
 * A server owns one device arena, allocated when it is created, from which
 * each admitted gulp takes an input buffer and an output buffer.  Gulps are
 * queued by dd_server_submit and admitted by dd_server_step as in-flight
 * launches retire and arena space frees up: at most one gulp per beam per
 * launch, a beam's gulps strictly in submission order, at most max_batch
 * gulps per launch and max_inflight launches queued on the GPU.  Each launch
 * copies its inputs in on a copy stream, runs every admitted beam's
 * transform as one batched persistent launch (dd_batch_launch) on the
 * compute stream, and copies outputs out on a second copy stream, so the
 * copies of one launch overlap the compute of another.  Results are those
 * of dd_stream_push on the same beam, bit for bit. */
typedef struct dd_server_s *dd_server;

/* Completed request, as returned by dd_server_poll. */
typedef struct {
  uint64_t request;     /* id returned by dd_server_submit */
  int beam;             /* beam id returned by dd_server_add_beam */
  int status;           /* dd_status of the request */
  int64_t nsamps_out;   /* output samples per trial (0 while the beam's
                           overlap tail is still filling) */
  const void *out_dev;  /* device output rows (uint32, or float for 32-bit
                           input), row stride out_stride; valid until
                           dd_server_release; null when copied to host_out */
  int64_t out_stride;   /* elements */
  double latency_ms;    /* dd_server_submit -> output ready on the GPU (or
                           in host_out when one was given) */
} dd_request_info;

/* Create a server on the current device with an arena of arena_bytes
 * (allocated here, once), at most max_batch (1..32) gulps per launch and
 * max_inflight (1..8) launches queued on the GPU. */
dd_status dd_server_create(dd_server *server, size_t arena_bytes, int max_batch,
                           int max_inflight);
/* Waits for every launch in flight (without a deadline: the arena cannot
 * be freed under running work; call dd_server_drain first to find out
 * whether the GPU still answers), then frees the server, its streams and its
 * arena (plans stay with the caller). */
void dd_server_destroy(dd_server server);

/* Deadline of the server's host waits, in milliseconds (0, the default: no
 * deadline).  A wait that reaches it returns DD_ERR_TIMEOUT and leaves the
 * launch in flight, where a later dd_server_step or dd_server_drain
 * retires it once it ends: the server stays usable.  The deadline guards
 * the host against a GPU or driver that stops answering; the kernels' own
 * waits are bounded on the device. */
dd_status dd_server_set_timeout(dd_server server, double timeout_ms);

/* Wait for every launch in flight and retire it, within the server's
 * deadline (DD_ERR_TIMEOUT when launches are still running at it). */
dd_status dd_server_drain(dd_server server);

/* Queue a pause of ms milliseconds (at most 60 s) on the compute stream
 * behind the transform of the next launch, before its completion is
 * signalled.  The pause is a host callback in the stream, with no device
 * work: it makes a launch late on purpose, so that deadlines and the
 * scheduler's handling of slow launches can be exercised without disturbing
 * the GPU.  (A request with host_out in pageable memory makes the launch's
 * own output copy wait on the host, pause included.) */
dd_status dd_server_pause_next_launch(dd_server server, double ms);

/* Register a beam: its plan (band, DM list; must outlive the server), input
 * bits and largest gulp.  The beam keeps its overlap tail on the device. */
dd_status dd_server_add_beam(dd_server server, dd_plan plan, int in_nbits, int64_t max_gulp,
                             int *beam);

/* Queue one gulp of nsamps_in rows (host memory, row stride
 * in_row_stride_bytes; page-locked memory lets the copy run asynchronously).
 * in_host must stay valid, unchanged, until the request completes.  host_out
 * (optional, null for device output) receives the output rows with row
 * stride out_row_stride_elems >= nsamps_in.  Non-blocking.  Returns
 * DD_ERR_REJECTED when the gulp's buffers could never fit in the arena. */
dd_status dd_server_submit(dd_server server, int beam, const void *in_host, int64_t nsamps_in,
                           int64_t in_row_stride_bytes, void *host_out,
                           int64_t out_row_stride_elems, uint64_t *request);

/* One scheduling pass: retire launches that finished, admit queued gulps
 * and launch them.  With wait != 0 and nothing admissible it first waits
 * for the oldest launch in flight, at most the server's deadline
 * (DD_ERR_TIMEOUT if it is still running then).  *admitted (may be null)
 * receives the gulps launched by this pass. */
dd_status dd_server_step(dd_server server, int wait, int *admitted);

/* Up to max completed requests, oldest first; *n receives the count. */
dd_status dd_server_poll(dd_server server, dd_request_info *out, int max, int *n);

/* Copy a completed request's device output into host rows of stride
 * host_row_stride_elems (synchronous). */
dd_status dd_server_copy_out(dd_server server, uint64_t request, void *host_dst,
                             int64_t host_row_stride_elems);

/* Return a completed request's device output to the arena.  Requests that
 * had a host_out are forgotten once polled and need no release. */
dd_status dd_server_release(dd_server server, uint64_t request);

/* Queued, in-flight and completed-but-unreleased requests, and arena bytes
 * in use (any pointer may be null). */
dd_status dd_server_stats(dd_server server, int *queued, int *inflight, int *completed,
                          size_t *arena_used);

/* ---- measurement */

/* Integer-add throughput of the current device, measured by a kernel of
 * independent 32-bit add chains (counted one per scalar add); the compute
 * roof of the roofline.  Synchronises. */
dd_status dd_probe_int_add(int64_t adds_per_thread, void *cuda_stream,
                           double *adds_per_second, double *kernel_ms);

#ifdef __cplusplus
}
#endif

#endif /* GB300_DEDISP_H */
