/*
 * corr.h -- C ABI of the GB300 X-engine library (libcorr.so).
 *
 * The library implements the cross-multiply-and-accumulate stage of an FX
 * correlator for 4+4-bit complex channelised voltages: for every fine
 * frequency channel f and every input pair 0 <= j <= i < N it accumulates
 *
 *     V_ij(f) = sum_t x_i(t,f) * conj(x_j(t,f))                       (1)
 *
 * over an integration and emits the packed lower triangle including the
 * autocorrelations.  Eq. 3 (Section 2) is the per-channel product of two
 * spectra; Section 3.4.2 integrates the products over a time I on the GPU;
 * Appendix C ("GPU Output") fixes the packed-triangle output.  The arithmetic
 * here is exact integer arithmetic, so every result equals the int64
 * reference sum bit for bit.
 *
 * Conventions shared by every call below
 * -------------------------------------
 * Voltage input (Appendix A "Data Format", Appendix C "GPU Input"):
 *   uint8 volt[n_time][n_chan][n_inputs], one byte per complex sample, real
 *   part = high nibble (bits 7..4), imaginary part = low nibble (bits 3..0),
 *   each 4-bit two's complement (-8..7).  The input index is
 *   n = 2*station + polarisation; the library is agnostic to input order
 *   (Appendix C: the GPU correlates in whatever order the inputs arrive).
 *   Nibble code 8 is the paper's "invalid" marker: by default it decodes as
 *   -8; with CORR_ZERO_INVALID a sample with either nibble equal to 8 is
 *   treated as 0 + 0i.
 *
 * Visibility output:
 *   int32 vis[n_chan][P][2], P = N(N+1)/2, element (i, j), j <= i, at index
 *   i(i+1)/2 + j, holding (Re, Im) of (1) with x_i unconjugated.
 *
 * Memory ownership: the caller owns every buffer it passes.  Device buffers
 * are plain device pointers (cudaMalloc or a framework allocator); the
 * library never frees or retains them beyond the call, except the workspace
 * bound with corr_bind_workspace, which it uses until the context is
 * destroyed or another workspace is bound.  The library itself allocates only
 * host memory for the context object; every device byte it touches is the
 * caller's.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls enqueue work and return without synchronising the host,
 * except corr_sync, corr_get_state and corr_set_state which synchronise the
 * given stream.  Argument and state errors are detected on the host and
 * returned synchronously before anything is enqueued.
 *
 * Errors: every call returns a corr_status (0 = success, negative = error)
 * and records it for corr_last_error() in the calling thread.  No call
 * aborts, exits or prints.
 */
#ifndef CORR_H
#define CORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum corr_status {
    CORR_OK = 0,
    CORR_E_ARG = -1,          /* invalid argument (NULL, size, alignment)        */
    CORR_E_STATE = -2,        /* call not valid in the context's current state   */
    CORR_E_OVERFLOW = -3,     /* integration would exceed n_time_per_int         */
    CORR_E_NOMEM = -4,        /* host allocation failed / workspace too small    */
    CORR_E_BUDGET = -5,       /* request exceeds a caller-set memory budget      */
    CORR_E_CUDA = -6,         /* a CUDA runtime call failed                      */
    CORR_E_TIMEOUT = -7,      /* a bounded device-side wait gave up              */
    CORR_E_UNSUPPORTED = -8   /* shape or path not supported on this device      */
} corr_status;

/* X-engine implementations (all bit-exact). */
typedef enum corr_path {
    CORR_PATH_AUTO = 0,       /* fastest supported path for the shape            */
    CORR_PATH_CUDACORE = 1,   /* register-tiled dp4a on CUDA cores (baseline)    */
    CORR_PATH_MMA_I8 = 2,     /* int8 warp-level mma.sync, int32 accumulation    */
    CORR_PATH_TC_FP8 = 3      /* tcgen05 E4M3 tensor cores, FP32 in TMEM         */
} corr_path;

/* Context flags (corr_set_flags). */
#define CORR_ZERO_INVALID 1u

typedef struct corr_ctx corr_ctx;

/* ---------------------------------------------------------------- context -- */

/*
 * Create a context for an array of n_inputs inputs and n_chan fine channels
 * integrating at most n_time_per_int samples per dump.  Binds to the current
 * CUDA device.  Returns NULL on error (corr_last_error() tells which):
 * CORR_E_ARG if any size is < 1 or 128 * n_time_per_int >= 2^31 (the int32
 * bound for |Re V_ij| when every component is -8), CORR_E_NOMEM if the host
 * context cannot be allocated, CORR_E_CUDA if no device is usable.
 */
corr_ctx *corr_create(int n_inputs, int n_chan, int n_time_per_int);

/* Release the context (host memory only; the workspace stays the caller's). */
int corr_destroy(corr_ctx *ctx);

/* Select the implementation.  CORR_E_UNSUPPORTED if the path cannot run on
 * this device (CORR_PATH_TC_FP8 needs an sm_103 device).  The tensor-core
 * path reads the voltage rows through TMA, which needs rows on 16-byte
 * boundaries: with n_inputs % 16 != 0 each call's samples are first copied
 * into rows of round_up(n_inputs, 16) bytes in the workspace (up to 4 GiB:
 * a whole integration where it fits, else chunks of a multiple of 64
 * samples), and in a batch such arrays are
 * correlated in launches of their own.  AUTO picks the tensor-core path from
 * 64 inputs on.  Valid only between integrations (corr_samples() == 0), else
 * CORR_E_STATE.  The default is CORR_PATH_AUTO. */
int corr_set_path(corr_ctx *ctx, int path);

/* Tile shape (Section 3.4.2, Eq. 4: the tile sets the arithmetic intensity).
 * CUDA-core path: 32 or 64 inputs per side.  tcgen05 path: 128 = every work
 * item one 128 x 128 tile pair (one TMEM accumulator each, so an item's
 * epilogue overlaps the next item's MMAs); 256 = pair items, a diagonal tile
 * and the tile left of it as one 256-row column of the triangle (one
 * conversion of the shared tile feeds two accumulators).  0 chooses by shape:
 * 32 when n_inputs <= 32 on the CUDA-core path; pair items from 64 stages
 * of 64 samples per launch on the tcgen05 path.  A value that does not apply
 * to the context's path is ignored by it.  Any other value: CORR_E_ARG.  Only
 * between integrations (CORR_E_STATE). */
int corr_set_tile(corr_ctx *ctx, int tile);

/* The path that accumulate calls will run (AUTO resolved). */
int corr_get_path(const corr_ctx *ctx);

/* Set CORR_* flags (only between integrations, else CORR_E_STATE). */
int corr_set_flags(corr_ctx *ctx, unsigned flags);

/* Bytes of device workspace the context needs for its current path (int32
 * accumulators, unpacked operand staging, host-transfer staging, status
 * word).  The caller allocates at least this many bytes, 256-byte aligned. */
size_t corr_workspace_bytes(const corr_ctx *ctx);

/* The same figure for a shape, without a context or a device (for planning
 * and admission control); 0 with CORR_E_ARG on invalid sizes. */
size_t corr_workspace_bytes_for(int n_inputs, int n_chan, int n_time_per_int);

/* Give the context its workspace (device pointer, caller-owned).  Resets the
 * integration (the accumulators are treated as zero).  CORR_E_ARG if d_ws is
 * NULL, not 256-byte aligned, or bytes < corr_workspace_bytes(). */
int corr_bind_workspace(corr_ctx *ctx, void *d_ws, size_t bytes);

/* ------------------------------------------------------------ integration -- */

/*
 * Add n_time samples of every channel and input to the running integration:
 * d_volt is a device pointer to uint8 [n_time][n_chan][n_inputs] (layout
 * above).  n_time == 0 is a no-op.  CORR_E_OVERFLOW (nothing enqueued) if
 * corr_samples() + n_time > n_time_per_int; CORR_E_STATE if no workspace is
 * bound; CORR_E_ARG on NULL d_volt or negative n_time, and on the tensor-core
 * path with n_inputs % 16 == 0 (read in place by TMA) if d_volt is not
 * 16-byte aligned.  Asynchronous.
 */
int corr_accumulate(corr_ctx *ctx, const uint8_t *d_volt, int n_time, void *stream);

/*
 * Write the current integration's packed triangle to d_vis (device int32
 * [n_chan][P][2]) and start a new integration.  Valid at any time, including
 * on a partial or empty integration (an empty one dumps zeros).
 */
int corr_dump(corr_ctx *ctx, int32_t *d_vis, void *stream);

/* Samples accumulated since the last dump (host-side count). */
long long corr_samples(const corr_ctx *ctx);

/*
 * One whole integration in one call: correlate n_time samples of d_volt
 * (device, [n_time][n_chan][n_inputs]) and write their packed triangle to
 * d_vis (device int32 [n_chan][P][2]), as corr_accumulate on an empty
 * integration followed by corr_dump would, but with the X-engine epilogue
 * storing straight into d_vis (Section 3.4.3: the products of one
 * integration are written out once) -- no accumulator pass and no copy.
 * The context's running integration and accumulators are not touched.
 * n_time 0 writes zeros; n_time above n_time_per_int is CORR_E_OVERFLOW.
 */
int corr_integrate(corr_ctx *ctx, const uint8_t *d_volt, int n_time, int32_t *d_vis, void *stream);

/*
 * corr_integrate plus the incoherent beam of the same samples (Section 3.4:
 * the XMAC's other mode, the total power of all inputs per channel and
 * sample, as corr_incoherent_beam computes it): d_beam (device int32
 * [n_time / n_avg][n_chan], overwritten) gets, per channel and block of n_avg
 * consecutive samples, the sum over inputs and samples of re^2 + im^2.  On
 * the tensor-core path the beam is formed by the X-engine's own unpack of the
 * voltages (no second pass over them): d_beam is zeroed on `stream`, then
 * each 128-input tile adds its power once.  On the other paths the
 * stand-alone beam kernel runs after the X-engine.  CORR_E_ARG on NULL
 * d_vis or d_beam, n_avg < 1, n_time % n_avg != 0 or 128 n_avg n_inputs >=
 * 2^31 (an int32 beam value could overflow); other errors as corr_integrate.
 */
int corr_integrate_beam(corr_ctx *ctx, const uint8_t *d_volt, int n_time, int32_t *d_vis, int32_t *d_beam,
                        int n_avg, void *stream);

/*
 * End-to-end variants over HOST buffers: h_volt is host memory
 * [n_time][n_chan][n_inputs] (pinned memory gives full copy bandwidth); the
 * library copies it in chunks of up to 500 samples through a ring of three
 * device staging buffers in the workspace, on its own copy stream, so that
 * each chunk's host-to-device copy overlaps the correlation of the previous
 * ones on `stream`.  h_volt must stay valid and unmodified until `stream`
 * has passed the call.
 *
 * corr_dump_host copies the triangle to host memory h_vis (int32
 * [n_chan][P][2]) and starts a new integration.  The device-to-host copy runs
 * on the context's own output stream, after the work already enqueued on
 * `stream`, so the next integration's correlation overlaps it (the first
 * later write of the accumulators waits for it).  h_vis is complete once
 * corr_sync(ctx, stream) has returned (or the device is synchronised); it
 * must not be read or reused before then.
 */
int corr_accumulate_host(corr_ctx *ctx, const uint8_t *h_volt, int n_time, void *stream);
int corr_dump_host(corr_ctx *ctx, int32_t *h_vis, void *stream);

/* Synchronise `stream` and the context's output stream (host dumps), then
 * report a device-side error recorded by a kernel
 * of this context (CORR_E_TIMEOUT if a bounded wait gave up) or CORR_OK.  The
 * error is cleared once reported.  After CORR_E_TIMEOUT the accumulators hold
 * a partial sum: dump (and discard) or restore a state before going on. */
int corr_sync(corr_ctx *ctx, void *stream);

/* Limit, in SM clock cycles, of every wait inside the tensor-core kernel
 * (between its producer, converter, MMA and epilogue roles).  A wait that
 * exceeds it records CORR_E_TIMEOUT (reported by corr_sync), and the kernel
 * drains its copies and MMAs, frees its tensor memory and returns instead of
 * hanging.  0 restores the default (2^31 cycles, about one second). */
int corr_set_wait_limit(corr_ctx *ctx, long long cycles);

/* Fault injection for tests, made without any GPU fault: with
 * CORR_INJECT_STALL the next tensor-core launch of this context first waits
 * on a barrier that nothing ever completes, so its bounded wait expires and
 * the launch ends with CORR_E_TIMEOUT.  One-shot; CORR_INJECT_NONE clears. */
#define CORR_INJECT_NONE 0u
#define CORR_INJECT_STALL 1u
int corr_debug_inject(corr_ctx *ctx, unsigned what);

/* ------------------------------------------------------ checkpoint/resume -- */

/* Size of the serialised integration state: a 32-byte header (magic, N, F,
 * samples) followed by the int32 accumulators [n_chan][P][2]. */
size_t corr_state_bytes(const corr_ctx *ctx);

/* Copy the running integration to host memory h_buf (synchronises stream). */
int corr_get_state(corr_ctx *ctx, void *h_buf, size_t bytes, void *stream);

/* Restore an integration saved by corr_get_state from a context of the same
 * shape (CORR_E_ARG on a size or header mismatch; synchronises stream). */
int corr_set_state(corr_ctx *ctx, const void *h_buf, size_t bytes, void *stream);

/* ------------------------------------------------------------- stand-alone -- */

/*
 * Unpack and corner-turn (the GPU form of the host-side reordering and 4-to-8
 * bit promotion of Section 3.4.1 and Appendix C "GPU Input"): reads d_volt
 * uint8 [n_time][n_chan][n_inputs] and writes d_out int8
 * [n_chan][n_inputs][n_time][2] (real, imaginary), time contiguous per input.
 * flags: CORR_ZERO_INVALID or 0.  d_out must hold 2*n_time*n_chan*n_inputs
 * bytes.  Asynchronous.
 */
int corr_unpack(const uint8_t *d_volt, int n_time, int n_chan, int n_inputs,
                int8_t *d_out, unsigned flags, void *stream);

/* ------------------------------------------------------------------- batch -- */

/*
 * Several arrays of uneven size correlated together (the MWA correlator runs
 * one X-engine per GPU over a fixed set of channels, Section 3.4; here one
 * GPU serves several arrays).  Arrays on the tensor-core path are correlated
 * by ONE persistent launch (up to CORR_BATCH_TC_GROUP arrays per launch; the
 * work items of all of them, longest first, shared by every SM); arrays on
 * other paths get their own kernels on the same stream.
 */
#define CORR_BATCH_MAX 16
#define CORR_BATCH_TC_GROUP 4

typedef struct corr_array_desc {
    int n_inputs;        /* N */
    int n_chan;          /* F */
    int n_time_per_int;  /* samples per integration (cap) */
    int path;            /* CORR_PATH_* for this array; AUTO picks per shape */
    unsigned flags;      /* CORR_ZERO_INVALID or 0 */
    int tile;            /* tile shape (corr_set_tile), 0 = by shape */
} corr_array_desc;

typedef struct corr_batch corr_batch;

/* NULL on error (corr_last_error): CORR_E_ARG for n_arrays outside
 * [1, CORR_BATCH_MAX] or an invalid descriptor (same rules as corr_create),
 * CORR_E_UNSUPPORTED if a requested path cannot run its shape. */
corr_batch *corr_batch_create(int n_arrays, const corr_array_desc *descs);
int corr_batch_destroy(corr_batch *b);

/* Device workspace for all arrays (one caller-owned, 256-byte aligned block). */
size_t corr_batch_workspace_bytes(const corr_batch *b);
int corr_batch_bind_workspace(corr_batch *b, void *d_ws, size_t bytes);

/* Resolved path of array a (CORR_PATH_*), or a negative status. */
int corr_batch_path(const corr_batch *b, int a);

/* Samples in array a's running integration. */
long long corr_batch_samples(const corr_batch *b, int a);

/* The context of array a (owned by the batch; valid until corr_batch_destroy):
 * for corr_profile_*, corr_get_state / corr_set_state and corr_sync. */
corr_ctx *corr_batch_array(corr_batch *b, int a);

/*
 * Accumulate d_volt[a] (device, [n_time[a]][F_a][N_a]) into array a for every
 * a with d_volt[a] != NULL and n_time[a] > 0.  All checks happen before
 * anything is enqueued: CORR_E_OVERFLOW if any array would exceed its cap.
 */
int corr_batch_accumulate(corr_batch *b, const uint8_t *const *d_volt, const int *n_time,
                          void *stream);

/* Dump every array a with d_vis[a] != NULL (device int32 [F_a][P_a][2]). */
int corr_batch_dump(corr_batch *b, int32_t *const *d_vis, void *stream);

/*
 * corr_integrate for every array a with d_vis[a] != NULL, the tensor-core
 * arrays sharing one persistent launch: array a's n_time[a] samples of
 * d_volt[a] become the triangle in d_vis[a].  Running integrations are not
 * touched.  All checks happen before anything is enqueued.
 */
int corr_batch_integrate(corr_batch *b, const uint8_t *const *d_volt, const int *n_time,
                         int32_t *const *d_vis, void *stream);

/* corr_sync for every array of the batch. */
int corr_batch_sync(corr_batch *b, void *stream);

/*
 * Capture one whole integration -- corr_batch_integrate(d_volt, n_time,
 * d_vis) -- into an executable CUDA graph (returned as an opaque handle in
 * *graph_exec).  Each corr_graph_launch replays it on the captured buffers:
 * whatever d_volt holds then becomes the triangles in d_vis.  The batch's
 * running integrations are not involved.  `stream` must not be the legacy
 * default stream (CORR_E_ARG).
 * Profiling events recorded during capture become graph nodes; launches that
 * cannot be timed from them are left out of corr_profile_read's "timed" and
 * "ms" (launch counts cover the capture only).
 */
int corr_batch_graph_capture(corr_batch *b, const uint8_t *const *d_volt, const int *n_time,
                             int32_t *const *d_vis, void *stream, void **graph_exec);
int corr_graph_launch(void *graph_exec, void *stream);
int corr_graph_destroy(void *graph_exec);

/* --------------------------------------------------- other modes and output -- */

/*
 * Incoherent beam (Section 3.4: one of the XMAC's modes besides correlation):
 * the total power of all inputs per channel and sample, summed over n_avg
 * consecutive samples:
 *
 *   d_beam[k][f] = sum over t in [k n_avg, (k+1) n_avg), over n < n_inputs, of |x_n(t,f)|^2
 *
 * d_volt: device uint8 [n_time][n_chan][n_inputs] (Appendix A encoding, real
 * part in the high nibble); d_beam: device int32 [n_time / n_avg][n_chan].
 * flags: CORR_ZERO_INVALID (samples with a nibble code 8 contribute 0) or 0.
 * CORR_E_ARG if n_time is not a multiple of n_avg or 128 n_avg n_inputs
 * reaches 2^31 (the int32 bound).  Asynchronous, allocates nothing.
 */
int corr_incoherent_beam(const uint8_t *d_volt, int n_time, int n_chan, int n_inputs, int n_avg,
                         unsigned flags, int32_t *d_beam, void *stream);

/*
 * Packet ingest (Appendix A "Data Format", Appendix B): one 50 ms bank of PFB
 * packets into the voltage block the X-engine reads.
 *
 * Packet (CORR_PKT_BYTES = 264): header word 0x0800; word two: sec_tick
 * (bit 0), pfb_id (bits 4-5), mgt_id (bits 6-8), mgt_bank (bits 9-13); word
 * three: mgt_frame (bits 0-8), mgt_group (bits 9-10), mgt_channel (bits
 * 11-15); 256 sample bytes; the XOR of the 128 data words.  Words are most
 * significant byte first.  The bit positions and mgt_frame's 9-bit width are
 * readings: the appendix lists the fields but not their placement, and gives
 * mgt_frame 5 bits for the values 0-499.  Sample byte 64 f2 + k is fine
 * channel 128 mgt_channel + 16 mgt_id + 4 mgt_group + f2 and input
 * 64 pfb_id + k (PFB order, the X-engine's input order).
 *
 * d_packets: device, n_packets x 264 bytes, 4-byte aligned, any order.
 * d_volt: device uint8 [CORR_PKT_FRAMES][CORR_PKT_CHANNELS][CORR_PKT_INPUTS],
 * 16-byte aligned, fully written: sample t of the bank is mgt_frame t.
 * d_seen: device scratch of CORR_PKT_SEEN_BYTES.  d_counters: device int32
 * [CORR_PKT_COUNTERS], zeroed then filled: good packets, rejected packets by
 * reason (header, checksum, field: mgt_bank != bank, mgt_channel >= 24,
 * mgt_frame >= 500, or sec_tick on a packet other than the second's first),
 * repeated slots (a repeated packet's bytes replace the earlier ones), and
 * slots (frame, four channels, PFB) no good packet filled, whose 256 bytes
 * are written as 0x88 (code 8 in both parts: invalid, see CORR_ZERO_INVALID).
 * Asynchronous; allocates nothing.
 */
#define CORR_PKT_BYTES 264
#define CORR_PKT_FRAMES 500
#define CORR_PKT_CHANNELS 3072
#define CORR_PKT_INPUTS 256
#define CORR_PKT_SLOTS (CORR_PKT_FRAMES * (CORR_PKT_CHANNELS / 4) * 4)
#define CORR_PKT_SEEN_BYTES CORR_PKT_SLOTS   /* one mark byte per slot */
#define CORR_PKT_GOOD 0
#define CORR_PKT_BAD_HEADER 1
#define CORR_PKT_BAD_CHECKSUM 2
#define CORR_PKT_BAD_FIELD 3
#define CORR_PKT_DUPLICATE 4
#define CORR_PKT_MISSING 5
#define CORR_PKT_COUNTERS 6
int corr_ingest_packets(const uint8_t *d_packets, long long n_packets, int bank, uint8_t *d_volt, void *d_seen,
                        int32_t *d_counters, void *stream);

#define CORR_REMAP_MAX_DUMPS 8
/*
 * Output remap (Appendix C, "GPU Output"): the X-engine correlates the inputs
 * in PFB order, so its triangle is over PFB positions; this writes the
 * products per station pair in natural input order, conjugating those the
 * triangle holds only as conjugates, and optionally integrates further over
 * f_avg adjacent channels and over n_dumps consecutive dumps (Section 3.4.3:
 * "integrate by a factor of two in each dimension" is f_avg = n_dumps = 2):
 *
 *   d_out[g][s1(s1+1)/2 + s2][p1][p2][re,im] = sum over d < n_dumps and the
 *       f_avg channels f of group g of  V_{2 s1 + p1, 2 s2 + p2}(f),   s2 <= s1
 *
 * d_tri: host array of n_dumps (<= CORR_REMAP_MAX_DUMPS) device pointers to
 * int32 [n_chan][n_inputs(n_inputs+1)/2][2] triangles as corr_dump writes
 * them.  d_nat_of_pfb: device int32 [n_inputs], the natural input carried at
 * each PFB position, or NULL for the Appendix A order (position k of each
 * PFB's 64 carries input (k mod 4) * 16 + k div 4; PFB blocks concatenated,
 * Appendix B), which needs n_inputs % 64 == 0.  Reading: natural input a is
 * station a / 2, polarisation a % 2.  d_out: device int32
 * [n_chan / f_avg][S(S+1)/2][2][2][2], 16-byte aligned, S = n_inputs / 2 (33024 complex
 * products per channel at 256 inputs).  Sums are int32: the caller keeps
 * n_dumps f_avg 128 n_time below 2^31.  A table that is not a permutation
 * gives undefined products but no out-of-bounds access.  Asynchronous.
 */
int corr_remap(const int32_t *const *d_tri, int n_dumps, int n_inputs, int n_chan, int f_avg,
               const int32_t *d_nat_of_pfb, int32_t *d_out, void *stream);

/*
 * Fine polyphase filterbank, the F stage's second channeliser (Section
 * 3.2.1): a critically sampled, n_taps-tap, 128-point filter-response-weighted
 * DFT turning each 1.28 MHz coarse channel into 128 fine channels of 10 kHz,
 * one output sample per 128 input samples.  For coarse channel q, input i and
 * frame m < M = n_samples / 128 - n_taps + 1:
 *
 *   u_m[n] = sum_{p < n_taps} window[p * 128 + n] * x_qi[(m + p) * 128 + n]      (n < 128)
 *   Y_m[k] = sum_{n < 128} u_m[n] * exp(-2 pi i k n / 128)                      (k < 128)
 *
 * written to fine channel q * 128 + c with c = (k + 64) mod 128 (c = 0 the
 * lowest frequency of the coarse channel, c = 64 its centre).  The paper gives
 * the 12-tap, 128-point structure but not the window, so the window is the
 * caller's.  Arithmetic is fp32 (the window, the sums and the FFT).
 *
 * d_x:      device int8 [n_coarse][n_inputs][n_samples][2] (real, imaginary),
 *           8-byte aligned; n_samples a multiple of 128 and >= 128 n_taps.
 * d_window: device float [n_taps][128], 16-byte aligned.  n_taps: 12 (the
 *           paper's) or 1 (a plain DFT per 128 samples); other counts give
 *           CORR_E_UNSUPPORTED.
 * d_volt:   device uint8 [M][n_coarse * 128][n_inputs] or NULL: the 4+4-bit
 *           sample (Appendix A, real part in the high nibble) of
 *           clamp(rint(scale * Y), -7, 7) per component, rounding half to even:
 *           the X-engine's input layout, so it can be passed to corr_accumulate
 *           with n_chan = 128 n_coarse.
 * d_spec:   device float [M][n_coarse * 128][n_inputs][2] or NULL, 8-byte
 *           aligned: Y itself.
 * At least one of d_volt and d_spec must be given.  CORR_E_ARG on sizes out of
 * range, NULL or misaligned pointers or a non-finite scale.  The caller owns
 * every buffer; asynchronous on `stream`, allocates nothing.
 */
#define CORR_PFB_POINTS 128
int corr_fine_pfb(const int8_t *d_x, int n_coarse, int n_inputs, long long n_samples, const float *d_window,
                  int n_taps, float scale, uint8_t *d_volt, float *d_spec, void *stream);

/* ------------------------------------------------------- no device allocation -- */

/* Size of the library's static device scratch used by corr_xmac_noalloc. */
#define CORR_NOALLOC_SCRATCH_BYTES (64u << 20)

/*
 * One whole integration of one block, for callers that may not allocate
 * device memory (no cudaMalloc, cudaFree or allocating library call happens
 * here or in anything it calls).  This has no counterpart in the paper: it
 * exists for hosts that own every byte of device memory through their own
 * pool, and for real-time loops in which an allocation (and the device
 * synchronisation it can cause) is not allowed once data is flowing.
 *
 * Correlates d_volt (device uint8 [n_time][n_chan][n_inputs], layout above)
 * with the CUDA-core X-engine and OVERWRITES d_vis (device int32
 * [n_chan][P][2]) with the packed triangle; n_time == 0 writes zeros.  Its
 * scratch is one static device array of CORR_NOALLOC_SCRATCH_BYTES (64 MiB)
 * that every GPU using the library holds until the process exits.  A request
 * whose unpacked operands need more than that, i.e.
 *     8 * n_chan * round_up(n_inputs, 64) * round_up(n_time, 64) / 2 bytes
 * > CORR_NOALLOC_SCRATCH_BYTES, returns CORR_E_BUDGET without enqueuing
 * anything (e.g. 256 inputs x 5000 samples fit 12 channels per call).
 * Other argument errors: CORR_E_ARG.  Asynchronous on `stream`.
 *
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it.  With lazy
 * module loading (the CUDA default) that lookup is also what loads the
 * library's device code on the device and reserves the 64 MiB, so the first
 * call may take device memory and synchronise the device: make one warm-up
 * call per device (n_time == 0 with a valid d_vis is enough) before data
 * flows, and before any stream capture.  All calls on a device share the same
 * scratch: calls whose work overlaps on the GPU (different streams, no
 * ordering between them) race and corrupt each other's results.  Calls
 * ordered on one stream are safe; the scratch keeps the previous call's
 * contents, which the next call fully rewrites before reading.
 */
int corr_xmac_noalloc(const uint8_t *d_volt, int n_time, int n_chan, int n_inputs,
                      int32_t *d_vis, unsigned flags, void *stream);

/* --------------------------------------------------------------- profiling -- */

/* Kernel kinds counted by the profiler. */
enum { CORR_K_UNPACK = 0, CORR_K_XENGINE = 1, CORR_K_DUMP = 2, CORR_K_OTHER = 3, CORR_K_KINDS = 4 };

typedef struct corr_profile {
    long long launches[CORR_K_KINDS];  /* kernels launched by this context, by kind */
    long long timed[CORR_K_KINDS];     /* of which bracketed by timing events       */
    double ms[CORR_K_KINDS];           /* summed device time of the timed launches  */
} corr_profile;

/* Launch counting is always on.  With on != 0 every kernel launch of the
 * context is also bracketed by a pair of CUDA events recorded on the launch
 * stream (device-side timing, no host synchronisation at launch). */
int corr_profile_enable(corr_ctx *ctx, int on);

/* Fill *out with the counts and the summed event times since the last reset
 * (waits for the recorded events to complete; pairs that cannot be timed are
 * not counted in timed[] and ms[]); reset != 0 clears them. */
int corr_profile_read(corr_ctx *ctx, corr_profile *out, int reset);

/* ------------------------------------------------------------------ errors -- */

int corr_last_error(void);            /* last status returned in this thread */
const char *corr_strerror(int status);  /* static string, never NULL         */

/* Library version as 10000*major + 100*minor + patch. */
int corr_version(void);

/* ---------------------------------------------------------------- probes -- */

/* Peak-rate probes: the rates the X-engine forms are measured against
 * (Section 3.4.2 compares the kernel with the GPU's peak; Eq. 4 sets the
 * intensity needed to reach it), taken on the device instead of assumed.
 * Each launches one block per SM running a fixed loop on register- or
 * shared-memory-resident values: */
#define CORR_PROBE_TC_FP8 0  /* tcgen05.mma kind::f8f6f4 E4M3 -> F32, M128 N256 K32, operands in SMEM  */
#define CORR_PROBE_MMA_S8 1  /* mma.sync m16n8k32 s8 -> s32 on registers                               */
#define CORR_PROBE_DP4A 2    /* dp4a (8 ops: four multiply-adds) on registers                          */
#define CORR_PROBE_FFMA 3    /* paired fp32 FMA (2 multiply-adds, 4 ops) on registers                 */
/* *ops_per_s: dense ops per second of the whole device (2 per multiply-add);
 * *launch_ms (may be NULL): the timed launch's CUDA-event time.  Runs a
 * warm-up launch and a timed one on `stream` and waits for them (the only
 * call here that synchronises the host besides corr_sync and the state
 * calls).  CORR_E_ARG on a bad kind or NULL ops_per_s; CORR_E_UNSUPPORTED
 * for CORR_PROBE_TC_FP8 off sm_103; CORR_E_TIMEOUT if the tensor-core
 * probe's completion wait gave up.  Allocates nothing. */
int corr_probe_rate(int kind, double *ops_per_s, double *launch_ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CORR_H */
