/*
 * rfr.h -- C ABI of the GB300 readout DSP library.
 *
 * The library turns a software radio's complex int16 ADC stream into
 * per-tone baseband timestreams, in the two forms of arXiv:1812.02200:
 *   - a polyphase filter bank (PFB, Sec. III.A): a windowed polyphase FIR
 *     over N channels x T taps, an N-point FFT per frame, and the full
 *     spectrum and/or a gather of the bins that hold the tones (critically
 *     sampled as in the paper, or oversampled with a hop below N);
 *   - direct multi-tone demodulation (Sec. III.B): a per-tone NCO mix, a
 *     low-pass FIR and decimation by D;
 * plus the chirped readout (Sec. III.C) and the GPU-generated transmit
 * buffers (a chirp; a multi-tone comb).
 *
 * Conventions shared by every call:
 *   - Samples are complex int16, I then Q interleaved (4 bytes per sample),
 *     as the radio delivers them (Sec. II.A).
 *   - Outputs are complex64 (float re, float im).
 *   - The stream starts at sample 0 with zero history.  Frame k is computed
 *     from the W samples that end at sample (k+1)*hop - 1 (W = N*T, hop = N
 *     for the PFB; W = L, hop = D for demodulation); samples before 0 are 0.
 *   - The PFB output of channel c is y_k[c] = sum_p v_k[p] exp(-2*pi*i*c*p/N)
 *     (for a hop below N, exp(-2*pi*i*c*(A_k + p)/N) with A_k the absolute
 *     index of the frame's first sample), natural bin order, no 1/N factor
 *     (the taps sum to 1 instead).
 *   - A tone is an NCO word w: a uint64 phase increment per sample in units
 *     of 2*pi/2^64.  Its phase at absolute sample m is w*m mod 2^64 (exact
 *     integer arithmetic); the mixer is exp(-i*phase).
 *   - Device pointers are plain CUDA device (or managed) addresses; "stream"
 *     is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Every call returns an rfr_status; nothing is thrown across the ABI.
 *     rfr_last_error() gives a message for the last failure of a plan.
 *   - Tracing: the calls that enqueue GPU work open NVTX ranges named after
 *     themselves.  RFR_DEBUG=1 in the environment (read once per process)
 *     makes them synchronise their stream after enqueueing, unless it is
 *     being captured, and return the first CUDA or device-status error at
 *     the call that caused it; results are unchanged.
 *
 * Thread safety: a plan is used by one host thread at a time.  Different
 * plans are independent.
 */
#ifndef RFR_H
#define RFR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rfr_plan rfr_plan;   /* opaque, owned by the library */

typedef enum {
    RFR_OK = 0,
    RFR_E_INVALID = -1,     /* bad argument or plan parameters */
    RFR_E_NOMEM = -2,       /* device or host allocation failed */
    RFR_E_CUDA = -3,        /* a CUDA call failed (message in rfr_last_error) */
    RFR_E_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    RFR_E_SHORT = -5,       /* output capacity too small; nothing consumed */
    RFR_E_BUSY = -6,        /* resource in use (e.g. server slot pool full) */
    RFR_E_UNSUPPORTED = -7  /* valid request this build does not implement */
} rfr_status;

typedef enum {
    RFR_WIN_RECT = 0,       /* square window: the paper's moving average (Sec. III.B) */
    RFR_WIN_HANN = 1,
    RFR_WIN_HAMMING = 2,    /* the paper's PFB window (Sec. III.A) */
    RFR_WIN_BLACKMAN = 3,
    RFR_WIN_KAISER = 4      /* uses beta */
} rfr_window_kind;

/* Low-pass prototype h[j] = w[j] * sinc(2*cutoff*(j - (W-1)/2)), normalised
 * to sum 1 in FP64 (DC gain 1), where w is the symmetric window of length W.
 * cutoff is in cycles per sample.  PFB: cutoff 0 selects 1/(2N), which puts
 * the cross-over of adjacent channels near -6 dB (Sec. III.A, Fig. 3).
 * Demodulation: cutoff 0 drops the sinc factor (pure window; with
 * RFR_WIN_RECT the moving average of Sec. III.B). */
typedef struct {
    int32_t kind;           /* rfr_window_kind */
    double beta;            /* Kaiser shape parameter; ignored otherwise */
    double cutoff;          /* cycles/sample, >= 0 */
} rfr_window;

/* Readout tones: NCO words (host memory; copied by rfr_plan_create). */
typedef struct {
    const uint64_t* words;
    int32_t count;
} rfr_tones;

enum { RFR_OUT_FULL = 1, RFR_OUT_TONES = 2 };
enum { RFR_MODE_PFB = 1, RFR_MODE_DEMOD = 2, RFR_MODE_CHIRP = 3 };

/* Caller-owned output buffers of one push (device memory).
 *   full : complex64 [frames][full_ld], channel c of frame f at
 *          full[(frame_offset + f) * full_ld + c]   (PFB with RFR_OUT_FULL)
 *   tones: complex64 [count][tones_ld], tone s of frame f at
 *          tones[s * tones_ld + frame_offset + f]  (PFB with RFR_OUT_TONES,
 *          and always for demodulation)
 * full_cap / tones_cap are the capacities in frames of each row range; a push
 * that would write past frame_offset + cap fails with RFR_E_SHORT before any
 * work is enqueued.  frames is written by the call (frames produced). */
typedef struct {
    void* full;
    int64_t full_ld;
    int64_t full_cap;
    void* tones;
    int64_t tones_ld;
    int64_t tones_cap;
    int64_t frame_offset;
    int64_t frames;
} rfr_output;

typedef struct {
    int32_t mode;           /* RFR_MODE_PFB, RFR_MODE_DEMOD or RFR_MODE_CHIRP */
    int32_t channels;       /* N (PFB) or 0 */
    int32_t taps;           /* T per channel (PFB) or L (demodulation) */
    int32_t decimation;     /* hop: N (PFB) or D */
    int32_t n_tones;
    uint32_t out_flags;
    int64_t samples_consumed;   /* stream position (samples pushed so far) */
    int64_t frames_produced;
    int64_t frames_pending;     /* produced by rfr_push, not yet pulled */
    double tap_scale;           /* demodulation: power-of-two tap scale used by the
                                   split-FP16 tensor-core path (diagnostic) */
} rfr_plan_info;

/*
 * rfr_plan_create -- build a plan (Sec. III.A for channels > 0, Sec. III.B
 * for channels == 0).
 *   channels   N > 0: PFB with N channels, 2 <= N <= 2^24 (Sec. III.A: Fig. 3
 *              uses N = 10^5, the section reports up to 10^7 bins).  N must have
 *              no prime factor above 7 (N = 2^a 3^b 5^c 7^d); any other N
 *              returns RFR_E_UNSUPPORTED.  Powers of two from 16 to 16384 run
 *              the single-CTA-per-frame kernels (FIR, FFT and gather fused
 *              where the delay line fits one SM; for N = 8192, 16384 or
 *              T > 8 the FIR as a separate pre-sum pass first), every other
 *              N the mixed-radix kernels (one pass up to 8192, a four-step
 *              two-pass form above).
 *              0: direct demodulation.
 *   taps       PFB: T taps per channel, 1 <= T <= 16 (prototype length N*T).
 *              Demodulation: filter length L, 1 <= L <= 16384.
 *   window     prototype window and cut-off (see rfr_window).
 *   tones      NCO words of the readout tones (0 <= count <= 65536).  PFB:
 *              tone s is read from bin rfr_word_to_bin(words[s], N).
 *   decimation PFB: the hop H between frames, 1 <= H <= N (H = N: critically
 *              sampled, the paper's PFB; H < N: oversampled, frame k ending
 *              at sample (k+1)*H - 1, each channel keeping the phase of the
 *              absolute time origin, so channel c equals the demodulator's
 *              output for the bin-centred word; oversampled plans run the
 *              mixed-radix kernels, except N = 4096, T = 8 at H = N/2 or N/4,
 *              which runs as exact phase passes of the fused kernel).  Demodulation: D >= 1 and D a multiple
 *              of 32 for the tensor-core path.
 *   out_flags  PFB: any non-empty combination of RFR_OUT_FULL, RFR_OUT_TONES
 *              (RFR_OUT_TONES needs count > 0).  Demodulation: RFR_OUT_TONES.
 * Allocates the plan's device tables and stream state on the current device.
 * Two-pass PFB plans (N > 8192 and not a power of two up to 16384) also hold
 * between-pass buffers for a batch of frames: Z, and (when the split of N has
 * an even second factor) the FIR outputs V, each up to 1 GB, allocated by the
 * first push that needs them (rfr_batch_push grows them before capturing its
 * graph; rfr_server_create sizes them for its largest buffer, so serving
 * never allocates).  Demodulation plans likewise allocate their per-push
 * scratch (the FP16 split of the stream and the rotation tables) on the first
 * push of a given size, and so do PFB plans that run their FIR as a separate
 * pre-sum pass (N = 8192; N = 16384 with T > 4; N = 256 to 4096 with T > 8:
 * 8 bytes per channel and frame) or the oversampled phase passes; a
 * push that grows scratch synchronises the device and sizes it for that many
 * samples after any carry.  Inside a stream capture such a push fails with
 * RFR_E_INVALID instead, so push once at the largest size outside capture
 * first.
 * Errors: RFR_E_INVALID (parameters), RFR_E_NOMEM, RFR_E_CUDA.
 */
rfr_status rfr_plan_create(rfr_plan** plan, int32_t channels, int32_t taps,
                           const rfr_window* window, const rfr_tones* tones,
                           int32_t decimation, uint32_t out_flags);

/*
 * Chirped readout (Sec. III.C, Eq. 1).  Eq. 1, phi_t = 2*pi*(f0*t + k*t^2), in
 * sample units t = m/fs is the exact uint64 phase
 *     p(m) = start*m + rate*m^2  (mod 2^64, units of 2*pi/2^64),
 * start = rfr_freq_to_word(f0, fs), rate = rfr_chirp_rate_word(k, fs).
 *
 * rfr_plan_create_chirp -- a plan that demodulates the stream against
 * n_chirps chirps (the algorithm of Sec. III.B with the chirp as the mixer):
 * for chirp c and frame k (b_k = (k+1)*D - L, zero history)
 *     out[c][k] = sum_{n<L} h[n] x[b_k+n] exp(-i*2*pi*p_c(b_k+n)/2^64),
 * h the low-pass of `window` (as for demodulation; cut-off 0 = pure window).
 * Output layout and streaming as for demodulation plans (RFR_OUT_TONES, one
 * row per chirp).  1 <= L <= 16384, 1 <= D, 1 <= n_chirps <= 4096; start and
 * rate words are host arrays, copied.
 */
rfr_status rfr_plan_create_chirp(rfr_plan** plan, int32_t taps, const rfr_window* window,
                                 const uint64_t* start_words, const uint64_t* rate_words,
                                 int32_t n_chirps, int32_t decimation);

/* Rate word of a chirp rate k (Hz/s) at sample rate fs: round(k/fs^2 * 2^64). */
uint64_t rfr_chirp_rate_word(double k_hz_per_s, double fs_hz);

/*
 * rfr_chirp_synthesize -- the transmit buffer of a chirp generated on the
 * GPU in real time (Sec. III.C): samples m0 .. m0+n-1 of
 *     x[m] = (round(A*cos(2*pi*p(m)/2^64)), round(A*sin(2*pi*p(m)/2^64)))
 * as complex int16 (round half to even, clamped to the int16 range) into the
 * device buffer iq_out [n][2].  Computed in FP32 on the phase reduced to a
 * quarter turn; a component whose FP32 value lies within twice its error
 * bound (A*(pi*(2^-27 + 2^-31) + 2^-23) + |fl(A) - A|) of a rounding tie is
 * recomputed in FP64, so every sample is the FP64-rounded value.
 * 0 <= amplitude <= 32767.  Asynchronous on `stream`; the first call on a
 * device uploads a small table synchronously (make it outside stream
 * capture).
 */
rfr_status rfr_chirp_synthesize(uint64_t start_word, uint64_t rate_word, double amplitude, int64_t m0,
                                int64_t n_samples, int16_t* iq_out, void* stream);

/*
 * Transmit buffer (Sec. III: the transmission buffer is generated on the GPU
 * from the tones the receiver demodulates).  A generator holds n_tones NCO
 * words w_t, phase words p_t (NULL: all zero) and amplitudes A_t >= 0
 * (sum A_t <= 10^6), copied from host arrays, and writes samples m0 .. m0+n-1
 *     s(m) = sum_t A_t exp(+i*2*pi*((w_t*m + p_t) mod 2^64) / 2^64)
 * as complex int16 (each component rounded half to even, clamped) into the
 * device buffer iq_out [n][2], asynchronously on `stream`.  A tone at word w
 * is brought to DC by the receiver's mixer for the same word.
 *
 * Precision: FP32 sines and cosines of the exact integer phase, FP32 sums over
 * 32 tones, FP64 over the chunks.  Before rounding each component is within
 * e = rfr_tx_error_bound(tx) of the exact sum, so every component whose exact
 * value lies farther than e from a rounding tie is the exact rounding; the few
 * within e of a tie are one of the two neighbouring integers.  Samples are
 * computed independently: any split of [m0, m0+n) gives the same samples.
 * Errors: RFR_E_INVALID (arguments), RFR_E_NOMEM, RFR_E_CUDA (launch).
 */
typedef struct rfr_tx rfr_tx;
rfr_status rfr_tx_create(rfr_tx** tx, const uint64_t* words, const uint64_t* phase_words,
                         const double* amplitudes, int32_t n_tones);
rfr_status rfr_tx_synthesize(rfr_tx* tx, int64_t m0, int64_t n, int16_t* iq_out, void* stream);
double rfr_tx_error_bound(const rfr_tx* tx);
void rfr_tx_destroy(rfr_tx* tx);

/* Frees everything the plan owns (waits for its outstanding work). */
void rfr_plan_destroy(rfr_plan* plan);

rfr_status rfr_plan_get_info(const rfr_plan* plan, rfr_plan_info* info);

/* Number of frames a push of n_samples would produce now. */
rfr_status rfr_frames_for(const rfr_plan* plan, int64_t n_samples, int64_t* frames);

/*
 * rfr_push_into -- process the next n_samples of the stream (device buffer
 * iq, [n_samples][2] int16) asynchronously on `stream`, writing the frames
 * that complete into the caller's buffers `out` (device).  Filter history,
 * the partial-frame residue and the stream position are kept in the plan, so
 * any split of a stream into pushes gives the same frames (bit-identical) as
 * one push of the whole stream.
 * iq must stay valid until the work on `stream` completes.  On error nothing
 * is enqueued and the stream state is unchanged.
 * Errors: RFR_E_INVALID, RFR_E_SHORT (output capacity), RFR_E_CUDA.
 */
rfr_status rfr_push_into(rfr_plan* plan, const int16_t* iq, int64_t n_samples,
                         rfr_output* out, void* stream);

/*
 * rfr_push / rfr_pull -- the queued form (Sec. III: the processing thread
 * hands finished buffers to a streaming thread).  rfr_push processes like
 * rfr_push_into but keeps the frames in a plan-owned device ring (grown on
 * demand); rfr_pull copies all pending frames, in order, into `out` (device
 * or host memory) on the stream of the last push and consumes them.  `out`
 * must have room for every pending frame (RFR_E_SHORT otherwise, nothing
 * consumed); out->frames is set to the number copied.
 */
rfr_status rfr_push(rfr_plan* plan, const int16_t* iq, int64_t n_samples, void* stream);
rfr_status rfr_pull(rfr_plan* plan, rfr_output* out);

/*
 * rfr_process_host -- end-to-end form for host-resident data: copies the
 * host samples to the device in chunks, processes them and copies the frames
 * back into host `out` buffers, overlapping the copies with the compute on
 * the plan's internal streams.  Host buffers should be pinned
 * (cudaHostAlloc / cudaHostRegister) for full speed.  Synchronous: returns
 * when `out` holds the results.  The stream state advances as for a push.
 */
rfr_status rfr_process_host(rfr_plan* plan, const int16_t* iq_host, int64_t n_samples,
                            rfr_output* out_host);

/* Zero history, residue and stream position (and drop pending frames): the
 * plan starts a new stream at sample 0, as after rfr_plan_create (the
 * buffered Rx stream of Sec. III restarted).  Synchronises the device.
 * Errors: RFR_E_INVALID (NULL plan), RFR_E_CUDA. */
rfr_status rfr_reset(rfr_plan* plan);

/*
 * Checkpoint / resume of the stream state (history, residue, position) of the
 * buffered Rx stream of Sec. III: the state a push carries to the next one.
 * Export with host == NULL stores the needed size in *bytes; otherwise *bytes
 * is the capacity of `host` (RFR_E_SHORT if too small) and receives the size
 * written.  Import needs a plan created with the same parameters
 * (RFR_E_INVALID otherwise, state unchanged); it restores the state exactly,
 * so the next push continues the stream bit-identically.  Both synchronise
 * with the plan's outstanding work; the blob is plain host memory owned by
 * the caller.
 */
rfr_status rfr_state_export(rfr_plan* plan, void* host, size_t* bytes);
rfr_status rfr_state_import(rfr_plan* plan, const void* host, size_t bytes);

/*
 * rfr_plan_set_demod_products -- demodulation only: the form of the tensor-
 * core contraction.  4: the real embedding of the complex product (four real
 * products per complex multiply-add).  3 (the default wherever D % 64 == 0,
 * 4 otherwise): the Gauss form
 *   P1 = sum ((xr+xi)/2) cr, P2 = sum xr (ci-cr), P3 = sum xi (cr+ci),
 *   Re = 2 P1 - P3, Im = 2 P1 + P2
 * (three real products; the same definition, Sec. III.B, rounded
 * differently), which needs D % 64 == 0 (RFR_E_UNSUPPORTED otherwise) and
 * builds its tap planes on the first switch (allocates, synchronises the
 * device).  Either switch resets the accumulation chunk to the form's
 * default (64 taps in the four-product form, 256 in the three-product
 * form).  Set it before the first push of a stream.
 */
rfr_status rfr_plan_set_demod_products(rfr_plan* plan, int32_t products);

/*
 * rfr_plan_set_accum_chunk -- demodulation only: how many K blocks (32 taps
 * each in the four-product form, 64 in the three-product form; 1..64,
 * default 2 in the four-product form, 4 in the three-product form) the
 * tensor cores accumulate in TMEM before the epilogue adds the partial sums
 * into FP32 registers.  Longer chunks are faster (fewer TMEM reads by the
 * epilogue, which compete with the MMAs) and less accurate (the tensor
 * cores' internal accumulation error grows with the partial sums): on the
 * weakest tones of the 2048-tone workload, 1.2e-6 / 1.9e-6 / 3.7e-6
 * relative error at 2 / 4 / 8 blocks of the three-product form, which runs
 * 16.7 / 18.2 / 19.1 Gs/s there.  Changes the results' rounding, so set it
 * before the first push.
 */
rfr_status rfr_plan_set_accum_chunk(rfr_plan* plan, int32_t k_blocks);

/*
 * rfr_plan_seek -- position a fresh or used plan at absolute sample
 * start_sample of a stream (a multiple of the hop), as if every sample before
 * it had been pushed: the next push's first frame is frame start_sample/hop,
 * with NCO phases taken from the absolute sample index.  `history` (device or
 * host) holds the n_history = min(H, start_sample) samples just before
 * start_sample, H = N*T - hop for the PFB and max(L - D, 0) for demodulation;
 * earlier samples count as zero.  This is how a
 * long stream is split along time across plans or GPUs: each shard gets its
 * slice plus this halo, and the shards' frames concatenate to the one-shot
 * result bit-identically.  Synchronises the device.
 */
rfr_status rfr_plan_seek(rfr_plan* plan, int64_t start_sample, const int16_t* history,
                         int64_t n_history);

/*
 * rfr_plan_inject_device_status -- failure injection on the host: writes the
 * plan's device status word exactly as a kernel whose bounded wait gave up
 * would (status 1 = timeout; 0 clears it), so that callers and tests can
 * exercise their RFR_E_TIMEOUT handling without faulting or hanging a GPU.
 * Kernels of a later push that find the word set leave their waits early.
 * Synchronises the device.  Errors: RFR_E_INVALID (status not 0, 1 or 2),
 * RFR_E_CUDA.
 */
rfr_status rfr_plan_inject_device_status(rfr_plan* plan, int32_t status);

/*
 * rfr_wait_selftest -- launch a kernel whose bounded device-side wait can
 * never be satisfied and check that it gives up after limit_ns (1 us .. 2 s)
 * with the library's timeout status: returns RFR_E_TIMEOUT (and the device
 * status word in *device_status) when the failure detection works.  Nothing
 * faults or traps; the context stays usable.
 */
rfr_status rfr_wait_selftest(int64_t limit_ns, int32_t* device_status);

/*
 * Prototype taps (host memory, caller-owned): the windowed-sinc low-pass of
 * Sec. III.A (PFB, length N*T, oldest sample first) or the demodulator's
 * filter of Sec. III.B (length L).  h64 in FP64 (may be NULL), h32 the FP32
 * values the PFB kernels use (may be NULL).  *n receives the length (N*T or
 * L); with both pointers NULL only *n is set.  Errors: RFR_E_INVALID.
 */
rfr_status rfr_plan_get_taps(const rfr_plan* plan, double* h64, float* h32, int64_t* n);

/* PFB: bin of each tone (host int32[count]). */
rfr_status rfr_plan_get_bins(const rfr_plan* plan, int32_t* bins, int32_t* count);

/*
 * rfr_plain_oneshot -- the plain FP32 GPU form of the same computation, for
 * comparison: PFB as an FP32 FIR kernel, a batched cuFFT C2C transform and a
 * gather kernel; demodulation as an FP32 CUDA-core kernel.  Processes one
 * whole buffer with zero history (does not touch the plan's stream state).
 * Scratch is allocated by the call on first use and cached in the plan.
 * Chirp plans have no separate plain form (RFR_E_UNSUPPORTED): their kernel
 * already is plain FP32 CUDA-core code.
 */
rfr_status rfr_plain_oneshot(rfr_plan* plan, const int16_t* iq, int64_t n_samples,
                             rfr_output* out, void* stream);

/*
 * rfr_plain_oneshot_form -- rfr_plain_oneshot with the comparison form named:
 *   RFR_PLAIN_DEFAULT  the forms above;
 *   RFR_PLAIN_CGEMM    demodulation plans only: the mix + filter of Sec. III.B
 *                      as the library matrix product the paper names for it,
 *                      cublasCgemm in pedantic FP32 (no TF32, no emulation) of
 *                      the Toeplitz matrix X[k][n] = x[(k+1)D - L + n],
 *                      materialised on the device in frame chunks of at most
 *                      512 MiB, by the modulated taps C_t[n]; then the rotation
 *                      exp(-i*phi_t((k+1)D - L)) into [tone][frame].
 * Same arguments, output layout and zero history as rfr_plain_oneshot.
 * Errors: RFR_E_INVALID (unknown form), RFR_E_UNSUPPORTED (Cgemm form on a
 * PFB or chirp plan), RFR_E_SHORT, RFR_E_CUDA (a cuBLAS failure included).
 */
enum { RFR_PLAIN_DEFAULT = 0, RFR_PLAIN_CGEMM = 1 };
rfr_status rfr_plain_oneshot_form(rfr_plan* plan, int32_t form, const int16_t* iq, int64_t n_samples,
                                  rfr_output* out, void* stream);

/* ------------------------------------------------------------------ batch */
typedef struct rfr_batch rfr_batch;

/*
 * rfr_batch_create -- group n distinct plans (PFB and/or demodulation, any
 * shapes) that advance together, one buffer per plan per step (the paper's
 * Rx processing of many detector readouts, Sec. III; the batched workload).
 * The batch borrows the plans (they must outlive it and must not be pushed
 * elsewhere while it runs).  Errors: RFR_E_INVALID (n < 1, NULL or repeated
 * plan), RFR_E_NOMEM, RFR_E_CUDA.
 */
rfr_status rfr_batch_create(rfr_batch** batch, rfr_plan* const* plans, int32_t n);
void rfr_batch_destroy(rfr_batch* batch);

/*
 * rfr_batch_push -- one step: plan i pushes bufs[i] (device, n_samples[i]
 * samples) into outs[i] exactly as rfr_push_into would (bit-identical
 * results, stream state kept per plan), but all plans' kernels run
 * concurrently from ONE CUDA-graph launch into `stream`.  Inside it, the
 * tensor-core GEMMs of every three-product demodulation plan run as one
 * persistent kernel over all those plans' tiles (one launch per tone-tile
 * width and per 16 plans), the other kernels on one graph branch per plan.
 * The executable graph is kept and updated in place on the next step.
 * outs[i].frames is set.
 * Every push is checked before anything is enqueued (RFR_E_INVALID /
 * RFR_E_SHORT leave all plans unchanged).  Scratch growth happens before the
 * graph is built.
 */
rfr_status rfr_batch_push(rfr_batch* batch, const int16_t* const* bufs, const int64_t* n_samples,
                          rfr_output* outs, void* stream);

/* Steps run, graph updates in place and graph instantiations so far. */
rfr_status rfr_batch_stats(const rfr_batch* batch, int64_t* steps, int64_t* graph_updates,
                           int64_t* graph_instantiations);
const char* rfr_batch_last_error(const rfr_batch* batch);

/*
 * rfr_plan_autotune -- time the plan's result-neutral launch choices (PFB:
 * ring look-ahead of 1..3 super-blocks; demodulation: GEMM tile raster
 * groups and, for the three-product form, the tile shape (128 frames x 128
 * or 64 tones) and whether the FP16 split of the stream is fused into the
 * GEMM) on a push of n_samples and keep the fastest (Sec. III: the
 * host runtime tunes the GPU kernels).  Outputs stay bit-identical whatever
 * is chosen.  With use_cache != 0 the choice is read
 * from / written to the JSON file named by RFR_TUNE_CACHE (default
 * ./rfr_tune_cache.json), keyed by plan shape, push size and GPU.  The
 * stream state is left unchanged.  *best_ms (may be NULL) receives the time
 * of the chosen configuration (-1 when it came from the cache).
 */
rfr_status rfr_plan_autotune(rfr_plan* plan, int64_t n_samples, int32_t use_cache, double* best_ms);
rfr_status rfr_plan_get_tune(const rfr_plan* plan, int32_t* pfb_lookahead, int32_t* demod_raster,
                             int32_t* tuned);
/* Tones per GEMM tile of a three-product demodulation plan (128 or 64, as
 * tuned; 128 by default); 0 for other plans.  Setting it is result-neutral
 * (the autotuner chooses it; set it by hand only to pin a choice).
 * Errors: RFR_E_INVALID (not a three-product demodulation plan, or a width
 * other than 64 or 128). */
rfr_status rfr_plan_get_tone_tile(const rfr_plan* plan, int32_t* tones_per_tile);
rfr_status rfr_plan_set_tone_tile(rfr_plan* plan, int32_t tones_per_tile);

/* Three-product demodulation: on = 1 fuses the FP16 hi/lo split of the int16
 * stream (the GEMM's A operand) into the GEMM's producer warps, which read
 * the stream and write the swizzled operand tiles themselves, instead of a
 * separate kernel writing six FP16 planes (12 bytes per sample) to device
 * memory for the GEMM to load (Sec. III.B's mix and filter as one kernel).
 * Result-neutral (bit-identical planes); the autotuner times both forms.
 * Errors: RFR_E_INVALID (not a three-product demodulation plan, on not 0/1). */
rfr_status rfr_plan_set_fused_presplit(rfr_plan* plan, int32_t on);
rfr_status rfr_plan_get_fused_presplit(const rfr_plan* plan, int32_t* on);

/* Three-product demodulation: on = 1 runs the GEMM in clusters of two CTAs
 * on two SMs that take the two tone tiles of one frame tile; the frames'
 * operand tiles (the Toeplitz view of the stream, Sec. III.B) are the same
 * for both, so each CTA loads half of every such tile and TMA multicasts it
 * into both CTAs' shared memory, a quarter less operand traffic from L2 per
 * CTA.  Default 0 (one CTA per tile; the cluster form measured about 3 %
 * slower on the 2048-tone workload, the two CTAs running in lock step).
 * Applies to the separate pre-split form only (get reports 0 while the
 * fused pre-split is on).  Result-neutral (the same MMAs in the same
 * order); the autotuner times both forms.
 * Errors: RFR_E_INVALID (not a three-product demodulation plan, on not 0/1). */
rfr_status rfr_plan_set_demod_pair(rfr_plan* plan, int32_t on);
rfr_status rfr_plan_get_demod_pair(const rfr_plan* plan, int32_t* on);

/* PFB plans of N = 8192 or 16384 channels with T <= 8 taps (Sec. III.A), whose
 * FP32 delay line of N*T points exceeds one SM's tensor memory: on = 1 runs
 * them on clusters of N/4096 CTAs on as many SMs, each holding a 4096-channel
 * slice's delay line in tensor memory and taps in registers; the N-point
 * FFT is split into a radix-(N/4096) step across the CTAs (filtered slices
 * exchanged through distributed shared memory) and a 4096-point FFT per
 * CTA, and the output rows are assembled the same way.  on = 0 (the
 * default): the direct kernel (one CTA per frame, the FIR as a separate
 * pre-sum pass for T > 4 at N = 16384 and any T at N = 8192, else through
 * L1/L2), which measured faster (132 against 58 Gs/s at N = 16384, T = 8):
 * with one frame in flight per CTA the cross-SM exchanges and cluster
 * barriers of every frame cannot be hidden.  The two round differently (both within the
 * oracle's tolerance), so choose before the first push; the autotuner times
 * both.  Errors: RFR_E_INVALID (another plan shape, on not 0/1). */
rfr_status rfr_plan_set_pfb_cluster(rfr_plan* plan, int32_t on);
rfr_status rfr_plan_get_pfb_cluster(const rfr_plan* plan, int32_t* on);

/* ---------------------------------------------------------------- serving */
typedef struct rfr_server rfr_server;

typedef struct {
    uint64_t tag;           /* as given to rfr_server_submit */
    int32_t readout;
    int32_t status;         /* rfr_status of the request */
    int64_t frames;         /* frames written to the request's output */
    int64_t samples;
    double t_submit_us;     /* rfr_now_us() clock: submit, admission, completion seen */
    double t_admit_us;
    double t_done_us;
} rfr_completion;

typedef struct {
    int64_t submitted, admitted, completed, queued, in_flight;
    int64_t budget_bytes, peak_bytes;   /* staging arena: size and high-water mark */
} rfr_server_stats;

/*
 * rfr_server_create -- a serving loop over n readouts (plans[i] serves
 * readout i; plans must outlive the server and not be pushed elsewhere).
 * The paper's host runtime passes acquired buffers between threads through
 * queues of pointers into pre-allocated memory (Sec. III); here one worker
 * thread admits submitted buffers in arrival order as device memory frees up
 * and enqueues each at once on its readout's stream (copy in, push, copy the
 * frames out, completion event), so requests that arrive while others are on
 * the GPU run concurrently with them (continuous batching).  Each readout's
 * buffers are processed in submission order and its filter history and NCO
 * phase stay on the device between buffers.
 *   mem_budget_bytes   device staging arena allocated once here (inputs of
 *                      host buffers + produced frames of every admitted
 *                      request must fit); nothing is allocated while serving.
 *   max_buffer_samples largest buffer a request may carry (plan scratch is
 *                      pre-sized for it).
 */
rfr_status rfr_server_create(rfr_server** server, rfr_plan* const* plans, int32_t n,
                             size_t mem_budget_bytes, int64_t max_buffer_samples);

/*
 * rfr_server_submit -- queue a buffer (host -- ideally pinned -- or device
 * memory, [n_samples][2] int16) of `readout`; its frames go to `out` (host or
 * device buffers, layout of rfr_output).  Returns immediately; iq and out must
 * stay valid until the request's completion is polled.  RFR_E_NOMEM if the
 * request could never fit in the budget, RFR_E_INVALID for bad arguments.
 */
rfr_status rfr_server_submit(rfr_server* server, int32_t readout, const int16_t* iq, int64_t n_samples,
                             const rfr_output* out, uint64_t tag);

/* Up to cap completions (oldest first); waits up to wait_ms for the first. */
rfr_status rfr_server_poll(rfr_server* server, rfr_completion* done, int32_t cap, int32_t* n_done,
                           int32_t wait_ms);
rfr_status rfr_server_get_stats(const rfr_server* server, rfr_server_stats* stats);

/* A completion's status is RFR_E_TIMEOUT when a bounded device-side wait of
 * that request's kernels gave up (the plan's device status word is copied
 * after each request and cleared), RFR_E_CUDA on a CUDA error. */

/* Finishes every submitted request, then frees the server. */
void rfr_server_destroy(rfr_server* server);

/* The host clock (microseconds, steady) the server stamps requests with. */
double rfr_now_us(void);

/*
 * rfr_demod_noalloc -- one-shot direct demodulation that allocates nothing.
 * (The paper has no counterpart; this is a deployment convenience.)
 *
 * Who needs it: code that must not call the CUDA allocator while it runs --
 * a real-time processing thread that cannot absorb the device-wide
 * synchronisation and allocator locking cudaMalloc/cudaFree may cause, or a
 * host application whose device-memory budget is owned by another allocator.
 * Plans allocate their tables and stream state; this call instead uses one
 * file-scope device array of about 6.7 MB that every GPU loading the library
 * holds until the process exits.  The caller still owns inputs and outputs.
 *
 * Computes the same frames as a fresh plan (zero history) pushed with the
 * whole buffer: tone s of frame k at tones[s * tones_ld + k], k < n_samples/D,
 * on the same split-FP16 tensor-core path.
 *   iq        device int16 [n_samples][2]
 *   taps      HOST FP64 low-pass taps h[0..L) (e.g. from rfr_plan_get_taps)
 *   words     HOST NCO words [n_tones]
 *   tones     device complex64 [n_tones][tones_ld], tones_ld >= n_samples/D
 * Limits (the size of the static scratch): n_samples <= 2^18, L <= 1024,
 * 1 <= n_tones <= 256, D a multiple of 32; anything larger returns
 * RFR_E_INVALID before any work is enqueued.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call shares the one array and leaves its contents behind
 * (each call clears or overwrites what it needs), so calls whose GPU work
 * overlaps -- on different streams or host threads -- race; serialise them.
 * Asynchronous on `stream`; the results are ready when the stream is.
 */
rfr_status rfr_demod_noalloc(const int16_t* iq, int64_t n_samples, const double* taps, int32_t L,
                             int32_t D, const uint64_t* words, int32_t n_tones, void* tones,
                             int64_t tones_ld, void* stream);

/*
 * rfr_demod_noalloc_status -- the device status word of the last
 * rfr_demod_noalloc call (it lives in the same shared static array, so it
 * belongs to whichever call ran last on this device).  Waits for `stream`
 * (pass the stream of that call), then copies the word into *device_status
 * (may be NULL) without allocating.  Returns RFR_E_TIMEOUT when a bounded
 * device-side wait of the call's GEMM gave up (its output is then incomplete),
 * RFR_E_CUDA for a CUDA error or any other non-zero word, RFR_OK otherwise.
 * (The paper has no counterpart.)
 */
rfr_status rfr_demod_noalloc_status(void* stream, int32_t* device_status);

/* The per-tone NCO of Sec. III.B (the mixer of each readout tone): frequency
 * f_hz at sample rate fs_hz -> NCO word, f/fs wrapped into [-1/2, 1/2), times
 * 2^64, rounded to nearest (two's complement).  Pure function, no device work. */
uint64_t rfr_freq_to_word(double f_hz, double fs_hz);

/* The user-selected channels of Sec. III.A (the PFB bins that hold the
 * readout tones): bin of an NCO word in an n-channel PFB, round(word*n/2^64)
 * mod n, ties up, i.e. floor((word*n + 2^63) / 2^64) mod n in exact 128-bit
 * integer arithmetic, for any n >= 2; -1 if n < 2.  Pure function. */
int32_t rfr_word_to_bin(uint64_t word, int32_t n);

const char* rfr_status_string(rfr_status status);
const char* rfr_last_error(const rfr_plan* plan);

/* Library version string. */
const char* rfr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RFR_H */
