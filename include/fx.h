/*
 * fx.h -- C ABI of the GB300 FX correlator library (libfx_gb300.so).
 *
 * The hot path of the Cobalt correlator pipeline (arXiv 1801.04834,
 * Sec. "Signal processing with GPU kernels"), per subband:
 *   fx_channelize  polyphase filter bank: T-tap FIR per channel + C-point FFT
 *   fx_correct     fine delay compensation + bandpass correction (+ gains),
 *                  transposing to the per-channel, all-stations layout
 *   fx_correlate   X-stage: all station pairs x 4 polarisation products,
 *                  integrated over the block
 *
 * Conventions for every call:
 *   - Pointers prefixed d_ are device pointers (cudaMalloc'd or torch tensors),
 *     h_ are host pointers. The caller owns every buffer it passes in; the
 *     library owns only what fx_create allocates (taps, twiddles, subband
 *     frequencies, the phase-table and status workspaces).
 *   - Complex values are interleaved (re, im) pairs of the stated real type.
 *   - Calls are asynchronous and stream-ordered on `stream` (NULL = legacy
 *     default stream). They never synchronise the device, so they can be
 *     captured in a CUDA graph. An error from earlier asynchronous work is
 *     reported by a later call that checks for it.
 *   - Return values are fx_status codes; nothing throws across the ABI.
 *     fx_last_error() returns a message for the last failure on this thread.
 *   - A handle is not thread-safe: use one handle per host thread / stream.
 *   - Nothing is allocated on the device after fx_create returns.
 *
 * Layouts (row-major; N stations, P = 2 polarisations, I = N*P inputs with
 * input index i = n*P + p, SB subbands, C channels, T taps, S spectra):
 *   raw   [SB][N][L][P]      complex int16, int8 or int4, L = (S + T - 1) * C samples
 *   chan  [SB][N][P][S][C]   complex float
 *   corr  FX_F32:            [SB][C][S16/16][N][16][P] complex float,
 *                            S16 = S rounded up to 16 ("spectrum-blocked":
 *                            sample (n, p) of spectrum s in channel k is at
 *                            (((sb*C + k)*S16/16 + s/16)*N + n)*16*P
 *                            + (s%16)*P + p; one channel's block is
 *                            contiguous, and within it each station's 16
 *                            spectra x 2 pols are one 256-byte run); spectra
 *                            S .. S16-1 are written as zeros
 *         FX_F16, FX_BF16:   [SB][C][2][I_pad][S_pad] half / bfloat16,
 *                            plane 0 real parts, plane 1 imaginary parts
 *         FX_F16_SPLIT:      [SB][C][4][I_pad][S_pad] half, planes hi.re,
 *                            hi.im, lo.re, lo.im (value = hi + lo)
 *         FX_TF32_SPLIT:     [SB][C][2][I_pad][S_pad] float (FP32 planes,
 *                            split into TF32 parts by the X-stage)
 *         I_pad = I rounded up to 16, S_pad = S rounded up to 64; the padding
 *         is written as zeros by fx_correct and fx_channelize_correct. A caller
 *         that fills corr itself must zero spectra S .. S_pad-1 (the X-stage
 *         sums them); padded inputs only reach visibilities that are not
 *         written.
 *   vis   [SB][C][B][4]      complex float, B = N(N+1)/2 baselines,
 *                            b = j(j+1)/2 + i for stations i <= j, products
 *                            (p,q) in the order XX, XY, YX, YY (index 2p+q):
 *                            V = sum_s Y[i,p] * conj(Y[j,q]).
 */
#ifndef FX_GB300_H
#define FX_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t, spelled without the CUDA headers. */
typedef struct CUstream_st *fx_stream;

typedef enum {
    FX_OK = 0,
    FX_ERR_INVALID = -1,     /* bad argument, NULL pointer, size mismatch */
    FX_ERR_CUDA = -2,        /* a CUDA runtime call or kernel launch failed */
    FX_ERR_NOMEM = -3,       /* device or host allocation failed in fx_create */
    FX_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    FX_ERR_UNSUPPORTED = -5  /* valid request this build does not implement */
} fx_status;

/* Complex sample formats of the station data. FX_CI4 (the 4-bit mode): one
 * byte per complex sample, real part in the high nibble and imaginary part
 * in the low nibble, each two's complement in [-8, 7]. */
typedef enum { FX_CI16 = 0, FX_CI8 = 1, FX_CI4 = 2 } fx_format;

/* Arithmetic type of the corrected samples and of the X-stage operands. The
 * FIR and FFT always run in FP32; the X-stage always accumulates in FP32.
 * FX_TF32_SPLIT: FP32 corrected samples in the planar layout; the X-stage
 * splits each into hi (the TF32 part) + lo on the tensor cores and forms
 * hi hi' as TF32 MMAs and the cross terms hi lo' + lo hi' as BF16 MMAs, all
 * with FP32 accumulation, which holds FP32's error bound; at most 512
 * stations, operand_scale must be 1. */
typedef enum { FX_F32 = 0, FX_F16 = 1, FX_BF16 = 2, FX_F16_SPLIT = 3, FX_TF32_SPLIT = 4 } fx_precision;

typedef struct {
    int n_stations;              /* N >= 1 (antenna fields) */
    int n_pols;                  /* P, must be 2 */
    int n_subbands;              /* SB >= 1 */
    int n_channels;              /* C in {16, 64, 256} */
    int n_taps;                  /* T in {4, 8, 16} */
    int n_spectra;               /* S >= 1, spectra integrated per block */
    int format;                  /* fx_format of the raw samples */
    int precision;               /* fx_precision of corr and of the X-stage */
    double sample_rate_hz;       /* subband width / complex sample rate, > 0 */
    const double *h_subband_centre_hz; /* [SB] sky frequency of each subband centre */
    const float *h_taps;         /* [T*C] prototype filter, tap k of channel c at
                                    k*C + c; copied at fx_create */
    float operand_scale;         /* power of two multiplied into FP16/BF16
                                    operands and divided out of vis; 0 means 1 */
    unsigned flags;              /* 0 or a set of FX_FLAG_* bits */
    int host_chunk_subbands;     /* > 0: allocate the double-buffered workspaces of
                                    fx_process_host for chunks of this many
                                    subbands; 0: no host pipeline */
    int max_coarse_shift;        /* with FX_FLAG_STREAMING: largest integer-sample
                                    coarse delay per station (>= 0) */
    int chunk_subbands;          /* with chunk_spectra > 0: subbands per piece of
                                    fx_channelize_correlate (>= 1) */
    int chunk_spectra;           /* > 0: allocate two operand buffers of
                                    chunk_subbands x chunk_spectra (a multiple of 64
                                    dividing n_spectra) for fx_channelize_correlate;
                                    precision FX_F32, FX_F16 or FX_BF16 */
    int max_beams;               /* in [0, 256]; > 0: allocate the beamformer's weight
                                    table for up to this many beams (fx_beamform);
                                    needs precision FX_F16 or FX_BF16 and
                                    n_stations <= 64 */
} fx_params;

/* Streaming form (fx_stream_block): the handle keeps the FIR history of every
 * (subband, station) and room for coarse delays of up to max_coarse_shift
 * samples, and allocates one assembled raw block as workspace. */
#define FX_FLAG_STREAMING 0x1u

/* Tuning hints for the FP32 X-stage (results agree up to FP32 rounding
 * order). Default: 4 x 4-station register tiles from 16 stations up (2 x 4
 * below). SMALL: 2 x 4 tiles. THREE_MULT: 2 x 4 tiles with the
 * three-multiplication complex product (sum xr yr, sum xi yi,
 * sum (xr + xi)(yr - yi)): 3 FMAs per complex MAC instead of 4. */
#define FX_FLAG_XF32_SMALL_TILES 0x2u
#define FX_FLAG_XF32_THREE_MULT 0x4u

/* Failure-detection test hook: the tensor-core X-stage issues no operand
 * loads, so its consumer waits run out after about a millisecond; the call
 * itself succeeds and fx_poll_status() then reports FX_ERR_TIMEOUT. The GPU
 * context stays usable. Never set in production. */
#define FX_FLAG_TEST_NO_LOADS 0x80000000u

typedef struct fx_handle fx_handle;

/* Buffer sizes and padded dimensions implied by a handle's parameters. */
typedef struct {
    size_t raw_bytes;            /* input of fx_channelize */
    size_t chan_bytes;           /* output of fx_channelize */
    size_t corr_bytes;           /* output of fx_correct (depends on precision) */
    size_t vis_bytes;            /* output of fx_correlate */
    int n_inputs;                /* I = N * P */
    int n_inputs_pad;            /* I_pad of the planar layouts */
    int n_spectra_pad;           /* S_pad of the planar layouts */
    int n_baselines;             /* B = N (N + 1) / 2 */
    int corr_planes;             /* 0 for FX_F32, else 2 or 4 */
} fx_sizes;

/* Validate params, copy taps and subband frequencies to the device, build the
 * FFT twiddle table (host FP64, stored FP32) and allocate the workspaces.
 * Uses the current CUDA device. On failure *out is NULL. */
fx_status fx_create(const fx_params *params, fx_handle **out);

/* Free everything fx_create allocated. Synchronises the device first. NULL is
 * a no-op. */
void fx_destroy(fx_handle *h);

/* Message for the last failed call on this thread ("" if none). */
const char *fx_last_error(void);

fx_status fx_query_sizes(const fx_handle *h, fx_sizes *out);

/* Polyphase filter bank (Sec. "Signal processing with GPU kernels": FIR and
 * FFT kernels that channelise each subband; Sec. "Processing steps": fixed
 * to floating point conversion). d_raw: raw layout, format from params;
 * d_chan: chan layout, complex float. For spectrum s and channel c the FIR is
 *   u_s[c] = sum_{k<T} h[k*C + c] * x[(s + k)*C + c],
 * then X_s[m] = sum_c u_s[c] exp(-2 pi i c m / C) (unnormalised), stored at
 * channel (m + C/2) mod C, so channel k has sky frequency
 * f_sb + (k - C/2) * fs / C. The first T-1 spectra' worth of samples in each
 * block are the FIR history carried over from the previous block. */
fx_status fx_channelize(fx_handle *h, const void *d_raw, float *d_chan, fx_stream stream);

/* Fine delay compensation and bandpass correction with the transposing
 * write-back (Sec. "Signal processing with GPU kernels"): for station n,
 *   tau_n(s) = d_delay_begin[n] + (d_delay_end[n] - d_delay_begin[n]) * s / S
 *   Y = X * bandpass[n][k] * gain[n][p] * exp(+2 pi i f_k tau_n(s)).
 * The phase at the block ends is formed in FP64 per (station, channel) and
 * reduced mod 2 pi; the per-sample interpolation, sin/cos and rotation run in
 * FP32. d_delay_begin, d_delay_end: [N] double seconds (device).
 * d_bandpass: [N][C] float or NULL (all ones). d_gains: [N][P] complex float
 * or NULL (all ones). d_chan: chan layout. d_corr: corr layout of the handle's
 * precision; FP16/BF16 values are multiplied by operand_scale before rounding. */
fx_status fx_correct(fx_handle *h, const float *d_chan, const double *d_delay_begin,
                     const double *d_delay_end, const float *d_bandpass,
                     const float *d_gains, void *d_corr, fx_stream stream);

/* fx_channelize followed by fx_correct in one pass, without the channelised
 * intermediate: the same arithmetic per sample (FIR, FFT, then bandpass x gain
 * x exp(i phi) with the FP64-formed phase) and the same corr output as the
 * two calls, for the handle's precision. The per-sample sin/cos is evaluated
 * with a fast intrinsic after an FP32 reduction to [-pi, pi] (absolute error
 * ~4e-7), so results agree with the two-call path to FP32 rounding, not bit
 * for bit. Arguments as for fx_channelize (d_raw) and fx_correct (the rest). */
fx_status fx_channelize_correct(fx_handle *h, const void *d_raw, const double *d_delay_begin,
                                const double *d_delay_end, const float *d_bandpass,
                                const float *d_gains, void *d_corr, fx_stream stream);

/* X-stage correlation (Sec. "Signal processing with GPU kernels": the last
 * kernel correlates all pairs of antenna fields and integrates ~1 s):
 *   vis[sb][k][b(i,j)][2p+q] = sum_{s<S} Y[i,p] conj(Y[j,q])  for i <= j.
 * d_corr: corr layout of the handle's precision; d_vis: vis layout. FP32
 * operands run on the CUDA cores; FP16/BF16/split operands on the tcgen05
 * tensor cores with FP32 accumulation (split: hi*hi' + hi*lo' + lo*hi',
 * accumulator chains restarted every 256 spectra and summed in IEEE FP32);
 * FX_TF32_SPLIT operands (FP32 planar) on the tcgen05 tensor cores as hi/lo
 * parts (hi*hi' in TF32, the cross terms in BF16) with FP32 accumulation,
 * accumulator chains restarted every 64 spectra and summed in IEEE FP32 (FP32
 * accuracy, any station count up to 512; results reproducible run to run). */
fx_status fx_correlate(fx_handle *h, const void *d_corr, float *d_vis, fx_stream stream);

/* End to end from host memory: raw samples in, visibilities out, for all
 * subbands of the handle. The subbands are processed in chunks of
 * host_chunk_subbands (set at fx_create) on three library streams so that the
 * host-to-device copy of chunk k+1 and the device-to-host copy of chunk k-1
 * overlap the fused channelise/correct and the X-stage of chunk k (double
 * buffered device workspaces). The paper's input and output stages run in
 * parallel with GPU processing in the same way (Sec. "Workload distribution":
 * task parallelism of input, GPU control and output). h_raw: raw layout,
 * h_vis: vis layout, h_delay_begin/h_delay_end: [N] double, h_bandpass: [N][C]
 * or NULL, h_gains: [N][P] complex or NULL, all host memory; h_raw and h_vis
 * should be page-locked (cudaHostAlloc / cudaHostRegister) for the copies to
 * overlap. Asynchronous: `stream` waits for the whole pipeline, so
 * synchronising `stream` makes h_vis valid; the host inputs must stay
 * unchanged until then. Uses its own streams, so it is not capturable.
 * FX_ERR_INVALID if the handle was created with host_chunk_subbands = 0. */
fx_status fx_process_host(fx_handle *h, const void *h_raw, const double *h_delay_begin,
                          const double *h_delay_end, const float *h_bandpass, const float *h_gains,
                          float *h_vis, fx_stream stream);

/* ---- F-stage and X-stage over L2-sized pieces ----------------------------
 * The same result as fx_channelize_correct + fx_correlate (integrated over the
 * whole block), computed piece by piece: for each group of chunk_subbands
 * subbands and each run of chunk_spectra spectra, the fused F-stage writes the
 * corrected operands of that piece into one of two handle-owned buffers (sized
 * to stay in L2) and the X-stage adds the piece's products into d_vis, so the
 * corrected block never goes through HBM as a whole. Buffers as in
 * fx_channelize_correct (d_raw, delays, bandpass, gains) and fx_correlate
 * (d_vis, overwritten). Handle needs chunk_spectra > 0 (else FX_ERR_INVALID).
 * Stream-ordered, allocation free, graph-capturable. */
fx_status fx_channelize_correlate(fx_handle *h, const void *d_raw, const double *d_delay_begin,
                                  const double *d_delay_end, const float *d_bandpass, const float *d_gains,
                                  float *d_vis, fx_stream stream);

/* ---- streaming form --------------------------------------------------------
 * Consecutive blocks of a continuous stream (Sec. "Signal processing with GPU
 * kernels": FIR history is carried to the next block; Sec. "Software
 * architecture": the transpose stage applies the coarse, whole-sample delay
 * with a circular buffer and lost data is recorded as metadata).
 *
 * Each call brings S*C new samples per (subband, station, pol):
 * d_new [SB][N][S*C][P] in the handle's format. Station n is read d_n samples
 * late (integer coarse delay, d_coarse_shift [N] int in [0, max_coarse_shift],
 * NULL = 0): the block's spectra use its stream samples
 * [t0 - (T-1)*C - d_n, t0 + S*C - d_n), t0 = first new sample, with samples
 * before the first call taken as zero. The residual (fine) delay is the
 * caller's d_delay_begin/d_delay_end, corrected as in fx_correct. d_flags
 * [N][S] float weights (0 = lost spectrum, NULL = all 1) multiply the
 * corrected samples. Writes d_corr (corr layout of the precision), d_vis (vis
 * layout; NULL = skip the X-stage) and d_counts [B] float = sum_s w_i(s) w_j(s)
 * per baseline (NULL = skip). A coarse shift outside [0, max] is clamped and
 * recorded: fx_poll_status then returns FX_ERR_INVALID. The history advances
 * by one block per call: each call also switches host-side state (which of
 * two history buffers is current), so it must not be captured in a CUDA
 * graph, and consecutive calls must be ordered (same stream, or events).
 * Allocation free; buffers are caller-owned and only read (d_new, delays,
 * bandpass, gains, flags, shifts) or written (d_corr, d_vis, d_counts).
 * Handle needs FX_FLAG_STREAMING; otherwise FX_ERR_INVALID. */
fx_status fx_stream_block(fx_handle *h, const void *d_new, const int *d_coarse_shift,
                          const double *d_delay_begin, const double *d_delay_end,
                          const float *d_bandpass, const float *d_gains, const float *d_flags,
                          void *d_corr, float *d_vis, float *d_counts, fx_stream stream);

/* Zero the streaming history (the stream restarts with zeros before it). */
fx_status fx_stream_reset(fx_handle *h, fx_stream stream);

/* ---- FP32 throughput probe (a measurement aid, not part of the method) ----
 * Not a step of the correlator: it exists only to measure the FP32 FMA peak
 * that the FFMA X-stage's roofline is judged against. Launches `blocks` CTAs of 256 threads that each run `iterations` x 128
 * packed FP32 FMAs (FFMA2) per thread on registers only: 512 flop per
 * iteration per thread, blocks * 256 * iterations * 512 flop in total. The
 * caller times it (events on `stream`) to measure the FP32 FMA peak that the
 * FP32 X-stage's roofline derives from the unit counts. d_sink: one float the
 * kernel may write (device memory, caller-owned). No handle needed. */
fx_status fx_ffma_probe(int iterations, int blocks, float *d_sink, fx_stream stream);

/* ---- coherent beamformer -------------------------------------------------
 * Sec. "Signal processing with GPU kernels": after delay compensation and
 * bandpass correction, coherent beamforming steers each beam with a phase
 * shift and sums over antenna fields, then optionally computes Stokes
 * parameters (otherwise complex voltages are kept). For beam b, pol p,
 * spectrum s, channel k (sky frequency f_k = centre + (k - C/2) fs / C):
 *   B_bp(s, k) = sum_n a_n exp(+2 pi i f_k delta[b][n]) Y_np(s, k)
 * Y = d_corr, the corrected block of fx_channelize_correct / fx_correct in
 * the handle's FP16/BF16 planar layout (divided by operand_scale on output).
 * d_beam_delays [n_beams][N] double: each beam's extra delay per station in
 * seconds, constant over the block; d_station_weights [N] float a_n or NULL
 * (= 1). n_beams in [1, max_beams]. With X = B_b0, Y = B_b1:
 *   FX_BEAM_VOLTAGES     d_out [SB][n_beams][C][S][4] float (Re X, Im X, Re Y, Im Y); tint = 1
 *   FX_BEAM_STOKES_I     d_out [SB][n_beams][C][S/tint] float, I = |X|^2 + |Y|^2
 *   FX_BEAM_STOKES_IQUV  d_out [SB][n_beams][C][S/tint][4] float, Q = |X|^2 - |Y|^2,
 *                        U = 2 Re(X conj Y), V = 2 Im(X conj Y)
 * Stokes values are summed over tint consecutive spectra: tint a power of two
 * <= 32 dividing S. Operands are FP16/BF16 with FP32 accumulation on the
 * tensor cores. Uses the handle's weight table (rewritten every call, so two
 * calls on one handle must be stream-ordered). FX_ERR_INVALID for bad
 * arguments or a handle without max_beams; asynchronous and graph-capturable.
 * A device-side wait that gives up is reported by fx_poll_status. */
typedef enum { FX_BEAM_VOLTAGES = 0, FX_BEAM_STOKES_I = 1, FX_BEAM_STOKES_IQUV = 2 } fx_beam_output;
fx_status fx_beamform(fx_handle *h, const void *d_corr, int n_beams, const double *d_beam_delays,
                      const float *d_station_weights, int output, int tint, float *d_out, fx_stream stream);

/* Incoherent beam (same section: incoherent beamforming first computes the
 * Stokes parameters of each antenna field, then sums over fields). For every
 * subband, channel and spectrum: sum_n a_n Stokes(Y_n0, Y_n1) (definitions as
 * in fx_beamform), summed over tint consecutive spectra (a power of two <= 32
 * dividing S). d_corr: the corrected block of the handle's precision (FP32
 * interleaved, FP16/BF16 planar divided by operand_scale^2 on output, or the
 * FX_TF32_SPLIT planar FP32 block; split FP16: FX_ERR_UNSUPPORTED).
 * d_station_weights [N] float or NULL (= 1). output FX_BEAM_STOKES_I:
 * d_out [SB][C][S/tint] float; FX_BEAM_STOKES_IQUV: d_out [SB][C][S/tint][4].
 * Asynchronous, allocation free, graph-capturable; needs no max_beams. */
fx_status fx_beamform_incoherent(fx_handle *h, const void *d_corr, const float *d_station_weights, int output,
                                 int tint, float *d_out, fx_stream stream);

/* ---- differentiation form ------------------------------------------------
 * With the delay held constant over the block (tau_begin = tau_end = tau) the
 * corrected sample is Y_a = c_a X_a, c_a(k) = g_a exp(2 pi i f_k tau_n(a))
 * (Sec. "Signal processing with GPU kernels": delay compensation is a
 * per-channel phase rotation), so V_ab = c_a conj(c_b) R_ab, where R ("raw
 * visibilities") is what fx_correct with NULL gains and zero delays followed
 * by fx_correlate produces (bandpass included). Both calls below read R in
 * the vis layout; d_gains is [N][P] complex float (NULL = ones), d_delays is
 * [N] double seconds. They need a handle with n_stations <= 512. */

/* Forward from raw visibilities: d_vis = c_a conj(c_b) R for every entry. */
fx_status fx_apply_gains(fx_handle *h, const float *d_raw_vis, const float *d_gains,
                         const double *d_delays, float *d_vis, fx_stream stream);

/* Adjoint of correct + correlate: given d_grad_vis = (dL/dRe V, dL/dIm V) per
 * entry (vis layout) of a real loss L, writes d_grad_gains [N][P] complex
 * float = (dL/dRe g, dL/dIm g) and d_grad_delays [N] double = dL/dtau. Either
 * output may be NULL. Deterministic (fixed-order reductions, FP64 sums). */
fx_status fx_correct_correlate_backward(fx_handle *h, const float *d_raw_vis, const float *d_gains,
                                        const double *d_delays, const float *d_grad_vis,
                                        float *d_grad_gains, double *d_grad_delays, fx_stream stream);

/* Adjoint of correct + correlate when each station's delay moves linearly
 * from d_delay_begin to d_delay_end over the block (the forward correction's
 * interpolation, Sec. "Signal processing with GPU kernels": phases formed at
 * the block's ends and interpolated in between). V then no longer factors
 * through R; with unit gains K = sum_s Y_a conj(Y_b) and
 * M1 = sum_s (s/S) Y_a conj(Y_b) of the delay- and bandpass-corrected block Y,
 * V_ab = g_a conj(g_b) K_ab, dV_ab/dtau_end = +-i 2 pi f_k g_a conj(g_b) M1_ab
 * and dV_ab/dtau_begin = +-i 2 pi f_k g_a conj(g_b) (K_ab - M1_ab) (+ for the
 * first station of the entry, - for the second). The call recomputes Y from
 * the channelised block (d_chan, chan layout) into d_work_corr (corr layout
 * of the handle's precision, caller-owned, corr_bytes of fx_query_sizes,
 * 128-byte aligned), forms K and M1 with the X-stage into d_work_vis
 * (2 x vis_bytes, caller-owned; K first) and writes d_grad_gains [N][P]
 * complex float, d_grad_delay_begin [N] and d_grad_delay_end [N] double
 * (each may be NULL) from d_grad_vis = (dL/dRe V, dL/dIm V). d_bandpass
 * [N][C] or NULL, d_gains [N][P] complex or NULL (= ones). Needs an FX_F32
 * or FX_TF32_SPLIT handle with n_stations <= 512; stream-ordered, allocation
 * free. At equal ends the two delay gradients add up to
 * fx_correct_correlate_backward's. */
fx_status fx_correct_correlate_backward_interp(fx_handle *h, const float *d_chan, const double *d_delay_begin,
                                               const double *d_delay_end, const float *d_bandpass,
                                               const float *d_gains, const float *d_grad_vis, void *d_work_corr,
                                               float *d_work_vis, float *d_grad_gains,
                                               double *d_grad_delay_begin, double *d_grad_delay_end,
                                               fx_stream stream);

/* ---- batching form ----------------------------------------------------------
 * Many uneven correlation jobs (each its own station count, subbands,
 * channels and spectra) in one persistent tensor-core launch. The paper maps
 * subbands statically to GPUs and compiles kernels per observation
 * (Sec. "Workload distribution"); here one launch walks a cost-sorted list of
 * (job, channel, tile) items so small and large jobs share the GPU, and the
 * tile plan (tile width, pipeline depth, item order) comes from an autotuner
 * that times the candidates on the batch itself. */
typedef struct {
    int n_stations;              /* N of this job (P = 2) */
    int n_subbands;              /* SB */
    int n_channels;              /* C (any, the X-stage does not care) */
    int n_spectra;               /* S */
    const void *d_corr;          /* planar corr layout of this job in the batch's
                                    precision: [SB][C][planes][I_pad][S_pad],
                                    I_pad = 2N rounded up to 16, S_pad = S rounded
                                    up to 64, 128-byte aligned, padding zero */
    float *d_vis;                /* vis layout [SB][C][N(N+1)/2][4] complex float */
} fx_job;

typedef struct fx_batch fx_batch;

/* Builds a plan for 1..64 jobs: tensor maps over each job's operands, the
 * device list of work items, a status word. precision is FX_F16, FX_BF16 or
 * FX_F16_SPLIT; operand_scale as in fx_params (0 = 1). Uses a tile plan tuned
 * earlier for the same job shapes in this process, else a default.
 * Allocates device memory (the item list); synchronises. */
fx_status fx_batch_create(const fx_job *jobs, int n_jobs, int precision, float operand_scale,
                          fx_batch **out);

/* Times each candidate tile plan (wide tiles / 128- / 64-column tiles,
 * longest-first / job-major order) with `reps` launches on `stream`, keeps the
 * fastest and remembers it for this set of job shapes. Writes every job's
 * visibilities while doing so. Synchronises; not capturable. */
fx_status fx_batch_autotune(fx_batch *b, int reps, fx_stream stream);

/* One persistent launch correlating every job of the plan; no host work
 * besides the launch, so it can be captured in a CUDA graph. */
fx_status fx_correlate_batched(fx_batch *b, fx_stream stream);

/* The plan in use, as text (tile mode, column tile, stages, accumulator
 * buffers, item order, item count). */
const char *fx_batch_describe(const fx_batch *b);

/* As fx_poll_status, for a batch plan's launches. */
fx_status fx_batch_poll_status(fx_batch *b, int *code);

void fx_batch_destroy(fx_batch *b);

/* Synchronises the device, then reports asynchronous failures of earlier
 * calls: FX_ERR_CUDA for a CUDA error, FX_ERR_TIMEOUT if a bounded device-side
 * wait gave up (each wait has a budget of about two seconds). In the
 * tensor-core X-stages the kernel then drains its in-flight copies, frees its
 * tensor memory and exits, and that call's visibilities are incomplete; in
 * the F-stage kernels (raw rows staged by bulk copies) the wait for a round's
 * rows gives up and the kernel finishes on stale rows, so that call's output
 * is invalid. *code (may be NULL) receives the role that gave up: 1 loader,
 * 2 MMA issuer, 3 epilogue, 4 operand converter (TF32-split X-stage), 6 the
 * F-stage's raw-row wait (code 5, a clamped coarse shift of fx_stream_block,
 * returns FX_ERR_INVALID instead).
 * The status word is cleared by the call. Not capturable in a CUDA graph. */
fx_status fx_poll_status(fx_handle *h, int *code);

/* The same correction as fx_correct with FP32 output, for callers that must
 * not allocate device memory: no handle (fx_create allocates) and no
 * cudaMalloc, cudaFree or allocating library call anywhere on this path. This
 * serves code that owns a fixed device-memory budget handed out at start-up,
 * hosts that forbid their plugins to touch the CUDA allocator, and real-time
 * threads that cannot risk the device-wide synchronisation an allocation may
 * cause. The paper has no counterpart; it is a packaging variant of the
 * delay/bandpass step.
 *
 * The per-call phase table (FP32 pairs: the phase at the block start reduced
 * mod 2 pi and the per-spectrum step, both computed in FP64) lives in a fixed
 * device array built into the library, FX_NOALLOC_MAX_PHASES entries (8 MiB
 * per GPU, held until the process exits); a request with
 * n_subbands * n_stations * n_channels above that limit, or with more than
 * 4096 stations, 65535 subbands or 4194240 spectra, is rejected with
 * FX_ERR_INVALID before anything is launched. The array is committed on a
 * device when the library's correction code is first loaded there (under
 * CUDA's lazy loading: the first call of this entry point or of any
 * correction launch on that device), and the first call on each device also
 * looks up the array's device address (with that device current) and caches
 * it; either may synchronise. So make one warm-up call per device outside any
 * real-time thread and before any stream capture. The cached address belongs
 * to the device's context; after cudaDeviceReset the next call looks it up
 * again. Every call reuses the same array and overwrites all of the entries
 * it reads, so no state carries over between calls; calls whose work overlaps
 * on the GPU (different streams, or different host threads without ordering)
 * race on the array and must be serialised by the caller.
 *
 * Arguments as for fx_correct with an FX_F32 handle: d_subband_centre_hz [SB]
 * double (device), d_delay_begin/d_delay_end [N] double seconds (device),
 * d_bandpass [N][C] float or NULL, d_gains [N][P] complex float or NULL,
 * d_chan the chan layout, d_corr the FP32 (spectrum-blocked) corr layout. Pols = 2,
 * channels in {16, 64, 256}. */
#define FX_NOALLOC_MAX_PHASES (1u << 20)
fx_status fx_correct_f32_noalloc(int n_stations, int n_subbands, int n_channels, int n_spectra,
                                 double sample_rate_hz, const double *d_subband_centre_hz,
                                 const double *d_delay_begin, const double *d_delay_end,
                                 const float *d_bandpass, const float *d_gains, const float *d_chan,
                                 float *d_corr, fx_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* FX_GB300_H */
