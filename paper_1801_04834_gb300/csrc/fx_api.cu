// fx_api.cu -- the C ABI declared in include/fx.h: parameter validation,
// handle and workspace ownership, dispatch to the kernels.
//
// One wrapper per kernel validates shapes and pointers before launching, in
// the spirit of the paper's per-kernel wrapper classes that hold execution
// configuration and buffer sizes (Sec. "Signal processing with GPU kernels").
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace {

thread_local char g_err[512] = "";

fx_status fail(fx_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

fx_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(FX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_pow2(float x)
{
    int e;
    float m = std::frexp(x, &e);
    return x > 0.f && m == 0.5f;
}

}  // namespace

struct fx_handle : fxi::Handle {};

namespace fxi {

bool xstage_supported(const Handle &h)
{
    if (h.p.precision == FX_F32) return true;
    if (h.p.precision == FX_TF32_SPLIT) return xtf32_supported(h.I_pad, h.S_pad);
    int rl, stg;
    unsigned sb;
    return xtc_plan(h, &rl, &stg, &sb);
}

cudaError_t launch_xstage(const Handle &h, const void *corr, float2 *vis, cudaStream_t st, bool accumulate)
{
    switch (h.p.precision) {
    case FX_F32: return launch_xcorr_f32(h, static_cast<const float2 *>(corr), vis, st, accumulate);
    case FX_TF32_SPLIT: return launch_xcorr_tf32(h, static_cast<const float *>(corr), vis, st, accumulate);
    default: return launch_xcorr_tc(h, corr, vis, st, accumulate);
    }
}

// Operand bytes of one piece of fx_channelize_correlate.
static size_t chunk_bytes(const Handle &h)
{
    const size_t G = (size_t)h.p.chunk_subbands, C = h.p.n_channels, T = h.p.chunk_spectra;
    return h.p.precision == FX_F32 ? G * C * T * h.I * sizeof(float2) : G * C * 2 * (size_t)h.I_pad * T * 2;
}

}  // namespace fxi

extern "C" const char *fx_last_error(void) { return g_err; }

extern "C" fx_status fx_create(const fx_params *pp, fx_handle **out)
{
    if (!out) return fail(FX_ERR_INVALID, "fx_create: out is NULL");
    *out = nullptr;
    if (!pp) return fail(FX_ERR_INVALID, "fx_create: params is NULL");
    const fx_params &p = *pp;
    if (p.n_pols != fxi::kPols) return fail(FX_ERR_UNSUPPORTED, "n_pols must be 2 (got %d)", p.n_pols);
    if (p.n_stations < 1 || p.n_stations > 4096)
        return fail(FX_ERR_INVALID, "n_stations out of range (%d)", p.n_stations);
    if (p.n_subbands < 1) return fail(FX_ERR_INVALID, "n_subbands must be >= 1 (got %d)", p.n_subbands);
    if (p.n_spectra < 1) return fail(FX_ERR_INVALID, "n_spectra must be >= 1 (got %d)", p.n_spectra);
    if (p.n_taps < 1) return fail(FX_ERR_INVALID, "n_taps must be >= 1 (got %d)", p.n_taps);
    if (!fxi::ppf_supported(p.n_channels, p.n_taps))
        return fail(FX_ERR_UNSUPPORTED, "channels %d / taps %d not built (C in {16,64,256}, T in {4,8,16})",
                    p.n_channels, p.n_taps);
    if (p.format != FX_CI16 && p.format != FX_CI8 && p.format != FX_CI4)
        return fail(FX_ERR_INVALID, "bad format %d", p.format);
    if (p.precision < FX_F32 || p.precision > FX_TF32_SPLIT)
        return fail(FX_ERR_INVALID, "bad precision %d", p.precision);
    if (!(p.sample_rate_hz > 0)) return fail(FX_ERR_INVALID, "sample_rate_hz must be > 0");
    if (!p.h_subband_centre_hz) return fail(FX_ERR_INVALID, "h_subband_centre_hz is NULL");
    if (!p.h_taps) return fail(FX_ERR_INVALID, "h_taps is NULL");
    if ((p.flags & ~(FX_FLAG_TEST_NO_LOADS | FX_FLAG_STREAMING | FX_FLAG_XF32_SMALL_TILES | FX_FLAG_XF32_THREE_MULT)) != 0)
        return fail(FX_ERR_INVALID, "unknown flags 0x%x", p.flags);
    if (p.max_coarse_shift < 0 || p.max_coarse_shift > (1 << 24))
        return fail(FX_ERR_INVALID, "max_coarse_shift out of range");
    if (p.host_chunk_subbands < 0) return fail(FX_ERR_INVALID, "host_chunk_subbands must be >= 0");
    if (p.max_beams < 0 || p.max_beams > 256) return fail(FX_ERR_INVALID, "max_beams must be in [0, 256]");
    if (p.chunk_spectra < 0 || (p.chunk_spectra > 0 && (p.chunk_spectra % 64 != 0 || p.n_spectra % p.chunk_spectra != 0 ||
                                                        p.chunk_subbands < 1 || p.chunk_subbands > p.n_subbands)))
        return fail(FX_ERR_INVALID, "chunk_spectra must be a multiple of 64 dividing n_spectra, chunk_subbands in [1, SB]");
    if (p.chunk_spectra > 0 && p.precision != FX_F32 && p.precision != FX_F16 && p.precision != FX_BF16)
        return fail(FX_ERR_UNSUPPORTED, "fx_channelize_correlate supports FX_F32, FX_F16 and FX_BF16");
    if (p.max_beams > 0 && ((p.precision != FX_F16 && p.precision != FX_BF16) || p.n_stations > 64))
        return fail(FX_ERR_UNSUPPORTED, "the beamformer needs FX_F16 or FX_BF16 operands and at most 64 stations");
    float scale = p.operand_scale == 0.f ? 1.f : p.operand_scale;
    if (!is_pow2(scale)) return fail(FX_ERR_INVALID, "operand_scale must be a power of two");
    if ((p.precision == FX_F32 || p.precision == FX_TF32_SPLIT) && scale != 1.f)
        return fail(FX_ERR_INVALID, "operand_scale applies to FP16/BF16 only");
    if (p.precision == FX_TF32_SPLIT && p.n_stations > 512)
        return fail(FX_ERR_UNSUPPORTED, "FX_TF32_SPLIT handles at most 512 stations");
    const long long I = 2LL * p.n_stations;
    const long long S = p.n_spectra;
    const long long SB = p.n_subbands;
    // keep every flattened index within 64-bit and the planar row length within int
    if (S > (1 << 24)) return fail(FX_ERR_INVALID, "n_spectra too large");

    fx_handle *h = new (std::nothrow) fx_handle();
    if (!h) return fail(FX_ERR_NOMEM, "host allocation failed");
    h->p = p;
    h->p.h_subband_centre_hz = nullptr;
    h->p.h_taps = nullptr;
    h->I = (int)I;
    h->I_pad = (int)((I + 15) / 16 * 16);
    h->S_pad = (int)((S + 63) / 64 * 64);
    h->B = p.n_stations * (p.n_stations + 1) / 2;
    h->operand_scale = scale;
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (h->num_sms <= 0) h->num_sms = 152;
    h->tc_test_no_tma = (p.flags & FX_FLAG_TEST_NO_LOADS) ? 1 : 0;
    // ~2 s at 2 GHz; ~1 ms for the failure-detection test hook
    h->tc_timeout_cycles = h->tc_test_no_tma ? 2000000LL : 4000000000LL;

    const int C = p.n_channels, T = p.n_taps, N = p.n_stations;
    std::vector<float2> tw(C);
    for (int m = 0; m < C; ++m) {
        const double a = 2.0 * 3.14159265358979323846 * (double)m / (double)C;
        tw[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    // FP32 X-stage form: 4 x 4 tiles from 16 stations up unless the caller asks otherwise
    h->xf32_mode = (p.flags & FX_FLAG_XF32_SMALL_TILES) ? 0 : (p.flags & FX_FLAG_XF32_THREE_MULT) ? 2
                   : N >= 16                              ? 1
                                                          : 0;
    const int rs = h->xf32_mode == 1 ? 4 : 2;
    int ntiles = fxi::xf32_build_tiles(N, rs, nullptr);
    std::vector<int2> tiles(ntiles);
    fxi::xf32_build_tiles(N, rs, tiles.data());
    h->xf32_ntiles = ntiles;

    cudaError_t e = cudaSuccess;
#define FX_TRY(call)                                             \
    do {                                                         \
        e = (call);                                              \
        if (e != cudaSuccess) {                                  \
            fx_destroy(h);                                       \
            return e == cudaErrorMemoryAllocation                \
                       ? fail(FX_ERR_NOMEM, "%s: %s", #call, cudaGetErrorString(e)) \
                       : cuda_fail(e, #call);                    \
        }                                                        \
    } while (0)
    FX_TRY(cudaMalloc(&h->d_taps, sizeof(float) * T * C));
    FX_TRY(cudaMalloc(&h->d_twiddle, sizeof(float2) * C));
    FX_TRY(cudaMalloc(&h->d_centres, sizeof(double) * SB));
    FX_TRY(cudaMalloc(&h->d_phase, sizeof(float2) * SB * N * C));
    FX_TRY(cudaMalloc(&h->d_status, sizeof(int) * 4));
    FX_TRY(cudaMalloc(&h->d_xf32_tiles, sizeof(int2) * ntiles));
    FX_TRY(cudaMalloc(&h->d_adj_partial, sizeof(double) * 4 * (size_t)fxi::adjoint_blocks(*h) * h->I));
    FX_TRY(cudaMemcpy(h->d_taps, p.h_taps, sizeof(float) * T * C, cudaMemcpyHostToDevice));
    FX_TRY(cudaMemcpy(h->d_twiddle, tw.data(), sizeof(float2) * C, cudaMemcpyHostToDevice));
    FX_TRY(cudaMemcpy(h->d_centres, p.h_subband_centre_hz, sizeof(double) * SB,
                      cudaMemcpyHostToDevice));
    FX_TRY(cudaMemcpy(h->d_xf32_tiles, tiles.data(), sizeof(int2) * ntiles, cudaMemcpyHostToDevice));
    FX_TRY(cudaMemset(h->d_status, 0, sizeof(int) * 4));
    if (p.host_chunk_subbands > 0) FX_TRY(fxi::pipe_create(*h, p.host_chunk_subbands));
    if (p.max_beams > 0) FX_TRY(cudaMalloc(&h->d_bfw, fxi::bf_weight_bytes(*h, p.max_beams)));
    if (p.chunk_spectra > 0) {
        FX_TRY(cudaMalloc(&h->d_chunk[0], fxi::chunk_bytes(*h)));
        FX_TRY(cudaMalloc(&h->d_chunk[1], fxi::chunk_bytes(*h)));
    }
    if (p.flags & FX_FLAG_STREAMING) {
        h->hist_len = (T - 1) * C + p.max_coarse_shift;
        const size_t hist_bytes = (size_t)SB * N * h->hist_len * fxi::raw_sample_bytes(*h);
        const size_t block_bytes = (size_t)SB * N * (size_t)(p.n_spectra + T - 1) * C * fxi::raw_sample_bytes(*h);
        FX_TRY(cudaMalloc(&h->d_hist[0], hist_bytes));
        FX_TRY(cudaMalloc(&h->d_hist[1], hist_bytes));
        FX_TRY(cudaMalloc(&h->d_block, block_bytes));
        FX_TRY(cudaMemset(h->d_hist[0], 0, hist_bytes));
        FX_TRY(cudaMemset(h->d_hist[1], 0, hist_bytes));
    }
#undef FX_TRY
    *out = h;
    g_err[0] = 0;
    return FX_OK;
}

extern "C" void fx_destroy(fx_handle *h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    cudaFree(h->d_taps);
    cudaFree(h->d_twiddle);
    cudaFree(h->d_centres);
    cudaFree(h->d_phase);
    cudaFree(h->d_status);
    cudaFree(h->d_xf32_tiles);
    cudaFree(h->d_adj_partial);
    cudaFree(h->d_hist[0]);
    cudaFree(h->d_hist[1]);
    cudaFree(h->d_block);
    cudaFree(h->d_bfw);
    cudaFree(h->d_chunk[0]);
    cudaFree(h->d_chunk[1]);
    fxi::pipe_destroy(*h);
    delete h;
}

extern "C" fx_status fx_query_sizes(const fx_handle *h, fx_sizes *o)
{
    if (!h || !o) return fail(FX_ERR_INVALID, "fx_query_sizes: NULL argument");
    const fx_params &p = h->p;
    const size_t SB = p.n_subbands, N = p.n_stations, C = p.n_channels, S = p.n_spectra;
    const size_t L = (S + p.n_taps - 1) * C;
    const size_t bpc = p.format == FX_CI16 ? 4 : p.format == FX_CI8 ? 2 : 1;   // bytes per complex sample
    o->raw_bytes = SB * N * L * 2 * bpc;
    o->chan_bytes = SB * N * 2 * S * C * sizeof(float2);
    switch (p.precision) {
    case FX_F32: o->corr_bytes = SB * C * ((S + 15) / 16 * 16) * N * 2 * sizeof(float2); o->corr_planes = 0; break;
    case FX_F16:
    case FX_BF16: o->corr_bytes = SB * C * 2 * (size_t)h->I_pad * h->S_pad * 2; o->corr_planes = 2; break;
    case FX_TF32_SPLIT: o->corr_bytes = SB * C * 2 * (size_t)h->I_pad * h->S_pad * 4; o->corr_planes = 2; break;
    default: o->corr_bytes = SB * C * 4 * (size_t)h->I_pad * h->S_pad * 2; o->corr_planes = 4; break;
    }
    o->vis_bytes = SB * C * (size_t)h->B * 4 * sizeof(float2);
    o->n_inputs = h->I;
    o->n_inputs_pad = h->I_pad;
    o->n_spectra_pad = h->S_pad;
    o->n_baselines = h->B;
    return FX_OK;
}

static fx_status check_handle(const fx_handle *h, const char *who)
{
    if (!h) return fail(FX_ERR_INVALID, "%s: handle is NULL", who);
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != h->device)
        return fail(FX_ERR_INVALID, "%s: current device %d is not the handle's device %d", who, dev,
                    h->device);
    return FX_OK;
}

static fx_status after_launch(cudaError_t e, const char *who)
{
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, who);
    return FX_OK;
}

extern "C" fx_status fx_channelize(fx_handle *h, const void *d_raw, float *d_chan, fx_stream stream)
{
    fx_status st = check_handle(h, "fx_channelize");
    if (st) return st;
    if (!d_raw || !d_chan) return fail(FX_ERR_INVALID, "fx_channelize: NULL buffer");
    if (((uintptr_t)d_raw & 15) || ((uintptr_t)d_chan & 15))
        return fail(FX_ERR_INVALID, "fx_channelize: buffers must be 16-byte aligned");
    return after_launch(fxi::launch_ppf(*h, d_raw, reinterpret_cast<float2 *>(d_chan),
                                        (cudaStream_t)stream),
                        "fx_channelize");
}

extern "C" fx_status fx_correct(fx_handle *h, const float *d_chan, const double *d_delay_begin,
                                const double *d_delay_end, const float *d_bandpass,
                                const float *d_gains, void *d_corr, fx_stream stream)
{
    fx_status st = check_handle(h, "fx_correct");
    if (st) return st;
    if (!d_chan || !d_corr || !d_delay_begin || !d_delay_end)
        return fail(FX_ERR_INVALID, "fx_correct: NULL buffer");
    if (((uintptr_t)d_chan & 15) || ((uintptr_t)d_corr & 15) || ((uintptr_t)d_gains & 7) ||
        ((uintptr_t)d_bandpass & 3) || ((uintptr_t)d_delay_begin & 7) || ((uintptr_t)d_delay_end & 7))
        return fail(FX_ERR_INVALID, "fx_correct: misaligned buffer");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = fxi::launch_phase_table(*h, d_delay_begin, d_delay_end, s);
    if (e == cudaSuccess)
        e = fxi::launch_correct(*h, reinterpret_cast<const float2 *>(d_chan), d_bandpass,
                                reinterpret_cast<const float2 *>(d_gains), d_corr, s);
    return after_launch(e, "fx_correct");
}

extern "C" fx_status fx_channelize_correct(fx_handle *h, const void *d_raw, const double *d_delay_begin,
                                           const double *d_delay_end, const float *d_bandpass,
                                           const float *d_gains, void *d_corr, fx_stream stream)
{
    const char *who = "fx_channelize_correct";
    fx_status st = check_handle(h, who);
    if (st) return st;
    if (!d_raw || !d_corr || !d_delay_begin || !d_delay_end) return fail(FX_ERR_INVALID, "%s: NULL buffer", who);
    if (((uintptr_t)d_raw & 15) || ((uintptr_t)d_corr & 15) || ((uintptr_t)d_gains & 7) ||
        ((uintptr_t)d_bandpass & 3) || ((uintptr_t)d_delay_begin & 7) || ((uintptr_t)d_delay_end & 7))
        return fail(FX_ERR_INVALID, "%s: misaligned buffer", who);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = fxi::launch_phase_table(*h, d_delay_begin, d_delay_end, s);
    if (e == cudaSuccess)
        e = fxi::launch_channelize_correct(*h, d_raw, d_bandpass, reinterpret_cast<const float2 *>(d_gains), d_corr, s);
    return after_launch(e, who);
}

extern "C" fx_status fx_process_host(fx_handle *h, const void *h_raw, const double *h_delay_begin,
                                     const double *h_delay_end, const float *h_bandpass, const float *h_gains,
                                     float *h_vis, fx_stream stream)
{
    const char *who = "fx_process_host";
    fx_status st = check_handle(h, who);
    if (st) return st;
    if (!h->pipe) return fail(FX_ERR_INVALID, "%s: handle was created with host_chunk_subbands = 0", who);
    if (!h_raw || !h_vis || !h_delay_begin || !h_delay_end) return fail(FX_ERR_INVALID, "%s: NULL buffer", who);
    if (!fxi::xstage_supported(*h)) return fail(FX_ERR_UNSUPPORTED, "%s: no tensor-core plan", who);
    return after_launch(fxi::pipe_run(*h, h_raw, h_delay_begin, h_delay_end, h_bandpass, h_gains, h_vis,
                                      (cudaStream_t)stream),
                        who);
}

extern "C" fx_status fx_ffma_probe(int iterations, int blocks, float *d_sink, fx_stream stream)
{
    if (iterations < 1 || blocks < 1 || !d_sink) return fail(FX_ERR_INVALID, "fx_ffma_probe: bad arguments");
    const cudaError_t e = fxi::launch_ffma_probe(iterations, blocks, d_sink, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fx_ffma_probe");
    return FX_OK;
}

extern "C" fx_status fx_beamform(fx_handle *h, const void *d_corr, int n_beams, const double *d_beam_delays,
                                 const float *d_station_weights, int output, int tint, float *d_out, fx_stream stream)
{
    const char *who = "fx_beamform";
    fx_status st = check_handle(h, who);
    if (st) return st;
    if (!h->d_bfw) return fail(FX_ERR_INVALID, "%s: handle was created with max_beams = 0", who);
    if (!d_corr || !d_beam_delays || !d_out) return fail(FX_ERR_INVALID, "%s: NULL buffer", who);
    if (n_beams < 1 || n_beams > h->p.max_beams)
        return fail(FX_ERR_INVALID, "%s: n_beams must be in [1, %d]", who, h->p.max_beams);
    if (output < FX_BEAM_VOLTAGES || output > FX_BEAM_STOKES_IQUV) return fail(FX_ERR_INVALID, "%s: bad output", who);
    if (tint < 1 || tint > 32 || !is_pow2(tint) || h->p.n_spectra % tint != 0 ||
        (output == FX_BEAM_VOLTAGES && tint != 1))
        return fail(FX_ERR_INVALID, "%s: tint must be a power of two <= 32 dividing S (1 for voltages)", who);
    if (((uintptr_t)d_corr & 15) || ((uintptr_t)d_out & 15) || ((uintptr_t)d_beam_delays & 7) ||
        ((uintptr_t)d_station_weights & 3))
        return fail(FX_ERR_INVALID, "%s: misaligned buffer", who);
    return after_launch(fxi::launch_beamform(*h, d_corr, n_beams, d_beam_delays, d_station_weights, output, tint,
                                             d_out, (cudaStream_t)stream),
                        who);
}

extern "C" fx_status fx_beamform_incoherent(fx_handle *h, const void *d_corr, const float *d_station_weights,
                                            int output, int tint, float *d_out, fx_stream stream)
{
    const char *who = "fx_beamform_incoherent";
    fx_status st = check_handle(h, who);
    if (st) return st;
    if (h->p.precision == FX_F16_SPLIT) return fail(FX_ERR_UNSUPPORTED, "%s: split FP16 operands", who);
    if (!d_corr || !d_out) return fail(FX_ERR_INVALID, "%s: NULL buffer", who);
    if (output != FX_BEAM_STOKES_I && output != FX_BEAM_STOKES_IQUV)
        return fail(FX_ERR_INVALID, "%s: output must be FX_BEAM_STOKES_I or FX_BEAM_STOKES_IQUV", who);
    if (tint < 1 || tint > 32 || !is_pow2(tint) || h->p.n_spectra % tint != 0)
        return fail(FX_ERR_INVALID, "%s: tint must be a power of two <= 32 dividing S", who);
    if (((uintptr_t)d_corr & 15) || ((uintptr_t)d_out & 15) || ((uintptr_t)d_station_weights & 3))
        return fail(FX_ERR_INVALID, "%s: misaligned buffer", who);
    return after_launch(fxi::launch_beamform_incoherent(*h, d_corr, d_station_weights, output, tint, d_out,
                                                        (cudaStream_t)stream),
                        who);
}

extern "C" fx_status fx_channelize_correlate(fx_handle *h, const void *d_raw, const double *d_delay_begin,
                                             const double *d_delay_end, const float *d_bandpass, const float *d_gains,
                                             float *d_vis, fx_stream stream)
{
    const char *who = "fx_channelize_correlate";
    fx_status st = check_handle(h, who);
    if (st) return st;
    if (!h->d_chunk[0]) return fail(FX_ERR_INVALID, "%s: handle was created with chunk_spectra = 0", who);
    if (!d_raw || !d_vis || !d_delay_begin || !d_delay_end) return fail(FX_ERR_INVALID, "%s: NULL buffer", who);
    if (((uintptr_t)d_raw & 15) || ((uintptr_t)d_vis & 15) || ((uintptr_t)d_gains & 7) ||
        ((uintptr_t)d_bandpass & 3) || ((uintptr_t)d_delay_begin & 7) || ((uintptr_t)d_delay_end & 7))
        return fail(FX_ERR_INVALID, "%s: misaligned buffer", who);
    if (!fxi::xstage_supported(*h)) return fail(FX_ERR_UNSUPPORTED, "%s: no tensor-core plan", who);
    cudaStream_t s = (cudaStream_t)stream;
    const int SB = h->p.n_subbands, N = h->p.n_stations, C = h->p.n_channels, S = h->p.n_spectra;
    const int G = h->p.chunk_subbands, TC = h->p.chunk_spectra;
    const size_t raw_sb = (size_t)N * (S + h->p.n_taps - 1) * C * fxi::raw_sample_bytes(*h);   // bytes per subband
    const size_t vis_sb = (size_t)C * h->B * 4;                                                 // float2 per subband
    const float2 *gains = reinterpret_cast<const float2 *>(d_gains);
    cudaError_t e = fxi::launch_phase_table(*h, d_delay_begin, d_delay_end, s);
    long long k = 0;
    for (int g0 = 0; g0 < SB && e == cudaSuccess; g0 += G) {
        fxi::Handle v = *h;                                   // view of subbands [g0, g0 + gs)
        const int gs = SB - g0 < G ? SB - g0 : G;
        v.p.n_subbands = gs;
        v.d_centres = h->d_centres + g0;
        v.d_phase = h->d_phase + (size_t)g0 * N * C;
        const void *raw_g = static_cast<const unsigned char *>(d_raw) + (size_t)g0 * raw_sb;
        float2 *vis_g = reinterpret_cast<float2 *>(d_vis) + (size_t)g0 * vis_sb;
        fxi::Handle x = v;                                    // the X-stage's view of one piece
        x.p.n_spectra = TC;
        x.S_pad = TC;
        for (int t0 = 0; t0 < S && e == cudaSuccess; t0 += TC, ++k) {
            void *buf = h->d_chunk[k & 1];
            const fxi::FWindow w{t0, t0 + TC, TC};
            e = fxi::launch_channelize_correct(v, raw_g, d_bandpass, gains, buf, s, nullptr, &w);
            if (e == cudaSuccess) e = fxi::launch_xstage(x, buf, vis_g, s, t0 > 0);
        }
    }
    return after_launch(e, who);
}

extern "C" fx_status fx_stream_reset(fx_handle *h, fx_stream stream)
{
    fx_status st = check_handle(h, "fx_stream_reset");
    if (st) return st;
    if (!h->d_block) return fail(FX_ERR_INVALID, "fx_stream_reset: handle was created without FX_FLAG_STREAMING");
    const size_t hist_bytes =
        (size_t)h->p.n_subbands * h->p.n_stations * h->hist_len * fxi::raw_sample_bytes(*h);
    cudaError_t e = cudaMemsetAsync(h->d_hist[0], 0, hist_bytes, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_hist[1], 0, hist_bytes, (cudaStream_t)stream);
    return after_launch(e, "fx_stream_reset");
}

extern "C" fx_status fx_stream_block(fx_handle *h, const void *d_new, const int *d_coarse_shift,
                                     const double *d_delay_begin, const double *d_delay_end,
                                     const float *d_bandpass, const float *d_gains, const float *d_flags,
                                     void *d_corr, float *d_vis, float *d_counts, fx_stream stream)
{
    const char *who = "fx_stream_block";
    fx_status st = check_handle(h, who);
    if (st) return st;
    if (!h->d_block) return fail(FX_ERR_INVALID, "%s: handle was created without FX_FLAG_STREAMING", who);
    if (!d_new || !d_corr || !d_delay_begin || !d_delay_end) return fail(FX_ERR_INVALID, "%s: NULL buffer", who);
    if (((uintptr_t)d_new & 15) || ((uintptr_t)d_corr & 15) || ((uintptr_t)d_vis & 15) ||
        ((uintptr_t)d_coarse_shift & 3) || ((uintptr_t)d_flags & 3) || ((uintptr_t)d_counts & 3) ||
        ((uintptr_t)d_gains & 7) || ((uintptr_t)d_bandpass & 3) || ((uintptr_t)d_delay_begin & 7) ||
        ((uintptr_t)d_delay_end & 7))
        return fail(FX_ERR_INVALID, "%s: misaligned buffer", who);
    if (d_vis && !fxi::xstage_supported(*h)) return fail(FX_ERR_UNSUPPORTED, "%s: no tensor-core plan", who);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = fxi::launch_stream_assemble(*h, d_new, d_coarse_shift, s);
    if (e == cudaSuccess) e = fxi::launch_phase_table(*h, d_delay_begin, d_delay_end, s);
    if (e == cudaSuccess)
        e = fxi::launch_channelize_correct(*h, h->d_block, d_bandpass, reinterpret_cast<const float2 *>(d_gains),
                                           d_corr, s, d_flags);
    if (e == cudaSuccess && d_vis) {
        float2 *vis = reinterpret_cast<float2 *>(d_vis);
        e = fxi::launch_xstage(*h, d_corr, vis, s);
    }
    if (e == cudaSuccess && d_counts) e = fxi::launch_baseline_counts(*h, d_flags, d_counts, s);
    if (e == cudaSuccess) e = fxi::launch_stream_history(*h, d_new, s);
    return after_launch(e, who);
}

extern "C" fx_status fx_poll_status(fx_handle *h, int *code)
{
    fx_status st = check_handle(h, "fx_poll_status");
    if (st) return st;
    if (code) *code = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "fx_poll_status: asynchronous error");
    int w[2] = {0, 0};
    e = cudaMemcpy(w, h->d_status, sizeof(w), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fx_poll_status");
    if (w[0] != 0) {
        cudaMemset(h->d_status, 0, sizeof(int) * 4);
        if (code) *code = w[0];
        if (w[0] == 5) return fail(FX_ERR_INVALID, "a coarse shift was outside [0, max_coarse_shift] and was clamped");
        return fail(FX_ERR_TIMEOUT, "device-side wait gave up (role %d, CTA %d)", w[0], w[1]);
    }
    return FX_OK;
}

extern "C" fx_status fx_correlate(fx_handle *h, const void *d_corr, float *d_vis, fx_stream stream)
{
    fx_status st = check_handle(h, "fx_correlate");
    if (st) return st;
    if (!d_corr || !d_vis) return fail(FX_ERR_INVALID, "fx_correlate: NULL buffer");
    if (((uintptr_t)d_corr & 127) || ((uintptr_t)d_vis & 15))
        return fail(FX_ERR_INVALID, "fx_correlate: corr must be 128-byte and vis 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    float2 *vis = reinterpret_cast<float2 *>(d_vis);
    if (!fxi::xstage_supported(*h))
        return fail(FX_ERR_UNSUPPORTED, "fx_correlate: tensor-core X-stage needs <= 128 stations (<= 100 for split FP16)");
    return after_launch(fxi::launch_xstage(*h, d_corr, vis, s), "fx_correlate");
}

extern "C" fx_status fx_apply_gains(fx_handle *h, const float *d_raw_vis, const float *d_gains,
                                    const double *d_delays, float *d_vis, fx_stream stream)
{
    fx_status st = check_handle(h, "fx_apply_gains");
    if (st) return st;
    if (!d_raw_vis || !d_delays || !d_vis) return fail(FX_ERR_INVALID, "fx_apply_gains: NULL buffer");
    if (((uintptr_t)d_raw_vis & 7) || ((uintptr_t)d_vis & 7) || ((uintptr_t)d_gains & 7) || ((uintptr_t)d_delays & 7))
        return fail(FX_ERR_INVALID, "fx_apply_gains: misaligned buffer");
    return after_launch(fxi::launch_apply_gains(*h, reinterpret_cast<const float2 *>(d_raw_vis),
                                                reinterpret_cast<const float2 *>(d_gains), d_delays,
                                                reinterpret_cast<float2 *>(d_vis), (cudaStream_t)stream),
                        "fx_apply_gains");
}

extern "C" fx_status fx_correct_correlate_backward(fx_handle *h, const float *d_raw_vis, const float *d_gains,
                                                   const double *d_delays, const float *d_grad_vis,
                                                   float *d_grad_gains, double *d_grad_delays, fx_stream stream)
{
    const char *who = "fx_correct_correlate_backward";
    fx_status st = check_handle(h, who);
    if (st) return st;
    if (!d_raw_vis || !d_delays || !d_grad_vis) return fail(FX_ERR_INVALID, "%s: NULL buffer", who);
    if (h->I > 1024) return fail(FX_ERR_UNSUPPORTED, "%s: at most 512 stations", who);
    if (((uintptr_t)d_raw_vis & 7) || ((uintptr_t)d_grad_vis & 7) || ((uintptr_t)d_gains & 7) ||
        ((uintptr_t)d_delays & 7) || ((uintptr_t)d_grad_gains & 7) || ((uintptr_t)d_grad_delays & 7))
        return fail(FX_ERR_INVALID, "%s: misaligned buffer", who);
    return after_launch(fxi::launch_adjoint(*h, reinterpret_cast<const float2 *>(d_raw_vis),
                                            reinterpret_cast<const float2 *>(d_grad_vis),
                                            reinterpret_cast<const float2 *>(d_gains), d_delays,
                                            reinterpret_cast<float2 *>(d_grad_gains), d_grad_delays,
                                            (cudaStream_t)stream),
                        who);
}

extern "C" fx_status fx_correct_correlate_backward_interp(
    fx_handle *h, const float *d_chan, const double *d_delay_begin, const double *d_delay_end,
    const float *d_bandpass, const float *d_gains, const float *d_grad_vis, void *d_work_corr, float *d_work_vis,
    float *d_grad_gains, double *d_grad_delay_begin, double *d_grad_delay_end, fx_stream stream)
{
    const char *who = "fx_correct_correlate_backward_interp";
    fx_status st = check_handle(h, who);
    if (st) return st;
    if (h->p.precision != FX_F32 && h->p.precision != FX_TF32_SPLIT)
        return fail(FX_ERR_UNSUPPORTED, "%s: needs an FX_F32 or FX_TF32_SPLIT handle", who);
    if (!d_chan || !d_delay_begin || !d_delay_end || !d_grad_vis || !d_work_corr || !d_work_vis)
        return fail(FX_ERR_INVALID, "%s: NULL buffer", who);
    if (h->I > 1024) return fail(FX_ERR_UNSUPPORTED, "%s: at most 512 stations", who);
    if (!fxi::xstage_supported(*h)) return fail(FX_ERR_UNSUPPORTED, "%s: X-stage not supported for this shape", who);
    if (((uintptr_t)d_chan & 15) || ((uintptr_t)d_work_corr & 127) || ((uintptr_t)d_work_vis & 15) ||
        ((uintptr_t)d_grad_vis & 7) || ((uintptr_t)d_gains & 7) || ((uintptr_t)d_bandpass & 3) ||
        ((uintptr_t)d_delay_begin & 7) || ((uintptr_t)d_delay_end & 7) || ((uintptr_t)d_grad_gains & 7) ||
        ((uintptr_t)d_grad_delay_begin & 7) || ((uintptr_t)d_grad_delay_end & 7))
        return fail(FX_ERR_INVALID, "%s: misaligned buffer", who);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vis_len = (size_t)h->p.n_subbands * h->p.n_channels * h->B * 4;   // float2 per visibility block
    float2 *K = reinterpret_cast<float2 *>(d_work_vis), *M1 = K + vis_len;
    cudaError_t e = fxi::launch_phase_table(*h, d_delay_begin, d_delay_end, s);
    if (e == cudaSuccess)   // the corrected block with unit gains: Y
        e = fxi::launch_correct(*h, reinterpret_cast<const float2 *>(d_chan), d_bandpass, nullptr, d_work_corr, s);
    if (e == cudaSuccess) e = fxi::launch_xstage(*h, d_work_corr, K, s);              // K = sum Y Y^H
    if (e == cudaSuccess) e = fxi::launch_weight_spectra(*h, d_work_corr, s);         // Y sqrt(s/S)
    if (e == cudaSuccess) e = fxi::launch_xstage(*h, d_work_corr, M1, s);             // M1 = sum (s/S) Y Y^H
    if (e == cudaSuccess)
        e = fxi::launch_adjoint_interp(*h, K, M1, reinterpret_cast<const float2 *>(d_grad_vis),
                                       reinterpret_cast<const float2 *>(d_gains),
                                       reinterpret_cast<float2 *>(d_grad_gains), d_grad_delay_begin,
                                       d_grad_delay_end, s);
    return after_launch(e, who);
}

extern "C" fx_status fx_batch_create(const fx_job *jobs, int n_jobs, int precision, float operand_scale,
                                     fx_batch **out)
{
    const char *who = "fx_batch_create";
    if (!out) return fail(FX_ERR_INVALID, "%s: out is NULL", who);
    *out = nullptr;
    if (!jobs || n_jobs < 1 || n_jobs > 64) return fail(FX_ERR_INVALID, "%s: need 1..64 jobs", who);
    if (precision != FX_F16 && precision != FX_BF16 && precision != FX_F16_SPLIT)
        return fail(FX_ERR_INVALID, "%s: precision must be FX_F16, FX_BF16 or FX_F16_SPLIT", who);
    const float scale = operand_scale == 0.f ? 1.f : operand_scale;
    if (!is_pow2(scale)) return fail(FX_ERR_INVALID, "%s: operand_scale must be a power of two", who);
    for (int j = 0; j < n_jobs; ++j) {
        const fx_job &J = jobs[j];
        if (J.n_stations < 1 || J.n_stations > 4096 || J.n_subbands < 1 || J.n_channels < 1 || J.n_spectra < 1 ||
            J.n_spectra > (1 << 24))
            return fail(FX_ERR_INVALID, "%s: job %d has bad sizes", who, j);
        if (!J.d_corr || !J.d_vis) return fail(FX_ERR_INVALID, "%s: job %d has a NULL buffer", who, j);
        if (((uintptr_t)J.d_corr & 127) || ((uintptr_t)J.d_vis & 15))
            return fail(FX_ERR_INVALID, "%s: job %d: corr must be 128-byte, vis 16-byte aligned", who, j);
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const char *why = "";
    cudaError_t e = fxi_batch_create(jobs, n_jobs, precision, scale, sms, out, &why);
    if (e == cudaErrorMemoryAllocation) return fail(FX_ERR_NOMEM, "%s: %s", who, why);
    if (e == cudaErrorNotSupported) return fail(FX_ERR_UNSUPPORTED, "%s: %s", who, why);
    if (e != cudaSuccess) return fail(FX_ERR_INVALID, "%s: %s (%s)", who, why, cudaGetErrorString(e));
    return FX_OK;
}

static fx_status check_batch(const fx_batch *b, const char *who)
{
    if (!b) return fail(FX_ERR_INVALID, "%s: batch is NULL", who);
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != fxi_batch_device(b)) return fail(FX_ERR_INVALID, "%s: wrong current device", who);
    return FX_OK;
}

extern "C" fx_status fx_batch_autotune(fx_batch *b, int reps, fx_stream stream)
{
    fx_status st = check_batch(b, "fx_batch_autotune");
    if (st) return st;
    if (reps < 1) reps = 1;
    return after_launch(fxi_batch_autotune(b, reps, (cudaStream_t)stream), "fx_batch_autotune");
}

extern "C" fx_status fx_correlate_batched(fx_batch *b, fx_stream stream)
{
    fx_status st = check_batch(b, "fx_correlate_batched");
    if (st) return st;
    return after_launch(fxi_batch_launch(b, (cudaStream_t)stream), "fx_correlate_batched");
}

extern "C" const char *fx_batch_describe(const fx_batch *b) { return b ? fxi_batch_describe(b) : ""; }

extern "C" fx_status fx_batch_poll_status(fx_batch *b, int *code)
{
    fx_status st = check_batch(b, "fx_batch_poll_status");
    if (st) return st;
    if (code) *code = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "fx_batch_poll_status: asynchronous error");
    int w[2] = {0, 0};
    e = cudaMemcpy(w, fxi_batch_status(b), sizeof(w), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fx_batch_poll_status");
    if (w[0] != 0) {
        cudaMemset(fxi_batch_status(b), 0, sizeof(int) * 4);
        if (code) *code = w[0];
        return fail(FX_ERR_TIMEOUT, "device-side wait gave up (role %d, CTA %d)", w[0], w[1]);
    }
    return FX_OK;
}

extern "C" void fx_batch_destroy(fx_batch *b) { fxi_batch_destroy(b); }

// Handle-free correction for callers that cannot allocate device memory; the
// phase table lives in a fixed device array in correct.cu (see fx.h).
extern "C" fx_status fx_correct_f32_noalloc(int n_stations, int n_subbands, int n_channels, int n_spectra,
                                            double sample_rate_hz, const double *d_subband_centre_hz,
                                            const double *d_delay_begin, const double *d_delay_end,
                                            const float *d_bandpass, const float *d_gains, const float *d_chan,
                                            float *d_corr, fx_stream stream)
{
    const char *who = "fx_correct_f32_noalloc";
    if (n_stations < 1 || n_subbands < 1 || n_spectra < 1)
        return fail(FX_ERR_INVALID, "%s: sizes must be >= 1", who);
    if (n_channels != 16 && n_channels != 64 && n_channels != 256)
        return fail(FX_ERR_UNSUPPORTED, "%s: channels must be 16, 64 or 256 (got %d)", who, n_channels);
    if (!(sample_rate_hz > 0)) return fail(FX_ERR_INVALID, "%s: sample_rate_hz must be > 0", who);
    const long long entries = (long long)n_subbands * n_stations * n_channels;
    if (entries > (long long)FX_NOALLOC_MAX_PHASES)
        return fail(FX_ERR_INVALID,
                    "%s: subbands x stations x channels = %lld exceeds the built-in phase table of %u entries",
                    who, entries, FX_NOALLOC_MAX_PHASES);
    // the correction kernel's grid: (stations, runs of four 16-spectrum blocks, subbands)
    if (n_subbands > 65535 || n_stations > 4096 || ((n_spectra + 15) / 16 + 3) / 4 > 65535)
        return fail(FX_ERR_INVALID, "%s: sizes out of range (subbands <= 65535, stations <= 4096, "
                    "spectra <= 4194240)", who);
    if (!d_subband_centre_hz || !d_delay_begin || !d_delay_end || !d_chan || !d_corr)
        return fail(FX_ERR_INVALID, "%s: NULL buffer", who);
    if (((uintptr_t)d_chan & 15) || ((uintptr_t)d_corr & 15) || ((uintptr_t)d_gains & 7) ||
        ((uintptr_t)d_bandpass & 3) || ((uintptr_t)d_delay_begin & 7) || ((uintptr_t)d_delay_end & 7) ||
        ((uintptr_t)d_subband_centre_hz & 7))
        return fail(FX_ERR_INVALID, "%s: misaligned buffer", who);
    cudaError_t e = fxi::launch_correct_f32_noalloc(
        n_stations, n_subbands, n_channels, n_spectra, sample_rate_hz, d_subband_centre_hz, d_delay_begin,
        d_delay_end, d_bandpass, reinterpret_cast<const float2 *>(d_gains), reinterpret_cast<const float2 *>(d_chan),
        reinterpret_cast<float2 *>(d_corr), (cudaStream_t)stream);
    return after_launch(e, who);
}
