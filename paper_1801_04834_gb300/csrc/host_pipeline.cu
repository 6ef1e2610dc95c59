// host_pipeline.cu -- fx_process_host: the hot path from host memory to host
// memory with the copies overlapped with compute.
//
// Paper, Sec. "Workload distribution": receiving input, GPU transfers and
// kernels, and output run as parallel tasks on the same hardware. Here that is
// a three-stream software pipeline over chunks of subbands (subbands are
// independent):
//
//   s_in   : H2D raw chunk k into buffer k%2        -> in_done[k%2]
//   s_comp : phase table, fused channelise+correct,
//            X-stage of chunk k                     -> comp_done[k%2]
//   s_out  : D2H visibilities of chunk k            -> out_done[k%2]
//
// Buffer b = k%2 is reused by chunk k+2 only after comp_done (raw, corr) and
// out_done (vis) of chunk k, so at any time one chunk is being uploaded, one
// computed and one downloaded. The kernels are the ordinary launchers run on a
// view of the handle restricted to the chunk's subbands.
#include "internal.h"

namespace fxi {

struct HostPipe {
    int chunk = 0;
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    void *d_raw[2] = {nullptr, nullptr};
    void *d_corr[2] = {nullptr, nullptr};
    float2 *d_vis[2] = {nullptr, nullptr};
    double *d_tau = nullptr;        // [2][N]: begin, end
    float *d_bp = nullptr;          // [N][C]
    float2 *d_gain = nullptr;       // [N][P]
    cudaEvent_t ev_start = nullptr, ev_params = nullptr;
    cudaEvent_t in_done[2] = {}, comp_done[2] = {}, out_done[2] = {};
    size_t raw_sb = 0, corr_sb = 0, vis_sb = 0;   // bytes per subband
};

static size_t corr_bytes_per_subband(const Handle &h)
{
    const size_t C = h.p.n_channels, S = h.p.n_spectra;
    switch (h.p.precision) {
    case FX_F32: return C * ((S + 15) / 16 * 16) * h.I * sizeof(float2);   // spectrum-blocked, ceil16(S)
    case FX_F16:
    case FX_BF16: return C * 2 * (size_t)h.I_pad * h.S_pad * 2;
    case FX_TF32_SPLIT: return C * 2 * (size_t)h.I_pad * h.S_pad * 4;
    default: return C * 4 * (size_t)h.I_pad * h.S_pad * 2;
    }
}

void pipe_destroy(Handle &h)
{
    HostPipe *P = h.pipe;
    if (!P) return;
    for (int b = 0; b < 2; ++b) {
        cudaFree(P->d_raw[b]);
        cudaFree(P->d_corr[b]);
        cudaFree(P->d_vis[b]);
        if (P->in_done[b]) cudaEventDestroy(P->in_done[b]);
        if (P->comp_done[b]) cudaEventDestroy(P->comp_done[b]);
        if (P->out_done[b]) cudaEventDestroy(P->out_done[b]);
    }
    cudaFree(P->d_tau);
    cudaFree(P->d_bp);
    cudaFree(P->d_gain);
    if (P->ev_start) cudaEventDestroy(P->ev_start);
    if (P->ev_params) cudaEventDestroy(P->ev_params);
    if (P->s_in) cudaStreamDestroy(P->s_in);
    if (P->s_comp) cudaStreamDestroy(P->s_comp);
    if (P->s_out) cudaStreamDestroy(P->s_out);
    delete P;
    h.pipe = nullptr;
}

cudaError_t pipe_create(Handle &h, int chunk)
{
    HostPipe *P = new HostPipe();
    h.pipe = P;
    const int SB = h.p.n_subbands, N = h.p.n_stations, C = h.p.n_channels;
    P->chunk = chunk < SB ? chunk : SB;
    const size_t L = (size_t)(h.p.n_spectra + h.p.n_taps - 1) * C;
    P->raw_sb = (size_t)N * L * 2 * (h.p.format == FX_CI16 ? 4 : h.p.format == FX_CI8 ? 2 : 1);
    P->corr_sb = corr_bytes_per_subband(h);
    P->vis_sb = (size_t)C * h.B * 4 * sizeof(float2);
    cudaError_t e = cudaSuccess;
#define PIPE_TRY(x)               \
    do {                          \
        e = (x);                  \
        if (e != cudaSuccess) {   \
            pipe_destroy(h);      \
            return e;             \
        }                         \
    } while (0)
    for (int b = 0; b < 2; ++b) {
        PIPE_TRY(cudaMalloc(&P->d_raw[b], P->raw_sb * P->chunk));
        PIPE_TRY(cudaMalloc(&P->d_corr[b], P->corr_sb * P->chunk));
        PIPE_TRY(cudaMalloc(&P->d_vis[b], P->vis_sb * P->chunk));
        PIPE_TRY(cudaEventCreateWithFlags(&P->in_done[b], cudaEventDisableTiming));
        PIPE_TRY(cudaEventCreateWithFlags(&P->comp_done[b], cudaEventDisableTiming));
        PIPE_TRY(cudaEventCreateWithFlags(&P->out_done[b], cudaEventDisableTiming));
    }
    PIPE_TRY(cudaMalloc(&P->d_tau, sizeof(double) * 2 * N));
    PIPE_TRY(cudaMalloc(&P->d_bp, sizeof(float) * N * C));
    PIPE_TRY(cudaMalloc(&P->d_gain, sizeof(float2) * N * kPols));
    PIPE_TRY(cudaEventCreateWithFlags(&P->ev_start, cudaEventDisableTiming));
    PIPE_TRY(cudaEventCreateWithFlags(&P->ev_params, cudaEventDisableTiming));
    PIPE_TRY(cudaStreamCreateWithFlags(&P->s_in, cudaStreamNonBlocking));
    PIPE_TRY(cudaStreamCreateWithFlags(&P->s_comp, cudaStreamNonBlocking));
    PIPE_TRY(cudaStreamCreateWithFlags(&P->s_out, cudaStreamNonBlocking));
#undef PIPE_TRY
    return cudaSuccess;
}

cudaError_t pipe_run(Handle &h, const void *h_raw, const double *h_tb, const double *h_te, const float *h_bp,
                     const float *h_gains, float *h_vis, cudaStream_t st)
{
    HostPipe &P = *h.pipe;
    const int SB = h.p.n_subbands, N = h.p.n_stations, C = h.p.n_channels;
    cudaError_t e;
#define RUN_TRY(x)                           \
    do {                                     \
        e = (x);                             \
        if (e != cudaSuccess) return e;      \
    } while (0)
    // order after earlier work on the caller's stream
    RUN_TRY(cudaEventRecord(P.ev_start, st));
    RUN_TRY(cudaStreamWaitEvent(P.s_in, P.ev_start, 0));
    RUN_TRY(cudaStreamWaitEvent(P.s_comp, P.ev_start, 0));
    RUN_TRY(cudaStreamWaitEvent(P.s_out, P.ev_start, 0));
    // small per-call parameters
    RUN_TRY(cudaMemcpyAsync(P.d_tau, h_tb, sizeof(double) * N, cudaMemcpyHostToDevice, P.s_in));
    RUN_TRY(cudaMemcpyAsync(P.d_tau + N, h_te, sizeof(double) * N, cudaMemcpyHostToDevice, P.s_in));
    if (h_bp) RUN_TRY(cudaMemcpyAsync(P.d_bp, h_bp, sizeof(float) * N * C, cudaMemcpyHostToDevice, P.s_in));
    if (h_gains)
        RUN_TRY(cudaMemcpyAsync(P.d_gain, h_gains, sizeof(float2) * N * kPols, cudaMemcpyHostToDevice, P.s_in));
    RUN_TRY(cudaEventRecord(P.ev_params, P.s_in));
    RUN_TRY(cudaStreamWaitEvent(P.s_comp, P.ev_params, 0));

    const int nch = (SB + P.chunk - 1) / P.chunk;
    const unsigned char *raw = static_cast<const unsigned char *>(h_raw);
    unsigned char *vis = reinterpret_cast<unsigned char *>(h_vis);
    for (int k = 0; k < nch; ++k) {
        const int b = k & 1;
        const int sb0 = k * P.chunk;
        const int cs = (SB - sb0) < P.chunk ? (SB - sb0) : P.chunk;
        // upload (buffer b is free once chunk k-2 has been computed)
        if (k >= 2) RUN_TRY(cudaStreamWaitEvent(P.s_in, P.comp_done[b], 0));
        RUN_TRY(cudaMemcpyAsync(P.d_raw[b], raw + (size_t)sb0 * P.raw_sb, (size_t)cs * P.raw_sb,
                                cudaMemcpyHostToDevice, P.s_in));
        RUN_TRY(cudaEventRecord(P.in_done[b], P.s_in));
        // compute (visibility buffer b is free once chunk k-2 has been downloaded)
        RUN_TRY(cudaStreamWaitEvent(P.s_comp, P.in_done[b], 0));
        if (k >= 2) RUN_TRY(cudaStreamWaitEvent(P.s_comp, P.out_done[b], 0));
        Handle v = h;                                   // view of the chunk's subbands
        v.p.n_subbands = cs;
        v.d_centres = h.d_centres + sb0;
        v.d_phase = h.d_phase + (size_t)sb0 * N * C;
        RUN_TRY(launch_phase_table(v, P.d_tau, P.d_tau + N, P.s_comp));
        RUN_TRY(launch_channelize_correct(v, P.d_raw[b], h_bp ? P.d_bp : nullptr, h_gains ? P.d_gain : nullptr,
                                          P.d_corr[b], P.s_comp));
        RUN_TRY(launch_xstage(v, P.d_corr[b], P.d_vis[b], P.s_comp));
        RUN_TRY(cudaEventRecord(P.comp_done[b], P.s_comp));
        // download
        RUN_TRY(cudaStreamWaitEvent(P.s_out, P.comp_done[b], 0));
        RUN_TRY(cudaMemcpyAsync(vis + (size_t)sb0 * P.vis_sb, P.d_vis[b], (size_t)cs * P.vis_sb,
                                cudaMemcpyDeviceToHost, P.s_out));
        RUN_TRY(cudaEventRecord(P.out_done[b], P.s_out));
    }
    // the caller's stream waits for the last download (s_out is in order)
    RUN_TRY(cudaStreamWaitEvent(st, P.out_done[(nch - 1) & 1], 0));
#undef RUN_TRY
    return cudaSuccess;
}

}  // namespace fxi
