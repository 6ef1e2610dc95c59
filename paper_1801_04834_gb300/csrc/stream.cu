// stream.cu -- streaming blocks: FIR history kept in the handle, integer-sample
// coarse delay per station, per-baseline counts of valid spectra.
//
// Paper, Sec. "Signal processing with GPU kernels": FIR filter history is
// carried across to the next block. Sec. "Software architecture": the coarse
// (whole-sample) delay is applied by the transpose stage through a circular
// buffer, and lost data is recorded in metadata.
//
// Stream coordinates: t = 0 is the first new sample of the current call, new
// samples are t in [0, S*C), the history holds the hist_len = (T-1)*C +
// max_shift samples before it (zeros before the first call). Station n's
// block is its stream over [-(T-1)*C - d_n, S*C - d_n): the assembled block
// is then an ordinary raw block for the channeliser. After the call the
// history becomes the last hist_len samples of the stream, written to the
// other buffer of a ping-pong pair.
#include "internal.h"

namespace fxi {
namespace {

constexpr int kStatusBadShift = 5;

template <typename U>
__global__ void stream_assemble_kernel(const U *__restrict__ hist, const U *__restrict__ nw,
                                       const int *__restrict__ shift, U *__restrict__ block, int *status,
                                       long long total, int N, int L, int hist_len, int new_len, int pre,
                                       int max_shift)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const long long sbn = idx / L;                  // (subband, station)
    const int t = (int)(idx - sbn * L);
    const int n = (int)(sbn % N);
    int d = shift ? shift[n] : 0;
    if (d < 0 || d > max_shift) {
        atomicCAS(status, 0, kStatusBadShift);
        d = d < 0 ? 0 : max_shift;
    }
    const int ts = t - pre - d;                     // stream time, >= -hist_len
    block[idx] = ts < 0 ? hist[sbn * hist_len + hist_len + ts] : nw[sbn * new_len + ts];
}

template <typename U>
__global__ void stream_history_kernel(const U *__restrict__ hist, const U *__restrict__ nw, U *__restrict__ out,
                                      long long total, int hist_len, int new_len)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const long long sbn = idx / hist_len;
    const int j = (int)(idx - sbn * hist_len);
    const int ts = new_len - hist_len + j;          // stream time of history entry j
    out[idx] = ts >= 0 ? nw[sbn * new_len + ts] : hist[sbn * hist_len + hist_len + ts];
}

// counts[b(i,j)] = sum_s w_i(s) w_j(s)
__global__ void baseline_counts_kernel(const float *__restrict__ flags, float *__restrict__ counts, int N, int S)
{
    const long long B = (long long)N * (N + 1) / 2;
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (!flags) {
        counts[b] = (float)S;
        return;
    }
    int j = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((long long)j * (j + 1) / 2 > b) --j;
    while ((long long)(j + 1) * (j + 2) / 2 <= b) ++j;
    const int i = (int)(b - (long long)j * (j + 1) / 2);
    float c = 0.f;
    for (int s = 0; s < S; ++s) c = fmaf(flags[(long long)i * S + s], flags[(long long)j * S + s], c);
    counts[b] = c;
}

template <typename U>
cudaError_t assemble_t(const Handle &h, const void *nw, const int *shift, cudaStream_t st)
{
    const int C = h.p.n_channels, T = h.p.n_taps, S = h.p.n_spectra;
    const int L = (S + T - 1) * C;
    const long long total = (long long)h.p.n_subbands * h.p.n_stations * L;
    const long long blocks = (total + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    stream_assemble_kernel<U><<<(unsigned)blocks, 256, 0, st>>>(
        static_cast<const U *>(h.d_hist[h.hist_cur]), static_cast<const U *>(nw), shift, static_cast<U *>(h.d_block),
        h.d_status, total, h.p.n_stations, L, h.hist_len, S * C, (T - 1) * C, h.p.max_coarse_shift);
    return cudaGetLastError();
}

template <typename U>
cudaError_t history_t(Handle &h, const void *nw, cudaStream_t st)
{
    const int S = h.p.n_spectra, C = h.p.n_channels;
    const long long total = (long long)h.p.n_subbands * h.p.n_stations * h.hist_len;
    const long long blocks = (total + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    stream_history_kernel<U><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const U *>(h.d_hist[h.hist_cur]),
                                                               static_cast<const U *>(nw),
                                                               static_cast<U *>(h.d_hist[1 - h.hist_cur]), total,
                                                               h.hist_len, S * C);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) h.hist_cur = 1 - h.hist_cur;
    return e;
}

}  // namespace

int raw_sample_bytes(const Handle &h)
{
    return kPols * (h.p.format == FX_CI16 ? 4 : h.p.format == FX_CI8 ? 2 : 1);
}

cudaError_t launch_stream_assemble(const Handle &h, const void *d_new, const int *shift, cudaStream_t st)
{
    switch (raw_sample_bytes(h)) {
    case 8: return assemble_t<uint2>(h, d_new, shift, st);
    case 4: return assemble_t<unsigned>(h, d_new, shift, st);
    default: return assemble_t<unsigned short>(h, d_new, shift, st);
    }
}

cudaError_t launch_stream_history(Handle &h, const void *d_new, cudaStream_t st)
{
    switch (raw_sample_bytes(h)) {
    case 8: return history_t<uint2>(h, d_new, st);
    case 4: return history_t<unsigned>(h, d_new, st);
    default: return history_t<unsigned short>(h, d_new, st);
    }
}

cudaError_t launch_baseline_counts(const Handle &h, const float *flags, float *counts, cudaStream_t st)
{
    const long long B = h.B;
    baseline_counts_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(flags, counts, h.p.n_stations,
                                                                        h.p.n_spectra);
    return cudaGetLastError();
}

}  // namespace fxi
