// xcorr_f32.cu -- X-stage correlator in FP32 on the CUDA cores (FFMA).
//
// Paper, Sec. "Signal processing with GPU kernels": the last kernel correlates
// all pairs of antenna fields and integrates to ~1 s. Sec. "Hardware
// requirements and design priorities": the correlator is compute bound and
// can run close to peak.
//
//   V[sb][k][b(i,j)][2p+q] = sum_s Y[s][i,p] * conj(Y[s][j,q]),  i <= j
//
// Input is the FP32 corrected layout [SB][C][S][I] (I = 2N interleaved complex),
// so one channel's block is one contiguous [S][I] matrix.
//
// Register tiling over the station triangle: a thread owns 2 stations (rows,
// 4 inputs) x 4 stations (columns, 8 inputs) = 32 complex accumulators, i.e.
// 128 FFMAs per time sample against 6 shared-memory vector loads. Tiles
// (row pair r, column quad q) are kept only where some pair i <= j exists
// (2r <= 4q+3), which gives N(N+1)/2 useful pairs out of ~N(N+2)/2 computed.
// A CTA holds the tile set of `cpb` channels; time is streamed through shared
// memory in chunks of KC samples with double-buffered cp.async.
#include <algorithm>

#include "internal.h"

namespace fxi {
namespace {

constexpr int kKC = 32;          // time samples per shared-memory chunk
constexpr int kMaxThreads = 544;   // 2 channels x 272 tiles at N = 64; 120 registers

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One CTA: channels [chb*cpb, +cpb) of the flattened (subband, channel) index
// and part `part` of the tile list (parts > 1 only when one channel's tiles
// exceed a CTA, then cpb = 1); thread t works on tile part*tpp + t % tpp of
// channel t / tpp.
__global__ void __launch_bounds__(kMaxThreads, 1)
xcorr_f32_kernel(const float2 *__restrict__ corr, float2 *__restrict__ vis,
                 const int2 *__restrict__ tiles, int ntiles, int tpp, int parts, int N, int S,
                 int IP, int cpb, long long total_ch)
{
    extern __shared__ float4 sm[];   // [2][cpb][KC][IP/2] float4
    const int I = 2 * N;
    const int row4 = IP / 2;                       // float4 per time row
    const int stage_f4 = cpb * kKC * row4;
    const int tid = threadIdx.x;
    const int part = blockIdx.x % parts;
    const long long ch0 = (long long)(blockIdx.x / parts) * cpb;
    const int nthr = blockDim.x;

    auto load_chunk = [&](int stage, int s0) {
        float4 *dst0 = sm + stage * stage_f4;
        for (int v = tid; v < stage_f4; v += nthr) {
            const int x = v % row4;
            const int s = (v / row4) % kKC;
            const int cl = v / (row4 * kKC);
            const long long gch = ch0 + cl;
            const bool ok = (2 * x < I) && (s0 + s < S) && (gch < total_ch);
            const float2 *src = corr;
            if (ok) src = corr + (gch * S + s0 + s) * (long long)I + 2 * x;
            cp_async16(dst0 + v, src, ok ? 16 : 0);
        }
    };

    const int cl = tid / tpp;
    const int tl = part * tpp + (tid - cl * tpp);
    const bool active = cl < cpb && (ch0 + cl) < total_ch && tl < ntiles;
    int2 rq = make_int2(0, 0);
    if (active) rq = tiles[tl];
    const int r = rq.x, q = rq.y;

    float are[4][8], aim[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) are[a][b] = aim[a][b] = 0.f;

    const int nchunks = (S + kKC - 1) / kKC;
    load_chunk(0, 0);
    cp_async_commit();
    for (int kc = 0; kc < nchunks; ++kc) {
        if (kc + 1 < nchunks) load_chunk((kc + 1) & 1, (kc + 1) * kKC);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        if (active) {
            const float4 *base = sm + (kc & 1) * stage_f4 + cl * kKC * row4;
#pragma unroll 2
            for (int s = 0; s < kKC; ++s) {
                const float4 *rowp = base + s * row4;
                const float4 x0 = rowp[2 * r], x1 = rowp[2 * r + 1];
                const float4 y0 = rowp[4 * q], y1 = rowp[4 * q + 1], y2 = rowp[4 * q + 2],
                             y3 = rowp[4 * q + 3];
                const float xr[4] = {x0.x, x0.z, x1.x, x1.z};
                const float xi[4] = {x0.y, x0.w, x1.y, x1.w};
                const float yr[8] = {y0.x, y0.z, y1.x, y1.z, y2.x, y2.z, y3.x, y3.z};
                const float yi[8] = {y0.y, y0.w, y1.y, y1.w, y2.y, y2.w, y3.y, y3.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        // x * conj(y)
                        are[a][b] = fmaf(xr[a], yr[b], are[a][b]);
                        are[a][b] = fmaf(xi[a], yi[b], are[a][b]);
                        aim[a][b] = fmaf(xi[a], yr[b], aim[a][b]);
                        aim[a][b] = fmaf(-xr[a], yi[b], aim[a][b]);
                    }
            }
        }
        __syncthreads();
    }
    if (!active) return;
    const long long gch = ch0 + cl;
    const long long B = (long long)N * (N + 1) / 2;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = 2 * r + a / 2, p = a % 2;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = 4 * q + jj;
            if (i <= j && j < N) {
                const long long b = (long long)j * (j + 1) / 2 + i;
                float4 v = make_float4(are[a][2 * jj], aim[a][2 * jj], are[a][2 * jj + 1], aim[a][2 * jj + 1]);
                *reinterpret_cast<float4 *>(vis + (gch * B + b) * 4 + 2 * p) = v;
            }
        }
    }
}

}  // namespace

// Tiles (r, q): row stations 2r, 2r+1; column stations 4q..4q+3; kept where
// 2r <= 4q + 3. Ordered by q, then r, so a warp mostly shares its column loads.
int xf32_build_tiles(int N, int2 *out)
{
    const int NR = (N + 1) / 2, NQ = (N + 3) / 4;
    int n = 0;
    for (int q = 0; q < NQ; ++q)
        for (int r = 0; r < NR; ++r)
            if (2 * r <= 4 * q + 3) {
                if (out) out[n] = make_int2(r, q);
                ++n;
            }
    return n;
}

cudaError_t launch_xcorr_f32(const Handle &h, const float2 *corr, float2 *vis, cudaStream_t st)
{
    const int N = h.p.n_stations, S = h.p.n_spectra;
    const int IP = 8 * ((N + 3) / 4);
    const int nt = h.xf32_ntiles;
    const int parts = (nt + kMaxThreads - 1) / kMaxThreads;
    const int tpp = (nt + parts - 1) / parts;          // tiles per CTA part
    const long long total = (long long)h.p.n_subbands * h.p.n_channels;
    const size_t per_ch = 2ull * kKC * IP * sizeof(float2);
    if (per_ch > 200 * 1024) return cudaErrorNotSupported;   // > ~400 stations
    int cpb = parts > 1 ? 1 : std::max(1, kMaxThreads / nt);
    cpb = (int)std::min<long long>(cpb, std::max<size_t>(1, (200 * 1024) / per_ch));
    // keep at least ~2 waves of CTAs on 152 SMs
    while (cpb > 1 && (total + cpb - 1) / cpb < 2 * 152) --cpb;
    const int threads = (cpb * tpp + 31) / 32 * 32;
    const size_t smem = per_ch * cpb;
    cudaError_t e = cudaFuncSetAttribute(xcorr_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (total + cpb - 1) / cpb * parts;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    xcorr_f32_kernel<<<(unsigned)blocks, threads, smem, st>>>(corr, vis, h.d_xf32_tiles, nt, tpp, parts,
                                                              N, S, IP, cpb, total);
    return cudaGetLastError();
}

}  // namespace fxi
