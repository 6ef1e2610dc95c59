// correct.cu -- fine delay compensation + bandpass correction (+ complex
// gains) with the transposing write-back to the per-channel layout the
// X-stage reads.
//
// Paper, Sec. "Signal processing with GPU kernels": the residual delays at the
// start and end of a block give channel-dependent phase angles computed in
// double precision; within the block the angle is interpolated linearly per
// sample and the rotation itself is single precision; the delay/bandpass
// kernel transposes on write-back so that the correlator reads all stations of
// one channel together. Sec. "Verification and validation": double precision
// is needed only for the delays.
//
// Two kernels per call:
//   phase_table  FP64, one thread per (subband, station, channel):
//                phi0 = 2 pi f_k tau_begin reduced mod 2 pi, and the
//                per-spectrum step 2 pi f_k (tau_end - tau_begin) / S; both
//                stored as FP32. FP64 work is SB*N*C, not per sample.
//   correct_*    FP32 per sample: phi = phi0 + s * step reduced to [-pi, pi]
//                (two-constant Cody-Waite split of 2 pi), __sincosf, rotate,
//                times bandpass * gain, transpose. Memory bound.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

#include "internal.h"

namespace fxi {
namespace {

__global__ void phase_table_kernel(const double *__restrict__ centres, const double *__restrict__ tau_b,
                                   const double *__restrict__ tau_e, float2 *__restrict__ table,
                                   int SB, int N, int C, int S, double fs)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)SB * N * C) return;
    const int k = (int)(idx % C);
    const int n = (int)((idx / C) % N);
    const int sb = (int)(idx / ((long long)C * N));
    const double two_pi = 6.283185307179586476925286766559;
    const double f = centres[sb] + (double)(k - C / 2) * fs / (double)C;
    const double phi0 = two_pi * f * tau_b[n];
    const double red = phi0 - two_pi * rint(phi0 / two_pi);
    const double step = two_pi * f * (tau_e[n] - tau_b[n]) / (double)S;
    table[idx] = make_float2((float)red, (float)step);
}

// ---- FP32 output, spectrum-blocked [SB][C][ceil16(S)/16][N][16][2] ---------
// CTA = (subband, station, run of kBPC blocks of 16 spectra), all C channels;
// stations run fastest in the grid so that CTAs resident together fill
// neighbouring 256-byte runs of each channel. Per block the CTA first
// tabulates exp(i phi) per (channel, spectrum) in shared memory
// (phi = phi0 + s * step in FP32, reduced to [-pi, pi] with a two-constant
// Cody-Waite split of 2 pi, then __sincosf: absolute error about 4e-7; both
// pols share an entry). Reads are C-channel runs of one (pol, spectrum);
// writes are 256-byte runs (16 spectra x 2 pols) of one channel; the tile
// [C][32 + 1] turns the corner in shared memory. Spectra S .. ceil16(S) - 1
// are written as zeros.
constexpr int kNT = 256;
constexpr int kBS = 16;                  // spectra per block of the FP32 layout
constexpr int kBPC = 4;                  // blocks per CTA

__global__ void __launch_bounds__(kNT)
correct_f32_kernel(const float2 *__restrict__ chan, const float2 *__restrict__ table,
                   const float *__restrict__ bandpass, const float2 *__restrict__ gains,
                   float2 *__restrict__ corr, int N, int C, int S)
{
    extern __shared__ float2 tile[];     // [C][2 * kBS + 1], then the phasors [kBS][C]
    constexpr int TW = 2 * kBS + 1;
    float2 *ph = tile + C * TW;
    const int n = blockIdx.x, sb = blockIdx.z;
    const int NB = (S + kBS - 1) / kBS;
    const float2 *tb = table + ((long long)sb * N + n) * C;
    float2 g[kPols];
#pragma unroll
    for (int p = 0; p < kPols; ++p) g[p] = gains ? gains[n * kPols + p] : make_float2(1.f, 0.f);
    const int blk_end = min(NB, (int)(blockIdx.y + 1) * kBPC);
    for (int blk = blockIdx.y * kBPC; blk < blk_end; ++blk) {
        if (blk > (int)blockIdx.y * kBPC) __syncthreads();   // the previous block's tile is written out
        for (int e = threadIdx.x; e < kBS * C; e += kNT) {
            const int k = e % C, j = e / C;
            const float2 pt = tb[k];
            const float phi = fmaf((float)(blk * kBS + j), pt.y, pt.x);
            const float kq = rintf(phi * 0.15915494309189535f);            // phi / (2 pi)
            float r = fmaf(-kq, 6.28125f, phi);                             // 2 pi = 6.28125 + 1.9353...e-3
            r = fmaf(-kq, 1.9353071795864769e-3f, r);
            float sn, cs;
            __sincosf(r, &sn, &cs);
            ph[e] = make_float2(cs, sn);
        }
        __syncthreads();
        // eight samples per thread in flight before any is used
        constexpr int U = 8;
        for (int e0 = threadIdx.x; e0 < kPols * kBS * C; e0 += U * kNT) {
            float2 xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * kNT;
                const int k = e % C, j = (e / C) % kBS, p = e / (C * kBS);
                const int s = blk * kBS + j;
                xv[u] = make_float2(0.f, 0.f);
                if (e < kPols * kBS * C && s < S) xv[u] = chan[((((long long)sb * N + n) * kPols + p) * S + s) * C + k];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * kNT;
                if (e >= kPols * kBS * C) break;
                const int k = e % C, j = (e / C) % kBS, p = e / (C * kBS);
                const int s = blk * kBS + j;
                float2 y = make_float2(0.f, 0.f);
                if (s < S) {
                    const float2 x = xv[u];
                    const float bp = bandpass ? bandpass[(long long)n * C + k] : 1.f;
                    const float2 xg =
                        make_float2(fmaf(x.x, g[p].x, -x.y * g[p].y), fmaf(x.x, g[p].y, x.y * g[p].x));
                    const float2 w = ph[j * C + k];
                    y = make_float2(bp * fmaf(xg.x, w.x, -xg.y * w.y), bp * fmaf(xg.x, w.y, xg.y * w.x));
                }
                tile[k * TW + j * kPols + p] = y;
            }
        }
        __syncthreads();
        float2 *out = corr + (((long long)sb * C * NB + blk) * N + n) * (2 * kBS);
        const long long kstride = (long long)NB * N * (2 * kBS);
        for (int e = threadIdx.x; e < C * 2 * kBS; e += kNT) {
            const int jp = e % (2 * kBS), k = e / (2 * kBS);
            out[k * kstride + jp] = tile[k * TW + jp];
        }
    }
}

static cudaError_t launch_correct_f32(const float2 *chan, const float2 *table, const float *bandpass,
                                      const float2 *gains, float2 *corr, int SB, int N, int C, int S, cudaStream_t st)
{
    const size_t smem = (size_t)C * (2 * kBS + 1 + kBS) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(correct_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(N, ((S + kBS - 1) / kBS + kBPC - 1) / kBPC, SB);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    correct_f32_kernel<<<grid, kNT, smem, st>>>(chan, table, bandpass, gains, corr, N, C, S);
    return cudaGetLastError();
}

// ---- planar output [SB][C][planes][I_pad][S_pad] (16-bit, hi/lo or FP32) ----
// CTA tile = one station (both pols) x CC channels (CC = min(C, 64)) x ST =
// 2048 / CC spectra. Reads are whole channel runs of one (pol, spectrum)
// (CC x 8 bytes: all of a 64-channel row), so a CTA reads contiguous memory
// and DRAM pages are not reopened by sibling CTAs; writes are ST-spectrum
// runs of one (channel, plane, input). The tile [pol][channel][ST + 1] turns
// the corner in shared memory without bank conflicts. CTAs past the last
// station (inputs I .. I_pad) and spectra S .. S_pad write zeros.
// All of a thread's samples are loaded before any is used (memory-level
// parallelism). The phase is reduced to [-pi, pi] by a two-constant
// Cody-Waite split of 2 pi, then __sincosf (absolute error about 4e-7, as in
// the fused F-stage).
constexpr int kPT_E = 4096;                 // samples per CTA tile

template <int CC>
constexpr int pt_st() { return kPT_E / (kPols * CC); }

template <int MODE, int CC>  // MODE 1: F16, 2: BF16, 3: F16 split, 4: FP32 (TF32 split X-stage)
__global__ void __launch_bounds__(kNT)
correct_planar_kernel(const float2 *__restrict__ chan, const float2 *__restrict__ table,
                      const float *__restrict__ bandpass, const float2 *__restrict__ gains,
                      void *__restrict__ corr, int N, int C, int S, int I_pad, int S_pad, float scale)
{
    constexpr int ST = pt_st<CC>();          // spectra per tile: 32 (CC = 64) or 128 (CC = 16)
    constexpr int TR = ST + 1;               // tile row (float2)
    constexpr int PER = kPT_E / kNT;
    __shared__ float2 tile[kPols * CC * TR];
    const int s0 = blockIdx.x * ST;
    const int n = blockIdx.y;                // station; n >= N: padding inputs (zeros)
    const int cblocks = C / CC;
    const int c0 = (blockIdx.z % cblocks) * CC;
    const int sb = blockIdx.z / cblocks;

    float2 xv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * kNT;
        const int c = e % CC, s = (e / CC) % ST, p = e / (CC * ST);
        const int ss = s0 + s;
        xv[u] = make_float2(0.f, 0.f);
        if (n < N && ss < S) xv[u] = chan[((((long long)sb * N + n) * kPols + p) * S + ss) * C + c0 + c];
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * kNT;
        const int c = e % CC, s = (e / CC) % ST, p = e / (CC * ST);
        const int ss = s0 + s, k = c0 + c;
        float2 y = make_float2(0.f, 0.f);
        if (n < N && ss < S) {
            const float2 ph = table[((long long)sb * N + n) * C + k];
            const float bp = (bandpass ? bandpass[(long long)n * C + k] : 1.f) * scale;
            const float2 g = gains ? gains[n * kPols + p] : make_float2(1.f, 0.f);
            const float phi = fmaf((float)ss, ph.y, ph.x);
            const float kq = rintf(phi * 0.15915494309189535f);            // phi / (2 pi)
            float r = fmaf(-kq, 6.28125f, phi);                             // 2 pi = 6.28125 + 1.9353...e-3
            r = fmaf(-kq, 1.9353071795864769e-3f, r);
            float sn, cs;
            __sincosf(r, &sn, &cs);
            const float2 x = xv[u];
            const float2 xg = make_float2(fmaf(x.x, g.x, -x.y * g.y), fmaf(x.x, g.y, x.y * g.x));
            y = make_float2(bp * fmaf(xg.x, cs, -xg.y * sn), bp * fmaf(xg.x, sn, xg.y * cs));
        }
        tile[(p * CC + c) * TR + s] = y;
    }
    __syncthreads();
    constexpr int planes = (MODE == 3) ? 4 : 2;
    const long long plane_stride = (long long)I_pad * S_pad;
    // task = (pol p, channel c, group of 8 spectra)
    for (int task = threadIdx.x; task < kPols * CC * (ST / 8); task += kNT) {
        const int g8 = task % (ST / 8);
        const int c = (task / (ST / 8)) % CC;
        const int p = task / ((ST / 8) * CC);
        const int sg = s0 + g8 * 8;
        if (sg >= S_pad) continue;
        const float2 *src = tile + (p * CC + c) * TR + g8 * 8;
        const long long base = (((long long)sb * C + c0 + c) * planes) * plane_stride +
                               (long long)(n * kPols + p) * S_pad + sg;
        if constexpr (MODE == 4) {
            float4 *re = reinterpret_cast<float4 *>(reinterpret_cast<float *>(corr) + base);
            float4 *im = reinterpret_cast<float4 *>(reinterpret_cast<float *>(corr) + base + plane_stride);
            re[0] = make_float4(src[0].x, src[1].x, src[2].x, src[3].x);
            re[1] = make_float4(src[4].x, src[5].x, src[6].x, src[7].x);
            im[0] = make_float4(src[0].y, src[1].y, src[2].y, src[3].y);
            im[1] = make_float4(src[4].y, src[5].y, src[6].y, src[7].y);
        } else {
            unsigned short re_hi[8], im_hi[8], re_lo[8], im_lo[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 y = src[q];
                if constexpr (MODE == 2) {
                    re_hi[q] = __bfloat16_as_ushort(__float2bfloat16_rn(y.x));
                    im_hi[q] = __bfloat16_as_ushort(__float2bfloat16_rn(y.y));
                } else {
                    const __half hr = __float2half_rn(y.x), hi = __float2half_rn(y.y);
                    re_hi[q] = __half_as_ushort(hr);
                    im_hi[q] = __half_as_ushort(hi);
                    if constexpr (MODE == 3) {
                        re_lo[q] = __half_as_ushort(__float2half_rn(y.x - __half2float(hr)));
                        im_lo[q] = __half_as_ushort(__float2half_rn(y.y - __half2float(hi)));
                    }
                }
            }
            unsigned short *out = reinterpret_cast<unsigned short *>(corr);
            auto store8 = [&](long long off, const unsigned short (&v)[8]) {
                uint4 w;
                w.x = v[0] | ((unsigned)v[1] << 16);
                w.y = v[2] | ((unsigned)v[3] << 16);
                w.z = v[4] | ((unsigned)v[5] << 16);
                w.w = v[6] | ((unsigned)v[7] << 16);
                *reinterpret_cast<uint4 *>(out + off) = w;
            };
            store8(base, re_hi);
            store8(base + plane_stride, im_hi);
            if constexpr (MODE == 3) {
                store8(base + 2 * plane_stride, re_lo);
                store8(base + 3 * plane_stride, im_lo);
            }
        }
    }
}

// Scratch of the no-allocation correction entry point (fx_correct_f32_noalloc):
// the phase table lives in this fixed-size device array instead of memory
// allocated by fx_create. Every GPU that loads the library holds these 8 MiB
// until the process exits.
static __device__ __align__(256) float2 g_noalloc_phase[FX_NOALLOC_MAX_PHASES];

}  // namespace

cudaError_t launch_phase_table(const Handle &h, const double *tau_b, const double *tau_e,
                               cudaStream_t st)
{
    const long long n = (long long)h.p.n_subbands * h.p.n_stations * h.p.n_channels;
    const int threads = 256;
    const long long blocks = (n + threads - 1) / threads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    phase_table_kernel<<<(unsigned)blocks, threads, 0, st>>>(h.d_centres, tau_b, tau_e, h.d_phase,
                                                             h.p.n_subbands, h.p.n_stations,
                                                             h.p.n_channels, h.p.n_spectra,
                                                             h.p.sample_rate_hz);
    return cudaGetLastError();
}

// The context current on this thread (driver entry point fetched through the
// runtime, so the library needs no -lcuda), or null.
static CUcontext current_context()
{
    typedef CUresult (*GetCurrentFn)(CUcontext *);
    static GetCurrentFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<GetCurrentFn>(p);
        return static_cast<GetCurrentFn>(nullptr);
    }();
    CUcontext ctx = nullptr;
    if (fn) fn(&ctx);
    return ctx;
}

// Device address of g_noalloc_phase on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device (the first call on that device does
// it, with that device current) and cached together with the context it
// belongs to; if the device's context was replaced since (cudaDeviceReset),
// the lookup is done again.
static cudaError_t noalloc_phase_ptr(float2 **out)
{
    static std::mutex mu;
    static float2 *ptrs[kMaxDevices] = {};
    static CUcontext ctxs[kMaxDevices] = {};
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev] || (ctxs[dev] && ctxs[dev] != current_context())) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_phase);
        if (e != cudaSuccess) return e;
        ptrs[dev] = static_cast<float2 *>(p);
        ctxs[dev] = current_context();
    }
    *out = ptrs[dev];
    return cudaSuccess;
}

cudaError_t launch_correct_f32_noalloc(int N, int SB, int C, int S, double fs, const double *centres,
                                       const double *tau_b, const double *tau_e, const float *bandpass,
                                       const float2 *gains, const float2 *chan, float2 *corr, cudaStream_t st)
{
    float2 *table = nullptr;
    cudaError_t e = noalloc_phase_ptr(&table);
    if (e != cudaSuccess) return e;
    const long long n = (long long)SB * N * C;
    phase_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(centres, tau_b, tau_e, table, SB, N, C, S,
                                                                    fs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_correct_f32(chan, table, bandpass, gains, corr, SB, N, C, S, st);
}

template <int CC>
static cudaError_t launch_planar(const Handle &h, const float2 *chan, const float *bandpass, const float2 *gains,
                                 void *corr, cudaStream_t st)
{
    const int N = h.p.n_stations, C = h.p.n_channels, S = h.p.n_spectra, SB = h.p.n_subbands;
    constexpr int ST = pt_st<CC>();
    dim3 grid((h.S_pad + ST - 1) / ST, h.I_pad / kPols, SB * (C / CC));
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    switch (h.p.precision) {
    case FX_F16:
        correct_planar_kernel<1, CC><<<grid, kNT, 0, st>>>(chan, h.d_phase, bandpass, gains, corr, N, C, S, h.I_pad,
                                                           h.S_pad, h.operand_scale);
        break;
    case FX_BF16:
        correct_planar_kernel<2, CC><<<grid, kNT, 0, st>>>(chan, h.d_phase, bandpass, gains, corr, N, C, S, h.I_pad,
                                                           h.S_pad, h.operand_scale);
        break;
    case FX_TF32_SPLIT:
        correct_planar_kernel<4, CC><<<grid, kNT, 0, st>>>(chan, h.d_phase, bandpass, gains, corr, N, C, S, h.I_pad,
                                                           h.S_pad, 1.f);
        break;
    default:
        correct_planar_kernel<3, CC><<<grid, kNT, 0, st>>>(chan, h.d_phase, bandpass, gains, corr, N, C, S, h.I_pad,
                                                           h.S_pad, h.operand_scale);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_correct(const Handle &h, const float2 *chan, const float *bandpass,
                           const float2 *gains, void *corr, cudaStream_t st)
{
    const int N = h.p.n_stations, C = h.p.n_channels, S = h.p.n_spectra, SB = h.p.n_subbands;
    if (h.p.precision == FX_F32)
        return launch_correct_f32(chan, h.d_phase, bandpass, gains, reinterpret_cast<float2 *>(corr), SB, N, C, S,
                                  st);
    if (C >= 64) return launch_planar<64>(h, chan, bandpass, gains, corr, st);
    return launch_planar<16>(h, chan, bandpass, gains, corr, st);
}

}  // namespace fxi
